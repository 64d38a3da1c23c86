"""Device arithmetic of the FP64 path checked against the CUDA library."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def D():
    from paper_1804_06205_gb300 import build
    build.build()
    from paper_1804_06205_gb300 import dpd
    return dpd


def test_box_muller_log_matches_library_log(D):
    # every uniform n 2^-24 (n odd); |ln u| <= 16.7, so a few units in the last
    # place of the largest values is ~1e-14: far below what the FP64 force
    # tolerance (1e-10 max|f|) could notice in theta = sqrt(-2 ln u) cos(2 pi v)
    assert D.ln_check() < 1e-14
