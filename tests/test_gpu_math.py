"""Device arithmetic of the FP64 path checked against the CUDA library."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def D():
    from paper_1804_06205_gb300 import build
    build.build()
    from paper_1804_06205_gb300 import dpd
    return dpd


def test_box_muller_functions_match_library(D):
    # every uniform n 2^-24 (n odd); |ln u| <= 16.7, so a few units in the last
    # place of the largest values is ~1e-14, and |cos| <= 1: both far below
    # what the FP64 force tolerance (1e-10 max|f|) could notice in
    # theta = sqrt(-2 ln u) cos(2 pi v)
    ln_err, cos_err = D.bm_check()
    assert ln_err < 1e-14
    assert cos_err < 1e-15
