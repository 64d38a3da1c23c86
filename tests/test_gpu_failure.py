"""Failure detection of the bounded device waits, without a fault: a wait
whose bytes never arrive gives up, the call reports DPD_ETIMEOUT promptly,
and the same CUDA context then runs a system normally."""
import time

import numpy as np
import pytest

from paper_1804_06205_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def D():
    from paper_1804_06205_gb300 import build
    build.build()
    from paper_1804_06205_gb300 import dpd
    return dpd


def test_delivered_wait_completes(D):
    assert D.wait_check(True, tries=1 << 20) == D.DPD_OK


def test_undelivered_wait_gives_up_and_context_survives(D):
    t0 = time.perf_counter()
    rc = D.wait_check(False, tries=4096)
    assert rc == D.DPD_ETIMEOUT
    assert time.perf_counter() - t0 < 30.0
    assert D.wait_check(True) == D.DPD_OK           # the context is still usable
    w = W.fluid_3k()
    g = D.System.from_workload(w, precision=D.DPD_FP32)
    g.set_state(w.pos, w.vel, 0)
    g.step(5)
    pos, vel, f, step = g.get_state()
    g.close()
    assert step == 5 and np.isfinite(pos).all() and np.isfinite(vel).all()


def test_force_overflow_is_reported_as_unstable(D):
    """A repulsion so strong that binary32 forces overflow: the force
    evaluation of set_state flags it and the call reports DPD_EUNSTABLE;
    cell indices stay in range for any value, so nothing else is affected."""
    w = W.fluid(6.0, a_same=3.0e38, seed=5)
    g = D.System.from_workload(w, precision=D.DPD_FP32)
    with pytest.raises(D.DPDError) as e:
        g.set_state(w.pos, w.vel, 0)
    assert e.value.code == D.DPD_EUNSTABLE
    g.close()
    w = W.fluid_3k()
    g = D.System.from_workload(w, precision=D.DPD_FP32)
    g.set_state(w.pos, w.vel, 0)
    g.step(3)
    assert np.isfinite(g.get_state()[2]).all()
    g.close()
