"""The persistent multi-system step (dpd_options.persistent = 1): every
dpd_step / dpd_batch_step call is one cooperative launch whose resident
blocks run all phases of all steps of Fig. 1 for all resident systems, with a
bounded grid-wide barrier between phases.  It calls the same device code as
the one-launch-per-kernel path, so the trajectories must be identical bit for
bit; and its barrier must give up (DPD_ETIMEOUT) rather than wait forever."""
import time

import numpy as np
import pytest

from paper_1804_06205_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FP32, FP64 = 0, 1


@pytest.fixture(scope="module")
def D():
    from paper_1804_06205_gb300 import build
    build.build()
    from paper_1804_06205_gb300 import dpd
    return dpd


def _systems():
    return [W.serving_system(7, edge=9.3, a_ab=41.0),
            W.fluid((12.0, 8.5, 10.2), ntypes=2, a_same=25.0, a_cross=30.0, seed=71),
            W.peptide_192k(L=10.0, nchains=6, chain_len=20, seed=72),
            W.serving_system(8, edge=15.7, a_ab=27.0)]


def _run_batch(D, prec, persistent, chunks, remove_after=None):
    ws = _systems()
    nb = sum(w.n for w in ws)
    nc = sum(int(np.prod(np.floor(w.L))) for w in ws)
    nbond = sum(w.nbonds for w in ws)
    b = D.Batch(nb, nc, nbond, max_systems=len(ws), precision=prec,
                persistent=1 if persistent else 0)
    ids = [b.add_workload(w) for w in ws]
    for k, n in enumerate(chunks):
        b.step(n)
        if remove_after is not None and k == remove_after:
            b.remove(ids[1])
            ids[1] = None
    out = [None if s is None else b.get_state(s) for s in ids]
    b.close()
    return out


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_persistent_batch_equals_direct_launches(D, prec):
    chunks = (7, 1, 12)
    a = _run_batch(D, prec, False, chunks, remove_after=1)
    b = _run_batch(D, prec, True, chunks, remove_after=1)
    for x, y in zip(a, b):
        if x is None:
            assert y is None
            continue
        for u, v in zip(x, y):
            if isinstance(u, np.ndarray):
                assert np.array_equal(u, v)
            else:
                assert u == v


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_persistent_single_system_equals_direct(D, prec):
    w = W.melt_98k(L=10.0, seed=73)
    out = []
    for persistent in (0, 1):
        g = D.System.from_workload(w, precision=prec, persistent=persistent)
        g.set_state(w.pos, w.vel, 0)
        g.step(9)
        g.step(4)
        out.append(g.get_state())
        o = g.observables()
        g.close()
        assert o["status"] == 0
    for u, v in zip(out[0][:3], out[1][:3]):
        assert np.array_equal(u, v)
    assert out[0][3] == out[1][3] == 13


def test_grid_barrier_wait_gives_up_and_context_survives(D):
    assert D.grid_wait_check(True, budget_cycles=200_000_000) == D.DPD_OK
    t0 = time.perf_counter()
    rc = D.grid_wait_check(False, budget_cycles=20_000_000)
    assert rc == D.DPD_ETIMEOUT
    assert time.perf_counter() - t0 < 30.0
    assert D.grid_wait_check(True, budget_cycles=200_000_000) == D.DPD_OK
    w = W.fluid_3k()
    g = D.System.from_workload(w, precision=FP32, persistent=1)
    g.set_state(w.pos, w.vel, 0)
    g.step(5)
    pos, vel, f, step = g.get_state()
    g.close()
    assert step == 5 and np.isfinite(pos).all() and np.isfinite(vel).all()
