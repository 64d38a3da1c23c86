"""Batches: many independent systems advanced by the same launches.

A system in a batch must follow exactly the arithmetic it follows alone
(same noise from its own seed and local ids, same per-bead summation order):
the tests compare batched and alone runs bit for bit, before and after
removals re-pack the pools, and check memory admission."""
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


def systems():
    """Uneven systems shaped like the serving stream (edge 8..11, two types,
    10% of beads in harmonic chains), plus a peptide-like one with Morse."""
    out = [W.serving_system(s, edge=e, a_ab=ab) for s, e, ab in
           ((1, 8.0, 27.0), (2, 9.7, 44.0), (3, 11.2, 33.0), (4, 8.4, 50.0))]
    out.append(W.peptide_192k(L=9.0, nchains=8, chain_len=20, seed=31))
    return out


def alone(D, w, nsteps, prec):
    g = D.System.from_workload(w, precision=prec)
    g.set_state(w.pos, w.vel, 0)
    g.step(nsteps)
    out = g.get_state()
    g.close()
    return out


def batch_for(D, ws, prec, **kw):
    nb = sum(w.n for w in ws)
    nc = sum(int(np.prod(np.floor(w.L))) for w in ws)
    nbond = sum(w.nbonds for w in ws)
    return D.Batch(nb, nc, nbond, max_systems=16, precision=prec, **kw)


@pytest.mark.parametrize("prec", [0, 1])
def test_batched_systems_equal_alone_runs(D, prec):
    ws = systems()
    b = batch_for(D, ws, prec)
    ids = [b.add_workload(w) for w in ws]
    assert all(i is not None for i in ids)
    b.step(12)
    for w, s in zip(ws, ids):
        ref = alone(D, w, 12, prec)
        got = b.get_state(s)
        assert got[3] == ref[3] == 12
        for x, y in zip(got[:3], ref[:3]):
            assert np.array_equal(x, y), w.name
    b.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_sampling_does_not_change_the_trajectory(D, prec):
    """Splitting a run into calls changes which steps fuse the next position
    update (the last step of a call does not), and observables asked for
    between calls run a sampled force pass on the state: none of it may change
    the trajectory."""
    w = systems()[4]
    ref = alone(D, w, 12, prec)
    g = D.System.from_workload(w, precision=prec)
    g.set_state(w.pos, w.vel, 0)
    for k in (5, 4, 1, 2):
        g.step(k)
        assert np.isfinite(g.observables()["p_total"])
    got = g.get_state()
    for x, y in zip(got[:3], ref[:3]):
        assert np.array_equal(x, y)


def test_removal_repacks_and_keeps_the_others_exact(D):
    ws = systems()
    b = batch_for(D, ws, 0)
    ids = [b.add_workload(w) for w in ws]
    b.step(5)
    b.remove(ids[1])          # a system in the middle of the pools
    b.step(4)
    b.remove(ids[0])          # the first one
    b.step(3)
    used, cap, ns = b.usage()
    assert ns == 3
    assert used[0] == sum(w.n for w in ws[2:])
    for w, s in zip(ws[2:], ids[2:]):
        ref = alone(D, w, 12, 0)
        got = b.get_state(s)
        for x, y in zip(got[:3], ref[:3]):
            assert np.array_equal(x, y), w.name
        # observables computed on demand from the re-packed pools
        g = D.System.from_workload(w, precision=0)
        g.set_state(w.pos, w.vel, 0)
        g.step(12)
        oa, ob = g.observables(), b.observables(s)
        g.close()
        for k in ("kT", "p_total", "e_pair", "e_bond"):
            assert oa[k] == ob[k], (w.name, k)
    b.close()


def test_late_arrival_joins_running_batch(D):
    """A system added after the others have advanced starts from its own
    step counter and matches its alone run."""
    ws = systems()
    b = batch_for(D, ws, 0)
    first = [b.add_workload(w) for w in ws[:3]]
    b.step(6)
    late = b.add_workload(ws[3])
    b.step(5)
    got = b.get_state(late)
    ref = alone(D, ws[3], 5, 0)
    assert got[3] == 5
    for x, y in zip(got[:3], ref[:3]):
        assert np.array_equal(x, y)
    got0 = b.get_state(first[0])
    ref0 = alone(D, ws[0], 11, 0)
    assert got0[3] == 11 and np.array_equal(got0[0], ref0[0])
    b.close()


def test_admission_by_memory_footprint(D):
    ws = systems()
    small = ws[0]
    b = D.Batch(2 * small.n + 10, 10 ** 5, 10 ** 5, max_systems=8)
    assert b.add_workload(small) is not None
    assert b.add_workload(small) is not None
    assert b.add_workload(small) is None       # beads exhausted: not admitted
    used, cap, ns = b.usage()
    assert ns == 2 and used[0] == 2 * small.n
    b.remove(0)
    assert b.add_workload(small) is not None   # room again after a departure
    b.close()
