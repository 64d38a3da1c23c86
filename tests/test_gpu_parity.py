"""GPU parity of the CUDA engine (through the C ABI) against the FP64 oracle.

Tolerances (from the arithmetic of each path):
  * cell keys, sort order, cell starts, g(r) counts of the FP64 path: bit-exact;
  * one force evaluation from an identical state: max|f_gpu - f_oracle| <=
    1e-4 max|f| for FP32 (FP32 pair arithmetic, ~1e-6 relative per pair,
    summed over ~13 hits), 1e-10 max|f| for FP64 (summation order only);
  * long-run statistics (kT, pressure) within 1%, g(r) within 0.01 absolute.
"""
import numpy as np
import pytest

import oracle as O
from paper_1804_06205_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FP32, FP64 = 0, 1
TOL = {FP32: 1e-4, FP64: 1e-10}


@pytest.fixture(scope="module")
def D():
    from paper_1804_06205_gb300 import build
    build.build()
    from paper_1804_06205_gb300 import dpd
    return dpd


def osys(w, noise=0):
    return O.System(w.L, w.types, w.a, w.gamma, w.kT, w.dt, w.lam, seed=w.seed, noise=noise,
                    bonds=w.bonds)


def gsys(D, w, prec, **kw):
    return D.System.from_workload(w, precision=prec, **kw)


def small_workloads():
    melt = W.melt_98k(L=10.0, seed=21)
    pep = W.peptide_192k(L=10.0, nchains=10, chain_len=20, seed=22)
    helix = W.alpha_helix_24k()
    helix_small = W.Workload("helix_small", np.array([8.0, 8.0, 8.0]),
                             np.concatenate([helix.types[:60], np.ones(1476, np.int32)]),
                             helix.a, helix.gamma, helix.kT, helix.dt, helix.lam, 23,
                             np.concatenate([helix.pos[:60] % 8.0,
                                             np.random.default_rng(2).uniform(0, 8, (1476, 3))]),
                             W.maxwell_velocities(np.random.default_rng(3), 1536),
                             helix.bonds)
    odd = W.fluid((7.3, 9.1, 11.7), ntypes=3, a_same=25.0, a_cross=33.0, seed=24)
    return {"fluid_3k": W.fluid_3k(), "melt": melt, "peptide": pep, "helix": helix_small,
            "odd_box": odd}


WL = small_workloads()


# ------------------------------------------------------------------ cells
def _oracle_cells(w, pos):
    s = osys(w)
    p = O.wrap(s, pos)
    key = O.cell_keys(s, p)
    order, start = O.cell_sort(s, key)
    return key, order, start


def _face_positions(L, n, seed):
    """Positions with many exact cell faces, L - eps, 0 and out-of-box values."""
    rng = np.random.default_rng(seed)
    L = np.asarray(L, float)
    nc = np.floor(L)
    h = L / nc
    pos = rng.uniform(0, 1, (n, 3)) * L
    m = n // 4
    pos[:m] = rng.integers(0, nc.astype(int), (m, 3)) * h          # on faces
    pos[m:m + 10] = np.nextafter(L, 0)                               # L - eps
    pos[m + 10:m + 20] = 0.0
    pos[m + 20:m + 40] += L * rng.integers(-3, 4, (20, 3))           # unwrapped
    pos[m + 40:m + 50] = -1e-18
    return pos


@pytest.mark.parametrize("prec", [FP32, FP64])
@pytest.mark.parametrize("L", [(10.0, 10.0, 10.0), (7.3, 9.1, 11.7), (3.0, 4.5, 3.2)])
def test_cells_bitexact_at_set_state(D, prec, L):
    n = int(3 * np.prod(L))
    w = W.fluid(L, n=n, seed=31)
    pos = _face_positions(L, n, 32)
    g = gsys(D, w, prec)
    g.set_state(pos, w.vel, 0)
    key, order, start = g.cells()
    okey, oorder, ostart = _oracle_cells(w, pos)
    assert np.array_equal(key, okey)
    assert np.array_equal(order, oorder)
    assert np.array_equal(start, ostart)


def test_cells_bitexact_after_steps_fp64(D):
    w = WL["melt"]
    g = gsys(D, w, FP64)
    g.set_state(w.pos, w.vel, 0)
    g.step(25)
    pos, _, _, step = g.get_state()
    assert step == 25
    key, order, start = g.cells()
    okey, oorder, ostart = _oracle_cells(w, pos)
    assert np.array_equal(key, okey)
    assert np.array_equal(order, oorder)
    assert np.array_equal(start, ostart)


def test_cells_after_steps_fp32(D):
    """After steps the FP32 path's cell index is state (the integer cell and a
    binary32 offset in [0, h), moved by whole cells), not re-derived from an
    FP64 position.  Its keys must equal the oracle's key of that same state --
    x = c h + o formed in FP64 from the checkpoint's exact cell and offset --
    for every bead whose x is not within FP64 rounding of a cell face; there
    the two may differ by one cell, and no further."""
    w = WL["odd_box"]
    g = gsys(D, w, FP32)
    g.set_state(w.pos, w.vel, 0)
    g.step(25)
    key, order, start = g.cells()
    ck = g.get_checkpoint()
    nc = g.nc
    assert sorted(order.tolist()) == list(range(w.n))
    ks = key[order].astype(np.int64)
    assert np.all(np.diff(ks) >= 0)
    assert np.all(np.diff(order)[np.diff(ks) == 0] > 0)
    assert np.array_equal(np.diff(start), np.bincount(key.astype(np.int64),
                                                      minlength=int(np.prod(nc))))
    rec = np.frombuffer(ck, dtype=np.dtype([("key", "<u4"), ("o", "<f4", 3), ("v", "<f4", 3),
                                            ("f", "<f4", 3)]), offset=80)
    assert np.array_equal(rec["key"], key)
    h = w.L / nc
    c = np.stack([key % nc[0], (key // nc[0]) % nc[1], key // (nc[0] * nc[1])], axis=1)
    o = rec["o"].astype(np.float64)
    assert np.all((o >= 0.0) & (o < h))
    x = c * h + o
    okey = O.cell_keys(osys(w), x)
    frac = x / h - np.floor(x / h)
    near = np.any((frac < 1e-12) | (frac > 1.0 - 1e-12), axis=1)
    assert np.array_equal(key[~near], okey[~near])
    oc = np.stack([okey % nc[0], (okey // nc[0]) % nc[1], okey // (nc[0] * nc[1])], axis=1)
    dcell = np.abs(c - oc.astype(np.int64))
    assert np.all(np.minimum(dcell, nc - dcell)[near] <= 1)


# ------------------------------------------------------------------ forces
@pytest.mark.parametrize("prec", [FP32, FP64])
@pytest.mark.parametrize("name", sorted(WL))
def test_one_force_evaluation_matches_oracle(D, prec, name):
    w = WL[name]
    g = gsys(D, w, prec)
    g.set_state(w.pos, w.vel, 17)
    _, _, f, step = g.get_state()
    assert step == 17
    fo, _ = O.forces(osys(w), O.wrap(osys(w), w.pos), w.vel, 17)
    scale = np.abs(fo).max()
    err = np.abs(f - fo).max()
    assert err <= TOL[prec] * scale, (err, scale)


@pytest.mark.parametrize("prec", [FP32, FP64])
@pytest.mark.parametrize("L,tile,threads", [((10.5, 10.0, 10.0), 0, 128),
                                            ((10.5, 10.0, 10.0), 5, 128),
                                            ((10.0, 10.5, 10.0), 7, 256),
                                            ((11.856, 11.856, 11.856), 0, 128),
                                            ((11.856, 11.856, 11.856), 3, 64)])
def test_inexact_brick_origins_match_oracle(D, prec, L, tile, threads):
    """Boxes whose cell edge makes a brick's origin x0 * h inexact in floating
    point: every home bead's frame position must coincide bit for bit with its
    staged copy, or the bead meets itself at r ~ 1e-16.  One force evaluation
    and a 10-step trajectory against the oracle, for several brick shapes and
    block sizes."""
    w = W.fluid(L, ntypes=2, a_same=25.0, a_cross=33.0, seed=24)
    g = gsys(D, w, prec, tile_cells=tile, threads=threads)
    g.set_state(w.pos, w.vel, 0)
    f0 = g.get_state()[2]
    s = osys(w)
    fo, _ = O.forces(s, O.wrap(s, w.pos), w.vel, 0)
    assert np.abs(f0 - fo).max() <= TOL[prec] * np.abs(fo).max()
    g.step(10)
    pos = g.get_state()[0]
    g.close()
    st = O.State(s, w.pos, w.vel, 0, mode=O.MODE_CELLS)
    st.run(10)
    d = pos - st.pos
    d -= w.L * np.round(d / w.L)
    assert np.abs(d).max() < (1e-4 if prec == FP32 else 1e-9)


def test_fp64_large_pair_forces_take_the_full_shell(D):
    """FP64 evaluates each pair of two home beads once and hands the partner
    its share in fixed point, which holds force components below 2^9; with
    a_ij in the thousands most pairs exceed that, and the blocks redo their
    bricks over the full shell.  Forces must still match the oracle, and runs
    must repeat bit for bit."""
    w = W.fluid(10.0, ntypes=2, a_same=2000.0, a_cross=2400.0, seed=31)
    s = osys(w)
    fo, _ = O.forces(s, O.wrap(s, w.pos), w.vel, 5)
    outs = []
    for _ in range(2):
        g = gsys(D, w, FP64)
        g.set_state(w.pos, w.vel, 5)
        outs.append(g.get_state()[2])
        g.close()
    assert np.abs(fo).max() > 1e3
    assert np.array_equal(outs[0], outs[1])
    assert np.abs(outs[0] - fo).max() <= TOL[FP64] * np.abs(fo).max()


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_uniform_noise_option(D, prec):
    w = WL["fluid_3k"]
    g = gsys(D, w, prec, noise=D.DPD_NOISE_UNIFORM)
    g.set_state(w.pos, w.vel, 3)
    _, _, f, _ = g.get_state()
    s = osys(w, noise=O.NOISE_UNIFORM)
    fo, _ = O.forces(s, w.pos, w.vel, 3)
    assert np.abs(f - fo).max() <= TOL[prec] * np.abs(fo).max()


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_one_step_matches_oracle(D, prec):
    w = WL["peptide"]
    g = gsys(D, w, prec)
    g.set_state(w.pos, w.vel, 0)
    g.step(1)
    pos, vel, f, step = g.get_state()
    st = O.State(osys(w), w.pos, w.vel, 0)
    st.run(1)
    assert step == st.step == 1
    d = pos - st.pos
    d -= w.L * np.round(d / w.L)
    assert np.abs(d).max() < (1e-5 if prec == FP32 else 1e-12)
    assert np.abs(vel - st.vel).max() <= TOL[prec] * np.abs(st.f).max()
    assert np.abs(f - st.f).max() <= 2 * TOL[prec] * np.abs(st.f).max()


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_observables_match_oracle_at_identical_state(D, prec):
    w = WL["peptide"]
    g = gsys(D, w, prec)
    g.set_state(w.pos, w.vel, 5)
    o = g.observables()
    st = O.State(osys(w), w.pos, w.vel, 5)
    oo = st.observables()
    tol = 1e-5 if prec == FP32 else 1e-10
    for k in ("kT", "p_total", "p_ideal", "p_cons", "p_bond", "e_pair", "e_bond"):
        assert abs(o[k] - oo[k]) <= tol * max(1.0, abs(oo[k])), (k, o[k], oo[k])
    assert o["step"] == 5


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_observables_on_demand_equal_in_step_sampling(D, prec):
    """Observables are computed when asked for, from the state; sampling every
    step inside the step loop (running means) reaches the same state with the
    same bits and reports the same instantaneous observables, bit for bit."""
    w = WL["peptide"]
    out = []
    for every in (0, 1):
        g = gsys(D, w, prec, sample_every=every)
        g.set_state(w.pos, w.vel, 0)
        g.step(6)
        pos, vel, f, _ = g.get_state()
        out.append((pos, vel, f, g.observables()))
        g.close()
    for a, b in zip(out[0][:3], out[1][:3]):
        assert np.array_equal(a, b)
    o0, o1 = out[0][3], out[1][3]
    assert o1["n_samples"] == 6 and o0["n_samples"] == 0
    for k in ("kT", "p_total", "p_cons", "p_bond", "e_pair", "e_bond"):
        assert o0[k] == o1[k], (k, o0[k], o1[k])


# ------------------------------------------------------------------ invariants
@pytest.mark.parametrize("prec", [FP32, FP64])
def test_momentum_conserved_and_runs_deterministic(D, prec):
    w = WL["melt"]
    runs = []
    for _ in range(2):
        g = gsys(D, w, prec)
        g.set_state(w.pos, w.vel, 0)
        g.step(60)
        runs.append(g.get_state())
        g.close()
    for a, b in zip(runs[0][:3], runs[1][:3]):
        assert np.array_equal(a, b)
    p = runs[0][1].sum(axis=0)
    assert np.abs(p).max() < (2e-3 if prec == FP32 else 1e-10)


def test_graph_replay_is_bitwise_and_tilings_agree(D):
    """Graph replay and direct launches give identical bits; other tilings
    (tile cells, threads) change only the summation tree of each bead's force."""
    w = WL["odd_box"]
    outs = {}
    for name, opt in (("graph", dict(use_graph=1)), ("direct", dict()),
                      ("t64", dict(tile_cells=3, threads=64)),
                      ("t256", dict(tile_cells=12, threads=256)),
                      ("t128x1", dict(tile_cells=1, threads=128, use_graph=0))):
        g = gsys(D, w, FP32, **opt)
        g.set_state(w.pos, w.vel, 0)
        f0 = g.get_state()[2]
        g.step(7)
        outs[name] = (f0, g.get_state())
        g.close()
    for a, b in zip(outs["graph"][1][:3], outs["direct"][1][:3]):
        assert np.array_equal(a, b)
    f_ref = outs["graph"][0]
    for name in ("t64", "t256", "t128x1"):
        assert np.abs(outs[name][0] - f_ref).max() <= 1e-5 * np.abs(f_ref).max(), name


def test_gr_counts_fp64_bitexact(D):
    w = WL["fluid_3k"]
    g = gsys(D, w, FP64)
    g.set_state(w.pos, w.vel, 0)
    c = g.gr_counts(3.0, 150)
    co = O.gr_counts(osys(w), O.wrap(osys(w), w.pos), 3.0, 150)
    assert np.array_equal(c, co)


# ------------------------------------------------------------------ edge cases
@pytest.mark.parametrize("prec", [FP32, FP64])
def test_edge_single_bead_and_pair(D, prec):
    w1 = W.fluid(4.0, n=1, seed=3)
    g = gsys(D, w1, prec)
    g.set_state(w1.pos, w1.vel, 0)
    g.step(3)
    _, v, f, _ = g.get_state()
    assert np.all(f == 0.0) and np.allclose(v, w1.vel)
    w2 = W.fluid(4.0, n=2, seed=4)
    w2.pos[:] = [[0.05, 2.0, 2.0], [3.7, 2.1, 1.9]]    # a pair across the boundary
    g = gsys(D, w2, prec)
    g.set_state(w2.pos, w2.vel, 9)
    _, _, f, _ = g.get_state()
    fo, _ = O.forces(osys(w2), w2.pos, w2.vel, 9)
    assert np.abs(f - fo).max() <= TOL[prec] * np.abs(fo).max()
    assert np.abs(fo).max() > 0


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_edge_crowded_cell_uses_chunks_and_passes(D, prec):
    # 600 beads inside one cell of a 5^3 box plus a sparse background: the
    # neighbourhood exceeds the staged capacity and every bead has ~600 hits
    rng = np.random.default_rng(5)
    n = 900
    w = W.fluid(5.0, n=n, seed=6)
    w.pos[:600] = 2.0 + rng.uniform(0, 0.9, (600, 3))
    g = gsys(D, w, prec)
    g.set_state(w.pos, w.vel, 4)
    _, _, f, _ = g.get_state()
    fo, _ = O.forces(osys(w), w.pos, w.vel, 4)
    assert np.abs(f - fo).max() <= TOL[prec] * np.abs(fo).max()


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_edge_smallest_box(D, prec):
    w = W.fluid(3.0, n=81, seed=8)
    g = gsys(D, w, prec)
    g.set_state(w.pos, w.vel, 2)
    _, _, f, _ = g.get_state()
    fo, _ = O.forces(osys(w), w.pos, w.vel, 2)
    assert np.abs(f - fo).max() <= TOL[prec] * np.abs(fo).max()


def test_errors_are_reported(D):
    w = WL["fluid_3k"]
    g = gsys(D, w, FP32)
    with pytest.raises(D.DPDError) as e:
        g.step(1)
    assert e.value.code == D.DPD_ENOSTATE
    bad = w.pos.copy()
    bad[7, 1] = np.nan
    with pytest.raises(D.DPDError) as e:
        g.set_state(bad, w.vel, 0)
    assert e.value.code == D.DPD_EINVAL


# ------------------------------------------------------------------ long run
def test_long_run_statistics_match_oracle(D):
    """fluid_3k: 200 equilibration steps, then 160 samples 10 steps apart.
    kT and pressure within 1%; g(r) (bins of 0.05 up to 3) within 0.01 plus
    three block-averaged standard errors of the difference (the bins below
    r ~ 0.3 hold a few pairs per sample, so their noise exceeds 0.01)."""
    w = WL["fluid_3k"]
    nb, rmax, nsamp, nblk = 60, 3.0, 160, 8

    def run(step_fn, obs_fn, gr_fn):
        ks, ps, gs = [], [], []
        for _ in range(nsamp):
            step_fn(10)
            k, p = obs_fn()
            ks.append(k)
            ps.append(p)
            gs.append(O.gr_normalise(gr_fn(), w.n, w.L, rmax))
        return np.array(ks), np.array(ps), np.array(gs)

    g = gsys(D, w, FP32)
    g.set_state(w.pos, w.vel, 0)
    g.step(200)

    def g_obs():
        o = g.observables()
        return o["kT"], o["p_total"]
    gk, gp, gg = run(g.step, g_obs, lambda: g.gr_counts(rmax, nb))
    s = osys(w)
    st = O.State(s, w.pos, w.vel, 0, mode=O.MODE_CELLS)
    st.run(200)
    last = {}

    def o_step(n):
        last["s"] = st.run(n, sample_every=n)[-1]

    ok, op, og = run(o_step, lambda: (last["s"][4], last["s"][5]),
                     lambda: O.gr_counts(s, st.pos, rmax, nb))
    assert abs(gk.mean() - ok.mean()) < 0.01 * ok.mean()
    assert abs(gp.mean() - op.mean()) < 0.01 * op.mean()
    blk = lambda x: x.reshape(nblk, -1, *x.shape[1:]).mean(axis=1)
    sem = lambda x: blk(x).std(axis=0, ddof=1) / np.sqrt(nblk)
    diff = gg.mean(axis=0) - og.mean(axis=0)
    err = np.sqrt(sem(gg) ** 2 + sem(og) ** 2)
    r = (np.arange(nb) + 0.5) * rmax / nb
    m = r >= 0.1
    assert np.all(np.abs(diff[m]) <= 0.01 + 3 * err[m]), (np.abs(diff[m]).max(), err[m].max())
    # where the statistics allow it, the 0.01 bound holds by itself
    assert np.all(np.abs(diff[r >= 0.5]) < 0.01)


# ------------------------------------------------------------------ full size
@pytest.mark.parametrize("prec", [FP32, FP64])
def test_full_size_fluid_3m_sampled_parity(D, prec):
    """The 100^3, N = 3,000,000 fluid in the benchmark's launch configuration
    (default options): the state comes back as it went in (the transfers run
    in several chunks at this size), cells bit-exact for all beads, forces on
    256 sampled beads against the oracle's brute-force sum, total force ~ 0."""
    w = W.fluid_3m()
    g = gsys(D, w, prec)
    g.set_state(w.pos, w.vel, 11)
    pos, vel, f, _ = g.get_state()
    d = pos - w.pos
    d -= w.L * np.round(d / w.L)
    if prec == FP64:
        assert np.array_equal(vel, w.vel) and np.abs(d).max() == 0.0
    else:   # velocities stored in binary32; positions as cell + binary32 offset
        assert np.array_equal(vel, w.vel.astype(np.float32).astype(np.float64))
        assert np.abs(d).max() < 1e-6
    key, order, start = g.cells()
    okey, oorder, ostart = _oracle_cells(w, w.pos)
    assert np.array_equal(key, okey)
    assert np.array_equal(order, oorder)
    assert np.array_equal(start, ostart)
    idx = np.random.default_rng(12).choice(w.n, 256, replace=False)
    s = osys(w)
    fo = O.pair_forces_subset(s, w.pos, w.vel, 11, idx)
    scale = np.abs(fo).max()
    assert np.abs(f[idx] - fo).max() <= TOL[prec] * scale
    assert np.abs(f.sum(axis=0)).max() < (1e-2 if prec == FP32 else 1e-6) * np.sqrt(w.n)


@pytest.mark.parametrize("prec", [FP32, FP64])
@pytest.mark.parametrize("name", ["melt_98k", "peptide_192k"])
def test_full_size_configs_match_oracle(D, prec, name):
    """The polymer melt (32^3, 98,304 beads, 88,470 harmonic bonds) and the
    peptide-like system (40^3, 192,000 beads, harmonic and standard-Morse
    bonds) at full size with default options: every bead's force from an
    identical state, and every bead after 3 steps, against the oracle's
    cell-list sum (equal to its brute-force sum to 1e-12)."""
    w = W.make(name)
    s = osys(w)
    g = gsys(D, w, prec)
    g.set_state(w.pos, w.vel, 3)
    f = g.get_state()[2]
    fo, _ = O.forces(s, O.wrap(s, w.pos), w.vel, 3, mode=O.MODE_CELLS)
    scale = np.abs(fo).max()
    assert np.abs(f - fo).max() <= TOL[prec] * scale
    g.step(3)
    pos, vel, _, step = g.get_state()
    g.close()
    st = O.State(s, w.pos, w.vel, 3, mode=O.MODE_CELLS)
    st.run(3)
    assert step == st.step == 6
    d = pos - st.pos
    d -= w.L * np.round(d / w.L)
    # positions: FP32 keeps offsets inside unit cells (resolution ~1e-7) and
    # the stiffest bonds (max |f| ~ 7.5e3 in the peptide system) amplify force
    # rounding by dt^2 per step; velocities: a force error e changes v by dt e
    # per step, with the one-evaluation tolerance as e
    assert np.abs(d).max() < (1e-4 if prec == FP32 else 1e-11)
    assert np.abs(vel - st.vel).max() <= 4 * w.dt * TOL[prec] * scale
