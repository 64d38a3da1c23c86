"""Pins of the oracle's force terms: eq. 4 (conservative), the Groot-Warren
dissipative / random terms, eqs. 6-8 and Fig. 3a (bonded terms), eq. 3
(pair sum) and the cell-list mode against the brute-force definition."""
import numpy as np
import pytest

import oracle as O
from paper_1804_06205_gb300 import workloads as W


def _two_beads(d, vi=(0, 0, 0), vj=(0, 0, 0), a=25.0, gamma=0.0, kT=0.0, dt=0.04, L=10.0):
    pos = np.array([[5.0, 5.0, 5.0], np.array([5.0, 5.0, 5.0]) - np.asarray(d, float)])
    vt = np.array([vi, vj], dtype=float)
    sys_ = O.System(L, [0, 0], [[a]], gamma, kT, dt, seed=11)
    return sys_, pos, vt


def test_conservative_single_pair_eq4():
    # a = 25 at r = 0.5: |F^C| = a (1 - r) = 12.5, pointing from j to i (repulsive)
    s, pos, vt = _two_beads([0.5, 0.0, 0.0])
    F = O.pair_force_one(s, pos, vt, 0, 1, 0)
    assert np.allclose(F, [12.5, 0.0, 0.0], rtol=0, atol=1e-13)
    rng = np.random.default_rng(3)
    for _ in range(200):
        r = rng.uniform(0.0, 1.2)
        e = rng.normal(size=3)
        e /= np.linalg.norm(e)
        a = rng.uniform(0.0, 80.0)
        s, pos, vt = _two_beads(r * e, a=a)
        F = O.pair_force_one(s, pos, vt, 0, 1, 0)
        expect = a * (1.0 - r) * e if r < 1.0 else np.zeros(3)
        assert np.allclose(F, expect, rtol=1e-12, atol=1e-12)
    # the cutoff itself contributes nothing, nor does r == 0
    s, pos, vt = _two_beads([1.0, 0.0, 0.0])
    assert np.all(O.pair_force_one(s, pos, vt, 0, 1, 0) == 0.0)
    s, pos, vt = _two_beads([0.0, 0.0, 0.0])
    assert np.all(O.pair_force_one(s, pos, vt, 0, 1, 0) == 0.0)


def test_conservative_through_periodic_boundary():
    s = O.System(10.0, [0, 0], [[25.0]], 0.0, 0.0, 0.04)
    pos = np.array([[0.1, 5.0, 5.0], [9.7, 5.0, 5.0]])   # image distance 0.4
    F = O.pair_force_one(s, pos, np.zeros((2, 3)), 0, 1, 0)
    assert np.allclose(F, [25.0 * 0.6, 0, 0], atol=1e-12)


def test_dissipative_worked_example():
    # kT = 0 switches the random term off (sigma^2 = 2 gamma kT).  i at the
    # origin moving towards j at +0.5 x with unit speed: e = -x, e.v_ij = -1,
    # w = 0.5, gamma w^2 = 4.5 * 0.25 = 1.125 -> F_i = -1.125 x (brakes i).
    s, pos, vt = _two_beads([-0.5, 0.0, 0.0], vi=(1.0, 0, 0), a=0.0, gamma=4.5, kT=0.0)
    F = O.pair_force_one(s, pos, vt, 0, 1, 0)
    assert np.allclose(F, [-1.125, 0.0, 0.0], atol=1e-13)
    # relative velocity perpendicular to the bond: no dissipative force
    s, pos, vt = _two_beads([-0.5, 0.0, 0.0], vi=(0.0, 2.0, -1.0), a=0.0, gamma=4.5, kT=0.0)
    assert np.allclose(O.pair_force_one(s, pos, vt, 0, 1, 0), 0.0, atol=1e-14)
    # power is never positive, linear in v
    rng = np.random.default_rng(5)
    for _ in range(100):
        d = rng.uniform(-0.55, 0.55, 3)
        vi, vj = rng.normal(size=3), rng.normal(size=3)
        s, pos, vt = _two_beads(d, vi=vi, vj=vj, a=0.0, gamma=4.5, kT=0.0)
        F1 = O.pair_force_one(s, pos, vt, 0, 1, 0)
        assert np.dot(F1, vi - vj) <= 1e-14
        s2, pos2, vt2 = _two_beads(d, vi=2 * vi, vj=2 * vj, a=0.0, gamma=4.5, kT=0.0)
        assert np.allclose(O.pair_force_one(s2, pos2, vt2, 0, 1, 0), 2 * F1, atol=1e-12)


def test_random_force_variance_fluctuation_dissipation():
    # with v~ = 0 and a = 0 only F^R remains: <(F.e)^2> dt / w^2 = sigma^2 = 2 gamma kT
    gamma, kT, dt, r = 4.5, 1.0, 0.04, 0.3
    s, pos, vt = _two_beads([r, 0, 0], a=0.0, gamma=gamma, kT=kT, dt=dt)
    fx = np.array([O.pair_force_one(s, pos, vt, 0, 1, step)[0] for step in range(40000)])
    w = 1.0 - r
    var = np.mean(fx ** 2) * dt / w ** 2
    assert abs(var - 2 * gamma * kT) < 4 * np.sqrt(2.0 / fx.size) * 2 * gamma * kT
    assert abs(fx.mean()) < 4 * np.sqrt(2 * gamma * kT) * w / np.sqrt(dt) / np.sqrt(fx.size)


def test_pair_sum_newton_third_law_and_cells_equal_brute():
    w = W.fluid(7.3, n=1200, ntypes=2, a_cross=40.0, seed=42)
    s = O.System(w.L, w.types, w.a, w.gamma, w.kT, w.dt, seed=77)
    vt = w.vel
    fb, tb = O.pair_forces(s, w.pos, vt, 5, O.MODE_BRUTE)
    fc, tc = O.pair_forces(s, w.pos, vt, 5, O.MODE_CELLS)
    scale = np.abs(fb).max()
    assert np.abs(fb.sum(axis=0)).max() < 1e-11 * scale * np.sqrt(w.n)
    assert np.abs(fb - fc).max() < 1e-12 * scale
    assert abs(tb.wc - tc.wc) < 1e-10 * abs(tb.wc)
    assert abs(tb.ep - tc.ep) < 1e-10 * abs(tb.ep)


@pytest.mark.parametrize("L", [(3.0, 3.0, 3.0), (3.5, 4.2, 9.9), (11.7, 5.0, 3.0)])
def test_cells_equal_brute_small_and_odd_boxes(L):
    rng = np.random.default_rng(int(sum(L) * 10))
    L = np.array(L)
    n = int(3 * np.prod(L))
    pos = rng.uniform(0, 1, (n, 3)) * L
    s = O.System(L, np.zeros(n, np.int32), [[25.0]], 4.5, 1.0, 0.04, seed=3)
    vt = rng.normal(size=(n, 3))
    fb, _ = O.pair_forces(s, pos, vt, 9, O.MODE_BRUTE)
    fc, _ = O.pair_forces(s, pos, vt, 9, O.MODE_CELLS)
    assert np.abs(fb - fc).max() < 1e-12 * np.abs(fb).max()


def _fd_force(kind, r0, k, alpha, d, h=1e-6):
    g = np.zeros(3)
    for c in range(3):
        dp, dm = d.copy(), d.copy()
        dp[c] += h
        dm[c] -= h
        g[c] = -(O.bond_one(kind, r0, k, alpha, dp)[1] - O.bond_one(kind, r0, k, alpha, dm)[1]) / (2 * h)
    return g


@pytest.mark.parametrize("kind,r0,k,alpha", [(1, 0.0, 4.0, 0.0), (1, 0.5, 4.0, 0.0),
                                              (1, 0.6, 160.0, 0.0), (3, 0.7, 5.0, 3.0),
                                              (3, 1.0, 5.0, 3.0)])
def test_bond_force_is_minus_gradient_of_energy(kind, r0, k, alpha):
    rng = np.random.default_rng(kind * 100 + int(r0 * 10))
    for _ in range(50):
        d = rng.normal(size=3) * 0.6
        F, _ = O.bond_one(kind, r0, k, alpha, d)
        g = _fd_force(kind, r0, k, alpha, d)
        assert np.allclose(F, g, rtol=1e-6, atol=1e-6 * max(1.0, np.abs(g).max()))


def test_harmonic_r0_zero_is_minus_k_d():
    # "F = -4 r" springs (k = 4, r0 = 0): the force is -k d exactly
    d = np.array([0.3, -0.2, 0.9])
    F, U = O.bond_one(1, 0.0, 4.0, 0.0, d)
    assert np.allclose(F, -4.0 * d, atol=1e-15)
    assert abs(U - 2.0 * d.dot(d)) < 1e-15


@pytest.mark.parametrize("kind", [2, 3])
def test_morse_force_vanishes_at_r0(kind):
    for r0 in (0.6, 0.7, 0.9, 1.0):
        e = np.array([1.0, 2.0, -2.0]) / 3.0
        F, _ = O.bond_one(kind, r0, 12.0, 8.0, r0 * e)
        assert np.abs(F).max() < 1e-12


def _fig3a(kind, r_e, const, const2, d):
    """The bond lines of Fig. 3a written out: dx = r_e - r (the sign that
    makes the harmonic line restoring), dr0 the unit vector from j to i."""
    r = np.linalg.norm(d)
    dr0 = d / r
    dx = r_e - r
    if kind == 1:
        return const * dx * dr0, 0.5 * const * dx * dx
    exppart = np.exp(-const2 * abs(dx))
    expminusone = exppart - 1.0
    const_exp = const * expminusone
    return 2.0 * const_exp * const2 * exppart * dr0, const_exp * expminusone


def test_bonds_match_fig3a_lines():
    rng = np.random.default_rng(8)
    # the alpha-helix deck values of Fig. 3b
    for kind, r_e, c1, c2 in [(1, 0.6, 160.0, 0.0), (1, 1.2, 80.0, 0.0), (2, 0.9, 12.0, 8.0),
                              (2, 0.6, 12.0, 8.0)]:
        for _ in range(40):
            d = rng.normal(size=3)
            d *= rng.uniform(0.05, 2.0) / np.linalg.norm(d)
            F, U = O.bond_one(kind, r_e, c1, c2, d)
            Fp, Up = _fig3a(kind, r_e, c1, c2, d)
            assert np.allclose(F, Fp, rtol=1e-13, atol=1e-13)
            assert abs(U - Up) < 1e-12 * max(1.0, abs(Up))
            if kind == 2:
                # same direction (towards j) on both sides of r_e, bounded by K alpha / 2
                assert np.dot(F, d) <= 0.0
                assert np.linalg.norm(F) <= c1 * c2 / 2.0 + 1e-12


def test_bond_forces_antisymmetric_through_boundary():
    L = 6.0
    pos = np.array([[0.2, 3.0, 3.0], [5.9, 3.1, 2.9], [1.0, 1.0, 1.0]])
    bonds = W.concat_bonds([W.bond_records([0], [1], 1, 0.5, 4.0),
                            W.bond_records([0], [2], 3, 0.7, 5.0, 3.0)])
    s = O.System(L, [0, 0, 0], [[25.0]], 4.5, 1.0, 0.04, bonds=bonds)
    f, t = O.bond_forces(s, pos)
    assert np.abs(f.sum(axis=0)).max() < 1e-13
    d = np.array([0.2 - 5.9 + 6.0, -0.1, 0.1])
    F01, _ = O.bond_one(1, 0.5, 4.0, 0.0, d)
    F02, _ = O.bond_one(3, 0.7, 5.0, 3.0, pos[0] - pos[2])
    assert np.allclose(f[0], F01 + F02, atol=1e-13)
    assert np.allclose(f[1], -F01, atol=1e-13)


def test_subset_forces_equal_full_rows():
    w = W.fluid(6.0, n=700, ntypes=2, a_cross=35.0, seed=4)
    s = O.System(w.L, w.types, w.a, w.gamma, w.kT, w.dt, seed=5)
    f, _ = O.pair_forces(s, w.pos, w.vel, 3)
    idx = np.array([0, 5, 699, 350, 5])
    fs = O.pair_forces_subset(s, w.pos, w.vel, 3, idx)
    assert np.array_equal(fs, f[idx])
