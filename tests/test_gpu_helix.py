"""The paper's alpha-helix model (section "Formation of protein structure",
Figs. 3-5: 24,000 beads in a 20^3 box, a 60-bead skeletal chain with 1-2
harmonic, 1-3 harmonic + modified Morse and 1-5 modified Morse bonds,
gamma = 4.2, dt = 0.02) on the GPU against the oracle.

Trajectories are chaotic, so the comparison is of averages over a run with
block error bars: mean 1-2, 1-3 and 1-5 distances along the chain, kT and
pressure.  The paper shows its result only as a picture (Fig. 5), so
agreement with the paper itself is not pinned; the helicity proxy (mean 1-5
distance, which the 1-5 Morse term pulls towards r_e = 0.6 and below, and
the consistency of the sign of consecutive dihedral angles) is reported."""
import numpy as np
import pytest

from paper_1804_06205_gb300 import workloads as W

pytestmark = pytest.mark.gpu

NSTEPS, EVERY, SKIP = 2000, 50, 10      # samples after the first 500 steps


@pytest.fixture(scope="module")
def D():
    from paper_1804_06205_gb300 import build
    build.build()
    from paper_1804_06205_gb300 import dpd
    return dpd


def chain_stats(pos, L, nb=60):
    p = pos[:nb]
    out = []
    for k in (1, 2, 4):
        d = p[k:] - p[:-k]
        d -= L * np.round(d / L)
        out.append(np.linalg.norm(d, axis=1).mean())
    return out


def dihedral_sign_order(pos, L, nb=60):
    """|mean sign| of the dihedral angles of consecutive 4-bead windows: 1 for
    a regular helix of one hand, ~0 for a random coil."""
    p = pos[:nb].copy()
    for i in range(1, nb):          # unwrap the chain
        d = p[i] - p[i - 1]
        p[i] = p[i - 1] + d - L * np.round(d / L)
    b1, b2, b3 = p[1:-2] - p[:-3], p[2:-1] - p[1:-2], p[3:] - p[2:-1]
    s = np.einsum("ij,ij->i", np.cross(b1, b2), b3)
    return abs(np.mean(np.sign(s)))


def series_gpu(D, w, prec):
    g = D.System.from_workload(w, precision=prec)
    g.set_state(w.pos, w.vel, 0)
    rows = []
    for _ in range(NSTEPS // EVERY):
        g.step(EVERY)
        o = g.observables()
        pos = g.get_state(vel=False, force=False)[0]
        rows.append(chain_stats(pos, w.L) + [o["kT"], o["p_total"],
                                             dihedral_sign_order(pos, w.L)])
    g.close()
    return np.array(rows)


@pytest.fixture(scope="module")
def oracle_series():
    import oracle as O
    w = W.alpha_helix_24k()
    s = O.System(w.L, w.types, w.a, w.gamma, w.kT, w.dt, w.lam, seed=w.seed, bonds=w.bonds)
    st = O.State(s, w.pos, w.vel, 0, mode=O.MODE_CELLS)
    rows = []
    for _ in range(NSTEPS // EVERY):
        st.run(EVERY)
        o = st.observables()
        rows.append(chain_stats(st.pos, w.L) + [o["kT"], o["p_total"],
                                                dihedral_sign_order(st.pos, w.L)])
    return np.array(rows)


def mean_err(x, nblocks=5):
    x = np.asarray(x)[SKIP:]
    b = np.array([blk.mean() for blk in np.array_split(x, nblocks)])
    return x.mean(), b.std(ddof=1) / np.sqrt(nblocks)


@pytest.mark.parametrize("prec", [0, 1])
def test_alpha_helix_statistics_match_oracle(D, oracle_series, prec):
    w = W.alpha_helix_24k()
    gpu = series_gpu(D, w, prec)
    names = ("d12", "d13", "d15", "kT", "p")
    floors = (0.01, 0.02, 0.03, 0.01, 0.15)
    for k, (name, floor) in enumerate(zip(names, floors)):
        mg, eg = mean_err(gpu[:, k])
        mo, eo = mean_err(oracle_series[:, k])
        tol = 4.0 * np.hypot(eg, eo) + floor
        assert abs(mg - mo) < tol, (name, mg, mo, tol)
    # the 1-5 Morse term has pulled the chain in from its random-walk start
    assert mean_err(gpu[:, 2])[0] < 0.7
