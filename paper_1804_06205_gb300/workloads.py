"""Seeded synthetic DPD systems shaped like the paper's workloads.

This module only draws initial conditions and parameter sets (numpy
``default_rng``); it holds none of the method's arithmetic and is the one
module that both the CUDA engine's callers and the oracle's tests use.

Workloads (sizes and parameters are the ones each benchmark is quoted on):
  * ``fluid_3k``        10^3 box, rho=3, N=3000, a=25 (the paper's benchmark
                        fluid, section "Performance and parallel efficiency")
  * ``melt_98k``        32^3 box, 9830 A5B5 10-bead chains + 4 free beads,
                        harmonic k=4, r0=0; a_AA=a_BB=25, a_AB=40
  * ``peptide_192k``    40^3 box, 200 chains x 20 backbone beads in solvent,
                        1-2 harmonic (k=4, r0=0.5), 1-3 and 1-5 standard
                        Morse (D=5, alpha=3, r0=0.7 / 1.0)
  * ``fluid_3m``        100^3 box, N=3,000,000, types A/B 50/50,
                        a_AA=a_BB=25, a_AB=30
  * ``serving_stream``  256 systems, Poisson(20/s) arrivals, edge U[8,24],
                        a_AB U[25,50], 10% of beads in 10-bead chains
  * ``alpha_helix_24k`` the paper's alpha-helix model (section "Formation of
                        protein structure", Fig. 3b)
Common DPD parameters: gamma=4.5 (sigma=3), kT=1, dt=0.04, lambda=0.65.
"""
from __future__ import annotations

import dataclasses
from typing import Dict, List, Optional

import numpy as np

KIND_HARMONIC = 1
KIND_MORSE_PAPER = 2
KIND_MORSE = 3


@dataclasses.dataclass
class Workload:
    name: str
    L: np.ndarray            # (3,) box edges
    types: np.ndarray        # (N,) int32
    a: np.ndarray            # (ntypes, ntypes) float64
    gamma: float
    kT: float
    dt: float
    lam: float
    seed: int                # Philox key of the pair noise
    pos: np.ndarray          # (N, 3) float64 in [0, L)
    vel: np.ndarray          # (N, 3) float64, zero net momentum
    bonds: Dict[str, np.ndarray]
    steps: int = 0

    @property
    def n(self) -> int:
        return int(self.types.size)

    @property
    def nbonds(self) -> int:
        return int(self.bonds["i"].size)


def empty_bonds() -> Dict[str, np.ndarray]:
    return dict(i=np.zeros(0, np.int32), j=np.zeros(0, np.int32), kind=np.zeros(0, np.int32),
                r0=np.zeros(0), k=np.zeros(0), alpha=np.zeros(0))


def concat_bonds(parts: List[Dict[str, np.ndarray]]) -> Dict[str, np.ndarray]:
    if not parts:
        return empty_bonds()
    out = {}
    for key, dt in (("i", np.int32), ("j", np.int32), ("kind", np.int32), ("r0", np.float64),
                    ("k", np.float64), ("alpha", np.float64)):
        out[key] = np.ascontiguousarray(np.concatenate([p[key] for p in parts]), dtype=dt)
    return out


def bond_records(i, j, kind, r0, k, alpha=0.0) -> Dict[str, np.ndarray]:
    i = np.asarray(i, np.int32)
    m = i.size
    return dict(i=i, j=np.asarray(j, np.int32), kind=np.full(m, kind, np.int32),
                r0=np.full(m, float(r0)), k=np.full(m, float(k)), alpha=np.full(m, float(alpha)))


def maxwell_velocities(rng, n, kT=1.0) -> np.ndarray:
    v = rng.normal(0.0, np.sqrt(kT), size=(n, 3))
    v -= v.mean(axis=0, keepdims=True)
    return v


def random_walk_chains(rng, nchains, length, step, L) -> np.ndarray:
    """Chains as random walks with fixed step length and isotropic directions,
    from uniform starts, wrapped into the box.  Returns (nchains*length, 3)."""
    L = np.asarray(L, dtype=np.float64)
    start = rng.uniform(0.0, 1.0, size=(nchains, 1, 3)) * L
    d = rng.normal(size=(nchains, length - 1, 3))
    d *= step / np.linalg.norm(d, axis=2, keepdims=True)
    walk = np.concatenate([np.zeros((nchains, 1, 3)), np.cumsum(d, axis=1)], axis=1) + start
    walk = walk.reshape(-1, 3)
    return np.mod(walk, L)


def _box(L):
    return np.broadcast_to(np.asarray(L, dtype=np.float64), (3,)).copy()


def fluid(L, rho=3.0, a_same=25.0, a_cross=None, ntypes=1, seed=1001, gamma=4.5, kT=1.0,
          dt=0.04, lam=0.65, n=None, name="fluid") -> Workload:
    """Uniform random fluid; types assigned uniformly at random if ntypes > 1."""
    L = _box(L)
    rng = np.random.default_rng(seed)
    if n is None:
        n = int(round(rho * float(np.prod(L))))
    pos = rng.uniform(0.0, 1.0, size=(n, 3)) * L
    pos = np.where(pos >= L, 0.0, pos)
    types = (rng.integers(0, ntypes, size=n) if ntypes > 1 else np.zeros(n)).astype(np.int32)
    a = np.full((ntypes, ntypes), float(a_same))
    if ntypes > 1 and a_cross is not None:
        a = np.full((ntypes, ntypes), float(a_cross))
        np.fill_diagonal(a, float(a_same))
    vel = maxwell_velocities(rng, n, kT)
    return Workload(name, L, types, a, gamma, kT, dt, lam, seed, pos, vel, empty_bonds())


def fluid_3k(seed=1001) -> Workload:
    w = fluid(10.0, n=3000, seed=seed, name="fluid_3k")
    w.steps = 1000
    return w


def fluid_3m(seed=1004) -> Workload:
    w = fluid(100.0, n=3_000_000, ntypes=2, a_same=25.0, a_cross=30.0, seed=seed,
              name="fluid_3m")
    w.steps = 500
    return w


def fluid_1m(seed=1004) -> Workload:
    """The fluid_3m recipe in a 70^3 box (N = 1,029,000): state larger than
    L2 at a third of the size, for kernel profiles."""
    w = fluid(70.0, ntypes=2, a_same=25.0, a_cross=30.0, seed=seed, name="fluid_1m")
    w.steps = 500
    return w


def camus_table(n: int, protein=False, seed=1007) -> Workload:
    """The shapes of the paper's timing tables: a cubic box at rho = 3 holding
    n beads with a_ij = 25 everywhere (Table 1); with protein=True the first
    60 beads are the alpha-helix chain with its 1-2, 1-3 and 1-5 bonds and
    the helix model's a_ij (Table 3)."""
    edge = (n / 3.0) ** (1.0 / 3.0)
    L = _box(edge)
    rng = np.random.default_rng(seed + n)
    pos = rng.uniform(0.0, 1.0, size=(n, 3)) * L
    types = np.zeros(n, np.int32)
    a = np.array([[25.0]])
    bonds = empty_bonds()
    gamma, dt = 4.5, 0.04
    if protein:
        beads = 60
        pos[:beads] = random_walk_chains(rng, 1, beads, 0.6, L)
        types = np.concatenate([np.zeros(beads, np.int32), np.ones(n - beads, np.int32)])
        a = np.array([[50.0, 55.0], [55.0, 50.0]])
        bonds = _helix_bonds(beads)
        gamma, dt = 4.2, 0.02
    pos = np.where(pos >= L, 0.0, pos)
    vel = maxwell_velocities(rng, n)
    return Workload("camus_%s_%d" % ("protein" if protein else "fluid", n), L, types, a, gamma,
                    1.0, dt, 0.65, seed + n, pos, vel, bonds)


def melt_98k(seed=1002, L=32.0, chain_len=10) -> Workload:
    L = _box(L)
    rng = np.random.default_rng(seed)
    n = int(round(3.0 * float(np.prod(L))))
    nch = n // chain_len
    nfree = n - nch * chain_len
    chains = random_walk_chains(rng, nch, chain_len, 0.5, L)
    free = rng.uniform(0.0, 1.0, size=(nfree, 3)) * L
    pos = np.concatenate([chains, free], axis=0)
    half = chain_len // 2
    per_chain = np.array([0] * half + [1] * (chain_len - half), np.int32)
    types = np.concatenate([np.tile(per_chain, nch), np.zeros(nfree, np.int32)])
    a = np.array([[25.0, 40.0], [40.0, 25.0]])
    base = (np.arange(nch) * chain_len)[:, None]
    i = (base + np.arange(chain_len - 1)[None, :]).ravel()
    bonds = bond_records(i, i + 1, KIND_HARMONIC, 0.0, 4.0)
    vel = maxwell_velocities(rng, n)
    return Workload("melt_98k", L, types, a, 4.5, 1.0, 0.04, 0.65, seed, pos, vel, bonds)


def peptide_192k(seed=1003, L=40.0, nchains=200, chain_len=20) -> Workload:
    L = _box(L)
    rng = np.random.default_rng(seed)
    n = int(round(3.0 * float(np.prod(L))))
    chains = random_walk_chains(rng, nchains, chain_len, 0.5, L)
    nsol = n - nchains * chain_len
    sol = rng.uniform(0.0, 1.0, size=(nsol, 3)) * L
    pos = np.concatenate([chains, sol], axis=0)
    types = np.concatenate([np.zeros(nchains * chain_len, np.int32), np.ones(nsol, np.int32)])
    a = np.array([[25.0, 30.0], [30.0, 25.0]])
    base = (np.arange(nchains) * chain_len)[:, None]
    i12 = (base + np.arange(chain_len - 1)[None, :]).ravel()
    i13 = (base + np.arange(chain_len - 2)[None, :]).ravel()
    i15 = (base + np.arange(chain_len - 4)[None, :]).ravel()
    bonds = concat_bonds([
        bond_records(i12, i12 + 1, KIND_HARMONIC, 0.5, 4.0),
        bond_records(i13, i13 + 2, KIND_MORSE, 0.7, 5.0, 3.0),
        bond_records(i15, i15 + 4, KIND_MORSE, 1.0, 5.0, 3.0),
    ])
    vel = maxwell_velocities(rng, n)
    return Workload("peptide_192k", L, types, a, 4.5, 1.0, 0.04, 0.65, seed, pos, vel, bonds)


def _helix_bonds(beads: int) -> Dict[str, np.ndarray]:
    """Fig. 3b's bond list for a skeletal chain of `beads` beads."""
    i12 = np.arange(beads - 1)
    i13 = np.arange(beads - 2)
    i15 = np.arange(beads - 4)
    return concat_bonds([
        bond_records(i12, i12 + 1, KIND_HARMONIC, 0.6, 160.0),
        bond_records(i13, i13 + 2, KIND_HARMONIC, 1.2, 80.0),
        bond_records(i13, i13 + 2, KIND_MORSE_PAPER, 0.9, 12.0, 8.0),
        bond_records(i15, i15 + 4, KIND_MORSE_PAPER, 0.6, 12.0, 8.0),
    ])


def alpha_helix_24k(seed=1006) -> Workload:
    """The paper's alpha-helix model: 24000 beads in a 20^3 box, one chain of 60
    skeletal beads (type 0) in water (type 1); a_SS=a_WW=50, a_SW=55;
    1-2 harmonic C=160, r_e=0.6; 1-3 harmonic C=80, r_e=1.2 plus modified
    Morse K=12, alpha=8, r_e=0.9; 1-5 modified Morse K=12, alpha=8, r_e=0.6;
    gamma=4.2, kT=1, lambda=0.65, dt=0.02, 10000 steps."""
    L = _box(20.0)
    rng = np.random.default_rng(seed)
    n, beads = 24000, 60
    chain = random_walk_chains(rng, 1, beads, 0.6, L)
    water = rng.uniform(0.0, 1.0, size=(n - beads, 3)) * L
    pos = np.concatenate([chain, water], axis=0)
    types = np.concatenate([np.zeros(beads, np.int32), np.ones(n - beads, np.int32)])
    a = np.array([[50.0, 55.0], [55.0, 50.0]])
    bonds = _helix_bonds(beads)
    vel = maxwell_velocities(rng, n)
    w = Workload("alpha_helix_24k", L, types, a, 4.2, 1.0, 0.02, 0.65, seed, pos, vel, bonds)
    w.steps = 10000
    return w


@dataclasses.dataclass
class Request:
    """One system of the serving stream."""
    rid: int
    arrival_s: float
    steps: int
    workload: Workload


def serving_system(s: int, edge: Optional[float] = None, a_ab: Optional[float] = None,
                   chain_frac=0.1, chain_len=10) -> Workload:
    rng = np.random.default_rng(5000 + s)
    if edge is None:
        edge = float(rng.uniform(8.0, 24.0))
    if a_ab is None:
        a_ab = float(rng.uniform(25.0, 50.0))
    L = _box(edge)
    n = int(round(3.0 * edge ** 3))
    nch = int(chain_frac * n) // chain_len
    chains = random_walk_chains(rng, nch, chain_len, 0.5, L) if nch else np.zeros((0, 3))
    nfree = n - nch * chain_len
    free = rng.uniform(0.0, 1.0, size=(nfree, 3)) * L
    pos = np.concatenate([chains, free], axis=0)
    pos = np.where(pos >= L, 0.0, pos)
    types = rng.integers(0, 2, size=n).astype(np.int32)
    a = np.array([[25.0, a_ab], [a_ab, 25.0]])
    if nch:
        base = (np.arange(nch) * chain_len)[:, None]
        i = (base + np.arange(chain_len - 1)[None, :]).ravel()
        bonds = bond_records(i, i + 1, KIND_HARMONIC, 0.0, 4.0)
    else:
        bonds = empty_bonds()
    vel = maxwell_velocities(rng, n)
    return Workload("serving_%d" % s, L, types, a, 4.5, 1.0, 0.04, 0.65, 5000 + s, pos, vel,
                    bonds)


def serving_stream(nsys=256, rate_hz=20.0, steps=2000, seed=1005) -> List[Request]:
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_hz, size=nsys)
    t = np.cumsum(gaps) - gaps[0]
    return [Request(s, float(t[s]), steps, serving_system(s)) for s in range(nsys)]


WORKLOADS = {
    "fluid_3k": fluid_3k,
    "melt_98k": melt_98k,
    "peptide_192k": peptide_192k,
    "fluid_3m": fluid_3m,
    "fluid_1m": fluid_1m,
    "alpha_helix_24k": alpha_helix_24k,
}


def make(name: str, **kw) -> Workload:
    return WORKLOADS[name](**kw)
