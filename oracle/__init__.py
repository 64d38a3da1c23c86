"""FP64 CPU oracle for the DPD step loop of arxiv 1804.06205 (CAMUS).

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may use this module; the CUDA engine never does.
It shares no code with the CUDA path: the arithmetic lives in
``dpd_oracle.c`` (plain C, FP64, built with ``-ffp-contract=off``) and this
file only marshals numpy arrays.

What each function computes, with the passage it follows:
  * ``pair_forces``  eq. 3-4 plus the Groot-Warren dissipative/random forms
    (w^D = (w^R)^2, sigma^2 = 2 gamma kT), brute force over all j != i;
    ``pair_forces_ids`` the same terms for beads given with their global ids
    (a spatial domain and its ghosts, ``oracle.slab``);
  * ``bond_forces``  eqs. 6-8, Fig. 3a;
  * ``run``          Fig. 1 (modified velocity-Verlet, lambda);
  * ``cell_keys`` / ``cell_sort``  the cell division of section "Design
    concept of CAMUS" (cell edge = cutoff), canonical (cell, id) order;
  * ``theta``        pair noise (Philox4x32-10 + Box-Muller, a reading: the
    paper only says "Gaussian statistics").
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dpd_oracle.c")
_HDR = os.path.join(_HERE, "dpd_oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

MODE_BRUTE = 0
MODE_CELLS = 1
NOISE_GAUSS = 0
NOISE_UNIFORM = 1

OBS_FIELDS = ("step", "px", "py", "pz", "kT", "p_total", "p_ideal", "p_cons", "p_bond",
              "e_pair", "e_bond", "sum_v2")


def build(force: bool = False) -> str:
    """Compile dpd_oracle.c with gcc into liboracle.so (in place)."""
    stale = (not os.path.exists(_LIB)
             or os.path.getmtime(_LIB) < max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)))
    if force or stale:
        tmp = _LIB + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", "-std=c11", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Sys(C.Structure):
    _fields_ = [
        ("L", C.c_double * 3), ("n", C.c_int64), ("ntypes", C.c_int32),
        ("types", C.c_void_p), ("a", C.c_void_p),
        ("gamma", C.c_double), ("kT", C.c_double), ("dt", C.c_double), ("lam", C.c_double),
        ("seed", C.c_uint64), ("noise", C.c_int32), ("nbonds", C.c_int64),
        ("bi", C.c_void_p), ("bj", C.c_void_p), ("bkind", C.c_void_p),
        ("br0", C.c_void_p), ("bk", C.c_void_p), ("balpha", C.c_void_p),
    ]


class Terms(C.Structure):
    _fields_ = [("wc", C.c_double), ("wb", C.c_double), ("ep", C.c_double), ("eb", C.c_double)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = C.CDLL(_LIB)
            P = C.c_void_p
            lib.orc_philox4x32_10.argtypes = [P, P, P]
            lib.orc_u01.argtypes = [C.c_uint32]
            lib.orc_u01.restype = C.c_double
            lib.orc_theta.argtypes = [C.c_uint64, C.c_int64, C.c_int64, C.c_int64, C.c_int32]
            lib.orc_theta.restype = C.c_double
            lib.orc_pair_force_one.argtypes = [P, P, P, C.c_int64, C.c_int64, C.c_int64, P]
            lib.orc_pair_forces.argtypes = [P, P, P, C.c_int64, C.c_int32, P, P]
            lib.orc_pair_forces_subset.argtypes = [P, P, P, C.c_int64, P, C.c_int64, P]
            lib.orc_pair_forces_ids.argtypes = [P, C.c_int64, P, P, P, P, C.c_int64, C.c_int64,
                                                P]
            lib.orc_bond_forces.argtypes = [P, P, P, P]
            lib.orc_bond_one.argtypes = [C.c_int32, C.c_double, C.c_double, C.c_double, P, P, P]
            lib.orc_forces.argtypes = [P, P, P, C.c_int64, C.c_int32, P, P]
            lib.orc_wrap.argtypes = [P, P]
            lib.orc_cell_dims.argtypes = [P, P, P]
            lib.orc_cell_keys.argtypes = [P, P, P]
            lib.orc_cell_sort.argtypes = [P, P, P, P]
            lib.orc_run.argtypes = [P, P, P, P, P, C.c_int64, C.c_int32, C.c_int32, P, P]
            lib.orc_observables.argtypes = [P, P, P, C.c_int64, P]
            lib.orc_gr_counts.argtypes = [P, P, C.c_double, C.c_int32, P]
            lib.orc_num_threads.restype = C.c_int
            _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


class System:
    """Parameters of one DPD system (all arrays copied to contiguous numpy)."""

    def __init__(self, L, types, a, gamma, kT, dt, lam=0.65, seed=0, noise=NOISE_GAUSS,
                 bonds=None):
        self.L = np.broadcast_to(np.asarray(L, dtype=np.float64), (3,)).copy()
        self.types = np.ascontiguousarray(types, dtype=np.int32)
        self.a = np.ascontiguousarray(a, dtype=np.float64)
        self.ntypes = int(round(np.sqrt(self.a.size)))
        self.n = int(self.types.size)
        if bonds is None:
            bonds = dict(i=[], j=[], kind=[], r0=[], k=[], alpha=[])
        self.bi = np.ascontiguousarray(bonds["i"], dtype=np.int32)
        self.bj = np.ascontiguousarray(bonds["j"], dtype=np.int32)
        self.bkind = np.ascontiguousarray(bonds["kind"], dtype=np.int32)
        self.br0 = np.ascontiguousarray(bonds["r0"], dtype=np.float64)
        self.bk = np.ascontiguousarray(bonds["k"], dtype=np.float64)
        self.balpha = np.ascontiguousarray(bonds["alpha"], dtype=np.float64)
        self.c = _Sys()
        self.c.L = (C.c_double * 3)(*self.L)
        self.c.n = self.n
        self.c.ntypes = self.ntypes
        self.c.types = _ptr(self.types)
        self.c.a = _ptr(self.a)
        self.c.gamma, self.c.kT, self.c.dt, self.c.lam = gamma, kT, dt, lam
        self.c.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
        self.c.noise = noise
        self.c.nbonds = int(self.bi.size)
        self.c.bi, self.c.bj, self.c.bkind = _ptr(self.bi), _ptr(self.bj), _ptr(self.bkind)
        self.c.br0, self.c.bk, self.c.balpha = _ptr(self.br0), _ptr(self.bk), _ptr(self.balpha)

    @property
    def ref(self):
        return C.byref(self.c)


def _f64(x, n=None):
    a = np.ascontiguousarray(x, dtype=np.float64)
    if n is not None:
        a = a.reshape(n, 3)
    return a


def philox4x32_10(ctr, key):
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def u01(x):
    return _load().orc_u01(int(x) & 0xFFFFFFFF)


def theta(seed, i, j, s, noise=NOISE_GAUSS):
    return _load().orc_theta(int(seed) & 0xFFFFFFFFFFFFFFFF, int(i), int(j), int(s), int(noise))


def pair_force_one(sys: System, pos, vt, i, j, s):
    pos = _f64(pos, sys.n)
    vt = _f64(vt, sys.n)
    F = np.zeros(3)
    _load().orc_pair_force_one(sys.ref, _ptr(pos), _ptr(vt), int(i), int(j), int(s), _ptr(F))
    return F


def pair_forces(sys: System, pos, vt, s, mode=MODE_BRUTE):
    pos = _f64(pos, sys.n)
    vt = _f64(vt, sys.n)
    f = np.zeros((sys.n, 3))
    t = Terms()
    rc = _load().orc_pair_forces(sys.ref, _ptr(pos), _ptr(vt), int(s), int(mode), _ptr(f),
                                 C.byref(t))
    if rc:
        raise RuntimeError("orc_pair_forces failed: %d" % rc)
    return f, t


def pair_forces_subset(sys: System, pos, vt, s, idx):
    """Pair forces on the beads idx only (brute force over all j != i)."""
    pos = _f64(pos, sys.n)
    vt = _f64(vt, sys.n)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    f = np.zeros((idx.size, 3))
    rc = _load().orc_pair_forces_subset(sys.ref, _ptr(pos), _ptr(vt), int(s), _ptr(idx),
                                        int(idx.size), _ptr(f))
    if rc:
        raise RuntimeError("orc_pair_forces_subset failed: %d" % rc)
    return f


def pair_forces_ids(sys: System, pos, vt, types, ids, m, s):
    """Pair forces on the first m of the given beads (their own positions,
    predicted velocities, types and global ids) from all of them: a domain's
    beads followed by its ghosts."""
    pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
    vt = np.ascontiguousarray(vt, dtype=np.float64).reshape(-1, 3)
    types = np.ascontiguousarray(types, dtype=np.int32)
    ids = np.ascontiguousarray(ids, dtype=np.int64)
    n = pos.shape[0]
    f = np.zeros((int(m), 3))
    rc = _load().orc_pair_forces_ids(sys.ref, n, _ptr(pos), _ptr(vt), _ptr(types), _ptr(ids),
                                     int(m), int(s), _ptr(f))
    if rc:
        raise RuntimeError("orc_pair_forces_ids failed: %d" % rc)
    return f


def bond_forces(sys: System, pos):
    pos = _f64(pos, sys.n)
    f = np.zeros((sys.n, 3))
    t = Terms()
    rc = _load().orc_bond_forces(sys.ref, _ptr(pos), _ptr(f), C.byref(t))
    if rc:
        raise RuntimeError("orc_bond_forces failed: %d" % rc)
    return f, t


def bond_one(kind, r0, k, alpha, d):
    d = np.ascontiguousarray(d, dtype=np.float64)
    Fi = np.zeros(3)
    U = C.c_double(0.0)
    _load().orc_bond_one(int(kind), float(r0), float(k), float(alpha), _ptr(d), _ptr(Fi),
                         C.byref(U))
    return Fi, U.value


def forces(sys: System, pos, vt, s, mode=MODE_BRUTE):
    pos = _f64(pos, sys.n)
    vt = _f64(vt, sys.n)
    f = np.zeros((sys.n, 3))
    t = Terms()
    rc = _load().orc_forces(sys.ref, _ptr(pos), _ptr(vt), int(s), int(mode), _ptr(f), C.byref(t))
    if rc:
        raise RuntimeError("orc_forces failed: %d" % rc)
    return f, t


def wrap(sys: System, pos):
    p = _f64(pos, sys.n).copy()
    _load().orc_wrap(sys.ref, _ptr(p))
    return p


def cell_dims(sys: System):
    nc = np.zeros(3, dtype=np.int64)
    inv_h = np.zeros(3)
    _load().orc_cell_dims(sys.ref, _ptr(nc), _ptr(inv_h))
    return nc, inv_h


def cell_keys(sys: System, pos):
    pos = _f64(pos, sys.n)
    key = np.zeros(sys.n, dtype=np.uint32)
    _load().orc_cell_keys(sys.ref, _ptr(pos), _ptr(key))
    return key


def cell_sort(sys: System, key):
    key = np.ascontiguousarray(key, dtype=np.uint32)
    nc, _ = cell_dims(sys)
    ncell = int(np.prod(nc))
    order = np.zeros(sys.n, dtype=np.int64)
    start = np.zeros(ncell + 1, dtype=np.int64)
    _load().orc_cell_sort(sys.ref, _ptr(key), _ptr(order), _ptr(start))
    return order, start


class State:
    """Oracle trajectory state: positions, velocities, force and counter."""

    def __init__(self, sys: System, pos, vel, step=0, mode=MODE_BRUTE):
        self.sys = sys
        self.mode = mode
        self.pos = wrap(sys, pos)
        self.vel = _f64(vel, sys.n).copy()
        self.step = int(step)
        # initial force f(0) evaluated with v~ = v at counter `step`
        self.f, self.terms = forces(sys, self.pos, self.vel, self.step, mode)

    def run(self, nsteps, sample_every=0):
        nsamp = (nsteps // sample_every + 1) if sample_every > 0 else 0
        samples = np.zeros((max(nsamp, 1), 12))
        stp = C.c_int64(self.step)
        t = Terms()
        rc = _load().orc_run(self.sys.ref, _ptr(self.pos), _ptr(self.vel), _ptr(self.f),
                             C.byref(stp), int(nsteps), int(self.mode), int(sample_every),
                             _ptr(samples) if sample_every > 0 else None, C.byref(t))
        if rc:
            raise RuntimeError("orc_run failed: %d" % rc)
        if nsteps > 0:
            self.terms = t
        first = self.step
        self.step = stp.value
        if sample_every > 0:
            # samples land at steps that are multiples of sample_every
            cnt = sum(1 for s in range(first + 1, self.step + 1) if s % sample_every == 0)
            return samples[:cnt]
        return None

    def observables(self):
        out = np.zeros(12)
        _load().orc_observables(self.sys.ref, _ptr(self.vel), C.byref(self.terms), self.step,
                                _ptr(out))
        return dict(zip(OBS_FIELDS, out))


def gr_counts(sys: System, pos, rmax, nbins):
    pos = _f64(pos, sys.n)
    counts = np.zeros(nbins, dtype=np.uint64)
    _load().orc_gr_counts(sys.ref, _ptr(pos), float(rmax), int(nbins), _ptr(counts))
    return counts


def gr_normalise(counts, n, L, rmax):
    """g(r) from unique-pair counts: counts / (ideal-gas pairs in each shell)."""
    L = np.broadcast_to(np.asarray(L, dtype=np.float64), (3,))
    V = float(np.prod(L))
    nb = len(counts)
    edges = np.linspace(0.0, rmax, nb + 1)
    shell = 4.0 / 3.0 * np.pi * (edges[1:] ** 3 - edges[:-1] ** 3)
    ideal = 0.5 * n * (n - 1) / V * shell
    return np.asarray(counts, dtype=np.float64) / ideal


def num_threads():
    return _load().orc_num_threads()
