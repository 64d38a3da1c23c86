"""ctypes binding of libdpd (include/dpd.h): argument marshalling only.

Every step of the DPD loop runs in the CUDA kernels of ``libdpd.so``; this
module converts numpy arrays to the C ABI's plain pointers and raises on
error codes.  Importing it loads the library and fails loudly if it has not
been built (``python -m paper_1804_06205_gb300.build``); there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libdpd.so")

DPD_OK = 0
DPD_EINVAL = -1
DPD_ENOMEM = -2
DPD_ECUDA = -3
DPD_EUNSTABLE = -4
DPD_ETIMEOUT = -5
DPD_ENOSTATE = -6

DPD_FP32 = 0
DPD_FP64 = 1
DPD_NOISE_GAUSS = 0
DPD_NOISE_UNIFORM = 1

EXPORTED = ("dpd_default_options", "dpd_create", "dpd_set_state", "dpd_step", "dpd_get_state",
            "dpd_observables", "dpd_gr", "dpd_get_cells", "dpd_cell_dims", "dpd_sync",
            "dpd_launch_count", "dpd_profile_begin", "dpd_profile_end", "dpd_destroy",
            "dpd_strerror", "dpd_last_error", "dpd_cells_noalloc", "dpd_batch_create",
            "dpd_batch_add", "dpd_batch_remove", "dpd_batch_step", "dpd_batch_get_state",
            "dpd_batch_observables", "dpd_batch_usage", "dpd_batch_sync", "dpd_batch_launch_count",
            "dpd_batch_last_error", "dpd_batch_destroy", "dpd_batch_profile_begin",
            "dpd_batch_profile_end", "dpd_wait_check", "dpd_bm_check", "dpd_checkpoint_bytes",
            "dpd_get_checkpoint", "dpd_set_checkpoint", "dpd_batch_checkpoint_bytes",
            "dpd_batch_get_checkpoint", "dpd_batch_set_checkpoint", "dpd_grid_wait_check")


class dpd_box(C.Structure):
    _fields_ = [("L", C.c_double * 3)]


class dpd_bond(C.Structure):
    _fields_ = [("i", C.c_int32), ("j", C.c_int32), ("kind", C.c_int32), ("pad", C.c_int32),
                ("r0", C.c_double), ("k", C.c_double), ("alpha", C.c_double)]


class dpd_options(C.Structure):
    _fields_ = [("lambda_", C.c_double), ("seed", C.c_uint64), ("precision", C.c_int32),
                ("noise", C.c_int32), ("sample_every", C.c_int32), ("tile_cells", C.c_int32),
                ("threads", C.c_int32), ("use_graph", C.c_int32), ("persistent", C.c_int32),
                ("pad", C.c_int32), ("cuda_stream", C.c_void_p)]


class dpd_batch_capacity(C.Structure):
    _fields_ = [("max_beads", C.c_int64), ("max_cells", C.c_int64), ("max_bonds", C.c_int64),
                ("max_systems", C.c_int32), ("pad", C.c_int32)]


class dpd_obs(C.Structure):
    _fields_ = [("step", C.c_int64), ("momentum", C.c_double * 3), ("kT", C.c_double),
                ("p_total", C.c_double), ("p_ideal", C.c_double), ("p_cons", C.c_double),
                ("p_bond", C.c_double), ("e_pair", C.c_double), ("e_bond", C.c_double),
                ("sum_v2", C.c_double), ("kT_mean", C.c_double), ("p_mean", C.c_double),
                ("n_samples", C.c_int64), ("status", C.c_int32), ("pad", C.c_int32)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k not in ("momentum", "pad")}
        d["momentum"] = list(self.momentum)
        return d


class DPDError(RuntimeError):
    def __init__(self, code, where, detail=""):
        self.code = code
        super().__init__("%s failed: %d (%s) %s" % (where, code, strerror(code), detail))


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libdpd.so is not built at %s; run "
                          "`python -m paper_1804_06205_gb300.build` (needs nvcc)" % LIB_PATH)
    lib = C.CDLL(LIB_PATH)
    P = C.c_void_p
    lib.dpd_default_options.argtypes = [P]
    lib.dpd_default_options.restype = None
    lib.dpd_create.argtypes = [P, C.c_int64, P, C.c_int32, P, C.c_double, C.c_double, C.c_double,
                               P, C.c_int64, P, C.c_int64, P, P]
    lib.dpd_set_state.argtypes = [P, P, P, C.c_int64]
    lib.dpd_step.argtypes = [P, C.c_int64]
    lib.dpd_get_state.argtypes = [P, P, P, P, P]
    lib.dpd_observables.argtypes = [P, P]
    lib.dpd_gr.argtypes = [P, C.c_double, C.c_int32, P]
    lib.dpd_get_cells.argtypes = [P, P, P, P]
    lib.dpd_cell_dims.argtypes = [P, P]
    lib.dpd_sync.argtypes = [P]
    lib.dpd_launch_count.argtypes = [P]
    lib.dpd_launch_count.restype = C.c_int64
    lib.dpd_profile_begin.argtypes = [P, C.c_int64]
    lib.dpd_profile_end.argtypes = [P, P, P]
    lib.dpd_destroy.argtypes = [P]
    lib.dpd_strerror.argtypes = [C.c_int]
    lib.dpd_strerror.restype = C.c_char_p
    lib.dpd_last_error.argtypes = [P]
    lib.dpd_last_error.restype = C.c_char_p
    lib.dpd_cells_noalloc.argtypes = [P, C.c_int64, P, P, P, P, P]
    lib.dpd_wait_check.argtypes = [C.c_int32, C.c_int32, P]
    lib.dpd_wait_check.restype = C.c_int
    lib.dpd_grid_wait_check.argtypes = [C.c_int32, C.c_int64, P]
    lib.dpd_grid_wait_check.restype = C.c_int
    lib.dpd_bm_check.argtypes = [P, P]
    lib.dpd_bm_check.restype = C.c_int
    lib.dpd_checkpoint_bytes.argtypes = [P, P]
    lib.dpd_get_checkpoint.argtypes = [P, P, C.c_int64]
    lib.dpd_set_checkpoint.argtypes = [P, P, C.c_int64]
    lib.dpd_batch_checkpoint_bytes.argtypes = [P, C.c_int32, P]
    lib.dpd_batch_get_checkpoint.argtypes = [P, C.c_int32, P, C.c_int64]
    lib.dpd_batch_set_checkpoint.argtypes = [P, C.c_int32, P, C.c_int64]
    lib.dpd_batch_create.argtypes = [P, P, P]
    lib.dpd_batch_add.argtypes = [P, P, C.c_int64, P, C.c_int32, P, C.c_double, C.c_double,
                                  C.c_double, P, C.c_int64, P, C.c_int64, C.c_double, C.c_uint64,
                                  C.c_int32, P, P, C.c_int64, P]
    lib.dpd_batch_profile_begin.argtypes = [P, C.c_int64]
    lib.dpd_batch_profile_end.argtypes = [P, P, P]
    lib.dpd_batch_remove.argtypes = [P, C.c_int32]
    lib.dpd_batch_step.argtypes = [P, C.c_int64]
    lib.dpd_batch_get_state.argtypes = [P, C.c_int32, P, P, P, P]
    lib.dpd_batch_observables.argtypes = [P, C.c_int32, P]
    lib.dpd_batch_usage.argtypes = [P, P, P, P]
    lib.dpd_batch_sync.argtypes = [P]
    lib.dpd_batch_launch_count.argtypes = [P]
    lib.dpd_batch_launch_count.restype = C.c_int64
    lib.dpd_batch_last_error.argtypes = [P]
    lib.dpd_batch_last_error.restype = C.c_char_p
    lib.dpd_batch_destroy.argtypes = [P]
    return lib


lib = _load()


def strerror(code):
    return lib.dpd_strerror(int(code)).decode()


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


NOALLOC_MAX_N = 4194304
NOALLOC_MAX_CELLS = 4194304


def cells_noalloc(pos_dev_ptr, n, L, key_dev_ptr, order_dev_ptr, cell_start_dev_ptr,
                  stream_ptr=None):
    """dpd_cells_noalloc on caller-owned device buffers (raw pointers); returns
    the DPD_* code.  Enqueued on the stream; the caller synchronises."""
    L = np.broadcast_to(np.asarray(L, dtype=np.float64), (3,))
    box = dpd_box((C.c_double * 3)(*L))
    return lib.dpd_cells_noalloc(C.c_void_p(pos_dev_ptr), int(n), C.byref(box),
                                 C.c_void_p(key_dev_ptr), C.c_void_p(order_dev_ptr),
                                 C.c_void_p(cell_start_dev_ptr), C.c_void_p(stream_ptr))


WAIT_CHECK_MAX_TRIES = 1 << 22


def wait_check(deliver, tries=4096, stream_ptr=None):
    """dpd_wait_check: one bounded mbarrier wait whose bytes are delivered
    (deliver=True, DPD_OK) or never delivered (deliver=False: the wait gives up
    after `tries` polls, DPD_ETIMEOUT).  Returns the DPD_* code."""
    return lib.dpd_wait_check(1 if deliver else 0, int(tries), C.c_void_p(stream_ptr))


GRID_WAIT_CHECK_MAX_CYCLES = 4000000000


def grid_wait_check(complete, budget_cycles=20_000_000, stream_ptr=None):
    """dpd_grid_wait_check: one grid-wide barrier of a 4-block cooperative
    grid that completes (complete=True, DPD_OK) or waits for a block that does
    not exist (complete=False: every block gives up after budget_cycles,
    DPD_ETIMEOUT).  Returns the DPD_* code."""
    return lib.dpd_grid_wait_check(1 if complete else 0, int(budget_cycles),
                                   C.c_void_p(stream_ptr))


def bm_check():
    """dpd_bm_check: largest absolute differences (ln, cos) between the FP64
    Box-Muller functions and the library's log and cospi over all 2^23
    uniforms."""
    le, ce = C.c_double(0.0), C.c_double(0.0)
    rc = lib.dpd_bm_check(C.byref(le), C.byref(ce))
    if rc != DPD_OK:
        raise DPDError(rc, "dpd_bm_check")
    return le.value, ce.value


def default_options(**kw) -> dpd_options:
    o = dpd_options()
    lib.dpd_default_options(C.byref(o))
    for k, v in kw.items():
        setattr(o, "lambda_" if k in ("lam", "lambda") else k, v)
    return o


def _records_fast(b):
    m = len(b["i"])
    dt = np.dtype([("i", "<i4"), ("j", "<i4"), ("kind", "<i4"), ("pad", "<i4"), ("r0", "<f8"),
                   ("k", "<f8"), ("alpha", "<f8")])
    rec = np.zeros(max(m, 1), dtype=dt)
    if m:
        rec["i"], rec["j"], rec["kind"] = b["i"], b["j"], b["kind"]
        rec["r0"], rec["k"], rec["alpha"] = b["r0"], b["k"], b["alpha"]
    return rec, m


class System:
    """One DPD system owned by libdpd (a thin wrapper over the C handle)."""

    def __init__(self, L, types, a, gamma, kT, dt, bonds=None, morse=None, options=None, **opt):
        self.h = C.c_void_p()
        L = np.broadcast_to(np.asarray(L, dtype=np.float64), (3,))
        box = dpd_box((C.c_double * 3)(*L))
        self.types = np.ascontiguousarray(types, dtype=np.int32)
        self.n = int(self.types.size)
        self.a = np.ascontiguousarray(a, dtype=np.float64)
        ntypes = int(round(np.sqrt(self.a.size)))
        if options is None:
            options = default_options(**opt)
        self.options = options
        empty = dict(i=[], j=[], kind=[], r0=[], k=[], alpha=[])
        brec, nb = _records_fast(bonds if bonds is not None else empty)
        mrec, nm = _records_fast(morse if morse is not None else empty)
        self._keep = (brec, mrec)
        rc = lib.dpd_create(C.byref(box), self.n, _ptr(self.types), ntypes, _ptr(self.a),
                            float(gamma), float(kT), float(dt), _ptr(brec), nb, _ptr(mrec), nm,
                            C.byref(options), C.byref(self.h))
        if rc != DPD_OK:
            raise DPDError(rc, "dpd_create", lib.dpd_last_error(None).decode())
        nc = np.zeros(3, np.int64)
        lib.dpd_cell_dims(self.h, _ptr(nc))
        self.nc = nc
        self.L = np.array(L)

    @classmethod
    def from_workload(cls, w, **opt):
        opt.setdefault("seed", w.seed)
        opt.setdefault("lam", w.lam)
        return cls(w.L, w.types, w.a, w.gamma, w.kT, w.dt, bonds=w.bonds, **opt)

    def _check(self, rc, where):
        if rc != DPD_OK:
            raise DPDError(rc, where, lib.dpd_last_error(self.h).decode())

    def set_state(self, pos, vel, step=0):
        pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(self.n, 3)
        vel = np.ascontiguousarray(vel, dtype=np.float64).reshape(self.n, 3)
        self._check(lib.dpd_set_state(self.h, _ptr(pos), _ptr(vel), int(step)), "dpd_set_state")

    def set_state_ptr(self, pos_ptr, vel_ptr, step=0):
        """Host pointers (e.g. of pinned buffers) of n*3 doubles each."""
        self._check(lib.dpd_set_state(self.h, C.c_void_p(pos_ptr), C.c_void_p(vel_ptr), int(step)),
                    "dpd_set_state")

    def step(self, nsteps=1):
        self._check(lib.dpd_step(self.h, int(nsteps)), "dpd_step")

    def get_state(self, pos=True, vel=True, force=True):
        out = [np.empty((self.n, 3)) if f else None for f in (pos, vel, force)]
        st = C.c_int64(0)
        self._check(lib.dpd_get_state(self.h, _ptr(out[0]), _ptr(out[1]), _ptr(out[2]),
                                      C.byref(st)), "dpd_get_state")
        return out[0], out[1], out[2], st.value

    def get_state_ptr(self, pos_ptr=None, vel_ptr=None, force_ptr=None):
        st = C.c_int64(0)
        self._check(lib.dpd_get_state(self.h, C.c_void_p(pos_ptr), C.c_void_p(vel_ptr),
                                      C.c_void_p(force_ptr), C.byref(st)), "dpd_get_state")
        return st.value

    def observables(self) -> dict:
        o = dpd_obs()
        self._check(lib.dpd_observables(self.h, C.byref(o)), "dpd_observables")
        return o.as_dict()

    def gr_counts(self, rmax, nbins):
        c = np.zeros(nbins, dtype=np.uint64)
        self._check(lib.dpd_gr(self.h, float(rmax), int(nbins), _ptr(c)), "dpd_gr")
        return c

    def cells(self):
        key = np.zeros(self.n, np.uint32)
        order = np.zeros(self.n, np.int64)
        start = np.zeros(int(np.prod(self.nc)) + 1, np.int64)
        self._check(lib.dpd_get_cells(self.h, _ptr(key), _ptr(order), _ptr(start)),
                    "dpd_get_cells")
        return key, order, start

    def get_checkpoint(self) -> bytes:
        """The exact state as an opaque byte string (dpd_get_checkpoint)."""
        nb = C.c_int64(0)
        self._check(lib.dpd_checkpoint_bytes(self.h, C.byref(nb)), "dpd_checkpoint_bytes")
        buf = C.create_string_buffer(nb.value)
        self._check(lib.dpd_get_checkpoint(self.h, buf, nb.value), "dpd_get_checkpoint")
        return buf.raw

    def set_checkpoint(self, data: bytes):
        self._check(lib.dpd_set_checkpoint(self.h, C.c_char_p(data), len(data)),
                    "dpd_set_checkpoint")

    def checkpoint_bytes(self) -> int:
        nb = C.c_int64(0)
        self._check(lib.dpd_checkpoint_bytes(self.h, C.byref(nb)), "dpd_checkpoint_bytes")
        return nb.value

    def get_checkpoint_ptr(self, ptr, nbytes):
        """The checkpoint into host memory at ptr (e.g. a pinned buffer)."""
        self._check(lib.dpd_get_checkpoint(self.h, C.c_void_p(ptr), int(nbytes)),
                    "dpd_get_checkpoint")

    def set_checkpoint_ptr(self, ptr, nbytes):
        self._check(lib.dpd_set_checkpoint(self.h, C.c_void_p(ptr), int(nbytes)),
                    "dpd_set_checkpoint")

    def sync(self):
        self._check(lib.dpd_sync(self.h), "dpd_sync")

    def launch_count(self) -> int:
        return int(lib.dpd_launch_count(self.h))

    def profile_begin(self, max_steps):
        self._check(lib.dpd_profile_begin(self.h, int(max_steps)), "dpd_profile_begin")

    def profile_end(self):
        """-> (ms per phase summed over timed steps [update+sort, pair, bond+v], steps)"""
        ms = np.zeros(3)
        n = C.c_int64(0)
        self._check(lib.dpd_profile_end(self.h, _ptr(ms), C.byref(n)), "dpd_profile_end")
        return ms, n.value

    def close(self):
        if self.h:
            lib.dpd_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Batch:
    """Many independent systems advanced by the same launches (dpd_batch_*)."""

    def __init__(self, max_beads, max_cells, max_bonds=0, max_systems=64, options=None, **opt):
        self.h = C.c_void_p()
        cap = dpd_batch_capacity(int(max_beads), int(max_cells), int(max_bonds),
                                 int(max_systems), 0)
        if options is None:
            options = default_options(**opt)
        self.options = options
        rc = lib.dpd_batch_create(C.byref(cap), C.byref(options), C.byref(self.h))
        if rc != DPD_OK:
            raise DPDError(rc, "dpd_batch_create", lib.dpd_batch_last_error(None).decode())
        self.n = {}

    def _check(self, rc, where):
        if rc != DPD_OK:
            raise DPDError(rc, where, lib.dpd_batch_last_error(self.h).decode())

    def try_add(self, L, types, a, gamma, kT, dt, pos, vel, bonds=None, morse=None, lam=0.65,
                seed=0, step=0, tile_cells=0):
        """Add a system with its state; returns its index, or None when it does
        not fit in the pools (DPD_ENOMEM: not admitted)."""
        L = np.broadcast_to(np.asarray(L, dtype=np.float64), (3,))
        box = dpd_box((C.c_double * 3)(*L))
        types = np.ascontiguousarray(types, dtype=np.int32)
        a = np.ascontiguousarray(a, dtype=np.float64)
        ntypes = int(round(np.sqrt(a.size)))
        empty = dict(i=[], j=[], kind=[], r0=[], k=[], alpha=[])
        brec, nb = _records_fast(bonds if bonds is not None else empty)
        mrec, nm = _records_fast(morse if morse is not None else empty)
        pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(types.size, 3)
        vel = np.ascontiguousarray(vel, dtype=np.float64).reshape(types.size, 3)
        sys_ = C.c_int32(-1)
        rc = lib.dpd_batch_add(self.h, C.byref(box), int(types.size), _ptr(types), ntypes,
                               _ptr(a), float(gamma), float(kT), float(dt), _ptr(brec), nb,
                               _ptr(mrec), nm, float(lam), int(seed) & 0xFFFFFFFFFFFFFFFF,
                               int(tile_cells), _ptr(pos), _ptr(vel), int(step), C.byref(sys_))
        if rc == DPD_ENOMEM:
            return None
        self._check(rc, "dpd_batch_add")
        self.n[sys_.value] = int(types.size)
        return sys_.value

    def add_workload(self, w, step=0, tile_cells=0):
        return self.try_add(w.L, w.types, w.a, w.gamma, w.kT, w.dt, w.pos, w.vel,
                            bonds=w.bonds, lam=w.lam, seed=w.seed, step=step,
                            tile_cells=tile_cells)

    def profile_begin(self, max_steps):
        self._check(lib.dpd_batch_profile_begin(self.h, int(max_steps)),
                    "dpd_batch_profile_begin")

    def profile_end(self):
        ms = np.zeros(3)
        n = C.c_int64(0)
        self._check(lib.dpd_batch_profile_end(self.h, _ptr(ms), C.byref(n)),
                    "dpd_batch_profile_end")
        return ms, n.value

    def remove(self, s):
        self._check(lib.dpd_batch_remove(self.h, int(s)), "dpd_batch_remove")
        self.n.pop(s, None)

    def step(self, nsteps=1):
        self._check(lib.dpd_batch_step(self.h, int(nsteps)), "dpd_batch_step")

    def get_state(self, s, pos=True, vel=True, force=True):
        n = self.n[s]
        out = [np.empty((n, 3)) if f else None for f in (pos, vel, force)]
        st = C.c_int64(0)
        self._check(lib.dpd_batch_get_state(self.h, int(s), _ptr(out[0]), _ptr(out[1]),
                                            _ptr(out[2]), C.byref(st)), "dpd_batch_get_state")
        return out[0], out[1], out[2], st.value

    def observables(self, s) -> dict:
        o = dpd_obs()
        self._check(lib.dpd_batch_observables(self.h, int(s), C.byref(o)),
                    "dpd_batch_observables")
        return o.as_dict()

    def get_checkpoint(self, s) -> bytes:
        nb = C.c_int64(0)
        self._check(lib.dpd_batch_checkpoint_bytes(self.h, int(s), C.byref(nb)),
                    "dpd_batch_checkpoint_bytes")
        buf = C.create_string_buffer(nb.value)
        self._check(lib.dpd_batch_get_checkpoint(self.h, int(s), buf, nb.value),
                    "dpd_batch_get_checkpoint")
        return buf.raw

    def set_checkpoint(self, s, data: bytes):
        self._check(lib.dpd_batch_set_checkpoint(self.h, int(s), C.c_char_p(data), len(data)),
                    "dpd_batch_set_checkpoint")

    def usage(self):
        used = np.zeros(4, np.int64)
        cap = np.zeros(4, np.int64)
        ns = C.c_int32(0)
        self._check(lib.dpd_batch_usage(self.h, _ptr(used), _ptr(cap), C.byref(ns)),
                    "dpd_batch_usage")
        return used, cap, ns.value

    def sync(self):
        self._check(lib.dpd_batch_sync(self.h), "dpd_batch_sync")

    def launch_count(self) -> int:
        return int(lib.dpd_batch_launch_count(self.h))

    def close(self):
        if self.h:
            lib.dpd_batch_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
