"""dpd_cells_noalloc: the cell division for callers that cannot allocate
device memory (their memory belongs to a framework allocator or a fixed
arena, or they must avoid cudaMalloc's implicit synchronisation).  The
caller owns every buffer; the library only uses its fixed scratch array.

Checked through the C ABI against the existing path (dpd_set_state +
dpd_get_cells) and against the FP64 oracle's cell division, on two calls in a
row with different sizes, so that the shared scratch's leftovers from the
first call cannot leak into the second; a clump of thousands of beads in one
cell checks the canonical order inside crowded cells.
This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_1804_06205_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _face_heavy(L, n, seed):
    rng = np.random.default_rng(seed)
    L = np.broadcast_to(np.asarray(L, float), (3,))
    nc = np.floor(L)
    pos = rng.uniform(0, 1, (n, 3)) * L
    m = n // 5
    pos[:m] = rng.integers(0, nc.astype(int), (m, 3)) * (L / nc)     # exactly on faces
    pos[m:m + 20] += L * rng.integers(-2, 3, (20, 3))                 # outside the box
    pos[m + 20:m + 30] = np.nextafter(L, 0)
    return pos


def _oracle_cells(L, pos):
    """Keys, canonical order and cell starts from the FP64 oracle."""
    import oracle as O
    s = O.System(L, np.zeros(len(pos), np.int32), np.array([[25.0]]), 4.5, 1.0, 0.04, 0.65)
    p = O.wrap(s, pos)
    key = O.cell_keys(s, p)
    order, start = O.cell_sort(s, key)
    return key, order, start


def _crowded(L, n, k, seed):
    """n beads, k of them packed inside one cell (a dense clump)."""
    rng = np.random.default_rng(seed)
    L = np.broadcast_to(np.asarray(L, float), (3,))
    pos = rng.uniform(0, 1, (n, 3)) * L
    h = L / np.floor(L)
    pos[rng.permutation(n)[:k]] = h * (1.0 + rng.uniform(0.05, 0.95, (k, 3)))
    return pos


def _noalloc(D, torch, L, pos):
    n = len(pos)
    ncell = int(np.prod(np.floor(L)))
    dev = torch.device("cuda", 0)
    pos_d = torch.tensor(pos, dtype=torch.float64, device=dev)
    key_d = torch.full((n,), -1, dtype=torch.int32, device=dev)
    order_d = torch.full((n,), -1, dtype=torch.int32, device=dev)
    start_d = torch.full((ncell + 1,), -1, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    rc = D.cells_noalloc(pos_d.data_ptr(), n, L, key_d.data_ptr(), order_d.data_ptr(),
                         start_d.data_ptr(), stream.cuda_stream)
    assert rc == D.DPD_OK
    torch.cuda.synchronize(dev)
    return (key_d.cpu().numpy().view(np.uint32), order_d.cpu().numpy().astype(np.int64),
            start_d.cpu().numpy().view(np.uint32).astype(np.int64))


def test_noalloc_cells_match_engine_on_two_calls():
    torch = pytest.importorskip("torch")
    from paper_1804_06205_gb300 import build
    build.build()
    from paper_1804_06205_gb300 import dpd as D

    cases = [((11.3, 9.0, 14.7), 4500, 1), ((6.0, 7.5, 5.2), 700, 2)]
    for L, n, seed in cases:
        w = W.fluid(L, n=n, seed=seed)
        pos = _face_heavy(L, n, seed + 10)
        # the existing path
        g = D.System.from_workload(w)
        g.set_state(pos, w.vel, 0)
        key_ref, order_ref, start_ref = g.cells()
        g.close()
        # the no-allocation path, on buffers the caller allocated
        key, order, start = _noalloc(D, torch, L, pos)
        assert np.array_equal(key, key_ref)
        assert np.array_equal(order, order_ref)
        assert np.array_equal(start, start_ref)
        # and directly against the oracle's cell division
        okey, oorder, ostart = _oracle_cells(L, pos)
        assert np.array_equal(key, okey)
        assert np.array_equal(order, oorder)
        assert np.array_equal(start, ostart)


def test_noalloc_crowded_cell_matches_oracle():
    """Hundreds to thousands of beads in one cell: the canonical (cell, id)
    order inside it is still exact, on two calls in a row."""
    torch = pytest.importorskip("torch")
    from paper_1804_06205_gb300 import build
    build.build()
    from paper_1804_06205_gb300 import dpd as D
    for L, n, k, seed in (((8.0, 9.5, 7.0), 5000, 3000, 41), ((5.0, 5.0, 6.3), 1500, 400, 42)):
        pos = _crowded(L, n, k, seed)
        key, order, start = _noalloc(D, torch, L, pos)
        okey, oorder, ostart = _oracle_cells(L, pos)
        assert np.diff(ostart).max() >= k
        assert np.array_equal(key, okey)
        assert np.array_equal(order, oorder)
        assert np.array_equal(start, ostart)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    pytest.importorskip("torch")
    from paper_1804_06205_gb300 import dpd as D
    # rejected before anything touches the device: no buffers needed
    fake = 0x1000
    assert D.cells_noalloc(fake, D.NOALLOC_MAX_N + 1, 200.0, fake, fake, fake) == D.DPD_EINVAL
    assert D.cells_noalloc(fake, 10, (2000.0, 2000.0, 3.0), fake, fake, fake) == D.DPD_EINVAL
    assert D.cells_noalloc(fake, 10, (2.5, 5.0, 5.0), fake, fake, fake) == D.DPD_EINVAL
