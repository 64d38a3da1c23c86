"""dpd_cells_noalloc: the cell division for callers that cannot allocate
device memory (their memory belongs to a framework allocator or a fixed
arena, or they must avoid cudaMalloc's implicit synchronisation).  The
caller owns every buffer; the library only uses its fixed scratch array.

Checked through the C ABI against the existing path (dpd_set_state +
dpd_get_cells) on two calls in a row, with different sizes, so that the
shared scratch's leftovers from the first call cannot leak into the second.
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
        key = key_d.cpu().numpy().view(np.uint32)
        order = order_d.cpu().numpy().astype(np.int64)
        start = start_d.cpu().numpy().view(np.uint32).astype(np.int64)
        assert np.array_equal(key, key_ref)
        assert np.array_equal(order, order_ref)
        assert np.array_equal(start, start_ref)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    pytest.importorskip("torch")
    from paper_1804_06205_gb300 import dpd as D
    # rejected before anything touches the device: no buffers needed
    fake = 0x1000
    assert D.cells_noalloc(fake, D.NOALLOC_MAX_N + 1, 200.0, fake, fake, fake) == D.DPD_EINVAL
    assert D.cells_noalloc(fake, 10, (2000.0, 2000.0, 3.0), fake, fake, fake) == D.DPD_EINVAL
    assert D.cells_noalloc(fake, 10, (2.5, 5.0, 5.0), fake, fake, fake) == D.DPD_EINVAL
