"""Host <-> device state transfers: the chunked copies through pinned host
buffers (the pointer API a caller with its own pinned memory uses) give the
same state and forces as the same calls with ordinary numpy arrays."""
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


@pytest.mark.parametrize("prec", [0, 1])
def test_pinned_and_pageable_transfers_agree(D, prec):
    torch = pytest.importorskip("torch")
    w = W.fluid_1m()          # 1,029,000 beads: the transfers run in three chunks
    a = D.System.from_workload(w, precision=prec)
    a.set_state(w.pos, w.vel, 4)
    a.step(2)
    ref = a.get_state()
    a.close()
    pos_h = torch.from_numpy(np.ascontiguousarray(w.pos)).pin_memory()
    vel_h = torch.from_numpy(np.ascontiguousarray(w.vel)).pin_memory()
    frc_h = torch.empty_like(pos_h).pin_memory()
    b = D.System.from_workload(w, precision=prec)
    b.set_state_ptr(pos_h.data_ptr(), vel_h.data_ptr(), 4)
    b.step(2)
    step = b.get_state_ptr(pos_h.data_ptr(), vel_h.data_ptr(), frc_h.data_ptr())
    b.close()
    assert step == ref[3] == 6
    for x, y in zip((pos_h.numpy(), vel_h.numpy(), frc_h.numpy()), ref[:3]):
        assert np.array_equal(x, y)
