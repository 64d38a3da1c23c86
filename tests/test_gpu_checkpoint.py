"""Checkpoint and resume through the C ABI (dpd_get_checkpoint /
dpd_set_checkpoint and the batch forms).

Fig. 1 carries r, v and the force f(t) from one step to the next; a
checkpoint stores all three in the engine's own representation, so a run
that stops after n steps and resumes from its checkpoint in a new handle (or
inside a batch) must reproduce the uninterrupted 2n-step run bit for bit.
"""
import numpy as np
import pytest

from paper_1804_06205_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FP32, FP64 = 0, 1


@pytest.fixture(scope="module")
def D():
    from paper_1804_06205_gb300 import build
    build.build()
    from paper_1804_06205_gb300 import dpd
    return dpd


def _workload():
    # chains with harmonic and standard-Morse bonds in solvent, odd box
    return W.peptide_192k(L=9.5, nchains=8, chain_len=20, seed=61)


def _straight(D, w, prec, nsteps):
    g = D.System.from_workload(w, precision=prec)
    g.set_state(w.pos, w.vel, 0)
    g.step(2 * nsteps)
    out = g.get_state()
    g.close()
    return out


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_resume_from_records_copied_in_chunks(D, prec):
    """A system of 600k beads: its records cross the host link in several
    chunks of ids, each restored (or read out) while the next one moves, and
    the resumed run still equals the uninterrupted one bit for bit."""
    w = W.fluid(58.5, ntypes=2, a_same=25.0, a_cross=30.0, seed=63)
    assert w.n >= 2 * (1 << 18)
    n = 2
    ref = _straight(D, w, prec, n)
    g = D.System.from_workload(w, precision=prec)
    g.set_state(w.pos, w.vel, 0)
    g.step(n)
    ck = g.get_checkpoint()
    g.close()
    h = D.System.from_workload(w, precision=prec)
    h.set_checkpoint(ck)
    assert h.get_checkpoint() == ck
    h.step(n)
    out = h.get_state()
    h.close()
    for a, b in zip(ref[:3], out[:3]):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_restored_state_answers_like_the_original(D, prec):
    """A restore leaves the beads in bead-id order (the next step sorts them);
    observables, g(r) and the cell arrays asked for before any step must
    still equal those of the handle the checkpoint came from, bit for bit."""
    w = _workload()
    g = D.System.from_workload(w, precision=prec)
    g.set_state(w.pos, w.vel, 0)
    g.step(7)
    ck = g.get_checkpoint()
    o_ref = g.observables()
    gr_ref = g.gr_counts(2.0, 100)
    cells_ref = g.cells()
    g.close()
    for ask in ("observables", "gr", "cells"):
        h = D.System.from_workload(w, precision=prec)
        h.set_checkpoint(ck)
        if ask == "observables":
            o = h.observables()
            for k in ("kT", "p_total", "p_cons", "p_bond", "e_pair", "e_bond"):
                assert o[k] == o_ref[k], (k, o[k], o_ref[k])
        elif ask == "gr":
            assert np.array_equal(h.gr_counts(2.0, 100), gr_ref)
        else:
            for a, b in zip(h.cells(), cells_ref):
                assert np.array_equal(a, b)
        assert h.get_checkpoint() == ck
        h.close()


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_resume_alone_is_bitwise(D, prec):
    w = _workload()
    n = 12
    ref = _straight(D, w, prec, n)
    g = D.System.from_workload(w, precision=prec)
    g.set_state(w.pos, w.vel, 0)
    g.step(n)
    ck = g.get_checkpoint()
    g.close()
    h = D.System.from_workload(w, precision=prec)
    h.set_checkpoint(ck)
    assert h.get_state()[3] == n
    h.step(n)
    out = h.get_state()
    h.close()
    for a, b in zip(ref[:3], out[:3]):
        assert np.array_equal(a, b)
    assert out[3] == ref[3] == 2 * n


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_resume_in_a_batch_and_back_is_bitwise(D, prec):
    w = _workload()
    other = W.fluid((8.2, 7.0, 9.9), ntypes=2, a_same=25.0, a_cross=35.0, seed=62)
    n = 10
    ref = _straight(D, w, prec, n)
    # run alone for n steps, checkpoint, restore into a batch next to another system
    g = D.System.from_workload(w, precision=prec)
    g.set_state(w.pos, w.vel, 0)
    g.step(n)
    ck = g.get_checkpoint()
    g.close()
    b = D.Batch(max_beads=8000, max_cells=2000, max_bonds=2000, max_systems=4, precision=prec)
    so = b.add_workload(other)
    s = b.add_workload(w)          # any state; replaced by the checkpoint
    b.set_checkpoint(s, ck)
    b.step(n // 2)
    ck2 = b.get_checkpoint(s)      # half-way, from inside the batch
    b.step(n - n // 2)
    out = b.get_state(s)
    for a, c in zip(ref[:3], out[:3]):
        assert np.array_equal(a, c)
    b.close()
    # the batch's checkpoint restores alone
    h = D.System.from_workload(w, precision=prec)
    h.set_checkpoint(ck2)
    h.step(n - n // 2)
    out2 = h.get_state()
    h.close()
    for a, c in zip(ref[:3], out2[:3]):
        assert np.array_equal(a, c)
    assert so is not None


def test_checkpoint_rejects_foreign_or_damaged_data(D):
    w = _workload()
    g = D.System.from_workload(w, precision=FP32)
    g.set_state(w.pos, w.vel, 0)
    g.step(2)
    ck = g.get_checkpoint()
    assert len(ck) == 80 + 40 * w.n
    # another precision, another seed, a truncated buffer
    g64 = D.System.from_workload(w, precision=FP64)
    gs = D.System.from_workload(w, precision=FP32, seed=w.seed + 1)
    for sysx, data in ((g64, ck), (gs, ck), (g, ck[:-1])):
        with pytest.raises(D.DPDError) as e:
            sysx.set_checkpoint(data)
        assert e.value.code == D.DPD_EINVAL
    # a cell key out of range and a non-finite velocity
    bad = bytearray(ck)
    bad[80:84] = (2 ** 31).to_bytes(4, "little")
    with pytest.raises(D.DPDError) as e:
        g.set_checkpoint(bytes(bad))
    assert e.value.code == D.DPD_EINVAL
    bad = bytearray(ck)
    bad[80 + 16:80 + 20] = np.float32(np.nan).tobytes()
    with pytest.raises(D.DPDError) as e:
        g.set_checkpoint(bytes(bad))
    assert e.value.code == D.DPD_EINVAL
    # the handle still works after a rejected restore
    g.set_checkpoint(ck)
    g.step(1)
    assert g.get_state()[3] == 3
    for x in (g, g64, gs):
        x.close()


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_pinned_host_buffers_are_restored_in_place(D, prec):
    """A page-locked host buffer is read by the restore kernel directly over
    the host link; an unaligned one (offset by 4 bytes) and pageable memory go
    through the chunked copies, as every read-out does.  All give the same
    bytes, and a run resumed from each equals the uninterrupted run bit for
    bit."""
    import torch
    w = W.fluid(24.5, ntypes=2, a_same=25.0, a_cross=30.0, seed=67)
    n = 2
    ref = _straight(D, w, prec, n)
    g = D.System.from_workload(w, precision=prec)
    g.set_state(w.pos, w.vel, 0)
    g.step(n)
    ck = g.get_checkpoint()          # pageable bytes: the copy path
    nb = g.checkpoint_bytes()
    assert nb == len(ck)
    pin = torch.zeros(nb + 16, dtype=torch.uint8, pin_memory=True)
    base = pin.data_ptr()
    assert base % 8 == 0
    for off in (0, 4):               # read-outs into pinned memory, aligned or not
        pin.zero_()
        g.get_checkpoint_ptr(base + off, nb)
        assert pin.numpy()[off:off + nb].tobytes() == ck
    g.close()
    for off in (0, 4):
        pin.zero_()
        pin.numpy()[off:off + nb] = np.frombuffer(ck, dtype=np.uint8)
        h = D.System.from_workload(w, precision=prec)
        h.set_checkpoint_ptr(base + off, nb)
        assert h.get_checkpoint() == ck
        h.step(n)
        out = h.get_state()
        h.close()
        for a, b in zip(ref[:3], out[:3]):
            assert np.array_equal(a, b)
        assert out[3] == ref[3]
