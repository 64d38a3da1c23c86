"""Spatial domain decomposition along z on CPU ranks (gloo, world size 2):
the slab-decomposed oracle (oracle.slab: ghost layers of width r_c, bead
migration between slabs, bond partners across slab faces found by global id)
must reproduce the undecomposed FP64 oracle's trajectory to summation-order
roundoff.  No GPU is involved."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import oracle as O  # noqa: E402
from paper_1804_06205_gb300 import workloads as W  # noqa: E402

NSTEPS = 8


def _system():
    # peptide-like chains (harmonic 1-2, standard-Morse 1-3 and 1-5) in
    # solvent, in a box that is long along z so that each slab is 5 cells thick
    w = W.peptide_192k(L=10.0, nchains=6, chain_len=20, seed=81)
    L = np.array([6.0, 6.0, 10.0])
    rng = np.random.default_rng(82)
    keep = np.concatenate([np.arange(120), 120 + rng.permutation(w.n - 120)[:int(3 * 360) - 120]])
    idmap = -np.ones(w.n, np.int64)
    idmap[keep] = np.arange(keep.size)
    pos = w.pos[keep] % 10.0
    pos[:, :2] *= 0.6                            # squeeze x, y into the 6 x 6 cross-section
    b = w.bonds
    ok = (idmap[b["i"]] >= 0) & (idmap[b["j"]] >= 0)
    bonds = {k: (idmap[v[ok]] if k in ("i", "j") else v[ok]) for k, v in b.items()}
    vel = W.maxwell_velocities(np.random.default_rng(83), keep.size)
    return dict(L=L, types=w.types[keep], a=w.a, gamma=w.gamma, kT=w.kT, dt=w.dt, lam=w.lam,
                seed=w.seed, bonds=bonds, pos=pos, vel=vel)


def _worker(rank, world, port, out_path):
    from oracle.slab import SlabRank
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        s = _system()
        r = SlabRank(s["L"], s["types"], s["a"], s["gamma"], s["kT"], s["dt"], s["lam"],
                     s["seed"], s["bonds"], rank, world, dist)
        r.setup(s["pos"], s["vel"], 0)
        f0 = r.gather()
        r.step(NSTEPS)
        ids, pos, vel, f = r.gather()
        counts = [None] * world
        dist.all_gather_object(counts, (r.migrated, r.fetched, r.ids.size))
        if rank == 0:
            np.savez(out_path, ids=ids, pos=pos, vel=vel, f=f, f0=f0[3],
                     counts=np.array(counts))
    finally:
        dist.destroy_process_group()


def _port():
    with socket.socket() as sck:
        sck.bind(("127.0.0.1", 0))
        return sck.getsockname()[1]


def test_slab_decomposed_oracle_equals_undecomposed(tmp_path):
    out = str(tmp_path / "slab.npz")
    mp.start_processes(_worker, args=(2, _port(), out), nprocs=2, join=True,
                       start_method="spawn")
    r = np.load(out)
    s = _system()
    n = s["types"].size
    assert np.array_equal(r["ids"], np.arange(n))
    sysd = O.System(s["L"], s["types"], s["a"], s["gamma"], s["kT"], s["dt"], s["lam"],
                    seed=s["seed"], bonds=s["bonds"])
    st = O.State(sysd, s["pos"], s["vel"], 0)
    scale0 = np.abs(st.f).max()
    assert np.abs(r["f0"] - st.f).max() <= 1e-12 * scale0
    st.run(NSTEPS)
    d = r["pos"] - st.pos
    d -= s["L"] * np.round(d / s["L"])
    assert np.abs(d).max() < 1e-10
    assert np.abs(r["vel"] - st.vel).max() < 1e-10
    assert np.abs(r["f"] - st.f).max() <= 1e-9 * np.abs(st.f).max()
    # the decomposition was exercised: beads crossed slab faces, bonded
    # partners were fetched from the other rank, both slabs hold beads
    migrated, fetched, held = r["counts"].T
    assert migrated.sum() > 0
    assert fetched.sum() > 0
    assert held.min() > 0.3 * n


def test_slab_bounds_cover_the_box_in_whole_cells():
    from oracle.slab import SlabRank

    class NoDist:
        pass
    for Lz, world in ((10.0, 2), (11.7, 3), (7.5, 4)):
        ranks = [SlabRank((4.0, 4.0, Lz), np.zeros(3, np.int32), np.array([[25.0]]), 4.5, 1.0,
                          0.04, 0.65, 1, None, r, world, NoDist()) for r in range(world)]
        h = Lz / np.floor(Lz)
        assert ranks[0].zlo == 0.0 and ranks[-1].zhi == Lz
        for a, b in zip(ranks, ranks[1:]):
            assert a.zhi == b.zlo
            assert abs(b.zlo / h - round(b.zlo / h)) < 1e-12 and b.zlo - a.zlo >= h - 1e-12
        z = np.linspace(0, Lz, 1001, endpoint=False)
        own = ranks[0].owner(z)
        for r in ranks:
            assert np.all((own == r.rank) == ((z >= r.zlo) & (z < r.zhi)))
