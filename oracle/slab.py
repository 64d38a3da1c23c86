"""Spatial domain decomposition of the FP64 oracle along z, on CPU ranks.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle``): it checks the host
logic of a slab decomposition -- the route the paper names for systems past
1e7 beads (closing remark of section "Performance and parallel efficiency"
on hybrid OpenMP + MPI) -- against the undecomposed oracle.

The periodic box is cut along z into one slab per rank, each a whole number
of cells (edge h = Lz / floor(Lz) >= r_c), so a bead interacts only with beads
of its own slab and of the neighbouring slabs' layers within r_c of the
shared faces.  One step of Fig. 1 per rank:
  1. r += dt v + dt^2/2 f for the owned beads, periodic wrap;
  2. migration: beads whose z left the slab go to the owning rank, with v, f;
  3. v~ = v + lambda dt f;
  4. ghost exchange: positions, v~, types and ids of the beads within r_c of
     each face go to the rank across that face;
  5. f' = pair forces on the owned beads from owned + ghost beads (the pair
     noise keys on global ids and the evaluation counter, so it is the same
     on any rank), plus bonded forces, whose partners are found by global id
     among owned and ghost beads or fetched from their owners;
  6. v += dt/2 (f + f'), f = f'.
Exchanges are all-gathers of small Python objects over torch.distributed
(the gloo backend on CPU); no GPU memory is involved.
"""
from __future__ import annotations

import math
from typing import Dict, List

import numpy as np

from . import System, bond_one, pair_forces_ids, wrap


class SlabRank:
    """One rank's slab of a periodic system.  ``bonds`` holds every record
    (i, j, kind, r0, k, alpha) by global id; each rank keeps the full table,
    which is a parameter of the system, and uses the records of its beads."""

    def __init__(self, L, types, a, gamma, kT, dt, lam, seed, bonds, rank, world, dist):
        self.L = np.broadcast_to(np.asarray(L, float), (3,)).copy()
        self.types_all = np.ascontiguousarray(types, dtype=np.int32)
        self.sys = System(self.L, self.types_all, a, gamma, kT, dt, lam, seed=seed, bonds=bonds)
        self.dt, self.lam = float(dt), float(lam)
        self.rank, self.world, self.dist = rank, world, dist
        nz = int(math.floor(self.L[2]))
        if nz < world:
            raise ValueError("fewer z cells than ranks")
        h = self.L[2] / nz
        self.zlo = (rank * nz // world) * h
        self.zhi = ((rank + 1) * nz // world) * h if rank + 1 < world else self.L[2]
        self.cuts = [(r * nz // world) * h for r in range(world)] + [self.L[2]]
        # bond records of every bead id (both ends hold the record)
        n = self.types_all.size
        recs: List[list] = [[] for _ in range(n)]
        for q in range(len(bonds["i"]) if bonds is not None else 0):
            i, j = int(bonds["i"][q]), int(bonds["j"][q])
            r = (int(bonds["kind"][q]), float(bonds["r0"][q]), float(bonds["k"][q]),
                 float(bonds["alpha"][q]))
            recs[i].append((j,) + r)
            recs[j].append((i,) + r)
        self.recs = recs
        self.migrated = 0          # beads received by migration (for the tests)
        self.fetched = 0           # bond partners fetched from other ranks

    # ---------------------------------------------------------------- geometry
    def owner(self, z):
        """Rank owning each wrapped z."""
        return np.clip(np.searchsorted(self.cuts, z, side="right") - 1, 0, self.world - 1)

    def _min_image(self, d):
        return d - self.L * np.round(d / self.L)

    # ---------------------------------------------------------------- exchange
    def _alltoall(self, out: Dict[int, dict]) -> List[dict]:
        """out[r] = payload for rank r; returns the payloads sent to this rank."""
        gathered: List[Dict[int, dict]] = [None] * self.world
        self.dist.all_gather_object(gathered, out)
        return [g[self.rank] for g in gathered if g is not None and self.rank in g]

    def setup(self, pos, vel, step):
        """Take the owned beads of a global initial state (bead-id order) and
        evaluate f(step) at v~ = v."""
        p = wrap(self.sys, pos)
        mine = self.owner(p[:, 2]) == self.rank
        self.ids = np.nonzero(mine)[0].astype(np.int64)
        self.pos = p[mine].copy()
        self.vel = np.asarray(vel, float)[mine].copy()
        self.step_n = int(step)
        self.f = self.forces(self.vel)

    def _ghosts(self, vt):
        """Owned beads within r_c of the lower and upper faces go to the ranks
        across them; returns the received ghosts (ids, pos, v~)."""
        z = self.pos[:, 2]
        lower = (self.rank - 1) % self.world
        upper = (self.rank + 1) % self.world
        out: Dict[int, dict] = {}
        for dst, sel in ((lower, z - self.zlo < 1.0), (upper, self.zhi - z < 1.0)):
            if dst == self.rank or not sel.any():
                continue
            d = out.setdefault(dst, {"ids": [], "pos": [], "vt": []})
            d["ids"].append(self.ids[sel])
            d["pos"].append(self.pos[sel])
            d["vt"].append(vt[sel])
        for d in out.values():
            for k in d:
                d[k] = np.concatenate(d[k])
        got = self._alltoall(out)
        if not got:
            return np.zeros(0, np.int64), np.zeros((0, 3)), np.zeros((0, 3))
        ids = np.concatenate([g["ids"] for g in got])
        pos = np.concatenate([g["pos"] for g in got])
        vt = np.concatenate([g["vt"] for g in got])
        ids, first = np.unique(ids, return_index=True)    # both faces of one neighbour
        return ids, pos[first], vt[first]

    def _migrate(self):
        """Beads whose wrapped z left the slab move to their owner with v, f."""
        own = self.owner(self.pos[:, 2])
        out: Dict[int, dict] = {}
        for r in np.unique(own[own != self.rank]):
            sel = own == r
            out[int(r)] = {"ids": self.ids[sel], "pos": self.pos[sel], "vel": self.vel[sel],
                           "f": self.f[sel]}
        keep = own == self.rank
        self.ids, self.pos = self.ids[keep], self.pos[keep]
        self.vel, self.f = self.vel[keep], self.f[keep]
        got = self._alltoall(out)
        for g in got:
            self.migrated += g["ids"].size
            self.ids = np.concatenate([self.ids, g["ids"]])
            self.pos = np.concatenate([self.pos, g["pos"]])
            self.vel = np.concatenate([self.vel, g["vel"]])
            self.f = np.concatenate([self.f, g["f"]])
        order = np.argsort(self.ids, kind="stable")
        self.ids, self.pos = self.ids[order], self.pos[order]
        self.vel, self.f = self.vel[order], self.f[order]

    def _fetch(self, need: np.ndarray) -> Dict[int, np.ndarray]:
        """Positions of bond partners that are neither owned nor ghosts, by
        global id, from whichever rank owns them (every rank takes part)."""
        asks: List[np.ndarray] = [None] * self.world
        self.dist.all_gather_object(asks, need)
        answers: Dict[int, dict] = {}
        for src, ask in enumerate(asks):
            if src == self.rank or ask is None or ask.size == 0:
                continue
            hit = np.isin(ask, self.ids)
            sel = np.searchsorted(self.ids, ask[hit])
            answers[src] = {"ids": ask[hit], "pos": self.pos[sel]}
        out: Dict[int, np.ndarray] = {}
        for g in self._alltoall(answers):
            for i, p in zip(g["ids"], g["pos"]):
                out[int(i)] = p
        self.fetched += len(out)
        return out

    # ------------------------------------------------------------------ forces
    def forces(self, vt):
        """Pair forces of the owned beads from owned + ghost beads, plus the
        bonded forces of the owned beads' records."""
        gids, gpos, gvt = self._ghosts(vt)
        ids = np.concatenate([self.ids, gids])
        pos = np.concatenate([self.pos, gpos])
        vtt = np.concatenate([vt, gvt])
        f = pair_forces_ids(self.sys, pos, vtt, self.types_all[ids], ids, self.ids.size,
                            self.step_n)
        where = {int(i): k for k, i in enumerate(ids)}
        need = sorted({j for i in self.ids for (j, *_r) in self.recs[int(i)]
                       if j not in where})
        far = self._fetch(np.asarray(need, np.int64)) if self.world > 1 else {}
        for q, i in enumerate(self.ids):
            for (j, kind, r0, k, alpha) in self.recs[int(i)]:
                pj = pos[where[j]] if j in where else far[j]
                d = self._min_image(self.pos[q] - pj)
                F, _ = bond_one(kind, r0, k, alpha, d)
                f[q] += F
        return f

    # -------------------------------------------------------------------- step
    def step(self, nsteps=1):
        """nsteps steps of Fig. 1 for the owned beads."""
        dt = self.dt
        for _ in range(nsteps):
            self.pos = wrap_rows(self.pos + dt * self.vel + 0.5 * dt * dt * self.f, self.L)
            self._migrate()
            vt = self.vel + self.lam * dt * self.f
            self.step_n += 1
            f_new = self.forces(vt)
            self.vel = self.vel + 0.5 * dt * (self.f + f_new)
            self.f = f_new

    def gather(self):
        """(ids, pos, vel, f) of every rank's owned beads, on every rank."""
        parts: List[tuple] = [None] * self.world
        self.dist.all_gather_object(parts, (self.ids, self.pos, self.vel, self.f))
        ids = np.concatenate([p[0] for p in parts])
        order = np.argsort(ids)
        return (ids[order],) + tuple(np.concatenate([p[k] for p in parts])[order]
                                     for k in (1, 2, 3))


def wrap_rows(pos, L):
    """x - L floor(x / L) with the fix-ups of the oracle's wrap (result in [0, L))."""
    y = pos - L * np.floor(pos / L)
    y = np.where(y < 0.0, y + L, y)
    return np.where(y >= L, y - L, y)
