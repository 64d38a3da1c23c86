"""Autotuner for the pair kernel's launch shape in batches.

Picks the threads per block (one value for a batch launch) and, per size
class of system (box edge), the brick length X (home cells along x of the
X x 2 x 2 bricks).  Each candidate is timed on the GPU with the library's
phase events: a batch of identical systems of the class advances a few steps
and the pair phase's mean time per bead is compared.
"""
from __future__ import annotations

import json

import numpy as np

from . import dpd as D
from . import workloads as W


def _time_pair(systems, threads, tile, steps):
    nb = sum(w.n for w in systems)
    nc = sum(int(np.prod(np.floor(w.L))) for w in systems)
    nbond = sum(w.nbonds for w in systems)
    b = D.Batch(nb, nc, max(nbond, 1), max_systems=len(systems), threads=threads)
    try:
        for w in systems:
            if b.add_workload(w, tile_cells=tile) is None:
                raise RuntimeError("tuning batch does not fit")
        b.step(3)
        b.profile_begin(steps)
        b.step(steps)
        ms, n = b.profile_end()
        return ms[1] / max(n, 1) / nb      # pair ms per bead per step
    finally:
        b.close()


def tune(edges=(8.0, 12.0, 16.0, 20.0, 24.0), threads=(64, 128, 256), beads=400_000,
         max_copies=96, steps=10, verbose=False) -> dict:
    """Time the pair phase for each thread count and brick length on batches
    of about `beads` beads made of identical systems of each edge class."""
    best_total, best = None, None
    classes = {}
    for e in edges:
        n1 = int(round(3.0 * e ** 3))
        copies = max(2, min(max_copies, beads // n1))
        classes[e] = [W.serving_system(900 + k, edge=e, a_ab=35.0) for k in range(copies)]
    for T in threads:
        tiles, total = {}, 0.0
        for e in edges:
            systems = classes[e]
            copies = len(systems)
            nx = int(np.floor(e))
            x0 = max(1, int(0.85 * T / (4 * 3.0)))     # ~0.85 T home beads at rho = 3
            cands = sorted({min(max(1, x), nx) for x in (x0 - 2, x0 - 1, x0, x0 + 1, x0 + 2,
                                                         x0 // 2)})
            times = {x: _time_pair(systems, T, x, steps) for x in cands}
            xb = min(times, key=times.get)
            tiles[e] = xb
            total += times[xb]
            if verbose:
                print("T=%d edge=%g copies=%d %s -> %d" % (
                    T, e, copies, {k: "%.3g" % (v * 1e6) for k, v in times.items()}, xb))
        if best_total is None or total < best_total:
            best_total, best = total, {"threads": T, "tiles": {str(k): v for k, v in tiles.items()}}
    best["pair_ns_per_bead_step"] = best_total * 1e6 / len(edges)
    return best


if __name__ == "__main__":
    import sys
    t = tune(verbose=True)
    print(json.dumps(t))
    if len(sys.argv) > 1:
        json.dump(t, open(sys.argv[1], "w"))
