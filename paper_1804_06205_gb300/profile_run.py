"""Run a named workload for a few steps (a target for kernel profilers).

    python -m paper_1804_06205_gb300.profile_run --workload fluid_1m --steps 6

Builds the system, sets its state (one force evaluation), advances `steps`
steps through CUDA-graph replay (or direct launches with --no-graph) and
prints the mean step time measured with CUDA events inside the library."""
from __future__ import annotations

import argparse
import time


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="fluid_1m")
    ap.add_argument("--steps", type=int, default=6)
    ap.add_argument("--precision", type=int, default=0)
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--graph", action="store_true")
    args = ap.parse_args()
    from . import dpd as D
    from . import workloads as W
    w = W.make(args.workload)
    g = D.System.from_workload(w, precision=args.precision, threads=args.threads,
                               use_graph=1 if args.graph else 0)
    g.set_state(w.pos, w.vel, 0)
    g.sync()
    t0 = time.perf_counter()
    g.step(args.steps)
    g.sync()
    dt = time.perf_counter() - t0
    print("%s N=%d steps=%d: %.3f ms/step (host clock), %d launches"
          % (w.name, w.n, args.steps, 1e3 * dt / max(args.steps, 1), g.launch_count()))
    g.close()


if __name__ == "__main__":
    main()
