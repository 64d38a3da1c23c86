"""Continuous-batching server for independent DPD systems.

Requests (one DPD system each, with a number of steps) arrive over time.  The
server keeps every admitted system resident in one batch (libdpd's
dpd_batch_*): all resident systems advance together, one launch per kernel
of the step loop for all of them, in chunks of a few dozen steps.  Between
chunks it
  * admits waiting requests first-come-first-served as long as they fit in
    the batch's pools (memory-based admission: dpd_batch_add refuses what
    does not fit, and the request waits for a departure);
  * reads back and removes the systems that have done all their steps.
Requests that arrive while others are on the GPU therefore join the running
batch within one chunk, and their work overlaps on the device.  Completion
latency = time the final state is on the host - arrival time.
"""
from __future__ import annotations

import collections
import dataclasses
import time
from typing import Dict, List, Optional, Sequence

import numpy as np

from .workloads import Request


@dataclasses.dataclass
class Completed:
    rid: int
    n: int
    steps: int
    arrival_s: float
    admit_s: float
    done_s: float
    state: Optional[tuple] = None

    @property
    def latency_s(self) -> float:
        return self.done_s - self.arrival_s


def tile_for(table: Optional[dict], L) -> int:
    """Brick length from an autotuner table {"tiles": {edge: X}} (nearest edge)."""
    if not table or not table.get("tiles"):
        return 0
    edges = sorted(float(e) for e in table["tiles"])
    e = min(edges, key=lambda x: abs(x - float(np.min(L))))
    for k, v in table["tiles"].items():
        if float(k) == e:
            return int(v)
    return 0


class Server:
    """precision 0 = FP32 path, 1 = FP64 path; table = autotuner output;
    use_graph: replay each step shape as a CUDA graph or launch the kernels
    directly (the default: direct launches overlap each kernel's start with
    the previous kernel's end through programmatic dependent launch, and
    admissions and departures would force the graphs to be captured again)."""

    def __init__(self, max_beads=2_000_000, max_cells=2_000_000, max_bonds=1_000_000,
                 max_systems=128, chunk=50, precision=0, table=None, keep_states=False,
                 clock=time.perf_counter, cuda_stream=None, use_graph=False):
        from . import dpd as D          # loads libdpd.so, fails loudly if it is not built
        threads = int(table.get("threads", 0)) if table else 0
        opts = dict(precision=precision, threads=threads, use_graph=1 if use_graph else 0)
        if cuda_stream is not None:
            opts["cuda_stream"] = cuda_stream
        self.batch = D.Batch(max_beads, max_cells, max_bonds, max_systems=max_systems, **opts)
        self.chunk = int(chunk)
        self.table = table
        self.keep = keep_states
        self.clock = clock
        self.max_resident = 0
        self.chunks = 0
        self.busy_s = 0.0     # host time spent waiting for chunks (the GPU is busy)

    def run(self, requests: Sequence[Request]) -> List[Completed]:
        """Serve the requests in real time (arrival_s relative to the start)."""
        b = self.batch
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival_s))
        waiting: collections.deque = collections.deque()
        resident: Dict[int, list] = {}
        done: List[Completed] = []
        t0 = self.clock()
        while pending or waiting or resident:
            now = self.clock() - t0
            while pending and pending[0].arrival_s <= now:
                waiting.append(pending.popleft())
            while waiting:               # first come, first served, while it fits
                r = waiting[0]
                sid = b.add_workload(r.workload, tile_cells=tile_for(self.table, r.workload.L))
                if sid is None:
                    if not resident:
                        raise RuntimeError("request %d does not fit in an empty batch" % r.rid)
                    break
                waiting.popleft()
                resident[sid] = [r, r.steps, self.clock() - t0]
            self.max_resident = max(self.max_resident, len(resident))
            if not resident:
                if pending:
                    time.sleep(max(0.0, pending[0].arrival_s - (self.clock() - t0)))
                continue
            k = min(self.chunk, min(v[1] for v in resident.values()))
            tb = self.clock()
            b.step(k)
            b.sync()
            self.busy_s += self.clock() - tb
            self.chunks += 1
            for v in resident.values():
                v[1] -= k
            for sid in [s for s, v in resident.items() if v[1] == 0]:
                r, _, admit_s = resident.pop(sid)
                st = b.get_state(sid, force=False)     # the result goes back to the client
                b.remove(sid)
                done.append(Completed(r.rid, r.workload.n, r.steps, r.arrival_s, admit_s,
                                      self.clock() - t0, st if self.keep else None))
        return done

    def close(self):
        self.batch.close()


def summarize(done: Sequence[Completed]) -> dict:
    lat = np.array([d.latency_s for d in done])
    work = float(sum(d.n * d.steps for d in done))
    t_first = min(d.arrival_s for d in done)
    t_last = max(d.done_s for d in done)
    return {"requests": len(done),
            "p50_latency_s": float(np.percentile(lat, 50)),
            "p99_latency_s": float(np.percentile(lat, 99)),
            "mean_latency_s": float(lat.mean()),
            "max_latency_s": float(lat.max()),
            "particle_steps": work,
            "throughput_particle_steps_per_s": work / (t_last - t_first),
            "span_s": t_last - t_first}
