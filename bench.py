#!/usr/bin/env python
"""Benchmark of the DPD step loop (arxiv 1804.06205, Fig. 1) on GB300.

One step = position update + wrap + cell division + pair forces (eqs. 3-4
with Groot-Warren dissipative/random terms) + bonds + velocity update, for
the whole system, on the device.

Default workload: the 100^3 periodic box at rho = 3 (N = 3,000,000), types
A/B 50/50, a_AA = a_BB = 25, a_AB = 30, gamma = 4.5, kT = 1, dt = 0.04;
synthetic, seeded.  Prints ONE JSON line (rank 0):
  value   FP32 particle-steps/s, state resident in HBM, the step kernels
          launched directly (programmatic dependent launch) on one stream
  e2e     the same metric through the public API with host buffers: every
          step restores the full state (a checkpoint) from pinned host memory,
          steps, and writes the new checkpoint back
  roofline    the pair kernel (dominant) against the plain-ALU issue peak,
          with the algorithmic operation count of the method per bead
  roofline_hbm_phases  cell division and bonds/velocity/update against the
          HBM peak, with the method's minimum bytes per bead
  cpu_baseline  the FP64 oracle (cell-list mode) on the host cores; the same
          leg measures each path's one-evaluation force error against the
          oracle's brute-force sum on sampled beads (error_vs_oracle)
  paper_tables  the shapes of the paper's Tables 1 and 3 (N = 5k..100k) on
          the GPU, beside CAMUS's quoted CPU times (context)
  alpha_helix   the paper's alpha-helix run, 10,000 steps
  serving the batched half of the metric: a stream of independent systems
          (box edge 8..24, two types, 10% of beads in chains) arriving as a
          Poisson process, served by continuous batching; p50/p99 completion
          latency and throughput, after the autotuner picked the launch shape;
          serving_saturated: the same stream all arriving at once
  launch_modes  ms/step with one launch per kernel vs one persistent
          cooperative launch per call (small systems, a batch, fluid_3m)
  fp64_plain    the plain FP64 path, one system per launch (last in the line)

--impl reference times the FP64 CPU oracle (the only reference: the paper
publishes no code) on a bounded sample of the same workload.
--profile-target WORKLOAD runs set_state and a few steps of a named
workload (a target for kernel profilers; prints nothing else).
Multi-GPU: replicas only (each rank advances its own copy; value sums them).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "particle-steps/s at N=3M rho=3 (FP32 vs FP64 plain); batched p50/p99 latency"
UNIT = "particle-steps/s"
WORKLOAD_DESC = ("fluid_3m: periodic 100^3 box, rho=3, N=3,000,000, types A/B 50/50, "
                 "a_AA=a_BB=25, a_AB=30, gamma=4.5 (sigma=3), kT=1, dt=0.04, lambda=0.65")

# Algorithmic work of one step of the pair force, per bead at rho = 3, as
# the method requires it (each unique pair counted once): 40.5 candidate
# pairs in the half shell of 27 cells at ~8 FP32 ops (3 sub, 3 mul/fma,
# compare), and 6.28 unique pairs within r_c at ~150 ops (distance, weight,
# projections and force ~35 FP32; Philox4x32-10 ~100 INT32; Box-Muller ~3
# transcendentals + ~8 FP32).
PAIR_OPS_PER_BEAD = 40.5 * 8 + 6.28 * 150
# The same work recounted from the kernel's own operations (7 ops per
# candidate test; 103 per unique pair: geometry 13, Philox 60, uniforms 6,
# Box-Muller 6, force 11, sums 6, id order 2), reported beside it.
PAIR_OPS_PER_BEAD_RECOUNT = 40.5 * 7 + 6.28 * 103
# Minimum HBM bytes per bead and step of the two HBM-bound phases together
# (cell division, bonds + velocity + position update): the state (offset
# 16 B, velocity 16 B, force 16 B, id and key 8 B) read once and written
# once, doubled by the sort's gather: 200 B.
HBM_MIN_BYTES_PER_BEAD = 200.0
PROFILE_FIGURES = os.path.join(ROOT, "profiles", "k_pair_fluid_3m.md")
KERNEL_SOURCE = os.path.join(ROOT, "paper_1804_06205_gb300", "csrc", "kernels.cuh")


def profile_figures():
    """ncu figures of one k_pair launch on fluid_3m, from the committed
    profile, if they were taken on the current kernel source (else None)."""
    import hashlib
    import re
    try:
        text = open(PROFILE_FIGURES).read()
        m = re.search(r"<!-- figures (\{.*?\}) -->", text)
        fig = json.loads(m.group(1))
        sha = hashlib.sha1(open(KERNEL_SOURCE, "rb").read()).hexdigest()
    except Exception:
        return None
    fig["current"] = fig.get("kernel_source_sha1") == sha
    return fig


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    out = {"hbm_gbs": 6800.0, "source": "fallback", "sm_max_mhz": 2070.0}
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            for k in ("hbm_gbs", "bf16_tflops", "bf16_tflops_sustained"):
                if k in d:
                    out[k] = float(d[k])
            out["source"] = "measured"
            for k in ("sm_max_mhz", "clocks_sm_max_mhz"):
                if k in d:
                    out["sm_max_mhz"] = float(d[k])
        except Exception:
            pass
    return out


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.idx = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", "dpd_clocks_%d.csv" % os.getpid())

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_over_ranks(x, op, dist=None, device="cpu"):
    """x reduced over the ranks of the default process group (op "max" or
    "sum"); x itself on a single process."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def replica_throughput(units_local, secs_local, dist=None, device="cpu"):
    """Whole-job throughput of independent replicas: the units all ranks
    processed divided by the slowest rank's time."""
    units = reduce_over_ranks(units_local, "sum", dist, device)
    secs = reduce_over_ranks(secs_local, "max", dist, device)
    return units / secs, secs


def run_cpu_oracle(w, warmup, steps):
    """The FP64 oracle's cell-list mode on all host cores."""
    import oracle as O
    s = O.System(w.L, w.types, w.a, w.gamma, w.kT, w.dt, w.lam, seed=w.seed, bonds=w.bonds)
    st = O.State(s, w.pos, w.vel, 0, mode=O.MODE_CELLS)
    st.run(warmup)
    t0 = time.perf_counter()
    st.run(steps)
    dt = time.perf_counter() - t0
    return w.n * steps / dt, dt, O.num_threads()


def oracle_force_error(w, forces, step, nsample=256, seed=12):
    """One force evaluation of each GPU path against the FP64 oracle's
    brute-force pair sum on `nsample` beads drawn with a fixed seed:
    max |f_gpu - f_oracle| / max |f_oracle| over the sample (per path)."""
    import oracle as O
    s = O.System(w.L, w.types, w.a, w.gamma, w.kT, w.dt, w.lam, seed=w.seed, bonds=w.bonds)
    idx = np.random.default_rng(seed).choice(w.n, nsample, replace=False)
    t0 = time.perf_counter()
    fo = O.pair_forces_subset(s, w.pos, w.vel, step, idx)
    out = {"sampled_beads": nsample, "oracle_s": time.perf_counter() - t0,
           "what": "one force evaluation from an identical state: max|f - f_oracle| / "
                   "max|f_oracle| over the sampled beads (FP64 brute-force pair sum)"}
    scale = float(np.abs(fo).max())
    for name, f in forces.items():
        out[name] = float(np.abs(f[idx] - fo).max()) / scale
    out["tolerance"] = {"f32": 1e-4, "f64": 1e-10}
    return out


def reference_arm(args):
    from paper_1804_06205_gb300 import workloads as W
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    # bounded sample: same density, composition and parameters, 40^3 box
    L = args.ref_box
    w = W.fluid(L, ntypes=2, a_same=25.0, a_cross=30.0, seed=1004, name="fluid_3m_sample")
    value, secs, cores = run_cpu_oracle(w, args.warmup, args.steps)
    sample = ("FP64 oracle, cell-list mode, %d^3 box of the same fluid (N=%d), %d warm-up + "
              "%d timed steps" % (L, w.n, args.warmup, args.steps))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD_DESC, "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# CAMUS's best ms/step on 2x Xeon E5-2640 (Table 1: fluid; Table 3: with the
# 60-bead protein model), quoted as context.
CAMUS_TABLE1_MS = {5000: 2.8, 10000: 5.1, 50000: 24.8, 100000: 48.7}
CAMUS_TABLE3_MS = {5000: 2.8, 10000: 5.2, 50000: 25.9, 100000: 49.4}


def paper_tables_leg(D, W, stream, steps=300, warmup=20):
    """The paper's timing-table shapes on the GPU (FP32 and FP64)."""
    import torch
    out = []
    for protein, ref in ((False, CAMUS_TABLE1_MS), (True, CAMUS_TABLE3_MS)):
        for n, cpu_ms in ref.items():
            w = W.camus_table(n, protein=protein)
            row = {"table": 3 if protein else 1, "N": n, "camus_best_ms": cpu_ms}
            for prec, tag in ((D.DPD_FP32, "f32"), (D.DPD_FP64, "f64")):
                g = D.System.from_workload(w, precision=prec, cuda_stream=stream.cuda_stream)
                g.set_state(w.pos, w.vel, 0)
                g.step(warmup)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                g.step(steps)
                e1.record(stream)
                e1.synchronize()
                ms = e0.elapsed_time(e1) / steps
                g.close()
                row["gpu_ms_" + tag] = ms
            row["speedup_f32_vs_camus"] = cpu_ms / row["gpu_ms_f32"]
            out.append(row)
    return out


def alpha_helix_leg(D, W, stream):
    """The paper's alpha-helix run (10,000 steps, FP32) with its chain proxy."""
    import torch
    w = W.alpha_helix_24k()
    g = D.System.from_workload(w, precision=D.DPD_FP32, cuda_stream=stream.cuda_stream)
    g.set_state(w.pos, w.vel, 0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    g.step(w.steps)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    pos = g.get_state(vel=False, force=False)[0]
    o = g.observables()
    g.close()
    p = pos[:60]
    dist = {}
    for k in (1, 2, 4):
        d = p[k:] - p[:-k]
        d -= w.L * np.round(d / w.L)
        dist["d1%d" % (k + 1)] = float(np.linalg.norm(d, axis=1).mean())
    return {"workload": "alpha_helix_24k: 24,000 beads, 20^3, 60-bead chain, Fig. 3b bonds, "
                        "gamma=4.2, dt=0.02", "steps": w.steps, "ms_total": ms,
            "ms_per_step": ms / w.steps, "final_chain_mean_distances": dist,
            "kT": o["kT"], "p_total": o["p_total"]}


def launch_modes_leg(D, W, stream, steps=400, warmup=20):
    """ms/step of the one-launch-per-kernel path (programmatic dependent
    launch) and of the persistent cooperative launch (one launch per call of
    `steps` steps), FP32, on the small and batched workloads where launches
    matter and on fluid_3m."""
    import torch
    cases = [("alpha_helix_24k", [W.alpha_helix_24k()]),
             ("table1_5k", [W.camus_table(5000)]),
             ("serving_batch_9", [W.serving_system(900 + k) for k in range(9)]),
             ("fluid_3m", [W.fluid_3m()])]
    out = {}
    for name, ws in cases:
        row = {"beads": int(sum(w.n for w in ws)), "systems": len(ws)}
        st = steps if row["beads"] < 1_000_000 else 100
        for persistent in (0, 1):
            b = D.Batch(sum(w.n for w in ws), sum(int(np.prod(np.floor(w.L))) for w in ws),
                        max(1, sum(w.nbonds for w in ws)), max_systems=len(ws),
                        persistent=persistent, cuda_stream=stream.cuda_stream)
            for w in ws:
                b.add_workload(w)
            b.step(warmup)
            b.sync()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            l0 = b.launch_count()
            e0.record(stream)
            b.step(st)
            e1.record(stream)
            e1.synchronize()
            row["persistent_ms" if persistent else "direct_ms"] = e0.elapsed_time(e1) / st
            row["persistent_launches" if persistent else "direct_launches"] = b.launch_count() - l0
            b.close()
        row["steps"] = st
        out[name] = row
    return out


def serving_leg(args, stream, saturated=False, table=None):
    """Continuous batching of a stream of independent systems: Poisson
    arrivals at the workload's rate, or (saturated) all of them at t = 0."""
    from paper_1804_06205_gb300 import autotune, serving
    from paper_1804_06205_gb300 import workloads as W
    tune_s = 0.0
    if table is None:
        t0 = time.perf_counter()
        table = autotune.tune(edges=(8.0, 12.0, 16.0, 20.0, 24.0), threads=(128, 256),
                              beads=300_000, steps=8)
        tune_s = time.perf_counter() - t0
    reqs = W.serving_stream(nsys=args.serve_requests, rate_hz=args.serve_rate,
                            steps=args.serve_steps)
    if saturated:
        for r in reqs:
            r.arrival_s = 0.0
    srv = serving.Server(max_beads=3_000_000, max_cells=1_500_000, max_bonds=600_000,
                         max_systems=160, chunk=args.serve_chunk, table=table,
                         cuda_stream=stream.cuda_stream)
    l0 = srv.batch.launch_count()
    sampler = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    sampler.start()
    done = srv.run(reqs)
    clocks = sampler.stop()
    launches = srv.batch.launch_count() - l0
    srv.close()
    out = serving.summarize(done)
    out.update({"arrivals": "all at t=0" if saturated else "Poisson %g/s" % args.serve_rate,
                "steps_per_request": args.serve_steps, "chunk_steps": args.serve_chunk,
                "max_resident": srv.max_resident, "chunks": srv.chunks,
                "gpu_busy_frac": srv.busy_s / max(out["span_s"], 1e-9),
                "gpu_launches": launches, "clocks": clocks,
                "latency": "completion (final state on the host) - arrival"})
    if not saturated:
        out.update({"autotune": table, "autotune_s": tune_s,
                    "workload": "serving stream: %d systems, box edge U(8,24), rho=3, types A/B, "
                                "a_AB U(25,50), 10%% of beads in harmonic 10-mers, dt=0.04; "
                                "FP32" % args.serve_requests})
    return out, table


def profile_target(args):
    """set_state and a few steps of a named workload, for kernel profilers."""
    from paper_1804_06205_gb300 import build as B
    B.build()
    from paper_1804_06205_gb300 import dpd as D
    from paper_1804_06205_gb300 import workloads as W
    w = W.make(args.profile_target)
    g = D.System.from_workload(w, precision=args.profile_precision,
                               threads=args.profile_threads)
    g.set_state(w.pos, w.vel, 0)
    g.step(args.steps)
    g.sync()
    g.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=100)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="fluid_3m")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--fp64-steps", type=int, default=None)
    ap.add_argument("--cpu-steps", type=int, default=8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--ref-box", type=int, default=40)
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=256)
    ap.add_argument("--serve-rate", type=float, default=20.0)
    ap.add_argument("--serve-steps", type=int, default=2000)
    ap.add_argument("--serve-chunk", type=int, default=50)
    ap.add_argument("--profile-target", default=None, metavar="WORKLOAD")
    ap.add_argument("--profile-precision", type=int, default=0)
    ap.add_argument("--profile-threads", type=int, default=0)
    args = ap.parse_args()
    if args.profile_target:
        return profile_target(args)
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return reference_arm(args)

    import torch
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(x):
        return reduce_over_ranks(x, "max", dist, "cuda")

    from paper_1804_06205_gb300 import build as B
    if rank == 0:
        B.build()
    if dist is not None:
        dist.barrier()
    from paper_1804_06205_gb300 import dpd as D
    from paper_1804_06205_gb300 import workloads as W

    w = W.make(args.workload)
    # a dedicated stream for all of the library's work
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    peaks = _peaks()
    err_step = 11          # evaluation counter of the error-check state

    def timed(prec, warmup, steps, profile=True, sampler=None):
        g = D.System.from_workload(w, precision=prec, cuda_stream=stream.cuda_stream)
        g.set_state(w.pos, w.vel, err_step)
        f0 = g.get_state(pos=False, vel=False)[2]     # for the oracle error, untimed
        g.step(warmup)
        barrier()
        if sampler:
            sampler.start()
        l0 = g.launch_count()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.step(steps)
        e1.record(stream)
        barrier()
        ms = e0.elapsed_time(e1)
        launches = g.launch_count() - l0
        clocks = sampler.stop() if sampler else None
        g.sync()
        phases = None
        if profile:
            g.profile_begin(steps)
            g.step(steps)
            pms, pn = g.profile_end()
            phases = (pms / max(pn, 1)).tolist()
        pairs = int(g.gr_counts(1.0, 1)[0])
        g.close()
        return ms, launches, clocks, phases, pairs, f0

    # ---- FP32, state resident in HBM
    sampler = ClockSampler(local)
    ms32, launches, clocks, phases, pairs, f32 = timed(D.DPD_FP32, args.warmup, args.steps,
                                                       sampler=sampler)
    value, secs32 = replica_throughput(w.n * args.steps, ms32 * 1e-3, dist, "cuda")
    ms32 = secs32 * 1e3

    # ---- plain FP64 path
    fp64, f64 = None, None
    if not args.no_fp64:
        k64 = args.fp64_steps or args.steps
        ms64, _, _, ph64, _, f64 = timed(D.DPD_FP64, max(3, args.warmup // 4), k64)
        ms64 = max_over_ranks(ms64)
        v64 = ws * w.n * k64 / (ms64 * 1e-3)
        fp64 = {"value": v64, "unit": UNIT, "ms_per_step": ms64 / k64, "steps": k64,
                "phases_ms": dict(zip(("update_sort", "pair", "bond_vel"), ph64)),
                "fp32_speedup": value / v64}

    # ---- end to end through the public API with pinned host buffers: every
    # step takes its whole input state (a checkpoint: cell, offset, v, f per
    # bead) from pinned host memory and returns the new one there
    g = D.System.from_workload(w, precision=D.DPD_FP32, cuda_stream=stream.cuda_stream)
    g.set_state(w.pos, w.vel, 0)
    nb = g.checkpoint_bytes()
    ck_h = torch.empty(nb, dtype=torch.uint8).pin_memory()
    g.get_checkpoint_ptr(ck_h.data_ptr(), nb)
    for _ in range(2):
        g.set_checkpoint_ptr(ck_h.data_ptr(), nb)
        g.step(1)
        g.get_checkpoint_ptr(ck_h.data_ptr(), nb)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        g.set_checkpoint_ptr(ck_h.data_ptr(), nb)
        g.step(1)
        g.get_checkpoint_ptr(ck_h.data_ptr(), nb)
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    g.close()
    e2e = {"value": ws * w.n * args.e2e_steps / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": nb, "d2h_bytes_per_step": nb, "steps": args.e2e_steps,
           "note": "per step: dpd_set_checkpoint from pinned host (the full state, 40 B per "
                   "bead: cell, offset, v, f), dpd_step(1), dpd_get_checkpoint to pinned host"}

    # ---- roofline of the pair kernel (plain-ALU bound)
    pair_ms = phases[1]
    alu_peak = 152 * 128 * peaks["sm_max_mhz"] * 1e6          # lane-ops/s at max SM clock
    achieved = PAIR_OPS_PER_BEAD * w.n / (pair_ms * 1e-3)
    fig = profile_figures()
    cur = bool(fig and fig.get("current"))
    scale = w.n / fig["n"] if cur else None
    roofline = {"bound": "alu", "kernel": "k_pair", "achieved": achieved / 1e12,
                "peak": alu_peak / 1e12, "unit": "Tops/s", "frac": achieved / alu_peak,
                "traffic": fig["dram_bytes"] * scale if cur else None,
                "traffic_note": ("ncu dram read+write of one launch (profiles/k_pair_fluid_3m.md, "
                                 "taken on this kernel source)" if cur else
                                 "null: the committed ncu figures predate the current kernel"),
                "ops_per_bead": PAIR_OPS_PER_BEAD,
                "ops_per_bead_recount": PAIR_OPS_PER_BEAD_RECOUNT,
                "frac_recount": PAIR_OPS_PER_BEAD_RECOUNT * w.n / (pair_ms * 1e-3) / alu_peak,
                "launch_ms": pair_ms,
                "peak_source": "152 SMs x 128 lanes x %.0f MHz (one op per lane per cycle)"
                               % peaks["sm_max_mhz"]}
    if cur:
        ti = fig["thread_inst"] * scale
        roofline["issued"] = {"thread_inst_per_bead": ti / w.n,
                              "frac": ti / (pair_ms * 1e-3) / alu_peak,
                              "note": "thread instructions the kernel issues (ncu), same peak"}
    hbm_ms = phases[0] + phases[2]
    hbm = {"bytes_per_bead": HBM_MIN_BYTES_PER_BEAD, "ms": hbm_ms,
           "GBs": HBM_MIN_BYTES_PER_BEAD * w.n / (hbm_ms * 1e-3) / 1e9,
           "frac": HBM_MIN_BYTES_PER_BEAD * w.n / (hbm_ms * 1e-3) / 1e9 / peaks["hbm_gbs"],
           "phases_ms": {"update_sort": phases[0], "bond_vel": phases[2]},
           "peak_GBs": peaks["hbm_gbs"], "peak_source": peaks["source"],
           "note": "cell division + bonds/velocity/update against the method's minimum "
                   "bytes (state read and written once, doubled by the sort's gather)"}
    step_ms = ms32 / args.steps

    # ---- the oracle on the host: timing, and each path's force error
    cpu = err = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        v, secs, cores = run_cpu_oracle(w, 1, args.cpu_steps)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "FP64 oracle, cell-list mode, full fluid_3m (N=3,000,000), 1 warm-up + "
                         "%d timed steps on all host cores" % args.cpu_steps}
        forces = {"f32": f32}
        if f64 is not None:
            forces["f64"] = f64
        err = oracle_force_error(w, forces, err_step)

    serve = serve_sat = tables = helix = modes = None
    if ws == 1 and not args.no_extras:
        modes = launch_modes_leg(D, W, stream)
    if ws == 1 and not args.no_serving:
        serve, table = serving_leg(args, stream)
        serve_sat, _ = serving_leg(args, stream, saturated=True, table=table)
    if ws == 1 and not args.no_extras:
        tables = paper_tables_leg(D, W, stream)
        helix = alpha_helix_leg(D, W, stream)

    if rank == 0:
        keep = lambda d, ks: None if d is None else {k: d[k] for k in ks if k in d}
        skeys = ("requests", "arrivals", "p50_latency_s", "p99_latency_s",
                 "throughput_particle_steps_per_s", "max_resident", "gpu_busy_frac")
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD_DESC, "N": w.n,
                           "l2": "inputs larger than L2 (~0.5 GB of state per replica)",
                           "parallelism": "replicas" if ws > 1 else "single"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches, "clocks": clocks,
                # bulky context first; the tail of the line keeps the key results
                "paper_tables": tables, "alpha_helix": helix, "launch_modes": modes,
                "serving_detail": serve, "serving_saturated_detail": serve_sat,
                "pair_interactions_per_s": ws * pairs * args.steps / (ms32 * 1e-3),
                "phases_ms": dict(zip(("update_sort", "pair", "bond_vel"), phases)),
                "roofline_hbm_phases": hbm,
                "serving": keep(serve, skeys), "serving_saturated": keep(serve_sat, skeys),
                "error_vs_oracle": err, "fp64_plain": fp64}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
