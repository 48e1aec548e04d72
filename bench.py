#!/usr/bin/env python3
"""Benchmark: ideal-MHD RK2 cell-updates/s on B300 (one JSON line on rank 0).

Workload (default): 3D periodic turbulent box 256^3, FP64, rho = 1, P = 1/gamma,
uniform B0 along x at beta = 1, seeded random-phase solenoidal velocity with
E(k) ~ k^-2 for 1 <= |k| <= 8 at rms Mach 1, gamma = 5/3, CFL 0.4.  A "step" is one
full RK2 cycle (two stages: primitives, PLM, HLLD on x/y/z faces, E^c EMFs, CT and
cell update, CFL reduction, dt).  value = cells x cycles / device time, summed over
ranks.  Inputs (state 134 MB plus intermediates of several GB) are larger than the
126 MB L2, so no flush is needed between cycles.

Multi-GPU: the method does not shard here -- `--gpus N` under torchrun runs N
independent replicas (one box per rank, no data-path collective); a barrier and a
max over ranks bracket the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--n 256] [--precision fp64|fp32]
  python bench.py --impl reference ...   # the FP64 CPU oracle on host cores, same metric
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ideal-MHD cell-updates/s per B300 (FP64 vs FP32, plain vs served) + p50/p99"
UNIT = "cell-updates/s"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--n", type=int, default=256)
    p.add_argument("--precision", default="fp64", choices=["fp64", "fp32"])
    p.add_argument("--impl", default="idx", choices=["idx", "reference"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--mode", default="plain", choices=["plain", "batched", "serve", "accuracy"],
                   help="plain: one box (the headline line); batched: the 64-instance mix, "
                        "batched vs one at a time")
    p.add_argument("--cycles", type=int, default=100, help="cycles per instance (batched mode)")
    p.add_argument("--requests", type=int, default=200, help="requests in the served stream")
    p.add_argument("--budget-gb", type=float, default=120.0, help="HBM budget of the server")
    p.add_argument("--serve-precisions", default="fp32,fp64", help="precisions of the serve mode")
    p.add_argument("--serve-caps", default="0",
                   help="comma list of max active cells for admission (0 = no cap), serve mode")
    return p.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(x, dist=None):
    """Largest value of x over all ranks (x on every rank; identity without a process group).
    The tensor lives on the GPU for NCCL and on the host for gloo."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(units_per_rank, steps, world, ms_max):
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return units_per_rank * steps * world / (ms_max * 1e-3)


def workload_config(args):
    return {"workload": f"3D periodic turbulent box {args.n}^3, ideal MHD, "
                        f"{'FP64' if args.precision == 'fp64' else 'FP32 bulk / FP64 accumulation'}, "
                        "beta=1 B0 along x, random-phase solenoidal v, E(k)~k^-2 (k=1..8), "
                        "rms Mach 1, gamma=5/3, PLM+HLLD+E^c CT+RK2, CFL 0.4",
            "n": args.n, "cells": args.n ** 3, "precision": args.precision, "seed": 0,
            "l2": "inputs larger than L2 (no flush)", "parallelism": "replicas"}


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except FileNotFoundError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------- CPU baseline
def cpu_baseline(n=96, cycles=3):
    """The FP64 oracle as it stands on this host's cores: a bounded sample of the same
    workload (an n^3 box of the same recipe, `cycles` RK2 cycles)."""
    import oracle
    from paper_2304_13746_b300 import inputs
    ic = inputs.turbulent_box(n, seed=0)
    sim = oracle.Sim.from_prims(ic.prim, ic.lengths, ic.gamma, 0.4)
    t0 = time.perf_counter()
    for _ in range(cycles):
        sim.step()
    el = time.perf_counter() - t0
    return {"value": ic.ncells * cycles / el, "unit": UNIT, "cores": oracle.threads(),
            "kind": "oracle",
            "sample": f"turbulent box {n}^3 (same recipe, seed 0), {cycles} FP64 RK2 cycles, "
                      f"{el:.1f} s wall"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_2304_13746_b300 import inputs
    n = 64
    ic = inputs.turbulent_box(n, seed=0)
    sim = oracle.Sim.from_prims(ic.prim, ic.lengths, ic.gamma, 0.4)
    for _ in range(args.warmup):
        sim.step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        sim.step()
    el = time.perf_counter() - t0
    value = ic.ncells * args.steps / el
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": el / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.threads(),
                             "kind": "oracle",
                             "sample": f"each step one RK2 cycle of a {n}^3 box of the same "
                                       "recipe on the host cores (bounded sample)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU arm
# DRAM bytes per face of the dominant kernel, from one ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum of one launch, 192^3 box, scaled by faces): reported only while
# the bench's dominant kernel is the variant that was captured.
MEASURED_TRAFFIC_PER_FACE = {("fp64", "x", 32): (1.281667e9 + 0.780322e9) / 192 ** 3}


def alg_flops_per_face(cons, lengths, gamma):
    """Algorithmic flops per face of each direction from the oracle's op counter on a
    small box of the same recipe: HLLD + half of the two-sided reconstruction (each
    cell's slope counted once)."""
    import oracle
    out = []
    for d in range(3):
        h, r = oracle.count_faces(cons, lengths, gamma, d)
        out.append(sum(h[k] for k in ("add", "mul", "div", "sqrt")) +
                   0.5 * sum(r[k] for k in ("add", "mul", "div", "sqrt")))
    return out


def c4_instances(seed=4):
    """The batched workload: 64 independent instances, 32 Orszag-Tang 2D boxes with N
    log-uniform in [64, 512] and 32 turbulent 3D boxes with N log-uniform in [32, 128]
    (N rounded to a multiple of 8), the boxes seeded 1..32."""
    from paper_2304_13746_b300 import inputs
    rng = np.random.Generator(np.random.PCG64(seed))

    def r8(x):
        return int(max(8, 8 * round(x / 8)))
    ics = []
    for i in range(32):
        ics.append(inputs.orszag_tang_2d(r8(math.exp(rng.uniform(math.log(64), math.log(512))))))
    for i in range(32):
        n = r8(math.exp(rng.uniform(math.log(32), math.log(128))))
        ics.append(inputs.turbulent_box(n, seed=i + 1))
    return ics


def run_batched(args):
    import torch
    from paper_2304_13746_b300 import build as idx_build
    from paper_2304_13746_b300 import idx
    idx_build.build()
    idx.lib()
    ics = c4_instances()
    cells = sum(ic.ncells for ic in ics)
    K = args.cycles
    results = {}
    for precision in ("fp64", "fp32"):
        stream = torch.cuda.Stream()
        # one batch for all 64 instances
        sims = [idx.Sim(ic.shape, ic.lengths, ic.gamma, 0.4, precision, stream=stream.cuda_stream)
                for ic in ics]
        for s, ic in zip(sims, ics):
            s.set_primitive(ic.prim)
        b = idx.Batch(precision, stream=stream.cuda_stream)
        for s in sims:
            b.add(s)
        b.step(args.warmup)
        b.poll()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.step(K)
        e1.record(stream)
        e1.synchronize()
        ms_b = e0.elapsed_time(e1)
        shapes = b.shapes()
        for s in sims:
            b.remove(s)
        b.close()
        for s in sims:
            s.close()
        # the same instances one at a time (each a graph of its own cycle)
        sims = [idx.Sim(ic.shape, ic.lengths, ic.gamma, 0.4, precision, stream=stream.cuda_stream)
                for ic in ics]
        for s, ic in zip(sims, ics):
            s.set_primitive(ic.prim)
            for _ in range(args.warmup):
                s.step()
        torch.cuda.synchronize()
        e0.record(stream)
        for s in sims:
            for _ in range(K):
                s.step()
        e1.record(stream)
        e1.synchronize()
        ms_s = e0.elapsed_time(e1)
        for s in sims:
            s.close()
        results[precision] = {
            "batched": cells * K / (ms_b * 1e-3), "sequential": cells * K / (ms_s * 1e-3),
            "speedup": ms_s / ms_b, "ms_batched": ms_b, "ms_sequential": ms_s,
            "batch_sweep_shapes_xyz": shapes}
    line = {"metric": METRIC, "value": results["fp64"]["batched"], "unit": UNIT, "n_gpus": 1,
            "steps": K, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "batched: 64 independent instances (32 Orszag-Tang 2D, N "
                                   "log-uniform 64..512; 32 turbulent 3D boxes, N log-uniform "
                                   "32..128), own CFL dt each, one batch vs one at a time",
                       "instances": len(ics), "cells": cells, "cycles_per_instance": K},
            "batched": results}
    print(json.dumps(line), flush=True)


def run_serve(args):
    """Served stream: seeded Poisson arrivals of 2D/3D requests admitted under an HBM budget
    into one running batch (continuous batching), against the same stream one at a time."""
    import torch
    from paper_2304_13746_b300 import build as idx_build
    from paper_2304_13746_b300 import idx, serve
    idx_build.build()
    idx.lib()
    budget = int(args.budget_gb * 1e9)
    base = serve.make_payloads(serve.poisson_stream(args.requests, 20.0, seed=7))
    stream = torch.cuda.Stream()

    def clone(reqs, rate):
        out = []
        for r in reqs:
            q = serve.Request(r.rid, r.arrival * 20.0 / rate, r.kind, r.n, r.t_end, r.seed,
                              payload=r.payload)
            q.cells = r.cells
            out.append(q)
        return out

    def served(precision, rate, cap=None, order="oldest"):
        be = serve.IdxBackend(precision, stream=stream.cuda_stream)
        st = serve.Server(be, budget, cycles_per_poll=4, chunk_s=0.01,
                          max_active_cells=cap, order=order).run(clone(base, rate))
        be.close()
        return st

    results = {}
    for precision in args.serve_precisions.split(","):
        cap = served(precision, 1e9)                    # everything arrives at once
        mean_work = cap["cell_updates"] / max(cap["done"], 1)
        capacity_rps = cap["cell_updates_per_s"] / mean_work
        rate70 = 0.7 * capacity_rps
        r = {"capacity_req_per_s": capacity_rps, "mean_cell_updates_per_request": mean_work,
             "all_at_once": cap}
        r["sequential_all_at_once"] = serve.serve_sequential(
            serve.IdxSequential(precision, stream=stream.cuda_stream), clone(base, 1e9),
            budget_bytes=budget)
        r["served_70pct"] = dict(served(precision, rate70), rate=rate70)
        for cap in [int(float(c)) for c in args.serve_caps.split(",") if float(c) > 0]:
            r[f"served_70pct_cap{cap}"] = dict(served(precision, rate70, cap), rate=rate70,
                                               max_active_cells=cap)
        r["served_70pct_least_work"] = dict(served(precision, rate70, order="least_work"),
                                            rate=rate70, order="least_work")
        r["sequential_70pct"] = dict(serve.serve_sequential(
            serve.IdxSequential(precision, stream=stream.cuda_stream), clone(base, rate70),
            budget_bytes=budget), rate=rate70)
        if precision == "fp32":
            r["served_20rps"] = dict(served(precision, 20.0), rate=20.0)
        r["offered_load_at_20rps"] = 20.0 / capacity_rps
        results[precision] = r
    head = results.get("fp64", results[next(iter(results))])
    line = {"metric": METRIC, "value": head["served_70pct"]["cell_updates_per_s"],
            "unit": UNIT, "n_gpus": 1, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"served: {args.requests} requests, Poisson arrivals (seed 7), "
                                   "kind 2D/3D p=1/2, 2D Orszag-Tang N log-uniform 64..512, 3D "
                                   "turbulent box N log-uniform 32..128, t_end U[0.01, 0.1], "
                                   f"HBM budget {args.budget_gb:g} GB, continuous batching vs "
                                   "one at a time", "budget_bytes": budget},
            "served": results}
    print(json.dumps(line), flush=True)


def run_accuracy(args):
    """FP32-bulk error budget at n^3 (default 512^3): per-field L1 difference from FP64 vs
    the Richardson estimate of the discretisation error (half-resolution FP64 run)."""
    from paper_2304_13746_b300 import accuracy
    from paper_2304_13746_b300 import build as idx_build
    idx_build.build()
    n = args.n if args.n != 256 else 512
    t_end = 0.0175  # about 200 RK2 cycles of the 512^3 box
    r = accuracy.fp32_error_budget(n, t_end)
    line = {"metric": "FP32-bulk L1 error / discretisation error (per field)", "value": r["max_ratio"],
            "unit": "ratio", "higher_is_better": False, "n_gpus": 1, "dtype": "f32/f64",
            "data": "synthetic",
            "config": {"workload": f"3D turbulent box {n}^3 to t={t_end} (FP32 bulk vs FP64, "
                                   f"discretisation error from {n // 2}^3, p=2)"},
            "accuracy": r}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.mode == "batched":
        return run_batched(args)
    if args.mode == "serve":
        return run_serve(args)
    if args.mode == "accuracy":
        return run_accuracy(args)
    rank, world, local = dist_env()
    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    from paper_2304_13746_b300 import build as idx_build
    from paper_2304_13746_b300 import idx, inputs
    if rank == 0:
        idx_build.build()
    if dist:
        dist.barrier()
    idx.lib()

    ic = inputs.turbulent_box(args.n, seed=0)
    ncell = ic.ncells
    stream = torch.cuda.Stream()
    sim = idx.Sim(ic.shape, ic.lengths, ic.gamma, 0.4, args.precision, stream=stream.cuda_stream)
    sim.set_primitive(ic.prim)
    cons_host = sim.get_state()

    for _ in range(args.warmup):
        sim.step()
    torch.cuda.synchronize()

    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")   # lets a profiler select the timed cycles
    e0.record(stream)
    for _ in range(args.steps):
        sim.step()
    e1.record(stream)
    e1.synchronize()
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    sim.time()  # surfaces any device error of the timed cycles
    ms = max_over_ranks(ms, dist)
    value = aggregate_rate(ncell, args.steps, world, ms)
    n_active = sum(1 for s in ic.shape if s > 1)
    launches_per_cycle = 2 + 2 * (3 + n_active)

    # dominant kernel: per-launch device time of each kernel (events between launches)
    kt = sim.kernel_times(reps=2)
    shapes = sim.sweep_shapes()
    flops_face = alg_flops_per_face(
        [np.ascontiguousarray(a[:32, :32, :32]) for a in cons_host] if args.n > 32 else cons_host,
        (32 / args.n,) * 3 if args.n > 32 else ic.lengths, ic.gamma)
    sweep_ms = {d: kt[f"sweep_{d}"] for d in "xyz"}
    dom = max(sweep_ms, key=sweep_ms.get)
    d_i = "xyz".index(dom)
    achieved_gflops = flops_face[d_i] * ncell / (sweep_ms[dom] * 1e-3) / 1e9
    rates = idx.pipe_rates()
    if args.precision == "fp64":
        peak = 2 * rates["fma64"] / 1e9
        peak_note = "measured FP64 FMA rate x 2 flop (idx_pipe_rates, this GPU)"
    else:
        peak = 2 * rates["fma32"] / 1e9
        peak_note = "measured FP32 FMA rate x 2 flop (idx_pipe_rates, this GPU)"
    tpf = MEASURED_TRAFFIC_PER_FACE.get((args.precision, dom, shapes["xyz".index(dom)]))
    roofline = {"bound": "alu", "kernel": f"k_sweep<{'double' if args.precision == 'fp64' else 'float'},{dom}>",
                "achieved": achieved_gflops, "peak": peak, "unit": "GFLOP/s",
                "frac": achieved_gflops / peak,
                "traffic": tpf * ncell if tpf else None, "traffic_unit": "bytes per launch",
                "alg_flops_per_face": flops_face[d_i], "launch_ms": sweep_ms[dom],
                "peak_source": peak_note, "kernel_ms": kt, "sweep_shapes_xyz": shapes,
                "pipe_rates_gops": {k: v / 1e9 for k, v in rates.items()}}

    # end to end through the C ABI with host buffers: H2D state, one cycle, D2H state
    pinned = [torch.from_numpy(a).pin_memory().numpy() for a in cons_host]
    out_pinned = [torch.empty(ic.shape, dtype=torch.float64).pin_memory().numpy() for _ in range(8)]
    e2e_steps = max(3, min(args.steps, 10))
    sim.set_state(pinned)
    sim.step()
    sim.get_state(out=out_pinned)
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        sim.set_state(pinned)
        sim.step()
        sim.get_state(out=out_pinned)
    el = time.perf_counter() - t0
    el = max_over_ranks(el, dist)
    e2e = {"value": aggregate_rate(ncell, e2e_steps, world, el * 1e3), "unit": UNIT,
           "h2d_bytes_per_step": 8 * 8 * ncell, "d2h_bytes_per_step": 8 * 8 * ncell,
           "note": "per step: idx_set_state from pinned host (incl. its signal-speed pass), "
                   "idx_step, idx_get_state to pinned host"}
    sim.close()

    def time_variant(precision, ic_v=None, **kw):
        # another configuration (same box unless given), same timing rules
        ic_v = ic if ic_v is None else ic_v
        sv = idx.Sim(ic_v.shape, ic_v.lengths, ic_v.gamma, 0.4, precision, stream=stream.cuda_stream,
                     **kw)
        sv.set_primitive(ic_v.prim)
        for _ in range(args.warmup):
            sv.step()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            sv.step()
        e1.record(stream)
        e1.synchronize()
        msv = max_over_ranks(e0.elapsed_time(e1), dist)
        sv.time()
        out = {"value": aggregate_rate(ncell, args.steps, world, msv), "unit": UNIT,
               "ms_per_step": msv / args.steps, "sweep_shapes_xyz": sv.sweep_shapes()}
        sv.close()
        return out

    def time_advance(precision, ic_v, t_end):
        # a whole run through idx_advance (graph replays in chunks, end time clamped on the
        # device), timed from the first cycle to the synchronised end; the warm-up run
        # captures the sim's graph, then the state is set again at t = 0
        sv = idx.Sim(ic_v.shape, ic_v.lengths, ic_v.gamma, 0.4, precision, stream=stream.cuda_stream)
        sv.set_primitive(ic_v.prim)
        sv.advance(0.05 * t_end)
        sv.set_primitive(ic_v.prim)
        torch.cuda.synchronize()
        e0.record(stream)
        nst = sv.advance(t_end)
        e1.record(stream)
        e1.synchronize()
        msv = max_over_ranks(e0.elapsed_time(e1), dist)
        ncv = math.prod(ic_v.shape)
        out = {"value": aggregate_rate(ncv, nst, world, msv), "unit": UNIT, "cycles": nst,
               "ms_per_step": msv / nst}
        sv.close()
        return out

    variants = {}
    if args.precision == "fp64":
        # the small 2D problem of the paper's Orszag-Tang test, whole run: launch-bound
        ot2 = inputs.orszag_tang_2d(128)
        for prec in ("fp64", "fp32"):
            key = f"{prec}_orszag_tang_2d_128_to_t0.5"
            variants[key] = time_advance(prec, ot2, 0.5)
            variants[key]["note"] = ("2D Orszag-Tang 128^2 to t = 0.5 through idx_advance (16384 cells: "
                                     "launch-bound, one CUDA graph per cycle)")
        variants["fp32_bulk"] = time_variant("fp32")
        variants["fp64_vector_potential"] = time_variant("fp64", induction="potential")
        variants["fp64_vector_potential"]["note"] = "Eqs. 7-8: edge potential stepped, B = Bref + curl A"
        variants["fp64_rk3"] = time_variant("fp64", rk_order=3)
        variants["fp64_rk3"]["note"] = "RK3 (Table 1): three stages per cycle instead of two"
        variants["fp64_limo3"] = time_variant("fp64", recon="limo3")
        variants["fp64_limo3"]["note"] = "LimO3 reconstruction (Sec. 2.3) instead of van Leer PLM"
        variants["fp64_limo3_rk3"] = time_variant("fp64", recon="limo3", rk_order=3)
        variants["fp64_limo3_rk3"]["note"] = "LimO3 + RK3, the paper's higher-accuracy pairing"
        # the paper's own performance problem (Sec. 5): 3D Orszag-Tang, FP64, at this box size
        ot = inputs.orszag_tang_3d(args.n)
        variants["fp64_orszag_tang_3d"] = time_variant("fp64", ot)
        variants["fp64_orszag_tang_3d"]["note"] = (
            f"3D Orszag-Tang {args.n}^3 (Sec. 5 performance problem); the paper reports ~121 Mcell/s "
            "per V100 at 256^3 per GPU (4-GPU node, 484 Mcell/s): context, another machine")

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64" if args.precision == "fp64" else "f32/f64",
                "data": "synthetic", "config": workload_config(args),
                "gpu_launches": launches_per_cycle * args.steps,
                "clocks": clk, "roofline": roofline, "e2e": e2e, "variants": variants}
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline()
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
