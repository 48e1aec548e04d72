#!/usr/bin/env python3
"""Benchmark: ideal-MHD RK2 cell-updates/s on B300 (one JSON line on rank 0).

Workload (default): 3D periodic turbulent box 256^3, FP64, rho = 1, P = 1/gamma,
uniform B0 along x at beta = 1, seeded random-phase solenoidal velocity with
E(k) ~ k^-2 for 1 <= |k| <= 8 at rms Mach 1, gamma = 5/3, CFL 0.4.  A "step" is one
full RK2 cycle (two stages: primitives, PLM, HLLD on x/y/z faces, E^c EMFs, CT and
cell update, CFL reduction, dt).  value = cells x cycles / device time of the median of
5 timed regions of K cycles each, summed over ranks.  Inputs (state 134 MB plus
intermediates of several GB) are larger than the 126 MB L2, so no flush is needed
between cycles.

Beside the headline the default run measures, on the same GPU (each under `variants`):
FP32 bulk at 256^3 and 512^3 and FP64 at 512^3, each with the roofline of the slower of
its HBM bytes, FP32 flops and FP64 flops; the batched 64-instance mix, batched vs one at
a time, FP64 and FP32; a served Poisson stream at 2D 64^2..1024^2 / 3D 64^3..256^3 sizes
and end times 0.1..1 crossing times, continuous batching vs one at a time, with p50/p99;
and the paper's 3D Orszag-Tang problem and the RK3, LimO3 and vector-potential forms.

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
REGIONS = 5                # timed regions of the headline; the median is reported
BYTES_PER_UPDATE = 320     # algorithmic HBM bytes per cell-update (RK2, FP64 state)
FP64_NOMINAL_GFLOPS = 1250.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--n", type=int, default=256)
    p.add_argument("--precision", default="fp64", choices=["fp64", "fp32"])
    p.add_argument("--impl", default="idx", choices=["idx", "reference"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--stage-kernels", default="auto", choices=["auto", "split", "fused", "carry"],
                   help="kernels of a stage for the headline box (fused, carry: FP32 bulk only)")
    p.add_argument("--sweep-shapes", default="",
                   help="x,y,z sweep shapes for the headline box instead of the autotuner's "
                        "(profiling runs; e.g. 32,116,116)")
    p.add_argument("--no-variants", action="store_true",
                   help="headline, roofline and e2e only (profiling runs)")
    p.add_argument("--mode", default="plain", choices=["plain", "batched", "serve", "accuracy"],
                   help="plain: the default line; batched / serve: that part alone, with all "
                        "its policies; accuracy: the FP32-bulk error budget")
    p.add_argument("--cycles", type=int, default=100, help="cycles per instance (batched mix)")
    p.add_argument("--instances", type=int, default=64,
                   help="batched mode: the first N instances of the 64-instance mix")
    p.add_argument("--batch-precisions", default="fp64,fp32", help="precisions of the batched mode")
    p.add_argument("--serve-requests-fp32", type=int, default=16)
    p.add_argument("--serve-requests-fp64", type=int, default=6)
    p.add_argument("--budget-gb", type=float, default=120.0, help="HBM budget of the server")
    p.add_argument("--serve-precisions", default="fp32,fp64", help="precisions of the serve mode")
    p.add_argument("--serve-caps", default="0",
                   help="comma list of max active cells for admission (0 = no cap), serve mode")
    return p.parse_args()


def parse_args_for_test(argv=()):
    """The options bench.py would take from argv (for host-side tests)."""
    saved = sys.argv
    try:
        sys.argv = ["bench.py", *argv]
        return parse()
    finally:
        sys.argv = saved


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
            "timing": f"median of {REGIONS} CUDA-event regions of --steps cycles each",
            "l2": "inputs larger than L2 (no flush)", "parallelism": "replicas",
            "stage_kernels": args.stage_kernels,
            "sweep_shapes": args.sweep_shapes or "autotuned"}


def measured_peaks():
    """HBM copy bandwidth (GB/s) from MEASURED_PEAKS.json, else the stated fallback."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "MEASURED_PEAKS.json hbm_gbs (of measured)"
    except (OSError, KeyError, ValueError):
        return 6400.0, "fallback 6.4 TB/s (of fallback)"


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


REFERENCE_SAMPLE_N = 64


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_2304_13746_b300 import inputs
    n = REFERENCE_SAMPLE_N
    ic = inputs.turbulent_box(n, seed=0)
    sim = oracle.Sim.from_prims(ic.prim, ic.lengths, ic.gamma, 0.4)
    for _ in range(args.warmup):
        sim.step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        sim.step()
    el = time.perf_counter() - t0
    value = ic.ncells * args.steps / el
    sample = (f"each step is one FP64 RK2 cycle of a {n}^3 box of the same recipe ({ic.ncells} "
              f"cells, seed 0), a bounded sample of the {args.n}^3 workload; value = sample "
              "cells x steps / host seconds")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": el / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args),
            "reference_sample": {"box": f"{n}^3", "cells_per_step": ic.ncells,
                                 "note": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- op counts
# DRAM bytes per face of the dominant kernel, from one ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum of one launch, 192^3 box, scaled by faces): reported only while
# the bench's dominant kernel is the variant that was captured.
# DRAM bytes per face of the dominant sweep, from one ncu capture at 192^3 of the current
# kernel (dram__bytes_read.sum + dram__bytes_write.sum over the faces of the launch)
MEASURED_TRAFFIC_PER_FACE = {("fp64", "x", 32): (1278596096 + 785182976) / 192 ** 3,
                             ("fp64", "x", -2): (453105920 + 412378880) / 192 ** 3,
                             ("fp32", "x", -2): (254834944 + 188080128) / 192 ** 3}


def op_counts(cons, lengths, gamma):
    """Algorithmic flops from the oracle's pinned op counter on a sample of the state:
    per cell-update of one RK2 cycle (whole, and the part the FP32-bulk variant keeps in
    FP64) and per face of each direction (HLLD, face values and each slope once)."""
    import oracle
    parts = oracle.count_cycle_parts(cons, lengths, gamma, 0.4)
    face = [oracle.algorithmic_face_flops(oracle.count_faces_parts(cons, lengths, gamma, d))
            for d in range(3)]
    total = sum(oracle.flops(c) for c in parts.values())
    return {"cycle_flops_counted": total, "cycle_flops": oracle.algorithmic_flops(parts),
            "fp64_island_flops": oracle.fp64_island_flops(parts), "face_flops": face,
            "parts": {p: oracle.flops(c) for p, c in parts.items()}}


def roofline_cycle(value, counts, rates, hbm_gbs, precision):
    """Roofline of a whole cycle: the slower of its algorithmic HBM bytes at the measured
    copy bandwidth, its FP64 flops at the FP64 flop peak and (FP32 bulk) its FP32 flops at
    the FP32 flop peak; frac = that bound's time / the measured time per cell-update."""
    f64 = 2 * rates["fma64"]
    f32 = 2 * rates["fma32"]
    t = {"hbm": BYTES_PER_UPDATE / (hbm_gbs * 1e9)}
    if precision == "fp64":
        t["fp64"] = counts["cycle_flops"] / f64
    else:
        t["fp64"] = counts["fp64_island_flops"] / f64
        t["fp32"] = (counts["cycle_flops"] - counts["fp64_island_flops"]) / f32
    bound = max(t, key=t.get)
    out = {"bound": bound, "bound_cell_updates_per_s": 1.0 / t[bound],
           "frac": value * t[bound],
           "ns_per_cell_update": {k: v * 1e9 for k, v in t.items()},
           "measured_ns_per_cell_update": 1e9 / value,
           "alg_flops_per_cell_update": counts["cycle_flops"],
           "bytes_per_cell_update": BYTES_PER_UPDATE}
    if precision != "fp64":
        out["fp64_island_flops_per_cell_update"] = counts["fp64_island_flops"]
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


def batched_mix(ics, precision, K, warmup):
    """The mix as one batch (K batched cycles) and one at a time (K cycles each)."""
    import torch
    from paper_2304_13746_b300 import idx
    cells = sum(ic.ncells for ic in ics)
    stream = torch.cuda.Stream()
    sims = [idx.Sim(ic.shape, ic.lengths, ic.gamma, 0.4, precision, stream=stream.cuda_stream)
            for ic in ics]
    for s, ic in zip(sims, ics):
        s.set_primitive(ic.prim)
    b = idx.Batch(precision, stream=stream.cuda_stream)
    for s in sims:
        b.add(s)
    b.step(warmup)
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
    sims = [idx.Sim(ic.shape, ic.lengths, ic.gamma, 0.4, precision, stream=stream.cuda_stream)
            for ic in ics]
    for s, ic in zip(sims, ics):
        s.set_primitive(ic.prim)
        for _ in range(warmup):
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
    return {"batched": cells * K / (ms_b * 1e-3), "sequential": cells * K / (ms_s * 1e-3),
            "speedup": ms_s / ms_b, "ms_batched": ms_b, "ms_sequential": ms_s,
            "batch_sweep_shapes_xyz": shapes}


def run_batched(args):
    from paper_2304_13746_b300 import build as idx_build
    from paper_2304_13746_b300 import idx
    idx_build.build()
    idx.lib()
    ics = c4_instances()
    ics = ics[:32][:max(0, args.instances // 2)] + ics[32:][:max(0, args.instances - args.instances // 2)]
    cells = sum(ic.ncells for ic in ics)
    results = {p: batched_mix(ics, p, args.cycles, args.warmup)
               for p in args.batch_precisions.split(",")}
    line = {"metric": METRIC, "value": results[next(iter(results))]["batched"], "unit": UNIT,
            "n_gpus": 1,
            "steps": args.cycles, "warmup": args.warmup, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": C4_WORKLOAD, "instances": len(ics), "cells": cells,
                       "cycles_per_instance": args.cycles},
            "batched": results}
    print(json.dumps(line), flush=True)


C4_WORKLOAD = ("batched: 64 independent instances (32 Orszag-Tang 2D, N log-uniform 64..512; "
               "32 turbulent 3D boxes, N log-uniform 32..128), own CFL dt each, one batch vs "
               "one at a time")

# the served stream at the survey's C5 reading: kind 2D/3D with p = 1/2, 2D Orszag-Tang N
# log-uniform in [64, 1024], 3D turbulent box N log-uniform in [64, 256], t_end uniform in
# [0.1, 1.0] crossing times (t_cross = 1 for both), Poisson arrivals, seed 7
C5 = {"sizes_2d": (64, 1024), "sizes_3d": (64, 256), "t_end": (0.1, 1.0), "seed": 7}


def served_stream(precision, nreq, budget, serve_mod, stream, orders=("oldest",), caps=()):
    """The first nreq requests of the C5 stream, served three ways: all arriving at once
    (capacity), then at 70 % of that capacity by continuous batching and one at a time."""
    base = serve_mod.make_payloads(serve_mod.poisson_stream(
        nreq, 20.0, seed=C5["seed"], sizes_2d=C5["sizes_2d"], sizes_3d=C5["sizes_3d"],
        t_end=C5["t_end"]))

    def clone(rate):
        out = []
        for r in base:
            q = serve_mod.Request(r.rid, r.arrival * 20.0 / rate, r.kind, r.n, r.t_end, r.seed,
                                  payload=r.payload)
            q.cells = r.cells
            out.append(q)
        return out

    def failures(reqs):
        # a request whose state turns non-physical ends with its error (the method has no
        # positivity safeguard); it is the same request alone and in the mix
        return [{"rid": q.rid, "kind": q.kind, "n": q.n, "t_end": round(q.t_end, 3),
                 "error": q.error} for q in reqs if q.status == "failed"]

    def served(rate, cap=None, order="oldest"):
        be = serve_mod.IdxBackend(precision, stream=stream)
        reqs = clone(rate)
        st = serve_mod.Server(be, budget, cycles_per_poll=4, chunk_s=0.01,
                              max_active_cells=cap, order=order).run(reqs)
        be.close()
        return dict(st, failed_requests=failures(reqs))

    def sequential(rate):
        reqs = clone(rate)
        st = serve_mod.serve_sequential(serve_mod.IdxSequential(precision, stream=stream),
                                        reqs, budget_bytes=budget)
        return dict(st, failed_requests=failures(reqs))

    cap = served(1e9)                     # everything at once: the batch's capacity
    seq_cap = sequential(1e9)             # everything at once, one at a time
    mean_work = cap["cell_updates"] / max(cap["done"], 1)
    capacity_rps = cap["cell_updates_per_s"] / mean_work
    rate70 = 0.7 * capacity_rps
    r = {"requests": nreq, "capacity_req_per_s": capacity_rps,
         "capacity_cell_updates_per_s": cap["cell_updates_per_s"],
         "mean_cell_updates_per_request": mean_work, "all_at_once": cap,
         "all_at_once_sequential": seq_cap,
         "capacity_vs_sequential": cap["cell_updates_per_s"] / max(seq_cap["cell_updates_per_s"], 1e-30),
         "sizes": [f"{q.kind} {q.n}" for q in base], "t_end": [round(q.t_end, 3) for q in base]}
    for order in orders:
        key = "served_70pct" if order == "oldest" else f"served_70pct_{order}"
        r[key] = dict(served(rate70, order=order), rate=rate70, order=order,
                      offered_load=0.7)
    for c in caps:
        r[f"served_70pct_cap{c}"] = dict(served(rate70, c), rate=rate70, max_active_cells=c)
    r["sequential_70pct"] = dict(sequential(rate70), rate=rate70, offered_load=0.7)
    s, q = r["served_70pct"], r["sequential_70pct"]
    r["summary"] = {"capacity_cell_updates_per_s": cap["cell_updates_per_s"],
                    "sequential_capacity_cell_updates_per_s": seq_cap["cell_updates_per_s"],
                    "served_p50_s": s["p50_s"], "served_p99_s": s["p99_s"],
                    "sequential_p50_s": q["p50_s"], "sequential_p99_s": q["p99_s"],
                    "served_cell_updates_per_s": s["cell_updates_per_s"],
                    "sequential_cell_updates_per_s": q["cell_updates_per_s"]}
    return r


def run_serve(args):
    """Served stream alone, with every admission policy."""
    import torch
    from paper_2304_13746_b300 import build as idx_build
    from paper_2304_13746_b300 import idx, serve
    idx_build.build()
    idx.lib()
    budget = int(args.budget_gb * 1e9)
    stream = torch.cuda.Stream()
    caps = [int(float(c)) for c in args.serve_caps.split(",") if float(c) > 0]
    results = {}
    for precision in args.serve_precisions.split(","):
        n = args.serve_requests_fp32 if precision == "fp32" else args.serve_requests_fp64
        results[precision] = served_stream(precision, n, budget, serve, stream.cuda_stream,
                                           orders=("oldest", "least_work"), caps=caps)
    head = results[next(iter(results))]
    line = {"metric": METRIC, "value": head["served_70pct"]["cell_updates_per_s"],
            "unit": UNIT, "n_gpus": 1, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": C5_WORKLOAD, "budget_bytes": budget}, "served": results}
    print(json.dumps(line), flush=True)


C5_WORKLOAD = ("served: Poisson arrivals (seed 7), kind 2D/3D p=1/2, 2D Orszag-Tang N "
               "log-uniform 64..1024, 3D turbulent box N log-uniform 64..256, t_end U[0.1, 1.0] "
               "crossing times, HBM budget 120 GB, first R requests of the stream at 70 % of "
               "the capacity an all-at-once run measures; continuous batching vs one at a time")


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


def guarded(fn, *a, **kw):
    """A variant's numbers, or the error that stopped it (the headline line still prints)."""
    try:
        return fn(*a, **kw)
    except Exception as e:  # noqa: BLE001 -- reported in the JSON line
        return {"error": f"{type(e).__name__}: {e}"}


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
    hbm_gbs, hbm_source = measured_peaks()

    ic = inputs.turbulent_box(args.n, seed=0)
    ncell = ic.ncells
    stream = torch.cuda.Stream()
    sim = idx.Sim(ic.shape, ic.lengths, ic.gamma, 0.4, args.precision, stream=stream.cuda_stream)
    sim.set_primitive(ic.prim)
    sim.set_stage_kernels(args.stage_kernels)
    if args.sweep_shapes:
        sim.set_sweep_shapes(tuple(int(v) for v in args.sweep_shapes.split(",")))
    fused = sim.stage_kernels() == "fused"
    carry = sim.stage_kernels() == "carry"
    cons_host = sim.get_state()

    for _ in range(args.warmup):
        sim.step()
    torch.cuda.synchronize()

    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    regions = []
    for _ in range(REGIONS):
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("timed")   # lets a profiler select the timed cycles
        e0.record(stream)
        for _ in range(args.steps):
            sim.step()
        e1.record(stream)
        e1.synchronize()
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        regions.append(max_over_ranks(e0.elapsed_time(e1), dist))
    clk = clocks.stop()
    # the pipe-rate probe runs with the GPU hot from the timed cycles: the first probe of a
    # process read ~6 % low while the clocks were still coming up from idle
    rates = idx.pipe_rates()
    sim.time()  # surfaces any device error of the timed cycles
    ms = statistics.median(regions)
    value = aggregate_rate(ncell, args.steps, world, ms)
    n_active = sum(1 for s in ic.shape if s > 1)
    # k_begin, k_end, and per stage: prims, the sweeps, E^c, update (fused: prims + one kernel;
    # carry: no prims kernel, the update recovers the next stage's primitives)
    launches_per_cycle = 2 + 2 * (2 if fused else (2 if carry else 3) + n_active)

    # op counts from the oracle's pinned counter on a 32^3 corner of the box's state
    sample = ([np.ascontiguousarray(a[:32, :32, :32]) for a in cons_host] if args.n > 32
              else cons_host)
    counts = op_counts(sample, (32 / args.n,) * 3 if args.n > 32 else ic.lengths, ic.gamma)

    # dominant kernel: per-launch device time of each kernel (events between launches)
    kt = sim.kernel_times(reps=2)
    shapes = sim.sweep_shapes()
    sweep_ms = {d: kt[f"sweep_{d}"] for d in "xyz"}
    dom = max(sweep_ms, key=sweep_ms.get)
    d_i = "xyz".index(dom)
    achieved_gflops = counts["face_flops"][d_i] * ncell / (sweep_ms[dom] * 1e-3) / 1e9
    kname = f"k_sweep<{'double' if args.precision == 'fp64' else 'float'},{dom}>"
    dom_ms, dom_flops = sweep_ms[dom], counts["face_flops"][d_i]
    if fused:
        # one kernel does a stage's faces, edges and update: its share of a cycle's count
        # is all of it but the primitive recovery, over the two stages
        dom_ms = kt["update"]
        dom_flops = (counts["cycle_flops"] - counts["parts"]["prims"]) / 2
        achieved_gflops = dom_flops * ncell / (dom_ms * 1e-3) / 1e9
        kname = "k_stage_fused<float>"
    fma = rates["fma64"] if args.precision == "fp64" else rates["fma32"]
    peak = 2 * fma / 1e9
    tpf = MEASURED_TRAFFIC_PER_FACE.get((args.precision, dom, shapes["xyz".index(dom)]))
    whole = roofline_cycle(value, counts, rates, hbm_gbs, args.precision)
    roofline = {"bound": "alu", "kernel": kname,
                "achieved": achieved_gflops, "peak": peak, "unit": "GFLOP/s",
                "frac": achieved_gflops / peak,
                "frac_of_nominal_fp64": (achieved_gflops / FP64_NOMINAL_GFLOPS
                                         if args.precision == "fp64" else None),
                "traffic": tpf * ncell if (tpf and not fused) else None,
                "traffic_unit": "bytes per launch",
                "alg_flops_per_unit": dom_flops, "launch_ms": dom_ms,
                "peak_source": (f"measured {'FP64' if args.precision == 'fp64' else 'FP32'} FMA "
                                "rate x 2 flop (idx_pipe_rates, this GPU; of measured)"),
                "kernel_ms": kt, "sweep_shapes_xyz": shapes,
                "pipe_rates_gops": {k: v / 1e9 for k, v in rates.items()},
                "whole_cycle": whole, "op_counts": counts, "hbm_gbs": hbm_gbs,
                "hbm_source": hbm_source}

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
    el_serial = max_over_ranks(time.perf_counter() - t0, dist)
    # a stream of independent states through two sims on their own streams: step k's
    # upload and speed pass run beside step k-1's cycle, its download beside step k+1's
    stream2 = torch.cuda.Stream()
    sim2 = idx.Sim(ic.shape, ic.lengths, ic.gamma, 0.4, args.precision, stream=stream2.cuda_stream)
    sim2.set_stage_kernels(args.stage_kernels)
    if args.sweep_shapes:
        sim2.set_sweep_shapes(tuple(int(v) for v in args.sweep_shapes.split(",")))
    pair = (sim, sim2)
    for s_ in pair:
        s_.set_state(pinned)
        s_.step()
        s_.get_state(out=out_pinned)
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    pair[0].set_state(pinned)
    pair[0].step()
    for k in range(1, e2e_steps):
        pair[k % 2].set_state(pinned)
        pair[k % 2].step()
        pair[(k - 1) % 2].get_state(out=out_pinned)
    pair[(e2e_steps - 1) % 2].get_state(out=out_pinned)
    el = max_over_ranks(time.perf_counter() - t0, dist)
    e2e = {"value": aggregate_rate(ncell, e2e_steps, world, el * 1e3), "unit": UNIT,
           "h2d_bytes_per_step": 8 * 8 * ncell, "d2h_bytes_per_step": 8 * 8 * ncell,
           "note": "per step: idx_set_state from pinned host (incl. its signal-speed pass), "
                   "idx_step, idx_get_state to pinned host; two sims on their own streams "
                   "alternate, so a step's copies run beside the neighbouring steps' cycles",
           "serial_value": aggregate_rate(ncell, e2e_steps, world, el_serial * 1e3),
           "serial_note": "one sim, each step's upload, cycle and download in turn"}
    sim2.close()
    sim.close()
    del pinned, out_pinned

    def time_variant(precision, ic_v=None, steps=None, warmup=None, stage=None, kernels=False,
                     **kw):
        # another configuration (same box unless given), same timing rules, one region
        ic_v = ic if ic_v is None else ic_v
        steps = args.steps if steps is None else steps
        warmup = args.warmup if warmup is None else warmup
        sv = idx.Sim(ic_v.shape, ic_v.lengths, ic_v.gamma, 0.4, precision,
                     stream=stream.cuda_stream, **kw)
        sv.set_primitive(ic_v.prim)
        if stage:
            sv.set_stage_kernels(stage)
        for _ in range(warmup):
            sv.step()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            sv.step()
        e1.record(stream)
        e1.synchronize()
        msv = max_over_ranks(e0.elapsed_time(e1), dist)
        sv.time()
        out = {"value": aggregate_rate(ic_v.ncells, steps, world, msv), "unit": UNIT,
               "ms_per_step": msv / steps, "steps": steps,
               "sweep_shapes_xyz": sv.sweep_shapes(), "stage_kernels": sv.stage_kernels()}
        if kernels:
            out["kernel_ms"] = sv.kernel_times(reps=2)
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

    def with_roofline(v, precision, cnt):
        if "value" in v:
            v["roofline"] = roofline_cycle(v["value"], cnt, rates, hbm_gbs, precision)
        return v

    variants = {}
    if args.precision == "fp64" and not args.no_variants:
        variants["fp32_bulk"] = with_roofline(guarded(time_variant, "fp32", kernels=True),
                                              "fp32", counts)
        # the six kernels per stage (primitive recovery a kernel of its own), for comparison
        variants["fp32_bulk_split"] = with_roofline(
            guarded(time_variant, "fp32", stage="split", kernels=True), "fp32", counts)
        # the 512^3 box: the FP32-bulk configuration, and FP64 beside it
        ic512 = inputs.turbulent_box(512, seed=0)
        variants["fp32_bulk_512"] = with_roofline(guarded(time_variant, "fp32", ic512),
                                                  "fp32", counts)
        variants["fp64_512"] = with_roofline(guarded(time_variant, "fp64", ic512, steps=5,
                                                     warmup=2), "fp64", counts)
        del ic512
        # the small 2D problem of the paper's Orszag-Tang test, whole run: launch-bound
        ot2 = inputs.orszag_tang_2d(128)
        for prec in ("fp64", "fp32"):
            key = f"{prec}_orszag_tang_2d_128_to_t0.5"
            variants[key] = guarded(time_advance, prec, ot2, 0.5)
            variants[key]["note"] = ("2D Orszag-Tang 128^2 to t = 0.5 through idx_advance (16384 cells: "
                                     "launch-bound, one CUDA graph per cycle)")
        variants["fp64_vector_potential"] = guarded(time_variant, "fp64", induction="potential")
        variants["fp64_vector_potential"]["note"] = "Eqs. 7-8: edge potential stepped, B = Bref + curl A"
        variants["fp64_rk3"] = guarded(time_variant, "fp64", rk_order=3)
        variants["fp64_rk3"]["note"] = "RK3 (Table 1): three stages per cycle instead of two"
        variants["fp64_limo3"] = guarded(time_variant, "fp64", recon="limo3")
        variants["fp64_limo3"]["note"] = "LimO3 reconstruction (Sec. 2.3) instead of van Leer PLM"
        variants["fp64_limo3_rk3"] = guarded(time_variant, "fp64", recon="limo3", rk_order=3)
        variants["fp64_limo3_rk3"]["note"] = "LimO3 + RK3, the paper's higher-accuracy pairing"
        # the paper's own performance problem (Sec. 5): 3D Orszag-Tang, FP64, at this box size
        ot = inputs.orszag_tang_3d(args.n)
        variants["fp64_orszag_tang_3d"] = guarded(time_variant, "fp64", ot)
        variants["fp64_orszag_tang_3d"]["note"] = (
            f"3D Orszag-Tang {args.n}^3 (Sec. 5 performance problem); the paper reports ~121 Mcell/s "
            "per V100 at 256^3 per GPU (4-GPU node, 484 Mcell/s): context, another machine")
        if world == 1:
            # batched mix (C4) and the served stream (C5 reading), single GPU
            ics = c4_instances()
            variants["batched_mix"] = {
                "workload": C4_WORKLOAD, "cycles_per_instance": args.cycles,
                "cells": sum(x.ncells for x in ics),
                "fp64": guarded(batched_mix, ics, "fp64", args.cycles, args.warmup),
                "fp32": guarded(batched_mix, ics, "fp32", args.cycles, args.warmup)}
            del ics
            from paper_2304_13746_b300 import serve
            budget = int(args.budget_gb * 1e9)
            variants["served"] = {"workload": C5_WORKLOAD, "budget_bytes": budget}
            for prec, nreq in (("fp32", args.serve_requests_fp32),
                               ("fp64", args.serve_requests_fp64)):
                if nreq > 0:
                    variants["served"][prec] = guarded(served_stream, prec, nreq, budget, serve,
                                                       stream.cuda_stream)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64" if args.precision == "fp64" else "f32/f64",
                "data": "synthetic", "config": workload_config(args),
                "regions_ms": regions,
                "spread": (max(regions) - min(regions)) / ms,
                "gpu_launches": launches_per_cycle * args.steps * REGIONS,
                "clocks": clk, "roofline": roofline,
                "whole_cycle_frac": whole["frac"], "e2e": e2e, "variants": variants}
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline()
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
