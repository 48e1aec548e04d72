"""The multi-rank host logic of bench.py on CPU with gloo, world size 2: the timed region's
max over ranks and the whole-job aggregate; and the reference arm under torchrun (rank 0
alone prints one JSON line, the other rank exits 0 without work)."""
import json
import os
import subprocess
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 10.0 * (rank + 1)                       # rank 1 is the slow one
        m = bench.max_over_ranks(ms, dist)
        rate = bench.aggregate_rate(1000, 5, world, m)
        dist.barrier()
        out.put((rank, m, rate))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_aggregate_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, m, rate in res:
        assert m == 20.0                              # the slowest rank's time on every rank
        assert rate == pytest.approx(1000 * 5 * 2 / 0.020)


def test_single_rank_identity():
    assert bench.max_over_ranks(3.5, None) == 3.5
    assert bench.aggregate_rate(10, 2, 1, 1000.0) == pytest.approx(20.0)


def test_reference_arm_under_torchrun_two_ranks():
    port = 30500 + os.getpid() % 1000
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py",
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["reference_sample"]["cells_per_step"] == bench.REFERENCE_SAMPLE_N ** 3
    assert d["config"] == bench.workload_config(bench.parse_args_for_test())


def test_roofline_of_a_cycle_picks_the_slowest_bound():
    rates = {"fma64": 500e9, "fma32": 32e12}
    counts = {"cycle_flops": 3000.0, "fp64_island_flops": 100.0}
    # FP64: 3000 flop at 1 TFLOP/s = 3 ns against 320 B at 6.4 TB/s = 0.05 ns
    r = bench.roofline_cycle(1e8, counts, rates, 6400.0, "fp64")
    assert r["bound"] == "fp64"
    assert r["ns_per_cell_update"]["fp64"] == pytest.approx(3.0)
    assert r["frac"] == pytest.approx(1e8 * 3e-9)
    # FP32 bulk: islands 100 flop at 1 TFLOP/s = 0.1 ns, 2900 flop at 64 TFLOP/s = 0.045 ns,
    # HBM 0.05 ns: the FP64 islands bind
    r = bench.roofline_cycle(5e9, counts, rates, 6400.0, "fp32")
    assert r["bound"] == "fp64"
    assert r["ns_per_cell_update"]["fp32"] == pytest.approx(2900 / 64e12 * 1e9)
    assert r["ns_per_cell_update"]["hbm"] == pytest.approx(320 / 6400e9 * 1e9)
    assert r["frac"] == pytest.approx(5e9 * 0.1e-9)
