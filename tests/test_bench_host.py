"""Host-side checks of bench.py (no GPU): the multi-rank timing path on 2 gloo ranks and the
reference arm (the CPU oracle) on the small configuration."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        bench.barrier(world)
        q.put((rank, bench.dist_max(1.5 + rank, world)))
        bench.barrier(world)
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_on_two_gloo_ranks():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=5) for _ in range(2))
    assert got == [(0, 2.5), (1, 2.5)]  # every rank sees the slowest rank's time


def test_reference_arm_small_config():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "small", "--steps", "1",
                          "--warmup", "0"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "GTEPS"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0
    # the same keys as the GPU arm's line, so that the two lines compare one to one
    for key in ("metric", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling", "dtype", "data"):
        assert key in d, key
    assert set(d["config"]) == {"workload", "n", "nnz", "d_max", "alpha", "epsilon", "L", "k", "parallelism", "l2"}
    assert d["ms_per_step"] > 0 and d["config"]["L"] == 34


def test_reference_arm_declines_sampled_and_adaptive_workloads():
    for wl in ("rmat_s", "rmat_a", "batch"):
        out = subprocess.run([sys.executable, "-c", "import sys, bench; sys.argv=['bench.py','--impl','reference',"
                              f"'--workload','{wl}']; import json; a=bench.parse(); print(json.dumps(bench.run_reference(a)))"],
                             cwd=ROOT, capture_output=True, text=True, timeout=120)
        assert out.returncode == 0, out.stderr
        d = json.loads(out.stdout.strip().splitlines()[-1])
        assert d["impl"] == "reference" and "unavailable" in d


def test_l2_note():
    import importlib

    sys.path.insert(0, ROOT)
    bench = importlib.import_module("bench")
    assert bench.l2_note(4_194_304, 128_309_616).startswith("inputs larger than L2")
    assert bench.l2_note(1000, 10_206).startswith("inputs fit in L2")


def test_reference_arm_other_ranks_print_nothing():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "small", "--steps", "1",
                          "--warmup", "0"], cwd=ROOT, capture_output=True, text=True, timeout=300, env=env)
    assert out.returncode == 0, out.stderr
    assert out.stdout.strip() == ""


def test_roofline_fields_from_profiler_counters():
    # the dominant kernel's algorithmic bytes over its measured time, against the measured peak;
    # DRAM GB/s only when a committed ncu summary matches the kernel and its source hash
    import importlib

    sys.path.insert(0, ROOT)
    bench = importlib.import_module("bench")
    prof = {"top_ms": 600.0, "top_bytes": 866_084_292 * 1000, "top_launches": 1000, "sweep_bytes": 1e12,
            "sweep_ms": 700.0, "sweep_launches": 1200, "top_fp64": 0, "top_cols": 8, "top_mode": 5}
    r = bench.roofline(prof, "rmat22")
    assert r["unit"] == "GB/s" and r["bound"] == "hbm"
    assert abs(r["achieved"] - 866_084_292 / 600e-6 / 1e9) < 0.1
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-4
    assert r["kernel"].startswith("sweep_kernel<float, 8, 5>")
    if r["traffic"] is not None:
        assert abs(r["dram_gbs"] - r["traffic"] / 600e-6 / 1e9) < 0.1
    assert bench.roofline(dict(prof, top_mode=4), "rmat22")["traffic"] is None  # no summary for that kernel
