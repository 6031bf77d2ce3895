"""bench.py's host-side contract, on the CPU: the reference arm's JSON line,
silence of ranks other than 0, and the replica timing reduction over two gloo
ranks (the path `bench.py --gpus N` takes under torchrun)."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

REQUIRED = {"impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
            "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
            "cpu_baseline", "e2e"}


def _run_bench(extra_env, *args):
    env = dict(os.environ, **extra_env)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args],
                          capture_output=True, text=True, env=env, timeout=600)


def test_reference_arm_prints_one_contract_line():
    r = _run_bench({}, "--impl", "reference", "--scale", "10", "--steps", "1", "--warmup", "1",
                   "--cpu-seconds", "0.3")
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert REQUIRED <= set(d)
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "GFLOP/s"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"] == "rmat-s10-ef16-n128-fp32-grid16x4"


def test_reference_arm_other_ranks_are_silent():
    r = _run_bench({"RANK": "1", "WORLD_SIZE": "2"}, "--impl", "reference", "--scale", "10",
                   "--steps", "1", "--warmup", "1")
    assert r.returncode == 0, r.stderr[-2000:]
    assert not [l for l in r.stdout.splitlines() if l.startswith("{")]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, local_ms, out):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        ms, value = bench.job_throughput(local_ms[rank], 4, 1e9, world, "cpu")
        out[rank] = (ms, value)
    finally:
        dist.destroy_process_group()


def test_replica_timing_takes_the_slowest_rank_gloo():
    world = 2
    local_ms = [8.0, 12.0]   # total over 4 steps on each rank
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, _free_port(), local_ms, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        ms, value = res[rank]
        assert ms == pytest.approx(3.0)                     # max(8, 12) / 4 steps
        assert value == pytest.approx(2 * 1e9 / 3e-3 / 1e9)  # both ranks' work / max time


def test_single_rank_throughput_needs_no_process_group():
    ms, value = bench.job_throughput(10.0, 5, 4e9, 1, "cpu")
    assert ms == pytest.approx(2.0)
    assert value == pytest.approx(4e9 / 2e-3 / 1e9)
