"""bench.py's host-side contract, on the CPU: the reference arm's JSON line,
silence of ranks other than 0, and the replica timing reduction over two gloo
ranks (the path `bench.py --gpus N` takes under torchrun)."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
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


def test_minimum_bytes_and_flops_match_hand_computed_values():
    """The local-SpMM byte count of Section 4 at p = 1 (CSR read once, B read
    once, C written once) and 2*nnz*N flops, against values worked out by hand
    for the R-MAT scale-22 workload (nnz 65,245,304, N = 128) and its N = 256
    storage variants with FP16 values."""
    M = K = 4194304
    nnz = 65245304
    # 4(M+1) + 8 nnz + 4 K N + 4 M N = 16,777,220 + 521,962,432 + 2 * 2,147,483,648
    assert bench.min_bytes(M, K, 128, nnz) == 4833706948
    assert 2.0 * nnz * 128 == 16702797824.0
    # FP16 values (2 bytes), N = 256; CSR part 16,777,220 + 6 nnz = 408,249,044 and
    # C = 4,294,967,296.  B in FP32 / BF16 / E4M3 is 4,294,967,296 / 2,147,483,648 /
    # 1,073,741,824 bytes, E4M3 plus 16,777,216 bytes of row scales.
    assert bench.min_bytes(M, K, 256, nnz, w_val=2, w_b=4) == 8998183636
    assert bench.min_bytes(M, K, 256, nnz, w_val=2, w_b=2) == 6850699988
    assert bench.min_bytes(M, K, 256, nnz, w_val=2, w_b=1) + 4 * K == 5793735380


def test_tile_imbalance_is_max_over_mean_of_row_blocks():
    rowptr = torch.tensor([0, 5, 5, 6, 6, 6, 10, 10, 12], dtype=torch.int32)   # M = 8
    # 4 row blocks of 2 rows: 5, 1, 4, 2 nonzeros -> max 5 / mean 3
    assert abs(bench.tile_nnz_imbalance(rowptr, 8, 4) - 5 / 3) < 1e-12
    # ragged: 3 blocks of ceil(8/3) = 3 rows: 6, 4, 2 -> 6 / 4
    assert abs(bench.tile_nnz_imbalance(rowptr, 8, 3) - 1.5) < 1e-12
    assert bench.tile_nnz_imbalance(torch.zeros(9, dtype=torch.int32), 8, 4) == 1.0


def test_trace_summary_of_hand_made_records():
    from paper_2311_18141_gb300 import binding
    rec = np.zeros(3, dtype=binding.TRACE_DTYPE)
    rec["t_start_ns"] = [10, 10, 20]
    rec["t_end_ns"] = [110, 60, 120]
    rec["units"] = [4, 2, 6]
    rec["stolen"] = [1, 0, 2]
    t = bench.trace_summary(rec)
    assert t["warps"] == 3 and t["launch_us"] == 0.11
    assert abs(t["busy_max_over_avg"] - 100 / (250 / 3)) < 1e-12      # busy 100, 50, 100
    assert abs(t["finish_spread_us"] - 0.06) < 1e-12
    assert abs(t["idle_share"] - (1 - 250 / 330)) < 1e-12
    assert abs(t["units_per_warp_max_over_avg"] - 1.5) < 1e-12
    assert abs(t["stolen_share"] - 0.25) < 1e-12
    assert bench.trace_summary(rec[:0]) is None


def test_clock_summary_of_hand_made_samples():
    """Median SM clock under load, the maximum, and every throttle reason seen
    Active in any sample (the fields a run is accepted or rejected on)."""
    s = bench.ClockSampler("0")
    row = "0, {sm}, 2070, 900.0, 0x0, {hw}, Not Active, Not Active, {pc}"
    s.out = [row.format(sm=sm, hw=hw, pc=pc).split(",")
             for sm, hw, pc in [(2070, "Not Active", "Not Active"),
                                (1980, "Not Active", "Active"),
                                (2070, "Not Active", "Not Active")]]
    c = s.summary()
    assert c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0 and c["samples"] == 3
    assert c["reasons"] == ["sw_power_cap"]
    s.out[0][5] = " Active"
    assert bench.ClockSampler.summary(s)["reasons"] == ["hw_slowdown", "sw_power_cap"]
    assert bench.ClockSampler("0").summary()["reasons"] == ["no samples"]
