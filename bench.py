#!/usr/bin/env python3
"""Benchmark of the local CSR SpMM C = A*B on one GB300 (replicas on N GPUs).

Workload (the power-law FP32 SpMM): A is an R-MAT graph of scale 22
(4,194,304 rows and columns), edge factor 16, (a,b,c,d) = (0.57,0.19,0.19,0.05),
duplicates merged, self-loops kept, values uniform (0,1] in FP32; B is
4,194,304 x 128 FP32 N(0,1); a 16 x 4 tile grid (16 C row blocks x 4 column
blocks of 32) is pulled by the persistent work-stealing kernel.  Inputs are
synthetic and seeded, and larger than L2.

One step = one spmm_csr call: the work counter's reset, the persistent product
kernel and the split-row sum kernel (which adds the pieces of rows that chunk
boundaries cut).
`value` is GFLOP/s = 2*nnz*N / step time over all ranks (N>1 runs independent
replicas: the path has no exchange step, so there is no collective).

--impl reference times the FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SpMM GFLOP/s (2·nnz·N) and % HBM roofline; BF16 vs FP32 at stated error"
WORKLOAD = "rmat-s22-ef16-n128-fp32-grid16x4"
NOMINAL_HBM_GBS = 7900.0   # GB300 HBM3e nominal bandwidth, for the second roofline fraction
FALLBACK_HBM_GBS = 6800.0
PROFILE = os.path.join(ROOT, "profiles", "spmm_csr_persistent_rmat_s22_n128.md")
KERNEL_SOURCES = ["common.cuh", "schedule.cuh", "spmm_kernel.cuh", "launch.cuh",
                  "spmm_launch_impl.cuh", "spmm_f32_f32.cu", "plan.cu", "fixup.cu"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--scale", type=int, default=22, help="R-MAT scale (22 = the workload)")
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--grid", default="16x4")
    ap.add_argument("--chunk", type=int, default=0)
    ap.add_argument("--warps", type=int, default=0,
                    help="spmm_tuning.warps_per_cta: 0 library default (7 or 8), 1 to 8")
    ap.add_argument("--order", type=int, default=16,
                    help="spmm_tuning.tile_order (16: one queue per tile row, chunks of its "
                         "tiles handed out in turn)")
    ap.add_argument("--kernel", type=int, default=0,
                    help="spmm_tuning.kernel: 0 library default, 1 staged 16-byte kernel, "
                         "2 32-byte-lane kernel, 3 warp-specialised staged kernel")
    ap.add_argument("--ksplit", type=int, default=0,
                    help="gather workload: also time the gathers in the orders of a K-split "
                         "3D grid with this many k-blocks")
    ap.add_argument("--lanes", type=int, default=0,
                    help="spmm_tuning.lanes_per_item: 0 default, 2 or 4 lanes per column "
                         "block of 4 or 8 vectors")
    ap.add_argument("--e2e-steps", type=int, default=12)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the precision (FP32/BF16/E4M3 B) and small-workload objects")
    ap.add_argument("--context", action="store_true",
                    help="also time torch.sparse.mm (cuSPARSE) on the same product, as context")
    ap.add_argument("--batch-count", type=int, default=512)
    ap.add_argument("--spgemm-scale", type=int, default=14,
                    help="R-MAT scale of the A*A SpGEMM workload")
    ap.add_argument("--workload", default="rmat",
                    choices=["rmat", "precision", "gcn", "batch", "spgemm", "loadsim", "gather",
                             "ksplit"],
                    help="rmat: the benchmark line; the others report the precision, "
                         "backward and batched forms")
    return ap.parse_args()


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2311_18141_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def stored_traffic(src_hash: str):
    """dram read+write bytes per launch from the committed ncu summary, if it was
    taken on the current kernel source."""
    try:
        text = open(PROFILE).read()
    except OSError:
        return None
    m_hash = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", text)
    m_traffic = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", text)
    if not m_hash or not m_traffic or m_hash.group(1) != src_hash:
        return None
    return float(m_traffic.group(1))


def kernel_name(N, TC, esz=4, kernel=0, tag="TagF32", lanes=0):
    """The persistent kernel the library launches for FP32 A and B of element
    size `esz` (aligned torch tensors, dense strides): the staged kernel by
    default, the 32-byte-lane kernel when asked for (kernel 2) and a column
    block is 2..32 whole 32-byte vectors, the warp-specialised kernel when
    asked for (kernel 3) and a block is 8..32 16-byte vectors."""
    epv = 16 // esz
    w = -(-N // TC)
    w = -(-w // epv) * epv
    nb = w * esz
    if kernel == 2 and nb % 32 == 0 and (N * esz) % 32 == 0 and 2 <= nb // 32 <= 32:
        lpn = 2
        while lpn < nb // 32:
            lpn *= 2
        return f"spmm_csr_wide<TagF32,{tag},{lpn},1>"
    nvec = nb // 16
    if nvec <= 32:
        lpn = 2
        while lpn < nvec:
            lpn *= 2
        if lanes in (2, 4) and nvec in (4, 8) and lpn == nvec and lanes < nvec and nvec // lanes <= 4:
            return f"spmm_csr_persistent<TagF32,{tag},{lanes},{nvec // lanes}>"
        if kernel == 3 and lpn >= 8:
            return f"spmm_csr_spec<TagF32,{tag},{lpn},1>"
        return f"spmm_csr_persistent<TagF32,{tag},{lpn},1>"
    return f"spmm_csr_persistent<TagF32,{tag},32,{2 if nvec <= 64 else 4}>"


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.out = []
        self.t0 = self.t1 = None

    def start(self):
        """Start sampling and wait for the first sample, so that nvidia-smi's
        own start-up is over before the timed region begins."""
        import threading
        try:
            sel = [f"--id={self.index}"] if self.index else []
            self.proc = subprocess.Popen(
                ["nvidia-smi", *sel, f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.lines = []
        first = threading.Event()

        def reader():
            for line in self.proc.stdout:
                self.lines.append(line)
                first.set()
        self.thread = threading.Thread(target=reader, daemon=True)
        self.thread.start()
        first.wait(timeout=10.0)
        time.sleep(0.3)
        self.skip = len(self.lines)   # samples taken before the timed region

    def stop(self):
        if self.proc is None:
            return
        timed = self.lines[self.skip:]
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        use = timed if timed else self.lines
        self.out = [l.split(",") for l in use if l.count(",") >= 8]

    def summary(self):
        if not self.out:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = sorted(float(r[1]) for r in self.out)
        mx = max(float(r[2]) for r in self.out)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.out for k in range(4)
                          if r[5 + k].strip().lower() == "active"})
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(sm)}


def make_workload(scale, n, device):
    from paper_2311_18141_gb300 import inputs
    A = inputs.rmat_csr(scale, 16, 0.57, 0.19, 0.19, seed=1, device=device, values="pos")
    B = inputs.dense_normal(A.K, n, seed=2, device=device)
    return A, B


def min_bytes(M, K, N, nnz, w_val=4, w_b=4, w_c=4):
    """Local SpMM bytes of Section 4 at p = 1: CSR (rowptr, colind, vals), B, C once."""
    return 4 * (M + 1) + nnz * (4 + w_val) + K * N * w_b + M * N * w_c


def tile_nnz_imbalance(rowptr, M: int, TR: int) -> float:
    """max/avg nonzeros per tile of a TR x TC grid (the load-imbalance figure of
    the evaluation, Section 6): every column block of a row block holds the
    row block's nonzeros, so the ratio is the one over row blocks."""
    rb = -(-M // TR)
    cuts = [min(i * rb, M) for i in range(TR + 1)]
    rp = rowptr.cpu() if hasattr(rowptr, "cpu") else rowptr
    per = [int(rp[cuts[i + 1]]) - int(rp[cuts[i]]) for i in range(TR)]
    avg = sum(per) / TR
    return max(per) / avg if avg > 0 else 1.0


def trace_summary(rec) -> dict | None:
    """Load balance of one traced launch from its per-warp records: busy time
    max/avg over warps, the spread of finish times (idle tail), the idle share
    of warp time within the launch, units per warp and the stolen share."""
    if rec is None or rec.size == 0:
        return None
    busy = (rec["t_end_ns"] - rec["t_start_ns"]).astype(np.float64)
    span = float(rec["t_end_ns"].max() - rec["t_start_ns"].min())
    units = rec["units"].astype(np.float64)
    return {"warps": int(rec.size), "launch_us": span / 1e3,
            "busy_max_over_avg": float(busy.max() / busy.mean()),
            "finish_spread_us": float(rec["t_end_ns"].max() - rec["t_end_ns"].min()) / 1e3,
            "idle_share": float(1.0 - busy.sum() / (rec.size * span)) if span > 0 else 0.0,
            "units_per_warp_max_over_avg": float(units.max() / units.mean()),
            "stolen_share": float(rec["stolen"].sum() / max(1.0, units.sum()))}


def _host_operands(A, B):
    """A's CSR arrays and B as host numpy arrays (copied once)."""
    return (A.rowptr.cpu().numpy(), A.colind.cpu().numpy(), A.vals.cpu().numpy(),
            B.cpu().numpy())


def _oracle_stride(host, M: int, seconds: float) -> int:
    """Row stride whose oracle sample takes about `seconds` (at least a quarter
    of it), found by growing the sample 4x at a time; 1 = every row."""
    import oracle
    rp, ci, v, Bh = host
    stride = 4096
    while stride > 1:
        rows = np.arange(0, M, stride, dtype=np.int64)
        t = time.perf_counter()
        oracle.spmm_rows(rp, ci, v, Bh, rows)
        if time.perf_counter() - t >= seconds / 4:
            break
        stride //= 4
    return max(stride, 1)


def _oracle_timed(host, M: int, stride: int, seconds: float):
    """One timed oracle sample at `stride` (whole passes repeated while a
    stride-1 pass is shorter than `seconds`): (GFLOP/s, threads, description,
    seconds spent)."""
    import oracle
    rp, ci, v, Bh = host
    N = Bh.shape[1]
    lens = np.diff(rp.astype(np.int64))
    rows = np.arange(0, M, stride, dtype=np.int64)
    flops = 2.0 * float(lens[rows].sum()) * N
    total_t, reps = 0.0, 0
    while reps == 0 or (stride == 1 and total_t < seconds):
        t = time.perf_counter()
        oracle.spmm_rows(rp, ci, v, Bh, rows)
        total_t += time.perf_counter() - t
        reps += 1
    desc = (f"every {stride}-th row of the workload ({rows.size} rows, "
            f"{flops / 2 / N:.0f} nnz) x {reps} pass(es), N={N}, FP64 oracle, "
            f"{total_t:.2f} s")
    return flops * reps / total_t / 1e9, oracle.get_threads(), desc, total_t


def cpu_oracle_sample(A, B, seconds: float):
    """Time the FP64 oracle on a stride sample of rows of about `seconds` of CPU
    work; returns (GFLOP/s, threads, description, seconds spent)."""
    import oracle
    oracle.set_threads(len(os.sched_getaffinity(0)))
    host = _host_operands(A, B)
    return _oracle_timed(host, A.M, _oracle_stride(host, A.M, seconds), seconds)


def job_throughput(local_total_ms: float, steps: int, flops_per_step: float, world: int,
                   device) -> tuple[float, float]:
    """Replicas: every rank runs the same product.  The job's step time is the
    slowest rank's (max over ranks, one all-reduce when world > 1), and its
    throughput counts the work of all ranks: (ms per step, job GFLOP/s)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([local_total_ms], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_step = float(t.item()) / steps
    return ms_step, flops_per_step * world / (ms_step * 1e-3) / 1e9


def workload_label(args, N: int) -> str:
    if (args.scale, N, args.grid) == (22, 128, "16x4"):
        return WORKLOAD
    return f"rmat-s{args.scale}-ef16-n{N}-fp32-grid{args.grid}"


def workload_config(args, M, K, N, nnz) -> dict:
    """The workload both arms run (the same keys and values in each arm's line)."""
    return {"workload": workload_label(args, N), "M": M, "K": K, "N": N, "nnz": nnz,
            "tile_grid": args.grid,
            "l2": "inputs larger than L2 (A+B+C = %.2f GB per step)" % (min_bytes(M, K, N, nnz) / 1e9)}


def run_reference(args):
    """The FP64 oracle on the host cores (rank 0 only)."""
    import torch
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    A, B = make_workload(args.scale, args.n, "cuda" if torch.cuda.is_available() else "cpu")
    oracle.set_threads(len(os.sched_getaffinity(0)))
    host = _host_operands(A, B)
    # every step is one bounded sample, sized so the whole run takes about two minutes
    per_step = max(0.02, min(args.cpu_seconds, 120.0 / max(1, args.steps + args.warmup)))
    stride = _oracle_stride(host, A.M, per_step)
    vals = []
    for _ in range(args.warmup):
        _oracle_timed(host, A.M, stride, per_step)
    desc = cores = None
    for _ in range(args.steps):
        g, cores, desc, _ = _oracle_timed(host, A.M, stride, per_step)
        vals.append(g)
    value = sum(vals) / len(vals)
    flops_step = 2.0 * A.nnz * args.n
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GFLOP/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": flops_step / (value * 1e9) * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args, A.M, A.K, args.n, A.nnz),
        "cpu_baseline": {"value": value, "unit": "GFLOP/s", "cores": cores, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": value, "unit": "GFLOP/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2311_18141_gb300 import binding

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    binding.load_library()
    TR, TC = (int(x) for x in args.grid.split("x"))
    if args.order < 0 or args.order > 31:
        raise SystemExit("--order is 0..31")
    A, B = make_workload(args.scale, args.n, dev)
    M, K, N, nnz = A.M, A.K, args.n, A.nnz
    C = torch.empty(M, N, device=dev)
    tun = binding.make_tuning(chunk_items=args.chunk, warps_per_cta=args.warps,
                              tile_order=args.order, kernel=args.kernel,
                              lanes_per_item=args.lanes)
    plan = binding.Plan(A.rowptr, M, K, nnz, N, TR, TC, tuning=tun)
    ws = binding.workspace(plan.workspace_bytes, dev)
    stream = torch.cuda.current_stream()

    def step():
        binding.spmm_csr(A.rowptr, A.colind, A.vals, B, C, M, K, N, nnz, plan=plan, ws=ws,
                         stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    assert binding.spmm_get_device_status(ws) == 0

    # this rank's GPU as nvidia-smi names it: its entry of CUDA_VISIBLE_DEVICES
    # (an index or a UUID), else its local index
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")
    gpu_id = vis[local].strip() if local < len(vis) and vis[local].strip() else str(local)
    sampler = ClockSampler(gpu_id)
    sampler.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    ev[0].record(stream)
    for k in range(args.steps):
        step()
        ev[k + 1].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    sampler.stop()
    total_ms = ev[0].elapsed_time(ev[-1])
    per_launch = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
    flops = 2.0 * nnz * N
    ms_step, value = job_throughput(total_ms, args.steps, flops, world, dev)

    # roofline of the dominant kernel, the persistent product.  Its duration is
    # taken as the whole step's (the split-row sum after it included), so the
    # fraction is a lower bound on the product kernel's own.
    peak, peak_kind = measured_peaks()
    algo_bytes = min_bytes(M, K, N, nnz)
    launch_ms = sum(per_launch) / len(per_launch)
    achieved = algo_bytes / (launch_ms * 1e-3) / 1e9
    src_hash = kernel_source_hash()
    traffic = stored_traffic(src_hash)

    # one traced launch after the timed region: per-warp busy time, units and
    # steals, the on-chip form of the computation / load-imbalance split
    tbuf = binding.trace_buffer(1 << 16, dev)
    plan.set_trace(tbuf)
    step()
    torch.cuda.synchronize()
    plan.set_trace(None)
    trace = trace_summary(binding.read_trace(tbuf))
    del tbuf

    # end-to-end through the C ABI's host-buffer pipeline (spmm_host_pipe_*):
    # every step copies A and B from pinned host memory to the device,
    # multiplies, and copies C back into host memory, all inside the timed
    # region.  depth 1 runs the steps one after the other; depth d keeps d
    # device slots, so the uploads of the next steps and the downloads of the
    # previous ones overlap the current step's product.
    e2e = None
    if rank == 0 or world > 1:
        rp_h = A.rowptr.cpu().pin_memory()
        ci_h = A.colind.cpu().pin_memory()
        v_h = A.vals.cpu().pin_memory()
        B_h = B.cpu().pin_memory()
        C_hs = [torch.empty(M, N).pin_memory() for _ in range(3)]
        h2d = sum(t.numel() * t.element_size() for t in (rp_h, ci_h, v_h, B_h))
        d2h = C_hs[0].numel() * C_hs[0].element_size()
        assert binding.spmm_get_device_status(ws) == 0
        del C, ws
        n_e2e = max(1, args.e2e_steps)

        def pipe_ms(depth):
            pipe = binding.HostPipe(plan, A.vals.dtype, B.dtype, depth=depth, stream=stream)
            pipe.submit(rp_h, ci_h, v_h, B_h, C_hs[0])   # warm-up step
            pipe.wait()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for k in range(n_e2e):
                pipe.submit(rp_h, ci_h, v_h, B_h, C_hs[k % len(C_hs)])
            pipe.wait()
            ms = (time.perf_counter() - t0) * 1e3 / n_e2e
            pipe.close()
            return ms

        depths = (1, 2, 3)
        by_depth = [pipe_ms(d) for d in depths]
        if world > 1:   # the job's step time is the slowest rank's
            t = torch.tensor(by_depth, dtype=torch.float64, device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            by_depth = [float(x) for x in t]
        # every depth is the same public call; how well the copies of
        # consecutive steps overlap on the host link varies from machine to
        # machine, so the pipeline depth is chosen by timing, like a tuning knob
        k_best = min(range(len(depths)), key=lambda k: by_depth[k])
        depth, best_ms = depths[k_best], by_depth[k_best]
        e2e = {"value": flops * world / (best_ms * 1e-3) / 1e9, "unit": "GFLOP/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": best_ms,
               "steps": n_e2e, "pipelined": depth > 1, "api": f"spmm_host_pipe (depth {depth})",
               "ms_per_step_by_depth": {str(d): ms for d, ms in zip(depths, by_depth)}}
        del rp_h, ci_h, v_h, B_h, C_hs

    # optional context: the paper's own local kernel, cuSPARSE SpMM (through
    # torch.sparse.mm), on the same A and B; not a target and not a backend
    context = None
    if args.context and rank == 0:
        At = torch.sparse_csr_tensor(A.rowptr, A.colind, A.vals, size=(M, K))
        for _ in range(3):
            torch.sparse.mm(At, B)
        torch.cuda.synchronize()
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n_ctx = 10
        c0.record(stream)
        for _ in range(n_ctx):
            torch.sparse.mm(At, B)
        c1.record(stream)
        torch.cuda.synchronize()
        ctx_ms = c0.elapsed_time(c1) / n_ctx
        context = {"torch_sparse_mm_ms": ctx_ms, "torch_sparse_mm_gflops": flops / (ctx_ms * 1e-3) / 1e9,
                   "what": "cuSPARSE SpMM through torch.sparse.mm on the same A and B (context only)"}
        del At

    # the metric's second half (BF16 vs FP32 at stated error) and the small
    # workload, measured in the same run on rank 0
    precision = small = None
    if rank == 0 and not args.no_forms:
        del B
        torch.cuda.empty_cache()
        precision = precision_results(A, dev, args.grid, max(5, min(args.steps, 20)),
                                      max(3, args.warmup), warps=args.warps)
        small = small_results(dev, warps=args.warps)
        B = None

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        if B is None:
            from paper_2311_18141_gb300 import inputs
            B = inputs.dense_normal(A.K, args.n, seed=2, device=dev)
        g, cores, desc, _ = cpu_oracle_sample(A, B, args.cpu_seconds)
        cpu = {"value": g, "unit": "GFLOP/s", "cores": cores, "kind": "oracle", "sample": desc}

    chunks, units = plan.units()
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": workload_config(args, M, K, N, nnz),
            "parallelism": f"replicas x{world}" if world > 1 else "1 gpu",
            "plan": {"chunks": chunks, "work_units": units, "tile_order": args.order,
                     "tile_nnz_max_over_avg": tile_nnz_imbalance(A.rowptr, M, TR)},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "nominal_peak": NOMINAL_HBM_GBS, "frac_of_nominal": achieved / NOMINAL_HBM_GBS,
                         "peak_source": f"{peak_kind} (copy bandwidth)",
                         "algorithmic_bytes_per_launch": algo_bytes,
                         "kernel": kernel_name(N, TC, kernel=args.kernel, lanes=args.lanes),
                         "launch_ms": launch_ms, "launch_ms_min": min(per_launch),
                         "launch_ms_max": max(per_launch), "kernel_source_sha256_16": src_hash},
            "cpu_baseline": cpu,
            "e2e": e2e,
            # per step: the persistent product and the split-row sum
            "gpu_launches": 2 * args.steps,
            "context": context,
            "precision": precision,
            "small": small,
            "trace": trace,
            "clocks": sampler.summary(),
        }
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        dist.destroy_process_group()


def _time_ms(fn, steps, warmup, stream):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def sample_rows(rowptr, n_random: int, seed: int):
    """Rows the error report samples: the 32 heaviest (split across many work
    units), up to 256 empty ones, up to 512 of 17..1999 nonzeros, n_random
    random rows, and the first/last rows and row-block edges."""
    lens = np.diff(rowptr.astype(np.int64))
    M = lens.size
    rng = np.random.default_rng(seed)
    heavy = np.argsort(lens)[-32:]
    empty = np.flatnonzero(lens == 0)
    empty = rng.choice(empty, min(256, empty.size), replace=False) if empty.size else empty
    mid = np.flatnonzero((lens > 16) & (lens < 2000))
    mid = rng.choice(mid, min(512, mid.size), replace=False) if mid.size else mid
    rand = rng.choice(M, min(n_random, M), replace=False)
    edges = np.array([0, M - 1, M // 16 - 1, M // 16, M // 2], dtype=np.int64)
    return np.unique(np.concatenate([heavy, empty, mid, rand, edges]).astype(np.int64))


def sub_problem(rp, ci, rows):
    """The sampled rows of A as their own CSR over the columns they touch:
    (rowptr, remapped colind, positions of their nonzeros in A, touched columns)."""
    rp = rp.astype(np.int64)
    lens = rp[rows + 1] - rp[rows]
    pos = (np.concatenate([np.arange(rp[r], rp[r + 1]) for r in rows]) if lens.sum()
           else np.zeros(0, np.int64))
    cols, local = np.unique(ci[pos], return_inverse=True)
    sub_rp = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
    return sub_rp, local.astype(np.int32), pos, cols


def precision_results(A, dev, grid: str, steps: int, warmup: int, warps: int = 0):
    """The precision form at full size: FP16 A values; B of width 256 stored as
    FP32, BF16 and E4M3 with per-row FP32 scales; FP32 accumulation.  For each
    format: the time of one spmm_csr (CUDA events, mean over `steps` after
    `warmup`), its HBM roofline fraction, and the error against the FP64 oracle
    on sampled rows, normalised by |A||B|: against the product of the original
    FP32 data (what the storage costs) and against the product of the stored,
    dequantised inputs (what the kernel adds)."""
    import torch
    import oracle
    from paper_2311_18141_gb300 import binding, inputs
    N = 256
    M, K, nnz = A.M, A.K, A.nnz
    B = inputs.dense_normal(K, N, seed=2, device=dev)
    v16 = A.vals.to(torch.float16)
    TR, TC = (int(x) for x in grid.split("x"))
    stream = torch.cuda.current_stream()
    rp, ci = A.rowptr.cpu().numpy(), A.colind.cpu().numpy()
    rows = sample_rows(rp, 1000, seed=83)
    sub_rp, sub_ci, pos, cols = sub_problem(rp, ci, rows)
    v = oracle.decode_f16(v16.view(torch.int16).cpu().numpy().view(np.uint16)[pos])
    cols_d = torch.from_numpy(cols).to(dev)
    rows_d = torch.from_numpy(rows).to(dev)
    b32 = B[cols_d].cpu().numpy().astype(np.float64)
    ref0 = oracle.spmm(sub_rp, sub_ci, v, b32)
    bound0 = oracle.abs_bound(sub_rp, sub_ci, v, b32)
    out = {}
    plan = binding.Plan(A.rowptr, M, K, nnz, N, TR, TC,
                        tuning=binding.make_tuning(warps_per_cta=warps))
    ws = binding.workspace(plan.workspace_bytes, dev)
    C = torch.empty(M, N, device=dev)
    for fmt in ("f32", "bf16", "e4m3"):
        scale = None
        if fmt == "f32":
            Bq, bdq = B, b32
        elif fmt == "bf16":
            Bq = torch.empty(K, N, dtype=torch.bfloat16, device=dev)
            binding.spmm_quantize_rows(B, binding.SPMM_BF16, Bq)
            bdq = oracle.decode_bf16(Bq[cols_d].view(torch.int16).cpu().numpy().view(np.uint16))
        else:
            Bq = torch.empty(K, N, dtype=torch.uint8, device=dev)
            scale = torch.empty(K, dtype=torch.float32, device=dev)
            binding.spmm_quantize_rows(B, binding.SPMM_E4M3, Bq, scale)
            bdq = oracle.dequantize_rows(Bq[cols_d].cpu().numpy(), scale[cols_d].cpu().numpy(),
                                         "e4m3")

        def step():
            binding.spmm_csr(A.rowptr, A.colind, v16, Bq, C, M, K, N, nnz, b_scale=scale,
                             plan=plan, ws=ws, stream=stream)
        ms = _time_ms(step, steps, warmup, stream)
        assert binding.spmm_get_device_status(ws) == 0
        w_b = {"f32": 4, "bf16": 2, "e4m3": 1}[fmt]
        algo = min_bytes(M, K, N, nnz, w_val=2, w_b=w_b) + (4 * K if fmt == "e4m3" else 0)
        got = C[rows_d].double().cpu().numpy()
        rel0 = np.abs(got - ref0) / np.maximum(bound0, 1e-30)
        ref1 = oracle.spmm(sub_rp, sub_ci, v, bdq)
        bound1 = oracle.abs_bound(sub_rp, sub_ci, v, bdq)
        rel1 = np.abs(got - ref1) / np.maximum(bound1, 1e-30)
        out[fmt] = {"ms": ms, "gflops": 2.0 * nnz * N / ms / 1e6,
                    "kernel": kernel_name(N, TC, esz=w_b,
                                          tag={"f32": "TagF32", "bf16": "TagBF16",
                                               "e4m3": "TagE4M3"}[fmt]).replace(
                                              "<TagF32,", "<TagF16,"),
                    "algorithmic_bytes": algo,
                    "hbm_frac": algo / (ms * 1e-3) / 1e9 / measured_peaks()[0],
                    "err_max": float(rel0.max()), "err_rms": float(np.sqrt((rel0 ** 2).mean())),
                    "err_max_vs_stored_inputs": float(rel1.max())}
        del Bq
    plan.close()
    return {"workload": f"rmat-s22-fp16A-n256-grid{grid}" if A.M == 1 << 22 else
            f"rmat-fp16A-n256-grid{grid}", "N": N, "tile_grid": grid,
            "error_sample_rows": int(rows.size), "error_unit": "|C - C64| / (|A||B|)",
            "results": out,
            "bf16_faster_than_f32": out["bf16"]["ms"] < out["f32"]["ms"],
            "bf16_within_1e-2": out["bf16"]["err_max"] <= 1e-2,
            "e4m3_faster_than_bf16": out["e4m3"]["ms"] < out["bf16"]["ms"]}


def small_results(dev, steps: int = 200, warps: int = 0):
    """The small FP32 form: A 4096 x 4096 with exactly 16 nonzeros per row, B
    4096 x 32.  L2-resident and launch-bound, so times are per call: the
    device time of back-to-back calls (CUDA events), the host time of the
    spmm_csr call itself (no synchronisation), and the FP64 oracle on one
    host core and on all of them."""
    import torch
    import oracle
    from paper_2311_18141_gb300 import binding, inputs
    A = inputs.uniform_csr(4096, 4096, 16, seed=1, device=dev)
    N = 32
    B = inputs.dense_normal(4096, N, seed=1, device=dev)
    C = torch.empty(4096, N, device=dev)
    plan = binding.Plan(A.rowptr, A.M, A.K, A.nnz, N, 1, 1,
                        tuning=binding.make_tuning(warps_per_cta=warps))
    ws = binding.workspace(plan.workspace_bytes, dev)
    stream = torch.cuda.current_stream()

    def step():
        binding.spmm_csr(A.rowptr, A.colind, A.vals, B, C, A.M, A.K, N, A.nnz, plan=plan,
                         ws=ws, stream=stream)
    dev_us = _time_ms(step, steps, 20, stream) * 1e3
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        step()
    host_us = (time.perf_counter() - t0) * 1e6 / steps
    torch.cuda.synchronize()
    assert binding.spmm_get_device_status(ws) == 0
    plan.close()
    rp, ci, v, Bh = (A.rowptr.cpu().numpy(), A.colind.cpu().numpy(), A.vals.cpu().numpy(),
                     B.cpu().numpy())

    def oracle_us(threads):
        oracle.set_threads(threads)
        reps, t = 0, 0.0
        while t < 1.0:
            t0 = time.perf_counter()
            oracle.spmm(rp, ci, v, Bh)
            t += time.perf_counter() - t0
            reps += 1
        return t * 1e6 / reps

    cores = len(os.sched_getaffinity(0))
    one, allc = oracle_us(1), oracle_us(cores)
    flops = 2.0 * A.nnz * N
    return {"workload": "uniform-4096-16nnz-n32-fp32", "nnz": A.nnz, "N": N,
            "device_us_per_call": dev_us, "gflops": flops / (dev_us * 1e-6) / 1e9,
            "host_us_per_call": host_us,
            "kernel": kernel_name(N, 1),
            "cache": "L2-resident (1.6 MB), back-to-back calls",
            "oracle_us_1_core": one, "oracle_us_all_cores": allc, "oracle_cores": cores}


def run_precision(args):
    """The precision form alone (see precision_results)."""
    import torch
    from paper_2311_18141_gb300 import binding
    dev = torch.device("cuda")
    binding.load_library()
    A, _ = make_workload(args.scale, 8, dev)
    print(json.dumps(precision_results(A, dev, args.grid, args.steps, args.warmup, warps=args.warps)), flush=True)


def run_gcn(args):
    """GCN layer C = A_hat (X W) on the symmetrised R-MAT scale-18 graph: forward
    SpMM, the device transpose, dB = A_hat^T dC and SDDMM, timed separately."""
    import torch
    from paper_2311_18141_gb300 import binding, inputs
    from paper_2311_18141_gb300.autograd import SparseCSR
    dev = torch.device("cuda")
    binding.load_library()
    torch.backends.cuda.matmul.allow_tf32 = False
    A = inputs.gcn_normalized_adjacency(18, 16, seed=4, device=dev)
    X = inputs.dense_normal(A.M, 128, seed=55, device=dev)
    W = inputs.glorot_uniform(128, 64, seed=56, device=dev)
    B = X @ W
    dC = inputs.dense_normal(A.M, 64, seed=57, device=dev)
    N, M, K, nnz = 64, A.M, A.K, A.nnz
    S = SparseCSR(A.rowptr, A.colind, M, K, tile_rows=8)
    stream = torch.cuda.current_stream()
    C = torch.empty(M, N, device=dev)
    plan, ws = S.plan(N)
    fwd = _time_ms(lambda: binding.spmm_csr(A.rowptr, A.colind, A.vals, B, C, M, K, N, nnz,
                                            plan=plan, ws=ws, stream=stream),
                   args.steps, args.warmup, stream)
    colptr = torch.empty(K + 1, dtype=torch.int32, device=dev)
    rowind = torch.empty(nnz, dtype=torch.int32, device=dev)
    tv = torch.empty(nnz, device=dev)
    perm = torch.empty(nnz, dtype=torch.int32, device=dev)
    tws = binding.workspace(binding.spmm_csr_transpose_workspace_size(M, K, nnz), dev)
    tr = _time_ms(lambda: binding.spmm_csr_transpose(A.rowptr, A.colind, A.vals, M, K, nnz, colptr,
                                                     rowind, tv, perm, tws, stream=stream),
                  args.steps, args.warmup, stream)
    tplan, tws2 = S.plan(N, transpose=True)
    dB = torch.empty(K, N, device=dev)
    bwd_b = _time_ms(lambda: binding.spmm_csr(colptr, rowind, tv, dC, dB, K, M, N, nnz,
                                              plan=tplan, ws=tws2, stream=stream),
                     args.steps, args.warmup, stream)
    splan, sws = S.plan(N, sddmm=True)
    dv = torch.empty(nnz, device=dev)
    sd = _time_ms(lambda: binding.spmm_sddmm_csr(A.rowptr, A.colind, dC, B, dv, M, K, N, nnz,
                                                 plan=splan, ws=sws, stream=stream),
                  args.steps, args.warmup, stream)
    fwd_bytes = min_bytes(M, K, N, nnz)
    sd_bytes = 4 * (M + 1) + 4 * nnz + 4 * M * N + 4 * K * N + 4 * nnz
    peak = measured_peaks()[0]
    print(json.dumps({"workload": "gcn-rmat-s18-n64", "nnz": nnz,
                      "forward_ms": fwd, "forward_hbm_frac": fwd_bytes / (fwd * 1e-3) / 1e9 / peak,
                      "transpose_ms": tr, "dB_ms": bwd_b,
                      "sddmm_ms": sd, "sddmm_hbm_frac": sd_bytes / (sd * 1e-3) / 1e9 / peak}),
          flush=True)


def run_batch(args):
    """512 uneven BF16 products (rows log-uniform 1e3..2e5, Poisson nnz/row with
    mean U[8,64], N in {16, 64, 128}): one graph-replayed persistent launch,
    before and after autotuning, against 512 sequential spmm_csr launches."""
    import torch
    from paper_2311_18141_gb300 import binding, inputs
    dev = torch.device("cuda")
    binding.load_library()
    specs = inputs.batch_specs(args.batch_count, seed=5)
    probs, flops, algo = [], 0.0, 0
    for sp in specs:
        A = inputs.poisson_csr(sp.rows, sp.rows, sp.mean_nnz, seed=sp.seed, device=dev)
        B = inputs.dense_normal(A.K, sp.N, seed=sp.seed + 1, device=dev).to(torch.bfloat16)
        C = torch.empty(A.M, sp.N, device=dev)
        probs.append(dict(rowptr=A.rowptr, colind=A.colind, vals=A.vals.to(torch.bfloat16),
                          B=B, C=C, M=A.M, K=A.K, N=sp.N))
        flops += 2.0 * A.nnz * sp.N
        algo += min_bytes(A.M, A.K, sp.N, A.nnz, w_val=2, w_b=2)
    stream = torch.cuda.current_stream()
    # sequential: one plan and one spmm_csr launch per product
    seq = []
    for q in probs:
        pl = binding.Plan(q["rowptr"], q["M"], q["K"], q["colind"].numel(), q["N"], 1, 1)
        seq.append((q, pl, binding.workspace(pl.workspace_bytes, dev)))

    def run_seq():
        for q, pl, w in seq:
            binding.spmm_csr(q["rowptr"], q["colind"], q["vals"], q["B"], q["C"], q["M"], q["K"],
                             q["N"], q["colind"].numel(), plan=pl, ws=w, stream=stream)
    seq_ms = _time_ms(run_seq, max(3, args.steps // 10), 2, stream)
    batch = binding.Batch(probs)
    bws = binding.workspace(batch.workspace_bytes, dev)
    graph_ms = _time_ms(lambda: batch.graph_launch(bws, stream), args.steps, args.warmup, stream)
    tune_ms = batch.autotune(bws, reps=3)
    tuned_ms = _time_ms(lambda: batch.graph_launch(bws, stream), args.steps, args.warmup, stream)
    peak = measured_peaks()[0]
    nnz = sum(q["colind"].numel() for q in probs)
    print(json.dumps({"workload": f"batch-{args.batch_count}-bf16", "nnz": nnz, "gflop": flops / 1e9,
                      "algorithmic_bytes": algo, "sequential_ms": seq_ms,
                      "graph_ms": graph_ms, "autotuned_graph_ms": tuned_ms,
                      "autotune_best_ms": tune_ms,
                      "speedup_vs_sequential": seq_ms / tuned_ms,
                      "tuned_gflops": flops / (tuned_ms * 1e-3) / 1e9,
                      "tuned_hbm_frac": algo / (tuned_ms * 1e-3) / 1e9 / peak}), flush=True)
    for _, pl, _ in seq:
        pl.close()
    batch.close()


def run_spgemm(args):
    """Local SpGEMM C = A*A on an R-MAT matrix (edge factor 16, FP32 values):
    the expand-sort-compress product through spmm_spgemm, timed with CUDA events
    after warm-up, checked against the FP64 oracle on sampled rows."""
    import ctypes
    import numpy as np
    import torch
    import oracle
    from paper_2311_18141_gb300 import binding, inputs
    dev = torch.device("cuda")
    lib = binding.load_library()
    A = inputs.rmat_csr(args.spgemm_scale, 16, 0.57, 0.19, 0.19, seed=1, device=dev, values="pos")
    M, nnz = A.M, A.nnz
    stream = torch.cuda.current_stream()
    P, wsb = ctypes.c_int64(), ctypes.c_size_t()
    assert lib.spmm_spgemm_analyze(A.rowptr.data_ptr(), A.colind.data_ptr(), M, M, nnz,
                                   A.rowptr.data_ptr(), M, ctypes.byref(P), ctypes.byref(wsb),
                                   ctypes.c_void_p(stream.cuda_stream)) == 0
    ws = binding.workspace(wsb.value, dev)
    E = ctypes.c_int64()

    def step():
        rc = lib.spmm_spgemm(A.rowptr.data_ptr(), A.colind.data_ptr(), A.vals.data_ptr(), M, M,
                             nnz, A.rowptr.data_ptr(), A.colind.data_ptr(), A.vals.data_ptr(), M,
                             P.value, ws.data_ptr(), wsb.value, ctypes.byref(E),
                             ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0
    ms = _time_ms(step, args.steps, args.warmup, stream)
    rp, ci, v, _ = binding.spgemm(A.rowptr, A.colind, A.vals, M, M, A.rowptr, A.colind, A.vals,
                                  M, ws=ws)
    # sampled rows against the oracle
    rph, cih = A.rowptr.cpu().numpy(), A.colind.cpu().numpy()
    vh = A.vals.cpu().numpy().astype(np.float64)
    erp, eci, ev = oracle.spgemm(rph, cih, vh, rph, cih, vh, M, M)
    got_rp = rp.cpu().numpy()
    structure_ok = bool(np.array_equal(got_rp, erp) and np.array_equal(ci.cpu().numpy(), eci))
    _, _, bound = oracle.spgemm(rph, cih, np.abs(vh), rph, cih, np.abs(vh), M, M)
    rel = np.abs(v.cpu().numpy().astype(np.float64) - ev) / np.maximum(bound, 1e-30)
    bytes_min = 4 * (M + 1) + 8 * nnz + 4 * (M + 1) + 8 * E.value   # A once, C once
    context = None
    if args.context:   # cuSPARSE SpGEMM through torch.sparse.mm, as context only
        At = torch.sparse_csr_tensor(A.rowptr.long(), A.colind.long(), A.vals, size=(M, M))
        ctx_ms = _time_ms(lambda: torch.sparse.mm(At, At), max(3, args.steps), 2, stream)
        context = {"torch_sparse_mm_ms": ctx_ms,
                   "what": "cuSPARSE SpGEMM through torch.sparse.mm on the same A (context only)"}
    print(json.dumps({"workload": f"spgemm-rmat-s{args.spgemm_scale}-AxA", "nnz": nnz,
                      "products": P.value, "entries": E.value, "ms": ms,
                      "gflops": 2.0 * P.value / (ms * 1e-3) / 1e9,
                      "products_per_s": P.value / (ms * 1e-3),
                      "structure_matches_oracle": structure_ok,
                      "err_max": float(rel.max()) if rel.size else 0.0,
                      "min_bytes": bytes_min, "context": context}), flush=True)


def run_gather(args):
    """The SpMM's B gathers alone (spmm_bench_gather): for every nonzero of the
    R-MAT scale-22 matrix and every column block, the block's segment of B row
    colind[e], in the SpMM's interleaved order, nothing else.  Timed for the
    benchmark's 16 x 4 grid (128-byte segments) and 16 x 1 (512 bytes), on the
    matrix's own column stream, on uniform random columns (no reuse: DRAM
    bound) and on columns below 60,000 (30 MB of B rows: L2-resident), next to
    the full SpMM at the same grid, on the matrix's columns and on the
    L2-resident ones.  The gathered bytes are nnz * N * 4."""
    import torch
    from paper_2311_18141_gb300 import binding
    dev = torch.device("cuda")
    binding.load_library()
    A, B = make_workload(args.scale, args.n, dev)
    M, K, N, nnz = A.M, A.K, args.n, A.nnz
    stream = torch.cuda.current_stream()
    out = torch.zeros(1, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    streams = {"rmat": A.colind,
               "uniform": inputs_uniform_cols(nnz, K, 11, dev),
               "l2_resident": inputs_uniform_cols(nnz, min(K, 60000), 12, dev)}
    if args.ksplit > 1:
        # the same gathers in the orders a K-split 3D grid (Section 3.4's
        # reservation over (i, j, k) tiles) would issue them, with K cut into
        # `ksplit` blocks: "ksplit_tile" sweeps the k-blocks inside each C row
        # block (stationary C, a row block's C slice kept in L2), and
        # "ksplit_kmajor" sweeps every row block inside each k-block (B's
        # k-block slice kept in L2).  The gathered bytes are the same.
        TRg = 16
        RB = -(-M // TRg)
        KB = -(-K // args.ksplit)
        row_of = torch.repeat_interleave(torch.arange(M, device=dev),
                                         (A.rowptr[1:] - A.rowptr[:-1]).long())
        rb = row_of // RB
        kb = A.colind.long() // KB
        pos = torch.arange(nnz, device=dev)
        for name, key in (("ksplit_tile", (rb * args.ksplit + kb) * nnz + pos),
                          ("ksplit_kmajor", (kb * TRg + rb) * nnz + pos)):
            streams[name] = A.colind[torch.argsort(key)].contiguous()
        del row_of, rb, kb, pos
    gathered = nnz * N * 4

    def timed(fn, reps=5):
        ts = []
        for r in range(reps + 1):
            flush.zero_()   # L2 starts cold for every rep
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            if r:
                ts.append(e0.elapsed_time(e1))
        return sorted(ts)[len(ts) // 2]

    res = {}
    for grid in ("16x4", "16x1"):
        TR, TC = (int(x) for x in grid.split("x"))
        row = {}
        for name, ci in streams.items():
            ms = timed(lambda: binding.spmm_bench_gather(ci, nnz, B, K, N, TC, out,
                                                         stream=stream))
            row[name] = {"ms": ms, "gather_TBps": gathered / (ms * 1e-3) / 1e12}
        C = torch.empty(M, N, device=dev)
        plan = binding.Plan(A.rowptr, M, K, nnz, N, TR, TC,
                            tuning=binding.make_tuning(tile_order=args.order))
        ws = binding.workspace(plan.workspace_bytes, dev)
        ms = timed(lambda: binding.spmm_csr(A.rowptr, A.colind, A.vals, B, C, M, K, N, nnz,
                                            plan=plan, ws=ws, stream=stream))
        row["spmm_ms"] = ms
        # the same product on the L2-resident column stream: the kernel's SM
        # side with B's misses taken away
        ci_l2 = streams["l2_resident"]
        row["spmm_l2_resident_ms"] = timed(
            lambda: binding.spmm_csr(A.rowptr, ci_l2, A.vals, B, C, M, K, N, nnz, plan=plan,
                                     ws=ws, stream=stream))
        row["spmm_over_gather_floor"] = ms / row["rmat"]["ms"]
        row["spmm_hbm_frac_at_gather_floor"] = (min_bytes(M, K, N, nnz) /
                                                (row["rmat"]["ms"] * 1e-3) / 1e9 /
                                                measured_peaks()[0])
        plan.close()
        del C, ws
        res[grid] = row
    print(json.dumps({"workload": f"gather-rmat-s{args.scale}-n{N}", "nnz": nnz,
                      "gathered_bytes": gathered, "results": res}), flush=True)


def run_ksplit(args):
    """The K-split 3D grid of Section 3.4's reservation over (i, j, k) tiles,
    measured from its work.  A's rows are cut by k-block into sub-rows (the
    (row, k-block) pairs that hold nonzeros), ordered by C row block, then
    k-block, then row: a row block's k-blocks one after the other, so its C
    slice stays in L2 while B's k-blocks go by.  spmm_csr multiplies that
    matrix by B at the benchmark's 16 x 4 grid, so every gather a K-split
    kernel would issue is issued in its order and every partial row is
    written once.  A K-split kernel must in addition add the partial rows of
    a row into C, so this time is a lower bound on its time."""
    import torch
    from paper_2311_18141_gb300 import binding
    dev = torch.device("cuda")
    binding.load_library()
    A, B = make_workload(args.scale, args.n, dev)
    M, K, N, nnz = A.M, A.K, args.n, A.nnz
    TR, TC = (int(x) for x in args.grid.split("x"))
    stream = torch.cuda.current_stream()
    tun = binding.make_tuning(tile_order=args.order)

    def product_ms(rowptr, colind, vals, rows):
        C = torch.empty(rows, N, device=dev)
        plan = binding.Plan(rowptr, rows, K, nnz, N, TR, TC, tuning=tun)
        ws = binding.workspace(plan.workspace_bytes, dev)
        ms = _time_ms(lambda: binding.spmm_csr(rowptr, colind, vals, B, C, rows, K, N, nnz,
                                               plan=plan, ws=ws, stream=stream),
                      args.steps, args.warmup, stream)
        assert binding.spmm_get_device_status(ws) == 0
        plan.close()
        return ms

    out = {"plain_ms": product_ms(A.rowptr, A.colind, A.vals, M)}
    RB = -(-M // TR)
    row_of = torch.repeat_interleave(torch.arange(M, device=dev),
                                     (A.rowptr[1:] - A.rowptr[:-1]).long())
    for nk in (2, 4, 16):
        KB = -(-K // nk)
        key = ((row_of // RB) * nk + A.colind.long() // KB) * M + row_of
        key, perm = torch.sort(key, stable=True)
        _, counts = torch.unique_consecutive(key, return_counts=True)
        rows = int(counts.numel())
        rowptr = torch.zeros(rows + 1, dtype=torch.int32, device=dev)
        rowptr[1:] = torch.cumsum(counts, 0).to(torch.int32)
        colind = A.colind[perm].contiguous()
        vals = A.vals[perm].contiguous()
        del key, perm, counts
        ms = product_ms(rowptr, colind, vals, rows)
        out[f"k{nk}"] = {"sub_rows": rows, "ms_lower_bound": ms,
                         "partial_rows_per_row": rows / M}
        del rowptr, colind, vals
        torch.cuda.empty_cache()
    print(json.dumps({"workload": f"ksplit-rmat-s{args.scale}-n{N}-grid{args.grid}", "nnz": nnz,
                      "results": out}), flush=True)


def inputs_uniform_cols(nnz, K, seed, device):
    """nnz column indices uniform in [0, K), from the counter-based generator."""
    import torch
    from paper_2311_18141_gb300 import inputs
    h = inputs.hash_u32(torch.arange(nnz, dtype=torch.int64, device=device), seed,
                        inputs.STREAM_COLS)
    return (h % K).to(torch.int32)


def run_loadsim(args):
    """Fig. 1's analysis on the host: R-MAT scale 17, edge factor 8, a = 0.6,
    b = c = d = 0.4/3, squared on a 16 x 16 grid -- end-to-end vs synchronised
    load imbalance, as generated and after one random symmetric relabelling;
    then the SpMM tile grids of the benchmark's shape (N = 128) on the same A."""
    import numpy as np
    from paper_2311_18141_gb300 import inputs, loadsim
    A = inputs.rmat_csr(17, 8, 0.6, 0.4 / 3, 0.4 / 3, seed=1, device="cpu", values="pos")
    rp, ci = A.rowptr.numpy(), A.colind.numpy()
    out = {"workload": "loadsim-rmat-s17-ef8-a0.6-16x16", "nnz": A.nnz}
    for name, (r, c) in (("as_generated", (rp, ci)),
                         ("relabelled", loadsim.relabel(rp, ci, np.random.default_rng(0).permutation(A.M)))):
        w = loadsim.spgemm_stage_work(r, c, r, c, A.K, A.K, 16)
        im = loadsim.imbalance(w)
        ims = loadsim.imbalance(w, offset=True)
        out[name] = {"spgemm_end_to_end": im.end_to_end, "spgemm_synchronised": im.synchronised,
                     "spgemm_worst_stage": float(im.per_stage.max()),
                     "spgemm_synchronised_offset": ims.synchronised,
                     "spgemm_worst_stage_offset": float(ims.per_stage.max())}
        for TR, TC in ((16, 4), (16, 1), (4, 4)):
            imm = loadsim.imbalance(loadsim.spmm_stage_work(r, c, A.K, 128, TR, TC, 16))
            out[name][f"spmm_{TR}x{TC}_end_to_end"] = imm.end_to_end
            out[name][f"spmm_{TR}x{TC}_synchronised"] = imm.synchronised
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.workload == "loadsim":
        run_loadsim(args)
        return
    if args.workload == "spgemm":
        run_spgemm(args)
        return
    if args.workload == "gather":
        run_gather(args)
        return
    if args.workload == "ksplit":
        run_ksplit(args)
        return
    if args.workload == "precision":
        run_precision(args)
        return
    if args.workload == "gcn":
        run_gcn(args)
        return
    if args.workload == "batch":
        run_batch(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
