"""Full-size parity, at the sizes and in the launch configurations bench.py
times, checked against the FP64 oracle on sampled rows: the heaviest rows
(split across many work units), rows cut by chunk boundaries, empty rows and a
random sample.
  * the power-law FP32 workload: R-MAT scale 22, edge factor 16, N = 128,
    16 x 4 tiles, with the default stealing order and with the interleaved
    tile-row queues bench.py uses (tile order 16);
  * the precision forms: FP16 A values, B of width 256 stored BF16 and E4M3
    with per-row scales, 16 x 4 tiles;
  * the batch: 512 uneven BF16 products in one persistent launch replayed from
    a CUDA graph after autotuning."""
import numpy as np
import pytest
import torch

import oracle
from paper_2311_18141_gb300 import binding, inputs

from gpu_util import TOL_F32, TOL_LOWP, assert_close_rel

pytestmark = pytest.mark.gpu


def _sample_rows(rowptr: np.ndarray, n_random: int, seed: int) -> np.ndarray:
    lens = np.diff(rowptr.astype(np.int64))
    M = lens.size
    rng = np.random.default_rng(seed)
    heavy = np.argsort(lens)[-32:]
    empty = np.flatnonzero(lens == 0)
    empty = rng.choice(empty, min(256, empty.size), replace=False) if empty.size else empty
    mid = np.flatnonzero((lens > 16) & (lens < 2000))
    mid = rng.choice(mid, min(512, mid.size), replace=False) if mid.size else mid
    rand = rng.choice(M, n_random, replace=False)
    edges = np.array([0, M - 1, M // 16 - 1, M // 16, M // 2], dtype=np.int64)
    return np.unique(np.concatenate([heavy, empty, mid, rand, edges]).astype(np.int64))


def _sub_problem(rp, ci, rows):
    """The sampled rows of A as their own CSR, over the columns they touch:
    (rowptr, remapped colind, positions of their nonzeros in A, touched columns)."""
    rp = rp.astype(np.int64)
    lens = rp[rows + 1] - rp[rows]
    pos = np.concatenate([np.arange(rp[r], rp[r + 1]) for r in rows]) if lens.sum() else \
        np.zeros(0, np.int64)
    cols, local = np.unique(ci[pos], return_inverse=True)
    sub_rp = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
    return sub_rp, local.astype(np.int32), pos, cols


@pytest.mark.parametrize("tile_order", [0, 16])
def test_rmat_s22_n128_grid16x4_sampled(tile_order):
    dev = torch.device("cuda")
    A = inputs.rmat_csr(22, 16, 0.57, 0.19, 0.19, seed=1, device=dev, values="pos")
    N = 128
    B = inputs.dense_normal(A.K, N, seed=2, device=dev)
    C = torch.full((A.M, N), float("nan"), device=dev)
    plan = binding.Plan(A.rowptr, A.M, A.K, A.nnz, N, 16, 4,
                        tuning=binding.make_tuning(tile_order=tile_order))
    ws = binding.workspace(plan.workspace_bytes, dev)
    binding.spmm_csr(A.rowptr, A.colind, A.vals, B, C, A.M, A.K, N, A.nnz, plan=plan, ws=ws)
    torch.cuda.synchronize()
    assert binding.spmm_get_device_status(ws) == 0
    assert not torch.isnan(C).any()
    rp = A.rowptr.cpu().numpy()
    ci = A.colind.cpu().numpy()
    v = A.vals.cpu().numpy()
    Bh = B.cpu().numpy()
    rows = _sample_rows(rp, 2000, seed=81)
    ref = oracle.spmm_rows(rp, ci, v, Bh, rows)
    bound = oracle.spmm_rows(rp, ci, np.abs(v.astype(np.float64)),
                             np.abs(Bh.astype(np.float64)), rows)
    got = C[torch.from_numpy(rows).to(dev)].cpu().numpy()
    assert_close_rel(got, ref, bound, TOL_F32, f"R-MAT s22 N=128 16x4 order {tile_order}")
    # empty rows are exact zeros, and the result is bitwise reproducible
    empty = np.diff(rp.astype(np.int64))[rows] == 0
    assert np.all(got[empty] == 0.0)
    C2 = torch.empty_like(C)
    binding.spmm_csr(A.rowptr, A.colind, A.vals, B, C2, A.M, A.K, N, A.nnz, plan=plan, ws=ws)
    torch.cuda.synchronize()
    assert torch.equal(C, C2)
    plan.close()


@pytest.mark.parametrize("fmt", ["bf16", "e4m3"])
def test_precision_s22_n256_sampled(fmt):
    """FP16 A values and quantised B at full size: sampled rows within 1e-5 of
    the FP64 product of the stored (dequantised) inputs, and BF16 within 1e-2 of
    the product of the original FP32 data."""
    dev = torch.device("cuda")
    A = inputs.rmat_csr(22, 16, 0.57, 0.19, 0.19, seed=1, device=dev, values="pos")
    N = 256
    B = inputs.dense_normal(A.K, N, seed=2, device=dev)
    v16 = A.vals.to(torch.float16)
    scale = None
    if fmt == "bf16":
        Bq = torch.empty(A.K, N, dtype=torch.bfloat16, device=dev)
        binding.spmm_quantize_rows(B, binding.SPMM_BF16, Bq)
    else:
        Bq = torch.empty(A.K, N, dtype=torch.uint8, device=dev)
        scale = torch.empty(A.K, dtype=torch.float32, device=dev)
        binding.spmm_quantize_rows(B, binding.SPMM_E4M3, Bq, scale)
    C = torch.full((A.M, N), float("nan"), device=dev)
    plan = binding.Plan(A.rowptr, A.M, A.K, A.nnz, N, 16, 4)
    ws = binding.workspace(plan.workspace_bytes, dev)
    binding.spmm_csr(A.rowptr, A.colind, v16, Bq, C, A.M, A.K, N, A.nnz, b_scale=scale,
                     plan=plan, ws=ws)
    torch.cuda.synchronize()
    assert binding.spmm_get_device_status(ws) == 0
    rp = A.rowptr.cpu().numpy()
    ci = A.colind.cpu().numpy()
    rows = _sample_rows(rp, 1000, seed=83)
    sub_rp, sub_ci, pos, cols = _sub_problem(rp, ci, rows)
    v = oracle.decode_f16(v16.view(torch.int16).cpu().numpy().view(np.uint16)[pos])
    cols_d = torch.from_numpy(cols).to(dev)
    if fmt == "bf16":
        b = oracle.decode_bf16(Bq[cols_d].view(torch.int16).cpu().numpy().view(np.uint16))
    else:
        b = oracle.dequantize_rows(Bq[cols_d].cpu().numpy(), scale[cols_d].cpu().numpy(), "e4m3")
    got = C[torch.from_numpy(rows).to(dev)].cpu().numpy()
    ref = oracle.spmm(sub_rp, sub_ci, v, b)
    bound = oracle.abs_bound(sub_rp, sub_ci, v, b)
    assert_close_rel(got, ref, bound, TOL_F32, f"{fmt} B, dequantised inputs")
    if fmt == "bf16":
        b32 = B[cols_d].cpu().numpy().astype(np.float64)
        ref0 = oracle.spmm(sub_rp, sub_ci, v, b32)
        bound0 = oracle.abs_bound(sub_rp, sub_ci, v, b32)
        assert_close_rel(got, ref0, bound0, TOL_LOWP, "bf16 B, original FP32 data")
    plan.close()


def test_batch_512_graph_autotuned_sampled():
    """The 512-product batch of bench.py, autotuned and replayed from the CUDA
    graph: sampled rows of every product against the FP64 oracle on the stored
    BF16 inputs."""
    dev = torch.device("cuda")
    specs = inputs.batch_specs(512, seed=5)
    probs = []
    for sp in specs:
        A = inputs.poisson_csr(sp.rows, sp.rows, sp.mean_nnz, seed=sp.seed, device=dev)
        B = inputs.dense_normal(A.K, sp.N, seed=sp.seed + 1, device=dev).to(torch.bfloat16)
        probs.append(dict(rowptr=A.rowptr, colind=A.colind, vals=A.vals.to(torch.bfloat16),
                          B=B, C=torch.full((A.M, sp.N), float("nan"), device=dev), M=A.M,
                          K=A.K, N=sp.N))
    batch = binding.Batch(probs)
    ws = binding.workspace(batch.workspace_bytes)
    batch.autotune(ws)
    for q in probs:
        q["C"].fill_(float("nan"))
    batch.graph_launch(ws)
    torch.cuda.synchronize()
    assert binding.spmm_get_device_status(ws) == 0
    for k, q in enumerate(probs):
        rp = q["rowptr"].cpu().numpy()
        ci = q["colind"].cpu().numpy()
        rows = _sample_rows(rp, min(q["M"], 48), seed=1000 + k)
        sub_rp, sub_ci, pos, cols = _sub_problem(rp, ci, rows)
        v = oracle.decode_bf16(q["vals"].view(torch.int16).cpu().numpy().view(np.uint16)[pos])
        cols_d = torch.from_numpy(cols).to(dev)
        b = oracle.decode_bf16(q["B"][cols_d].view(torch.int16).cpu().numpy().view(np.uint16))
        b = b.reshape(cols.size, q["N"])
        got = q["C"][torch.from_numpy(rows).to(dev)].cpu().numpy()
        ref = oracle.spmm(sub_rp, sub_ci, v, b)
        bound = oracle.abs_bound(sub_rp, sub_ci, v, b)
        assert_close_rel(got, ref, bound, TOL_F32, f"batch product {k}")
    batch.close()


def test_max_size_nnz_near_int32_limit():
    """The largest nonzero count the API takes (2^31 - 8 here, with 2^28 - 1 rows
    of 8), so merge-path positions (rows + nonzeros, about 2.4e9) pass 2^31:
    the plan's 64-bit coordinates and the kernel's 32-bit per-chunk offsets are
    both exercised.  Columns are hashed (repeats allowed, unsorted), B is 2^20 x 4.
    Sampled rows, including both ends of every row block, against the oracle."""
    dev = torch.device("cuda")
    free, _ = torch.cuda.mem_get_info()
    if free < 80 * (1 << 30):
        pytest.skip("needs about 80 GB of free device memory")
    per, M, K, N, TR = 8, (1 << 28) - 1, 1 << 20, 4, 16
    nnz = M * per
    assert nnz == (1 << 31) - 8
    rowptr = (torch.arange(M + 1, dtype=torch.int64, device=dev) * per).to(torch.int32)
    colind = torch.empty(nnz, dtype=torch.int32, device=dev)
    vals = torch.empty(nnz, dtype=torch.float32, device=dev)
    step = 1 << 27
    for lo in range(0, nnz, step):
        e = torch.arange(lo, min(nnz, lo + step), dtype=torch.int64, device=dev)
        colind[lo:lo + e.numel()] = ((e * 2654435761) % K).to(torch.int32)
        vals[lo:lo + e.numel()] = (e % 1021).to(torch.float32) / 1021.0 - 0.5
        del e
    B = inputs.dense_normal(K, N, seed=91, device=dev)
    C = torch.full((M, N), float("nan"), device=dev)
    plan = binding.Plan(rowptr, M, K, nnz, N, TR, 1)
    ws = binding.workspace(plan.workspace_bytes, dev)
    binding.spmm_csr(rowptr, colind, vals, B, C, M, K, N, nnz, plan=plan, ws=ws)
    torch.cuda.synchronize()
    assert binding.spmm_get_device_status(ws) == 0
    rb = -(-M // TR)
    edges = [x for i in range(TR + 1) for x in (i * rb - 1, i * rb) if 0 <= x < M]
    rng = np.random.default_rng(92)
    rows = np.unique(np.concatenate([rng.choice(M, 2000, replace=False), edges, [0, M - 1]]))
    rows_d = torch.from_numpy(rows).to(dev)
    idx = (rows_d.to(torch.int64) * per)[:, None] + torch.arange(per, device=dev)[None, :]
    cols = colind[idx.flatten()].cpu().numpy()
    v = vals[idx.flatten()].cpu().numpy()
    ucols, local = np.unique(cols, return_inverse=True)
    sub_rp = np.arange(rows.size + 1, dtype=np.int32) * per
    b = B[torch.from_numpy(ucols).to(dev)].cpu().numpy()
    ref = oracle.spmm(sub_rp, local.astype(np.int32), v, b)
    bound = oracle.abs_bound(sub_rp, local.astype(np.int32), v, b)
    got = C[rows_d].cpu().numpy()
    assert_close_rel(got, ref, bound, TOL_F32, "nnz = 2^31 - 8")
    plan.close()
