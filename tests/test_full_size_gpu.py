"""Full-size parity: the power-law FP32 workload exactly as bench.py runs it
(R-MAT scale 22, edge factor 16, N = 128, 16 x 4 tile grid, default plan and
launch), checked against the FP64 oracle on sampled rows: the heaviest rows
(split across many work units), rows cut by chunk boundaries, empty rows and
a random sample."""
import numpy as np
import pytest
import torch

import oracle
from paper_2311_18141_gb300 import binding, inputs

from gpu_util import TOL_F32, assert_close_rel

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


def test_rmat_s22_n128_grid16x4_sampled():
    dev = torch.device("cuda")
    A = inputs.rmat_csr(22, 16, 0.57, 0.19, 0.19, seed=1, device=dev, values="pos")
    N = 128
    B = inputs.dense_normal(A.K, N, seed=2, device=dev)
    C = torch.full((A.M, N), float("nan"), device=dev)
    plan = binding.Plan(A.rowptr, A.M, A.K, A.nnz, N, 16, 4)
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
    assert_close_rel(got, ref, bound, TOL_F32, "R-MAT s22 N=128 16x4 sampled rows")
    # empty rows are exact zeros, and the result is bitwise reproducible
    empty = np.diff(rp.astype(np.int64))[rows] == 0
    assert np.all(got[empty] == 0.0)
    C2 = torch.empty_like(C)
    binding.spmm_csr(A.rowptr, A.colind, A.vals, B, C2, A.M, A.K, N, A.nnz, plan=plan, ws=ws)
    torch.cuda.synchronize()
    assert torch.equal(C, C2)
    plan.close()
