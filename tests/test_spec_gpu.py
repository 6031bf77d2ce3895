"""The warp-specialised staged kernel (spmm_tuning.kernel = SPMM_KERNEL_SPEC).

Producer warps decode and gather, consumer warps sum: the same item order and
the same FFMA2 sums as the staged kernel, so its C must equal the staged
kernel's bit for bit, and the FP64 oracle's within the FP32 tolerance.  The
shapes cover the three lane widths it is built for (8, 16 and 32 lanes per
item: column blocks of 32, 64 and 128 FP32 values), ragged column blocks,
empty rows, a heavy row cut into many pieces, beta, row scales and BF16 B.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2311_18141_gb300 import binding, inputs
from paper_2311_18141_gb300.inputs import CSR

from gpu_util import TOL_F32, TOL_LOWP, assert_close_rel, run_spmm

pytestmark = pytest.mark.gpu

SPEC = binding.SPMM_KERNEL_SPEC
STAGED = binding.SPMM_KERNEL_STAGED


def heavy_matrix(seed=13):
    M, K = 1001, 5000
    rng = np.random.default_rng(seed)
    lens = np.zeros(M, np.int64)
    lens[::7] = rng.integers(1, 40, lens[::7].size)
    lens[500] = 4000                      # cut into ~60 pieces at chunk 64
    lens[1000] = 3
    rowptr = np.zeros(M + 1, np.int64)
    rowptr[1:] = np.cumsum(lens)
    colind = np.concatenate([np.sort(rng.choice(K, l, replace=False)) for l in lens if l])
    vals = rng.uniform(-1, 1, colind.size).astype(np.float32)
    return CSR(torch.from_numpy(rowptr.astype(np.int32)), torch.from_numpy(colind.astype(np.int32)),
               torch.from_numpy(vals), M, K), lens


@pytest.mark.parametrize("N,grid,chunk,order", [
    (32, (3, 1), 0, 0),       # 8 lanes per item
    (64, (4, 1), 0, 16),      # 16 lanes per item (two stages per decoded batch)
    (128, (2, 1), 0, 0),      # 32 lanes per item (four stages per batch)
    (128, (16, 4), 0, 16),    # the benchmark grid shape
    (40, (5, 1), 96, 0),      # ragged block: 10 vectors on 16 lanes
    (96, (3, 2), 64, 16),     # ragged: 48 columns per block, 12 vectors on 16 lanes
])
def test_spec_matches_oracle_and_staged_bitwise(N, grid, chunk, order):
    A = inputs.rmat_csr(12, 16, seed=31)
    B = inputs.dense_normal(A.K, N, seed=32)
    ref = oracle.spmm(A.rowptr, A.colind, A.vals, B)
    bound = oracle.abs_bound(A.rowptr, A.colind, A.vals, B)
    kw = dict(tile_rows=grid[0], tile_cols=grid[1], chunk_items=chunk, tile_order=order)
    Cs, st = run_spmm(A, B, N, kernel=SPEC, **kw)
    assert st == 0
    assert_close_rel(Cs.numpy(), ref, bound, TOL_F32, f"spec N={N} grid={grid}")
    Ct, st = run_spmm(A, B, N, kernel=STAGED, **kw)
    assert st == 0
    assert torch.equal(Cs, Ct)


def test_spec_empty_rows_and_heavy_row():
    A, lens = heavy_matrix()
    N = 128   # grids 1x1, 5x2, 13x4: 32, 16 and 8 lanes per item
    B = inputs.dense_normal(A.K, N, seed=14)
    ref = oracle.spmm(A.rowptr, A.colind, A.vals, B)
    bound = oracle.abs_bound(A.rowptr, A.colind, A.vals, B)
    for grid, chunk in [((1, 1), 64), ((5, 2), 64), ((13, 4), 50), ((1, 1), 0)]:
        C, st = run_spmm(A, B, N, tile_rows=grid[0], tile_cols=grid[1], chunk_items=chunk,
                         kernel=SPEC)
        assert st == 0
        assert_close_rel(C.numpy(), ref, bound, TOL_F32, f"spec heavy {grid} {chunk}")
        assert np.all(C.numpy()[lens == 0] == 0.0)


def test_spec_beta_and_row_scales():
    A = inputs.rmat_csr(11, 16, seed=33)
    N = 64
    B = inputs.dense_normal(A.K, N, seed=34)
    C0 = inputs.dense_normal(A.M, N, seed=35)
    a_scale = torch.rand(A.M) + 0.5
    beta = 0.75
    v = A.vals * a_scale.repeat_interleave(torch.diff(A.rowptr.long()))
    ref = oracle.spmm(A.rowptr, A.colind, v, B, beta=beta, C0=C0.numpy())
    bound = oracle.abs_bound(A.rowptr, A.colind, v, B) + beta * np.abs(C0.numpy())
    C, st = run_spmm(A, B, N, tile_rows=4, tile_cols=2, beta=beta, C0=C0, a_scale=a_scale,
                     chunk_items=64, kernel=SPEC)
    assert st == 0
    assert_close_rel(C.numpy(), ref, bound, TOL_F32, "spec beta + a_scale")


def test_spec_bf16_b():
    A = inputs.rmat_csr(11, 16, seed=36)
    N = 64
    B = inputs.dense_normal(A.K, N, seed=37)
    Bq = B.to(torch.bfloat16)
    C, st = run_spmm(A, B, N, tile_rows=2, tile_cols=1, Bdev=Bq.cuda(), kernel=SPEC)
    assert st == 0
    ref = oracle.spmm(A.rowptr, A.colind, A.vals, B)
    bound = oracle.abs_bound(A.rowptr, A.colind, A.vals, B)
    assert_close_rel(C.numpy(), ref, bound, TOL_LOWP, "spec bf16 B")
    Ct, _ = run_spmm(A, B, N, tile_rows=2, tile_cols=1, Bdev=Bq.cuda(), kernel=STAGED)
    assert torch.equal(C, Ct)


def test_spec_unsupported_shapes_are_refused():
    A = inputs.uniform_csr(64, 64, 4, seed=38)
    Ad = A.to("cuda")
    for N, TC in [(512, 1), (16, 1)]:     # 4 vectors per lane; 4 lanes per item
        B = torch.zeros(64, N, device="cuda")
        C = torch.zeros(64, N, device="cuda")
        plan = binding.Plan(Ad.rowptr, 64, 64, A.nnz, N, 1, TC,
                            tuning=binding.make_tuning(kernel=SPEC))
        ws = binding.workspace(plan.workspace_bytes)
        with pytest.raises(binding.SpmmError) as e:
            binding.spmm_csr(Ad.rowptr, Ad.colind, Ad.vals, B, C, 64, 64, N, A.nnz, plan=plan,
                             ws=ws)
        assert e.value.status == binding.SPMM_ERR_UNSUPPORTED
        plan.close()


def test_spec_trace_and_exactly_once():
    """Every unit is reserved once: with unit values and B = 1, C's first
    column is each row's length exactly; the producers' trace records account
    for all units."""
    M, K, N = 4096, 4096, 128   # 32 columns per block on the 16 x 4 grid: 8 lanes per item
    rng = np.random.default_rng(27)
    lens = np.zeros(M, np.int64)
    lens[0] = 4000
    lens[1::3] = 2
    rowptr = np.zeros(M + 1, np.int64)
    rowptr[1:] = np.cumsum(lens)
    colind = np.concatenate([np.sort(rng.choice(K, l, replace=False)) for l in lens if l])
    A = CSR(torch.from_numpy(rowptr.astype(np.int32)), torch.from_numpy(colind.astype(np.int32)),
            torch.ones(colind.size), M, K)
    Ad = A.to("cuda")
    B = torch.ones(K, N, device="cuda")
    TR, TC = 16, 4
    plan = binding.Plan(Ad.rowptr, M, K, A.nnz, N, TR, TC,
                        tuning=binding.make_tuning(chunk_items=32, tile_order=16, kernel=SPEC))
    ws = binding.workspace(plan.workspace_bytes)
    buf = binding.trace_buffer(1 << 15)
    plan.set_trace(buf)
    C = torch.empty(M, N, device="cuda")
    binding.spmm_csr(Ad.rowptr, Ad.colind, Ad.vals, B, C, M, K, N, A.nnz, plan=plan, ws=ws)
    torch.cuda.synchronize()
    assert binding.spmm_get_device_status(ws) == 0
    assert torch.equal(C[:, 0].cpu(), torch.from_numpy(lens.astype(np.float32)))
    rec = binding.read_trace(buf)
    chunks, _ = plan.units()
    G = 4   # 8 lanes per item
    total = int(rec["units"].sum())
    assert chunks * TC / G <= total <= chunks * TC / G + TR * TC
    plan.set_trace(None)
    plan.close()
