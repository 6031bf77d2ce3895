"""Parity of the CUDA SpMM path with the FP64 oracle (Section 2.1 local product).

Every test calls the library through the C ABI (binding.spmm_csr) and
compares with oracle.spmm element by element within the stated tolerance.
Sizes span many work units and ragged tails; the full-size R-MAT workload is
checked on sampled rows in test_full_size_gpu.py.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2311_18141_gb300 import binding, inputs
from paper_2311_18141_gb300.inputs import CSR

from gpu_util import KERNELS, TOL_F32, assert_close_rel, run_spmm

pytestmark = pytest.mark.gpu


def ref_and_bound(A, B, vals=None, beta=0.0, C0=None):
    v = A.vals if vals is None else vals
    ref = oracle.spmm(A.rowptr, A.colind, v, B, beta=beta,
                      C0=None if C0 is None else C0.numpy())
    bound = oracle.abs_bound(A.rowptr, A.colind, v, B)
    if C0 is not None and beta != 0.0:
        bound = bound + abs(beta) * np.abs(C0.numpy().astype(np.float64))
    return ref, bound


@pytest.mark.parametrize("kernel", KERNELS)
def test_uniform_4096_n32_full(kernel):
    """4096 x 4096, exactly 16 nonzeros per row, B 4096 x 32 (the small FP32 workload)."""
    A = inputs.uniform_csr(4096, 4096, 16, seed=1)
    B = inputs.dense_normal(4096, 32, seed=1)
    C, st = run_spmm(A, B, 32, kernel=kernel)
    assert st == 0
    ref, bound = ref_and_bound(A, B)
    assert_close_rel(C.numpy(), ref, bound, TOL_F32, "uniform 4096 N=32")


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("grid", [(1, 1), (16, 4), (3, 2), (7, 1), (1, 4)])
@pytest.mark.parametrize("chunk", [0, 64, 333])
def test_rmat_grids_and_chunks(grid, chunk, kernel):
    A = inputs.rmat_csr(12, 16, seed=2)
    N = 64
    B = inputs.dense_normal(A.K, N, seed=3)
    C, st = run_spmm(A, B, N, tile_rows=grid[0], tile_cols=grid[1], chunk_items=chunk,
                     kernel=kernel)
    assert st == 0
    ref, bound = ref_and_bound(A, B)
    assert_close_rel(C.numpy(), ref, bound, TOL_F32, f"rmat grid {grid} chunk {chunk}")


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("N", [4, 8, 16, 32, 64, 128, 256, 512])
def test_widths(N, kernel):
    A = inputs.rmat_csr(11, 8, seed=4)
    B = inputs.dense_normal(A.K, N, seed=5)
    C, st = run_spmm(A, B, N, chunk_items=96, kernel=kernel)
    assert st == 0
    ref, bound = ref_and_bound(A, B)
    assert_close_rel(C.numpy(), ref, bound, TOL_F32, f"N={N}")


@pytest.mark.parametrize("opts", [dict(warps_per_cta=4), dict(tile_order=1), dict(tile_order=2),
                                  dict(tile_order=4), dict(plan=False),
                                  dict(warps_per_cta=4, tile_order=5), dict(tile_order=8),
                                  dict(tile_order=9), dict(tile_order=16), dict(tile_order=24),
                                  dict(warps_per_cta=4, tile_order=16), dict(warps_per_cta=7),
                                  dict(warps_per_cta=5, tile_order=16), dict(warps_per_cta=3)])
@pytest.mark.parametrize("kernel", KERNELS)
def test_launch_options(opts, kernel):
    A = inputs.rmat_csr(12, 8, seed=6)
    N = 32
    B = inputs.dense_normal(A.K, N, seed=7)
    C, st = run_spmm(A, B, N, tile_rows=4, tile_cols=2, kernel=kernel, **opts)
    assert st == 0
    ref, bound = ref_and_bound(A, B)
    assert_close_rel(C.numpy(), ref, bound, TOL_F32, str(opts))


@pytest.mark.parametrize("kernel", KERNELS)
def test_beta_accumulate_and_scale(kernel):
    A = inputs.rmat_csr(11, 16, seed=8)
    N = 32
    B = inputs.dense_normal(A.K, N, seed=9)
    C0 = inputs.dense_normal(A.M, N, seed=10)
    for beta in (1.0, -0.5):
        C, st = run_spmm(A, B, N, tile_rows=2, tile_cols=2, beta=beta, C0=C0, chunk_items=128,
                         kernel=kernel)
        assert st == 0
        ref, bound = ref_and_bound(A, B, beta=beta, C0=C0)
        assert_close_rel(C.numpy(), ref, bound, TOL_F32, f"beta={beta}")


def test_beta_zero_ignores_nan_in_c():
    A = inputs.uniform_csr(300, 200, 5, seed=11)
    B = inputs.dense_normal(200, 16, seed=12)
    C0 = torch.full((300, 16), float("nan"))
    C, st = run_spmm(A, B, 16, beta=0.0, C0=C0)
    assert st == 0 and not torch.isnan(C).any()


@pytest.mark.parametrize("kernel", KERNELS)
def test_empty_rows_ragged_blocks_and_heavy_row(kernel):
    # rows: many empty, one enormous row split across many chunks, ragged M
    M, K, N = 1001, 5000, 32
    rng = np.random.default_rng(13)
    lens = np.zeros(M, np.int64)
    lens[::7] = rng.integers(1, 40, lens[::7].size)
    lens[500] = 4000                      # heavy row, cut into ~60 pieces at chunk 64
    lens[1000] = 3                        # last row
    rowptr = np.zeros(M + 1, np.int64)
    rowptr[1:] = np.cumsum(lens)
    colind = np.concatenate([np.sort(rng.choice(K, l, replace=False)) for l in lens if l])
    vals = rng.uniform(-1, 1, colind.size).astype(np.float32)
    A = CSR(torch.from_numpy(rowptr.astype(np.int32)), torch.from_numpy(colind.astype(np.int32)),
            torch.from_numpy(vals), M, K)
    B = inputs.dense_normal(K, N, seed=14)
    ref, bound = ref_and_bound(A, B)
    for grid, chunk in [((1, 1), 64), ((5, 2), 64), ((13, 4), 50), ((1, 1), 0)]:
        C, st = run_spmm(A, B, N, tile_rows=grid[0], tile_cols=grid[1], chunk_items=chunk,
                         kernel=kernel)
        assert st == 0
        assert_close_rel(C.numpy(), ref, bound, TOL_F32, f"heavy grid {grid} chunk {chunk}")
        empty = lens == 0
        assert np.all(C.numpy()[empty] == 0.0)


def test_row_sums_positive_terms_gamma_bound():
    """A*1 = row sums.  All terms positive, so the FP32 error is bounded by
    gamma_n = n*u/(1-n*u) times the sum (n = row length + split pieces)."""
    A = inputs.rmat_csr(12, 16, seed=15)          # positive values
    N = 4
    B = torch.ones(A.K, N)
    C, st = run_spmm(A, B, N, tile_rows=2, chunk_items=100)
    assert st == 0
    lens = A.row_lengths().numpy().astype(np.float64)
    rows = np.repeat(np.arange(A.M), A.row_lengths().numpy())
    sums = np.bincount(rows, weights=A.vals.numpy().astype(np.float64), minlength=A.M)
    u = 2.0 ** -24
    n = lens + 64
    lim = (n * u / (1 - n * u)) * sums
    err = np.abs(C.numpy()[:, 0].astype(np.float64) - sums)
    assert np.all(err <= lim)
    assert np.all(C.numpy() == C.numpy()[:, :1])   # all columns identical


def test_identity_and_permutation_exact():
    n, N = 5000, 64
    B = inputs.dense_normal(n, N, seed=16)
    perm = torch.from_numpy(np.random.default_rng(17).permutation(n).astype(np.int32))
    eye = CSR(torch.arange(n + 1, dtype=torch.int32), perm, torch.ones(n), n, n)
    C, st = run_spmm(eye, B, N, tile_rows=3, tile_cols=2)
    assert st == 0
    assert torch.equal(C, B[perm.long()])


def test_empty_matrix_and_degenerate_shapes():
    # nnz == 0: C = beta * C (0 for beta = 0)
    M, K, N = 77, 50, 16
    A = CSR(torch.zeros(M + 1, dtype=torch.int32), torch.zeros(0, dtype=torch.int32),
            torch.zeros(0), M, K)
    B = inputs.dense_normal(K, N, seed=18)
    C, st = run_spmm(A, B, N, tile_rows=4)
    assert st == 0 and torch.equal(C, torch.zeros(M, N))
    C0 = inputs.dense_normal(M, N, seed=19)
    C, st = run_spmm(A, B, N, beta=2.0, C0=C0)
    assert torch.equal(C, 2.0 * C0)
    # single row, single column
    A1 = CSR(torch.tensor([0, 1], dtype=torch.int32), torch.tensor([0], dtype=torch.int32),
             torch.tensor([3.0]), 1, 1)
    B1 = torch.arange(4, dtype=torch.float32).view(1, 4)
    C, st = run_spmm(A1, B1, 4)
    assert torch.equal(C, 3.0 * B1)
    # more tile rows than rows
    A2 = inputs.uniform_csr(5, 9, 3, seed=20)
    B2 = inputs.dense_normal(9, 8, seed=21)
    C, st = run_spmm(A2, B2, 8, tile_rows=16, tile_cols=2)
    ref, bound = ref_and_bound(A2, B2)
    assert_close_rel(C.numpy(), ref, bound, TOL_F32, "tiny")


@pytest.mark.parametrize("kernel", KERNELS)
def test_deterministic_bitwise(kernel):
    A = inputs.rmat_csr(13, 16, seed=22)
    N = 128
    B = inputs.dense_normal(A.K, N, seed=23)
    C1, _ = run_spmm(A, B, N, tile_rows=16, tile_cols=4, chunk_items=77, kernel=kernel)
    C2, _ = run_spmm(A, B, N, tile_rows=16, tile_cols=4, chunk_items=77, kernel=kernel)
    assert torch.equal(C1, C2)


def test_wide_kernel_rejects_16_byte_layouts():
    """The 32-byte-lane kernel, asked for explicitly, refuses column blocks,
    strides or pointers that are not whole 32-byte vectors (the default choice
    then runs the staged kernel instead)."""
    A = inputs.uniform_csr(64, 64, 4, seed=24)
    Ad = A.to("cuda")
    tun = binding.make_tuning(kernel=binding.SPMM_KERNEL_WIDE)
    for N, TC, off in [(4, 1, 0), (12, 1, 0), (16, 4, 0), (16, 1, 4)]:
        B = inputs.dense_normal(64, N, seed=25).cuda()
        Cbuf = torch.zeros(64 * N + off, device="cuda")
        C = Cbuf[off:].view(64, N)
        plan = binding.Plan(Ad.rowptr, 64, 64, A.nnz, N, 2, TC, tuning=tun)
        ws = binding.workspace(plan.workspace_bytes)
        with pytest.raises(binding.SpmmError) as e:
            binding.spmm_csr(Ad.rowptr, Ad.colind, Ad.vals, B, C, 64, 64, N, A.nnz, plan=plan,
                             ws=ws)
        assert e.value.status == binding.SPMM_ERR_MISALIGNED, (N, TC, off)
        plan.close()


def test_misaligned_and_plan_mismatch_rejected():
    A = inputs.uniform_csr(64, 64, 4, seed=24)
    Ad = A.to("cuda")
    B = inputs.dense_normal(64, 8, seed=25).cuda()
    C = torch.zeros(64, 8, device="cuda")
    plan = binding.Plan(Ad.rowptr, 64, 64, A.nnz, 8, 2, 1)
    ws = binding.workspace(plan.workspace_bytes)
    with pytest.raises(binding.SpmmError) as e:
        Cbad = torch.zeros(64 * 8 + 1, device="cuda")[1:].view(64, 8)
        binding.spmm_csr(Ad.rowptr, Ad.colind, Ad.vals, B, Cbad, 64, 64, 8, A.nnz, plan=plan, ws=ws)
    assert e.value.status == binding.SPMM_ERR_MISALIGNED
    with pytest.raises(binding.SpmmError) as e:
        binding.spmm_csr(Ad.rowptr, Ad.colind, Ad.vals, B, C, 64, 64, 8, A.nnz, plan=plan, ws=ws,
                         tile_rows=4)
    assert e.value.status == binding.SPMM_ERR_PLAN_MISMATCH
    with pytest.raises(binding.SpmmError) as e:
        binding.spmm_csr(Ad.rowptr, Ad.colind, Ad.vals, B, C, 64, 64, 8, A.nnz, plan=plan,
                         ws=ws[:16])
    assert e.value.status == binding.SPMM_ERR_WORKSPACE
    plan.close()


def test_validator():
    A = inputs.uniform_csr(100, 50, 4, seed=26).to("cuda")
    ws = binding.workspace(256)
    binding.spmm_csr_validate(A.rowptr, A.colind, 100, 50, A.nnz, ws)
    assert binding.spmm_get_device_status(ws) == 0
    bad_col = A.colind.clone()
    bad_col[17] = 50
    binding.spmm_csr_validate(A.rowptr, bad_col, 100, 50, A.nnz, ws)
    assert binding.spmm_get_device_status(ws) == binding.SPMM_ERR_BAD_CSR
    bad_rp = A.rowptr.clone()
    bad_rp[40] = bad_rp[41] + 1
    binding.spmm_csr_validate(bad_rp, A.colind, 100, 50, A.nnz, ws)
    assert binding.spmm_get_device_status(ws) == binding.SPMM_ERR_BAD_CSR
    binding.spmm_csr_validate(A.rowptr, A.colind, 100, 50, A.nnz - 1, ws)
    assert binding.spmm_get_device_status(ws) == binding.SPMM_ERR_BAD_CSR
    neg = A.colind.clone()
    neg[0] = -1
    binding.spmm_csr_validate(A.rowptr, neg, 100, 50, A.nnz, ws)
    assert binding.spmm_get_device_status(ws) == binding.SPMM_ERR_BAD_CSR
    # status clears after reading
    assert binding.spmm_get_device_status(ws) == 0


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("tile_order", [0, 9, 16])
def test_every_unit_reserved_exactly_once_under_imbalance(tile_order, kernel):
    """Work reservation (Section 3.4): with one huge row and many empty ones on a
    16 x 4 grid, the result equals the oracle, so every chunk of every tile was
    processed exactly once (a missed unit leaves NaN, a doubled one doubles)."""
    M, K, N = 4096, 4096, 32
    rng = np.random.default_rng(27)
    lens = np.zeros(M, np.int64)
    lens[0] = 4000
    lens[1::3] = 2
    rowptr = np.zeros(M + 1, np.int64)
    rowptr[1:] = np.cumsum(lens)
    colind = np.concatenate([np.sort(rng.choice(K, l, replace=False)) for l in lens if l])
    A = CSR(torch.from_numpy(rowptr.astype(np.int32)), torch.from_numpy(colind.astype(np.int32)),
            torch.ones(colind.size), M, K)
    B = torch.ones(K, N)
    C, st = run_spmm(A, B, N, tile_rows=16, tile_cols=4, chunk_items=32, tile_order=tile_order,
                     kernel=kernel)
    assert st == 0
    assert torch.equal(C[:, 0], torch.from_numpy(lens.astype(np.float32)))


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("tile_order", [0, 16])
def test_trace_records_account_for_every_unit(tile_order, kernel):
    """A traced launch computes the same C bit for bit; its per-warp records
    cover every work unit once (units of G = 32/LPN chunks per tile, summed over
    tiles), stolen units are a subset, times are ordered and SM ids valid."""
    A = inputs.rmat_csr(14, 16, seed=77)
    N, TR, TC = 128, 16, 4
    # a column block is 32 FP32 values: 8 lanes of 16 bytes (G = 4 groups per
    # warp) in the staged kernel, 4 lanes of 32 bytes (G = 8) in the wide one
    G = 4 if kernel == binding.SPMM_KERNEL_STAGED else 8   # wide: N=128, TC=4 qualifies
    Ad = A.to("cuda")
    B = inputs.dense_normal(A.K, N, seed=78, device="cuda")
    plan = binding.Plan(Ad.rowptr, A.M, A.K, A.nnz, N, TR, TC,
                        tuning=binding.make_tuning(tile_order=tile_order, kernel=kernel))
    ws = binding.workspace(plan.workspace_bytes)
    C0 = torch.empty(A.M, N, device="cuda")
    binding.spmm_csr(Ad.rowptr, Ad.colind, Ad.vals, B, C0, A.M, A.K, N, A.nnz, plan=plan, ws=ws)
    buf = binding.trace_buffer(1 << 15)
    plan.set_trace(buf)
    C1 = torch.empty_like(C0)
    binding.spmm_csr(Ad.rowptr, Ad.colind, Ad.vals, B, C1, A.M, A.K, N, A.nnz, plan=plan, ws=ws)
    torch.cuda.synchronize()
    assert binding.spmm_get_device_status(ws) == 0
    assert torch.equal(C0, C1)
    rec = binding.read_trace(buf)
    assert rec.size > 0
    # units: per row block, ceil(chunks / G) units in each of the TC column blocks
    chunks, _ = plan.units()
    total = int(rec["units"].sum())
    assert chunks * TC / G <= total <= chunks * TC / G + TR * TC
    assert np.all(rec["stolen"] <= rec["units"]) and np.all(rec["stolen"] >= 0)
    assert np.all(rec["t_end_ns"] >= rec["t_start_ns"]) and np.all(rec["t_start_ns"] > 0)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert np.all((rec["smid"] >= 0) & (rec["smid"] < sms))
    # tracing off: the buffer is left alone
    plan.set_trace(None)
    buf.zero_()
    binding.spmm_csr(Ad.rowptr, Ad.colind, Ad.vals, B, C1, A.M, A.K, N, A.nnz, plan=plan, ws=ws)
    torch.cuda.synchronize()
    assert torch.count_nonzero(buf) == 0
    plan.close()


@pytest.mark.parametrize("warps", [0, 5, 8])
def test_cta_size_of_the_persistent_grid(warps):
    """The launch fills every SM with whole CTAs of the requested size; the
    default (0) is 7-warp CTAs, four per SM, where they fit the registers and
    shared memory, else 8-warp CTAs, three per SM. With short chunks there are
    more warp units than resident warps, so the grid is not cut short, and the
    trace holds one record per launched warp."""
    A = inputs.rmat_csr(14, 16, seed=79)
    N, TR, TC = 128, 16, 4
    Ad = A.to("cuda")
    B = inputs.dense_normal(A.K, N, seed=80, device="cuda")
    plan = binding.Plan(Ad.rowptr, A.M, A.K, A.nnz, N, TR, TC,
                        tuning=binding.make_tuning(chunk_items=32, warps_per_cta=warps,
                                                   tile_order=16))
    ws = binding.workspace(plan.workspace_bytes)
    buf = binding.trace_buffer(1 << 15)
    plan.set_trace(buf)
    C = torch.empty(A.M, N, device="cuda")
    binding.spmm_csr(Ad.rowptr, Ad.colind, Ad.vals, B, C, A.M, A.K, N, A.nnz, plan=plan, ws=ws)
    torch.cuda.synchronize()
    assert binding.spmm_get_device_status(ws) == 0
    rec = binding.read_trace(buf)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    chunks, _ = plan.units()
    assert chunks * TC // 4 > sms * 32   # more warp units (4 chunks each) than warps
    assert rec.size % sms == 0
    per_sm = rec.size // sms
    if warps == 0:
        assert per_sm in (28, 24)
    elif warps == 5:
        assert per_sm == 25   # 5 CTAs: 5 x (40 KB of staging + 1 KB) fit 228 KB
    else:
        assert per_sm == 24   # 3 CTAs: a fourth 64 KB of staging does not fit
    ref, bound = ref_and_bound(A, B.cpu())
    assert_close_rel(C.cpu().numpy(), ref, bound, TOL_F32, f"warps={warps}")
    plan.set_trace(None)
    plan.close()
