"""Backward pieces on the GPU: CSR->CSC transpose (bit-exact against the
oracle's stable transpose), dB = A^T dC through the transpose and the SpMM
kernel, and SDDMM at A's pattern, against the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2311_18141_gb300 import binding, inputs
from paper_2311_18141_gb300.inputs import CSR

from gpu_util import TOL_F32, assert_close_rel, run_spmm

pytestmark = pytest.mark.gpu


def transpose_gpu(A, with_vals=True):
    Ad = A.to("cuda")
    colptr = torch.empty(A.K + 1, dtype=torch.int32, device="cuda")
    rowind = torch.empty(max(A.nnz, 1), dtype=torch.int32, device="cuda")
    tv = torch.empty(max(A.nnz, 1), dtype=Ad.vals.dtype, device="cuda") if with_vals else None
    perm = torch.empty(max(A.nnz, 1), dtype=torch.int32, device="cuda")
    ws = binding.workspace(binding.spmm_csr_transpose_workspace_size(A.M, A.K, A.nnz))
    binding.spmm_csr_transpose(Ad.rowptr, Ad.colind, Ad.vals, A.M, A.K, A.nnz, colptr, rowind,
                               tv, perm, ws)
    torch.cuda.synchronize()
    n = A.nnz
    return (colptr.cpu(), rowind.cpu()[:n], None if tv is None else tv.cpu()[:n],
            perm.cpu()[:n])


# column keys of 12, 15, 17, 9, 21 and 26 bits: two 8-bit passes, two 9-bit
# passes, one 9-bit pass, three 8-bit passes and three 9-bit passes
@pytest.mark.parametrize("shape", [("rmat", 12), ("rmat", 15), ("uniform", (3000, 70000, 9)),
                                   ("gcn", 12), ("uniform", (2000, 300, 7)),
                                   ("uniform", (1500, (1 << 20) + 77, 4)),
                                   ("uniform", (1200, (1 << 25) + 12345, 5))])
def test_transpose_bit_exact(shape):
    kind, s = shape
    if kind == "rmat":
        A = inputs.rmat_csr(s, 16, seed=41)
    elif kind == "gcn":
        A = inputs.gcn_normalized_adjacency(s, 16, seed=42)
    else:
        M, K, per_row = s
        A = inputs.uniform_csr(M, K, per_row, seed=43)
    colptr, rowind, tv, perm = transpose_gpu(A)
    c_ref, r_ref, v_ref, p_ref = oracle.csr_transpose(A.rowptr, A.colind, A.vals, A.K)
    np.testing.assert_array_equal(colptr.numpy(), c_ref)
    np.testing.assert_array_equal(rowind.numpy(), r_ref)
    np.testing.assert_array_equal(perm.numpy(), p_ref)
    np.testing.assert_array_equal(tv.numpy().astype(np.float64), v_ref)


def test_transpose_empty_and_single():
    A = CSR(torch.zeros(11, dtype=torch.int32), torch.zeros(0, dtype=torch.int32),
            torch.zeros(0), 10, 6)
    colptr, rowind, tv, perm = transpose_gpu(A)
    assert torch.equal(colptr, torch.zeros(7, dtype=torch.int32))
    A = CSR(torch.tensor([0, 0, 1], dtype=torch.int32), torch.tensor([2], dtype=torch.int32),
            torch.tensor([5.0]), 2, 3)
    colptr, rowind, tv, perm = transpose_gpu(A)
    assert colptr.tolist() == [0, 0, 0, 1] and rowind.tolist() == [1] and tv.tolist() == [5.0]


def test_gather_values_matches_transpose():
    A = inputs.rmat_csr(12, 8, seed=44)
    colptr, rowind, tv, perm = transpose_gpu(A)
    out = torch.empty(A.nnz, device="cuda")
    binding.spmm_gather_values(A.vals.cuda(), perm.cuda(), A.nnz, out)
    torch.cuda.synchronize()
    assert torch.equal(out.cpu(), tv)


@pytest.mark.parametrize("sym", [False, True])
def test_dB_through_transpose(sym):
    # a non-symmetric A catches transpose mistakes a symmetric one would hide
    A = inputs.gcn_normalized_adjacency(12, 16, seed=45) if sym else inputs.rmat_csr(12, 16, seed=46)
    N = 64
    dC = inputs.dense_normal(A.M, N, seed=47)
    colptr, rowind, tv, _ = transpose_gpu(A)
    At = CSR(colptr, rowind, tv, A.K, A.M)
    dB, st = run_spmm(At, dC, N, tile_rows=4, chunk_items=256)
    assert st == 0
    ref = oracle.spmm_t_push(A.rowptr, A.colind, A.vals, dC, A.K)
    bound = oracle.spmm_t_push(A.rowptr, A.colind, np.abs(A.vals.numpy().astype(np.float64)),
                               np.abs(dC.numpy().astype(np.float64)), A.K)
    assert_close_rel(dB.numpy(), ref, bound, TOL_F32, "dB = A^T dC")


@pytest.mark.parametrize("N,bdtype", [(8, torch.float32), (16, torch.float32),
                                       (32, torch.float32), (64, torch.float32),
                                       (128, torch.float32), (256, torch.float32),
                                       (512, torch.float32), (16, torch.bfloat16),
                                       (64, torch.bfloat16), (256, torch.bfloat16),
                                       (512, torch.bfloat16)])
@pytest.mark.parametrize("use_plan", [False, True])
def test_sddmm(N, bdtype, use_plan):
    """Every lane shape (2 to 32 lanes, 1 to 4 vectors per lane), with the dC
    row held in registers (narrow shapes) or staged per nonzero (wide ones),
    FP32 and BF16 B, against the FP64 oracle on the stored inputs."""
    A = inputs.rmat_csr(12, 16, seed=48)
    dC = inputs.dense_normal(A.M, N, seed=49)
    B = inputs.dense_normal(A.K, N, seed=50).to(bdtype)
    Ad = A.to("cuda")
    out = torch.full((A.nnz,), float("nan"), device="cuda")
    if use_plan:
        plan = binding.Plan(Ad.rowptr, A.M, A.K, A.nnz, N, tile_rows=8, tile_cols=1,
                            tuning=binding.make_tuning(chunk_items=150))
        ws = binding.workspace(plan.workspace_bytes)
    else:
        plan = None
        ws = binding.workspace(binding.spmm_csr_workspace_size(A.M, A.nnz, N, 1, 1))
    binding.spmm_sddmm_csr(Ad.rowptr, Ad.colind, dC.cuda(), B.cuda(), out, A.M, A.K, N, A.nnz,
                           plan=plan, ws=ws)
    torch.cuda.synchronize()
    assert binding.spmm_get_device_status(ws) == 0
    if bdtype == torch.bfloat16:
        B64 = oracle.decode_bf16(B.view(torch.int16).numpy().view(np.uint16))
    else:
        B64 = B.numpy().astype(np.float64)
    ref = oracle.sddmm(A.rowptr, A.colind, dC, B64)
    bound = oracle.sddmm(A.rowptr, A.colind, np.abs(dC.numpy().astype(np.float64)), np.abs(B64))
    assert_close_rel(out.cpu().numpy(), ref, bound, TOL_F32, f"sddmm N={N} {bdtype}")
    if plan is not None:
        plan.close()
