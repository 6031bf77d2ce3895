"""GCN-style layer C = A_hat (X W) through the autograd Function: forward and
hand-written backward (dB = A_hat^T dC via the device transpose, dA_vals =
SDDMM(dC, B^T)) against the FP64 oracle, and against FP64 central finite
differences of L = sum(dC * C) on the 2,048-node induced subgraph."""
import numpy as np
import pytest
import torch

import oracle
from paper_2311_18141_gb300 import autograd as ag
from paper_2311_18141_gb300 import inputs

from gpu_util import TOL_F32, assert_close_rel

pytestmark = pytest.mark.gpu


def run_layer(A, X, W, dC, tile_rows=1):
    torch.backends.cuda.matmul.allow_tf32 = False
    Ad = A.to("cuda")
    S = ag.SparseCSR(Ad.rowptr, Ad.colind, A.M, A.K, tile_rows=tile_rows)
    vals = Ad.vals.clone().requires_grad_(True)
    Xd = X.cuda()
    Wd = W.cuda().requires_grad_(True)
    B = (Xd @ Wd).detach().requires_grad_(True)
    C = ag.spmm(S, vals, B)
    (C * dC.cuda()).sum().backward()
    torch.cuda.synchronize()
    return C.detach().cpu(), vals.grad.cpu(), B.grad.cpu(), B.detach().cpu()


def check_against_oracle(A, C, dvals, dB, B, dC):
    ref = oracle.spmm(A.rowptr, A.colind, A.vals, B)
    assert_close_rel(C.numpy(), ref, oracle.abs_bound(A.rowptr, A.colind, A.vals, B), TOL_F32,
                     "forward")
    absv = np.abs(A.vals.numpy().astype(np.float64))
    absdC = np.abs(dC.numpy().astype(np.float64))
    dB64 = oracle.spmm_t_push(A.rowptr, A.colind, A.vals, dC, A.K)
    assert_close_rel(dB.numpy(), dB64, oracle.spmm_t_push(A.rowptr, A.colind, absv, absdC, A.K),
                     TOL_F32, "dB")
    dv64 = oracle.sddmm(A.rowptr, A.colind, dC, B)
    assert_close_rel(dvals.numpy(), dv64,
                     oracle.sddmm(A.rowptr, A.colind, absdC, np.abs(B.numpy().astype(np.float64))),
                     TOL_F32, "dvals")
    return dB64, dv64


def test_gcn_subgraph_2048_finite_differences():
    A = inputs.gcn_induced_subgraph(18, 2048, 16, seed=4)
    X = inputs.dense_normal(A.M, 128, seed=51)
    W = inputs.glorot_uniform(128, 64, seed=52)
    dC = inputs.dense_normal(A.M, 64, seed=53)
    C, dvals, dB, B = run_layer(A, X, W, dC)
    dB64, dv64 = check_against_oracle(A, C, dvals, dB, B, dC)

    Bn = B.numpy().astype(np.float64)
    vn = A.vals.numpy().astype(np.float64)
    dCn = dC.numpy().astype(np.float64)

    def loss(vv, BB):
        return float((dCn * oracle.spmm(A.rowptr, A.colind, vv, BB)).sum())

    rng = np.random.default_rng(54)
    h = 1e-3
    for _ in range(48):
        k, n = int(rng.integers(A.K)), int(rng.integers(64))
        Bp, Bm = Bn.copy(), Bn.copy()
        Bp[k, n] += h
        Bm[k, n] -= h
        fd = (loss(vn, Bp) - loss(vn, Bm)) / (2 * h)
        scale = float(np.abs(A.vals.numpy()[A.colind.numpy() == k]).sum() * np.abs(dCn).max()) + 1e-30
        assert abs(fd - dB64[k, n]) <= 1e-7 * scale + 1e-9
        assert abs(float(dB[k, n]) - fd) <= 1e-5 * scale + 1e-7
    for _ in range(48):
        e = int(rng.integers(A.nnz))
        vp, vm = vn.copy(), vn.copy()
        vp[e] += h
        vm[e] -= h
        fd = (loss(vp, Bn) - loss(vm, Bn)) / (2 * h)
        assert abs(fd - dv64[e]) <= 1e-7 * (abs(dv64[e]) + 1)
        assert abs(float(dvals[e]) - fd) <= 1e-5 * (np.abs(dCn).sum(1).max() * np.abs(Bn).max())


def test_gcn_full_scale18_forward_backward():
    """The differentiation workload: symmetrised R-MAT scale 18 (262,144 nodes),
    X 262,144 x 128, W 128 x 64, dC N(0,1)."""
    A = inputs.gcn_normalized_adjacency(18, 16, seed=4)
    X = inputs.dense_normal(A.M, 128, seed=55)
    W = inputs.glorot_uniform(128, 64, seed=56)
    dC = inputs.dense_normal(A.M, 64, seed=57)
    C, dvals, dB, B = run_layer(A, X, W, dC, tile_rows=8)
    check_against_oracle(A, C, dvals, dB, B, dC)


def test_nonsymmetric_backward():
    A = inputs.rmat_csr(13, 16, seed=58, values="sym")
    B = inputs.dense_normal(A.K, 32, seed=59)
    dC = inputs.dense_normal(A.M, 32, seed=60)
    Ad = A.to("cuda")
    S = ag.SparseCSR(Ad.rowptr, Ad.colind, A.M, A.K, tile_rows=4, tile_cols=2)
    vals = Ad.vals.clone().requires_grad_(True)
    Bd = B.cuda().requires_grad_(True)
    C = ag.spmm(S, vals, Bd)
    (C * dC.cuda()).sum().backward()
    check_against_oracle(A, C.detach().cpu(), vals.grad.cpu(), Bd.grad.cpu(), B, dC)
