"""torch.autograd.Function over the C ABI: C = A*B with a hand-written backward.

For L(C), with A's pattern fixed:
  dB      = A^T dC                 SpMM on A^T, whose CSR is A's CSC built once on
                                   the device by spmm_csr_transpose; its values are
                                   re-gathered from A's current values through the
                                   stored permutation at every backward.
  dA_vals = SDDMM(dC, B^T)         dA_vals[e] = <dC[row_e, :], B[col_e, :]>.
Both run in the CUDA library; this module only allocates and marshals.
"""
from __future__ import annotations

import torch

from . import binding


class SparseCSR:
    """A's pattern on the device, with cached plans, transpose and workspaces."""

    def __init__(self, rowptr: torch.Tensor, colind: torch.Tensor, M: int, K: int,
                 tile_rows: int = 1, tile_cols: int = 1):
        self.rowptr = rowptr.contiguous()
        self.colind = colind.contiguous()
        self.M, self.K = int(M), int(K)
        self.nnz = int(colind.numel())
        self.tile_rows, self.tile_cols = int(tile_rows), int(tile_cols)
        self._plans = {}
        self._ws = {}
        self._t = None

    def plan(self, N: int, transpose: bool = False, sddmm: bool = False):
        key = (N, transpose, sddmm)
        if key not in self._plans:
            if transpose:
                colptr, rowind, _ = self.transpose_pattern()
                p = binding.Plan(colptr, self.K, self.M, self.nnz, N, self.tile_rows, 1)
            else:
                p = binding.Plan(self.rowptr, self.M, self.K, self.nnz, N, self.tile_rows,
                                 1 if sddmm else self.tile_cols)
            self._plans[key] = p
            self._ws[key] = binding.workspace(p.workspace_bytes, self.rowptr.device)
        return self._plans[key], self._ws[key]

    def transpose_pattern(self):
        """(colptr, rowind, perm) of A^T, built once by spmm_csr_transpose."""
        if self._t is None:
            dev = self.rowptr.device
            colptr = torch.empty(self.K + 1, dtype=torch.int32, device=dev)
            n = max(self.nnz, 1)
            rowind = torch.empty(n, dtype=torch.int32, device=dev)
            perm = torch.empty(n, dtype=torch.int32, device=dev)
            ws = binding.workspace(
                binding.spmm_csr_transpose_workspace_size(self.M, self.K, self.nnz), dev)
            binding.spmm_csr_transpose(self.rowptr, self.colind, None, self.M, self.K, self.nnz,
                                       colptr, rowind, None, perm, ws)
            self._t = (colptr, rowind, perm)
        return self._t


class SpmmCSRFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vals: torch.Tensor, B: torch.Tensor, A: SparseCSR):
        B = B.contiguous()
        N = B.shape[1]
        C = torch.empty(A.M, N, dtype=torch.float32, device=B.device)
        plan, ws = A.plan(N)
        binding.spmm_csr(A.rowptr, A.colind, vals, B, C, A.M, A.K, N, A.nnz, plan=plan, ws=ws)
        ctx.save_for_backward(vals, B)
        ctx.A = A
        return C

    @staticmethod
    def backward(ctx, dC: torch.Tensor):
        vals, B = ctx.saved_tensors
        A: SparseCSR = ctx.A
        dC = dC.contiguous().to(torch.float32)
        N = dC.shape[1]
        dvals = dB = None
        if ctx.needs_input_grad[0]:
            dvals = torch.empty(A.nnz, dtype=torch.float32, device=dC.device)
            plan, ws = A.plan(N, sddmm=True)
            binding.spmm_sddmm_csr(A.rowptr, A.colind, dC, B, dvals, A.M, A.K, N, A.nnz,
                                   plan=plan, ws=ws)
            dvals = dvals.to(vals.dtype)
        if ctx.needs_input_grad[1]:
            colptr, rowind, perm = A.transpose_pattern()
            vt = torch.empty(max(A.nnz, 1), dtype=vals.dtype, device=vals.device)
            binding.spmm_gather_values(vals, perm, A.nnz, vt)
            dB = torch.empty(A.K, N, dtype=torch.float32, device=dC.device)
            plan, ws = A.plan(N, transpose=True)
            binding.spmm_csr(colptr, rowind, vt, dC, dB, A.K, A.M, N, A.nnz, plan=plan, ws=ws)
            dB = dB.to(B.dtype)
        return dvals, dB, None


def spmm(A: SparseCSR, vals: torch.Tensor, B: torch.Tensor) -> torch.Tensor:
    """Differentiable C = A*B (gradients for vals and B)."""
    return SpmmCSRFunction.apply(vals, B, A)


def gcn_layer(A: SparseCSR, a_vals: torch.Tensor, X: torch.Tensor, W: torch.Tensor) -> torch.Tensor:
    """GCN propagation C = A_hat (X W): the dense X W is a plain library GEMM,
    the sparse product and its backward run in the CUDA library."""
    return spmm(A, a_vals, X @ W)
