"""spmm_csr_noalloc: the entry point for callers that cannot allocate device
memory (it keeps its scratch in a fixed device array inside the library).

Two calls in a row, through the C ABI, must match spmm_csr with a caller
workspace within the FP32 tolerance; the second call also checks that the
array's leftover contents from the first call do not leak into the result.
This file is collected last so that a failure here leaves every other test
already run."""
import numpy as np
import pytest
import torch

from paper_2311_18141_gb300 import binding, inputs

from gpu_util import TOL_F32, assert_close_rel

pytestmark = pytest.mark.gpu


def _reference(Ad, B, N, grid, beta, C0):
    C = C0.clone()
    ws = binding.workspace(binding.spmm_csr_workspace_size(Ad.M, Ad.nnz, N, *grid))
    binding.spmm_csr(Ad.rowptr, Ad.colind, Ad.vals, B, C, Ad.M, Ad.K, N, Ad.nnz,
                     tile_rows=grid[0], tile_cols=grid[1], beta=beta, ws=ws)
    return C


def _noalloc(Ad, B, N, grid, beta, C0):
    C = C0.clone()
    binding.spmm_csr_noalloc(Ad.rowptr, Ad.colind, Ad.vals, B, C, Ad.M, Ad.K, N, Ad.nnz,
                             tile_rows=grid[0], tile_cols=grid[1], beta=beta)
    return C


def test_noalloc_matches_workspace_entry_point_twice():
    cases = [
        (inputs.rmat_csr(13, 16, seed=61).to("cuda"), 64, (8, 2), 0.0),
        (inputs.uniform_csr(3000, 2000, 7, seed=62).to("cuda"), 32, (3, 1), 1.0),
    ]
    for A, N, grid, beta in cases:
        B = inputs.dense_normal(A.K, N, seed=63, device="cuda")
        C0 = inputs.dense_normal(A.M, N, seed=64, device="cuda")
        ref = _reference(A, B, N, grid, beta, C0)
        got = _noalloc(A, B, N, grid, beta, C0)
        torch.cuda.synchronize()
        absA = A.vals.abs().cpu().numpy().astype(np.float64)
        rows = np.repeat(np.arange(A.M), A.row_lengths().cpu().numpy())
        absB = B.abs().cpu().numpy().astype(np.float64)
        bound = np.zeros((A.M, N))
        np.add.at(bound, rows, absA[:, None] * absB[A.colind.cpu().numpy()])
        bound += abs(beta) * C0.abs().cpu().numpy()
        assert_close_rel(got.cpu().numpy(), ref.cpu().numpy().astype(np.float64), 2 * bound,
                         TOL_F32, "noalloc vs spmm_csr")


def test_noalloc_rejects_problems_beyond_its_scratch():
    # a problem whose workspace exceeds the fixed array is refused before any device work
    M, nnz, N = 1 << 24, 1 << 26, 128
    assert binding.spmm_csr_workspace_size(M, nnz, N, 1, 1) > (16 << 20)
    fake = torch.zeros(16, dtype=torch.int32, device="cuda")
    Bf = torch.zeros(4, N, device="cuda")
    with pytest.raises(binding.SpmmError) as e:
        binding.spmm_csr_noalloc(fake, fake, fake.float(), Bf, Bf, M, 4, N, nnz)
    assert e.value.status == binding.SPMM_ERR_WORKSPACE
