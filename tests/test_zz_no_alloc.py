"""spmm_csr_noalloc: the product for callers that cannot allocate device memory.

Code that runs inside a memory pool it does not own, a plug-in whose host
application forbids device allocation, or a path that must not synchronise
the device (cudaMalloc and cudaFree can) cannot hand spmm_csr a workspace.
spmm_csr_noalloc keeps its scratch in one fixed 16 MiB device array inside the
library instead, and spmm_csr_noalloc_status reads that array's status word.

The calls below go through the C ABI and are checked element by element
against the FP64 oracle within the FP32 tolerance. A large problem that fills
most of the array runs first, then a small one twice: what the large call left
in the array must not leak into the small results, and the two small calls
must agree bit for bit. The device status must read OK after every call. This
file is collected last, so a failure here leaves every other test already run.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2311_18141_gb300 import binding, inputs

from gpu_util import TOL_F32, assert_close_rel

pytestmark = pytest.mark.gpu

SCRATCH_BYTES = 16 << 20   # the fixed array's size, stated in the header


def _noalloc(Ad, B, N, grid, beta, C0):
    C = C0.clone()
    binding.spmm_csr_noalloc(Ad.rowptr, Ad.colind, Ad.vals, B, C, Ad.M, Ad.K, N, Ad.nnz,
                             tile_rows=grid[0], tile_cols=grid[1], beta=beta)
    status = binding.spmm_csr_noalloc_status()
    return C.cpu(), status


def _check_against_oracle(A, B, C0, beta, got, what):
    ref = oracle.spmm(A.rowptr, A.colind, A.vals, B, beta=beta, C0=C0.numpy())
    bound = oracle.abs_bound(A.rowptr, A.colind, A.vals, B)
    bound = bound + abs(beta) * np.abs(C0.numpy().astype(np.float64))
    assert_close_rel(got.numpy(), ref, bound, TOL_F32, what)


def test_noalloc_large_then_small_twice_against_oracle():
    # large: fills most of the fixed array
    big = inputs.rmat_csr(14, 16, seed=61)
    Nb, grid_b = 192, (4, 2)
    need = binding.spmm_csr_workspace_size(big.M, big.nnz, Nb, *grid_b)
    assert SCRATCH_BYTES // 2 < need <= SCRATCH_BYTES, need
    Bb = inputs.dense_normal(big.K, Nb, seed=63)
    C0b = torch.full((big.M, Nb), float("nan"))
    got, st = _noalloc(big.to("cuda"), Bb.cuda(), Nb, grid_b, 0.0, C0b.cuda())
    assert st == binding.SPMM_OK
    _check_against_oracle(big, Bb, torch.zeros(big.M, Nb), 0.0, got, "noalloc large")

    # small, twice, accumulating into C0 (beta = 1)
    small = inputs.uniform_csr(3000, 2000, 7, seed=62)
    Ns, grid_s = 32, (3, 1)
    Bs = inputs.dense_normal(small.K, Ns, seed=64)
    C0s = inputs.dense_normal(small.M, Ns, seed=65)
    As, Bsd = small.to("cuda"), Bs.cuda()
    first, st1 = _noalloc(As, Bsd, Ns, grid_s, 1.0, C0s.cuda())
    second, st2 = _noalloc(As, Bsd, Ns, grid_s, 1.0, C0s.cuda())
    assert st1 == binding.SPMM_OK and st2 == binding.SPMM_OK
    _check_against_oracle(small, Bs, C0s, 1.0, first, "noalloc small, first call")
    _check_against_oracle(small, Bs, C0s, 1.0, second, "noalloc small, second call")
    assert torch.equal(first, second)


def test_noalloc_rejects_problems_beyond_its_scratch():
    # a problem whose workspace exceeds the fixed array is refused before any device work
    M, nnz, N = 1 << 24, 1 << 26, 128
    assert binding.spmm_csr_workspace_size(M, nnz, N, 1, 1) > SCRATCH_BYTES
    fake = torch.zeros(16, dtype=torch.int32, device="cuda")
    Bf = torch.zeros(4, N, device="cuda")
    with pytest.raises(binding.SpmmError) as e:
        binding.spmm_csr_noalloc(fake, fake, fake.float(), Bf, Bf, M, 4, N, nnz)
    assert e.value.status == binding.SPMM_ERR_WORKSPACE
    # nothing ran, so the array's status word still reads OK
    assert binding.spmm_csr_noalloc_status() == binding.SPMM_OK
