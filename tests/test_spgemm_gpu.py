"""Local SpGEMM C = A*B on the GPU against the FP64 oracle: structure (row
pointers and column indices) bit-exact, values within 1e-5 * (|A||B|) per entry,
results reproducible, explicit zeros kept, empty operands and bad indices."""
import numpy as np
import pytest
import torch

import oracle
from paper_2311_18141_gb300 import binding, inputs

from gpu_util import TOL_F32, assert_close_rel

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _gpu(rp, ci, v):
    return (torch.as_tensor(np.asarray(rp, np.int32), device=DEV),
            torch.as_tensor(np.asarray(ci, np.int32), device=DEV),
            torch.as_tensor(np.asarray(v, np.float32), device=DEV))


def _check(a, b, M, K, N):
    A = _gpu(*a)
    B = _gpu(*b)
    rp, ci, v, P = binding.spgemm(A[0], A[1], A[2], M, K, B[0], B[1], B[2], N)
    torch.cuda.synchronize()
    av = np.asarray(a[2], np.float32).astype(np.float64)
    bv = np.asarray(b[2], np.float32).astype(np.float64)
    erp, eci, ev = oracle.spgemm(a[0], a[1], av, b[0], b[1], bv, K, N)
    _, _, bound = oracle.spgemm(a[0], a[1], np.abs(av), b[0], b[1], np.abs(bv), K, N)
    np.testing.assert_array_equal(rp.cpu().numpy(), erp)
    np.testing.assert_array_equal(ci.cpu().numpy(), eci)
    assert_close_rel(v.cpu().numpy().astype(np.float64), ev, bound, TOL_F32, "spgemm values")
    a_rows = np.diff(np.asarray(a[0], np.int64))
    b_rows = np.diff(np.asarray(b[0], np.int64))
    assert P == int(b_rows[np.asarray(a[1], np.int64)].sum()) if a_rows.sum() else P == 0
    return rp, ci, v


@pytest.mark.parametrize("scale", [8, 10, 12])
def test_rmat_square(scale):
    A = inputs.rmat_csr(scale, 16, seed=31, values="pos")
    a = (A.rowptr.numpy(), A.colind.numpy(), A.vals.numpy())
    _check(a, a, A.M, A.K, A.K)


def test_rectangular_with_empty_rows_duplicates_and_signs():
    rng = np.random.default_rng(5)
    M, K, N = 300, 200, 150
    def rand_csr(R, C, p, dup):
        rows = []
        for i in range(R):
            cs = np.flatnonzero(rng.random(C) < p)
            if i % 7 == 0:
                cs = cs[:0]
            if dup and cs.size:
                cs = np.sort(np.concatenate([cs, cs[:2]]))
            rows.append(cs)
        rp = np.zeros(R + 1, np.int64)
        rp[1:] = np.cumsum([c.size for c in rows])
        ci = np.concatenate(rows).astype(np.int32)
        return rp.astype(np.int32), ci, rng.standard_normal(ci.size).astype(np.float32)
    a = rand_csr(M, K, 0.05, True)
    b = rand_csr(K, N, 0.08, False)
    _check(a, b, M, K, N)


def test_explicit_zeros_and_empty_operands():
    a = (np.array([0, 1, 1], np.int32), np.array([0], np.int32), np.array([0.0], np.float32))
    b = (np.array([0, 2], np.int32), np.array([0, 1], np.int32), np.array([1.0, 2.0], np.float32))
    rp, ci, v = _check(a, b, 2, 1, 2)
    assert v.cpu().tolist() == [0.0, 0.0]
    empty = (np.zeros(4, np.int32), np.zeros(0, np.int32), np.zeros(0, np.float32))
    _check(empty, b, 3, 1, 2)
    b_empty = (np.zeros(2, np.int32), np.zeros(0, np.int32), np.zeros(0, np.float32))
    _check(a, b_empty, 2, 1, 2)


def test_reproducible_bitwise():
    A = inputs.rmat_csr(11, 16, seed=32, values="pos")
    Ad = A.to(DEV)
    r1 = binding.spgemm(Ad.rowptr, Ad.colind, Ad.vals, A.M, A.K, Ad.rowptr, Ad.colind, Ad.vals, A.K)
    r2 = binding.spgemm(Ad.rowptr, Ad.colind, Ad.vals, A.M, A.K, Ad.rowptr, Ad.colind, Ad.vals, A.K)
    torch.cuda.synchronize()
    for x, y in zip(r1[:3], r2[:3]):
        assert torch.equal(x, y)


def test_column_out_of_range_is_reported():
    a = _gpu(np.array([0, 1], np.int32), np.array([5], np.int32), np.array([1.0], np.float32))
    b = _gpu(np.array([0, 1, 1], np.int32), np.array([0], np.int32), np.array([1.0], np.float32))
    with pytest.raises(binding.SpmmError) as e:
        binding.spgemm(a[0], a[1], a[2], 1, 2, b[0], b[1], b[2], 1)
    assert e.value.status == binding.SPMM_ERR_BAD_CSR


def test_wide_shapes_take_the_two_sort_path():
    # bits(M) + bits(N) > 32: products are sorted by column, then by row
    rng = np.random.default_rng(9)
    M, K, N = 100_000, 64, 90_000
    a_rows = rng.integers(0, 3, M)
    a_rp = np.zeros(M + 1, np.int64)
    a_rp[1:] = np.cumsum(a_rows)
    a_ci = np.concatenate([np.sort(rng.choice(K, n, replace=False)) for n in a_rows]).astype(np.int32)
    b_rows = rng.integers(0, 6, K)
    b_rp = np.zeros(K + 1, np.int64)
    b_rp[1:] = np.cumsum(b_rows)
    b_ci = np.concatenate([np.sort(rng.choice(N, n, replace=False)) for n in b_rows]).astype(np.int32)
    a = (a_rp.astype(np.int32), a_ci, rng.standard_normal(a_ci.size).astype(np.float32))
    b = (b_rp.astype(np.int32), b_ci, rng.standard_normal(b_ci.size).astype(np.float32))
    _check(a, b, M, K, N)
