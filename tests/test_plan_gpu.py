"""The merge-path plan, bit for bit: chunk counts per row block and every chunk
boundary (rows finished, nonzeros consumed), against a brute-force walk of each
row block's merge path item by item, including the move of a boundary that
falls inside a light row (fewer than D/8 items) back to the row's start."""
import math

import numpy as np
import pytest
import torch

from paper_2311_18141_gb300 import binding, inputs
from paper_2311_18141_gb300.inputs import CSR

pytestmark = pytest.mark.gpu


def brute_force_plan(rowptr, M, TR, D):
    rp = [int(x) for x in rowptr]
    RB = max(1, -(-M // TR))
    counts, points = [], []
    for i in range(TR):
        lo, hi = min(M, i * RB), min(M, i * RB + RB)
        nlo = rp[lo]
        is_end = []                       # the block's merge path: nonzeros, then the row end
        for r in range(lo, hi):
            is_end += [False] * (rp[r + 1] - rp[r]) + [True]
        total = len(is_end)
        ends_before = np.concatenate([[0], np.cumsum(is_end)]) if total else np.zeros(1, int)
        chunks = math.ceil(total / D)
        counts.append(chunks)
        for c in range(chunks + 1):
            d = min(c * D, total)
            x = int(ends_before[d])       # rows finished before item d
            y = d - x                     # nonzeros consumed
            if x < hi - lo:
                rs, re = rp[lo + x] - nlo, rp[lo + x + 1] - nlo
                if y > rs and 8 * (re - rs + 1) < D:
                    y = rs
            points.append((lo + x, nlo + y))
    base = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
    return base, np.array(points, dtype=np.int64).reshape(-1, 2)


def _matrix(kind, seed):
    if kind == "rmat":
        return inputs.rmat_csr(11, 8, seed=seed)
    rng = np.random.default_rng(seed)
    M = 1500
    lens = np.where(rng.random(M) < 0.4, 0, rng.integers(1, 12, M))
    lens[rng.choice(M, 5, replace=False)] = rng.integers(300, 3000, 5)   # heavy rows
    rowptr = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
    nnz = int(rowptr[-1])
    return CSR(torch.from_numpy(rowptr), torch.from_numpy(rng.integers(0, 500, nnz).astype(np.int32)),
               torch.ones(nnz), M, 500)


@pytest.mark.parametrize("kind,seed", [("rmat", 3), ("skewed", 4), ("skewed", 5)])
@pytest.mark.parametrize("TR,D", [(1, 64), (3, 150), (7, 333), (16, 96), (5, 2048)])
def test_plan_matches_brute_force_merge_path(kind, seed, TR, D):
    A = _matrix(kind, seed)
    plan = binding.Plan(A.rowptr.cuda(), A.M, A.K, A.nnz, 8, TR, 1,
                        tuning=binding.make_tuning(chunk_items=D))
    base, bnd_row, bnd_nnz = plan.boundaries()
    want_base, want_pts = brute_force_plan(A.rowptr.numpy(), A.M, TR, D)
    np.testing.assert_array_equal(base, want_base)
    assert bnd_row.size == want_pts.shape[0]
    np.testing.assert_array_equal(bnd_row, want_pts[:, 0])
    np.testing.assert_array_equal(bnd_nnz, want_pts[:, 1])
    plan.close()
