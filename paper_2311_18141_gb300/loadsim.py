"""Load-imbalance simulator for tiled sparse products (host side, numpy).

The paper's introduction (Fig. 1) squares an R-MAT matrix with a sparse 2D
algorithm on a p x p process grid and compares two kinds of balance:

* end to end -- the work of process (i, j) summed over all stages, max/avg over
  the p*p processes (processes that never synchronise);
* per stage -- in stage k every process (i, j) multiplies A's tile (i, k') by
  B's tile (k', j); if processes synchronise after every stage, the run takes
  sum_k max_ij w(i,j,k') against an ideal sum_k avg_ij w(i,j,k').  With the
  iteration offset of Section 3.3 (stationary C) process (i, j) takes
  k' = (i + j + k) mod p in stage k, so the tiles multiplied in one stage come
  from p different block columns; without it (SUMMA's lockstep) k' = k.

The work of a tile product is its number of scalar products: for SpGEMM
w(i,j,k) = sum over the columns l of block k of nnz(A[rows of block i, l]) *
nnz(B[l, columns of block j]); for SpMM with a dense B of width N split in TC
column blocks, w(i,j,k) = nnz(A tile (i, k)) * (columns of block j).

These figures help pick a tile grid: the asynchronous, work-stealing schedule
pays the end-to-end imbalance at most, a synchronised one the per-stage one.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def _block_of(n: int, parts: int) -> np.ndarray:
    """Block index of each of n indices cut into `parts` near-equal blocks."""
    size = -(-n // parts) if n else 1
    return np.minimum(np.arange(n, dtype=np.int64) // max(size, 1), parts - 1)


def _row_of(rowptr: np.ndarray) -> np.ndarray:
    lens = np.diff(np.asarray(rowptr, dtype=np.int64))
    return np.repeat(np.arange(lens.size, dtype=np.int64), lens)


def spgemm_stage_work(A_rowptr, A_colind, B_rowptr, B_colind, K: int, N: int, p: int,
                      stages: int | None = None) -> np.ndarray:
    """w[k, i, j] for C = A*B on a p x p grid: A (M x K) in p row blocks and
    `stages` column blocks (default p), B (K x N) in `stages` row blocks and p
    column blocks."""
    s = p if stages is None else stages
    arp = np.asarray(A_rowptr, np.int64)
    brp = np.asarray(B_rowptr, np.int64)
    M = arp.size - 1
    a_rows = _block_of(M, p)[_row_of(arp)]          # row block of each A nonzero
    a_cols = np.asarray(A_colind, np.int64)
    b_rows = _row_of(brp)                           # row l of each B nonzero
    b_cols = _block_of(N, p)[np.asarray(B_colind, np.int64)]
    # ca[l, i] = nnz of A in column l and row block i; rb[l, j] = nnz of B row l in column block j
    ca = np.zeros((K, p), np.float64)
    np.add.at(ca, (a_cols, a_rows), 1.0)
    rb = np.zeros((K, p), np.float64)
    np.add.at(rb, (b_rows, b_cols), 1.0)
    stage_of_l = _block_of(K, s)
    w = np.zeros((s, p, p), np.float64)
    for k in range(s):
        sel = stage_of_l == k
        w[k] = ca[sel].T @ rb[sel]
    return w


def spmm_stage_work(A_rowptr, A_colind, K: int, N: int, TR: int, TC: int,
                    stages: int) -> np.ndarray:
    """w[k, i, j] for C = A*B with a dense B of width N: A in TR row blocks and
    `stages` column blocks, C in TR x TC tiles."""
    arp = np.asarray(A_rowptr, np.int64)
    M = arp.size - 1
    a_rows = _block_of(M, TR)[_row_of(arp)]
    a_stage = _block_of(K, stages)[np.asarray(A_colind, np.int64)]
    nnz_tile = np.zeros((stages, TR), np.float64)
    np.add.at(nnz_tile, (a_stage, a_rows), 1.0)
    width = np.bincount(_block_of(N, TC), minlength=TC).astype(np.float64)
    return nnz_tile[:, :, None] * width[None, None, :]


@dataclass
class Imbalance:
    end_to_end: float          # max/avg over processes of the summed work
    synchronised: float        # sum_k max / sum_k avg (stages separated by barriers)
    per_stage: np.ndarray      # max/avg of every stage
    per_process: np.ndarray    # summed work of every process (the heat map)


def staggered(w: np.ndarray) -> np.ndarray:
    """Stage work reordered by the iteration offset of Section 3.3: entry
    [k, i, j] becomes the work process (i, j) does in stage k, which is its
    product for block (i + j + k) mod s (s stages)."""
    s, p, q = w.shape
    ii, jj = np.meshgrid(np.arange(p), np.arange(q), indexing="ij")
    return np.stack([w[(ii + jj + k) % s, ii, jj] for k in range(s)])


def imbalance(w: np.ndarray, offset: bool = False) -> Imbalance:
    """Both load-imbalance figures of stage work w[k, i, j]; with `offset`, the
    stages follow the iteration offset (see staggered)."""
    if offset:
        w = staggered(w)
    total = w.sum(axis=0)
    avg = total.mean()
    e2e = float(total.max() / avg) if avg > 0 else 1.0
    smax = w.reshape(w.shape[0], -1).max(axis=1)
    savg = w.reshape(w.shape[0], -1).mean(axis=1)
    sync = float(smax.sum() / savg.sum()) if savg.sum() > 0 else 1.0
    with np.errstate(invalid="ignore", divide="ignore"):
        per_stage = np.where(savg > 0, smax / savg, 1.0)
    return Imbalance(e2e, sync, per_stage, total)


def relabel(rowptr, colind, perm) -> tuple[np.ndarray, np.ndarray]:
    """CSR of P A P^T for a square A: vertex v becomes perm[v] (rows and
    columns alike); rows come out with increasing columns."""
    rp = np.asarray(rowptr, np.int64)
    ci = np.asarray(colind, np.int64)
    perm = np.asarray(perm, np.int64)
    n = rp.size - 1
    r = perm[_row_of(rp)]
    c = perm[ci]
    order = np.lexsort((c, r))
    r, c = r[order], c[order]
    out = np.zeros(n + 1, np.int64)
    out[1:] = np.cumsum(np.bincount(r, minlength=n))
    return out, c
