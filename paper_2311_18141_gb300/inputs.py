"""Seeded synthetic inputs for the CSR SpMM workloads.

This module is the one piece shared by the FP64 oracle tests and the CUDA path.
It holds no SpMM arithmetic: it only draws random matrices and assembles them
into CSR arrays.

Randomness comes from a counter-based generator (a 32-bit integer hash of
(seed, stream, counter) built from the MurmurHash3 32-bit finaliser), written
with int64 tensor ops that never overflow.  The same counters give the same
integers on the CPU and on a GPU, so a matrix drawn on the device for a
benchmark is bit-identical to the one a CPU test draws.  Dense normal values
go through Box-Muller in float64 and are rounded to float32.

Workloads (the synthetic stand-ins for the paper's SuiteSparse/SNAP matrices,
Table 1, and its dense widths n of 128/256/512, Section 6):
  * ``uniform_csr``   fixed nnz per row, distinct sorted columns (4096^2, 16/row)
  * ``rmat_csr``      R-MAT power-law graph (Section 1 uses R-MAT for Figure 1)
  * ``gcn_normalized_adjacency``  D^-1/2 (A + I) D^-1/2 of a symmetrised R-MAT
  * ``poisson_csr``   Poisson row lengths, distinct sorted uniform columns
  * ``dense_normal`` / ``dense_uniform``  dense B, C, X operands
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import torch

_M32 = 0xFFFFFFFF

# stream identifiers: independent counters for each kind of draw
STREAM_RMAT = 1
STREAM_VALS = 2
STREAM_COLS = 3
STREAM_DENSE_U1 = 4
STREAM_DENSE_U2 = 5
STREAM_ROWLEN = 6
STREAM_DENSE_UNIFORM = 7


def _mul32(h: torch.Tensor, m: int) -> torch.Tensor:
    """(h * m) mod 2^32 for int64 tensors holding values in [0, 2^32)."""
    m_lo = m & 0xFFFF
    m_hi = (m >> 16) & 0xFFFF
    return (h * m_lo + (((h * m_hi) & 0xFFFF) << 16)) & _M32


def _fmix32(h: torch.Tensor) -> torch.Tensor:
    h = h ^ (h >> 16)
    h = _mul32(h, 0x85EBCA6B)
    h = h ^ (h >> 13)
    h = _mul32(h, 0xC2B2AE35)
    h = h ^ (h >> 16)
    return h


def _fmix32_int(h: int) -> int:
    h &= _M32
    h ^= h >> 16
    h = (h * 0x85EBCA6B) & _M32
    h ^= h >> 13
    h = (h * 0xC2B2AE35) & _M32
    h ^= h >> 16
    return h


def hash_u32(counter: torch.Tensor, seed: int, stream: int) -> torch.Tensor:
    """32-bit hash of a non-negative int64 counter tensor (values < 2^62)."""
    k1 = _fmix32_int(seed * 0x9E3779B1 + stream * 0x7F4A7C15 + 0x165667B1)
    k2 = _fmix32_int(k1 ^ (stream * 0x27D4EB2F + 0x61C88647))
    lo = counter & _M32
    hi = counter >> 32
    h = _fmix32(lo ^ k1)
    h = _fmix32(h ^ hi ^ k2)
    return h


def _uniform_open01_f64(h: torch.Tensor) -> torch.Tensor:
    """Map 32-bit hashes to float64 in (0, 1]."""
    return (h.to(torch.float64) + 1.0) * (1.0 / 4294967296.0)


def uniform_f32(counter: torch.Tensor, seed: int, stream: int, lo: float, hi: float,
                open_low: bool = False) -> torch.Tensor:
    """Uniform float32 from 24 hashed bits: [lo, hi), or (lo, hi] if open_low."""
    h = hash_u32(counter, seed, stream) >> 8  # 24 bits
    if open_low:
        u = (h.to(torch.float64) + 1.0) * (1.0 / 16777216.0)
    else:
        u = h.to(torch.float64) * (1.0 / 16777216.0)
    return (lo + (hi - lo) * u).to(torch.float32)


_CHUNK = 1 << 24


def dense_normal(rows: int, cols: int, seed: int, device="cpu",
                 dtype=torch.float32) -> torch.Tensor:
    """rows x cols row-major N(0, 1) by Box-Muller over hashed counters."""
    n = rows * cols
    out = torch.empty(n, dtype=dtype, device=device)
    for start in range(0, n, _CHUNK):
        end = min(n, start + _CHUNK)
        idx = torch.arange(start, end, dtype=torch.int64, device=device)
        u1 = _uniform_open01_f64(hash_u32(idx, seed, STREAM_DENSE_U1))
        u2 = _uniform_open01_f64(hash_u32(idx, seed, STREAM_DENSE_U2))
        z = torch.sqrt(-2.0 * torch.log(u1)) * torch.cos((2.0 * math.pi) * u2)
        out[start:end] = z.to(dtype)
    return out.view(rows, cols)


def dense_uniform(rows: int, cols: int, seed: int, lo: float, hi: float,
                  device="cpu") -> torch.Tensor:
    """rows x cols row-major float32 uniform in [lo, hi)."""
    n = rows * cols
    out = torch.empty(n, dtype=torch.float32, device=device)
    for start in range(0, n, _CHUNK):
        end = min(n, start + _CHUNK)
        idx = torch.arange(start, end, dtype=torch.int64, device=device)
        out[start:end] = uniform_f32(idx, seed, STREAM_DENSE_UNIFORM, lo, hi)
    return out.view(rows, cols)


@dataclass
class CSR:
    """CSR matrix: int32 rowptr[M+1], int32 colind[nnz] sorted per row, float32 vals."""
    rowptr: torch.Tensor
    colind: torch.Tensor
    vals: torch.Tensor
    M: int
    K: int

    @property
    def nnz(self) -> int:
        return int(self.colind.numel())

    def to(self, device) -> "CSR":
        return CSR(self.rowptr.to(device), self.colind.to(device), self.vals.to(device),
                   self.M, self.K)

    def row_lengths(self) -> torch.Tensor:
        return (self.rowptr[1:] - self.rowptr[:-1]).to(torch.int64)


def _csr_from_sorted_keys(keys: torch.Tensor, M: int, K: int) -> tuple[torch.Tensor, torch.Tensor]:
    """Sorted unique int64 keys row*K + col -> (rowptr int32, colind int32)."""
    rows = keys // K
    cols = keys - rows * K
    counts = torch.bincount(rows, minlength=M)
    rowptr = torch.zeros(M + 1, dtype=torch.int64, device=keys.device)
    rowptr[1:] = torch.cumsum(counts, 0)
    return rowptr.to(torch.int32), cols.to(torch.int32)


def _values(nnz: int, seed: int, kind: str, device) -> torch.Tensor:
    idx = torch.arange(nnz, dtype=torch.int64, device=device)
    if kind == "sym":        # uniform [-1, 1)
        return uniform_f32(idx, seed, STREAM_VALS, -1.0, 1.0)
    if kind == "pos":        # uniform (0, 1]
        return uniform_f32(idx, seed, STREAM_VALS, 0.0, 1.0, open_low=True)
    if kind == "ones":
        return torch.ones(nnz, dtype=torch.float32, device=device)
    raise ValueError(kind)


def _distinct_sorted_columns(row_of: torch.Tensor, K: int, seed: int, device) -> torch.Tensor:
    """Draw one uniform column in [0, K) per entry of ``row_of`` (row id per slot,
    non-decreasing), redrawing collisions until every row's columns are distinct.
    Returns int64 keys row*K + col, sorted."""
    n = row_of.numel()
    if n == 0:
        return row_of.clone()
    lens = torch.bincount(row_of)
    dense = (lens * 8 >= K).nonzero().flatten()
    if dense.numel() > 0:
        # rows asking for at least K/8 columns: rank every column of the row by a
        # hashed key and keep the first L (redraws would converge too slowly)
        keep = ~torch.isin(row_of, dense)
        sparse_keys = _distinct_sorted_columns(row_of[keep], K, seed, device)
        cand = torch.arange(K, dtype=torch.int64, device=device)
        parts = [sparse_keys]
        for r in dense.tolist():
            L = int(lens[r])
            score = hash_u32(r * (K + 1) + cand, seed, STREAM_COLS + 100)
            pick = torch.sort(torch.argsort(score)[:L]).values
            parts.append(r * K + pick)
        return torch.sort(torch.cat(parts)).values
    slot = torch.arange(n, dtype=torch.int64, device=device)
    cols = hash_u32(slot * 64, seed, STREAM_COLS) % K
    for attempt in range(1, 64):
        keys, order = torch.sort(row_of * K + cols)
        dup = torch.zeros(n, dtype=torch.bool, device=device)
        if n > 1:
            dup[1:] = keys[1:] == keys[:-1]
        if not bool(dup.any()):
            return keys
        # redraw the later copy of each collision with a fresh counter
        redraw_slots = order[dup]
        cols = cols.clone()
        cols[redraw_slots] = hash_u32(redraw_slots * 64 + attempt, seed, STREAM_COLS) % K
    raise RuntimeError("could not draw distinct columns")


def uniform_csr(M: int, K: int, nnz_per_row: int, seed: int, device="cpu",
                values: str = "sym") -> CSR:
    """Exactly ``nnz_per_row`` distinct uniformly drawn columns per row, sorted."""
    assert nnz_per_row <= K
    row_of = torch.arange(M, dtype=torch.int64, device=device).repeat_interleave(nnz_per_row)
    keys = _distinct_sorted_columns(row_of, K, seed, device)
    rowptr, colind = _csr_from_sorted_keys(keys, M, K)
    return CSR(rowptr, colind, _values(keys.numel(), seed, values, device), M, K)


def poisson_row_lengths(M: int, mean: float, cap: int, seed: int, device="cpu") -> torch.Tensor:
    """Poisson(mean) row lengths by inverse CDF over hashed uniforms, capped at ``cap``."""
    kmax = int(mean + 12.0 * math.sqrt(mean) + 16)
    pmf = [math.exp(-mean)]
    for k in range(1, kmax + 1):
        pmf.append(pmf[-1] * mean / k)
    cdf = torch.tensor(pmf, dtype=torch.float64).cumsum(0)
    cdf[-1] = 1.0
    u = _uniform_open01_f64(hash_u32(torch.arange(M, dtype=torch.int64, device=device),
                                     seed, STREAM_ROWLEN))
    k = torch.searchsorted(cdf.to(device), u)
    return torch.clamp(k, max=cap)


def poisson_csr(M: int, K: int, mean: float, seed: int, device="cpu", values: str = "sym") -> CSR:
    """Poisson(mean) nnz per row (capped at K), distinct uniform sorted columns."""
    lens = poisson_row_lengths(M, mean, K, seed, device)
    row_of = torch.arange(M, dtype=torch.int64, device=device).repeat_interleave(lens)
    keys = _distinct_sorted_columns(row_of, K, seed, device)
    rowptr, colind = _csr_from_sorted_keys(keys, M, K)
    return CSR(rowptr, colind, _values(keys.numel(), seed, values, device), M, K)


def rmat_edges(scale: int, edge_factor: int, a: float, b: float, c: float, seed: int,
               device="cpu") -> tuple[torch.Tensor, torch.Tensor]:
    """R-MAT edge list: each edge takes ``scale`` independent quadrant draws,
    most significant bit first, with probabilities (a, b, c, d = 1-a-b-c) for the
    quadrants (top-left, top-right, bottom-left, bottom-right).  No noise and no
    vertex permutation."""
    m = edge_factor << scale
    t_a = int(a * 4294967296.0)
    t_ab = int((a + b) * 4294967296.0)
    t_abc = int((a + b + c) * 4294967296.0)
    rows = torch.empty(m, dtype=torch.int64, device=device)
    cols = torch.empty(m, dtype=torch.int64, device=device)
    for start in range(0, m, _CHUNK):
        end = min(m, start + _CHUNK)
        idx = torch.arange(start, end, dtype=torch.int64, device=device)
        r = torch.zeros_like(idx)
        q = torch.zeros_like(idx)
        for level in range(scale):
            u = hash_u32(idx * 64 + level, seed, STREAM_RMAT)
            rbit = (u >= t_ab).to(torch.int64)
            cbit = (((u >= t_a) & (u < t_ab)) | (u >= t_abc)).to(torch.int64)
            r = (r << 1) | rbit
            q = (q << 1) | cbit
        rows[start:end] = r
        cols[start:end] = q
    return rows, cols


def rmat_csr(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19,
             c: float = 0.19, seed: int = 1, device="cpu", values: str = "pos") -> CSR:
    """R-MAT CSR with duplicates merged and self-loops kept, values drawn after
    deduplication (uniform (0, 1] by default)."""
    n = 1 << scale
    rows, cols = rmat_edges(scale, edge_factor, a, b, c, seed, device)
    keys = torch.unique(rows * n + cols, sorted=True)
    del rows, cols
    rowptr, colind = _csr_from_sorted_keys(keys, n, n)
    return CSR(rowptr, colind, _values(keys.numel(), seed, values, device), n, n)


def _gcn_from_edge_keys(keys: torch.Tensor, n: int, device) -> CSR:
    """Binary symmetric pattern (no self-loops) -> D^-1/2 (A + I) D^-1/2 in FP64,
    rounded to FP32."""
    diag = torch.arange(n, dtype=torch.int64, device=device) * (n + 1)
    keys = torch.unique(torch.cat([keys, diag]), sorted=True)
    rowptr, colind = _csr_from_sorted_keys(keys, n, n)
    deg = (rowptr[1:] - rowptr[:-1]).to(torch.float64)
    rows = keys // n
    cols = keys - rows * n
    vals = (1.0 / torch.sqrt(deg[rows] * deg[cols])).to(torch.float32)
    return CSR(rowptr, colind, vals, n, n)


def symmetric_pattern_keys(scale: int, edge_factor: int, seed: int, device="cpu",
                           a: float = 0.57, b: float = 0.19, c: float = 0.19) -> torch.Tensor:
    """Sorted unique keys of the symmetrised R-MAT pattern A u A^T without self-loops."""
    n = 1 << scale
    rows, cols = rmat_edges(scale, edge_factor, a, b, c, seed, device)
    keep = rows != cols
    rows, cols = rows[keep], cols[keep]
    keys = torch.cat([rows * n + cols, cols * n + rows])
    return torch.unique(keys, sorted=True)


def gcn_normalized_adjacency(scale: int, edge_factor: int = 16, seed: int = 4,
                             device="cpu") -> CSR:
    """A_hat = D^-1/2 (A + I) D^-1/2 of the symmetrised, binarised R-MAT graph."""
    n = 1 << scale
    return _gcn_from_edge_keys(symmetric_pattern_keys(scale, edge_factor, seed, device), n, device)


def gcn_induced_subgraph(scale: int, n_sub: int, edge_factor: int = 16, seed: int = 4,
                         device="cpu") -> CSR:
    """A_hat re-normalised on the subgraph induced by nodes 0 .. n_sub-1."""
    n = 1 << scale
    keys = symmetric_pattern_keys(scale, edge_factor, seed, device)
    rows = keys // n
    cols = keys - rows * n
    keep = (rows < n_sub) & (cols < n_sub)
    sub = rows[keep] * n_sub + cols[keep]
    return _gcn_from_edge_keys(sub, n_sub, device)


def glorot_uniform(fan_in: int, fan_out: int, seed: int, device="cpu") -> torch.Tensor:
    bound = math.sqrt(6.0 / (fan_in + fan_out))
    return dense_uniform(fan_in, fan_out, seed, -bound, bound, device)


def log_uniform_int(count: int, lo: int, hi: int, seed: int, stream: int) -> list[int]:
    """``count`` integers with log drawn uniformly in [log lo, log hi]."""
    u = _uniform_open01_f64(hash_u32(torch.arange(count, dtype=torch.int64), seed, stream))
    v = torch.exp(math.log(lo) + (math.log(hi) - math.log(lo)) * u)
    return [int(min(hi, max(lo, int(x)))) for x in v.tolist()]


def uniform_list(count: int, lo: float, hi: float, seed: int, stream: int) -> list[float]:
    u = _uniform_open01_f64(hash_u32(torch.arange(count, dtype=torch.int64), seed, stream))
    return (lo + (hi - lo) * u).tolist()


@dataclass
class BatchProblemSpec:
    rows: int
    mean_nnz: float
    N: int
    seed: int


def batch_specs(count: int = 512, seed: int = 5, rows_lo: int = 1000, rows_hi: int = 200000,
                mean_lo: float = 8.0, mean_hi: float = 64.0,
                widths: tuple[int, ...] = (16, 64, 128)) -> list[BatchProblemSpec]:
    """Shapes of the uneven batch: rows log-uniform, mean nnz/row uniform, N from ``widths``."""
    rows = log_uniform_int(count, rows_lo, rows_hi, seed, 101)
    means = uniform_list(count, mean_lo, mean_hi, seed, 102)
    pick = hash_u32(torch.arange(count, dtype=torch.int64), seed, 103) % len(widths)
    return [BatchProblemSpec(rows[p], means[p], widths[int(pick[p])], seed * 100003 + p)
            for p in range(count)]
