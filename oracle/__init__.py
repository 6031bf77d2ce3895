"""FP64 CPU oracle for the CSR SpMM path (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It loads ``liboracle.so`` built from
``spmm_oracle.c`` (plain C, compiled with gcc) and wraps it with numpy.  It
imports nothing from the CUDA library and the CUDA library imports nothing
from it.

Every function follows the definition of the local product in Section 2.1 of
the paper (C_ij += sum_k A_ik B_kj) or a published number format; see the C
source for the passage each one follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "spmm_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp"]


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (OpenMP if available)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", *CFLAGS, _SRC, "-o", tmp, "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:  # retry without OpenMP
        cmd = ["gcc", *[f for f in CFLAGS if f != "-fopenmp"], _SRC, "-o", tmp, "-lm"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("oracle build failed:\n" + r.stderr)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            i64, i32p, vp, dp = ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p
            ci, cd = ctypes.c_int, ctypes.c_double
            lib.oracle_spmm.argtypes = [i64, i64, i64, i32p, i32p, vp, ci, vp, ci, i64, cd, dp,
                                        i64, dp, i64]
            lib.oracle_spmm_rows.argtypes = [i64, i32p, i32p, vp, ci, vp, ci, i64, cd, dp, i64,
                                             vp, i64, dp]
            lib.oracle_csr_transpose.argtypes = [i64, i64, i32p, i32p, dp, i32p, i32p, dp, vp]
            lib.oracle_sddmm.argtypes = [i64, i64, i32p, i32p, vp, ci, i64, vp, ci, i64, dp]
            lib.oracle_spmm_t_push.argtypes = [i64, i64, i64, i32p, i32p, vp, ci, vp, ci, i64,
                                               dp, i64]
            for name in ("oracle_decode_bf16", "oracle_decode_f16", "oracle_decode_e4m3",
                         "oracle_encode_bf16", "oracle_encode_f16", "oracle_encode_e4m3"):
                getattr(lib, name).argtypes = [vp, i64, vp]
                getattr(lib, name).restype = None
            lib.oracle_quantize_rows_e4m3.argtypes = [vp, i64, i64, i64, vp, i64, vp]
            lib.oracle_quantize_rows_e4m3.restype = None
            lib.oracle_set_threads.argtypes = [ci]
            lib.oracle_spgemm.argtypes = [i64, i64, i64, i32p, i32p, dp, i32p, i32p, dp, i32p,
                                          vp, vp]
            lib.oracle_set_threads.restype = None
            lib.oracle_get_threads.restype = ci
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _np(x, dtype=None) -> np.ndarray:
    """Accept numpy arrays or CPU torch tensors; return a C-contiguous numpy array."""
    if hasattr(x, "detach"):
        x = x.detach().cpu().numpy()
    a = np.ascontiguousarray(x)
    if dtype is not None and a.dtype != dtype:
        a = a.astype(dtype)
    return a


def _float_arr(x) -> tuple[np.ndarray, int]:
    a = _np(x)
    if a.dtype == np.float32:
        return a, 1
    return a.astype(np.float64, copy=False), 0


def set_threads(n: int) -> None:
    _load().oracle_set_threads(int(n))


def get_threads() -> int:
    return int(_load().oracle_get_threads())


def spmm(rowptr, colind, vals, B, beta: float = 0.0, C0=None) -> np.ndarray:
    """C = beta*C0 + A*B in FP64 (Section 2.1).  vals/B may be float32 or float64."""
    lib = _load()
    rp = _np(rowptr, np.int32)
    ci = _np(colind, np.int32)
    v, vf = _float_arr(vals)
    b, bf = _float_arr(B)
    M = rp.size - 1
    K, N = b.shape
    c0 = None if C0 is None else _np(C0, np.float64)
    C = np.empty((M, N), dtype=np.float64)
    rc = lib.oracle_spmm(M, K, N, _p(rp), _p(ci), _p(v), vf, _p(b), bf, N, float(beta),
                         None if c0 is None else _p(c0), N, _p(C), N)
    assert rc == 0
    return C


def spmm_rows(rowptr, colind, vals, B, rows, beta: float = 0.0, C0_rows=None) -> np.ndarray:
    """Rows ``rows`` of beta*C0 + A*B.  ``C0_rows`` holds C0 at those rows only."""
    lib = _load()
    rp = _np(rowptr, np.int32)
    ci = _np(colind, np.int32)
    v, vf = _float_arr(vals)
    b, bf = _float_arr(B)
    r = _np(rows, np.int64)
    N = b.shape[1]
    out = np.empty((r.size, N), dtype=np.float64)
    c0 = None if (C0_rows is None or beta == 0.0) else _np(C0_rows, np.float64)
    rc = lib.oracle_spmm_rows(N, _p(rp), _p(ci), _p(v), vf, _p(b), bf, N, float(beta),
                              None if c0 is None else _p(c0), N, _p(r), r.size, _p(out))
    assert rc == 0
    return out


def csr_transpose(rowptr, colind, vals, K: int):
    """CSR (M x K) -> (colptr[K+1], rowind[nnz], tvals[nnz], perm[nnz]), rows increasing."""
    lib = _load()
    rp = _np(rowptr, np.int32)
    ci = _np(colind, np.int32)
    v = _np(vals, np.float64)
    M = rp.size - 1
    nnz = ci.size
    colptr = np.empty(K + 1, dtype=np.int32)
    rowind = np.empty(nnz, dtype=np.int32)
    tvals = np.empty(nnz, dtype=np.float64)
    perm = np.empty(nnz, dtype=np.int64)
    rc = lib.oracle_csr_transpose(M, K, _p(rp), _p(ci), _p(v), _p(colptr), _p(rowind),
                                  _p(tvals), _p(perm))
    if rc != 0:
        raise ValueError("column index out of range")
    return colptr, rowind, tvals, perm


def sddmm(rowptr, colind, dC, B) -> np.ndarray:
    """out[e] = sum_n dC[row_e, n] * B[col_e, n] in FP64."""
    lib = _load()
    rp = _np(rowptr, np.int32)
    ci = _np(colind, np.int32)
    d, df = _float_arr(dC)
    b, bf = _float_arr(B)
    M = rp.size - 1
    N = b.shape[1]
    out = np.empty(ci.size, dtype=np.float64)
    lib.oracle_sddmm(M, N, _p(rp), _p(ci), _p(d), df, N, _p(b), bf, N, _p(out))
    return out


def spmm_t_push(rowptr, colind, vals, dC, K: int) -> np.ndarray:
    """dB = A^T dC by scattering rows of dC (no transpose), FP64."""
    lib = _load()
    rp = _np(rowptr, np.int32)
    ci = _np(colind, np.int32)
    v, vf = _float_arr(vals)
    d, df = _float_arr(dC)
    M = rp.size - 1
    N = d.shape[1]
    dB = np.empty((K, N), dtype=np.float64)
    lib.oracle_spmm_t_push(M, K, N, _p(rp), _p(ci), _p(v), vf, _p(d), df, N, _p(dB), N)
    return dB


def _codec(name: str, x, in_dtype, out_dtype) -> np.ndarray:
    a = _np(x, in_dtype)
    out = np.empty(a.shape, dtype=out_dtype)
    getattr(_load(), name)(_p(a), a.size, _p(out))
    return out


def decode_bf16(bits) -> np.ndarray:
    return _codec("oracle_decode_bf16", bits, np.uint16, np.float64)


def decode_f16(bits) -> np.ndarray:
    return _codec("oracle_decode_f16", bits, np.uint16, np.float64)


def decode_e4m3(bits) -> np.ndarray:
    return _codec("oracle_decode_e4m3", bits, np.uint8, np.float64)


def encode_bf16(x) -> np.ndarray:
    return _codec("oracle_encode_bf16", x, np.float32, np.uint16)


def encode_f16(x) -> np.ndarray:
    return _codec("oracle_encode_f16", x, np.float32, np.uint16)


def encode_e4m3(x) -> np.ndarray:
    return _codec("oracle_encode_e4m3", x, np.float32, np.uint8)


def quantize_rows_e4m3(X):
    """(codes uint8 [rows x cols], scales float32 [rows]) with s = amax/448 per row."""
    x = _np(X, np.float32)
    rows, cols = x.shape
    q = np.empty((rows, cols), dtype=np.uint8)
    s = np.empty(rows, dtype=np.float32)
    _load().oracle_quantize_rows_e4m3(_p(x), rows, cols, cols, _p(q), cols, _p(s))
    return q, s


def dequantize_rows(codes, scales, fmt: str) -> np.ndarray:
    """FP64 value of stored rows: decode(code) * scale (scale 1 when None)."""
    dec = {"bf16": decode_bf16, "f16": decode_f16, "e4m3": decode_e4m3}[fmt](codes)
    if scales is None:
        return dec
    return dec * _np(scales, np.float32).astype(np.float64)[:, None]


def abs_bound(rowptr, colind, vals, B) -> np.ndarray:
    """|A|*|B| in FP64: the elementwise scale of the error tolerances."""
    v, _ = _float_arr(vals)
    b, _ = _float_arr(B)
    return spmm(rowptr, colind, np.abs(v.astype(np.float64)), np.abs(b.astype(np.float64)))


def spgemm(A_rowptr, A_colind, A_vals, B_rowptr, B_colind, B_vals, K: int, N: int):
    """C = A*B for CSR A (M x K) and CSR B (K x N): (rowptr, colind, vals) in FP64,
    columns of each row increasing; an entry exists wherever some product
    A_ik B_kj is formed (explicit zeros count)."""
    lib = _load()
    arp, aci = _np(A_rowptr, np.int32), _np(A_colind, np.int32)
    brp, bci = _np(B_rowptr, np.int32), _np(B_colind, np.int32)
    av, bv = _np(A_vals, np.float64), _np(B_vals, np.float64)
    M = arp.size - 1
    rowptr = np.empty(M + 1, dtype=np.int32)
    rc = lib.oracle_spgemm(M, K, N, _p(arp), _p(aci), _p(av), _p(brp), _p(bci), _p(bv),
                           _p(rowptr), None, None)
    if rc != 0:
        raise ValueError("column index out of range")
    nnz = int(rowptr[-1])
    colind = np.empty(max(nnz, 1), dtype=np.int32)
    vals = np.empty(max(nnz, 1), dtype=np.float64)
    rc = lib.oracle_spgemm(M, K, N, _p(arp), _p(aci), _p(av), _p(brp), _p(bci), _p(bv),
                           _p(rowptr), _p(colind), _p(vals))
    assert rc == 0
    return rowptr, colind[:nnz], vals[:nnz]
