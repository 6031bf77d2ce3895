"""Thin ctypes binding of the C ABI in include/spmm_gb300.h.

Functions carry the C names and only marshal arguments: torch tensors become
device pointers, the current torch stream becomes the cudaStream_t, and a
non-zero status becomes an ``SpmmError``.  Every step of the computation runs
in the CUDA library; if the library cannot be loaded, importing this module's
functions raises, and there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libspmm_gb300.so")

SPMM_OK = 0
SPMM_ERR_INVALID_ARG = -1
SPMM_ERR_MISALIGNED = -2
SPMM_ERR_UNSUPPORTED = -3
SPMM_ERR_CUDA = -4
SPMM_ERR_BAD_CSR = -5
SPMM_ERR_TIMEOUT = -6
SPMM_ERR_WORKSPACE = -7
SPMM_ERR_PLAN_MISMATCH = -8
SPMM_ERR_INTERNAL = -9

SPMM_F32, SPMM_F16, SPMM_BF16, SPMM_E4M3 = 0, 1, 2, 3

EXPORTED = [
    "spmm_status_string", "spmm_version", "spmm_plan_create", "spmm_plan_destroy",
    "spmm_plan_workspace_size", "spmm_plan_units", "spmm_csr_workspace_size", "spmm_csr",
    "spmm_csr_validate", "spmm_get_device_status", "spmm_csr_transpose_workspace_size",
    "spmm_csr_transpose", "spmm_gather_values", "spmm_sddmm_csr", "spmm_quantize_rows",
    "spmm_csr_noalloc", "spmm_csr_noalloc_status", "spmm_bench_gather", "spmm_batch_create", "spmm_batch_destroy", "spmm_batch_workspace_size",
    "spmm_batch_set_shapes", "spmm_batch_get_shapes", "spmm_csr_batched",
    "spmm_batch_graph_launch", "spmm_batch_autotune", "spmm_spgemm_analyze", "spmm_spgemm",
    "spmm_spgemm_copy", "spmm_host_pipe_create", "spmm_host_pipe_submit", "spmm_host_pipe_wait",
    "spmm_host_pipe_destroy", "spmm_selftest_wait_timeout", "spmm_plan_set_trace",
    "spmm_plan_get_boundaries",
]

# spmm_trace_record: per-warp record of a traced spmm_csr launch
TRACE_DTYPE = np.dtype([("t_start_ns", "<i8"), ("t_end_ns", "<i8"), ("units", "<i4"),
                        ("stolen", "<i4"), ("home", "<i4"), ("smid", "<i4")])


class SpmmError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} ({status})")


class spmm_tuning(ctypes.Structure):
    _fields_ = [("chunk_items", ctypes.c_int32), ("warps_per_cta", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32), ("tile_order", ctypes.c_int32),
                ("kernel", ctypes.c_int32), ("lanes_per_item", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 2)]


# spmm_tuning.kernel
SPMM_KERNEL_AUTO, SPMM_KERNEL_STAGED, SPMM_KERNEL_WIDE, SPMM_KERNEL_SPEC = 0, 1, 2, 3


class spmm_problem(ctypes.Structure):
    _fields_ = [("rowptr", ctypes.c_void_p), ("colind", ctypes.c_void_p),
                ("vals", ctypes.c_void_p), ("a_scale", ctypes.c_void_p),
                ("B", ctypes.c_void_p), ("b_scale", ctypes.c_void_p), ("C", ctypes.c_void_p),
                ("M", ctypes.c_int64), ("K", ctypes.c_int64), ("N", ctypes.c_int64),
                ("nnz", ctypes.c_int64), ("ldb", ctypes.c_int64), ("ldc", ctypes.c_int64),
                ("beta", ctypes.c_float), ("tile_rows", ctypes.c_int32),
                ("tile_cols", ctypes.c_int32), ("chunk_items", ctypes.c_int32)]


_lib = None
_lock = threading.Lock()


def load_library(path: str | None = None):
    """Load libspmm_gb300.so (raises if it is missing: there is no fallback)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = path or os.environ.get("SPMM_GB300_LIB") or LIB_PATH
        if not os.path.exists(path):
            raise ImportError(f"CUDA library not built: {path} (run __graft_entry__.build())")
        lib = ctypes.CDLL(path)
        i32, i64, vp, f32 = ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p, ctypes.c_float
        sz = ctypes.c_size_t
        lib.spmm_status_string.argtypes = [ctypes.c_int]
        lib.spmm_status_string.restype = ctypes.c_char_p
        lib.spmm_version.restype = ctypes.c_int
        lib.spmm_plan_create.argtypes = [ctypes.POINTER(vp), vp, i64, i64, i64, i64, i32, i32,
                                         ctypes.POINTER(spmm_tuning), vp]
        lib.spmm_plan_destroy.argtypes = [vp]
        lib.spmm_plan_workspace_size.argtypes = [vp, ctypes.POINTER(sz)]
        lib.spmm_plan_units.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64)]
        lib.spmm_spgemm_analyze.argtypes = [vp, vp, i64, i64, i64, vp, i64, ctypes.POINTER(i64),
                                            ctypes.POINTER(sz), vp]
        lib.spmm_spgemm.argtypes = [vp, vp, vp, i64, i64, i64, vp, vp, vp, i64, i64, vp, sz,
                                    ctypes.POINTER(i64), vp]
        lib.spmm_spgemm_copy.argtypes = [vp, i64, i64, i64, i64, vp, vp, vp, vp]
        lib.spmm_csr_workspace_size.argtypes = [i64, i64, i64, i32, i32,
                                                ctypes.POINTER(spmm_tuning), ctypes.POINTER(sz)]
        lib.spmm_csr.argtypes = [vp, vp, vp, i32, vp, vp, i32, vp, i64, vp, i64, i64, i64, i64,
                                 i64, i32, i32, f32, vp, vp, sz, vp]
        lib.spmm_csr_validate.argtypes = [vp, vp, i64, i64, i64, vp, sz, vp]
        lib.spmm_get_device_status.argtypes = [vp, ctypes.POINTER(i32), vp]
        lib.spmm_csr_transpose_workspace_size.argtypes = [i64, i64, i64, ctypes.POINTER(sz)]
        lib.spmm_csr_transpose.argtypes = [vp, vp, vp, i32, i64, i64, i64, vp, vp, vp, vp, vp,
                                           sz, vp]
        lib.spmm_gather_values.argtypes = [vp, i32, vp, i64, vp, vp]
        lib.spmm_sddmm_csr.argtypes = [vp, vp, vp, i64, vp, i32, i64, vp, i64, i64, i64, i64, vp,
                                       vp, sz, vp]
        lib.spmm_quantize_rows.argtypes = [vp, i64, i64, i64, i32, vp, i64, vp, vp]
        P = ctypes.POINTER
        lib.spmm_batch_create.argtypes = [P(vp), P(spmm_problem), i32, i32, i32, vp]
        lib.spmm_batch_destroy.argtypes = [vp]
        lib.spmm_batch_workspace_size.argtypes = [vp, P(sz)]
        lib.spmm_batch_set_shapes.argtypes = [vp, P(i32), P(i32), P(i32), vp]
        lib.spmm_batch_get_shapes.argtypes = [vp, P(i32), P(i32), P(i32)]
        lib.spmm_csr_batched.argtypes = [vp, vp, sz, vp]
        lib.spmm_batch_graph_launch.argtypes = [vp, vp, sz, vp]
        lib.spmm_batch_autotune.argtypes = [vp, vp, sz, i32, vp, P(ctypes.c_float)]
        lib.spmm_selftest_wait_timeout.argtypes = [vp, sz, i64, vp]
        lib.spmm_plan_set_trace.argtypes = [vp, vp, i32]
        lib.spmm_plan_get_boundaries.argtypes = [vp, vp, vp, vp]
        lib.spmm_host_pipe_create.argtypes = [P(vp), vp, i32, i32, i32, vp]
        lib.spmm_host_pipe_submit.argtypes = [vp, vp, vp, vp, vp, vp]
        lib.spmm_host_pipe_wait.argtypes = [vp]
        lib.spmm_host_pipe_destroy.argtypes = [vp]
        lib.spmm_csr_noalloc.argtypes = [vp, vp, vp, i32, vp, vp, i32, vp, i64, vp, i64, i64, i64,
                                         i64, i64, i32, i32, f32, vp]
        lib.spmm_csr_noalloc_status.argtypes = [vp, vp]
        lib.spmm_bench_gather.argtypes = [vp, i64, vp, i32, i64, i64, i64, i32, i32, i32, vp, vp]
        for name in EXPORTED:
            if name not in ("spmm_status_string",):
                getattr(lib, name).restype = ctypes.c_int
        _lib = lib
        return lib


def status_string(status: int) -> str:
    try:
        return load_library().spmm_status_string(int(status)).decode()
    except ImportError:
        return "library not loaded"


def _check(status: int, where: str) -> None:
    if status != SPMM_OK:
        raise SpmmError(status, where)


def dtype_code(t: torch.dtype) -> int:
    if t == torch.float32:
        return SPMM_F32
    if t == torch.float16:
        return SPMM_F16
    if t == torch.bfloat16:
        return SPMM_BF16
    if t in (torch.float8_e4m3fn, torch.uint8):
        return SPMM_E4M3
    raise TypeError(f"unsupported dtype {t}")


def _ptr(t: torch.Tensor | None):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def make_tuning(chunk_items=0, warps_per_cta=0, ctas_per_sm=0, tile_order=0,
                kernel=SPMM_KERNEL_AUTO, lanes_per_item=0) -> spmm_tuning:
    t = spmm_tuning()
    t.chunk_items, t.warps_per_cta = int(chunk_items), int(warps_per_cta)
    t.ctas_per_sm, t.tile_order = int(ctas_per_sm), int(tile_order)
    t.kernel, t.lanes_per_item = int(kernel), int(lanes_per_item)
    return t


def trace_buffer(records: int, device=None) -> torch.Tensor:
    """Zeroed device buffer for ``records`` trace records."""
    return torch.zeros(records * TRACE_DTYPE.itemsize, dtype=torch.uint8, device=device or "cuda")


def read_trace(buf: torch.Tensor) -> np.ndarray:
    """The records of a trace buffer that a launch wrote (t_end_ns > 0)."""
    rec = buf.cpu().numpy().view(TRACE_DTYPE)
    return rec[rec["t_end_ns"] > 0]


def workspace(nbytes: int, device=None) -> torch.Tensor:
    """Device scratch of at least ``nbytes`` (256-byte aligned by the caching allocator)."""
    return torch.zeros(max(int(nbytes), 256), dtype=torch.uint8, device=device or "cuda")


class Plan:
    """Owner of a spmm_plan handle (spmm_plan_create / spmm_plan_destroy)."""

    def __init__(self, rowptr: torch.Tensor, M: int, K: int, nnz: int, N: int,
                 tile_rows: int = 1, tile_cols: int = 1, tuning: spmm_tuning | None = None,
                 stream=None):
        lib = load_library()
        self.handle = ctypes.c_void_p()
        self.M, self.K, self.nnz, self.N = int(M), int(K), int(nnz), int(N)
        self.tile_rows, self.tile_cols = int(tile_rows), int(tile_cols)
        tp = ctypes.byref(tuning) if tuning is not None else None
        _check(lib.spmm_plan_create(ctypes.byref(self.handle), _ptr(rowptr), self.M, self.K,
                                    self.nnz, self.N, self.tile_rows, self.tile_cols, tp,
                                    _stream(stream)), "spmm_plan_create")
        n = ctypes.c_size_t()
        _check(lib.spmm_plan_workspace_size(self.handle, ctypes.byref(n)),
               "spmm_plan_workspace_size")
        self.workspace_bytes = int(n.value)

    def set_trace(self, records: torch.Tensor | None) -> None:
        """Trace later spmm_csr calls with this plan into ``records`` (a device
        buffer from trace_buffer), or stop tracing (None)."""
        n = 0 if records is None else records.numel() * records.element_size() // TRACE_DTYPE.itemsize
        _check(load_library().spmm_plan_set_trace(self.handle, _ptr(records), int(n)),
               "spmm_plan_set_trace")
        self._trace = records   # the plan writes into it: keep it alive

    def boundaries(self):
        """(blk_base[TR+1], bnd_row, bnd_nnz) of the plan as numpy int32 arrays."""
        chunks, _ = self.units()
        bb = np.empty(self.tile_rows + 1, np.int32)
        br = np.empty(chunks + self.tile_rows, np.int32)
        bz = np.empty(chunks + self.tile_rows, np.int32)
        _check(load_library().spmm_plan_get_boundaries(
            self.handle, bb.ctypes.data_as(ctypes.c_void_p), br.ctypes.data_as(ctypes.c_void_p),
            bz.ctypes.data_as(ctypes.c_void_p)), "spmm_plan_get_boundaries")
        return bb, br, bz

    def units(self) -> tuple[int, int]:
        c, u = ctypes.c_int64(), ctypes.c_int64()
        _check(load_library().spmm_plan_units(self.handle, ctypes.byref(c), ctypes.byref(u)),
               "spmm_plan_units")
        return int(c.value), int(u.value)

    def close(self):
        if self.handle:
            load_library().spmm_plan_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class HostPipe:
    """Owner of a spmm_host_pipe (host-buffer pipeline over a plan): submit()
    enqueues one product of host tensors A (rowptr, colind, vals), B into host
    C; wait() blocks until every submitted C is in host memory."""

    def __init__(self, plan: Plan, a_dtype: torch.dtype, b_dtype: torch.dtype, depth: int = 2,
                 stream=None):
        self.plan = plan   # the pipeline uses the plan: keep it alive
        self.handle = ctypes.c_void_p()
        _check(load_library().spmm_host_pipe_create(ctypes.byref(self.handle), plan.handle,
                                                    dtype_code(a_dtype), dtype_code(b_dtype),
                                                    int(depth), _stream(stream)),
               "spmm_host_pipe_create")

    def submit(self, rowptr, colind, vals, B, C) -> None:
        for t in (rowptr, colind, vals, B, C):
            if t.is_cuda or not t.is_contiguous():
                raise ValueError("host pipeline operands are contiguous host tensors")
        _check(load_library().spmm_host_pipe_submit(self.handle, _ptr(rowptr), _ptr(colind),
                                                    _ptr(vals), _ptr(B), _ptr(C)),
               "spmm_host_pipe_submit")

    def wait(self) -> None:
        _check(load_library().spmm_host_pipe_wait(self.handle), "spmm_host_pipe_wait")

    def close(self):
        if self.handle:
            load_library().spmm_host_pipe_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def spmm_csr_workspace_size(M: int, nnz: int, N: int, tile_rows: int = 1,
                            tile_cols: int = 1) -> int:
    n = ctypes.c_size_t()
    _check(load_library().spmm_csr_workspace_size(int(M), int(nnz), int(N), int(tile_rows),
                                                  int(tile_cols), None, ctypes.byref(n)),
           "spmm_csr_workspace_size")
    return int(n.value)


def spmm_csr(rowptr, colind, vals, B, C, M, K, N, nnz, *, a_scale=None, b_scale=None,
             tile_rows=0, tile_cols=0, beta=0.0, plan: Plan | None = None, ws=None,
             stream=None, ldb=None, ldc=None) -> None:
    """C = beta*C + diag(a_scale) A (diag(b_scale) B) through the C ABI."""
    lib = load_library()
    if plan is None and tile_rows == 0:
        tile_rows = 1
    if plan is None and tile_cols == 0:
        tile_cols = 1
    ldb = B.stride(0) if ldb is None else ldb
    ldc = C.stride(0) if ldc is None else ldc
    ws_bytes = ws.numel() * ws.element_size() if ws is not None else 0
    _check(lib.spmm_csr(_ptr(rowptr), _ptr(colind), _ptr(vals), dtype_code(vals.dtype),
                        _ptr(a_scale), _ptr(B), dtype_code(B.dtype), _ptr(b_scale), int(ldb),
                        _ptr(C), int(ldc), int(M), int(K), int(N), int(nnz), int(tile_rows),
                        int(tile_cols), float(beta), plan.handle if plan is not None else None,
                        _ptr(ws), int(ws_bytes), _stream(stream)), "spmm_csr")


def spmm_csr_noalloc(rowptr, colind, vals, B, C, M, K, N, nnz, *, a_scale=None, b_scale=None,
                     tile_rows=1, tile_cols=1, beta=0.0, stream=None) -> None:
    """spmm_csr without a workspace (the library's fixed device scratch array)."""
    _check(load_library().spmm_csr_noalloc(
        _ptr(rowptr), _ptr(colind), _ptr(vals), dtype_code(vals.dtype), _ptr(a_scale), _ptr(B),
        dtype_code(B.dtype), _ptr(b_scale), int(B.stride(0)), _ptr(C), int(C.stride(0)), int(M),
        int(K), int(N), int(nnz), int(tile_rows), int(tile_cols), float(beta), _stream(stream)),
        "spmm_csr_noalloc")


def spmm_bench_gather(colind, nnz, B, K, N, tile_cols, out, *, items_per_group=64,
                      ctas_per_sm=0, stream=None) -> None:
    """The B gathers of spmm_csr alone (measurement kernel); adds the sum of all
    values read to ``out[0]``."""
    _check(load_library().spmm_bench_gather(
        _ptr(colind), int(nnz), _ptr(B), dtype_code(B.dtype), int(B.stride(0)), int(K), int(N),
        int(tile_cols), int(items_per_group), int(ctas_per_sm), _ptr(out), _stream(stream)),
        "spmm_bench_gather")


def spmm_csr_noalloc_status(stream=None) -> int:
    """Read and clear the device status word of spmm_csr_noalloc's fixed array
    on the current device (synchronises ``stream``)."""
    st = ctypes.c_int32()
    _check(load_library().spmm_csr_noalloc_status(ctypes.byref(st), _stream(stream)),
           "spmm_csr_noalloc_status")
    return int(st.value)


def spmm_selftest_wait_timeout(ws, limit_cycles: int = 1 << 20, stream=None) -> None:
    """Run the bounded-wait self-test; the status word of ``ws`` then holds
    SPMM_ERR_TIMEOUT (read it with spmm_get_device_status)."""
    _check(load_library().spmm_selftest_wait_timeout(_ptr(ws), ws.numel() * ws.element_size(),
                                                     int(limit_cycles), _stream(stream)),
           "spmm_selftest_wait_timeout")


def spmm_csr_validate(rowptr, colind, M, K, nnz, ws, stream=None) -> None:
    _check(load_library().spmm_csr_validate(_ptr(rowptr), _ptr(colind), int(M), int(K), int(nnz),
                                            _ptr(ws), ws.numel() * ws.element_size(),
                                            _stream(stream)), "spmm_csr_validate")


def spmm_get_device_status(ws, stream=None) -> int:
    st = ctypes.c_int32()
    _check(load_library().spmm_get_device_status(_ptr(ws), ctypes.byref(st), _stream(stream)),
           "spmm_get_device_status")
    return int(st.value)


def spmm_csr_transpose_workspace_size(M, K, nnz) -> int:
    n = ctypes.c_size_t()
    _check(load_library().spmm_csr_transpose_workspace_size(int(M), int(K), int(nnz),
                                                            ctypes.byref(n)),
           "spmm_csr_transpose_workspace_size")
    return int(n.value)


def spmm_csr_transpose(rowptr, colind, vals, M, K, nnz, out_colptr, out_rowind, out_vals=None,
                       out_perm=None, ws=None, stream=None) -> None:
    dt = dtype_code(vals.dtype) if vals is not None else SPMM_F32
    _check(load_library().spmm_csr_transpose(
        _ptr(rowptr), _ptr(colind), _ptr(vals), dt, int(M), int(K), int(nnz), _ptr(out_colptr),
        _ptr(out_rowind), _ptr(out_vals), _ptr(out_perm), _ptr(ws),
        ws.numel() * ws.element_size() if ws is not None else 0, _stream(stream)),
        "spmm_csr_transpose")


def spmm_gather_values(vals, perm, nnz, out_vals, stream=None) -> None:
    _check(load_library().spmm_gather_values(_ptr(vals), dtype_code(vals.dtype), _ptr(perm),
                                             int(nnz), _ptr(out_vals), _stream(stream)),
           "spmm_gather_values")


def spmm_sddmm_csr(rowptr, colind, dC, B, out_vals, M, K, N, nnz, plan: Plan | None = None,
                   ws=None, stream=None) -> None:
    _check(load_library().spmm_sddmm_csr(
        _ptr(rowptr), _ptr(colind), _ptr(dC), int(dC.stride(0)), _ptr(B), dtype_code(B.dtype),
        int(B.stride(0)), _ptr(out_vals), int(M), int(K), int(N), int(nnz),
        plan.handle if plan is not None else None, _ptr(ws),
        ws.numel() * ws.element_size() if ws is not None else 0, _stream(stream)),
        "spmm_sddmm_csr")


def spmm_quantize_rows(X, dtype: int, Xq, scale=None, stream=None) -> None:
    rows, cols = X.shape
    _check(load_library().spmm_quantize_rows(_ptr(X), rows, cols, int(X.stride(0)), int(dtype),
                                             _ptr(Xq), int(Xq.stride(0)), _ptr(scale),
                                             _stream(stream)), "spmm_quantize_rows")


class Batch:
    """Owner of a spmm_batch handle: many products in one persistent launch.

    ``problems`` is a list of dicts with keys rowptr, colind, vals, B, C (device
    tensors), M, K, N and optionally a_scale, b_scale, beta, tile_rows,
    tile_cols, chunk_items.  The tensors must outlive the batch."""

    def __init__(self, problems, stream=None):
        lib = load_library()
        self.count = len(problems)
        self._keep = problems
        arr = (spmm_problem * self.count)()
        a_dt = b_dt = None
        for k, q in enumerate(problems):
            e = arr[k]
            e.rowptr, e.colind = q["rowptr"].data_ptr(), q["colind"].data_ptr()
            e.vals = q["vals"].data_ptr()
            e.a_scale = q["a_scale"].data_ptr() if q.get("a_scale") is not None else None
            e.B, e.C = q["B"].data_ptr(), q["C"].data_ptr()
            e.b_scale = q["b_scale"].data_ptr() if q.get("b_scale") is not None else None
            e.M, e.K, e.N = int(q["M"]), int(q["K"]), int(q["N"])
            e.nnz = int(q["colind"].numel())
            e.ldb, e.ldc = int(q["B"].stride(0)), int(q["C"].stride(0))
            e.beta = float(q.get("beta", 0.0))
            e.tile_rows = int(q.get("tile_rows", 0))
            e.tile_cols = int(q.get("tile_cols", 0))
            e.chunk_items = int(q.get("chunk_items", 0))
            a_dt = dtype_code(q["vals"].dtype) if a_dt is None else a_dt
            b_dt = dtype_code(q["B"].dtype) if b_dt is None else b_dt
        self.handle = ctypes.c_void_p()
        _check(lib.spmm_batch_create(ctypes.byref(self.handle), arr, self.count, a_dt, b_dt,
                                     _stream(stream)), "spmm_batch_create")
        n = ctypes.c_size_t()
        _check(lib.spmm_batch_workspace_size(self.handle, ctypes.byref(n)),
               "spmm_batch_workspace_size")
        self.workspace_bytes = int(n.value)

    def run(self, ws, stream=None):
        _check(load_library().spmm_csr_batched(self.handle, _ptr(ws), ws.numel(),
                                               _stream(stream)), "spmm_csr_batched")

    def graph_launch(self, ws, stream=None):
        _check(load_library().spmm_batch_graph_launch(self.handle, _ptr(ws), ws.numel(),
                                                      _stream(stream)), "spmm_batch_graph_launch")

    def autotune(self, ws, reps=3, stream=None, cache: str | None = None) -> float:
        """Tune the per-size-class shapes (spmm_batch_autotune) and return the
        best time in ms.  With ``cache`` (a JSON path), shapes stored there for
        a batch of the same signature are set instead of tuning, and newly
        tuned shapes are stored."""
        from . import tuning_cache
        sig = None
        self.last_tune_from_cache = False
        if cache is not None:
            sig = tuning_cache.batch_signature(self._keep, torch.cuda.get_device_name())
            hit = tuning_cache.load(cache, sig, self.count)
            if hit is not None:
                self.set_shapes(hit["tile_rows"], hit["tile_cols"], hit["chunk_items"], stream)
                self.last_tune_from_cache = True
                return hit["ms"]
        ms = ctypes.c_float()
        _check(load_library().spmm_batch_autotune(self.handle, _ptr(ws), ws.numel(), int(reps),
                                                  _stream(stream), ctypes.byref(ms)),
               "spmm_batch_autotune")
        if cache is not None:
            tuning_cache.store(cache, sig, *self.shapes(), float(ms.value))
        return float(ms.value)

    def shapes(self):
        n = self.count
        tr, tc, d = (ctypes.c_int32 * n)(), (ctypes.c_int32 * n)(), (ctypes.c_int32 * n)()
        _check(load_library().spmm_batch_get_shapes(self.handle, tr, tc, d),
               "spmm_batch_get_shapes")
        return list(tr), list(tc), list(d)

    def set_shapes(self, tile_rows=None, tile_cols=None, chunk_items=None, stream=None):
        n = self.count

        def arr(v):
            return None if v is None else (ctypes.c_int32 * n)(*[int(x) for x in v])
        _check(load_library().spmm_batch_set_shapes(self.handle, arr(tile_rows), arr(tile_cols),
                                                    arr(chunk_items), _stream(stream)),
               "spmm_batch_set_shapes")

    def close(self):
        if self.handle:
            load_library().spmm_batch_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def spgemm(A_rowptr, A_colind, A_vals, M: int, K: int, B_rowptr, B_colind, B_vals, N: int,
           stream=None, ws: torch.Tensor | None = None):
    """C = A * B for device CSR A (M x K) and B (K x N), FP32 values: spmm_spgemm_analyze,
    spmm_spgemm and spmm_spgemm_copy.  Returns (rowptr, colind, vals) on the device."""
    lib = load_library()
    nnzA = int(A_colind.numel())
    P, wsb = ctypes.c_int64(), ctypes.c_size_t()
    st = _stream(stream)
    _check(lib.spmm_spgemm_analyze(_ptr(A_rowptr), _ptr(A_colind), int(M), int(K), nnzA,
                                   _ptr(B_rowptr), int(N), ctypes.byref(P), ctypes.byref(wsb),
                                   st), "spmm_spgemm_analyze")
    dev = A_rowptr.device
    if ws is None or ws.numel() < wsb.value:
        ws = workspace(wsb.value, dev)
    E = ctypes.c_int64()
    _check(lib.spmm_spgemm(_ptr(A_rowptr), _ptr(A_colind), _ptr(A_vals), int(M), int(K), nnzA,
                           _ptr(B_rowptr), _ptr(B_colind), _ptr(B_vals), int(N), P.value,
                           _ptr(ws), wsb.value, ctypes.byref(E), st), "spmm_spgemm")
    rowptr = torch.empty(int(M) + 1, dtype=torch.int32, device=dev)
    colind = torch.empty(max(E.value, 1), dtype=torch.int32, device=dev)
    vals = torch.empty(max(E.value, 1), dtype=torch.float32, device=dev)
    _check(lib.spmm_spgemm_copy(_ptr(ws), int(M), nnzA, P.value, E.value, _ptr(rowptr),
                                _ptr(colind), _ptr(vals), st), "spmm_spgemm_copy")
    return rowptr, colind[:E.value], vals[:E.value], P.value
