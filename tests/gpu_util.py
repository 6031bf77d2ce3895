"""Helpers for the GPU parity tests: run the CUDA path through the C ABI and
compare with the FP64 oracle element by element."""
import numpy as np
import torch

import oracle
from paper_2311_18141_gb300 import binding

DEV = "cuda"

# Tolerances, from the arithmetic: an FP32 sum of products with random signs has
# a normalised error of a few units of 2^-24, far inside 1e-5; BF16 storage
# rounds each input by at most 2^-9 relative, inside 1e-2.
#   FP32 storage: |C - C64| <= 1e-5 * (|A| |B|) elementwise.
#   BF16/FP16 storage vs the FP64 product of the ORIGINAL fp32 data:
#                 |C - C64| <= 1e-2 * (|A| |B|).
#   any storage vs the FP64 product of the DEQUANTISED inputs: 1e-5 * (|A| |B|).
TOL_F32 = 1e-5
TOL_LOWP = 1e-2


# kernels a test can ask for (spmm_tuning.kernel): the 16-byte staged kernel, and
# the 32-byte-lane kernel wherever B, C and the column blocks are whole 32-byte
# vectors (elsewhere run_spmm asks for the library's default instead)
KERNELS = [binding.SPMM_KERNEL_STAGED, binding.SPMM_KERNEL_WIDE]


def wide_ok(N, TC, esz=4):
    """Whether the 32-byte-lane kernel accepts N columns in TC blocks (dense,
    aligned tensors)."""
    epv = 16 // esz
    w = -(-N // TC)
    w = -(-w // epv) * epv
    nb = w * esz
    return nb % 32 == 0 and (N * esz) % 32 == 0 and 2 <= nb // 32 <= 32


def run_spmm(A, B, N, *, tile_rows=1, tile_cols=1, beta=0.0, C0=None, chunk_items=0,
             warps_per_cta=0, tile_order=0, vals=None, a_scale=None, b_scale=None, plan=True,
             Bdev=None, kernel=binding.SPMM_KERNEL_AUTO):
    """Run spmm_csr on the GPU; returns C (float32, on the host) and the status word."""
    Ad = A.to(DEV)
    v = (vals if vals is not None else A.vals).to(DEV)
    Bd = Bdev if Bdev is not None else B.to(DEV)
    if C0 is not None:
        C = C0.clone().to(DEV)
    else:
        C = torch.full((A.M, N), float("nan"), device=DEV)
    esz = (Bdev.element_size() if Bdev is not None else 4)
    if kernel == binding.SPMM_KERNEL_WIDE and not wide_ok(N, tile_cols, esz):
        kernel = binding.SPMM_KERNEL_AUTO
    tun = binding.make_tuning(chunk_items=chunk_items, warps_per_cta=warps_per_cta,
                              tile_order=tile_order, kernel=kernel)
    if plan:
        pl = binding.Plan(Ad.rowptr, A.M, A.K, A.nnz, N, tile_rows, tile_cols, tuning=tun)
        ws = binding.workspace(pl.workspace_bytes)
        binding.spmm_csr(Ad.rowptr, Ad.colind, v, Bd, C, A.M, A.K, N, A.nnz, beta=beta,
                         plan=pl, ws=ws, a_scale=None if a_scale is None else a_scale.to(DEV),
                         b_scale=None if b_scale is None else b_scale.to(DEV))
    else:
        pl = None
        ws = binding.workspace(binding.spmm_csr_workspace_size(A.M, A.nnz, N, tile_rows,
                                                               tile_cols))
        binding.spmm_csr(Ad.rowptr, Ad.colind, v, Bd, C, A.M, A.K, N, A.nnz, beta=beta,
                         tile_rows=tile_rows, tile_cols=tile_cols, ws=ws,
                         a_scale=None if a_scale is None else a_scale.to(DEV),
                         b_scale=None if b_scale is None else b_scale.to(DEV))
    torch.cuda.synchronize()
    status = binding.spmm_get_device_status(ws)
    out = C.cpu()
    if pl is not None:
        pl.close()
    return out, status


def assert_close_rel(C, ref, bound, tol, what=""):
    C = np.asarray(C, dtype=np.float64)
    err = np.abs(C - ref)
    lim = tol * bound
    bad = ~(err <= lim)  # catches NaN too
    if bad.any():
        idx = np.argwhere(bad)[:5]
        raise AssertionError(
            f"{what}: {int(bad.sum())} elements out of tolerance; first {idx.tolist()} "
            f"got {[float(C[tuple(i)]) for i in idx]} want {[float(ref[tuple(i)]) for i in idx]} "
            f"bound {[float(lim[tuple(i)]) for i in idx]}")
    return float((err / np.maximum(bound, 1e-300)).max()) if err.size else 0.0
