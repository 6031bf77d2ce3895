"""Narrow storage: quantisation is bit-exact against the oracle's codecs, and
SpMM on BF16/FP16/E4M3 storage matches the FP64 product of the dequantised
inputs to FP32 accuracy, and the FP64 product of the original FP32 data within
the storage format's error."""
import numpy as np
import pytest
import torch

import oracle
from paper_2311_18141_gb300 import binding, inputs

from gpu_util import TOL_F32, TOL_LOWP, assert_close_rel, run_spmm

pytestmark = pytest.mark.gpu


def quantize_gpu(X, dtype):
    Xd = X.cuda()
    rows, cols = X.shape
    if dtype == binding.SPMM_E4M3:
        q = torch.empty(rows, cols, dtype=torch.uint8, device="cuda")
        s = torch.empty(rows, dtype=torch.float32, device="cuda")
    else:
        q = torch.empty(rows, cols, dtype=torch.bfloat16 if dtype == binding.SPMM_BF16
                        else torch.float16, device="cuda")
        s = None
    binding.spmm_quantize_rows(Xd, dtype, q, s)
    torch.cuda.synchronize()
    return q, s


def test_quantize_e4m3_bit_exact():
    X = inputs.dense_normal(3000, 256, seed=31)
    X[7] = 0.0
    X[9, :5] = torch.tensor([1e-9, -3e-4, 2.0 ** -10, 5.0, -5.0])
    q, s = quantize_gpu(X, binding.SPMM_E4M3)
    q_ref, s_ref = oracle.quantize_rows_e4m3(X.numpy())
    np.testing.assert_array_equal(s.cpu().numpy(), s_ref)
    np.testing.assert_array_equal(q.cpu().numpy(), q_ref)


@pytest.mark.parametrize("dt,enc", [(binding.SPMM_BF16, oracle.encode_bf16),
                                    (binding.SPMM_F16, oracle.encode_f16)])
def test_quantize_16bit_bit_exact(dt, enc):
    X = inputs.dense_normal(2000, 64, seed=32) * 1000.0
    q, _ = quantize_gpu(X, dt)
    bits = q.cpu().view(torch.int16).numpy().view(np.uint16)
    np.testing.assert_array_equal(bits, enc(X.numpy()))


def _store_b(B, fmt):
    if fmt == "f32":
        return B.cuda(), None, B.numpy().astype(np.float64)
    if fmt == "e4m3":
        q, s = quantize_gpu(B, binding.SPMM_E4M3)
        deq = oracle.dequantize_rows(q.cpu().numpy(), s.cpu().numpy(), "e4m3")
        return q, s, deq
    dt = binding.SPMM_BF16 if fmt == "bf16" else binding.SPMM_F16
    q, _ = quantize_gpu(B, dt)
    bits = q.cpu().view(torch.int16).numpy().view(np.uint16)
    deq = oracle.decode_bf16(bits) if fmt == "bf16" else oracle.decode_f16(bits)
    return q, None, deq


def _store_vals(vals, fmt):
    if fmt == "f32":
        return vals, vals.numpy().astype(np.float64), None
    if fmt == "f16":
        v = vals.to(torch.float16)
        return v, oracle.decode_f16(v.view(torch.int16).numpy().view(np.uint16)), None
    if fmt == "bf16":
        v = vals.to(torch.bfloat16)
        return v, oracle.decode_bf16(v.view(torch.int16).numpy().view(np.uint16)), None
    q, s = oracle.quantize_rows_e4m3(vals.numpy()[None, :])  # one scale for the whole matrix
    deq = oracle.decode_e4m3(q[0]) * float(s[0])
    return torch.from_numpy(q[0]), deq, float(s[0])


@pytest.mark.parametrize("afmt", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("bfmt", ["f32", "bf16", "f16", "e4m3"])
def test_spmm_storage_formats(afmt, bfmt):
    A = inputs.rmat_csr(12, 16, seed=33)
    N = 256 if bfmt != "f32" else 128
    B = inputs.dense_normal(A.K, N, seed=34)
    Bq, bscale, Bdeq = _store_b(B, bfmt)
    vq, vdeq, _ = _store_vals(A.vals, afmt)
    C, st = run_spmm(A, B, N, vals=vq, b_scale=bscale, Bdev=Bq, tile_rows=4, tile_cols=2,
                     chunk_items=200)
    assert st == 0
    # kernel error: against the FP64 product of exactly what was stored
    ref_deq = oracle.spmm(A.rowptr, A.colind, vdeq, Bdeq)
    bound_deq = oracle.spmm(A.rowptr, A.colind, np.abs(vdeq), np.abs(Bdeq))
    assert_close_rel(C.numpy(), ref_deq, bound_deq, TOL_F32, f"{afmt}/{bfmt} vs dequantised")
    # storage error: against the FP64 product of the original FP32 data
    ref = oracle.spmm(A.rowptr, A.colind, A.vals, B)
    bound = oracle.abs_bound(A.rowptr, A.colind, A.vals, B)
    if bfmt in ("f32", "bf16", "f16"):
        assert_close_rel(C.numpy(), ref, bound, TOL_LOWP if (afmt, bfmt) != ("f32", "f32")
                         else TOL_F32, f"{afmt}/{bfmt} vs original")
    else:
        # E4M3: |err| <= (2^-4 + u_A) |A||B| + |A| s 2^-10 (subnormal step), u_A of A's format
        uA = {"f32": 2.0 ** -24, "f16": 2.0 ** -11, "bf16": 2.0 ** -8}[afmt]
        sub = oracle.spmm(A.rowptr, A.colind, np.abs(A.vals.numpy().astype(np.float64)),
                          np.repeat(bscale.cpu().numpy().astype(np.float64)[:, None], N, 1))
        err = np.abs(C.numpy().astype(np.float64) - ref)
        assert np.all(err <= (2.0 ** -4 + uA + 1e-5) * bound + 2.0 ** -10 * sub)


def test_e4m3_values_with_row_scale():
    A = inputs.rmat_csr(11, 16, seed=35, values="sym")
    N = 64
    B = inputs.dense_normal(A.K, N, seed=36)
    vq, vdeq, s = _store_vals(A.vals, "e4m3")
    ascale = torch.full((A.M,), s, dtype=torch.float32)
    C, st = run_spmm(A, B, N, vals=vq.view(torch.uint8), a_scale=ascale, tile_rows=2)
    assert st == 0
    ref = oracle.spmm(A.rowptr, A.colind, vdeq, B)
    bound = oracle.spmm(A.rowptr, A.colind, np.abs(vdeq), np.abs(B.numpy().astype(np.float64)))
    assert_close_rel(C.numpy(), ref, bound, TOL_F32, "e4m3 vals + row scale")


def test_storage_formats_error_against_fp64():
    """The precision workload's error check at test size: FP32, BF16 and E4M3
    storage of B (FP16 A values) against the FP64 product of the original data,
    max and RMS normalised by |A||B|; BF16 within 1e-2, E4M3 within its stated
    bound.  (Which format is faster is measured by bench.py, not here.)"""
    A = inputs.rmat_csr(12, 16, seed=37)
    N = 256
    B = inputs.dense_normal(A.K, N, seed=38)
    ref = oracle.spmm(A.rowptr, A.colind, A.vals, B)
    bound = oracle.abs_bound(A.rowptr, A.colind, A.vals, B)
    v16 = A.vals.to(torch.float16)
    out = {}
    for fmt in ("f32", "bf16", "e4m3"):
        Bq, bscale, _ = _store_b(B, fmt)
        C, st = run_spmm(A, B, N, vals=v16, b_scale=bscale, Bdev=Bq)
        err = np.abs(C.numpy().astype(np.float64) - ref)
        rel = err / np.maximum(bound, 1e-30)
        out[fmt] = (float(rel.max()), float(np.sqrt((rel ** 2).mean())))
        if fmt == "e4m3":
            # E4M3 with per-row scale s: relative step 2^-4 for normal codes, absolute
            # step s*2^-10 below 2^-6*s (subnormals, and values that round to zero)
            sub = oracle.spmm(A.rowptr, A.colind, np.abs(A.vals.numpy().astype(np.float64)),
                              np.repeat(bscale.cpu().numpy().astype(np.float64)[:, None], N, 1))
            assert np.all(err <= (2.0 ** -4 + 2.0 ** -11 + 1e-5) * bound + 2.0 ** -10 * sub)
    assert out["bf16"][0] <= 1e-2 and out["f32"][0] <= 1e-2
    print("normalised error max/rms:", out)
