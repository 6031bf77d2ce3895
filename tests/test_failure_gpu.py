"""Failure detection on the GPU without a fault: a bounded wait that nothing
completes runs out, the kernel records SPMM_ERR_TIMEOUT in the workspace status
word and returns, the host reads the status, and the context stays usable for
the next product."""
import time

import numpy as np
import pytest
import torch

import oracle
from paper_2311_18141_gb300 import binding, inputs

from gpu_util import TOL_F32, assert_close_rel, run_spmm

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("limit", [1, 1 << 12, 1 << 20])
def test_bounded_wait_times_out_and_reports(limit):
    ws = binding.workspace(256)
    t0 = time.perf_counter()
    binding.spmm_selftest_wait_timeout(ws, limit)
    torch.cuda.synchronize()
    elapsed = time.perf_counter() - t0
    assert binding.spmm_get_device_status(ws) == binding.SPMM_ERR_TIMEOUT
    assert elapsed < 5.0
    # reading the status clears it
    assert binding.spmm_get_device_status(ws) == binding.SPMM_OK


def test_first_error_is_kept_and_context_stays_usable():
    ws = binding.workspace(256)
    binding.spmm_selftest_wait_timeout(ws, 1 << 10)
    binding.spmm_selftest_wait_timeout(ws, 1 << 10)
    torch.cuda.synchronize()
    assert binding.spmm_get_device_status(ws) == binding.SPMM_ERR_TIMEOUT
    A = inputs.rmat_csr(10, 16, seed=61)
    B = inputs.dense_normal(A.K, 32, seed=62)
    C, st = run_spmm(A, B, 32, tile_rows=4, tile_cols=2)
    assert st == 0
    ref = oracle.spmm(A.rowptr, A.colind, A.vals, B)
    bound = oracle.abs_bound(A.rowptr, A.colind, A.vals, B)
    assert_close_rel(C.numpy(), ref, bound, TOL_F32, "product after a timed-out wait")
