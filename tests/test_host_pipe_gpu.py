"""Host-buffer pipeline (spmm_host_pipe_*): every step's C, copied back into
host memory, equals the device call on the same inputs bit for bit and the
FP64 oracle within the FP32 tolerance, whatever the pipeline depth, with inputs
that change from step to step (so a slot reused too early would show)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2311_18141_gb300 import binding, inputs

from gpu_util import TOL_F32, TOL_LOWP, assert_close_rel

pytestmark = pytest.mark.gpu
DEV = "cuda"


def device_product(A, vals, B, N, plan):
    ws = binding.workspace(plan.workspace_bytes)
    Ad = A.to(DEV)
    C = torch.empty(A.M, N, device=DEV)
    binding.spmm_csr(Ad.rowptr, Ad.colind, vals.to(DEV), B.to(DEV), C, A.M, A.K, N, A.nnz,
                     plan=plan, ws=ws)
    torch.cuda.synchronize()
    assert binding.spmm_get_device_status(ws) == 0
    return C.cpu()


def step_inputs(A, N, k, vdtype=torch.float32, bdtype=torch.float32):
    vals = (A.vals * (1.0 + 0.25 * k)).to(vdtype)
    B = inputs.dense_normal(A.K, N, seed=100 + k).to(bdtype)
    return vals, B


@pytest.mark.parametrize("depth", [1, 2, 3])
@pytest.mark.parametrize("pinned", [True, False])
def test_pipe_matches_device_call_and_oracle(depth, pinned):
    A = inputs.rmat_csr(12, 16, seed=3)
    N, steps = 64, 5
    plan = binding.Plan(A.rowptr.to(DEV), A.M, A.K, A.nnz, N, 4, 2)
    pipe = binding.HostPipe(plan, torch.float32, torch.float32, depth=depth)
    pin = (lambda t: t.pin_memory()) if pinned else (lambda t: t.contiguous())
    rp, ci = pin(A.rowptr), pin(A.colind)
    ins, outs = [], []
    for k in range(steps):
        vals, B = step_inputs(A, N, k)
        vals, B = pin(vals), pin(B)
        C = pin(torch.full((A.M, N), float("nan")))
        pipe.submit(rp, ci, vals, B, C)
        ins.append((vals, B))
        outs.append(C)
    pipe.wait()
    for k in range(steps):
        vals, B = ins[k]
        want = device_product(A, vals, B, N, plan)
        assert torch.equal(outs[k], want), f"step {k}"
    vals, B = ins[-1]
    ref = oracle.spmm(A.rowptr, A.colind, vals, B)
    bound = oracle.abs_bound(A.rowptr, A.colind, vals, B)
    assert_close_rel(outs[-1].numpy(), ref, bound, TOL_F32, f"pipe depth {depth}")
    pipe.close()
    plan.close()


def test_pipe_narrow_storage():
    """FP16 A values and BF16 B through the pipeline."""
    A = inputs.rmat_csr(11, 16, seed=4)
    N, steps = 128, 3
    plan = binding.Plan(A.rowptr.to(DEV), A.M, A.K, A.nnz, N, 2, 4)
    pipe = binding.HostPipe(plan, torch.float16, torch.bfloat16, depth=2)
    ins, outs = [], []
    for k in range(steps):
        vals, B = step_inputs(A, N, k, torch.float16, torch.bfloat16)
        C = torch.empty(A.M, N).pin_memory()
        pipe.submit(A.rowptr.pin_memory(), A.colind.pin_memory(), vals.pin_memory(),
                    B.pin_memory(), C)
        ins.append((vals, B))
        outs.append(C)
    pipe.wait()
    for k in range(steps):
        vals, B = ins[k]
        assert torch.equal(outs[k], device_product(A, vals, B, N, plan)), f"step {k}"
        v64 = vals.double()
        b64 = B.double()
        ref = oracle.spmm(A.rowptr, A.colind, v64.numpy(), b64.numpy())
        bound = oracle.abs_bound(A.rowptr, A.colind, v64.numpy(), b64.numpy())
        assert_close_rel(outs[k].numpy(), ref, bound, TOL_F32, "dequantised inputs")
    pipe.close()
    plan.close()


def test_pipe_empty_matrix_and_many_steps():
    """nnz = 0 gives C = 0; twelve steps through two slots reuse each slot six times."""
    M, K, N = 300, 200, 32
    rowptr = torch.zeros(M + 1, dtype=torch.int32)
    colind = torch.zeros(0, dtype=torch.int32)
    vals = torch.zeros(0)
    plan = binding.Plan(rowptr.to(DEV), M, K, 0, N, 3, 1)
    pipe = binding.HostPipe(plan, torch.float32, torch.float32, depth=2)
    outs = []
    for _ in range(12):
        C = torch.full((M, N), 7.0).pin_memory()
        pipe.submit(rowptr.pin_memory(), colind, vals, torch.zeros(K, N).pin_memory(), C)
        outs.append(C)
    pipe.wait()
    for C in outs:
        assert torch.count_nonzero(C) == 0
    pipe.close()
    plan.close()


def test_pipe_rejects_bad_arguments():
    A = inputs.uniform_csr(64, 64, 4, seed=5)
    plan = binding.Plan(A.rowptr.to(DEV), A.M, A.K, A.nnz, 8, 1, 1)
    with pytest.raises(binding.SpmmError):
        binding.HostPipe(plan, torch.float32, torch.float32, depth=0)
    with pytest.raises(binding.SpmmError):
        binding.HostPipe(plan, torch.float32, torch.float32, depth=5)
    pipe = binding.HostPipe(plan, torch.float32, torch.float32, depth=2)
    with pytest.raises(ValueError):
        pipe.submit(A.rowptr.to(DEV), A.colind, A.vals, torch.zeros(64, 8), torch.zeros(64, 8))
    pipe.wait()
    pipe.close()
    # B width that breaks the BF16 vector rule (8 elements per 16 bytes)
    plan6 = binding.Plan(A.rowptr.to(DEV), A.M, A.K, A.nnz, 12, 1, 1)
    with pytest.raises(binding.SpmmError):
        binding.HostPipe(plan6, torch.float32, torch.bfloat16)
    plan.close()
    plan6.close()
