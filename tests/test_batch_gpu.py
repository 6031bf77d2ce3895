"""Batched SpMM: many uneven products in one persistent launch, plain and from a
CUDA graph, before and after autotuning, against the FP64 oracle (on the stored
BF16 values) and against one spmm_csr call per product."""
import numpy as np
import pytest
import torch

import oracle
from paper_2311_18141_gb300 import binding, inputs

from gpu_util import TOL_F32, assert_close_rel

pytestmark = pytest.mark.gpu


def make_batch(count, seed, dtype, widths, rows_hi=20000, beta=0.0):
    specs = inputs.batch_specs(count, seed=seed, rows_lo=50, rows_hi=rows_hi, widths=widths)
    probs, host = [], []
    for k, sp in enumerate(specs):
        A = inputs.poisson_csr(sp.rows, sp.rows, sp.mean_nnz, seed=sp.seed, device="cuda")
        B = inputs.dense_normal(A.K, sp.N, seed=sp.seed + 1, device="cuda")
        vals = A.vals.to(dtype)
        Bq = B.to(dtype)
        C = inputs.dense_normal(A.M, sp.N, seed=sp.seed + 2, device="cuda") if beta else \
            torch.full((A.M, sp.N), float("nan"), device="cuda")
        probs.append(dict(rowptr=A.rowptr, colind=A.colind, vals=vals, B=Bq, C=C, M=A.M, K=A.K,
                          N=sp.N, beta=beta))
        host.append((A, vals, Bq, C.clone()))
    return probs, host


def as_f64(t):
    if t.dtype == torch.bfloat16:
        return oracle.decode_bf16(t.view(torch.int16).cpu().numpy().view(np.uint16))
    return t.cpu().numpy().astype(np.float64)


def check(probs, host, what):
    for q, (A, vals, Bq, C0) in zip(probs, host):
        v = as_f64(vals)
        b = as_f64(Bq).reshape(A.K, q["N"])
        beta = q["beta"]
        ref = oracle.spmm(A.rowptr.cpu(), A.colind.cpu(), v, b, beta=beta,
                          C0=C0.cpu().numpy() if beta else None)
        bound = oracle.spmm(A.rowptr.cpu(), A.colind.cpu(), np.abs(v), np.abs(b))
        if beta:
            bound = bound + abs(beta) * np.abs(C0.cpu().numpy())
        assert_close_rel(q["C"].cpu().numpy(), ref, bound, TOL_F32, what)


@pytest.mark.parametrize("dtype,widths", [(torch.bfloat16, (16, 64, 128)),
                                          (torch.float32, (16, 32, 128, 256))])
def test_batch_matches_oracle_plain_graph_autotuned(dtype, widths):
    probs, host = make_batch(24, seed=71, dtype=dtype, widths=widths)
    batch = binding.Batch(probs)
    ws = binding.workspace(batch.workspace_bytes)
    batch.run(ws)
    torch.cuda.synchronize()
    check(probs, host, "batched")
    first = [q["C"].clone() for q in probs]
    # CUDA-graph replay, twice: same bits as the plain launch
    for q in probs:
        q["C"].fill_(float("nan"))
    batch.graph_launch(ws)
    batch.graph_launch(ws)
    torch.cuda.synchronize()
    for q, c in zip(probs, first):
        assert torch.equal(q["C"], c)
    # autotune, then the tuned shapes still give the right answer
    ms = batch.autotune(ws, reps=2)
    assert ms > 0
    tr, tc, d = batch.shapes()
    assert all(x >= 1 for x in tr + tc) and all(x >= 256 for x in d)
    for q in probs:
        q["C"].fill_(float("nan"))
    batch.graph_launch(ws)
    torch.cuda.synchronize()
    check(probs, host, "autotuned")
    batch.close()


def test_batch_equals_sequential_calls_and_accumulates():
    probs, host = make_batch(12, seed=72, dtype=torch.bfloat16, widths=(16, 64), beta=1.0)
    seq = []
    for q, (A, vals, Bq, C0) in zip(probs, host):
        C = C0.clone()
        ws = binding.workspace(binding.spmm_csr_workspace_size(A.M, A.nnz, q["N"], 1, 1))
        binding.spmm_csr(A.rowptr, A.colind, vals, Bq, C, A.M, A.K, q["N"], A.nnz, beta=1.0,
                         ws=ws)
        seq.append(C)
    batch = binding.Batch(probs)
    ws = binding.workspace(batch.workspace_bytes)
    batch.run(ws)
    torch.cuda.synchronize()
    check(probs, host, "batched beta=1")
    for q, c in zip(probs, seq):
        torch.testing.assert_close(q["C"], c, rtol=1e-5, atol=1e-5)
    batch.close()


def test_batch_rejects_mixed_or_bad_problems():
    probs, _ = make_batch(3, seed=73, dtype=torch.float32, widths=(16,))
    probs[1]["C"] = torch.zeros(probs[1]["M"] * 16 + 1, device="cuda")[1:].view(-1, 16)
    with pytest.raises(binding.SpmmError) as e:
        binding.Batch(probs)
    assert e.value.status == binding.SPMM_ERR_MISALIGNED


def test_autotune_cache_round_trip(tmp_path):
    """Tuned shapes are stored under the batch's signature; a new batch over the
    same problems sets them from the cache (no tuning) and still computes the
    oracle's products."""
    path = str(tmp_path / "tune.json")
    probs, host = make_batch(16, seed=73, dtype=torch.bfloat16, widths=(16, 64, 128))
    batch = binding.Batch(probs)
    ws = binding.workspace(batch.workspace_bytes)
    ms = batch.autotune(ws, cache=path)
    assert ms > 0 and not batch.last_tune_from_cache
    tuned = batch.shapes()
    batch.close()
    again = binding.Batch(probs)
    assert again.autotune(ws, cache=path) == pytest.approx(ms)
    assert again.last_tune_from_cache and again.shapes() == tuned
    for q in probs:
        q["C"].fill_(float("nan"))
    again.graph_launch(ws)
    torch.cuda.synchronize()
    assert binding.spmm_get_device_status(ws) == 0
    check(probs, host, "batch with cached shapes")
    again.close()


def test_batch_heavy_rows_cut_into_many_pieces():
    """Products each holding rows of thousands of nonzeros, which the plan cuts
    across dozens of chunks: the batched split-row sum adds more pieces per row
    than it has slot loads in flight, for several products of one launch, with
    beta = 1 on a random C."""
    rng = np.random.default_rng(74)
    probs, host = [], []
    for k, (M, K, N, heavy) in enumerate([(700, 8000, 16, 6000), (1500, 9000, 64, 8000),
                                          (900, 4000, 64, 3500), (400, 12000, 16, 11000)]):
        lens = rng.integers(0, 30, M)
        lens[rng.integers(0, M, 3)] = heavy        # three heavy rows per product
        lens[0] = 0
        lens[-1] = 5
        rowptr = np.zeros(M + 1, np.int64)
        rowptr[1:] = np.cumsum(lens)
        colind = np.concatenate([np.sort(rng.choice(K, int(l), replace=False)) for l in lens if l])
        vals = torch.from_numpy(rng.uniform(-1, 1, colind.size).astype(np.float32)).to(torch.bfloat16)
        B = inputs.dense_normal(K, N, seed=80 + k, device="cuda").to(torch.bfloat16)
        C0 = inputs.dense_normal(M, N, seed=90 + k, device="cuda")
        rp = torch.from_numpy(rowptr.astype(np.int32)).cuda()
        ci = torch.from_numpy(colind.astype(np.int32)).cuda()
        probs.append(dict(rowptr=rp, colind=ci, vals=vals.cuda(), B=B, C=C0.clone(), M=M, K=K, N=N,
                          beta=1.0))
        A = inputs.CSR(rp, ci, vals.float().cuda(), M, K)
        host.append((A, vals, B, C0.clone()))
    batch = binding.Batch(probs)
    ws = binding.workspace(batch.workspace_bytes)
    batch.run(ws)
    torch.cuda.synchronize()
    assert binding.spmm_get_device_status(ws) == 0
    check(probs, host, "batched heavy rows")
    batch.close()
