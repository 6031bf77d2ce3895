"""spmm_bench_gather, the measurement kernel that issues the SpMM's B gathers
alone (Section 4's B term, reloads included): it must read, for every nonzero
and column block, the block's segment of B row colind[e].

B's row k holds k mod 97 plus a column pattern, so the sum of everything read
is N * sum_e (colind[e] mod 97) + nnz * sum_n (n mod 5), exactly; a gather of a
wrong row, or a missed or doubled one, moves the sum far outside the FP32
rounding of the float atomics."""
import numpy as np
import pytest
import torch

from paper_2311_18141_gb300 import binding, inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N,TC,S", [(128, 4, 64), (128, 1, 64), (64, 1, 8), (256, 4, 4096),
                                    (96, 3, 16), (512, 2, 32)])
def test_gather_reads_the_rows_of_colind(N, TC, S):
    A = inputs.rmat_csr(12, 16, seed=90)
    K = A.K
    rows = (torch.arange(K, dtype=torch.float32) % 97)[:, None]
    cols = (torch.arange(N, dtype=torch.float32) % 5)[None, :]
    B = (rows + cols).cuda()
    ci = A.colind.numpy().astype(np.int64)
    expected = N * float((ci % 97).sum()) + A.nnz * float((np.arange(N) % 5).sum())
    out = torch.zeros(1, device="cuda")
    binding.spmm_bench_gather(A.colind.cuda(), A.nnz, B, K, N, TC, out, items_per_group=S)
    torch.cuda.synchronize()
    # all terms are positive: FP32 sums of up to 4096 terms per lane stay far
    # inside 1e-4 of the total, while reading wrong rows, or missing or doubling
    # a column block, moves it by percents
    assert abs(float(out.item()) - expected) <= 1e-4 * expected


def test_gather_rejects_unaligned_segments():
    A = inputs.uniform_csr(64, 64, 4, seed=91)
    out = torch.zeros(1, device="cuda")
    for N, TC in [(8, 1), (36, 1), (128, 16), (64, 3)]:
        B = torch.zeros(64, N, device="cuda")
        with pytest.raises(binding.SpmmError):
            binding.spmm_bench_gather(A.colind.cuda(), A.nnz, B, 64, N, TC, out)
