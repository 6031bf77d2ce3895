"""Pins for the FP64 oracle, independent of the oracle's own code.

Each check rests on something other than the oracle: a brute-force dense
product written here, a closed form, an invariant of the definition
(Section 2.1: C_ij = C_ij + sum_k A_ik B_kj), a hand-worked fixture, or an
independent library routine (numpy, torch) for the number formats.  A dropped
term, a wrong sign or index, or a transposed operand in the oracle fails at
least one of them.
"""
import math
import os

import numpy as np
import pytest
import torch

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def random_csr(rng, M, K, density, sorted_cols=True):
    dense = (rng.random((M, K)) < density) * rng.uniform(-1, 1, (M, K))
    rowptr = [0]
    colind, vals = [], []
    for r in range(M):
        cols = np.nonzero(dense[r])[0]
        if not sorted_cols:
            cols = rng.permutation(cols)
        colind.extend(cols.tolist())
        vals.extend(dense[r, cols].tolist())
        rowptr.append(len(colind))
    return (np.array(rowptr, np.int32), np.array(colind, np.int32),
            np.array(vals, np.float64), dense)


def brute_force(dense, B):
    """Triple loop over the dense form, k increasing, zeros skipped."""
    M, K = dense.shape
    N = B.shape[1]
    C = np.zeros((M, N))
    for r in range(M):
        for n in range(N):
            s = 0.0
            for k in range(K):
                if dense[r, k] != 0.0:
                    s += dense[r, k] * B[k, n]
            C[r, n] = s
    return C


@pytest.mark.parametrize("density", [0.0, 0.15, 0.6, 1.0])
@pytest.mark.parametrize("shape", [(1, 1, 1), (7, 5, 3), (13, 17, 4), (24, 9, 8)])
def test_brute_force_exact(shape, density):
    M, K, N = shape
    rng = np.random.default_rng(M * 131 + K * 7 + int(density * 100))
    rp, ci, v, dense = random_csr(rng, M, K, density)
    B = rng.standard_normal((K, N))
    C = oracle.spmm(rp, ci, v, B)
    np.testing.assert_array_equal(C, brute_force(dense, B))
    np.testing.assert_allclose(C, dense @ B, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("threads", [1, 3])
def test_abs_bound_is_the_product_of_absolute_values(threads):
    """The tolerance scale |A|.|B|: brute force over |A| and |B|, the same for
    one thread or several, and never below |A.B|."""
    rng = np.random.default_rng(5150)
    rp, ci, v, dense = random_csr(rng, 19, 11, 0.4)
    B = rng.standard_normal((11, 6))
    prev = oracle.get_threads()
    oracle.set_threads(threads)
    try:
        bound = oracle.abs_bound(rp, ci, v, B)
    finally:
        oracle.set_threads(prev)
    np.testing.assert_array_equal(bound, brute_force(np.abs(dense), np.abs(B)))
    assert np.all(bound >= np.abs(oracle.spmm(rp, ci, v, B)))


def test_golden_hand_worked():
    fields = {}
    with open(os.path.join(GOLDEN, "spmm_3x4.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            key, *rest = line.split()
            fields[key] = [float(x) for x in rest]
    M, K, N = int(fields["M"][0]), int(fields["K"][0]), int(fields["N"][0])
    B = np.array(fields["B"]).reshape(K, N)
    C = oracle.spmm(np.array(fields["rowptr"], np.int32), np.array(fields["colind"], np.int32),
                    np.array(fields["vals"]), B)
    np.testing.assert_array_equal(C, np.array(fields["C"]).reshape(M, N))


def test_identity_permutation_scaled():
    rng = np.random.default_rng(3)
    n, N = 37, 6
    B = rng.standard_normal((n, N)).astype(np.float32)
    eye_rp = np.arange(n + 1, dtype=np.int32)
    eye_ci = np.arange(n, dtype=np.int32)
    np.testing.assert_array_equal(oracle.spmm(eye_rp, eye_ci, np.ones(n), B), B.astype(np.float64))
    perm = rng.permutation(n).astype(np.int32)
    np.testing.assert_array_equal(oracle.spmm(eye_rp, perm, np.ones(n), B), B[perm].astype(np.float64))
    np.testing.assert_array_equal(oracle.spmm(eye_rp, eye_ci, np.full(n, 0.25), B),
                                  0.25 * B.astype(np.float64))
    # A non-square identity-like selector picks the listed rows of B
    sel = np.array([4, 0, 36], np.int32)
    np.testing.assert_array_equal(oracle.spmm(np.arange(4, dtype=np.int32), sel, np.ones(3), B),
                                  B[sel].astype(np.float64))


def test_row_sums_and_closed_form():
    rng = np.random.default_rng(5)
    rp, ci, v, dense = random_csr(rng, 50, 40, 0.3)
    C = oracle.spmm(rp, ci, v, np.ones((40, 1)))
    for r in range(50):
        assert C[r, 0] == pytest.approx(math.fsum(v[rp[r]:rp[r + 1]]), abs=1e-13)
    # a single row holding k ones against B = 1 gives exactly k
    for k in (0, 1, 5, 64):
        rp1 = np.array([0, k], np.int32)
        C1 = oracle.spmm(rp1, np.arange(k, dtype=np.int32), np.ones(k), np.ones((max(k, 1), 3)))
        np.testing.assert_array_equal(C1, np.full((1, 3), float(k)))


def test_beta_accumulate():
    rng = np.random.default_rng(9)
    rp, ci, v, dense = random_csr(rng, 20, 15, 0.4)
    B = rng.standard_normal((15, 5))
    C0 = rng.standard_normal((20, 5))
    np.testing.assert_allclose(oracle.spmm(rp, ci, v, B, beta=1.0, C0=C0), C0 + dense @ B,
                               rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(oracle.spmm(rp, ci, v, B, beta=-2.0, C0=C0), -2 * C0 + dense @ B,
                               rtol=1e-13, atol=1e-13)
    # beta = 0 ignores C0 entirely, NaNs included
    bad = np.full((20, 5), np.nan)
    np.testing.assert_array_equal(oracle.spmm(rp, ci, v, B, beta=0.0, C0=bad),
                                  oracle.spmm(rp, ci, v, B))
    rows = np.array([19, 0, 7])
    np.testing.assert_array_equal(oracle.spmm_rows(rp, ci, v, B, rows, beta=1.0, C0_rows=C0[rows]),
                                  oracle.spmm(rp, ci, v, B, beta=1.0, C0=C0)[rows])


def test_linearity():
    rng = np.random.default_rng(11)
    rp, ci, v, dense = random_csr(rng, 30, 25, 0.3)
    B1 = rng.standard_normal((25, 4))
    B2 = rng.standard_normal((25, 4))
    np.testing.assert_allclose(oracle.spmm(rp, ci, v, B1 + B2),
                               oracle.spmm(rp, ci, v, B1) + oracle.spmm(rp, ci, v, B2),
                               rtol=1e-12, atol=1e-12)
    v2 = rng.uniform(-1, 1, v.size)
    np.testing.assert_allclose(oracle.spmm(rp, ci, v + v2, B1),
                               oracle.spmm(rp, ci, v, B1) + oracle.spmm(rp, ci, v2, B1),
                               rtol=1e-12, atol=1e-12)


def test_unsorted_and_duplicate_columns_sum():
    # duplicates in a row are summed; column order inside a row does not matter
    rp = np.array([0, 3], np.int32)
    ci = np.array([2, 0, 2], np.int32)
    v = np.array([1.0, 2.0, 3.0])
    B = np.array([[1.0], [10.0], [100.0]])
    np.testing.assert_array_equal(oracle.spmm(rp, ci, v, B), [[402.0]])


def test_transpose_twice_and_adjoint():
    rng = np.random.default_rng(13)
    M, K = 33, 21
    rp, ci, v, dense = random_csr(rng, M, K, 0.25)
    colptr, rowind, tv, perm = oracle.csr_transpose(rp, ci, v, K)
    # the transposed CSR densifies to dense.T, and every column lists rows in order
    dT = np.zeros((K, M))
    for c in range(K):
        rows = rowind[colptr[c]:colptr[c + 1]]
        assert np.all(np.diff(rows) > 0)
        dT[c, rows] = tv[colptr[c]:colptr[c + 1]]
    np.testing.assert_array_equal(dT, dense.T)
    np.testing.assert_array_equal(tv, v[perm])
    rp2, ci2, v2, _ = oracle.csr_transpose(colptr, rowind, tv, M)
    np.testing.assert_array_equal(rp2, rp)
    np.testing.assert_array_equal(ci2, ci)
    np.testing.assert_array_equal(v2, v)
    x = rng.standard_normal((M, 1))
    y = rng.standard_normal((K, 1))
    lhs = float((oracle.spmm(colptr, rowind, tv, x) * y).sum())   # <A^T x, y>
    rhs = float((x * oracle.spmm(rp, ci, v, y)).sum())            # <x, A y>
    assert lhs == pytest.approx(rhs, rel=1e-12, abs=1e-12)


def test_sddmm_is_sampled_dense_product():
    rng = np.random.default_rng(17)
    M, K, N = 19, 23, 7
    rp, ci, v, dense = random_csr(rng, M, K, 0.3)
    dC = rng.standard_normal((M, N))
    B = rng.standard_normal((K, N))
    full = dC @ B.T
    out = oracle.sddmm(rp, ci, dC, B)
    rows = np.repeat(np.arange(M), np.diff(rp))
    np.testing.assert_allclose(out, full[rows, ci], rtol=1e-12, atol=1e-12)


def test_backward_push_matches_transpose_and_dense():
    rng = np.random.default_rng(19)
    M, K, N = 27, 31, 5
    rp, ci, v, dense = random_csr(rng, M, K, 0.2)
    dC = rng.standard_normal((M, N))
    dB = oracle.spmm_t_push(rp, ci, v, dC, K)
    np.testing.assert_allclose(dB, dense.T @ dC, rtol=1e-12, atol=1e-12)
    colptr, rowind, tv, _ = oracle.csr_transpose(rp, ci, v, K)
    np.testing.assert_allclose(dB, oracle.spmm(colptr, rowind, tv, dC), rtol=1e-12, atol=1e-12)


def test_finite_difference_gradients():
    """L = sum(dC * (A B)).  Central differences (h = 1e-3) in FP64 on the oracle
    forward match dB = A^T dC and dvals = SDDMM(dC, B^T)."""
    rng = np.random.default_rng(23)
    M, K, N = 16, 12, 6
    rp, ci, v, _ = random_csr(rng, M, K, 0.35)
    B = rng.standard_normal((K, N))
    dC = rng.standard_normal((M, N))

    def loss(vv, BB):
        return float((dC * oracle.spmm(rp, ci, vv, BB)).sum())

    h = 1e-3
    dB = oracle.spmm_t_push(rp, ci, v, dC, K)
    for (k, n) in [(0, 0), (3, 2), (K - 1, N - 1), (5, 4)]:
        Bp, Bm = B.copy(), B.copy()
        Bp[k, n] += h
        Bm[k, n] -= h
        assert (loss(v, Bp) - loss(v, Bm)) / (2 * h) == pytest.approx(dB[k, n], rel=1e-8, abs=1e-9)
    dv = oracle.sddmm(rp, ci, dC, B)
    for e in range(0, v.size, max(1, v.size // 6)):
        vp, vm = v.copy(), v.copy()
        vp[e] += h
        vm[e] -= h
        assert (loss(vp, B) - loss(vm, B)) / (2 * h) == pytest.approx(dv[e], rel=1e-8, abs=1e-9)


# ---------------- number formats ----------------

def test_e4m3_decode_table():
    codes = np.arange(256, dtype=np.uint8)
    mine = oracle.decode_e4m3(codes)
    ref = torch.from_numpy(codes.copy()).view(torch.float8_e4m3fn).to(torch.float64).numpy()
    np.testing.assert_array_equal(np.isnan(mine), np.isnan(ref))
    ok = ~np.isnan(ref)
    np.testing.assert_array_equal(mine[ok], ref[ok])
    # spot values from the OCP FP8 E4M3 definition
    assert mine[0x01] == 2.0 ** -9 and mine[0x07] == 7 * 2.0 ** -9 and mine[0x08] == 2.0 ** -6
    assert mine[0x38] == 1.0 and mine[0x7E] == 448.0 and mine[0xFE] == -448.0
    assert np.isnan(mine[0x7F]) and np.isnan(mine[0xFF])
    assert mine[0x80] == 0.0 and np.signbit(mine[0x80])


def test_e4m3_encode_rne_satfinite():
    rng = np.random.default_rng(29)
    x = np.concatenate([rng.uniform(-448, 448, 20000), rng.uniform(-1, 1, 20000),
                        rng.uniform(-0.02, 0.02, 20000),
                        oracle.decode_e4m3(np.arange(0, 0x7F, dtype=np.uint8))]).astype(np.float32)
    mine = oracle.encode_e4m3(x)
    ref = torch.from_numpy(x).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    np.testing.assert_array_equal(mine, ref)
    # ties go to the even code; out-of-range values saturate to +-448
    ties = np.array([1.0625, 1.1875, 2.0 ** -10, 3 * 2.0 ** -10, 464.0, 1e9, -1e9, np.inf],
                    np.float32)
    np.testing.assert_array_equal(oracle.encode_e4m3(ties),
                                  [0x38, 0x3A, 0x00, 0x02, 0x7E, 0x7E, 0xFE, 0x7E])


def test_bf16_codec_vs_torch():
    rng = np.random.default_rng(31)
    x = np.concatenate([rng.standard_normal(50000) * 10.0 ** rng.integers(-30, 30, 50000),
                        [0.0, -0.0, 1.0, 3.0e38, -3.39e38, 1e-40, 1.00390625, 1.01171875]]
                       ).astype(np.float32)
    mine = oracle.encode_bf16(x)
    ref = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    np.testing.assert_array_equal(mine, ref)
    codes = np.arange(65536, dtype=np.uint32).astype(np.uint16)
    dec = oracle.decode_bf16(codes)
    tref = torch.from_numpy(codes.view(np.int16)).view(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(np.isnan(dec), np.isnan(tref))
    ok = ~np.isnan(tref)
    np.testing.assert_array_equal(dec[ok], tref[ok])


def test_f16_codec_vs_numpy():
    codes = np.arange(65536, dtype=np.uint32).astype(np.uint16)
    dec = oracle.decode_f16(codes)
    ref = codes.view(np.float16).astype(np.float64)
    np.testing.assert_array_equal(np.isnan(dec), np.isnan(ref))
    ok = ~np.isnan(ref)
    np.testing.assert_array_equal(dec[ok], ref[ok])
    rng = np.random.default_rng(37)
    x = np.concatenate([rng.standard_normal(50000) * 2.0 ** rng.integers(-30, 18, 50000),
                        [65504.0, 65519.0, 65520.0, 2.0 ** -24, 2.0 ** -25, 3 * 2.0 ** -26]]
                       ).astype(np.float32)
    with np.errstate(over="ignore"):
        ref = x.astype(np.float16).view(np.uint16)
    np.testing.assert_array_equal(oracle.encode_f16(x), ref)


def test_quantize_rows_e4m3():
    rng = np.random.default_rng(41)
    X = rng.standard_normal((64, 40)).astype(np.float32)
    X[5] = 0.0
    q, s = oracle.quantize_rows_e4m3(X)
    amax = np.abs(X).max(axis=1)
    expect = (amax / np.float32(448.0)).astype(np.float32)
    expect[5] = 1.0
    np.testing.assert_array_equal(s, expect)
    deq = oracle.dequantize_rows(q, s, "e4m3")
    # relative error of a normal E4M3 value is at most 2^-4; subnormal step is 2^-9 * s
    err = np.abs(deq - X)
    bound = 2.0 ** -4 * np.abs(X) + 2.0 ** -10 * s[:, None]
    assert np.all(err <= bound)
    assert np.all(q[5] == 0)
    # the row maximum maps to +-448
    for r in range(64):
        if r == 5:
            continue
        j = int(np.argmax(np.abs(X[r])))
        assert q[r, j] & 0x7F == 0x7E


# ---------------------------------------------------------------- SpGEMM ----

def _rand_csr(rng, M, K, density, dup=False):
    rows, cols = [], []
    for i in range(M):
        cs = np.flatnonzero(rng.random(K) < density)
        if dup and cs.size:
            cs = np.sort(np.concatenate([cs, rng.choice(cs, 1)]))
        rows.append(np.full(cs.size, i))
        cols.append(cs)
    rp = np.zeros(M + 1, np.int64)
    rp[1:] = np.cumsum([c.size for c in cols])
    ci = np.concatenate(cols).astype(np.int32) if rp[-1] else np.zeros(0, np.int32)
    v = rng.standard_normal(ci.size)
    return rp.astype(np.int32), ci, v


def _dense(rp, ci, v, K):
    M = rp.size - 1
    D = np.zeros((M, K))
    S = np.zeros((M, K), bool)
    for i in range(M):
        for e in range(rp[i], rp[i + 1]):
            D[i, ci[e]] += v[e]
            S[i, ci[e]] = True
    return D, S


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_spgemm_equals_dense_product_on_small_matrices(seed):
    rng = np.random.default_rng(seed)
    M, K, N = 9, 7, 11
    a = _rand_csr(rng, M, K, 0.3, dup=seed % 2 == 1)
    b = _rand_csr(rng, K, N, 0.35)
    rp, ci, v = oracle.spgemm(*a, *b, K, N)
    Ad, As = _dense(*a, K)
    Bd, Bs = _dense(*b, N)
    # structure: where some stored A_ik meets some stored B_kj (boolean product)
    S = (As.astype(int) @ Bs.astype(int)) > 0
    Cd = np.zeros((M, N))
    Cs = np.zeros((M, N), bool)
    for i in range(M):
        cols = ci[rp[i]:rp[i + 1]]
        assert np.all(np.diff(cols) > 0)            # increasing, no duplicates
        Cd[i, cols] = v[rp[i]:rp[i + 1]]
        Cs[i, cols] = True
    assert np.array_equal(Cs, S)
    np.testing.assert_allclose(Cd, Ad @ Bd, rtol=1e-12, atol=1e-12)


def test_spgemm_identity_and_permutation_and_diagonal_are_exact():
    rng = np.random.default_rng(7)
    K, N = 8, 10
    b = _rand_csr(rng, K, N, 0.4)
    eye = (np.arange(K + 1, dtype=np.int32), np.arange(K, dtype=np.int32), np.ones(K))
    rp, ci, v = oracle.spgemm(*eye, *b, K, N)
    assert np.array_equal(rp, b[0]) and np.array_equal(ci, b[1]) and np.array_equal(v, b[2])
    perm = rng.permutation(K)
    P = (np.arange(K + 1, dtype=np.int32), perm.astype(np.int32), np.ones(K))
    rp, ci, v = oracle.spgemm(*P, *b, K, N)
    for i in range(K):
        k = perm[i]
        assert np.array_equal(ci[rp[i]:rp[i + 1]], b[1][b[0][k]:b[0][k + 1]])
        assert np.array_equal(v[rp[i]:rp[i + 1]], b[2][b[0][k]:b[0][k + 1]])
    d = rng.standard_normal(K)
    Dg = (np.arange(K + 1, dtype=np.int32), np.arange(K, dtype=np.int32), d)
    rp, ci, v = oracle.spgemm(*Dg, *b, K, N)
    for i in range(K):
        assert np.array_equal(v[rp[i]:rp[i + 1]], d[i] * b[2][b[0][i]:b[0][i + 1]])


def test_spgemm_keeps_explicit_zeros_and_empty_rows():
    # A = [[0 (stored), 0], [none]] times B = [[1, 2]]: row 0 gets both columns, valued 0
    a = (np.array([0, 1, 1], np.int32), np.array([0], np.int32), np.array([0.0]))
    b = (np.array([0, 2], np.int32), np.array([0, 1], np.int32), np.array([1.0, 2.0]))
    rp, ci, v = oracle.spgemm(*a, *b, 1, 2)
    assert rp.tolist() == [0, 2, 2] and ci.tolist() == [0, 1] and v.tolist() == [0.0, 0.0]
    empty = (np.zeros(4, np.int32), np.zeros(0, np.int32), np.zeros(0))
    rp, ci, v = oracle.spgemm(*empty, *b, 1, 2)
    assert rp.tolist() == [0, 0, 0, 0] and ci.size == 0


def test_spgemm_is_associative_with_the_spmm_oracle():
    # (A B) x == A (B x), the right side through the independent SpMM oracle
    rng = np.random.default_rng(11)
    M, K, N = 30, 25, 20
    a = _rand_csr(rng, M, K, 0.15)
    b = _rand_csr(rng, K, N, 0.2)
    x = rng.standard_normal((N, 3))
    rp, ci, v = oracle.spgemm(*a, *b, K, N)
    left = oracle.spmm(rp, ci, v, x)
    right = oracle.spmm(a[0], a[1], a[2], oracle.spmm(b[0], b[1], b[2], x))
    np.testing.assert_allclose(left, right, rtol=1e-10, atol=1e-10)
