"""The load-imbalance simulator (host side): stage work against brute force on
small matrices, conservation of the total work, and the two imbalance figures
on cases whose answer is known."""
import numpy as np

from paper_2311_18141_gb300 import inputs, loadsim


def _rand(rng, R, C, p):
    rows = [np.flatnonzero(rng.random(C) < p) for _ in range(R)]
    rp = np.zeros(R + 1, np.int64)
    rp[1:] = np.cumsum([r.size for r in rows])
    return rp, np.concatenate(rows).astype(np.int64)


def test_spgemm_stage_work_matches_brute_force():
    rng = np.random.default_rng(3)
    M, K, N, p, s = 13, 11, 9, 3, 4
    arp, aci = _rand(rng, M, K, 0.3)
    brp, bci = _rand(rng, K, N, 0.3)
    w = loadsim.spgemm_stage_work(arp, aci, brp, bci, K, N, p, stages=s)
    blk = lambda n, parts: [min(x // -(-n // parts), parts - 1) for x in range(n)]
    rb, kb, cb = blk(M, p), blk(K, s), blk(N, p)
    ref = np.zeros((s, p, p))
    for i in range(M):
        for e in range(arp[i], arp[i + 1]):
            l = aci[e]
            for f in range(brp[l], brp[l + 1]):
                ref[kb[l], rb[i], cb[bci[f]]] += 1
    np.testing.assert_array_equal(w, ref)


def test_total_work_is_conserved():
    A = inputs.rmat_csr(10, 8, seed=4)
    rp, ci = A.rowptr.numpy(), A.colind.numpy()
    w = loadsim.spgemm_stage_work(rp, ci, rp, ci, A.K, A.K, 8)
    products = np.diff(rp.astype(np.int64))[ci].sum()
    assert w.sum() == products
    w2 = loadsim.spmm_stage_work(rp, ci, A.K, 100, 8, 3, 5)
    assert w2.sum() == A.nnz * 100


def test_balanced_and_skewed_cases():
    # a diagonal matrix on a grid dividing it evenly: every process, every stage equal
    n, p = 64, 4
    rp = np.arange(n + 1)
    ci = np.arange(n)
    w = loadsim.spmm_stage_work(rp, ci, n, 8, p, 2, p)
    im = loadsim.imbalance(w)
    assert abs(im.end_to_end - 1.0) < 1e-12
    # all work in row block 0 of stage 0: ratios equal the number of blocks
    rp = np.zeros(n + 1, np.int64)
    rp[1:] = 4
    rp[0] = 0
    rp[1:] = np.minimum(np.arange(1, n + 1), 1) * 4
    ci = np.arange(4)
    w = loadsim.spmm_stage_work(rp, ci, n, 8, p, 1, p)
    im = loadsim.imbalance(w)
    assert abs(im.end_to_end - p) < 1e-12        # one busy process of p
    assert abs(im.synchronised - p) < 1e-12


def test_relabel_is_a_symmetric_permutation():
    A = inputs.rmat_csr(9, 8, seed=5)
    rp, ci = A.rowptr.numpy(), A.colind.numpy()
    perm = np.random.default_rng(1).permutation(A.M)
    nrp, nci = loadsim.relabel(rp, ci, perm)
    assert nrp[-1] == rp[-1]
    inv = np.argsort(perm)
    for v in range(0, A.M, 37):
        old = set(ci[rp[v]:rp[v + 1]].tolist())
        new = set(inv[nci[nrp[perm[v]]:nrp[perm[v] + 1]]].tolist())
        assert old == new
    # the SpGEMM work is unchanged by relabelling
    lens, nlens = np.diff(rp.astype(np.int64)), np.diff(nrp)
    assert lens[ci].sum() == nlens[nci].sum()


def test_staggered_stages_follow_the_iteration_offset():
    """Section 3.3's offset: in stage k process (i, j) takes block (i + j + k)
    mod s.  Brute force on random stage work; the end-to-end figure is the same
    either way (each process still does every block once)."""
    rng = np.random.default_rng(7)
    s, p = 5, 5
    w = rng.integers(0, 100, (s, p, p)).astype(np.float64)
    st = loadsim.staggered(w)
    for k in range(s):
        for i in range(p):
            for j in range(p):
                assert st[k, i, j] == w[(i + j + k) % s, i, j]
    a, b = loadsim.imbalance(w), loadsim.imbalance(w, offset=True)
    assert abs(a.end_to_end - b.end_to_end) < 1e-12
    # all work in block 0: lockstep stage 0 keeps every process equally busy
    # (synchronised 1), while under the offset only the p processes with
    # i + j = -k (mod p) have work in stage k (max 1, mean 1/p: synchronised p)
    w = np.zeros((p, p, p))
    w[0] = 1.0
    assert abs(loadsim.imbalance(w).synchronised - 1.0) < 1e-12
    assert abs(loadsim.imbalance(w, offset=True).synchronised - p) < 1e-12


def test_figure1_setting_relabelled_rmat_offset_schedule():
    """Fig. 1's R-MAT (scale 17, edge factor 8, a = 0.6, b = c = d = 0.4/3),
    randomly relabelled, squared on a 16 x 16 grid: end-to-end imbalance near
    1.2 and, for the staggered schedule synchronised after every stage, about
    2 (the paper reports ~1.2 and ~2.3 for its own draw; draws here give
    1.14-1.25 and 1.8-2.2)."""
    A = inputs.rmat_csr(17, 8, 0.6, 0.4 / 3, 0.4 / 3, seed=1, device="cpu", values="pos")
    rp, ci = A.rowptr.numpy(), A.colind.numpy()
    r, c = loadsim.relabel(rp, ci, np.random.default_rng(1).permutation(A.M))
    w = loadsim.spgemm_stage_work(r, c, r, c, A.K, A.K, 16)
    lock, stag = loadsim.imbalance(w), loadsim.imbalance(w, offset=True)
    assert 1.05 < lock.end_to_end < 1.4
    assert lock.synchronised < 1.4          # lockstep stages stay balanced
    assert 1.6 < stag.synchronised < 2.6    # the offset schedule is what amplifies it
