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
