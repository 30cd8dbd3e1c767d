"""Pins of the oracle's NN-descent (CPU).

The oracle follows the synchronous NN-descent stated above oracle_nndescent
(Dong, Charikar & Li 2011; the paper's CPU neighbour search is PyNNDescent,
Methods, "Benchmarking").  What pins it to something other than itself:

* the FP32 squared distance against the FP64 one within the rounding bound of
  d fused multiply-adds;
* k = n: the initial lists hold every point, so they are the exact kNN;
* on tiny inputs whose ids and sources map to distinct slots, whole iterations
  against the same steps written as set algebra over an FP64 distance matrix
  (a pull formulation: each point collects the join partners it shares a join
  list with, where the oracle pushes pairs from each join list);
* with colliding slots, every offered candidate that is missing from a list is
  beaten by the smaller key that held its slot (the slot keeps the minimum);
* convergence: recall against a k-d tree on a clustered set, and the early stop
  rule.
"""
import numpy as np
import pytest
from scipy.spatial import cKDTree

import oracle
from paper_2603_02402_gb300 import synth


def exact_sq(X):
    X = X.astype(np.float64)
    diff = X[:, None, :] - X[None, :, :]
    return (diff * diff).sum(-1)


def fib_slot(ids, bits):
    return ((np.asarray(ids, dtype=np.uint64) * np.uint64(0x9E3779B1)) & np.uint64(0xFFFFFFFF)) >> np.uint64(32 - bits)


def test_squared_distance_is_the_fp32_euclidean():
    rng = np.random.default_rng(0)
    for d in (1, 7, 50, 64):
        X = rng.normal(0, 3, (40, d)).astype(np.float32)
        idx, d2, _, run = oracle.nndescent(X, 8, iters=0, seed=5)
        assert run == 0
        ex = exact_sq(X)
        want = ex[np.arange(40)[:, None], idx]
        bound = (2 * d + 2) * 2.0 ** -24 * want + 1e-30
        assert (np.abs(d2.astype(np.float64) - want) <= bound).all(), d


def test_initial_lists_are_valid_and_sorted():
    X = synth.mixture(500, 12, n_comp=5, seed=1)
    k = 12
    idx, d2, _, _ = oracle.nndescent(X, k, iters=0, seed=3)
    for u in range(len(X)):
        assert u in idx[u]
        assert len(set(idx[u])) == k
        assert ((idx[u] >= 0) & (idx[u] < len(X))).all()
        keys = list(zip(d2[u].tolist(), idx[u].tolist()))
        assert keys == sorted(keys)
    # different seeds draw different initial neighbours
    idx2, _, _, _ = oracle.nndescent(X, k, iters=0, seed=4)
    assert (idx != idx2).any()


def test_k_equal_to_n_gives_the_exact_lists():
    rng = np.random.default_rng(2)
    X = rng.normal(0, 1, (9, 5)).astype(np.float32)
    idx, d2, _, _ = oracle.nndescent(X, 9, iters=0, seed=1)
    ex = exact_sq(X)
    for u in range(9):
        assert list(idx[u]) == list(np.lexsort((np.arange(9), ex[u])))


def pull_iterations(X, k, S, iters, seed, idx0, d2):
    """The iterations as set algebra (collision-free slots): returns the list
    ids after every iteration and the changes.  idx0 is the initial list (the
    oracle's, pinned above); flags start new except for the point itself."""
    n = len(X)
    B = [list(idx0[u]) for u in range(n)]
    new = [{v: (v != u) for v in B[u]} for u in range(n)]
    out, changes = [], []
    for _ in range(iters):
        newf, oldf = [], []
        for u in range(n):
            cand_new = [v for v in B[u] if new[u][v] and v != u]
            take = cand_new[:S]
            newf.append(set(take))
            oldf.append({v for v in B[u] if not new[u][v] and v != u})
            for v in take:
                new[u][v] = False
        rnew = [set() for _ in range(n)]
        rold = [set() for _ in range(n)]
        for u in range(n):
            for w in newf[u]:
                rnew[w].add(u)
            for w in oldf[u]:
                rold[w].add(u)
        jn = [newf[v] | rnew[v] for v in range(n)]
        jo = [(oldf[v] | rold[v]) - jn[v] for v in range(n)]
        offered = [set() for _ in range(n)]
        for a in range(n):
            for v in range(n):
                allv = jn[v] | jo[v]
                if a in jn[v]:
                    offered[a] |= allv - {a}
                elif a in jo[v]:
                    offered[a] |= jn[v] - {a}
        ch = 0
        for a in range(n):
            pool = set(B[a]) | offered[a]
            order = sorted(pool, key=lambda b: (d2[a, b], b))[:k]
            ch += sum(1 for b in order if b not in B[a])
            flags = {b: (new[a][b] if b in B[a] else True) for b in order}
            B[a], new[a] = order, flags
        out.append([list(r) for r in B])
        changes.append(ch)
    return out, changes


@pytest.mark.parametrize("n,d,k,S,seed", [(24, 4, 5, 5, 0), (32, 3, 6, 3, 1), (20, 6, 8, 2, 2), (32, 2, 4, 4, 3)])
def test_iterations_match_the_set_algebra(n, d, k, S, seed):
    rng = np.random.default_rng(10 + seed)
    X = rng.normal(0, 1, (n, d)).astype(np.float32)
    ex = exact_sq(X)
    # no two distances of a row within 1e-5 relative: FP32 and FP64 order alike
    for u in range(n):
        s = np.sort(ex[u])
        assert (np.diff(s) > 1e-5 * s[1:]).all()
    # with n <= 32 ids, 64 reverse and candidate slots never collide
    assert len(set(fib_slot(range(n), 6).tolist())) == n
    idx0, _, _, _ = oracle.nndescent(X, k, sample=S, rev_slots=64, cand_slots=64, iters=0, seed=seed)
    want, want_ch = pull_iterations(X, k, S, 4, seed, idx0, ex)
    for t in range(1, 5):
        idx, _, ch, run = oracle.nndescent(X, k, sample=S, rev_slots=64, cand_slots=64, iters=t, seed=seed)
        assert run == t
        assert [list(r) for r in idx] == want[t - 1], t
        assert list(ch) == want_ch[:t]


def test_a_slot_keeps_its_smallest_candidate():
    """Colliding slots (C = 16 for 300 ids): after one iteration from the
    initial lists, an offered candidate b missing from a's list either lies at
    or beyond the list's last key or shares its slot with a smaller offered
    key (whose winner is in the list or also beyond the last key)."""
    rng = np.random.default_rng(7)
    n, d, k = 300, 5, 8
    X = rng.normal(0, 1, (n, d)).astype(np.float32)
    idx0, d0, _, _ = oracle.nndescent(X, k, rev_slots=1024, cand_slots=16, iters=0, seed=9)
    idx1, d1, _, _ = oracle.nndescent(X, k, rev_slots=1024, cand_slots=16, iters=1, seed=9)
    ex = exact_sq(X)
    # iteration 0: every non-self entry is new and sampled (S = k); with 1024
    # reverse slots for 300 sources the reverse lists are complete
    assert len(set(fib_slot(range(n), 10).tolist())) == n
    jn = [set(idx0[v]) - {v} for v in range(n)]
    for u in range(n):
        for w in set(idx0[u]) - {u}:
            jn[w].add(u)
    offered = [set() for _ in range(n)]
    for v in range(n):
        for a in jn[v]:
            offered[a] |= jn[v] - {a}
    slot = fib_slot(np.arange(n), 4)
    checked = 0
    for a in range(n):
        last = (float(d1[a, -1]), int(idx1[a, -1]))
        lst = set(idx1[a].tolist())
        thr = (float(d0[a, -1]), int(idx0[a, -1]))
        for b in offered[a]:
            kb = (float(ex[a, b]), b)
            if b in lst or kb >= thr:
                continue
            # b was offered below the threshold and is not in the list
            rivals = [c for c in offered[a] if slot[c] == slot[b] and (float(ex[a, c]), c) < kb]
            assert rivals or kb > last, (a, b)
            checked += 1
    assert checked > 0


def test_converges_on_a_clustered_set():
    X = synth.mixture(3000, 10, n_comp=20, seed=4)
    k = 10
    idx, d2, ch, run = oracle.nndescent(X, k, iters=12, seed=2)
    assert run == 12
    _, want = cKDTree(X.astype(np.float64)).query(X.astype(np.float64), k)
    recall = np.mean([len(set(idx[u]) & set(want[u])) / k for u in range(len(X))])
    assert recall >= 0.97, recall
    assert ch[-1] * 20 < ch[0]
    # the lists only improve: the k-th distance never grows
    prev = None
    for t in (1, 3, 6):
        _, d2t, _, _ = oracle.nndescent(X, k, iters=t, seed=2)
        if prev is not None:
            assert (d2t[:, -1] <= prev).all()
        prev = d2t[:, -1]


def test_early_stop_rule():
    X = synth.mixture(2000, 8, n_comp=10, seed=5)
    k, delta = 8, 0.02
    _, _, ch, run = oracle.nndescent(X, k, iters=30, delta=delta, seed=1)
    assert 1 <= run < 30
    lim = delta * len(X) * k
    assert ch[run - 1] < lim
    assert (ch[:run - 1] >= lim).all()
    assert (ch[run:] == 0).all()


def test_duplicate_points():
    rng = np.random.default_rng(8)
    P = rng.normal(0, 1, (150, 6)).astype(np.float32)
    X = np.concatenate([P, P])
    idx, d2, _, _ = oracle.nndescent(X, 6, iters=10, seed=4)
    n = len(X)
    found = 0
    for u in range(n):
        assert len(set(idx[u])) == 6
        twin = u + 150 if u < 150 else u - 150
        found += twin in idx[u]
        # both zero-distance entries lead the list, in index order
        if twin in idx[u]:
            assert list(idx[u][:2]) == sorted([u, twin]) and d2[u][0] == 0 and d2[u][1] == 0
    assert found >= 0.95 * n


def test_bad_arguments():
    X = np.zeros((5, 3), dtype=np.float32)
    with pytest.raises(ValueError):
        oracle.nndescent(X, 6)             # k > n
    with pytest.raises(ValueError):
        oracle.nndescent(X, 3, rev_slots=12)   # not a power of two
    with pytest.raises(ValueError):
        oracle.nndescent(X, 3, sample=4)   # S > k


def test_caller_lists_start_the_iterations():
    """Initial lists from caller lists: the row itself, then the caller's valid
    distinct entries in order, then hashed draws; k exact lists are a fixed point."""
    rng = np.random.default_rng(13)
    n, d, k = 60, 4, 6
    X = rng.normal(0, 1, (n, d)).astype(np.float32)
    ex = exact_sq(X)
    exact = np.array([np.lexsort((np.arange(n), ex[u]))[:k] for u in range(n)], dtype=np.int32)
    idx0, _, _, _ = oracle.nndescent(X, k, iters=0, init=exact)
    assert (idx0 == exact).all()
    idx5, _, ch, _ = oracle.nndescent(X, k, iters=5, init=exact)
    assert (idx5 == exact).all() and (ch == 0).all()
    # invalid, repeated and self entries are skipped; the rest keeps its order
    init = np.full((n, k), -1, dtype=np.int32)
    init[:, 0] = (np.arange(n) + 7) % n
    init[:, 1] = (np.arange(n) + 7) % n
    init[:, 2] = np.arange(n)
    init[:, 3] = n + 5
    init[:, 4] = (np.arange(n) + 3) % n
    idx0, _, _, _ = oracle.nndescent(X, k, iters=0, init=init, seed=2)
    plain, _, _, _ = oracle.nndescent(X, k, iters=0, seed=2)
    for u in range(n):
        s = set(idx0[u].tolist())
        assert {u, (u + 7) % n, (u + 3) % n} <= s and len(s) == k
        # the remaining entries are the hashed draws of the plain initial list
        assert s - {(u + 7) % n, (u + 3) % n} <= set(plain[u].tolist())
