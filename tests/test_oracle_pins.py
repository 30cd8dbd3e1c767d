"""Pins for the FP64 oracle, against things other than itself.

Each check ties the oracle to an independent fact: a hand derivation
(tests/golden), exact integer brute force, a library routine (scipy's k-d tree,
scipy's cosine cdist, scipy.sparse arithmetic), a closed form of the
smooth-kNN equation, or an invariant the definitions imply.
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle
from paper_2603_02402_gb300 import synth

scipy_spatial = pytest.importorskip("scipy.spatial")
scipy_sparse = pytest.importorskip("scipy.sparse")


def _read_golden(path):
    rec = {"idx": [], "dist": [], "next": [], "w": [], "G": []}
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            if key == "points":
                rec["points"] = [float(v) for v in vals]
            elif key == "k":
                rec["k"] = int(vals[0])
            else:
                rec[key].append(vals)
    return rec


def _eval(expr, c):
    return float(eval(expr, {"__builtins__": {}}, {"c": c}))


# ----------------------------------------------------------------- kNN pins

def test_golden_line4(golden_dir):
    g = _read_golden(os.path.join(golden_dir, "line4_k3.txt"))
    X = np.array(g["points"], dtype=np.float32)[:, None]
    k = g["k"]
    idx, dist, nxt = oracle.knn(X, k)
    np.testing.assert_array_equal(idx, np.array(g["idx"], dtype=np.int32))
    np.testing.assert_array_equal(dist, np.array(g["dist"], dtype=np.float64))
    np.testing.assert_array_equal(nxt, np.array([v[0] for v in g["next"]], dtype=np.float64))

    c = math.log2(3.0) - 1.0
    s = oracle.connectivities(idx, dist)
    want_w = np.array([[_eval(e, c) for e in row] for row in g["w"]])
    np.testing.assert_allclose(s["weights"], want_w, atol=1e-5, rtol=0)
    # sigma solves 1 + exp(-(d - rho)/sigma) = log2 3 to the bisection tolerance
    for i in range(4):
        gap = dist[i, 2] - s["rho"][i]
        psum = 1.0 + math.exp(-gap / s["sigma"][i])
        assert abs(psum - math.log2(3.0)) < 1e-5
    want = {(int(r), int(cc)): _eval(e, c) for r, cc, e in g["G"]}
    got = {}
    for i in range(4):
        for p in range(s["indptr"][i], s["indptr"][i + 1]):
            got[(i, int(s["indices"][p]))] = s["data"][p]
    assert set(got) == set(want)
    for key in want:
        assert abs(got[key] - want[key]) < 2e-5, key


def _brute_int(P, k, rows=None):
    """Exact kNN on integer points: squared distances as Python ints."""
    n = len(P)
    rows = range(n) if rows is None else rows
    out = []
    for i in rows:
        order = sorted((sum((int(a) - int(b)) ** 2 for a, b in zip(P[i], P[j])), j) for j in range(n))
        out.append(order[:k + 1])
    return out


def test_ties_by_index_on_integer_grid():
    # a 3 x 4 integer grid plus a duplicate of one point: many exact ties
    pts = [(x, y) for x in range(3) for y in range(4)] + [(1, 1)]
    P = np.array(pts, dtype=np.float32)
    n = len(P)
    for k in (1, 2, 5, n - 1, n):
        idx, dist, nxt = oracle.knn(P, k)
        ref = _brute_int(pts, k)
        for i in range(n):
            assert [j for _, j in ref[i][:k]] == idx[i].tolist()
            assert [math.sqrt(d2) for d2, _ in ref[i][:k]] == dist[i].tolist()
            if k < n:
                assert nxt[i] == math.sqrt(ref[i][k][0])
            else:
                assert math.isinf(nxt[i])
    # the duplicate (index 12) of point 5 = (1, 1): point 5 lists itself first,
    # the duplicate lists point 5 first (same distance 0, smaller index)
    idx, dist, _ = oracle.knn(P, 2)
    assert idx[5].tolist() == [5, 12] and idx[12].tolist() == [5, 12]
    assert dist[12].tolist() == [0.0, 0.0]


def test_exhaustive_subsets_tiny():
    # every subset of 8 integer points (in 3-D) of size >= k, against brute force
    rng = np.random.Generator(np.random.PCG64(11))
    base = rng.integers(-3, 4, size=(8, 3))
    k = 3
    for m in range(k, 9):
        for sub in itertools.combinations(range(8), m):
            pts = [tuple(base[s]) for s in sub]
            idx, dist, _ = oracle.knn(np.array(pts, dtype=np.float32), k)
            ref = _brute_int(pts, k)
            for i in range(m):
                assert [j for _, j in ref[i][:k]] == idx[i].tolist()


def test_line_d1_by_sorting():
    # d = 1: the kNN of a point on a line is a sort of |x_i - x_j|
    rng = np.random.Generator(np.random.PCG64(3))
    x = rng.permutation(200).astype(np.float32) * 0.5
    idx, dist, _ = oracle.knn(x[:, None], 7)
    for i in range(len(x)):
        order = sorted(range(len(x)), key=lambda j: (abs(float(x[i]) - float(x[j])), j))[:7]
        assert idx[i].tolist() == order


@pytest.mark.parametrize("n,d,k", [(3000, 50, 15), (4000, 5, 30)])
def test_knn_matches_kdtree(n, d, k):
    X = synth.mixture(n, d, n_comp=20, seed=5)
    idx, dist, nxt = oracle.knn(X, k)
    tree = scipy_spatial.cKDTree(X.astype(np.float64))
    dd, ii = tree.query(X.astype(np.float64), k=k + 1)
    np.testing.assert_array_equal(idx, ii[:, :k])
    np.testing.assert_allclose(dist, dd[:, :k], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(nxt, dd[:, k], rtol=1e-12, atol=1e-12)
    assert (idx[:, 0] == np.arange(n)).all()   # each cell is its own 0-distance neighbour
    assert (dist[:, 0] == 0).all()


def test_knn_query_subset_equals_rows_of_full():
    X = synth.mixture(1500, 50, n_comp=10, seed=8)
    full_i, full_d, _ = oracle.knn(X, 10)
    q = synth.query_sample(1500, 100, seed=1)
    sub_i, sub_d, _ = oracle.knn(X, 10, queries=q)
    np.testing.assert_array_equal(sub_i, full_i[q])
    np.testing.assert_array_equal(sub_d, full_d[q])


def test_cosine_matches_scipy_cdist():
    X = synth.mixture(600, 50, n_comp=8, seed=2)
    k = 12
    idx, dist, _ = oracle.knn(X, k, metric=oracle.COSINE)
    D = scipy_spatial.distance.cdist(X.astype(np.float64), X.astype(np.float64), metric="cosine")
    for i in range(len(X)):
        order = np.lexsort((np.arange(len(X)), D[i]))[:k]
        # scipy and the oracle round 1 - cos differently by ~1e-16; compare sets
        # via distances and require identical order where gaps exceed 1e-12
        np.testing.assert_allclose(dist[i], D[i, order], rtol=0, atol=1e-12)
        gaps = np.diff(D[i, order])
        if (gaps > 1e-12).all():
            assert idx[i].tolist() == order.tolist()


def test_cosine_is_half_squared_euclidean_of_unit_rows():
    # 1 - cos(x, y) = ||x/|x| - y/|y|||^2 / 2: same ranking, related distances
    X = synth.mixture(800, 50, n_comp=8, seed=4).astype(np.float64)
    U = (X / np.linalg.norm(X, axis=1, keepdims=True)).astype(np.float32)
    ci, cd, _ = oracle.knn(X.astype(np.float32), 9, metric=oracle.COSINE)
    ei, ed, _ = oracle.knn(U, 9, metric=oracle.EUCLIDEAN)
    np.testing.assert_allclose(cd, ed ** 2 / 2, rtol=2e-6, atol=1e-7)
    assert (ci == ei).mean() > 0.99


def test_cosine_zero_rows_convention():
    X = np.array([[0, 0], [1, 0], [0, 0], [0, 2], [3, 3]], dtype=np.float32)
    idx, dist, _ = oracle.knn(X, 3, metric=oracle.COSINE)
    assert idx[0].tolist() == [0, 2, 1] and dist[0].tolist() == [0.0, 0.0, 1.0]
    assert idx[1, 0] == 1 and dist[1, 0] == 0.0
    assert 0 not in idx[4].tolist()[:2]


def test_knn_rejects_bad_args():
    X = np.zeros((4, 2), dtype=np.float32)
    with pytest.raises(ValueError):
        oracle.knn(X, 5)
    with pytest.raises(ValueError):
        oracle.knn(X, 0)


# ------------------------------------------------------- smooth-kNN pins

def test_sigma_closed_form_k15():
    # one neighbour at rho, the other 13 non-self ones at rho + delta:
    # 1 + 13 exp(-delta/sigma) = log2 15  =>  exp(-delta/sigma) = (log2 15 - 1)/13
    k, rho, delta = 15, 0.7, 0.25
    idx = np.arange(k, dtype=np.int32)[None, :]
    dist = np.array([[0.0, rho] + [rho + delta] * 13])
    s = oracle.smooth_knn(idx, dist)
    e = (math.log2(15) - 1) / 13
    sigma_star = delta / -math.log(e)
    assert s["rho"][0] == rho
    assert s["converged"][0] == 1 and s["floored"][0] == 0
    psum = 1 + 13 * math.exp(-delta / s["sigma"][0])
    assert abs(psum - math.log2(15)) < 1e-5
    assert abs(s["sigma"][0] - sigma_star) < 1e-4
    np.testing.assert_allclose(s["weights"][0, 2:], e, atol=1e-5 / 13 * 1.01)
    assert s["weights"][0, 0] == 0.0 and s["weights"][0, 1] == 1.0


def test_sigma_no_solution_hits_floor():
    # every non-self neighbour at rho: psum = k - 1 > log2 k for every sigma;
    # bisection keeps halving, never converges, and the 1e-3 * row-mean floor binds
    k = 10
    idx = np.arange(k, dtype=np.int32)[None, :]
    dist = np.array([[0.0] + [2.0] * (k - 1)])
    s = oracle.smooth_knn(idx, dist)
    assert s["converged"][0] == 0 and s["iters"][0] == 64
    assert s["floored"][0] == 1
    assert s["sigma"][0] == pytest.approx(1e-3 * dist.mean(), rel=1e-15)
    assert (s["weights"][0, 1:] == 1.0).all()


def test_rho_zero_uses_global_mean_floor():
    # row 0: all distances zero (duplicates) -> rho = 0, floor from global mean
    idx = np.array([[0, 1, 2], [1, 0, 2], [2, 1, 0]], dtype=np.int32)
    dist = np.array([[0.0, 0.0, 0.0], [0.0, 1.0, 3.0], [0.0, 2.0, 3.0]])
    s = oracle.smooth_knn(idx, dist)
    assert s["rho"][0] == 0.0
    assert s["sigma"][0] == pytest.approx(1e-3 * dist.mean(), rel=1e-15)
    assert s["weights"][0].tolist() == [0.0, 1.0, 1.0]


def test_invariants_on_random_mixture():
    X = synth.mixture(2000, 50, n_comp=20, seed=9)
    k = 15
    idx, dist, _ = oracle.knn(X, k)
    s = oracle.connectivities(idx, dist)
    rho, sig, w = s["rho"], s["sigma"], s["weights"]
    # rho = first non-zero distance
    for i in range(len(X)):
        nz = dist[i][dist[i] > 0]
        assert rho[i] == (nz[0] if len(nz) else 0.0)
    # sum_j exp(-max(0, d - rho)/sigma) = log2 k where converged and not floored
    ok = (s["converged"] == 1) & (s["floored"] == 0)
    assert ok.mean() > 0.99
    g = np.maximum(dist[:, 1:] - rho[:, None], 0.0)
    psum = np.exp(-g / sig[:, None]).sum(axis=1)
    assert np.abs(psum[ok] - math.log2(k)).max() < 1e-5
    # weights in [0, 1], self 0, the rho neighbour 1
    assert (w >= 0).all() and (w <= 1).all()
    assert (w[:, 0] == 0).all()
    assert (w[:, 1] == 1).all()
    assert (w[:, 1:] > 0).all()


def _dense_graph(indptr, indices, data, n):
    G = np.zeros((n, n))
    for i in range(n):
        G[i, indices[indptr[i]:indptr[i + 1]]] = data[indptr[i]:indptr[i + 1]]
    return G


def test_union_against_scipy_sparse_and_invariants():
    X = synth.mixture(700, 50, n_comp=7, seed=12)
    n, k = len(X), 15
    idx, dist, _ = oracle.knn(X, k)
    s = oracle.connectivities(idx, dist)
    ip, ind, dat = s["indptr"], s["indices"], s["data"]
    for i in range(n):   # ascending, unique columns, no diagonal, no zeros
        cols = ind[ip[i]:ip[i + 1]]
        assert (np.diff(cols) > 0).all() and i not in cols
    assert (dat != 0).all()
    rows = np.repeat(np.arange(n), k)
    A = scipy_sparse.csr_matrix((s["weights"].ravel(), (rows, idx.ravel())), shape=(n, n))
    Gs = (A + A.T - A.multiply(A.T)).toarray()
    np.fill_diagonal(Gs, 0.0)
    G = _dense_graph(ip, ind, dat, n)
    np.testing.assert_allclose(G, Gs, rtol=0, atol=1e-15)
    assert (G == G.T).all()                                   # symmetric
    Ad = A.toarray()
    a, b = Ad, Ad.T
    m = (a > 0) | (b > 0)
    np.fill_diagonal(m, False)
    assert (G[m] >= np.maximum(a, b)[m] - 1e-15).all()       # max(a, b) <= G
    assert (G[m] <= (a + b)[m] + 1e-15).all()                # G <= a + b
    one = ((a == 1) | (b == 1)) & m
    assert np.abs(G[one] - 1).max() <= 4.5e-16               # either is 1 -> 1 (to rounding)


def test_union_hub_row():
    # centre at the origin, 40 points on orthogonal axes: every axis point's
    # nearest other row is the centre (distance 5 < 5*sqrt(2)), so the
    # centre's row of G gets all 40 columns
    X = np.concatenate([np.zeros((1, 40)), 5 * np.eye(40)]).astype(np.float32)
    idx, dist, _ = oracle.knn(X, 3)
    assert (idx[1:, 1] == 0).all()
    s = oracle.connectivities(idx, dist)
    deg = np.diff(s["indptr"])
    assert deg[0] == 40
    assert (s["indices"][:40] == np.arange(1, 41)).all()


def test_knn_qd_matches_kdtree_and_self_join():
    X = synth.mixture(2500, 50, n_comp=10, seed=21)
    Q = synth.mixture(300, 50, n_comp=10, seed=22)
    idx, dist, nxt = oracle.knn_qd(Q, X, 9)
    tree = scipy_spatial.cKDTree(X.astype(np.float64))
    dd, ii = tree.query(Q.astype(np.float64), k=10)
    np.testing.assert_array_equal(idx, ii[:, :9])
    np.testing.assert_allclose(dist, dd[:, :9], rtol=1e-12)
    # querying a set against itself is the self-join
    si, sd, _ = oracle.knn(X, 9)
    qi, qd, _ = oracle.knn_qd(X, X, 9)
    np.testing.assert_array_equal(si, qi)
    np.testing.assert_array_equal(sd, qd)


def test_batched_oracle_by_brute_force():
    X = synth.mixture(120, 5, n_comp=3, seed=23)
    off = np.array([0, 30, 70, 120])
    wi, wd, xi, xd = oracle.batched_knn(X, off, 4, 2)
    D = np.sqrt(((X[:, None, :].astype(np.float64) - X[None, :, :]) ** 2).sum(-1))
    for q in range(len(X)):
        s = np.searchsorted(off, q, side="right") - 1
        cols = np.arange(off[s], off[s + 1])
        order = cols[np.lexsort((cols, D[q, cols]))][:4]
        assert wi[q].tolist() == order.tolist()
        exp = []
        for t in range(3):
            c = np.arange(off[t], off[t + 1])
            exp += c[np.lexsort((c, D[q, c]))][:2].tolist()
        exp = sorted(exp, key=lambda j: (D[q, j], j))
        assert xi[q].tolist() == exp
        np.testing.assert_allclose(xd[q], D[q, exp], rtol=1e-12)


def _mlp_case(seed=5, B=6, dims=(7, 9, 8, 11)):
    rng = np.random.Generator(np.random.PCG64(seed))
    D, H1, H2, P = dims
    X = rng.standard_normal((B, D)).astype(np.float32)
    T = rng.uniform(size=(B, P)).astype(np.float32)
    T /= T.sum(axis=1, keepdims=True)
    params = (rng.standard_normal(oracle.mlp_param_count(*dims)) * 0.4).astype(np.float32)
    return X, T, params, dims


def test_mlp_gradient_matches_central_differences():
    # the analytic FP64 backward against central differences of the FP64 loss
    X, T, params, dims = _mlp_case()
    loss, grad = oracle.mlp_loss_grad(X, T, params, dims)
    p64 = params.astype(np.float64)
    rng = np.random.Generator(np.random.PCG64(1))
    for i in rng.choice(params.size, size=60, replace=False):
        # perturb in float64 through a float32 parameter vector is too coarse:
        # evaluate the loss as a function of a scaled direction instead
        h = 1e-3
        e = np.zeros_like(p64)
        e[i] = h
        lp, _ = oracle.mlp_loss_grad(X, T, (p64 + e).astype(np.float32), dims, need_grad=False)
        lm, _ = oracle.mlp_loss_grad(X, T, (p64 - e).astype(np.float32), dims, need_grad=False)
        hp = float(np.float32(p64[i] + h)) - p64[i]
        hm = p64[i] - float(np.float32(p64[i] - h))
        fd = (lp - lm) / (hp + hm)
        assert abs(fd - grad[i]) <= 1e-4 * max(1.0, abs(grad[i])), (i, fd, grad[i])


def test_mlp_loss_closed_forms():
    # zero weights and biases: uniform softmax, loss = log P for any targets
    X, T, params, dims = _mlp_case(seed=6)
    zero = np.zeros_like(params)
    loss, grad = oracle.mlp_loss_grad(X, T, zero, dims)
    T64 = T.astype(np.float64)
    tsum = T64.sum(axis=1, keepdims=True)          # 1 up to float32 rounding of the targets
    assert abs(loss - np.log(dims[3]) * tsum.mean()) < 1e-12
    # gradient of b3 at zero weights: mean over the batch of (sum(t)/P - t)
    P = dims[3]
    gb3 = grad[-P:]
    np.testing.assert_allclose(gb3, (tsum / P - T64).mean(axis=0), atol=1e-12)


def test_bf16_rounding_rule():
    # round to nearest, ties to even, on the 16 upper bits of the float32
    X, T, params, dims = _mlp_case(seed=7)
    v = np.array([1.0, 1.00390625, 1.005859375, 1.0078125, 3.14159265], dtype=np.float32)
    # 1 + 2^-8 is exactly halfway between bf16 1.0 and 1.0078125: ties to even -> 1.0;
    # 1 + 1.5 * 2^-8 rounds up; 1.0078125 is representable
    expect = [1.0, 1.0, 1.0078125, 1.0078125, 3.140625]
    X1 = np.zeros((1, dims[0]), dtype=np.float32)
    got = []
    for x in v:
        # identity network: read back the rounded input through the bias-free first layer
        p = np.zeros_like(params)
        D, H1 = dims[0], dims[1]
        p[0] = 1.0                              # W1[0, 0] = 1
        X1[0, 0] = x
        # loss depends on z1 only through relu(z1) -> h1 -> W2 = 0 -> constant; use the gradient of W1[0,0]
        # with targets favouring class 0 and W3, W2 set so the chain is linear in h1[0]
        p2 = p.copy()
        off_W2 = H1 * D + H1
        p2[off_W2] = 1.0                        # W2[0, 0] = 1
        off_W3 = off_W2 + dims[2] * H1 + dims[2]
        p2[off_W3] = 1.0                        # W3[0, 0] = 1
        t = np.zeros((1, dims[3]), dtype=np.float32)
        t[0, 0] = 1.0
        _, g = oracle.mlp_loss_grad(X1, t, p2, dims, bf16=True)
        # dL/dW1[0,0] = dz1[0] * bf16(x); dL/db1[0] = dz1[0]
        got.append(g[0] / g[H1 * D])
    np.testing.assert_array_equal(np.array(got), np.array(expect))
