"""Pins for the oracle's UMAP layout epochs, against things other than itself.

The layout follows the UMAP method's embedding optimisation (McInnes, Healy &
Melville 2018): attraction along the gradient of log phi, repulsion along the
gradient of gamma log(1 - phi) with the squared distance offset by 0.001,
phi(d) = 1 / (1 + a d^(2b)).  The checks below tie the oracle to finite
differences of those functions, to a scalar recurrence of a two-vertex graph
written through |x|^(2b-1) instead of d2^(b-1) x, to exact rational arithmetic
for the sampling schedule, to published SplitMix64 outputs, and to invariants
(antisymmetric attraction preserves the centroid; translation invariance).
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle

A, B = 0.583, 1.334


def _sym_graph(n, m, rng, dyadic=False):
    """Random symmetric CSR graph with m undirected edges (no diagonal)."""
    pairs = set()
    while len(pairs) < m:
        i, j = rng.integers(0, n, 2)
        if i != j:
            pairs.add((min(i, j), max(i, j)))
    w = {}
    for p in pairs:
        w[p] = (rng.integers(1, 65) / 64.0) if dyadic else float(np.float32(rng.uniform(0.02, 1.0)))
    rows = [[] for _ in range(n)]
    for (i, j), v in w.items():
        rows[i].append((j, v))
        rows[j].append((i, v))
    indptr = [0]
    indices, data = [], []
    for r in rows:
        r.sort()
        indices += [c for c, _ in r]
        data += [v for _, v in r]
        indptr.append(len(indices))
    return np.array(indptr, np.int64), np.array(indices, np.int32), np.array(data, np.float32)


def _log_phi(y0, y1):
    d2 = float(np.sum((y0 - y1) ** 2))
    return -math.log1p(A * d2 ** B)


def _grad(f, y, h=1e-6):
    g = np.zeros_like(y)
    for t in range(len(y)):
        e = np.zeros_like(y)
        e[t] = h
        g[t] = (f(y + e) - f(y - e)) / (2 * h)
    return g


def test_splitmix64_published_vectors(golden_dir):
    with open(os.path.join(golden_dir, "splitmix64.txt")) as f:
        rows = [line.split() for line in f if line.strip() and not line.startswith("#")]
    assert rows
    for seed, i, value in rows:
        assert oracle.splitmix64(int(seed), int(i)) == int(value)


def test_negative_sampler_is_uniform_and_in_range():
    nv, draws = 50, 100000
    counts = np.zeros(nv)
    for e in range(draws // 5):
        for q in range(5):
            v = oracle.umap_negative(7, 3, draws // 5, e, 5, q, nv)
            assert 0 <= v < nv
            counts[v] += 1
    chi2 = float(np.sum((counts - draws / nv) ** 2 / (draws / nv)))
    # 49 degrees of freedom: chi2 above 100 has probability below 1e-5
    assert chi2 < 100.0
    assert all(oracle.umap_negative(1, 1, 10, e, 5, q, 1) == 0 for e in range(10) for q in range(5))
    # different epochs, entries and sample numbers draw from different counters
    a = [oracle.umap_negative(9, 1, 100, 3, 5, q, 2**31 - 1) for q in range(5)]
    b = [oracle.umap_negative(9, 2, 100, 3, 5, q, 2**31 - 1) for q in range(5)]
    c = [oracle.umap_negative(9, 1, 100, 4, 5, q, 2**31 - 1) for q in range(5)]
    assert len(set(a + b + c)) == 15


@pytest.mark.parametrize("y0,y1", [([0.3, -1.2], [2.1, 0.4]), ([0.0, 0.0], [0.2, -0.1]), ([5.0, 1.0], [-3.0, 2.0])])
def test_attraction_is_twice_the_gradient_of_log_phi(y0, y1):
    # one undirected edge stored as entries 0->1 and 1->0, both sampled in epoch 1
    indptr, indices, data = np.array([0, 1, 2]), np.array([1, 0]), np.array([0.7, 0.7], np.float32)
    Y = np.array([y0, y1], np.float32)
    lr = 0.01
    out, _, samples = oracle.umap_epochs(indptr, indices, data, Y, A, B, lr=lr, neg_rate=0, n_epochs=10,
                                         first=1, last=1)
    assert list(samples) == [1, 1]
    Yd = Y.astype(np.float64)
    g0 = _grad(lambda y: _log_phi(y, Yd[1]), Yd[0].copy())
    # vertex 0 moves as the head of 0->1 and as the tail of 1->0: 2 alpha grad
    np.testing.assert_allclose(out[0] - Yd[0], 2 * lr * g0, rtol=1e-6, atol=1e-12)
    np.testing.assert_allclose(out[1] - Yd[1], -2 * lr * g0, rtol=1e-6, atol=1e-12)


def test_repulsion_is_the_offset_gradient_of_log_one_minus_phi():
    indptr, indices, data = np.array([0, 1, 2]), np.array([1, 0]), np.array([1.0, 1.0], np.float32)
    Y = np.array([[0.4, 0.9], [2.5, -1.5]], np.float32)
    lr, gamma, r, seed, epoch = 0.02, 1.7, 6, 12345, 4
    out, _, _ = oracle.umap_epochs(indptr, indices, data, Y, A, B, gamma=gamma, lr=lr, neg_rate=r,
                                   n_epochs=10, first=epoch, last=epoch, seed=seed)
    alpha = lr * (1 - (epoch - 1) / 10)
    Yd = Y.astype(np.float64)
    d2 = float(np.sum((Yd[0] - Yd[1]) ** 2))
    for head, other, e in ((0, 1, 0), (1, 0, 1)):
        # negatives of entry e that land on the other vertex (landing on the head moves nothing)
        hits = sum(oracle.umap_negative(seed, epoch, 2, e, r, q, 2) == other for q in range(r))
        ga = _grad(lambda y: _log_phi(y, Yd[other]), Yd[head].copy())
        gr = _grad(lambda y: gamma * math.log(1.0 - math.exp(_log_phi(y, Yd[other]))), Yd[head].copy())
        expect = 2 * alpha * ga + hits * alpha * gr * d2 / (d2 + 0.001)
        np.testing.assert_allclose(out[head] - Yd[head], expect, rtol=1e-6, atol=1e-12)


def _pair_recurrence(x, lr, N, a, b, first=1, last=None):
    last = N if last is None else last
    for n in range(first, last + 1):
        alpha = lr * (1 - (n - 1) / N)
        ax = abs(x)
        pull = min(4.0, 2 * a * b * ax ** (2 * b - 1) / (1 + a * ax ** (2 * b))) if ax > 0 else 0.0
        x = x - 4 * alpha * math.copysign(pull, x)
    return x


@pytest.mark.parametrize("a,b,x0,lr", [(A, B, 6.0, 0.05), (1.58, 0.9, 3.0, 0.2), (10.0, 0.6, 0.01, 0.001)])
def test_two_vertex_separation_follows_scalar_recurrence(a, b, x0, lr):
    # 1-D, one undirected edge, no negatives: the midpoint stays, the separation
    # x follows x' = x - 4 alpha sgn(x) min(4, 2ab |x|^(2b-1) / (1 + a |x|^(2b)))
    indptr, indices, data = np.array([0, 1, 2]), np.array([1, 0]), np.array([0.5, 0.5], np.float32)
    y = np.array([[1.25], [1.25 + x0]], np.float32)
    x0 = float(y[1, 0]) - float(y[0, 0])
    N = 40
    out, _, samples = oracle.umap_epochs(indptr, indices, data, y, a, b, lr=lr, neg_rate=0, n_epochs=N)
    assert list(samples) == [N, N]
    assert abs((out[0, 0] + out[1, 0]) - float(y[0, 0] + y[1, 0])) < 1e-12
    np.testing.assert_allclose(out[1, 0] - out[0, 0], _pair_recurrence(x0, lr, N, a, b), rtol=1e-9, atol=1e-12)


def test_sampling_schedule_matches_exact_rationals():
    rng = np.random.default_rng(5)
    indptr, indices, data = _sym_graph(30, 60, rng, dyadic=True)
    N = 37
    assert data.max() == 1.0   # f = w exactly, so n f is exact in float32
    wmax = Fraction(float(data.max()))
    Y = rng.uniform(-5, 5, (30, 2)).astype(np.float32)
    total = np.zeros(len(data), np.int64)
    for n in range(1, N + 1):
        _, _, s = oracle.umap_epochs(indptr, indices, data, Y, A, B, neg_rate=0, n_epochs=N, first=n, last=n)
        for e, w in enumerate(data):
            f = Fraction(float(w)) / wmax
            assert s[e] == int(math.floor(n * f) > math.floor((n - 1) * f))
        total += s
    _, _, s_all = oracle.umap_epochs(indptr, indices, data, Y, A, B, neg_rate=0, n_epochs=N)
    expect = [math.floor(N * Fraction(float(w)) / wmax) for w in data]
    assert list(s_all) == expect == list(total)


def test_attraction_preserves_the_centroid():
    rng = np.random.default_rng(8)
    indptr, indices, data = _sym_graph(40, 150, rng)
    Y = rng.uniform(-10, 10, (40, 2)).astype(np.float32)
    out, _, _ = oracle.umap_epochs(indptr, indices, data, Y, A, B, lr=1.0, neg_rate=0, n_epochs=20)
    np.testing.assert_allclose(out.mean(0), Y.astype(np.float64).mean(0), atol=1e-11)
    assert np.abs(out - Y).max() > 0.1


def test_translation_invariance_with_negatives():
    rng = np.random.default_rng(9)
    indptr, indices, data = _sym_graph(50, 120, rng)
    # positions on a 2^-12 grid, so that adding the shift is exact in float32
    Y = (np.round(rng.uniform(-4, 4, (50, 3)) * 4096) / 4096).astype(np.float32)
    shift = np.array([8.0, -16.0, 2.0], np.float32)
    o1, _, _ = oracle.umap_epochs(indptr, indices, data, Y, A, B, n_epochs=10, seed=3)
    o2, _, _ = oracle.umap_epochs(indptr, indices, data, Y + shift, A, B, n_epochs=10, seed=3)
    np.testing.assert_allclose(o2 - shift, o1, atol=1e-9)


def test_moves_are_clipped_per_coordinate():
    # offsets of 0.02: the repulsion coefficient (about 1500) times the offset
    # exceeds 4, while the attraction moves about 0.003 per sample
    indptr, indices, data = np.array([0, 1, 2]), np.array([1, 0]), np.array([1.0, 1.0], np.float32)
    Y = np.array([[0.0, 0.0], [0.02, 0.02]], np.float32)
    out, absmove, _ = oracle.umap_epochs(indptr, indices, data, Y, A, B, lr=1.0, neg_rate=8, n_epochs=100,
                                         first=1, last=1, seed=1)
    hits = [sum(oracle.umap_negative(1, 1, 2, e, 8, q, 2) == 1 - e for q in range(8)) for e in (0, 1)]
    assert min(hits) > 0
    Yd = Y.astype(np.float64)
    # each repulsive sample moves the head by exactly -4 / +4 per coordinate; attraction is tiny
    for v in (0, 1):
        sgn = -1.0 if v == 0 else 1.0
        assert np.all(np.abs(out[v] - Yd[v] - sgn * 4.0 * hits[v]) < 1e-2)


def test_masked_epoch_matches_full_epoch():
    rng = np.random.default_rng(10)
    indptr, indices, data = _sym_graph(60, 200, rng)
    Y = rng.uniform(-6, 6, (60, 2)).astype(np.float32)
    full, am_full, _ = oracle.umap_epochs(indptr, indices, data, Y, A, B, n_epochs=50, first=7, last=7, seed=4)
    mask = np.zeros(60, bool)
    mask[rng.choice(60, 17, replace=False)] = True
    part, am_part, _ = oracle.umap_epochs(indptr, indices, data, Y, A, B, n_epochs=50, first=7, last=7, seed=4,
                                          mask=mask)
    np.testing.assert_array_equal(part[mask], full[mask])
    np.testing.assert_array_equal(am_part[mask], am_full[mask])
    np.testing.assert_array_equal(part[~mask], Y[~mask].astype(np.float64))


def test_layout_separates_two_cliques():
    # two 15-vertex cliques joined by one weak edge, random initial positions
    n, h = 30, 15
    rows = [[] for _ in range(n)]
    for c in (0, h):
        for i in range(c, c + h):
            for j in range(c, c + h):
                if i != j:
                    rows[i].append((j, 1.0))
    rows[0].append((h, 0.05))
    rows[h].append((0, 0.05))
    indptr, indices, data = [0], [], []
    for r in rows:
        r.sort()
        indices += [c for c, _ in r]
        data += [v for _, v in r]
        indptr.append(len(indices))
    rng = np.random.default_rng(2)
    Y = rng.uniform(-10, 10, (n, 2)).astype(np.float32)
    out, _, _ = oracle.umap_epochs(np.array(indptr), np.array(indices), np.array(data, np.float32), Y, A, B,
                                   n_epochs=200, seed=11)
    d = np.linalg.norm(out[:, None] - out[None], axis=2)
    intra = np.concatenate([d[:h, :h][np.triu_indices(h, 1)], d[h:, h:][np.triu_indices(h, 1)]])
    inter = d[:h, h:].ravel()
    assert intra.max() < inter.min()
    assert np.median(inter) > 3 * np.median(intra)


def test_negative_pairs_share_one_generator_output():
    # negatives 2h and 2h + 1 of an entry take the high and low halves of one
    # SplitMix64 output (the generator itself is pinned by published outputs)
    seed, epoch, nnz, e, r, n = 21, 3, 1000, 17, 5, 123457
    for q in range(r):
        u = oracle.splitmix64(seed, ((epoch - 1) * nnz + e) * 3 + q // 2 + 1)
        h = (u >> 32) if q % 2 == 0 else (u & 0xFFFFFFFF)
        assert oracle.umap_negative(seed, epoch, nnz, e, r, q, n) == (h * n) >> 32
