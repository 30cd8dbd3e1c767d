"""Seeded synthetic inputs shared by the CUDA path, the oracle and the benchmark.

This module draws random numbers only; it holds none of the neighbour-graph
arithmetic.  Every array is drawn in float64 from numpy's PCG64 generator and
cast once to float32, so the GPU path and the FP64 oracle read identical bytes.

The shapes stand in for the paper's PCA embeddings (cells x 50 principal
components) of the 1.3M-cell mouse-brain, 2.4M brain and 11M embryo datasets
(Benchmarking section), which are not available here:

* ``mixture``     -- Gaussian mixture, cluster means ~ N(0, 4 I), noise on PC t
                     ~ N(0, 1/t) (decaying PC variance, like a PCA embedding).
* ``batched``     -- many samples of log-uniform size sharing one mixture (the
                     same cell types), each shifted by its own offset
                     ~ N(0, 0.5 I) (a batch effect).
* ``anisotropic`` -- mixture whose components have random rotated covariances
                     Q diag(lambda) Q^T, lambda log-uniform in [0.05, 2].
* ``positions``   -- starting positions for UMAP layout epochs: uniform in
                     [-10, 10]^dim (a random initial layout) or Gaussian blobs
                     (a layout part-way through its epochs).
"""
from __future__ import annotations

import numpy as np

_CHUNK = 1 << 20


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def mixture(n: int, d: int = 50, n_comp: int = 20, seed: int = 0,
            mean_std: float = 2.0, offset: np.ndarray | None = None,
            means: np.ndarray | None = None) -> np.ndarray:
    """n x d float32 rows of a Gaussian mixture with uniform component weights.

    mean_c ~ N(0, mean_std^2 I) (or the given `means`); row = mean_c + eps,
    eps_t ~ N(0, 1/t) for t = 1..d.  Drawn chunk by chunk so 11M-row inputs
    stay within memory.
    """
    rng = _rng(seed)
    if means is None:
        means = rng.standard_normal((n_comp, d)) * mean_std
    n_comp = len(means)
    if offset is not None:
        means = means + offset[None, :]
    scale = 1.0 / np.sqrt(np.arange(1, d + 1, dtype=np.float64))
    out = np.empty((n, d), dtype=np.float32)
    for s in range(0, n, _CHUNK):
        e = min(n, s + _CHUNK)
        comp = rng.integers(0, n_comp, size=e - s)
        eps = rng.standard_normal((e - s, d)) * scale[None, :]
        out[s:e] = (means[comp] + eps).astype(np.float32)
    return out


def batched_sizes(n_samples: int = 64, lo: float = 2e3, hi: float = 2e5,
                  total: float = 3e6, seed: int = 0) -> np.ndarray:
    """Sample sizes, log-uniform in [lo, hi], rescaled so they sum to ~total."""
    rng = _rng(seed)
    sz = np.exp(rng.uniform(np.log(lo), np.log(hi), size=n_samples))
    sz = sz * (total / sz.sum())
    return np.maximum(1, np.round(sz)).astype(np.int64)


def batched(sizes, d: int = 50, n_comp: int = 30, seed: int = 0):
    """Concatenated samples and their offsets (category offsets, CSR-like).

    The samples share one ``n_comp``-component mixture (the same cell types,
    means ~ N(0, 4 I)); sample s is shifted by its own o_s ~ N(0, 0.5 I) (a
    batch effect) and draws its own rows.
    Returns (X float32 [sum(sizes), d], offsets int64 [len(sizes) + 1]).
    """
    rng = _rng(seed)
    means = rng.standard_normal((n_comp, d)) * 2.0
    sizes = np.asarray(sizes, dtype=np.int64)
    offsets = np.zeros(len(sizes) + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(sizes)
    X = np.empty((int(offsets[-1]), d), dtype=np.float32)
    for s, ns in enumerate(sizes):
        off = rng.standard_normal(d) * np.sqrt(0.5)
        sub_seed = int(rng.integers(0, 2**62))
        X[offsets[s]:offsets[s + 1]] = mixture(int(ns), d, seed=sub_seed, offset=off, means=means)
    return X, offsets


def anisotropic(n: int, d: int = 50, n_comp: int = 200, seed: int = 0,
                lam_lo: float = 0.05, lam_hi: float = 2.0, mean_std: float = 2.0) -> np.ndarray:
    """Mixture with per-component covariance Q diag(lambda) Q^T (Q Haar-random)."""
    rng = _rng(seed)
    means = rng.standard_normal((n_comp, d)) * mean_std
    factors = np.empty((n_comp, d, d))
    for c in range(n_comp):
        g = rng.standard_normal((d, d))
        q, r = np.linalg.qr(g)
        q = q * np.sign(np.diag(r))[None, :]          # Haar measure
        lam = np.exp(rng.uniform(np.log(lam_lo), np.log(lam_hi), size=d))
        factors[c] = q * np.sqrt(lam)[None, :]         # cov = F F^T
    out = np.empty((n, d), dtype=np.float32)
    for s in range(0, n, _CHUNK):
        e = min(n, s + _CHUNK)
        comp = rng.integers(0, n_comp, size=e - s)
        z = rng.standard_normal((e - s, d))
        x = np.empty((e - s, d))
        for c in np.unique(comp):                      # one matrix product per component
            m = comp == c
            x[m] = means[c] + z[m] @ factors[c].T
        out[s:e] = x.astype(np.float32)
    return out


def query_sample(n: int, m: int, seed: int = 0) -> np.ndarray:
    """m distinct query ids in [0, n), sorted (a seeded subsample)."""
    rng = _rng(seed + 7919)
    m = min(m, n)
    return np.sort(rng.choice(n, size=m, replace=False)).astype(np.int64)


def knn_lists(n: int, k: int, seed: int = 0, dup_frac: float = 0.0):
    """Random but well-formed kNN lists for connectivities-only tests.

    Row i holds itself at distance 0 in column 0, then k-1 distinct other
    rows at ascending positive distances.  With dup_frac > 0, that share of
    rows gets a run of equal distances (exact ties at rho).
    Returns (idx int32 [n, k], dist float32 [n, k]).
    """
    rng = _rng(seed)
    idx = np.empty((n, k), dtype=np.int32)
    dist = np.empty((n, k), dtype=np.float32)
    for i in range(n):
        others = rng.choice(n - 1, size=k - 1, replace=False)
        others = others + (others >= i)
        idx[i, 0] = i
        idx[i, 1:] = others
        gaps = rng.exponential(0.3, size=k - 1)
        dd = 0.5 + np.cumsum(gaps)
        if dup_frac > 0 and rng.uniform() < dup_frac:
            run = int(rng.integers(2, k))
            dd[:run] = dd[0]
        dist[i, 0] = 0.0
        dist[i, 1:] = dd.astype(np.float32)
    return idx, dist


def positions(n: int, dim: int = 2, seed: int = 0, clusters: int = 0, scale: float = 10.0) -> np.ndarray:
    """n x dim float32 positions: uniform in [-scale, scale]^dim, or with
    clusters > 0 blobs around centres uniform in that box (spread scale / 10)."""
    rng = _rng(seed + 104729)
    if clusters <= 0:
        return rng.uniform(-scale, scale, size=(n, dim)).astype(np.float32)
    centres = rng.uniform(-scale, scale, size=(clusters, dim))
    comp = rng.integers(0, clusters, size=n)
    return (centres[comp] + rng.standard_normal((n, dim)) * (scale / 10.0)).astype(np.float32)
