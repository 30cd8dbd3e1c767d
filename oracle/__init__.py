"""FP64 CPU oracle for the neighbourhood graph (TEST INFRASTRUCTURE ONLY).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  It shares no code with the CUDA library: the
arithmetic lives in ``oracle.c`` (plain C, double precision, OpenMP) and this
module only marshals numpy arrays through ctypes.

Functions and the definitions they follow (paper, Methods: "Custom GPU
kernels" for the distances, "Implementation" for following scanpy, whose
neighbours step uses the UMAP smooth-kNN / fuzzy-union construction):

* ``knn``          -- brute-force exact kNN, ties broken by ascending index.
* ``knn_qd``       -- the same for external queries against a row set.
* ``batched_knn``  -- per-sample kNN and k_cross nearest from every sample.
* ``smooth_knn``   -- rho, sigma (64-step bisection to log2 k) and weights.
* ``fuzzy_union``  -- G = A + A^T - A o A^T as CSR with sorted columns.
* ``connectivities`` -- smooth_knn followed by fuzzy_union.
* ``mlp_loss_grad`` -- the partitioner MLP's soft cross-entropy and gradients.
* ``umap_epochs``  -- epochs of the UMAP layout SGD on a CSR graph (Methods,
  "Dimensionality reduction and graph analysis": UMAP on the graph).
* ``splitmix64`` / ``umap_negative`` -- the counter-based negative sampler.
* ``edistance_sums`` / ``edistance`` -- group-pair sums of Euclidean distances
  and the energy distance (Methods, "Perturbation distance computation").
* ``leiden``       -- Leiden communities on a CSR graph (synchronous rounds,
  fixed-point weights; Methods, "Dimensionality reduction and graph analysis").
* ``nndescent``    -- approximate kNN by synchronous NN-descent with
  deterministic sampling (the paper's CPU neighbour search is PyNNDescent,
  Methods, "Benchmarking"); list decisions on FP32 squared distances.

Parity is pinned by tests/test_oracle_pins.py (brute force on tiny inputs,
closed forms, a library kNN, invariants).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.c")
_lock = threading.Lock()
_lib = None

EUCLIDEAN, COSINE = 0, 1


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_lib/liboracle.so (gcc, OpenMP)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
               "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            i64, i32, dbl = ctypes.c_int64, ctypes.c_int, ctypes.c_double
            vp = ctypes.c_void_p
            lib.oracle_knn.argtypes = [vp, i64, i32, vp, i64, i32, i32, vp, vp, vp]
            lib.oracle_knn.restype = i32
            lib.oracle_knn_qd.argtypes = [vp, i64, vp, i64, i32, i32, i32, vp, vp, vp]
            lib.oracle_knn_qd.restype = i32
            lib.oracle_smooth_knn.argtypes = [vp, vp, i64, i32, vp, vp, vp, vp, vp, vp, vp]
            lib.oracle_smooth_knn.restype = i32
            lib.oracle_fuzzy_union.argtypes = [vp, vp, i64, i32, vp, vp, vp, i64]
            lib.oracle_fuzzy_union.restype = i32
            lib.oracle_mlp_loss_grad.argtypes = [vp, vp, i64, i32, i32, i32, i32, vp, i32, vp, vp]
            lib.oracle_mlp_loss_grad.restype = i32
            u64 = ctypes.c_uint64
            lib.oracle_splitmix64.argtypes = [u64, u64]
            lib.oracle_splitmix64.restype = u64
            lib.oracle_umap_negative.argtypes = [u64, i32, i64, i64, i32, i32, i64]
            lib.oracle_umap_negative.restype = i64
            lib.oracle_umap_epochs.argtypes = [vp, vp, vp, i64, i32, vp, dbl, dbl, dbl, dbl, i32, i32,
                                               i32, i32, u64, vp, vp, vp]
            lib.oracle_umap_epochs.restype = i32
            lib.oracle_edistance_sums.argtypes = [vp, i64, i32, vp, vp, i32, vp, i64, vp]
            lib.oracle_edistance_sums.restype = i32
            lib.oracle_edistance_assemble.argtypes = [vp, i32, vp, vp, vp]
            lib.oracle_edistance_assemble.restype = i32
            lib.oracle_nndescent.argtypes = [vp, i64, i32, i32, i32, i32, i32, i32, dbl, u64, vp, vp, vp, vp, vp, vp]
            lib.oracle_nndescent.restype = i32
            lib.oracle_leiden.argtypes = [vp, vp, vp, i64, dbl, i32, i32, i32, vp, vp, vp, vp, vp]
            lib.oracle_leiden.restype = i32
            lib.oracle_num_threads.argtypes = []
            lib.oracle_num_threads.restype = i32
            _ = dbl
            _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def knn(X: np.ndarray, k: int, metric: int = EUCLIDEAN, queries=None):
    """Exact kNN of `queries` (row ids, default all rows) against all rows.

    Returns (idx int32 [nq, k], dist float64 [nq, k], next float64 [nq]) where
    ``next`` is the (k+1)-th distance, for judging ties at the boundary.
    Euclidean distances are metric (square-rooted); cosine is 1 - cos.
    """
    X = np.ascontiguousarray(X, dtype=np.float32)
    n, d = X.shape
    q = None if queries is None else np.ascontiguousarray(queries, dtype=np.int64)
    nq = n if q is None else len(q)
    idx = np.empty((nq, k), dtype=np.int32)
    dist = np.empty((nq, k), dtype=np.float64)
    nxt = np.empty(nq, dtype=np.float64)
    rc = _load().oracle_knn(_ptr(X), n, d, _ptr(q), nq, k, metric, _ptr(idx), _ptr(dist), _ptr(nxt))
    if rc != 0:
        raise ValueError(f"oracle_knn failed with status {rc}")
    return idx, dist, nxt


def knn_qd(Q: np.ndarray, D: np.ndarray, k: int, metric: int = EUCLIDEAN):
    """Exact kNN of the rows of Q among the rows of D (ids index D)."""
    Q = np.ascontiguousarray(Q, dtype=np.float32)
    D = np.ascontiguousarray(D, dtype=np.float32)
    nq, d = Q.shape
    idx = np.empty((nq, k), dtype=np.int32)
    dist = np.empty((nq, k), dtype=np.float64)
    nxt = np.empty(nq, dtype=np.float64)
    rc = _load().oracle_knn_qd(_ptr(Q), nq, _ptr(D), len(D), d, k, metric, _ptr(idx), _ptr(dist), _ptr(nxt))
    if rc != 0:
        raise ValueError(f"oracle_knn_qd failed with status {rc}")
    return idx, dist, nxt


def batched_knn(X: np.ndarray, offsets, k_within: int, k_cross: int, metric: int = EUCLIDEAN):
    """Per-sample kNN and cross-sample lists, by definition.

    within: rows of sample s against rows of sample s (global ids);
    cross: for every sample t the k_cross nearest rows of t, the row's
    n_samples * k_cross entries ordered by (distance, id).
    """
    X = np.ascontiguousarray(X, dtype=np.float32)
    off = np.asarray(offsets, dtype=np.int64)
    S, n = len(off) - 1, len(X)
    wi = np.empty((n, k_within), dtype=np.int32)
    wd = np.empty((n, k_within))
    xi = np.empty((n, S * k_cross), dtype=np.int64)
    xd = np.empty((n, S * k_cross))
    for s in range(S):
        a, b = off[s], off[s + 1]
        i, d_, _ = knn_qd(X[a:b], X[a:b], k_within, metric)
        wi[a:b], wd[a:b] = i + a, d_
    for t in range(S):
        a, b = off[t], off[t + 1]
        i, d_, _ = knn_qd(X, X[a:b], k_cross, metric)
        xi[:, t * k_cross:(t + 1) * k_cross] = i + a
        xd[:, t * k_cross:(t + 1) * k_cross] = d_
    order = np.lexsort((xi, xd), axis=1)
    xi = np.take_along_axis(xi, order, axis=1).astype(np.int32)
    xd = np.take_along_axis(xd, order, axis=1)
    return wi, wd, xi, xd


def smooth_knn(idx: np.ndarray, dist: np.ndarray):
    """Per-row rho, sigma, directed weights and bisection diagnostics."""
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    dist = np.ascontiguousarray(dist, dtype=np.float64)
    n, k = idx.shape
    out = {
        "rho": np.empty(n), "sigma": np.empty(n), "weights": np.empty((n, k)),
        "iters": np.empty(n, dtype=np.int32), "stop_margin": np.empty(n),
        "floored": np.empty(n, dtype=np.int32), "converged": np.empty(n, dtype=np.int32),
    }
    rc = _load().oracle_smooth_knn(_ptr(idx), _ptr(dist), n, k, _ptr(out["rho"]), _ptr(out["sigma"]),
                                   _ptr(out["weights"]), _ptr(out["iters"]), _ptr(out["stop_margin"]),
                                   _ptr(out["floored"]), _ptr(out["converged"]))
    if rc != 0:
        raise ValueError(f"oracle_smooth_knn failed with status {rc}")
    return out


def fuzzy_union(idx: np.ndarray, weights: np.ndarray):
    """CSR (indptr int64, indices int32, data float64) of A + A^T - A o A^T."""
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    weights = np.ascontiguousarray(weights, dtype=np.float64)
    n, k = idx.shape
    cap = 2 * n * k
    indptr = np.empty(n + 1, dtype=np.int64)
    indices = np.empty(cap, dtype=np.int32)
    data = np.empty(cap, dtype=np.float64)
    rc = _load().oracle_fuzzy_union(_ptr(idx), _ptr(weights), n, k, _ptr(indptr), _ptr(indices), _ptr(data), cap)
    if rc != 0:
        raise ValueError(f"oracle_fuzzy_union failed with status {rc}")
    nnz = int(indptr[-1])
    return indptr, indices[:nnz].copy(), data[:nnz].copy()


def connectivities(idx: np.ndarray, dist: np.ndarray):
    """smooth_knn then fuzzy_union; returns the smooth_knn dict plus the CSR."""
    s = smooth_knn(idx, dist)
    indptr, indices, data = fuzzy_union(idx, s["weights"])
    s.update(indptr=indptr, indices=indices, data=data)
    return s


def mlp_param_count(D, H1, H2, P):
    return H1 * D + H1 + H2 * H1 + H2 + P * H2 + P


def mlp_loss_grad(X, T, params, dims, bf16=False, need_grad=True):
    """Loss and gradient (double) of the MLP relu(W1 x+b1) -> relu(W2 .+b2) ->
    W3 .+b3 with soft-target cross-entropy, params flat [W1, b1, W2, b2, W3, b3]."""
    D, H1, H2, P = dims
    X = np.ascontiguousarray(X, dtype=np.float32)
    T = np.ascontiguousarray(T, dtype=np.float32)
    params = np.ascontiguousarray(params, dtype=np.float32)
    assert params.size == mlp_param_count(D, H1, H2, P)
    loss = ctypes.c_double(0)
    grad = np.empty(params.size, dtype=np.float64) if need_grad else None
    rc = _load().oracle_mlp_loss_grad(_ptr(X), _ptr(T), len(X), D, H1, H2, P, _ptr(params), int(bf16),
                                      ctypes.byref(loss), _ptr(grad))
    if rc != 0:
        raise ValueError(f"oracle_mlp_loss_grad failed with status {rc}")
    return loss.value, grad


def splitmix64(seed: int, i: int) -> int:
    """Output number i (i >= 1) of SplitMix64 started from `seed`."""
    return int(_load().oracle_splitmix64(seed & (2**64 - 1), i & (2**64 - 1)))


def umap_negative(seed: int, epoch: int, nnz: int, entry: int, neg_rate: int, q: int, n: int) -> int:
    """Vertex of negative sample q of graph entry `entry` in epoch `epoch` (1-based)."""
    return int(_load().oracle_umap_negative(seed & (2**64 - 1), epoch, nnz, entry, neg_rate, q, n))


def umap_epochs(indptr, indices, data, Y, a, b, gamma=1.0, lr=1.0, neg_rate=5, n_epochs=200,
                first=1, last=None, seed=0, mask=None):
    """Epochs first..last (1-based, inclusive) of the N-epoch UMAP layout.

    Y is the float embedding the epochs start from ([n, dim]); returns
    (Y double [n, dim], absmove double [n], samples int64 [nnz]): absmove is the
    sum of |move| over the coordinates of every move applied to a vertex in the
    last epoch run; samples counts the epochs in which each entry was sampled.
    With `mask` (bool [n]) a single epoch moves only the masked vertices.
    """
    indptr = np.ascontiguousarray(indptr, dtype=np.int64)
    indices = np.ascontiguousarray(indices, dtype=np.int32)
    data = np.ascontiguousarray(data, dtype=np.float32)
    Yd = np.ascontiguousarray(np.asarray(Y, dtype=np.float32), dtype=np.float64).copy()
    n, dim = Yd.shape
    last = n_epochs if last is None else last
    m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    absmove = np.zeros(n)
    samples = np.zeros(max(1, int(indptr[-1])), dtype=np.int64)
    rc = _load().oracle_umap_epochs(_ptr(indptr), _ptr(indices), _ptr(data), n, dim, _ptr(Yd), float(a), float(b),
                                    float(gamma), float(lr), neg_rate, n_epochs, first, last,
                                    seed & (2**64 - 1), _ptr(m), _ptr(absmove), _ptr(samples))
    if rc != 0:
        raise ValueError(f"oracle_umap_epochs failed with status {rc}")
    return Yd, absmove, samples[:int(indptr[-1])]


def edistance_sums(X, offsets, cell_index=None, pairs=None):
    """Sums of Euclidean distances per group pair, float64 [G, G]: entry (a, b),
    a <= b, of every requested pair (pairs [P, 2] with a <= b; None: all); the
    rest NaN.  Pairs a != b sum over all cells of a and of b; a == b over the
    pairs i < j of positions inside the group."""
    X = np.ascontiguousarray(X, dtype=np.float32)
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    G = len(off) - 1
    ci = None if cell_index is None else np.ascontiguousarray(cell_index, dtype=np.int32)
    pr = None if pairs is None else np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)
    sums = np.full((G, G), np.nan)
    rc = _load().oracle_edistance_sums(_ptr(X), len(X), X.shape[1], _ptr(ci), _ptr(off), G, _ptr(pr),
                                       0 if pr is None else len(pr), _ptr(sums))
    if rc != 0:
        raise ValueError(f"oracle_edistance_sums failed with status {rc}")
    return sums


def edistance(X, offsets, cell_index=None):
    """All pairs: (sums, mean distances, E), float64 [G, G] each."""
    sums = edistance_sums(X, offsets, cell_index)
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    G = len(off) - 1
    mean = np.empty((G, G))
    E = np.empty((G, G))
    rc = _load().oracle_edistance_assemble(_ptr(off), G, _ptr(np.ascontiguousarray(sums)), _ptr(mean), _ptr(E))
    if rc != 0:
        raise ValueError(f"oracle_edistance_assemble failed with status {rc}")
    return sums, mean, E


def nndescent(X, k, sample=None, rev_slots=32, cand_slots=64, iters=10, delta=0.0, seed=0, init=None,
              with_pairs=False):
    """Synchronous NN-descent (definition above oracle_nndescent in oracle.c).

    init: caller lists int32 [n, k] the initial lists start from (or None).
    Returns (idx int32 [n, k], d2 float32 [n, k] FP32 squared distances in list
    order, changes int64 [iters], iterations run), and pairs joined per
    iteration (int64 [iters]) last with_pairs."""
    X = np.ascontiguousarray(X, dtype=np.float32)
    n, d = X.shape
    S = k if sample is None else sample
    idx = np.empty((n, k), dtype=np.int32)
    d2 = np.empty((n, k), dtype=np.float32)
    ch = np.zeros(max(1, iters), dtype=np.int64)
    pr = np.zeros(max(1, iters), dtype=np.int64)
    run = ctypes.c_int(0)
    ini = None if init is None else np.ascontiguousarray(init, dtype=np.int32).reshape(n, k)
    rc = _load().oracle_nndescent(_ptr(X), n, d, k, S, rev_slots, cand_slots, iters, float(delta),
                                  seed & (2**64 - 1), _ptr(ini), _ptr(idx), _ptr(d2), _ptr(ch), _ptr(pr),
                                  ctypes.byref(run))
    if rc != 0:
        raise ValueError(f"oracle_nndescent failed with status {rc}")
    if with_pairs:
        return idx, d2, ch[:iters], run.value, pr[:iters]
    return idx, d2, ch[:iters], run.value


def leiden(indptr, indices, data, resolution=1.0, n_iter=2, max_levels=32, max_rounds=8, init=None):
    """Leiden communities (definition above oracle_leiden in oracle.c).

    Returns (membership int32 [n] numbered by first appearance, number of
    communities, modularity on the fixed-point weights, levels of the last run)."""
    indptr = np.ascontiguousarray(indptr, dtype=np.int64)
    indices = np.ascontiguousarray(indices, dtype=np.int32)
    data = np.ascontiguousarray(data, dtype=np.float32)
    n = len(indptr) - 1
    mem = np.empty(n, dtype=np.int32)
    ini = None if init is None else np.ascontiguousarray(init, dtype=np.int32)
    nc = ctypes.c_int64(0)
    q = ctypes.c_double(0.0)
    lv = ctypes.c_int(0)
    rc = _load().oracle_leiden(_ptr(indptr), _ptr(indices), _ptr(data), n, float(resolution), n_iter, max_levels,
                               max_rounds, _ptr(ini), _ptr(mem), ctypes.byref(nc), ctypes.byref(q), ctypes.byref(lv))
    if rc != 0:
        raise ValueError(f"oracle_leiden failed with status {rc}")
    return mem, int(nc.value), float(q.value), int(lv.value)
