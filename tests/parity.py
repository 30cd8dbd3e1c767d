"""Comparison helpers for the GPU-vs-oracle parity tests.

Tolerances (from the method's definition of the exact graph):
  * neighbour ids: identical, except positions where the oracle's own
    distances tie within 1e-6 relative (then any of the tied ids is valid);
  * distances: within 1e-5 relative of the oracle's FP64 value;
  * connectivity weights: within 1e-5 absolute, compared densely on the union
    of both sparsity patterns (an entry missing on one side counts as 0).
"""
import numpy as np

TIE_REL = 1e-6
DIST_REL = 1e-5
W_ABS = 1e-5


def exact_distances(X, rows, cols, metric):
    """FP64 distances between X[rows[i]] and X[cols[i, c]] (test-side check)."""
    X = np.asarray(X, dtype=np.float64)
    A = X[rows][:, None, :]
    B = X[cols]
    if metric == "euclidean":
        return np.sqrt(((A - B) ** 2).sum(-1))
    na = np.linalg.norm(A, axis=-1)
    nb = np.linalg.norm(B, axis=-1)
    with np.errstate(invalid="ignore", divide="ignore"):
        cos = (A * B).sum(-1) / (na * nb)
    d = 1.0 - cos
    d = np.where((na == 0) & (nb == 0), 0.0, d)
    d = np.where((na == 0) ^ (nb == 0), 1.0, d)
    return d


def check_knn(X, gi, gd, oi, od, onext, metric="euclidean", rows=None, dist_rel=DIST_REL,
              allow_miss=0.0):
    """Assert GPU kNN (gi, gd) matches the oracle (oi, od, onext) on `rows`.

    Returns a dict of statistics.  `allow_miss` > 0 relaxes the id check to a
    recall bound (for reduced-precision candidate search).
    """
    nq, k = oi.shape
    rows = np.arange(nq) if rows is None else np.asarray(rows)
    gi = np.asarray(gi)
    gd = np.asarray(gd, dtype=np.float64)
    assert gi.shape == (nq, k) and gd.shape == (nq, k)
    assert (gi >= 0).all(), "missing neighbours"
    dex = exact_distances(X, rows, gi, metric)             # exact distance of each returned id
    scale = np.maximum(od[:, -1], 1e-30)
    kth = od[:, -1]
    # ids: equal, or the returned neighbour is tied (within 1e-6 rel) with the oracle's
    same = gi == oi
    tied = np.abs(dex - od) <= TIE_REL * scale[:, None]
    inside = dex <= (kth + TIE_REL * scale)[:, None]
    ok_id = same | (tied & inside)
    recall = _recall(gi, oi, dex, kth, scale)
    if allow_miss == 0.0:
        bad = np.argwhere(~ok_id)
        assert bad.size == 0, f"{len(bad)} id mismatches beyond ties, first {bad[:5].tolist()} " \
                              f"gpu={gi[bad[0][0]].tolist()} oracle={oi[bad[0][0]].tolist()}"
        for i in range(nq):                                 # no id twice
            assert len(set(gi[i].tolist())) == k
    else:
        assert recall >= 1.0 - allow_miss, f"recall {recall}"
    # distances: relative to the oracle's distance at the same rank
    err = np.abs(gd - od)
    tol = dist_rel * od + 1e-7 * scale[:, None]
    if allow_miss == 0.0:
        assert (err <= tol).all(), f"max rel dist err {np.max(err / np.maximum(od, 1e-30))}"
    # each returned distance is the exact distance of the returned id
    assert (np.abs(gd - dex) <= dist_rel * dex + 1e-7 * scale[:, None]).all()
    # rows ascending
    assert (np.diff(gd, axis=1) >= 0).all()
    return {"id_exact": float(same.mean()), "recall": recall,
            "max_rel_dist_err": float(np.max(np.abs(gd - dex) / np.maximum(dex, 1e-30)))}


def _recall(gi, oi, dex, kth, scale):
    """recall@k, counting a returned id correct when its exact distance is
    within the oracle's k-th distance (tie-tolerant)."""
    good = dex <= (kth * (1 + TIE_REL) + 1e-30)[:, None]
    return float(good.mean())


def _coo_keys(indptr, indices, data, n):
    """Row-major keys row * n + col and values of a CSR graph."""
    indptr = np.asarray(indptr, dtype=np.int64)
    nnz = int(indptr[-1])
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(indptr))
    keys = rows * n + np.asarray(indices[:nnz], dtype=np.int64)
    return keys, np.asarray(data[:nnz], dtype=np.float64)


def check_csr_structure(indptr, indices, data, n):
    indptr = np.asarray(indptr)
    assert indptr[0] == 0 and (np.diff(indptr) >= 0).all()
    nnz = int(indptr[-1])
    ind, dat = np.asarray(indices)[:nnz], np.asarray(data)[:nnz]
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(indptr))
    same_row = rows[1:] == rows[:-1]
    bad = np.nonzero(same_row & (np.diff(ind.astype(np.int64)) <= 0))[0]
    assert bad.size == 0, f"row {rows[bad[0]]} not strictly ascending"
    diag = np.nonzero(ind == rows)[0]
    assert diag.size == 0, f"diagonal in row {rows[diag[0]]}"
    assert ((dat > 0) & (dat <= 1)).all()
    assert ((ind >= 0) & (ind < n)).all()
    return ind, dat


def compare_graphs(gpu, ref, n, exclude_rows=(), atol=W_ABS):
    """Dense-on-union comparison (an entry missing on one side counts as 0);
    entries in a row or column of `exclude_rows` are skipped.  Returns (max
    error, entries compared)."""
    gk, gv = _coo_keys(*gpu, n)
    rk, rv = _coo_keys(*ref, n)
    keys = np.union1d(gk, rk)
    a = np.zeros(len(keys))
    b = np.zeros(len(keys))
    a[np.searchsorted(keys, gk)] = gv
    b[np.searchsorted(keys, rk)] = rv
    rows, cols = keys // n, keys % n
    keep = np.ones(len(keys), dtype=bool)
    if len(exclude_rows):
        ex = np.zeros(n, dtype=bool)
        ex[np.asarray(exclude_rows, dtype=np.int64)] = True
        keep = ~(ex[rows] | ex[cols])
    err = np.abs(a - b)
    bad = np.nonzero(keep & (err > atol))[0]
    if bad.size:
        e = bad[0]
        raise AssertionError(f"{bad.size} entries beyond {atol}; first ({rows[e]}, {cols[e]}): "
                             f"gpu {a[e]} oracle {b[e]}")
    return (float(err[keep].max()) if keep.any() else 0.0), int(keep.sum())


def near_branch_rows(ref, margin=1e-6):
    """Rows whose FP64 bisection came within `margin` of flipping its stop
    test (|psum - log2 k| within margin of 1e-5 at some step).  The FP32
    psum (compensated sum of 2-ulp exps) is accurate to about 1e-6, so FP32
    may stop one step earlier or later on exactly these rows; about 13% of
    rows of a Gaussian-mixture graph qualify, because the last step's error
    is spread over [0, 1e-5).  They are compared at 5e-5 instead of 1e-5."""
    return np.nonzero(ref["stop_margin"] < margin)[0]


def propagated_weight_slack(ref, od, delta):
    """First-order change of the oracle's directed weights when its kNN
    distances move by delta [n, k] (absolute, per entry).

    rho moves by delta at rho's column (its first non-zero distance); sigma
    solves sum_{c>=1} exp(-(d_c - rho) / sigma) = log2 k, so to first order
    dsigma / sigma = sum w_c (dd_c - drho) / sum w_c (d_c - rho) over the
    columns with d_c > rho (a floored sigma moves like the mean distance);
    w_c = exp(-(d_c - rho) / sigma) then moves by
    w_c ((dd_c - drho) - (d_c - rho) dsigma / sigma) / sigma.  Bounded term by
    term with |dd_c| + |drho| in place of the signed differences; a column at
    rho (weight 1) may leave it, so it gets e_c / sigma.  Returns [n, k].
    """
    od = np.asarray(od, dtype=np.float64)
    n, k = od.shape
    rho, sigma, w = ref["rho"], ref["sigma"], ref["weights"]
    delta = np.abs(np.asarray(delta, dtype=np.float64))
    first = np.argmax(od > 0, axis=1)                       # rho's column
    drho = np.where(rho > 0, delta[np.arange(n), first], 0.0)
    e = delta + drho[:, None]
    beyond = od - rho[:, None]
    pos = beyond > 0
    pos[:, 0] = False
    num = np.where(pos, w * e, 0.0).sum(1)
    den = np.where(pos, w * beyond, 0.0).sum(1)
    rel_sigma = np.where(den > 0, num / np.where(den > 0, den, 1.0), 0.0)
    floored = ref["floored"].astype(bool)
    rel_mean = (delta / np.maximum(od, 1e-30)).max(1)
    rel_sigma = np.where(floored, rel_mean, rel_sigma)
    s = sigma[:, None]
    slack = np.where(pos, w, 1.0) * (e / s + np.maximum(beyond, 0.0) / s * rel_sigma[:, None])
    slack[:, 0] = 0.0                                       # the row itself: weight 0
    return slack


def compare_pipeline_graphs(gpu, ref, oi, slack, n, near, atol=W_ABS, atol_near=5e-5, exclude=None):
    """Dense-on-union comparison of a GPU graph with the oracle's graph of the
    oracle's own kNN lists oi: per entry tolerance atol (atol_near when either
    end is a near-branch row) + 2 (slack_ij + slack_ji), the directed slacks
    of propagated_weight_slack placed at (i, oi[i, c]) and transposed.
    Entries touching a row of `exclude` (bool [n]) are skipped.
    Returns (max error / tolerance, entries compared)."""
    gk, gv = _coo_keys(*gpu, n)
    rk, rv = _coo_keys(*ref, n)
    keys = np.union1d(gk, rk)
    a = np.zeros(len(keys))
    b = np.zeros(len(keys))
    a[np.searchsorted(keys, gk)] = gv
    b[np.searchsorted(keys, rk)] = rv
    k = oi.shape[1]
    rows = np.repeat(np.arange(n, dtype=np.int64), k)
    cols = np.asarray(oi, dtype=np.int64).ravel()
    sl = np.asarray(slack).ravel()
    extra = np.zeros(len(keys))
    for kk in (rows * n + cols, cols * n + rows):
        pos = np.searchsorted(keys, kk)
        hit = (pos < len(keys)) & (keys[np.minimum(pos, len(keys) - 1)] == kk)
        np.add.at(extra, pos[hit], sl[hit])
    r, c = keys // n, keys % n
    base = np.where(near[r] | near[c], atol_near, atol)
    tol = base + 2.0 * extra
    err = np.abs(a - b)
    keep = np.ones(len(keys), dtype=bool) if exclude is None else ~(exclude[r] | exclude[c])
    bad = np.nonzero(keep & (err > tol))[0]
    if bad.size:
        e = bad[0]
        raise AssertionError(f"{bad.size} entries beyond tolerance; first ({r[e]}, {c[e]}): gpu {a[e]} "
                             f"oracle {b[e]} tol {tol[e]}")
    return float((err[keep] / tol[keep]).max()), int(keep.sum())


def check_pipeline_graph(gpu, gi, gd, oi, od, ref, n):
    """GPU kNN -> GPU connectivities against oracle kNN -> oracle
    connectivities (the oracle never sees a GPU value).  rho: the distance at
    the same column, within the kNN distance tolerance; weights: 1e-5 (5e-5 on
    near-branch rows) plus the first-order effect of the measured distance
    differences |gd - od| (propagated_weight_slack).  Rows whose id sets differ
    (reduced-precision misses, ties) are left out and counted."""
    ip, ind, dat, rho, _ = gpu
    od = np.asarray(od, dtype=np.float64)
    same = np.all(np.sort(gi, axis=1) == np.sort(oi, axis=1), axis=1)
    delta = np.where(same[:, None], np.asarray(gd, dtype=np.float64) - od, 0.0)
    np.testing.assert_allclose(rho[same], ref["rho"][same], rtol=DIST_REL, atol=1e-7)
    near = np.zeros(n, dtype=bool)
    near[near_branch_rows(ref)] = True
    slack = propagated_weight_slack(ref, od, delta)
    ratio, cnt = compare_pipeline_graphs((ip, ind, dat), (ref["indptr"], ref["indices"], ref["data"]), oi, slack,
                                         n, near, exclude=~same)
    return {"ratio": ratio, "entries": cnt, "rows_left_out": int((~same).sum()),
            "median_slack": float(np.median(slack[:, 1:]))}
