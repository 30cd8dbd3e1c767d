"""GPU parity of rsc_knn_batched (per-sample and cross-sample kNN) against the
FP64 oracle's definition of both lists."""
import numpy as np
import pytest

import oracle
from paper_2603_02402_gb300 import synth
from parity import check_knn, exact_distances

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rsc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_02402_gb300 import rsc as mod
    mod.lib()
    return mod


def _recall(gi, gd, oi, od):
    # tie-tolerant recall: a returned id is right when its distance is within
    # the oracle's last distance of the row
    ok = gd <= od[:, -1:] * (1 + 1e-6) + 1e-12
    return float(ok.mean())


def run(rsc, X, off, kw, kx, metric="euclidean", use_stream=True, **opts):
    Xd = torch.from_numpy(X).cuda()
    stream = torch.cuda.Stream() if use_stream else None
    ctx = torch.cuda.stream(stream) if use_stream else torch.cuda.stream(torch.cuda.default_stream())
    with ctx:
        ws = torch.empty(rsc.rsc_knn_batched_workspace_size(len(X), X.shape[1], off, kw, kx, metric, **opts),
                         dtype=torch.uint8, device="cuda")
        out = rsc.rsc_knn_batched(Xd, off, kw, kx, metric, stream=stream, workspace=ws, **opts)
        out2 = rsc.rsc_knn_batched(Xd, off, kw, kx, metric, stream=stream, workspace=ws, **opts)   # graph replay
        assert rsc.rsc_workspace_status(ws, stream) == rsc.RSC_OK
    torch.cuda.synchronize()
    res = [t.cpu().numpy() for t in out]
    res2 = [t.cpu().numpy() for t in out2]
    for a, b in zip(res, res2):
        np.testing.assert_array_equal(a, b)
    return res


@pytest.mark.parametrize("metric", ["euclidean", "cosine"])
def test_batched_small_samples(rsc, metric):
    sizes = [300, 1000, 129, 2048, 517, 40]
    X, off = synth.batched(sizes, d=50, n_comp=5, seed=3)
    kw, kx = 15, 3
    m = oracle.EUCLIDEAN if metric == "euclidean" else oracle.COSINE
    wi, wd, xi, xd = oracle.batched_knn(X, off, kw, kx, m)
    gi, gd, gxi, gxd = run(rsc, X, off, kw, kx, metric)
    # within-sample lists: ids in the cell's own sample, exact up to the recall bound
    samp = np.searchsorted(off, np.arange(len(X)), side="right") - 1
    assert (np.searchsorted(off, gi, side="right") - 1 == samp[:, None]).all()
    check_knn(X, gi, gd, wi, wd, np.full(len(X), np.inf), metric=metric, allow_miss=1e-3)
    # cross lists: k_cross from every sample, whole row ordered by (distance, id)
    S = len(sizes)
    gs = np.searchsorted(off, gxi, side="right") - 1
    for t in range(S):
        assert ((gs == t).sum(axis=1) == kx).all()
    assert (np.diff(gxd, axis=1) >= 0).all()
    assert _recall(gxi, gxd, xi, xd) >= 0.999
    _cross_distances_ok(X, gxi, gxd, xd, metric)


def _cross_distances_ok(X, gxi, gxd, xd, metric):
    # every returned distance is the exact distance of the returned id, and
    # (almost) every row holds exactly the oracle's distances
    dex = exact_distances(X, np.arange(len(X)), gxi, metric)
    np.testing.assert_allclose(gxd, dex, rtol=1e-5, atol=1e-6)
    row_ok = np.all(np.abs(gxd - xd) <= 1e-5 * xd + 1e-6, axis=1)
    assert row_ok.mean() >= 0.99


def test_batched_legacy_stream_and_k_limits(rsc):
    X, off = synth.batched([200, 300, 250], d=20, n_comp=3, seed=4)
    wi, wd, xi, xd = oracle.batched_knn(X, off, 16, 4)
    gi, gd, gxi, gxd = run(rsc, X, off, 16, 4, use_stream=False)
    check_knn(X, gi, gd, wi, wd, np.full(len(X), np.inf), allow_miss=1e-3)
    _cross_distances_ok(X, gxi, gxd, xd, "euclidean")
    with pytest.raises(rsc.RscError):
        rsc.rsc_knn_batched(torch.from_numpy(X).cuda(), off, 17, 3)
    with pytest.raises(rsc.RscError):
        rsc.rsc_knn_batched(torch.from_numpy(X).cuda(), off, 15, 5)
    with pytest.raises(rsc.RscError):
        rsc.rsc_knn_batched(torch.from_numpy(X).cuda(), [0, 10, len(X)], 15, 3)   # sample smaller than k


def test_batched_full_size_sampled(rsc):
    # the 64-sample, ~3M-cell workload: a seeded sample of rows against the oracle
    sizes = synth.batched_sizes(64, seed=0)
    X, off = synth.batched(sizes, d=50, n_comp=30, seed=0)
    n = len(X)
    Xd = torch.from_numpy(X).cuda()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        gi, gd, gxi, gxd = [t.cpu().numpy() for t in rsc.rsc_knn_batched(Xd, off, 15, 3, stream=stream)]
    q = synth.query_sample(n, 60, seed=3)
    samp = np.searchsorted(off, q, side="right") - 1
    OI = np.empty((len(q), 15), dtype=np.int32)
    OD = np.empty((len(q), 15))
    for i, (r, s) in enumerate(zip(q, samp)):
        a, b = off[s], off[s + 1]
        oi, od, _ = oracle.knn_qd(X[r:r + 1], X[a:b], 15)
        OI[i], OD[i] = oi[0] + a, od[0]
    check_knn(X, gi[q], gd[q], OI, OD, np.full(len(q), np.inf), rows=q, allow_miss=1e-3)
    # cross lists of the sample rows, from every sample
    exp_d = []
    for t in range(64):
        a, b = off[t], off[t + 1]
        _, od, _ = oracle.knn_qd(X[q], X[a:b], 3)
        exp_d.append(od)
    exp_d = np.sort(np.concatenate(exp_d, axis=1), axis=1)
    assert _recall(gxi[q], gxd[q], None, exp_d) >= 0.999
    dex = exact_distances(X, q, gxi[q], "euclidean")
    np.testing.assert_allclose(gxd[q], dex, rtol=1e-5, atol=1e-6)
    row_ok = np.all(np.abs(gxd[q] - exp_d) <= 1e-5 * exp_d + 1e-6, axis=1)
    assert row_ok.mean() >= 0.95


@pytest.mark.parametrize("metric", ["euclidean", "cosine"])
@pytest.mark.parametrize("prune", ["on", "off"])
def test_batched_ordered_and_pruned(rsc, metric, prune):
    # above the ordering threshold: rows in cluster order inside each sample,
    # window pass + sphere bounds + list pass (or the ordered full scan); both
    # against the FP64 oracle on every row
    sizes = [9000, 14000, 2500, 8000, 700]
    X, off = synth.batched(sizes, d=50, n_comp=12, seed=21)
    kw, kx = 15, 3
    m = oracle.COSINE if metric == "cosine" else oracle.EUCLIDEAN
    wi, wd, xi, xd = oracle.batched_knn(X, off, kw, kx, m)
    gi, gd, gxi, gxd = run(rsc, X, off, kw, kx, metric, locality="on", prune=prune)
    assert _recall(gi, gd, wi, wd) >= 0.999
    assert _recall(gxi, gxd, xi, xd) >= 0.999
    np.testing.assert_allclose(np.sort(gd, axis=1)[:, 0], wd[:, 0], rtol=1e-5, atol=1e-6)
    assert (np.diff(gxd, axis=1) >= 0).all()


def test_batched_scan_stats(rsc):
    # (128-row query tile, 256-row database tile) pairs of one sample the last
    # call computed: all of them without pruning, fewer with it
    sizes = [9000, 14000, 2500, 8000, 700]
    X, off = synth.batched(sizes, d=50, n_comp=12, seed=21)
    n = len(X)
    Xd = torch.from_numpy(X).cuda()
    T = sum(-(-s // 128) for s in sizes)
    DT = sum(-(-s // 256) for s in sizes)
    for prune in ("off", "on"):
        ws = torch.empty(rsc.rsc_knn_batched_workspace_size(n, 50, off, 15, 3, locality="on", prune=prune),
                         dtype=torch.uint8, device="cuda")
        rsc.rsc_knn_batched(Xd, off, 15, 3, workspace=ws, locality="on", prune=prune)
        scanned, total = rsc.rsc_knn_batched_scan_stats(n, 50, off, 15, 3, ws, locality="on", prune=prune)
        assert total == T * DT
        if prune == "off":
            assert scanned == total
        else:
            assert 0 < scanned < total
