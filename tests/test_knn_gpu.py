"""GPU parity of rsc_knn against the FP64 oracle (through the C ABI)."""
import numpy as np
import pytest

import oracle
from paper_2603_02402_gb300 import synth
from parity import check_knn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rsc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_02402_gb300 import rsc as mod
    mod.lib()
    return mod


def run_knn(rsc, X, k, metric="euclidean", precision="fp32", **kw):
    Xd = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).cuda()
    ws = torch.empty(rsc.rsc_knn_workspace_size(*X.shape, k, metric, precision,
                                                kw.get("candidates", 0), kw.get("db_splits", 0),
                                                kw.get("locality", "auto")),
                     dtype=torch.uint8, device="cuda")
    idx, dist = rsc.rsc_knn(Xd, k, metric, precision, workspace=ws, **kw)
    assert rsc.rsc_workspace_status(ws) == rsc.RSC_OK
    torch.cuda.synchronize()
    return idx.cpu().numpy(), dist.cpu().numpy()


PRECISIONS = ["fp32", "bf16"]
# BF16 candidate search + exact re-rank targets recall@k >= 0.999; FP32 is exact
MISS = {"fp32": 0.0, "bf16": 1e-3}


def _maybe(rsc, fn):
    try:
        return fn()
    except rsc.RscError as e:
        if e.status == rsc.RSC_ERR_UNSUPPORTED:
            pytest.skip(str(e))
        raise


@pytest.mark.parametrize("precision", PRECISIONS)
def test_10k_mixture_full_parity(rsc, precision):
    # 10,000 cells x 50 PCs, 20-cluster mixture, k = 15 (the small workload)
    X = synth.mixture(10_000, 50, n_comp=20, seed=0)
    oi, od, on = oracle.knn(X, 15)
    gi, gd = _maybe(rsc, lambda: run_knn(rsc, X, 15, precision=precision))
    stats = check_knn(X, gi, gd, oi, od, on, allow_miss=MISS[precision])
    assert stats["id_exact"] > 0.999


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("n,d,k", [
    (1, 50, 1), (14, 50, 14), (15, 50, 15), (16, 50, 15), (127, 50, 15), (128, 50, 15),
    (129, 50, 15), (257, 16, 15), (1000, 1, 7), (1000, 64, 15), (2049, 50, 32), (3001, 50, 64),
    (700, 3, 1), (4097, 50, 15),
])
def test_shapes_and_ragged_tails(rsc, precision, n, d, k):
    X = synth.mixture(n, d, n_comp=5, seed=n + d)
    oi, od, on = oracle.knn(X, k)
    gi, gd = _maybe(rsc, lambda: run_knn(rsc, X, k, precision=precision))
    check_knn(X, gi, gd, oi, od, on, allow_miss=MISS[precision])


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("splits", [1, 3, 8])
def test_database_splits(rsc, precision, splits):
    X = synth.mixture(3000, 50, n_comp=10, seed=3)
    oi, od, on = oracle.knn(X, 15)
    gi, gd = _maybe(rsc, lambda: run_knn(rsc, X, 15, precision=precision, db_splits=splits))
    check_knn(X, gi, gd, oi, od, on, allow_miss=MISS[precision])


@pytest.mark.parametrize("precision", PRECISIONS)
def test_cosine_with_zero_rows(rsc, precision):
    X = synth.mixture(5000, 50, n_comp=20, seed=4)
    X[[7, 100, 4999]] = 0.0          # all-zero rows: distance 0 between them, 1 to others
    oi, od, on = oracle.knn(X, 30, metric=oracle.COSINE)
    gi, gd = _maybe(rsc, lambda: run_knn(rsc, X, 30, metric="cosine", precision=precision))
    check_knn(X, gi, gd, oi, od, on, metric="cosine", allow_miss=MISS[precision])
    assert gi[7].tolist()[:3] == [7, 100, 4999]


@pytest.mark.parametrize("precision", PRECISIONS)
def test_exact_ties_and_duplicates_integer_grid(rsc, precision):
    # integer points: every distance is exact in FP32, so ties must be broken
    # by ascending index exactly as the oracle does
    g = np.stack(np.meshgrid(np.arange(12), np.arange(12), np.arange(6)), -1).reshape(-1, 3)
    X = np.concatenate([g, g[:50]]).astype(np.float32)   # 50 duplicates
    oi, od, on = oracle.knn(X, 15)
    gi, gd = _maybe(rsc, lambda: run_knn(rsc, X, 15, precision=precision))
    if precision == "fp32":
        np.testing.assert_array_equal(gi, oi)
        np.testing.assert_array_equal(gd, od.astype(np.float32))
    else:
        check_knn(X, gi, gd, oi, od, on, allow_miss=MISS[precision])


def test_large_offset_is_translation_invariant(rsc):
    # a common offset of 1e3 leaves Euclidean distances unchanged; the
    # centring in the prep pass keeps the candidate search accurate
    X = synth.mixture(4000, 50, n_comp=10, seed=6) + np.float32(1000.0)
    oi, od, on = oracle.knn(X, 15)
    gi, gd = run_knn(rsc, X, 15)
    check_knn(X, gi, gd, oi, od, on)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_query_sample_of_large_input(rsc, precision):
    # 200,000 cells: compare a seeded sample of rows with the oracle
    X = synth.mixture(200_000, 50, n_comp=100, seed=1)
    q = synth.query_sample(len(X), 200, seed=1)
    oi, od, on = oracle.knn(X, 15, queries=q)
    gi, gd = _maybe(rsc, lambda: run_knn(rsc, X, 15, precision=precision))
    check_knn(X, gi[q], gd[q], oi, od, on, rows=q, allow_miss=MISS[precision])


# ---- locality ordering (coarse k-means + stable sort, window-first scan)

@pytest.mark.parametrize("n,d,k,splits", [
    (300, 50, 15, 0), (2049, 50, 15, 0), (5000, 50, 15, 3), (9001, 50, 30, 0), (4097, 16, 7, 2),
    (20000, 50, 15, 0),
])
def test_locality_order_parity(rsc, n, d, k, splits):
    # forced ordering on several tiles, ragged tails and database splits: the
    # oracle's neighbours, and the same output as the unordered scan
    X = synth.mixture(n, d, n_comp=12, seed=n)
    oi, od, on = oracle.knn(X, k)
    gi, gd = run_knn(rsc, X, k, precision="bf16", db_splits=splits, locality="on")
    check_knn(X, gi, gd, oi, od, on, allow_miss=MISS["bf16"])
    ui, ud = run_knn(rsc, X, k, precision="bf16", db_splits=splits, locality="off")
    np.testing.assert_array_equal(gi, ui)
    np.testing.assert_array_equal(gd, ud)


def test_locality_order_cosine_zero_rows(rsc):
    X = synth.mixture(6000, 50, n_comp=20, seed=9)
    X[[3, 2500, 5999]] = 0.0
    oi, od, on = oracle.knn(X, 30, metric=oracle.COSINE)
    gi, gd = run_knn(rsc, X, 30, metric="cosine", precision="bf16", locality="on")
    check_knn(X, gi, gd, oi, od, on, metric="cosine", allow_miss=MISS["bf16"])
    assert gi[3].tolist()[:3] == [3, 2500, 5999]


def test_locality_order_integer_ties(rsc):
    # exact FP32 distances with many ties: ties still break by original row id
    g = np.stack(np.meshgrid(np.arange(16), np.arange(16), np.arange(12)), -1).reshape(-1, 3)
    X = np.concatenate([g, g[:100]]).astype(np.float32)
    oi, od, on = oracle.knn(X, 15)
    gi, gd = run_knn(rsc, X, 15, precision="bf16", locality="on")
    check_knn(X, gi, gd, oi, od, on, allow_miss=MISS["bf16"])


def test_locality_order_is_deterministic(rsc):
    X = synth.mixture(30000, 50, n_comp=40, seed=12)
    a = run_knn(rsc, X, 15, precision="bf16", locality="on")
    b = run_knn(rsc, X, 15, precision="bf16", locality="on")
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])
