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
                                                kw.get("locality", "auto"), kw.get("prune", "auto")),
                     dtype=torch.uint8, device="cuda")
    idx, dist = rsc.rsc_knn(Xd, k, metric, precision, workspace=ws, **kw)
    assert rsc.rsc_workspace_status(ws) == rsc.RSC_OK
    torch.cuda.synchronize()
    return idx.cpu().numpy(), dist.cpu().numpy()


PRECISIONS = ["fp32", "bf16", "fp8"]
# BF16 / FP8 candidate search + exact re-rank targets recall@k >= 0.999; FP32 is exact
MISS = {"fp32": 0.0, "bf16": 1e-3, "fp8": 1e-3}


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


@pytest.mark.parametrize("metric,n,d", [("euclidean", 3001, 50), ("euclidean", 700, 7), ("euclidean", 5000, 64),
                                         ("cosine", 3001, 50), ("cosine", 700, 7), ("cosine", 5000, 63)])
def test_fp32_list_widths_agree(rsc, metric, n, d):
    # FP32 candidate lists of 32 come from 8 x 8 register blocks over 64-row
    # tiles, lists of 64 from 8 x 4 blocks over 32-row tiles; both must give
    # the exact lists
    X = synth.mixture(n, d, n_comp=8, seed=d + 1)
    om = oracle.COSINE if metric == "cosine" else oracle.EUCLIDEAN
    oi, od, on = oracle.knn(X, 15, metric=om)
    ai, ad = run_knn(rsc, X, 15, metric=metric, precision="fp32", candidates=24)
    bi, bd = run_knn(rsc, X, 15, metric=metric, precision="fp32", candidates=40)
    check_knn(X, ai, ad, oi, od, on, metric=metric, allow_miss=0.0)
    np.testing.assert_array_equal(ai, bi)
    np.testing.assert_array_equal(ad, bd)


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
    # oracle's neighbours.  The ordering moves rows between column parts, so
    # the BF16 candidate sets (beyond each part's best) may differ from the
    # unordered scan's; both must meet the recall bound and agree almost
    # everywhere.
    X = synth.mixture(n, d, n_comp=12, seed=n)
    oi, od, on = oracle.knn(X, k)
    gi, gd = run_knn(rsc, X, k, precision="bf16", db_splits=splits, locality="on")
    check_knn(X, gi, gd, oi, od, on, allow_miss=MISS["bf16"])
    ui, ud = run_knn(rsc, X, k, precision="bf16", db_splits=splits, locality="off")
    check_knn(X, ui, ud, oi, od, on, allow_miss=MISS["bf16"])
    assert (gi == ui).mean() >= 0.995


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


# ---- exact tile pruning (window pass, sphere bounds, list pass)

@pytest.mark.parametrize("n,d,k,comp,cands", [
    (20000, 50, 15, 30, 0), (33333, 50, 15, 60, 0), (40000, 50, 30, 40, 0), (25000, 32, 7, 20, 0),
    (30000, 50, 15, 25, 64),
])
def test_prune_equals_full_scan(rsc, n, d, k, comp, cands):
    # the pruned scan keeps exactly the unpruned scan's candidates, so the
    # re-ranked output is bit-identical; both match the oracle
    X = synth.mixture(n, d, n_comp=comp, seed=n + k)
    pi, pd = run_knn(rsc, X, k, precision="bf16", locality="on", prune="on", candidates=cands)
    fi, fd = run_knn(rsc, X, k, precision="bf16", locality="on", prune="off", candidates=cands)
    np.testing.assert_array_equal(pi, fi)
    np.testing.assert_array_equal(pd, fd)
    q = synth.query_sample(n, 300, seed=k)
    oi, od, on = oracle.knn(X, k, queries=q)
    check_knn(X, pi[q], pd[q], oi, od, on, rows=q, allow_miss=MISS["bf16"])


def test_prune_anisotropic_and_offset(rsc):
    X = synth.anisotropic(50000, 50, n_comp=40, seed=3) + np.float32(7.0)
    pi, pd = run_knn(rsc, X, 15, precision="bf16", locality="on", prune="on")
    fi, fd = run_knn(rsc, X, 15, precision="bf16", locality="on", prune="off")
    np.testing.assert_array_equal(pi, fi)
    np.testing.assert_array_equal(pd, fd)


def test_prune_cosine_zero_rows(rsc):
    X = synth.mixture(30000, 50, n_comp=30, seed=17)
    X[[5, 15000, 29999]] = 0.0
    pi, pd = run_knn(rsc, X, 30, metric="cosine", precision="bf16", locality="on", prune="on")
    fi, fd = run_knn(rsc, X, 30, metric="cosine", precision="bf16", locality="on", prune="off")
    np.testing.assert_array_equal(pi, fi)
    np.testing.assert_array_equal(pd, fd)
    assert pi[5].tolist()[:3] == [5, 15000, 29999]
    q = np.concatenate([[5, 15000], synth.query_sample(len(X), 200, seed=2)])
    oi, od, on = oracle.knn(X, 30, metric=oracle.COSINE, queries=q)
    check_knn(X, pi[q], pd[q], oi, od, on, rows=q, metric="cosine", allow_miss=MISS["bf16"])


def test_prune_integer_ties(rsc):
    # many exact distance ties (integer points: BF16 keys are exact): pruning
    # must not change which tied ids survive, and both are exact kNN lists up
    # to the choice among tied ids
    g = np.stack(np.meshgrid(np.arange(32), np.arange(32), np.arange(24)), -1).reshape(-1, 3)
    X = np.concatenate([g, g[:500]]).astype(np.float32)
    pi, pd = run_knn(rsc, X, 15, precision="bf16", locality="on", prune="on")
    fi, fd = run_knn(rsc, X, 15, precision="bf16", locality="on", prune="off")
    np.testing.assert_array_equal(pi, fi)
    np.testing.assert_array_equal(pd, fd)
    q = synth.query_sample(len(X), 400, seed=4)
    oi, od, on = oracle.knn(X, 15, queries=q)
    for gi, gd in ((pi, pd), (fi, fd)):
        check_knn(X, gi[q], gd[q], oi, od, on, rows=q, allow_miss=MISS["bf16"])


def test_prune_requires_ordering(rsc):
    X = torch.zeros((20000, 50), device="cuda")
    with pytest.raises(rsc.RscError):
        rsc.rsc_knn(X, 15, precision="bf16", locality="off", prune="on")


def test_scan_stats(rsc):
    # pairs of (128-row query tile, 256-row database tile) the search computed
    n = 40000
    X = synth.mixture(n, 50, n_comp=40, seed=8)
    Xd = torch.from_numpy(X).cuda()
    total = -(-n // 128) * -(-n // 256)
    for prune in ("off", "on"):
        ws = torch.empty(rsc.rsc_knn_workspace_size(n, 50, 15, "euclidean", "bf16", locality="on", prune=prune),
                         dtype=torch.uint8, device="cuda")
        rsc.rsc_knn(Xd, 15, precision="bf16", workspace=ws, locality="on", prune=prune)
        scanned, tot = rsc.rsc_knn_scan_stats(n, 50, 15, ws, "euclidean", "bf16", locality="on", prune=prune)
        assert tot == total
        if prune == "off":
            assert scanned == total
        else:
            assert 0 < scanned < total   # 40 separated clusters: most tile pairs are provably useless


@pytest.mark.parametrize("precision", PRECISIONS)
def test_input_rows_off_16_byte_boundary(rsc, precision):
    # X as a view one row into a larger buffer (d = 50: rows start 8 bytes off
    # a 16-byte boundary): the prep's vector loads must fall back, results equal
    # those of an aligned copy
    n, d, k = 20000, 50, 15
    X = synth.mixture(n + 1, d, n_comp=20, seed=31)
    base = torch.from_numpy(X).cuda()
    Xv = base[1:]
    assert Xv.data_ptr() % 16 != 0
    ws = torch.empty(rsc.rsc_knn_workspace_size(n, d, k, "euclidean", precision), dtype=torch.uint8, device="cuda")
    gi, gd = [t.cpu().numpy() for t in rsc.rsc_knn(Xv, k, "euclidean", precision, workspace=ws)]
    ai, ad = run_knn(rsc, X[1:], k, precision=precision)
    np.testing.assert_array_equal(gi, ai)
    np.testing.assert_array_equal(gd, ad)


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_rerank_vector_and_scalar_loads_agree(rsc, precision):
    # d = 48: rows of an aligned X are re-ranked with 16-byte loads, rows of a
    # copy placed 4 bytes off a 16-byte boundary with scalar loads; the partial
    # sums are the same either way, so the results are identical (below the
    # ordering's size, the re-rank reads the caller's rows)
    n, d, k = 6000, 48, 15
    X = synth.mixture(n, d, n_comp=12, seed=41)
    flat = torch.zeros(n * d + 1, dtype=torch.float32, device="cuda")
    flat[1:] = torch.from_numpy(X.reshape(-1)).cuda()
    Xv = flat[1:].view(n, d)
    assert Xv.data_ptr() % 16 != 0
    ws = torch.empty(rsc.rsc_knn_workspace_size(n, d, k, "euclidean", precision), dtype=torch.uint8, device="cuda")
    gi, gd = [t.cpu().numpy() for t in rsc.rsc_knn(Xv, k, "euclidean", precision, workspace=ws)]
    ai, ad = run_knn(rsc, X, k, precision=precision)
    np.testing.assert_array_equal(gi, ai)
    np.testing.assert_array_equal(gd, ad)
    oi, od, on = oracle.knn(X, k)
    check_knn(X, gi, gd, oi, od, on, allow_miss=MISS[precision])


def test_fp8_on_ordered_rows(rsc):
    # 30,000 rows take the locality ordering (window first, no pruning for
    # FP8); default candidates (8k, at most 128)
    X = synth.mixture(30_000, 50, n_comp=20, seed=21)
    q = synth.query_sample(len(X), 400, seed=21)
    oi, od, on = oracle.knn(X, 15, queries=q)
    gi, gd = run_knn(rsc, X, 15, precision="fp8")
    st = check_knn(X, gi[q], gd[q], oi, od, on, rows=q, allow_miss=MISS["fp8"])
    assert st["recall"] >= 0.999


def test_headline_1m_on_20k_query_sample(rsc):
    # the 1,000,000-cell x 50-PC workload (100-component mixture, k = 15) in
    # the bench's launch configuration (automatic options: BF16 candidates on
    # ordered rows with tile pruning, exact FP32 re-rank), and the plain FP32
    # path, against the FP64 oracle on a seeded 20,000-query subsample
    X = synth.mixture(1_000_000, 50, n_comp=100, seed=0)
    q = synth.query_sample(len(X), 20_000, seed=5)
    oi, od, on = oracle.knn(X, 15, queries=q)
    for precision in ("bf16", "fp32"):
        gi, gd = run_knn(rsc, X, 15, precision=precision)
        st = check_knn(X, gi[q], gd[q], oi, od, on, rows=q, allow_miss=MISS[precision])
        print(f"1M {precision} on 20k queries:", st)
        assert st["recall"] >= 0.999
        assert st["max_rel_dist_err"] <= 1e-5


def test_bounded_wait_times_out_and_the_next_call_recovers(rsc):
    # a wait budget of a few hundred SM clocks makes the tensor-core search's
    # first barrier wait give up: the kernel records RSC_ERR_TIMEOUT in the
    # workspace status word (after letting its in-flight copies and MMAs
    # finish), and the next call with the default budget is correct
    X = synth.mixture(4097, 50, n_comp=5, seed=3)
    oi, od, on = oracle.knn(X, 15)
    Xd = torch.from_numpy(X).cuda()
    ws = torch.empty(rsc.rsc_knn_workspace_size(len(X), 50, 15, "euclidean", "bf16"), dtype=torch.uint8,
                     device="cuda")
    rsc.rsc_set_wait_budget(300)
    try:
        rsc.rsc_knn(Xd, 15, precision="bf16", workspace=ws)
        assert rsc.rsc_workspace_status(ws) == rsc.RSC_ERR_TIMEOUT
    finally:
        rsc.rsc_set_wait_budget(0)
    gi, gd = rsc.rsc_knn(Xd, 15, precision="bf16", workspace=ws)
    assert rsc.rsc_workspace_status(ws) == rsc.RSC_OK
    check_knn(X, gi.cpu().numpy(), gd.cpu().numpy(), oi, od, on, allow_miss=MISS["bf16"])
    with pytest.raises(rsc.RscError):
        rsc.rsc_set_wait_budget(-1)
