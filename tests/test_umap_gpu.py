"""GPU parity of rsc_umap_layout against the oracle's UMAP layout epochs.

Graphs come from the oracle (its exact kNN, or a k-d tree on low-dimensional
mixtures at full size, followed by its connectivities), starting positions
from the seeded generator: no oracle input comes from the GPU.  One epoch is a
function of the graph and the positions it starts from, so single epochs are
compared vertex by vertex at several epochs of the schedule and from several
states; a run of many epochs is checked to equal the composition of single
epochs bit for bit, and whole runs are compared by the layout they reach.

Tolerance of a vertex (single epoch): 4e-6 times the sum of |move| over the
coordinates of every move applied to it (FP32 moves carry a relative error of
a few units of 2^-24 from the power and the products, and the lanes' partial
sums and the warp's tree add about ten roundings more), plus 2^-21 |y|
(FP32 rounding of the new position) plus 1e-9.
"""
import numpy as np
import pytest

import oracle
from paper_2603_02402_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

A, B = 0.583, 1.334


@pytest.fixture(scope="module")
def rsc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_02402_gb300 import rsc as mod
    mod.lib()
    return mod


def oracle_graph(X, k):
    idx, dist, _ = oracle.knn(X, k)
    g = oracle.connectivities(idx, dist.astype(np.float32).astype(np.float64))
    return g["indptr"], g["indices"], g["data"].astype(np.float32)


def kdtree_graph(X, k):
    spatial = pytest.importorskip("scipy.spatial")
    dist, idx = spatial.cKDTree(X.astype(np.float64)).query(X.astype(np.float64), k, workers=-1)
    g = oracle.connectivities(idx.astype(np.int32), dist.astype(np.float32).astype(np.float64))
    return g["indptr"], g["indices"], g["data"].astype(np.float32)


@pytest.fixture(scope="module")
def graph3k():
    return oracle_graph(synth.mixture(3000, 50, n_comp=12, seed=21), 15)


def gpu_epochs(rsc, graph, Y, first, last, N=200, **kw):
    ip, ind, dat = graph
    emb = torch.from_numpy(np.ascontiguousarray(Y, dtype=np.float32)).cuda()
    t = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (ip, ind, dat)]
    ws = torch.empty(rsc.rsc_umap_workspace_size(len(Y), len(ind), Y.shape[1]), dtype=torch.uint8, device="cuda")
    rsc.rsc_umap_layout(t[0], t[1], t[2], emb, kw.pop("a", A), kw.pop("b", B), n_epochs=N, epoch_first=first,
                        epoch_last=last, nnz=len(ind), workspace=ws, **kw)
    status = rsc.rsc_workspace_status(ws)
    return emb.cpu().numpy(), status


def assert_epoch_parity(got, Y, ref, absmove, mask=None):
    rows = np.arange(len(Y)) if mask is None else np.flatnonzero(mask)
    err = np.abs(got[rows].astype(np.float64) - ref[rows]).max(axis=1)
    tol = 4e-6 * absmove[rows] + 2.0 ** -21 * np.abs(ref[rows]).max(axis=1) + 1e-9
    bad = np.flatnonzero(err > tol)
    assert len(bad) == 0, (f"{len(bad)} of {len(rows)} vertices outside tolerance; worst ratio "
                           f"{(err / tol).max():.3g} at row {rows[np.argmax(err / tol)]}")
    moved = np.abs(ref[rows] - Y[rows]).max(axis=1) > 0
    return float((err / tol).max()), int(moved.sum())


@pytest.mark.parametrize("epoch", [1, 2, 77, 150, 200])
@pytest.mark.parametrize("state", ["uniform", "clustered"])
def test_single_epoch_matches_oracle(rsc, graph3k, epoch, state):
    Y = synth.positions(3000, 2, seed=epoch, clusters=12 if state == "clustered" else 0)
    got, status = gpu_epochs(rsc, graph3k, Y, epoch, epoch, seed=17)
    assert status == rsc.RSC_OK
    ref, absmove, samples = oracle.umap_epochs(*graph3k, Y, A, B, n_epochs=200, first=epoch, last=epoch, seed=17)
    ratio, moved = assert_epoch_parity(got, Y, ref, absmove)
    assert moved > 100 and samples.sum() > 0


@pytest.mark.parametrize("dim", [1, 3, 4])
def test_single_epoch_other_dimensions(rsc, graph3k, dim):
    Y = synth.positions(3000, dim, seed=40 + dim, clusters=6)
    got, status = gpu_epochs(rsc, graph3k, Y, 9, 9, N=50, seed=5, negative_sample_rate=3, gamma=0.7,
                             learning_rate=0.8)
    assert status == rsc.RSC_OK
    ref, absmove, _ = oracle.umap_epochs(*graph3k, Y, A, B, gamma=0.7, lr=0.8, neg_rate=3, n_epochs=50, first=9,
                                         last=9, seed=5)
    assert_epoch_parity(got, Y, ref, absmove)


def test_other_curve_parameters_and_rates(rsc, graph3k):
    a, b = 1.577, 0.895    # min_dist 0.1, spread 1
    Y = synth.positions(3000, 2, seed=3)
    for r in (0, 1, 12):
        got, _ = gpu_epochs(rsc, graph3k, Y, 3, 3, N=10, seed=2, negative_sample_rate=r, a=a, b=b)
        ref, absmove, _ = oracle.umap_epochs(*graph3k, Y, a, b, neg_rate=r, n_epochs=10, first=3, last=3, seed=2)
        assert_epoch_parity(got, Y, ref, absmove)


def test_epochs_compose_bit_for_bit(rsc, graph3k):
    Y = synth.positions(3000, 2, seed=8)
    whole, _ = gpu_epochs(rsc, graph3k, Y, 1, 20, N=20, seed=4)
    again, _ = gpu_epochs(rsc, graph3k, Y, 1, 20, N=20, seed=4)
    np.testing.assert_array_equal(whole, again)
    split, _ = gpu_epochs(rsc, graph3k, Y, 1, 7, N=20, seed=4)
    split, _ = gpu_epochs(rsc, graph3k, split, 8, 20, N=20, seed=4)
    np.testing.assert_array_equal(whole, split)
    step = Y
    for e in range(1, 21):
        step, _ = gpu_epochs(rsc, graph3k, step, e, e, N=20, seed=4)
    np.testing.assert_array_equal(whole, step)
    assert np.abs(whole - Y).max() > 1.0


def _csr(rows, n):
    indptr, indices, data = [0], [], []
    for i in range(n):
        r = sorted(rows.get(i, []))
        indices += [c for c, _ in r]
        data += [w for _, w in r]
        indptr.append(len(indices))
    return np.array(indptr, np.int64), np.array(indices, np.int32), np.array(data, np.float32)


def test_hub_rows_isolated_vertices_and_a_clique(rsc):
    rng = np.random.default_rng(3)
    n, hub_leaves = 1500, 1000
    rows = {}
    def add(i, j, w):
        rows.setdefault(i, []).append((j, w))
        rows.setdefault(j, []).append((i, w))
    for leaf in range(1, hub_leaves + 1):   # row 0 holds 1000 entries (32-entry chunks and a ragged tail)
        add(0, leaf, float(np.float32(rng.uniform(0.05, 1.0))))
    for i in range(1100, 1140):             # a 40-clique of weight-1 edges
        for j in range(i + 1, 1140):
            add(i, j, 1.0)
    # rows 1200 .. 1499 stay isolated
    graph = _csr(rows, n)
    Y = synth.positions(n, 2, seed=12)
    for epoch in (1, 5, 30):
        got, status = gpu_epochs(rsc, graph, Y, epoch, epoch, N=30, seed=9)
        assert status == rsc.RSC_OK
        ref, absmove, _ = oracle.umap_epochs(*graph, Y, A, B, n_epochs=30, first=epoch, last=epoch, seed=9)
        assert_epoch_parity(got, Y, ref, absmove)
        np.testing.assert_array_equal(got[1200:], Y[1200:])


@pytest.mark.parametrize("case", ["single_vertex", "no_entries", "zero_weights", "one_epoch"])
def test_degenerate_graphs(rsc, case):
    if case == "single_vertex":
        graph, Y = _csr({}, 1), np.array([[1.5, -2.0]], np.float32)
    elif case == "no_entries":
        graph, Y = _csr({}, 64), synth.positions(64, 2, seed=1)
    elif case == "zero_weights":
        graph, Y = _csr({0: [(1, 0.0)], 1: [(0, 0.0)]}, 2), np.array([[0.0, 0.0], [3.0, 4.0]], np.float32)
    else:
        graph, Y = _csr({0: [(1, 0.25)], 1: [(0, 0.25)], 2: [(3, 1.0)], 3: [(2, 1.0)]}, 4), \
            synth.positions(4, 2, seed=2)
    N = 1 if case == "one_epoch" else 5
    got, status = gpu_epochs(rsc, graph, Y, 1, N, N=N, seed=1)
    assert status == rsc.RSC_OK
    ref, _, _ = oracle.umap_epochs(*graph, Y, A, B, n_epochs=N, seed=1)
    if case == "one_epoch":
        assert np.abs(got[2:] - Y[2:]).max() > 0       # the weight-1 pair is sampled in epoch 1
        np.testing.assert_array_equal(got[:2], Y[:2])   # f = 1/4: floor(1/4) = 0, not sampled
    else:
        np.testing.assert_array_equal(got, Y)
    np.testing.assert_allclose(got, ref, rtol=1e-5, atol=1e-5)


def test_bad_graph_is_recorded_and_skipped(rsc):
    ip, ind, dat = _csr({0: [(1, 1.0)], 1: [(0, 1.0)], 2: [(3, 1.0)], 3: [(2, 1.0)]}, 4)
    Y = synth.positions(4, 2, seed=5)
    bad_col = ind.copy()
    bad_col[0] = 7    # column outside [0, n)
    got, status = gpu_epochs(rsc, (ip, bad_col, dat), Y, 1, 3, N=3)
    assert status == rsc.RSC_ERR_INVALID_ARG and np.all(np.isfinite(got))
    bad_ptr = ip.copy()
    bad_ptr[2] = 5    # indptr beyond nnz
    got, status = gpu_epochs(rsc, (bad_ptr, ind, dat), Y, 1, 3, N=3)
    assert status == rsc.RSC_ERR_INVALID_ARG and np.all(np.isfinite(got))


def _preservation(layout, ip, ind, k=10):
    spatial = pytest.importorskip("scipy.spatial")
    _, nn = spatial.cKDTree(layout).query(layout, k + 1)
    hits = 0
    for i in range(len(layout)):
        row = ind[ip[i]:ip[i + 1]]
        hits += len(np.intersect1d(row, nn[i, 1:]))
    return hits / (k * len(layout))


def test_whole_layout_matches_oracle_run(rsc):
    X = synth.mixture(2000, 50, n_comp=6, seed=33)
    graph = oracle_graph(X, 15)
    Y = synth.positions(2000, 2, seed=6)
    got, status = gpu_epochs(rsc, graph, Y, 1, 200, N=200, seed=13)
    assert status == rsc.RSC_OK
    ref, _, _ = oracle.umap_epochs(*graph, Y, A, B, n_epochs=200, seed=13)
    pg, po = _preservation(got, graph[0], graph[1]), _preservation(ref, graph[0], graph[1])
    rand = _preservation(Y, graph[0], graph[1])
    assert pg > 0.3 > 5 * rand
    assert abs(pg - po) < 0.03, (pg, po)


@pytest.fixture(scope="module")
def graph1m():
    # 1,000,000 cells, k = 15 (exact lists of an 8-dimensional mixture)
    return kdtree_graph(synth.mixture(1_000_000, 8, n_comp=100, seed=2), 15)


@pytest.mark.parametrize("epoch,state", [(1, "uniform"), (150, "clustered")])
def test_full_size_graph_on_sampled_vertices(rsc, graph1m, epoch, state):
    # the layout the benchmark times: N = 200 epochs, 5 negatives, 2-D
    n = 1_000_000
    graph = graph1m
    Y = synth.positions(n, 2, seed=epoch, clusters=100 if state == "clustered" else 0)
    got, status = gpu_epochs(rsc, graph, Y, epoch, epoch, seed=99)
    assert status == rsc.RSC_OK
    mask = np.zeros(n, bool)
    mask[synth.query_sample(n, 3000, seed=epoch)] = True
    ref, absmove, _ = oracle.umap_epochs(*graph, Y, A, B, n_epochs=200, first=epoch, last=epoch, seed=99, mask=mask)
    assert_epoch_parity(got, Y, ref, absmove, mask=mask)
    np.testing.assert_array_equal(np.isfinite(got), True)


def test_connectivities_graph_is_exactly_symmetric(rsc):
    # the layout's precondition, on the GPU's own graph of a mixture
    X = torch.from_numpy(synth.mixture(20000, 50, n_comp=20, seed=4)).cuda()
    idx, dist = rsc.rsc_knn(X, 15, precision="bf16")
    ip, ind, dat, _, _ = rsc.rsc_connectivities(idx, dist)
    nnz = int(ip[-1])
    ip, ind, dat = ip.cpu().numpy(), ind[:nnz].cpu().numpy(), dat[:nnz].cpu().numpy()
    rows = np.repeat(np.arange(len(ip) - 1), np.diff(ip))
    fwd = rows.astype(np.int64) * len(ip) + ind
    back = ind.astype(np.int64) * len(ip) + rows
    order = np.argsort(fwd)
    pos = np.searchsorted(fwd[order], back)
    assert np.all(fwd[order][pos] == back)
    np.testing.assert_array_equal(dat[order][pos].view(np.uint32), dat.view(np.uint32))
