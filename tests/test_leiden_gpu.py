"""GPU parity of rsc_leiden against the oracle's Leiden, through the C ABI.

Both sides take every decision on the same fixed-point weights with exact
integer gains, so the partitions must be identical: the same membership
(numbered by first appearance), the same community count, and the same
modularity (up to the last bits of its final floating-point sum).  Graphs come
from the oracle (its kNN and connectivities of seeded mixtures, or a k-d tree
for the 1M-cell graph) or are built by hand.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.csgraph  # noqa: F401

import oracle
from paper_2603_02402_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rsc():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2603_02402_gb300 import rsc as r
    r.lib()
    return r


def csr(rows, cols, vals, n):
    A = sp.csr_matrix((np.asarray(vals, dtype=np.float32), (rows, cols)), shape=(n, n))
    A.sum_duplicates()
    A.sort_indices()
    return A.indptr.astype(np.int64), A.indices.astype(np.int32), A.data.astype(np.float32)


def knn_graph(n, d, comps, seed, k=15):
    X = synth.mixture(n, d, n_comp=comps, seed=seed)
    i, dist, _ = oracle.knn(X, k)
    g = oracle.connectivities(i.astype(np.int32), dist)
    return g["indptr"].astype(np.int64), g["indices"].astype(np.int32), g["data"].astype(np.float32)


def run_both(rsc, graph, init=None, **kw):
    ip, ind, dat = graph
    dev = torch.device("cuda")
    mem, K, Q = rsc.rsc_leiden(torch.from_numpy(ip).to(dev), torch.from_numpy(ind).to(dev),
                               torch.from_numpy(dat).to(dev),
                               init=None if init is None else torch.from_numpy(init).to(dev), **kw)
    okw = {"resolution": kw.get("resolution", 1.0), "n_iter": kw.get("n_iterations", 2),
           "max_levels": kw.get("max_levels", 32), "max_rounds": kw.get("max_rounds", 8)}
    om, oK, oQ, _ = oracle.leiden(ip, ind, dat, init=init, **okw)
    return mem.cpu().numpy(), K, Q, om, oK, oQ


def assert_same(gm, gK, gQ, om, oK, oQ):
    assert gK == oK
    assert np.array_equal(gm, om), f"{(gm != om).sum()} vertices differ"
    assert gQ == pytest.approx(oQ, rel=1e-12, abs=1e-15)


def ring_of_cliques(n_cliques, size, weight=1.0):
    rows, cols = [], []
    n = n_cliques * size
    for c in range(n_cliques):
        m = range(size * c, size * c + size)
        for a in m:
            for b in m:
                if a != b:
                    rows.append(a)
                    cols.append(b)
        a, b = size * c + size - 1, (size * c + size) % n
        rows += [a, b]
        cols += [b, a]
    return csr(rows, cols, np.full(len(rows), weight), n)


@pytest.mark.parametrize("n,d,comps,seed", [(3000, 50, 20, 0), (6000, 10, 8, 1), (10000, 50, 60, 2)])
def test_knn_graphs_match_oracle(rsc, n, d, comps, seed):
    r = run_both(rsc, knn_graph(n, d, comps, seed))
    assert_same(*r)
    assert r[1] > 1


def test_cosine_k30_graph(rsc):
    """The oracle's cosine kNN (k = 30) and connectivities of a 5,000-cell mixture."""
    X = synth.mixture(5000, 40, n_comp=25, seed=12)
    i, dist, _ = oracle.knn(X, 30, metric=oracle.COSINE)
    g = oracle.connectivities(i.astype(np.int32), dist)
    graph = (g["indptr"].astype(np.int64), g["indices"].astype(np.int32), g["data"].astype(np.float32))
    assert_same(*run_both(rsc, graph))


@pytest.mark.parametrize("gamma", [0.1, 0.3, 2.5, 7.0])
def test_resolutions(rsc, gamma):
    assert_same(*run_both(rsc, knn_graph(3000, 20, 12, 4), resolution=gamma))
    assert_same(*run_both(rsc, ring_of_cliques(16, 5), resolution=gamma))


def test_iterations_levels_rounds(rsc):
    g = knn_graph(4000, 30, 15, 5)
    for kw in ({"n_iterations": 1}, {"n_iterations": 3}, {"max_levels": 1}, {"max_rounds": 2},
               {"max_rounds": 1, "n_iterations": 1}, {"max_rounds": 16}, {"max_rounds": 64}):
        assert_same(*run_both(rsc, g, **kw))


def test_starting_partition(rsc):
    g = knn_graph(3000, 20, 10, 6)
    rng = np.random.default_rng(7)
    for init in (rng.integers(0, 3000, 3000).astype(np.int32), np.zeros(3000, dtype=np.int32),
                 (np.arange(3000) // 300).astype(np.int32)):
        assert_same(*run_both(rsc, g, init=init))


def test_small_and_degenerate_graphs(rsc):
    assert_same(*run_both(rsc, ring_of_cliques(16, 5)))
    # cliques of uneven sizes, a hub joining four cliques, self-loops, zero weights
    rows, cols, vals, off = [], [], [], 0
    for s in (4, 7, 3, 12):
        for a in range(off, off + s):
            for b in range(off, off + s):
                if a != b:
                    rows.append(a)
                    cols.append(b)
                    vals.append(0.5 + 0.01 * ((a * 7 + b * 3) % 11))
        off += s
    hub = off
    for start in (0, 4, 11, 14):
        rows += [hub, start]
        cols += [start, hub]
        vals += [0.3, 0.3]
    rows += [1, 5, 5]
    cols += [1, 5, 6]
    vals += [2.0, 0.0, 0.0]   # self-loops and zero weights (6 -> 5 stays absent)
    g = csr(rows, cols, vals, hub + 1)
    assert_same(*run_both(rsc, g))
    # no edges; one vertex; two vertices joined by one edge
    assert_same(*run_both(rsc, (np.zeros(6, np.int64), np.zeros(0, np.int32), np.zeros(0, np.float32))))
    assert_same(*run_both(rsc, (np.zeros(2, np.int64), np.zeros(0, np.int32), np.zeros(0, np.float32))))
    assert_same(*run_both(rsc, csr([0, 1], [1, 0], [1.0, 1.0], 2)))


def test_bad_graphs_are_refused(rsc):
    dev = torch.device("cuda")
    ip = torch.tensor([0, 1, 2], dtype=torch.int64, device=dev)
    data = torch.ones(2, dtype=torch.float32, device=dev)
    with pytest.raises(rsc.RscError) as e:
        rsc.rsc_leiden(ip, torch.tensor([1, 5], dtype=torch.int32, device=dev), data)
    assert e.value.status == rsc.RSC_ERR_INVALID_ARG
    with pytest.raises(rsc.RscError) as e:
        rsc.rsc_leiden(torch.tensor([0, 2, 1], dtype=torch.int64, device=dev),
                       torch.tensor([1, 0], dtype=torch.int32, device=dev), data)
    assert e.value.status == rsc.RSC_ERR_INVALID_ARG
    with pytest.raises(rsc.RscError) as e:
        rsc.rsc_leiden(ip, torch.tensor([1, 0], dtype=torch.int32, device=dev), data,
                       init=torch.tensor([0, 7], dtype=torch.int32, device=dev))
    assert e.value.status == rsc.RSC_ERR_INVALID_ARG
    # the library still works after a refusal
    mem, K, _ = rsc.rsc_leiden(ip, torch.tensor([1, 0], dtype=torch.int32, device=dev), data)
    assert K == 1


def test_runs_are_identical(rsc):
    ip, ind, dat = knn_graph(20000, 50, 40, 8)
    dev = torch.device("cuda")
    args = (torch.from_numpy(ip).to(dev), torch.from_numpy(ind).to(dev), torch.from_numpy(dat).to(dev))
    a = rsc.rsc_leiden(*args)
    b = rsc.rsc_leiden(*args)
    assert torch.equal(a[0], b[0]) and a[1:] == b[1:]


def test_graph_of_200k_cells_matches_oracle(rsc):
    """A 200,000-cell graph (exact lists of an 8-dimensional mixture from a k-d
    tree, the oracle's connectivities): the whole partition."""
    spatial = pytest.importorskip("scipy.spatial")
    X = synth.mixture(200_000, 8, n_comp=60, seed=9)
    dist, idx = spatial.cKDTree(X.astype(np.float64)).query(X.astype(np.float64), 15, workers=-1)
    g = oracle.connectivities(idx.astype(np.int32), dist.astype(np.float32).astype(np.float64))
    graph = (g["indptr"].astype(np.int64), g["indices"].astype(np.int32), g["data"].astype(np.float32))
    assert_same(*run_both(rsc, graph))


def test_full_size_graph_properties(rsc):
    """The bench's 1M-cell graph size (exact lists of an 8-dimensional mixture):
    the returned modularity equals an independent computation from the
    membership, and every community is connected."""
    spatial = pytest.importorskip("scipy.spatial")
    n = 1_000_000
    X = synth.mixture(n, 8, n_comp=100, seed=2)
    dist, idx = spatial.cKDTree(X.astype(np.float64)).query(X.astype(np.float64), 15, workers=-1)
    g = oracle.connectivities(idx.astype(np.int32), dist.astype(np.float32).astype(np.float64))
    ip, ind, dat = g["indptr"].astype(np.int64), g["indices"].astype(np.int32), g["data"].astype(np.float32)
    dev = torch.device("cuda")
    mem, K, Q = rsc.rsc_leiden(torch.from_numpy(ip).to(dev), torch.from_numpy(ind).to(dev),
                               torch.from_numpy(dat).to(dev))
    m = mem.cpu().numpy()
    assert m.min() == 0 and m.max() == K - 1
    first = np.full(K, n)
    np.minimum.at(first, m, np.arange(n))
    assert (np.diff(first) > 0).all()   # numbered by first appearance
    W = np.rint(dat.astype(np.float64) * 2.0 ** 32)
    rows = np.repeat(np.arange(n), np.diff(ip))
    M = W.sum()
    tot = np.bincount(m, weights=np.bincount(rows, weights=W, minlength=n), minlength=K)
    inside = np.bincount(m[rows], weights=np.where(m[rows] == m[ind], W, 0.0), minlength=K)
    q = (inside / M - (tot / M) ** 2).sum()
    assert Q == pytest.approx(q, abs=1e-9)
    assert Q > 0.9
    # connected communities: dropping the edges between communities leaves K components
    keep = m[rows] == m[ind]
    A = sp.csr_matrix((np.ones(keep.sum()), (rows[keep], ind[keep])), shape=(n, n))
    ncomp, lab = sp.csgraph.connected_components(A, directed=False)
    assert ncomp == K
