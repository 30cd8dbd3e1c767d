"""Pins of the oracle's Leiden communities (CPU).

The oracle follows the synchronous Leiden stated above oracle_leiden (Traag,
Waltman & van Eck 2019; the paper clusters the stored graph with Leiden,
Methods, "Dimensionality reduction and graph analysis").  What pins it to
something other than itself:

* its modularity against networkx's modularity of the same partition;
* graphs whose best partition is known: a ring of cliques, disjoint cliques,
  a graph without edges, one vertex;
* networkx's Louvain on kNN graphs of mixtures: the same modularity within
  0.005, and a similar partition (adjusted Rand index);
* the paper's guarantee of well-connected communities: each community
  induces a connected subgraph;
* resolution: more communities as gamma grows; a starting partition.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from paper_2603_02402_gb300 import synth

nx = pytest.importorskip("networkx")


def csr(rows, cols, vals, n):
    A = sp.csr_matrix((np.asarray(vals, dtype=np.float32), (rows, cols)), shape=(n, n))
    A.sum_duplicates()
    A.sort_indices()
    return A


def ring_of_cliques(n_cliques, size):
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
    return csr(rows, cols, np.ones(len(rows)), n)


def knn_graph(n, d, comps, seed, k=15):
    X = synth.mixture(n, d, n_comp=comps, seed=seed)
    i, dist, _ = oracle.knn(X, k)
    g = oracle.connectivities(i.astype(np.int32), dist)
    return sp.csr_matrix((g["data"].astype(np.float32), g["indices"], g["indptr"]), shape=(n, n))


def fixed_point(A):
    """The oracle's fixed-point weights (w * 2^32 rounded) as floats: the graph
    whose modularity it computes."""
    B = A.copy().astype(np.float64)
    B.data = np.rint(A.data.astype(np.float64) * 2.0 ** 32) / 2.0 ** 32
    return B


def nx_modularity(A, mem, gamma=1.0):
    G = nx.from_scipy_sparse_array(fixed_point(A))
    comms = [set(np.flatnonzero(mem == c).tolist()) for c in range(mem.max() + 1)]
    return nx.community.modularity(G, comms, weight="weight", resolution=gamma), G, comms


def ari(a, b):
    from scipy.special import comb
    ct = {}
    for x, y in zip(a, b):
        ct[(x, y)] = ct.get((x, y), 0) + 1
    sa = np.bincount(a)
    sb = np.bincount(b)
    idx = sum(comb(v, 2) for v in ct.values())
    ea = sum(comb(v, 2) for v in sa)
    eb = sum(comb(v, 2) for v in sb)
    tot = comb(len(a), 2)
    exp = ea * eb / tot
    return (idx - exp) / (0.5 * (ea + eb) - exp)


def run(A, **kw):
    return oracle.leiden(A.indptr, A.indices, A.data, **kw)


def test_ring_of_cliques_and_disjoint_cliques():
    A = ring_of_cliques(16, 5)
    mem, K, Q, _ = run(A)
    assert K == 16
    assert (mem == np.repeat(np.arange(16), 5)).all()
    q, _, _ = nx_modularity(A, mem)
    assert Q == pytest.approx(q, abs=1e-12)
    # three disjoint cliques of different sizes
    rows, cols, off = [], [], 0
    for s in (4, 7, 3):
        for a in range(off, off + s):
            for b in range(off, off + s):
                if a != b:
                    rows.append(a)
                    cols.append(b)
        off += s
    mem, K, _, _ = run(csr(rows, cols, np.ones(len(rows)), off))
    assert K == 3 and list(mem) == [0] * 4 + [1] * 7 + [2] * 3


def test_no_edges_and_one_vertex():
    A = sp.csr_matrix((5, 5), dtype=np.float32)
    mem, K, Q, _ = run(A)
    assert K == 5 and list(mem) == [0, 1, 2, 3, 4] and Q == 0.0
    mem, K, _, _ = run(sp.csr_matrix((1, 1), dtype=np.float32))
    assert K == 1 and list(mem) == [0]


@pytest.mark.parametrize("n,d,comps,seed", [(3000, 50, 20, 0), (4000, 10, 8, 1)])
def test_matches_louvain_quality_on_knn_graphs(n, d, comps, seed):
    A = knn_graph(n, d, comps, seed)
    mem, K, Q, levels = run(A)
    q, G, comms = nx_modularity(A, mem)
    assert Q == pytest.approx(q, abs=1e-9)
    lc = nx.community.louvain_communities(G, weight="weight", seed=0)
    ql = nx.community.modularity(G, lc, weight="weight")
    assert Q >= ql - 0.005, (Q, ql)
    lab = np.empty(n, dtype=np.int64)
    for c, s in enumerate(lc):
        lab[list(s)] = c
    assert ari(mem, lab) > 0.6
    # well-connected communities: each one is connected
    assert all(nx.is_connected(G.subgraph(c)) for c in comms)
    assert levels >= 1


def test_resolution_and_starting_partition():
    R = ring_of_cliques(16, 5)
    assert run(R, resolution=0.1)[1] == 8 and run(R, resolution=1.0)[1] == 16   # pairs of cliques, then cliques
    A = knn_graph(2500, 20, 10, 3)
    counts = [run(A, resolution=g)[1] for g in (1.0, 3.0)]
    assert counts[0] < counts[1], counts
    mem, K, Q, _ = run(A)
    q3, _, _ = nx_modularity(A, run(A, resolution=3.0)[0], gamma=3.0)
    assert run(A, resolution=3.0)[2] == pytest.approx(q3, abs=1e-9)
    # starting from the result and running again keeps the quality
    mem2, K2, Q2, _ = run(A, init=mem, n_iter=1)
    assert Q2 >= Q - 1e-12
    # a bad starting label is refused
    with pytest.raises(ValueError):
        run(A, init=np.full(2500, 2500, dtype=np.int32))


def test_refinement_splits_a_disconnected_community():
    """Two cliques joined only through a hub: Louvain-style moving can leave
    the hub's clique pieces in one community; every community of the result is
    connected, and the cliques are found."""
    rows, cols = [], []
    size = 6
    for c in range(4):
        m = range(size * c, size * c + size)
        for a in m:
            for b in m:
                if a != b:
                    rows.append(a)
                    cols.append(b)
    hub = 4 * size
    for c in range(4):
        rows += [hub, size * c]
        cols += [size * c, hub]
    A = csr(rows, cols, np.ones(len(rows)), hub + 1)
    mem, K, Q, _ = run(A)
    _, G, comms = nx_modularity(A, mem)
    assert all(nx.is_connected(G.subgraph(c)) for c in comms)
    for c in range(4):
        assert len(set(mem[size * c:size * c + size].tolist())) == 1
