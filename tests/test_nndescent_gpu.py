"""GPU parity of rsc_knn_descent (NN-descent) against the oracle, through the C ABI.

Both sides take every decision on the same FP32 squared distances (t-ordered
fused multiply-adds) and the same integer hashing, so the lists must agree
bit for bit: ids, distances (sqrtf of the same squared distance) and the
per-iteration change counts.  At full size, where the oracle cannot run the
iterations, the sampled rows are checked against the oracle's exact distances
and exact neighbours.
"""
import numpy as np
import pytest

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


def run_both(rsc, X, k, S=0, R=32, C=64, T=4, delta=0.0, seed=0, init=None):
    dev = torch.device("cuda")
    gi, gd, gch = rsc.rsc_knn_descent(torch.from_numpy(X).to(dev), k, sample=S, rev_slots=R, cand_slots=C,
                                      max_iters=T, delta=delta, seed=seed, with_changes=True,
                                      init=None if init is None else torch.from_numpy(init).to(dev))
    torch.cuda.synchronize()
    oi, od2, och, run = oracle.nndescent(X, k, sample=S or k, rev_slots=R, cand_slots=C, iters=T, delta=delta,
                                         seed=seed, init=init)
    return gi.cpu().numpy(), gd.cpu().numpy(), gch.cpu().numpy(), oi, od2, och, run


def assert_same(gi, gd, gch, oi, od2, och, T):
    assert np.array_equal(gi, oi), f"ids differ in {(gi != oi).any(1).sum()} rows"
    want = np.sqrt(od2.astype(np.float32))
    assert np.array_equal(gd.view(np.uint32), want.view(np.uint32))
    assert list(gch[:T]) == list(och[:T])
    assert (gch[T:] == 0).all()


@pytest.mark.parametrize("n,d,k,S,R,C,T,seed", [
    (500, 50, 15, 0, 32, 64, 1, 0),
    (500, 50, 15, 0, 32, 64, 5, 1),
    (1999, 50, 15, 8, 16, 32, 6, 2),     # ragged n, smaller samples and slots
    (3001, 20, 30, 0, 64, 64, 4, 3),     # k = 30, entries beyond one warp of ids
    (1000, 7, 64, 20, 8, 16, 3, 4),      # k = 64 (two entries per lane), heavy collisions
    (800, 3, 2, 1, 1, 1, 5, 5),          # one reverse and one candidate slot
    (300, 64, 10, 10, 64, 64, 8, 6),     # d = 64
    (257, 1, 5, 3, 4, 8, 6, 7),          # d = 1: many equal distances, ties by id
    (1500, 100, 20, 0, 32, 64, 3, 8),    # d = 100: rows beyond one tensor-core K block (the join is FP32 SIMT)
])
def test_iterations_bit_exact(rsc, n, d, k, S, R, C, T, seed):
    X = synth.mixture(n, d, n_comp=7, seed=seed) if d > 1 else \
        np.random.default_rng(seed).integers(0, 40, (n, 1)).astype(np.float32)
    assert_same(*run_both(rsc, X, k, S, R, C, T, seed=seed)[:6], T)


def test_k_equals_n_and_tiny_sets(rsc):
    rng = np.random.default_rng(11)
    for n, k in ((2, 2), (5, 5), (17, 17), (40, 33)):
        X = rng.normal(0, 1, (n, 6)).astype(np.float32)
        assert_same(*run_both(rsc, X, k, T=3, seed=n)[:6], 3)


def test_caller_lists(rsc):
    """Seeded caller lists with out-of-range ids, repeats and the row itself."""
    X = synth.mixture(3000, 24, n_comp=12, seed=14)
    n, k = len(X), 12
    rng = np.random.default_rng(15)
    init = rng.integers(-50, n + 50, (n, k)).astype(np.int32)
    init[::7, 3] = init[::7, 2]
    init[::5, 0] = np.arange(0, n, 5)
    for T in (1, 2, 4):
        assert_same(*run_both(rsc, X, k, T=T, seed=6, init=init)[:6], T)


def test_duplicate_points(rsc):
    rng = np.random.default_rng(12)
    P = rng.normal(0, 1, (400, 9)).astype(np.float32)
    X = np.concatenate([P, P, P[:100]])
    assert_same(*run_both(rsc, X, 12, T=6, seed=3)[:6], 6)


def test_early_stop_matches(rsc):
    X = synth.mixture(4000, 30, n_comp=15, seed=8)
    k, delta = 10, 0.01
    gi, gd, gch, oi, od2, och, run = run_both(rsc, X, k, T=30, delta=delta, seed=2)
    assert 1 <= run < 30
    assert_same(gi, gd, gch, oi, od2, och, 30)
    lim = delta * len(X) * k
    assert gch[run - 1] < lim and (gch[:run - 1] >= lim).all()


def test_pair_counts(rsc):
    """The join's pair counters equal the oracle's count of joined pairs."""
    X = synth.mixture(2500, 16, n_comp=9, seed=16)
    k, T = 12, 5
    Xd = torch.from_numpy(X).cuda()
    o = rsc.nnd_opts(max_iters=T, seed=7)
    ws = torch.empty(rsc.rsc_knn_descent_workspace_size(len(X), 16, k, o), dtype=torch.uint8, device="cuda")
    rsc.rsc_knn_descent(Xd, k, max_iters=T, seed=7, workspace=ws)
    got = rsc.rsc_knn_descent_pairs(ws)
    _, _, _, _, want = oracle.nndescent(X, k, iters=T, seed=7, with_pairs=True)
    assert list(got[:T]) == list(want) and (got[T:] == 0).all()


def test_runs_are_identical(rsc):
    X = synth.mixture(20000, 50, n_comp=40, seed=9)
    Xd = torch.from_numpy(X).cuda()
    a = rsc.rsc_knn_descent(Xd, 15, max_iters=6, seed=4)
    b = rsc.rsc_knn_descent(Xd, 15, max_iters=6, seed=4)
    c = rsc.rsc_knn_descent(Xd, 15, max_iters=6, seed=5)
    torch.cuda.synchronize()
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    assert not torch.equal(a[0], c[0])


def test_bad_arguments(rsc):
    X = torch.zeros((10, 4), dtype=torch.float32, device="cuda")
    for kw in ({"k": 11}, {"k": 1}, {"k": 4, "sample": 5}, {"k": 4, "rev_slots": 3}, {"k": 4, "cand_slots": 128},
               {"k": 4, "max_iters": 65}, {"k": 4, "delta": -1.0}):
        k = kw.pop("k")
        with pytest.raises(rsc.RscError) as e:
            rsc.rsc_knn_descent(X, k, **kw)
        assert e.value.status == rsc.RSC_ERR_INVALID_ARG


def test_full_size_workload_on_sampled_rows(rsc):
    """The bench's 1M-cell workload and launch configuration: sampled rows'
    distances against the oracle's FP64 distances of the returned ids, list
    order, and recall against the oracle's exact neighbours."""
    n, k = 1_000_000, 15
    X = synth.mixture(n, 50, n_comp=100, seed=0)
    idx, dist = rsc.rsc_knn_descent(torch.from_numpy(X).cuda(), k, max_iters=8, delta=0.001, seed=0)
    torch.cuda.synchronize()
    gi, gd = idx.cpu().numpy(), dist.cpu().numpy()
    q = synth.query_sample(n, 400, seed=5)
    Xq = X[q].astype(np.float64)
    for r, u in enumerate(q):
        row = gi[u]
        assert len(set(row.tolist())) == k and u in row
        ex = np.sqrt(((X[row].astype(np.float64) - Xq[r]) ** 2).sum(1))
        assert np.allclose(gd[u], ex, rtol=2e-6, atol=1e-6)
        keys = list(zip(gd[u].tolist(), row.tolist()))
        assert keys == sorted(keys)
    want, _, _ = oracle.knn(X, k, queries=q)
    recall = np.mean([len(set(gi[u]) & set(want[r])) / k for r, u in enumerate(q)])
    assert recall >= 0.85, recall

