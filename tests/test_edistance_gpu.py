"""GPU parity of rsc_edistance against the oracle's E-distance (through the C ABI).

Inputs come from the seeded generators (mixtures, group sizes, permutations);
the oracle sums the same float32 rows by direct difference in FP64.

Error model of one GPU distance.  The squared distance is an FP32 tensor-core
accumulation of split-BF16 products of rows y = x - c (c the mean of the
kernel's row sample): FP32 rounding of terms as large as |y|^2, and the
split's residuals (the dropped low x low products, the rounding of the low
parts), about 2^-18 |y_i| |y_j| each.  The tolerance takes
e_ij = 2^-16 (|y_i| + |y_j|)^2 per squared distance (measured worst 107 x 2^-24,
so 2.4 x margin), hence |dd_ij| <= min(sqrt(e_ij), e_ij / d_ij).  A pair's sum
may be off by the sum of those bounds over its distances, plus 2^-18 of the
sum for the FP32 partial sums of 64 columns, plus 1e-9.  Means follow from the
sums; E = 2 m_ab - m_aa - m_bb from the three means' bounds.  Large groups
average the errors out (relative differences near 1e-6); the bound is what the
test asserts, and it also reports the ratio used.
"""
import numpy as np
import pytest

import oracle
from paper_2603_02402_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

E_REL = 2.0 ** -16   # squared-distance error per (|y_i| + |y_j|)^2
SUM_REL = 2.0 ** -18  # FP32 partial sums of 64 columns


def centre_of(X, ci, n):
    """The kernel's centre: mean of up to 4096 rows at positions r * n // m."""
    m = min(n, 4096)
    pos = (np.arange(m, dtype=np.int64) * n) // m
    rows = pos if ci is None else ci[pos]
    return X[rows].astype(np.float64).mean(0)


def sum_bounds(X, off, ci, pairs):
    """Bound on |GPU sum - exact sum| for each pair (a, b) (see the module text)."""
    n = int(off[-1])
    c = centre_of(X, ci, n)
    rows = np.arange(n) if ci is None else ci.astype(np.int64)
    Y = X[rows].astype(np.float64)
    ny = np.linalg.norm(Y - c, axis=1)
    out = {}
    for a, b in pairs:
        ia, ib = np.arange(off[a], off[a + 1]), np.arange(off[b], off[b + 1])
        tot = 0.0
        for s0 in range(0, len(ia), 256):
            ra = ia[s0:s0 + 256]
            D = np.sqrt(np.maximum(((Y[ra, None, :] - Y[None, ib, :]) ** 2).sum(-1), 0.0))
            e = E_REL * (ny[ra, None] + ny[None, ib]) ** 2
            bnd = np.minimum(np.sqrt(e), e / np.maximum(D, 1e-300))
            if a == b:
                bnd = np.where(ib[None, :] > ra[:, None], bnd, 0.0)
            tot += bnd.sum()
        out[(a, b)] = tot
    return out


@pytest.fixture(scope="module")
def rsc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_02402_gb300 import rsc as mod
    mod.lib()
    return mod


def groups_of(sizes, n_rows, seed, permute=True):
    rng = np.random.default_rng(seed)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    ci = rng.permutation(n_rows)[:off[-1]].astype(np.int32) if permute else None
    return off, ci


def gpu_ed(rsc, X, off, ci=None, pairs=None):
    Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    cd = None if ci is None else torch.from_numpy(ci).cuda()
    ws = torch.empty(rsc.rsc_edistance_workspace_size(len(X), X.shape[1], off, pairs), dtype=torch.uint8,
                     device="cuda")
    s, m, E = rsc.rsc_edistance(Xd, off, cd, pairs=pairs, workspace=ws)
    status = rsc.rsc_workspace_status(ws)
    return s.cpu().numpy(), m.cpu().numpy(), E.cpu().numpy(), status


def check(sums, mean, E, ref_sums, off, X, ci, pairs=None):
    """Assert sums, means and E against the oracle's sums within the bounds of
    the error model; returns (largest share of a bound used, largest relative
    difference of a sum)."""
    G = len(off) - 1
    want = np.zeros((G, G), bool)
    if pairs is None:
        want[np.triu_indices(G)] = True
    else:
        for a, b in pairs:
            want[a, b] = True
    plist = list(zip(*np.nonzero(want)))
    bnd = sum_bounds(X, off, ci, plist)
    rs = np.where(want, ref_sums, 0.0)
    tol = np.zeros((G, G))
    for (a, b), v in bnd.items():
        tol[a, b] = v + SUM_REL * abs(rs[a, b]) + 1e-9
    err = np.abs(sums - rs)
    assert np.all(err[want] <= tol[want]), f"worst share {np.max(err[want] / tol[want]):.3g}"
    assert np.all(sums[~want] == 0.0)
    n = np.diff(off).astype(np.float64)
    cnt = np.where(np.eye(G, dtype=bool), n[:, None] * (n[:, None] - 1) / 2, n[:, None] * n[None, :])
    with np.errstate(invalid="ignore", divide="ignore"):
        rm = np.where(cnt > 0, rs / cnt, 0.0)
        tm = np.where(cnt > 0, tol / cnt, 0.0)
    rm = np.where(want, rm, np.nan)
    rm = np.where(np.isnan(rm), rm.T, rm)
    tm = np.where(want, tm, tm.T)
    ok_m = ~np.isnan(rm)
    np.testing.assert_array_equal(np.isnan(mean), ~ok_m)
    assert np.all(np.abs(mean[ok_m] - rm[ok_m]) <= tm[ok_m] * (1 + 1e-9) + 1e-12)
    d, td = np.diag(rm), np.diag(tm)
    rE = 2 * rm - d[:, None] - d[None, :]
    tE = 2 * tm + td[:, None] + td[None, :]
    ok = ~np.isnan(rE)
    np.testing.assert_array_equal(np.isnan(E), ~ok)
    assert np.all(np.abs(E[ok] - rE[ok]) <= tE[ok] * (1 + 1e-9) + 1e-12)
    with np.errstate(invalid="ignore", divide="ignore"):
        return float(np.max(err[want] / tol[want])), float(np.nanmax(err[want] / np.maximum(rs[want], 1e-30)))


@pytest.mark.parametrize("sizes,d", [
    ([300, 1, 0, 700, 129, 1000], 50),
    ([128, 128, 256, 1], 50),
    ([1000], 50),
    ([77, 5, 400, 33, 260], 7),
    ([500, 600], 1),
    ([250, 250, 250], 58),
])
def test_all_pairs_match_oracle(rsc, sizes, d):
    n_rows = int(sum(sizes)) + 37
    X = synth.mixture(n_rows, d, n_comp=8, seed=len(sizes) * 10 + d)
    off, ci = groups_of(sizes, n_rows, seed=d)
    sums, mean, E, status = gpu_ed(rsc, X, off, ci)
    assert status == rsc.RSC_OK
    ref = oracle.edistance_sums(X, off, ci)
    share, rel = check(sums, mean, E, ref, off, X, ci)
    print(sizes, d, "bound share", share, "max rel sum err", rel)


def test_rows_of_x_without_cell_index(rsc):
    X = synth.mixture(3000, 50, n_comp=10, seed=4)
    off = np.array([0, 900, 2000, 2500], np.int64)   # the last 500 rows belong to no group
    sums, mean, E, status = gpu_ed(rsc, X, off)
    assert status == rsc.RSC_OK
    check(sums, mean, E, oracle.edistance_sums(X, off), off, X, None)


def test_many_tiny_groups(rsc):
    rng = np.random.default_rng(9)
    sizes = rng.integers(0, 5, 300)
    X = synth.mixture(int(sizes.sum()) + 10, 50, n_comp=30, seed=9)
    off, ci = groups_of(sizes, len(X), seed=9)
    sums, mean, E, status = gpu_ed(rsc, X, off, ci)
    assert status == rsc.RSC_OK
    share, rel = check(sums, mean, E, oracle.edistance_sums(X, off, ci), off, X, ci)
    print("tiny groups: bound share", share, "max rel sum err", rel)


@pytest.mark.parametrize("ref_group", [0, 3, 9])
def test_onesided_pairs(rsc, ref_group):
    from paper_2603_02402_gb300 import rsc as mod
    rng = np.random.default_rng(ref_group)
    sizes = rng.integers(50, 400, 10)
    X = synth.mixture(int(sizes.sum()), 50, n_comp=10, seed=ref_group)
    off, ci = groups_of(sizes, len(X), seed=ref_group)
    pairs = mod.edistance_onesided_pairs(10, ref_group)
    sums, mean, E, status = gpu_ed(rsc, X, off, ci, pairs=pairs)
    assert status == rsc.RSC_OK
    ref = oracle.edistance_sums(X, off, ci, pairs=pairs)
    check(sums, mean, E, np.nan_to_num(ref), off, X, ci, pairs=pairs)
    assert np.all(np.isfinite(E[ref_group])) and np.isnan(E[(ref_group + 1) % 10, (ref_group + 2) % 10])


def test_bad_cell_index_is_recorded(rsc):
    X = synth.mixture(500, 50, n_comp=4, seed=1)
    off = np.array([0, 200, 400], np.int64)
    ci = np.arange(400, dtype=np.int32)
    ci[17] = 5000
    _, _, E, status = gpu_ed(rsc, X, off, ci)
    assert status == rsc.RSC_ERR_INVALID_ARG and np.all(np.isfinite(E))


def test_screen_workload_on_sampled_pairs(rsc):
    # 100,000 cells x 50 PCs in 300 groups of log-uniform sizes (a perturbation
    # screen): every pair on the GPU, 40 sampled pairs from the oracle
    sizes = synth.batched_sizes(300, lo=20, hi=2000, total=100_000, seed=5)
    X = synth.mixture(int(sizes.sum()), 50, n_comp=60, seed=5)
    off, ci = groups_of(sizes, len(X), seed=5)
    sums, mean, E, status = gpu_ed(rsc, X, off, ci)
    assert status == rsc.RSC_OK
    rng = np.random.default_rng(1)
    a = rng.integers(0, 300, 12)
    b = rng.integers(0, 300, 12)
    pairs = np.stack([np.minimum(a, b), np.maximum(a, b)], 1).astype(np.int32)
    pairs = np.concatenate([pairs, np.array([[g, g] for g in np.unique(pairs)[:8]], np.int32)])
    ref = oracle.edistance_sums(X, off, ci, pairs=pairs)
    bnd = sum_bounds(X, off, ci, [tuple(p) for p in pairs])
    worst = 0.0
    for p, q in pairs:
        tol = bnd[(p, q)] + SUM_REL * abs(ref[p, q]) + 1e-9
        assert abs(sums[p, q] - ref[p, q]) <= tol, (p, q)
        worst = max(worst, abs(sums[p, q] - ref[p, q]) / abs(ref[p, q]))
    print("screen: max rel sum err", worst)
