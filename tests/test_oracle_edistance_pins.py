"""Pins for the oracle's E-distance, against things other than itself.

Hand-derived cases (tests/golden/edistance_line.txt), scipy's cdist summed per
group pair, scipy's one-dimensional energy_distance (a V-statistic: its
within-group means include the zero self distances, so they are (n - 1) / n
of the oracle's), the closed form E(X, X) = -2 m / n for two copies of one
point set (m its mean within-group distance), and invariance under rigid
motions.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle

spatial = pytest.importorskip("scipy.spatial")
stats = pytest.importorskip("scipy.stats")


def _golden(path):
    cases, cur = [], None
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        key, *vals = line.split()
        if key == "case":
            cur = {"sum": {}, "E": {}}
            cases.append(cur)
        elif key == "points":
            cur["points"] = np.array([float(v) for v in vals], np.float32)[:, None]
        elif key == "offsets":
            cur["offsets"] = [int(v) for v in vals]
        else:
            a, b, v = int(vals[0]), int(vals[1]), float(Fraction(vals[2]))
            cur[key][(a, b)] = v
    return cases


def test_hand_derived_cases(golden_dir):
    for case in _golden(os.path.join(golden_dir, "edistance_line.txt")):
        sums, mean, E = oracle.edistance(case["points"], case["offsets"])
        for (a, b), v in case["sum"].items():
            assert sums[a, b] == pytest.approx(v, abs=1e-12)
        for (a, b), v in case["E"].items():
            assert E[a, b] == pytest.approx(v, abs=1e-12) and E[b, a] == pytest.approx(v, abs=1e-12)


def _groups(rng, sizes, d, shuffle=True):
    n = int(sum(sizes))
    X = rng.standard_normal((n, d)).astype(np.float32) * 2.0
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    ci = rng.permutation(n).astype(np.int32) if shuffle else None
    return X, off, ci


def test_sums_match_scipy_cdist():
    rng = np.random.default_rng(1)
    sizes = [5, 1, 0, 17, 40, 2]
    X, off, ci = _groups(rng, sizes, 7)
    sums = oracle.edistance_sums(X, off, ci)
    G = len(sizes)
    Xd = X.astype(np.float64)
    for a in range(G):
        for b in range(a, G):
            ra, rb = ci[off[a]:off[a + 1]], ci[off[b]:off[b + 1]]
            if len(ra) == 0 or len(rb) == 0:
                want = 0.0
            else:
                D = spatial.distance.cdist(Xd[ra], Xd[rb])
                want = np.triu(D, 1).sum() if a == b else D.sum()
            assert sums[a, b] == pytest.approx(want, rel=1e-12, abs=1e-12)
    assert np.isnan(sums[1, 0])


def test_one_dimensional_energy_distance_of_scipy():
    rng = np.random.default_rng(2)
    for na, nb in ((30, 45), (2, 9), (100, 3)):
        u = rng.normal(0, 1, na).astype(np.float32)
        v = rng.normal(0.7, 1.5, nb).astype(np.float32)
        X = np.concatenate([u, v])[:, None]
        _, mean, E = oracle.edistance(X, [0, na, na + nb])
        # scipy: sqrt(2 E|U-V| - E|U-U'| - E|V-V'|) with self pairs inside the means
        v_stat = 2 * mean[0, 1] - (na - 1) / na * mean[0, 0] - (nb - 1) / nb * mean[1, 1]
        assert np.sqrt(v_stat) == pytest.approx(stats.energy_distance(u.astype(np.float64), v.astype(np.float64)),
                                                rel=1e-10)
        assert E[0, 1] == pytest.approx(2 * mean[0, 1] - mean[0, 0] - mean[1, 1], rel=1e-14)


def test_two_copies_of_one_set():
    rng = np.random.default_rng(3)
    P = rng.standard_normal((25, 6)).astype(np.float32)
    X = np.concatenate([P, P])
    _, mean, E = oracle.edistance(X, [0, 25, 50])
    m = mean[0, 0]
    assert mean[1, 1] == pytest.approx(m, rel=1e-14)
    assert E[0, 1] == pytest.approx(-2 * m / 25, rel=1e-10)


def test_rigid_motion_invariance_and_pair_subsets():
    rng = np.random.default_rng(4)
    sizes = [12, 30, 7, 21]
    X, off, ci = _groups(rng, sizes, 5)
    q, _ = np.linalg.qr(rng.standard_normal((5, 5)))
    Y = (X.astype(np.float64) @ q + 3.0).astype(np.float32)
    s1 = oracle.edistance_sums(X, off, ci)
    s2 = oracle.edistance_sums(Y, off, ci)
    ok = ~np.isnan(s1)
    np.testing.assert_allclose(s2[ok], s1[ok], rtol=1e-5)   # float32 rounding of the moved points
    pairs = np.array([[0, 0], [0, 2], [1, 3], [3, 3]], np.int32)
    sp = oracle.edistance_sums(X, off, ci, pairs=pairs)
    for a, b in pairs:
        assert sp[a, b] == s1[a, b]
    assert np.isnan(sp[0, 1]) and np.isnan(sp[2, 2])
