"""The benchmark's recall helpers on the CPU: a returned id counts when its
FP64 distance to the query is within the oracle's k-th distance, so the
oracle's own lists score 1, a list with an equally distant id in place of a
listed one (a tie) scores 1, and every far id costs exactly one entry."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402
import oracle  # noqa: E402
from paper_2603_02402_gb300 import synth  # noqa: E402


def test_exact_distances_match_the_oracle():
    X = synth.mixture(2000, 20, n_comp=6, seed=3)
    X[[5, 9]] = 0.0   # zero rows for the cosine convention
    q = np.array([0, 5, 17, 1999])
    for metric, om in (("euclidean", oracle.EUCLIDEAN), ("cosine", oracle.COSINE)):
        oi, od, _ = oracle.knn(X, 10, metric=om, queries=q)
        np.testing.assert_allclose(bench.exact_distances(X, q, oi, metric), od, rtol=0, atol=1e-12)


def test_recall_counts_ties_and_misses():
    # points on a line: query 0's neighbours at distances 0, 1, 1 (ids 1 and 2 tie), 2, 3
    X = np.array([[0.0], [1.0], [-1.0], [2.0], [3.0], [10.0]], dtype=np.float32)
    q = np.array([0])
    oi, od, _ = oracle.knn(X, 3, queries=q)
    assert oi.tolist() == [[0, 1, 2]]
    kth = od[:, -1]
    assert bench.recall_by_distance(bench.exact_distances(X, q, oi), kth) == 1.0
    tie = np.array([[0, 2, 1]])           # the tied ids in the other order
    assert bench.recall_by_distance(bench.exact_distances(X, q, tie), kth) == 1.0
    one_far = np.array([[0, 1, 5]])       # id 5 at distance 10 is outside
    assert bench.recall_by_distance(bench.exact_distances(X, q, one_far), kth) == 2 / 3
    beyond = np.array([[0, 1, 3]])        # id 3 at distance 2 is beyond the 3rd (1)
    assert bench.recall_by_distance(bench.exact_distances(X, q, beyond), kth) == 2 / 3
