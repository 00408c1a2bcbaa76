"""Pins for exact kNN (Definition 1, Sec. 2.1.1) and the medoid entry point (Sec. 4.3)."""
import numpy as np

import oracle


def _lib_topk(Q, X, k):
    # library route: exact integer scores, then a lexicographic sort (dist, id)
    s = -(Q.astype(np.int64) @ X.astype(np.int64).T)
    ids = np.empty((Q.shape[0], k), np.uint32)
    for i in range(Q.shape[0]):
        order = np.lexsort((np.arange(X.shape[0]), s[i]))
        ids[i] = order[:k]
    return ids, s


def test_knn_matches_sorted_brute_force_with_ties():
    rng = np.random.default_rng(11)
    X = rng.integers(-3, 4, size=(400, 8)).astype(np.float32)
    X[50] = X[10]          # planted exact duplicates -> exact ties
    X[399] = X[10]
    Q = rng.integers(-3, 4, size=(60, 8)).astype(np.float32)
    Q[0] = X[10]
    ids, dist = oracle.knn_f64(Q, X, 25)
    ref_ids, s = _lib_topk(Q, X, 25)
    assert np.array_equal(ids, ref_ids)
    assert np.array_equal(dist, np.take_along_axis(s, ref_ids.astype(np.int64), 1).astype(np.float64))
    row0 = list(ids[0])
    assert row0.index(10) < row0.index(50) < row0.index(399)


def test_knn_k_equals_n_is_a_full_sort():
    rng = np.random.default_rng(12)
    X = rng.integers(-2, 3, size=(30, 4)).astype(np.float32)
    Q = rng.integers(-2, 3, size=(5, 4)).astype(np.float32)
    ids, _ = oracle.knn_f64(Q, X, 30)
    ref_ids, _ = _lib_topk(Q, X, 30)
    assert np.array_equal(ids, ref_ids)
    assert all(sorted(r) == list(range(30)) for r in ids.tolist())


def test_medoid_closed_form():
    rng = np.random.default_rng(13)
    X = rng.integers(-5, 6, size=(300, 6)).astype(np.float32)
    mu = X.astype(np.float64).mean(axis=0)
    d2 = ((X.astype(np.float64) - mu) ** 2).sum(axis=1)
    assert oracle.medoid(X) == int(np.argmin(d2))
    # a point placed at the exact mean of a symmetric set is the medoid
    Y = np.array([[1, 0], [-1, 0], [0, 1], [0, -1], [0, 0]], np.float32)
    assert oracle.medoid(Y) == 4
