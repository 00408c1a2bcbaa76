"""Pins for Alg. 3 AcquireNeighbors (Sec. 4.2.3)."""
import numpy as np
import pytest

import oracle
from conftest import load_golden


def _angles_to_X(deg):
    r = np.deg2rad(np.asarray(deg, np.float64))
    X = np.zeros((len(deg), 4), np.float32)
    X[:, 0] = np.cos(r)
    X[:, 1] = np.sin(r)
    return X


def test_hand_case():
    g = load_golden("acquire_angles.json")
    X = _angles_to_X(g["angles"])
    for c in g["cases"]:
        res = oracle.acquire_neighbors(X, 0, [1, 2, 3, 4], c["M"], c["fill"])
        assert res.tolist() == c["res"], c


def _d(X, a, b):
    return -float(np.dot(X[a].astype(np.float64), X[b].astype(np.float64)))


@pytest.mark.parametrize("seed", range(12))
def test_rng_property_verifier(seed):
    """Checks the result against what Alg. 3 guarantees, without re-running it."""
    rng = np.random.default_rng(seed)
    n, d = 120, 16
    X = rng.standard_normal((n, d)).astype(np.float32)
    X /= np.linalg.norm(X, axis=1, keepdims=True)
    x = 0
    cand = np.arange(1, n)
    dx = np.array([_d(X, x, c) for c in cand])
    cand = cand[np.lexsort((cand, dx))]
    M = int(rng.integers(2, 24))
    res = oracle.acquire_neighbors(X, x, cand, M, fill=False).tolist()
    eps = 1e-9
    assert 1 <= len(res) <= M
    assert res[0] == cand[0]
    pos = {int(c): i for i, c in enumerate(cand)}
    assert [pos[r] for r in res] == sorted(pos[r] for r in res)      # a subsequence of C
    for i in range(1, len(res)):                                     # kept edges obey the rule
        for j in range(i):
            assert _d(X, x, res[i]) < _d(X, res[i], res[j]) + eps
    stop = pos[res[-1]] if len(res) == M else len(cand) - 1
    kept = set(res)
    for c in cand[:stop + 1]:                                         # dropped ones are dominated
        c = int(c)
        if c in kept:
            continue
        earlier = [p for p in res if pos[p] < pos[c]]
        assert any(_d(X, x, c) >= _d(X, c, p) - eps for p in earlier)
    full = oracle.acquire_neighbors(X, x, cand, M, fill=True).tolist()
    assert full[:len(res)] == res
    rest = [int(c) for c in cand if int(c) not in kept]
    assert full[len(res):] == rest[:M - len(res)]
    assert len(full) == min(M, len(cand))


def test_skips_self_and_duplicates():
    X = _angles_to_X([0, 10, 20, 30, -40])
    res = oracle.acquire_neighbors(X, 0, [0, 1, 1, 2, 3, 4], 4, fill=True)
    assert res.tolist() == [1, 4, 2, 3]
    assert oracle.acquire_neighbors(X, 0, [], 4, fill=True).tolist() == []
