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


# Alg. 3 with FP64 distances, and the same steps with FP32 fixed-order
# distances (the precision of the GPU pruning kernel); both obey the pins below.
FORMS = [(oracle.acquire_neighbors, 1e-9), (oracle.acquire_neighbors_f32, 1e-5)]


@pytest.mark.parametrize("acquire,eps", FORMS)
def test_hand_case(acquire, eps):
    g = load_golden("acquire_angles.json")
    X = _angles_to_X(g["angles"])
    for c in g["cases"]:
        res = acquire(X, 0, [1, 2, 3, 4], c["M"], c["fill"])
        assert res.tolist() == c["res"], c


def _d(X, a, b):
    return -float(np.dot(X[a].astype(np.float64), X[b].astype(np.float64)))


@pytest.mark.parametrize("acquire,eps", FORMS)
@pytest.mark.parametrize("seed", range(12))
def test_rng_property_verifier(seed, acquire, eps):
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
    res = acquire(X, x, cand, M, fill=False).tolist()
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
    full = acquire(X, x, cand, M, fill=True).tolist()
    assert full[:len(res)] == res
    rest = [int(c) for c in cand if int(c) not in kept]
    assert full[len(res):] == rest[:M - len(res)]
    assert len(full) == min(M, len(cand))


@pytest.mark.parametrize("acquire,eps", FORMS)
def test_skips_self_and_duplicates(acquire, eps):
    X = _angles_to_X([0, 10, 20, 30, -40])
    res = acquire(X, 0, [0, 1, 1, 2, 3, 4], 4, fill=True)
    assert res.tolist() == [1, 4, 2, 3]
    assert acquire(X, 0, [], 4, fill=True).tolist() == []


def test_f32_form_agrees_with_fp64_when_margins_are_wide():
    """Where no keep / drop comparison is within FP32 rounding, the FP32 and
    FP64 forms must keep the same ids."""
    rng = np.random.default_rng(7)
    same = 0
    for t in range(40):
        n, d = 200, 32
        X = rng.standard_normal((n, d)).astype(np.float32)
        X /= np.linalg.norm(X, axis=1, keepdims=True)
        cand = np.arange(1, n)
        dx = np.array([_d(X, 0, c) for c in cand])
        cand = cand[np.lexsort((cand, dx))]
        a = oracle.acquire_neighbors(X, 0, cand, 16, fill=False).tolist()
        b = oracle.acquire_neighbors_f32(X, 0, cand, 16, fill=False).tolist()
        if a == b:
            same += 1
            continue
        # a difference needs a decisive comparison within FP32 rounding
        margins = [abs(_d(X, 0, c) - _d(X, c, p)) for c in cand for p in set(a) | set(b) if p != c]
        assert min(margins) < 1e-5
    assert same >= 36
