"""Pins for the oracle's fixed-order FP32 dot product (inner-product distance, Sec. 5.1)."""
import numpy as np
import pytest

import oracle
from conftest import load_golden


def test_hand_case_separates_lane_orders():
    g = load_golden("dot_fixed_d8.json")
    q = np.array(g["q"], np.float32)
    x = np.array(g["x"], np.float32)
    assert oracle.dot_fixed(q, x) == np.float32(g["dot_fixed"])
    assert float(np.dot(q.astype(np.float64), x.astype(np.float64))) == g["exact"]


@pytest.mark.parametrize("d", [4, 8, 64, 200, 512, 516])
def test_exact_on_integer_inputs(d):
    # every partial sum is an integer below 2^24, so any order is exact
    rng = np.random.default_rng(d)
    q = rng.integers(-8, 9, size=d).astype(np.float32)
    x = rng.integers(-8, 9, size=d).astype(np.float32)
    exact = int(np.dot(q.astype(np.int64), x.astype(np.int64)))
    assert oracle.dot_fixed(q, x) == np.float32(exact)


@pytest.mark.parametrize("d", [64, 200, 512])
def test_higham_bound(d):
    # |fl(dot) - dot| <= gamma_m * sum |q_i x_i| with m = ceil(d/128)*4 + 5
    rng = np.random.default_rng(1000 + d)
    m = -(-d // 128) * 4 + 5
    u = 2.0 ** -24
    gamma = m * u / (1 - m * u)
    for _ in range(200):
        q = rng.standard_normal(d).astype(np.float32)
        x = rng.standard_normal(d).astype(np.float32)
        ref = float(np.dot(q.astype(np.float64), x.astype(np.float64)))
        bound = gamma * float(np.abs(q.astype(np.float64) * x.astype(np.float64)).sum())
        assert abs(float(oracle.dot_fixed(q, x)) - ref) <= bound


def test_single_nonzero_and_zero():
    d = 200
    for i in (0, 3, 4, 127, 128, 199):
        q = np.zeros(d, np.float32)
        x = np.zeros(d, np.float32)
        q[i], x[i] = 1.5, -2.25
        assert oracle.dot_fixed(q, x) == np.float32(-3.375)
    assert oracle.dot_fixed(np.zeros(8, np.float32), np.ones(8, np.float32)) == 0.0
