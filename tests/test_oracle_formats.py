"""Pins for the oracle's BF16 / FP8-E4M3 conversions against torch's CPU casts."""
import numpy as np
import pytest
import torch

import oracle


def _torch_bf16_bits(a):
    return torch.from_numpy(a).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)


def test_bf16_decode_all_codes():
    codes = np.arange(65536, dtype=np.uint16)
    ref = torch.from_numpy(codes.view(np.int16)).view(torch.bfloat16).float().numpy()
    got = np.array([oracle.bf16_to_f32(int(c)) for c in codes[::97]], np.float32)
    r = ref[::97]
    fin = np.isfinite(r)
    assert np.array_equal(got[fin], r[fin])
    assert np.all(np.isnan(got[np.isnan(r)]))


def test_bf16_encode_matches_torch_rne():
    rng = np.random.default_rng(5)
    a = np.concatenate([
        rng.standard_normal(1 << 20).astype(np.float32),
        (rng.standard_normal(1 << 18) * 1e30).astype(np.float32),
        (rng.standard_normal(1 << 18) * 1e-30).astype(np.float32),
        # exact halfway points: low 16 bits 0x8000 with odd and even kept parts
        (rng.integers(0, 1 << 15, 1 << 16, dtype=np.uint32) << 16 | 0x8000).view(np.float32),
        np.array([0.0, -0.0, np.inf, -np.inf, 3.3895314e38, 1e-45], np.float32),
    ])
    a = a[np.isfinite(a) | np.isinf(a)]
    assert np.array_equal(oracle.f32_to_bf16(a), _torch_bf16_bits(a))


def test_e4m3_decode_all_codes():
    codes = np.arange(256, dtype=np.uint8)
    ref = torch.from_numpy(codes).view(torch.float8_e4m3fn).float().numpy()
    got = np.array([oracle.e4m3_to_f32(int(c)) for c in codes], np.float32)
    fin = np.isfinite(ref)
    assert np.array_equal(got[fin], ref[fin])
    assert np.isnan(got[0x7F]) and np.isnan(got[0xFF])
    assert got[0x7E] == 448.0 and got[0x01] == 2.0 ** -9


def test_e4m3_encode_matches_torch_in_range():
    rng = np.random.default_rng(6)
    vals = torch.arange(256, dtype=torch.uint8).view(torch.float8_e4m3fn).float().numpy()
    vals = vals[np.isfinite(vals)]
    mids = []
    s = np.sort(np.unique(np.abs(vals)))
    mids = ((s[1:].astype(np.float64) + s[:-1]) / 2).astype(np.float32)   # exact ties
    a = np.concatenate([
        rng.uniform(-448, 448, 1 << 20).astype(np.float32),
        (rng.standard_normal(1 << 18) * 0.01).astype(np.float32),
        mids, -mids, s, -s,
        np.array([0.0, -0.0, 2.0 ** -10, 3 * 2.0 ** -11], np.float32),
    ])
    ref = torch.from_numpy(a).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    assert np.array_equal(oracle.f32_to_e4m3(a), ref)


def test_e4m3_saturates():
    a = np.array([448.0, 460.0, 500.0, 1e6, -1e6, np.inf, -np.inf], np.float32)
    got = oracle.f32_to_e4m3(a)
    assert list(got) == [0x7E, 0x7E, 0x7E, 0x7E, 0xFE, 0x7E, 0xFE]


def test_quant_e4m3_rows():
    rng = np.random.default_rng(7)
    X = rng.standard_normal((64, 200)).astype(np.float32)
    X[3] = 0.0
    codes, sc = oracle.quant_e4m3(X)
    maxabs = np.abs(X).max(axis=1)
    expect = np.where(maxabs == 0, np.float32(1.0), maxabs / np.float32(448.0)).astype(np.float32)
    assert np.array_equal(sc, expect)
    # the largest element of each nonzero row lands on +-448
    for r in range(64):
        if r == 3:
            assert np.all(codes[r] == 0)
            continue
        j = int(np.argmax(np.abs(X[r])))
        assert codes[r, j] & 0x7F == 0x7E
    # decoded values times the scale are within half an E4M3 step of x
    dec = torch.from_numpy(codes).view(torch.float8_e4m3fn).float().numpy() * sc[:, None]
    assert np.all(np.abs(dec - X) <= np.maximum(np.abs(X) * 2.0 ** -4, sc[:, None] * 2.0 ** -10) + 1e-12)
