"""Deletion by tombstones (Sec. 5.7) on the GPU against the oracle: deleted rows
route but are not answers; ids, visits and hops bit-exact."""
import numpy as np
import pytest

import oracle
from gpu_util import assert_same, dev_index, run

pytestmark = pytest.mark.gpu
MV = 16384


def _tomb_dev(words):
    import torch

    return torch.from_numpy(words.view(np.int32)).to("cuda:0")


def _deleted(n, frac, seed):
    return np.random.default_rng(seed).random(n) < frac


@pytest.mark.parametrize("L,tw", [(50, 1), (400, 1), (100, 4)])   # staged, register and team paths
def test_fp32_tombstones_match_oracle(tiny, L, tw):
    X, adj, entry = tiny["X"], tiny["adj"], tiny["entry"]
    words = oracle.pack_tombstones(_deleted(X.shape[0], 0.25, L + tw))
    idx = dev_index(X, adj, entry, max_visits=MV)
    idx.set_tuning(L, tw, 0, 0)
    idx.set_tombstones(_tomb_dev(words))
    Q = tiny["Q"][:300]
    ref = oracle.beam_search(X, adj, entry, Q, 10, L, max_visits=MV, tomb=words)
    assert_same(run(idx, Q, 10, L), ref, f"L={L} tw={tw}")
    # clearing the tombstones restores the plain answers
    idx.set_tombstones(None)
    assert_same(run(idx, Q, 10, L), oracle.beam_search(X, adj, entry, Q, 10, L, max_visits=MV), "cleared")
    idx.close()


@pytest.mark.parametrize("dtype", ["bf16", "fp8"])
def test_quantized_tombstones_match_oracle(tiny, dtype):
    X, adj, entry = tiny["X"], tiny["adj"], tiny["entry"]
    if dtype == "bf16":
        codes, sc = oracle.quant_bf16(X), None
    else:
        codes, sc = oracle.quant_e4m3(X)
    words = oracle.pack_tombstones(_deleted(X.shape[0], 0.3, 11))
    idx = dev_index(X, adj, entry, dtype=dtype, trav=codes.view(np.int16) if dtype == "bf16" else codes,
                    scales=sc, max_visits=MV)
    idx.set_tombstones(_tomb_dev(words))
    Q = tiny["Q"][:300]
    ref = oracle.beam_search(X, adj, entry, Q, 10, 100, max_visits=MV, dtype=dtype, Xt=codes, scales=sc,
                             tomb=words)
    assert_same(run(idx, Q, 10, 100), ref, dtype)
    idx.close()


def test_everything_deleted_returns_padding(tiny):
    X, adj, entry = tiny["X"], tiny["adj"], tiny["entry"]
    words = oracle.pack_tombstones(np.ones(X.shape[0], dtype=bool))
    idx = dev_index(X, adj, entry, max_visits=MV)
    idx.set_tombstones(_tomb_dev(words))
    Q = tiny["Q"][:40]
    got = run(idx, Q, 10, 60)
    ref = oracle.beam_search(X, adj, entry, Q, 10, 60, max_visits=MV, tomb=words)
    assert_same(got, ref, "all deleted")
    assert np.all(got[0] == 0xFFFFFFFF)
    idx.close()
