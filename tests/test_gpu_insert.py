"""Insertion through the saved bipartite graph (Sec. 5.7) on the GPU against
the oracle, row for row: graph rows, N_out lists and chosen queries identical.

The GPU inserts in windows of speculative searches and keeps a search only
while the nodes it expanded are unchanged; the result must be the oracle's
one-at-a-time order for every window size (1 is the plain sequential order,
small windows force many re-searches, large ones many kept searches)."""
import functools

import numpy as np
import pytest

import oracle
import roarsynth as rs

pytestmark = pytest.mark.gpu
NONE = 0xFFFFFFFF
CASES = [(3000, 2700, 16, 64), (2500, 2400, 8, 40), (8000, 5000, 16, 64)]


@functools.lru_cache(maxsize=None)
def _case(n, n_old, M, L):
    w = rs.scaled(rs.TINY, n=n, n_train=n, n_test=10)
    X = rs.base(w)
    T = rs.train_queries(w)
    nq = 32
    knn, _ = oracle.knn_f64(T, X[:n_old], nq)
    entry = oracle.medoid(X[:n_old])
    adj0, _, _ = oracle.build_index(X[:n_old], knn, M, L, entry)
    R = adj0.shape[1]
    adj = np.full((n, R), NONE, dtype=np.uint32)
    adj[:n_old] = adj0
    cap = nq + 48
    nout = np.full((T.shape[0], cap), NONE, dtype=np.uint32)
    nout[:, :nq - 1] = knn[:, 1:]
    cnt = np.full(T.shape[0], nq - 1, dtype=np.int32)
    ref = oracle.insert(X, adj, entry, n_old, T, knn[:, 0], nout.copy(), cnt.copy(), M, L, max_visits=16384)
    return X, T, knn, entry, adj, nout, cnt, ref


@pytest.mark.parametrize("window", [1, 7, 64, 256])
@pytest.mark.parametrize("n,n_old,M,L", CASES)
def test_insert_matches_oracle(n, n_old, M, L, window):
    import torch

    import paper_2408_08933_gb300 as pkg

    X, T, knn, entry, adj, nout, cnt, (r_adj, r_nout, r_cnt, r_q) = _case(n, n_old, M, L)
    dev = torch.device("cuda:0")
    Xd = torch.from_numpy(X).to(dev)
    Ad = torch.from_numpy(adj.view(np.int32)).to(dev)
    g_nout, g_cnt = nout.copy(), cnt.copy()
    g_q, st = pkg.insert(Xd, Ad, entry, n_old, T, knn[:, 0], g_nout, g_cnt, M, L, window=window,
                         return_stats=True)
    g_adj = Ad.cpu().numpy().view(np.uint32)
    assert np.array_equal(g_q, r_q)
    assert np.array_equal(g_cnt, r_cnt)
    assert np.array_equal(g_nout, r_nout)
    bad = np.nonzero(np.any(g_adj != r_adj, axis=1))[0]
    assert bad.size == 0, f"{bad.size} rows differ, first {bad[:5].tolist()}"
    inserted = n - n_old
    assert st["searches"] >= inserted
    if window == 1:
        assert st["windows"] == inserted and st["searches"] == inserted
    else:
        assert st["windows"] < inserted         # windows did apply several rows at once
