"""Insertion through the saved bipartite graph (Sec. 5.7) in the oracle: a
hand-traced case (two insertions, one re-pruning a full row) plus structural
and quality properties on a larger input."""
import numpy as np
import pytest

import oracle
import roarsynth as rs

NONE = 0xFFFFFFFF


@pytest.fixture(scope="module")
def inserted():
    w = rs.scaled(rs.TINY, n=3000, n_train=3000, n_test=200)
    X = rs.base(w)
    T = rs.train_queries(w)
    n_old, M, L, nq = 2700, 16, 64, 32
    knn, _ = oracle.knn_f64(T, X[:n_old], nq)
    entry = oracle.medoid(X[:n_old])
    adj0, _, _ = oracle.build_index(X[:n_old], knn, M, L, entry)
    R = adj0.shape[1]
    adj = np.full((X.shape[0], R), NONE, dtype=np.uint32)
    adj[:n_old] = adj0
    cap = nq + 64
    nout = np.full((T.shape[0], cap), NONE, dtype=np.uint32)
    nout[:, :nq - 1] = knn[:, 1:]
    cnt = np.full(T.shape[0], nq - 1, dtype=np.int32)
    out = oracle.insert(X, adj, entry, n_old, T, knn[:, 0], nout, cnt, M, L, max_visits=16384)
    return dict(X=X, T=T, w=w, n_old=n_old, M=M, L=L, R=R, entry=entry, knn=knn, before=(adj, nout, cnt),
                after=out)


def test_rows_stay_valid(inserted):
    adj, nout, cnt, chosen = inserted["after"]
    n, R, M, n_old = adj.shape[0], inserted["R"], inserted["M"], inserted["n_old"]
    for v in range(n):
        row = [int(u) for u in adj[v] if u != NONE]
        assert len(row) == len(set(row)) and v not in row and all(u < n for u in row)
        assert all(u == NONE for u in adj[v][len(row):])          # padding only at the end
        assert len(row) <= R
        if v >= n_old:
            assert len(row) >= 1       # N(v) (at most M), plus reverse edges of later insertions
    # old rows only gained new ids or were re-pruned to exactly R entries
    adj0 = inserted["before"][0]
    for v in range(n_old):
        old = set(int(u) for u in adj0[v] if u != NONE)
        new = set(int(u) for u in adj[v] if u != NONE)
        assert new - old <= set(range(n_old, n)) and (new >= old or len(new) == R)


def test_bipartite_lists_grow_with_the_chosen_queries(inserted):
    adj, nout, cnt, chosen = inserted["after"]
    _, nout0, cnt0 = inserted["before"]
    n_old = inserted["n_old"]
    grown = cnt - cnt0
    assert grown.sum() == int((chosen >= 0).sum())
    assert (chosen >= 0).mean() > 0.9                                # nearly every row finds a connected query
    for i, q in enumerate(chosen):
        if q >= 0:
            assert n_old + i in nout[q, :cnt[q]].tolist()


def test_inserted_rows_are_found_and_recall_holds(inserted):
    X, w, n_old = inserted["X"], inserted["w"], inserted["n_old"]
    adj = inserted["after"][0]
    entry = inserted["entry"]
    new = np.arange(n_old, X.shape[0])
    ids, *_ = oracle.beam_search(X, adj, entry, X[new], 1, 64)
    assert (ids[:, 0] == new).mean() >= 0.85                          # self-recall of inserted rows
    Q = rs.test_queries(w)
    gt, _ = oracle.knn_f64(Q, X, 10)
    got, *_ = oracle.beam_search(X, adj, entry, Q, 10, 64)
    # the same index rebuilt over all rows, for comparison (Sec. 5.7 compares with a rebuild)
    knn_all, _ = oracle.knn_f64(inserted["T"], X, 32)
    reb, _, _ = oracle.build_index(X, knn_all, inserted["M"], inserted["L"], oracle.medoid(X))
    got_r, *_ = oracle.beam_search(X, reb, oracle.medoid(X), Q, 10, 64)
    assert oracle.recall_at_k(got, gt, 10) >= oracle.recall_at_k(got_r, gt, 10) - 0.1


def test_insertion_hand_traced_on_a_circle():
    """Two insertions into the hand-traced circle graph (Sec. 5.7)."""
    import json
    import os

    with open(os.path.join(os.path.dirname(__file__), "golden", "insertion_circle.json")) as f:
        g = json.load(f)

    def unit(angles):
        r = np.deg2rad(np.asarray(angles, np.float64))
        V = np.zeros((len(r), 4), np.float32)
        V[:, 0], V[:, 1] = np.cos(r), np.sin(r)
        return V

    X, T = unit(g["angles"]), unit(g["query_angles"])
    knn = np.asarray(g["knn"], dtype=np.uint32)
    M = g["M"]
    R = 2 * M
    adj = np.full((X.shape[0], R), NONE, dtype=np.uint32)
    for v, row in enumerate(g["graph"]):
        adj[v, :len(row)] = row
    cap = 8
    nout = np.full((T.shape[0], cap), NONE, dtype=np.uint32)
    nout[:, :knn.shape[1] - 1] = knn[:, 1:]
    cnt = np.full(T.shape[0], knn.shape[1] - 1, dtype=np.int32)
    n_old = len(g["graph"])
    a, no, c, q = oracle.insert(X, adj, g["entry"], n_old, T, knn[:, 0], nout, cnt, M, g["L"], max_visits=16384)  # does not bind: each traced search visits at most n rows
    for v, row in enumerate(g["adj"]):
        assert [int(u) for u in a[v] if u != NONE] == row, (v, a[v].tolist())
    assert q.tolist() == g["chosen_q"]
    assert no[1, :c[1]].tolist() == g["nout_t1"]
