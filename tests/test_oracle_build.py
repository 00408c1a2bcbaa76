"""Pins of the oracle's index construction (Alg. 1-3, Sec. 4.2).

Hand-traced cases fix the projection, connectivity enhancement and the
reachability repair step by step; invariants check what the paper states
the graph must satisfy. (No graph from the authors exists to compare a
whole index against.)
"""
from collections import deque

import numpy as np
import pytest

import oracle
from conftest import load_golden

NONE = 0xFFFFFFFF


def _lists(adj):
    return [[int(u) for u in row if u != NONE] for row in adj]


def test_degree_bounds_no_self_loops_no_duplicates(tiny):
    M = tiny["M"]
    pj, fin = _lists(tiny["pj"]), _lists(tiny["adj"])
    for v, (a, b) in enumerate(zip(pj, fin)):
        assert len(a) <= M and len(b) <= 2 * M
        assert v not in a and v not in b
        assert len(set(a)) == len(a) and len(set(b)) == len(b)
        # padding only at the end of a row
        row = tiny["adj"][v]
        assert np.all(row[len(b):] == NONE)


def test_every_node_reachable_from_entry(tiny):
    fin = _lists(tiny["adj"])
    seen = np.zeros(len(fin), bool)
    seen[tiny["entry"]] = True
    dq = deque([tiny["entry"]])
    while dq:
        v = dq.popleft()
        for u in fin[v]:
            if not seen[u]:
                seen[u] = True
                dq.append(u)
    assert seen.all()


def test_projection_edges_come_from_bipartite_candidates(tiny):
    """Every G_pj edge a->b links a pivot to a node reached through one of
    its bridge queries (Alg. 2's candidate collection), either forward (b in U(a)) or as
    the reverse edge of a pivot b (a in U(b))."""
    knn = tiny["knn"]
    n = tiny["X"].shape[0]
    U = [set() for _ in range(n)]
    for t in range(knn.shape[0]):
        U[int(knn[t, 0])].update(int(c) for c in knn[t, 1:])
    for a, row in enumerate(_lists(tiny["pj"])):
        for b in row:
            assert b in U[a] or a in U[b]


def test_final_lists_start_with_projection_lists(tiny):
    pj, fin = _lists(tiny["pj"]), _lists(tiny["adj"])
    for a, b in zip(pj, fin):
        assert b[:len(a)] == a
    assert tiny["stats"]["repairs"] >= (1 if tiny["stats"]["unreachable_before_repair"] else 0)


def test_pivots_are_the_1nn_of_some_training_query(tiny):
    knn = tiny["knn"]
    assert tiny["stats"]["pivots"] == len(set(knn[:, 0].tolist()))


def test_recall_non_decreasing_in_L(tiny):
    X, Q, gt = tiny["X"], tiny["Q"], tiny["gt"]
    rec = []
    for L in (10, 20, 50, 100):
        ids, *_ = oracle.beam_search(X, tiny["adj"], tiny["entry"], Q, 10, L)
        rec.append(oracle.recall_at_k(ids, gt, 10))
    assert all(b >= a for a, b in zip(rec, rec[1:])), rec
    assert rec[-1] > 0.6


def test_tiny_search_reaches_exact_result_at_full_L(tiny):
    """L >= N on the connected final graph gives the exact top-k (Sec. 4.3)."""
    X, Q = tiny["X"], tiny["Q"][:3]
    ids, dist, visits, *_ = oracle.beam_search(X, tiny["adj"], tiny["entry"], Q, 10, X.shape[0])
    for i in range(len(Q)):
        dd = np.array([-oracle.dot_fixed(Q[i], x) for x in X], np.float32)
        order = np.lexsort((np.arange(len(X)), dd))[:10]
        assert ids[i].tolist() == order.tolist()
    assert np.all(visits == X.shape[0])


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_projection_hand_traced_on_a_circle(precision):
    """G_pj of the oracle's construction against a hand-traced case (Alg. 1-3).
    Every margin in the case is far above FP32 rounding, so the FP32 form of
    the construction must take the same decisions."""
    import json
    import os

    with open(os.path.join(os.path.dirname(__file__), "golden", "projection_circle.json")) as f:
        g = json.load(f)
    r = np.deg2rad(np.asarray(g["angles"], np.float64))
    X = np.zeros((len(r), 4), np.float32)
    X[:, 0], X[:, 1] = np.cos(r), np.sin(r)
    knn = np.asarray(g["knn"], dtype=np.uint32)
    adj, pj, stats = oracle.build_index(X, knn, g["M"], 10, 0, precision=precision)
    for v, row in g["pj"]:
        got = [int(u) for u in pj[v] if u != 0xFFFFFFFF]
        assert got == row, (v, got, row)


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_construction_hand_traced_on_a_circle(precision):
    """The oracle's whole construction (projection, connectivity enhancement,
    final union, repair) against a hand-traced case (Alg. 1-3), in FP64 and in
    the FP32 fixed-order form (margins far above FP32 rounding)."""
    import json
    import os

    with open(os.path.join(os.path.dirname(__file__), "golden", "construction_circle.json")) as f:
        g = json.load(f)
    r = np.deg2rad(np.asarray(g["angles"], np.float64))
    X = np.zeros((len(r), 4), np.float32)
    X[:, 0], X[:, 1] = np.cos(r), np.sin(r)
    knn = np.asarray(g["knn"], dtype=np.uint32)
    adj, pj, stats = oracle.build_index(X, knn, g["M"], g["L"], g["entry"], precision=precision)
    for v, row in g["pj"]:
        assert [int(u) for u in pj[v] if u != 0xFFFFFFFF] == row, ("pj", v)
    for v, row in g["adj"]:
        assert [int(u) for u in adj[v] if u != 0xFFFFFFFF] == row, ("adj", v, adj[v].tolist())


def test_hand_traced_reachability_repair():
    """The repair step (an addition to Alg. 1) on a hand-traced case with all
    three of its branches: nearest reachable node with room, nearest full but
    another with room, every reachable node full (the last edge is evicted)."""
    g = load_golden("repair_circle.json")
    a = np.deg2rad(np.array(g["angles_deg"], np.float64))
    X = np.zeros((len(a), 4), np.float32)
    X[:, 0], X[:, 1] = np.cos(a), np.sin(a)
    adj, repairs, unreach = oracle.repair(X, np.array(g["adj"], np.uint32), g["entry"])
    assert adj.tolist() == g["expect_adj"]
    assert (repairs, unreach) == (g["expect_repairs"], g["expect_unreachable_before"])
    # already connected: nothing to do
    adj2, r2, u2 = oracle.repair(X, adj, g["entry"])
    assert adj2.tolist() == adj.tolist() and (r2, u2) == (0, 0)


def test_fp32_construction_close_to_fp64(tiny):
    """The FP32 fixed-order construction on the tiny workload: the same
    invariants, and nearly the same graph as FP64 (decisions differ only
    where two distances fall within FP32 rounding)."""
    X, knn = tiny["X"], tiny["knn"]
    adj32, pj32, st32 = oracle.build_index(X, knn, 32, 500, tiny["entry"], precision="f32")
    adj64, pj64 = tiny["adj"], tiny["pj"]
    same_pj = np.mean([np.array_equal(a, b) for a, b in zip(pj32, pj64)])
    same_adj = np.mean([np.array_equal(a, b) for a, b in zip(adj32, adj64)])
    assert same_pj > 0.95 and same_adj > 0.9, (same_pj, same_adj)
    deg = (adj32 != NONE).sum(1)
    assert deg.max() <= 64 and st32["unreachable_before_repair"] >= 0
