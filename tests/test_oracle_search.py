"""Pins for the oracle's beam search (Sec. 4.3)."""
import numpy as np
import pytest

import oracle
from conftest import load_golden, path_graph

NONE = 0xFFFFFFFF


def test_hand_traced_path_graph():
    g = load_golden("beam_path6.json")
    X, adj = path_graph(g["a"])
    q = np.array([1, 0, 0, 0], np.float32)
    for c in g["cases"]:
        pid, pdist, trace, visits, hops, st = oracle.beam_search_trace(
            X, adj, g["entry"], q, c["L"], c["max_visits"])
        assert trace.tolist() == c["trace"], c
        assert pid.tolist() == c["pool_ids"]
        assert pdist.tolist() == c["pool_dist"]
        assert (visits, hops, st) == (c["visits"], c["hops"], c["status"])


def _exact_topk_fixed(X, q, k):
    dist = np.array([-oracle.dot_fixed(q, x) for x in X], np.float32)
    order = np.lexsort((np.arange(len(X)), dist))
    return order[:k], dist[order[:k]]


def test_complete_graph_gives_exact_topk():
    rng = np.random.default_rng(21)
    n, d = 40, 16
    X = rng.standard_normal((n, d)).astype(np.float32)
    adj = np.array([[u for u in range(n) if u != v] for v in range(n)], np.uint32)
    Q = rng.standard_normal((10, d)).astype(np.float32)
    ids, dist, visits, hops, st = oracle.beam_search(X, adj, 7, Q, 5, 5)
    for i in range(len(Q)):
        ref_ids, ref_d = _exact_topk_fixed(X, Q[i], 5)
        assert ids[i].tolist() == ref_ids.tolist()
        assert np.array_equal(dist[i], ref_d)
    assert np.all(visits == n) and np.all(st == 0)


def test_large_L_on_connected_graph_is_exact():
    rng = np.random.default_rng(22)
    n, d, r = 300, 8, 6
    X = rng.standard_normal((n, d)).astype(np.float32)
    adj = np.full((n, r), NONE, np.uint32)
    for v in range(n):                      # ring plus random chords: connected
        nb = {(v + 1) % n, (v - 1) % n} | set(rng.integers(0, n, 3).tolist())
        nb.discard(v)
        nb = sorted(nb)[:r]
        adj[v, :len(nb)] = nb
    Q = rng.standard_normal((12, d)).astype(np.float32)
    ids, dist, visits, hops, st = oracle.beam_search(X, adj, 0, Q, 10, n)
    for i in range(len(Q)):
        assert ids[i].tolist() == _exact_topk_fixed(X, Q[i], 10)[0].tolist()
    assert np.all(visits == n) and np.all(hops == n)


def test_padding_when_reachable_set_is_small():
    X, adj = path_graph([0, 1, 3, 2, 5, 4])
    adj[2, :] = NONE        # cut the path after node 2: only {0, 1, 2} reachable
    q = np.array([[1, 0, 0, 0]], np.float32)
    ids, dist, visits, hops, st = oracle.beam_search(X, adj, 0, q, 5, 8)
    assert ids[0].tolist() == [2, 1, 0, NONE, NONE]
    assert np.isinf(dist[0, 3:]).all() and dist[0, :3].tolist() == [-3.0, -1.0, -0.0]
    assert visits[0] == 3 and hops[0] == 3


def test_ties_broken_by_lower_id():
    X = np.array([[0, 0, 0, 0], [2, 0, 0, 0], [2, 0, 0, 0], [1, 0, 0, 0], [2, 0, 0, 0]], np.float32)
    adj = np.array([[4, 3, 2, 1]] + [[0, NONE, NONE, NONE]] * 4, np.uint32)
    ids, dist, *_ = oracle.beam_search(X, adj, 0, np.array([[1, 0, 0, 0]], np.float32), 3, 3)
    assert ids[0].tolist() == [1, 2, 4]


def test_rejects_bad_arguments():
    X, adj = path_graph([0, 1, 2])
    q = np.zeros((1, 4), np.float32)
    with pytest.raises(ValueError):
        oracle.beam_search(X, adj, 5, q, 1, 1)       # entry out of range
    with pytest.raises(ValueError):
        oracle.beam_search(X, adj, 0, q, 3, 2)       # k > L


def test_tombstones_hand_traced_path_graph():
    """Deleted rows route but are not answers (Sec. 5.7), on the hand-traced graph."""
    g = load_golden("beam_path6_tomb.json")
    X, adj = path_graph(g["a"])
    q = np.array([[1, 0, 0, 0]], dtype=np.float32)
    for c in g["cases"]:
        deleted = np.zeros(len(g["a"]), dtype=bool)
        deleted[c["deleted"]] = True
        ids, dist, visits, hops, st = oracle.beam_search(X, adj, g["entry"], q, c["k"], c["L"],
                                                         tomb=oracle.pack_tombstones(deleted))
        assert ids[0].tolist() == c["ids"], c
        assert dist[0].tolist() == [float(v) for v in c["dist"]], c
        assert (int(visits[0]), int(hops[0])) == (c["visits"], c["hops"]), c


def test_tombstones_filter_the_same_traversal(tiny):
    """With tombstones the visits and hops are unchanged and the answers are the
    untombstoned search's final pool with the deleted ids removed."""
    rng = np.random.default_rng(3)
    deleted = rng.random(tiny["X"].shape[0]) < 0.2
    Q = tiny["Q"][:64]
    L = 50
    full = oracle.beam_search(tiny["X"], tiny["adj"], tiny["entry"], Q, L, L)
    got = oracle.beam_search(tiny["X"], tiny["adj"], tiny["entry"], Q, 10, L,
                             tomb=oracle.pack_tombstones(deleted))
    assert np.array_equal(full[2], got[2]) and np.array_equal(full[3], got[3])
    for i in range(Q.shape[0]):
        alive = [u for u in full[0][i].tolist() if u != 0xFFFFFFFF and not deleted[u]][:10]
        assert got[0][i].tolist() == alive + [0xFFFFFFFF] * (10 - len(alive))


def quant_fan_inputs(g):
    """Arrays of the hand-traced quantised-search case (tests/golden/quant_search_fan.json)."""
    X32 = np.array(g["x32"], np.float32)
    adj = np.array(g["adj"], np.uint32)
    q = np.array([g["q"]], np.float32)
    fp8 = np.array(g["fp8_codes"], np.uint8)
    scales = np.array(g["fp8_scale_bits"], np.uint32).view(np.float32)
    bf16 = np.array(g["bf16_codes"], np.uint16)
    return X32, adj, q, fp8, scales, bf16


def test_hand_traced_quantized_search_and_rerank():
    """BF16 / FP8 traversal with one FP32 scale multiply after the fixed-order
    dot, the FP32 re-rank of the whole final pool, ties by id (hand-traced)."""
    g = load_golden("quant_search_fan.json")
    X32, adj, q, fp8, scales, bf16 = quant_fan_inputs(g)
    assert [oracle.e4m3_to_f32(int(c)) for c in fp8[1]] == [0.125, 0.625, 0.0, 0.0]
    assert scales[1] == np.float32(1 + 2.0 ** -23)
    forms = {"fp8": dict(dtype="fp8", Xt=fp8, scales=scales), "bf16": dict(dtype="bf16", Xt=bf16),
             "f32": dict(dtype="f32")}
    for name, kw in forms.items():
        e = g["expect"][name]
        for k in (1, 2):
            ids, dist, visits, hops, st = oracle.beam_search(X32, adj, g["entry"], q, k, g["L"], **kw)
            assert ids[0].tolist() == e[str(k)]["ids"], (name, k)
            assert dist[0].tolist() == e[str(k)]["dist"], (name, k)
            assert (int(visits[0]), int(hops[0]), int(st[0])) == (e["visits"], e["hops"], 0), name


def test_hand_traced_bipartite_graph_search():
    """G_bi (Alg. 1's bipartite step, every x -> t edge kept) and the greedy
    search through query nodes (Sec. 4.1), traced by hand."""
    g = load_golden("bipartite_search.json")
    X, _ = path_graph(g["a"])
    knn = np.array(g["knn"], np.uint32)
    off, qids = oracle.bipartite(knn, X.shape[0])
    assert off.tolist() == g["expect_off"] and qids.tolist() == g["expect_qids"]
    q = np.array([[1, 0, 0, 0]], np.float32)
    for c in g["cases"]:
        ids, dist, visits, hops, st = oracle.beam_search_bi(X, knn, g["entry"], q, c["k"], c["L"], c["max_visits"])
        assert ids[0].tolist() == c["ids"] and dist[0].tolist() == c["dist"], c["derivation"]
        assert (int(visits[0]), int(hops[0]), int(st[0])) == (c["visits"], c["hops"], c["status"])


def test_bipartite_search_complete_is_exact():
    """One training query linked to every base row: expanding the entry scores
    every row, so the result is the exact top-k under dot_fixed."""
    rng = np.random.default_rng(23)
    n, d = 50, 12
    X = rng.standard_normal((n, d)).astype(np.float32)
    knn = np.array([[5] + [u for u in range(n) if u != 5]], np.uint32)
    Q = rng.standard_normal((6, d)).astype(np.float32)
    ids, dist, visits, hops, st = oracle.beam_search_bi(X, knn, 5, Q, 7, 7)
    for i in range(len(Q)):
        ref_ids, ref_d = _exact_topk_fixed(X, Q[i], 7)
        assert ids[i].tolist() == ref_ids.tolist() and np.array_equal(dist[i], ref_d)
    assert np.all(visits == n) and np.all(st == 0)
