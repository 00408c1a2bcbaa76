"""The ablation graphs of Sec. 5.4 on the GPU: the bipartite graph G_bi
(Alg. 1's bipartite step, searched through query nodes as in Sec. 4.1) and
the projected graph G_pj, each against the oracle."""
import numpy as np
import pytest

import oracle
from conftest import load_golden, path_graph
from gpu_util import assert_same, dev_index

pytestmark = pytest.mark.gpu
MV = 16384


def _bi_index(X, knn, entry, max_visits=MV):
    import torch

    import paper_2408_08933_gb300 as pkg

    Xd = torch.from_numpy(np.ascontiguousarray(X, np.float32)).to("cuda:0")
    kd = torch.from_numpy(np.ascontiguousarray(knn, np.uint32).view(np.int32)).to("cuda:0")
    off, qids, nout, stats = pkg.bipartite(kd, X.shape[0])
    torch.cuda.synchronize()
    return pkg.BipartiteIndex(Xd, nout, off, qids, entry, max_visits=max_visits), off, qids, nout, stats


def _run(idx, Q, k, L):
    import torch

    Qd = torch.from_numpy(np.ascontiguousarray(Q, np.float32)).to("cuda:0")
    ids, dist, visits, hops, st = idx.search(Qd, k, L)
    torch.cuda.synchronize()
    return (ids.cpu().numpy().view(np.uint32), dist.cpu().numpy(), visits.cpu().numpy().view(np.uint32),
            hops.cpu().numpy().view(np.uint32), st.cpu().numpy())


def bi_entry(X, off, entry):
    """The G_bi search entry: the medoid when it has a query out-neighbour,
    else the base node with one nearest to it (FP64 inner product, ties by id)."""
    if off[entry + 1] > off[entry]:
        return int(entry)
    piv = np.nonzero(np.diff(off) > 0)[0]
    s = X[piv].astype(np.float64) @ X[entry].astype(np.float64)
    return int(piv[np.lexsort((piv, -s))[0]])


def test_hand_traced_bipartite_search():
    g = load_golden("bipartite_search.json")
    X, _ = path_graph(g["a"])
    knn = np.array(g["knn"], np.uint32)
    q = np.array([[1, 0, 0, 0]], np.float32)
    for c in g["cases"]:
        idx, off, qids, nout, stats = _bi_index(X, knn, g["entry"], max_visits=c["max_visits"])
        assert off.cpu().numpy().tolist() == g["expect_off"]
        assert qids.cpu().numpy().tolist() == g["expect_qids"]
        ids, dist, visits, hops, st = _run(idx, q, c["k"], c["L"])
        assert ids[0].tolist() == c["ids"] and dist[0].tolist() == c["dist"], c["derivation"]
        assert (int(visits[0]), int(hops[0]), int(st[0])) == (c["visits"], c["hops"], c["status"])
        assert stats == {"base_nodes_with_query_edges": 3, "widest_base_row": 2}
        idx.close()


@pytest.mark.parametrize("L", [10, 50, 100])
def test_bipartite_search_matches_oracle_tiny(tiny, L):
    X, knn = tiny["X"], tiny["knn"]
    idx, off, qids, nout, _ = _bi_index(X, knn, 0)
    ref_off, ref_q = oracle.bipartite(knn, X.shape[0])
    assert np.array_equal(off.cpu().numpy(), ref_off)
    assert np.array_equal(qids.cpu().numpy().view(np.uint32), ref_q)
    assert np.array_equal(nout.cpu().numpy().view(np.uint32), knn[:, 1:])
    entry = bi_entry(X, ref_off, tiny["entry"])
    idx.close()
    idx, *_ = _bi_index(X, knn, entry)
    Q = tiny["Q"]
    ref = oracle.beam_search_bi(X, knn, entry, Q, 10, L, max_visits=MV)
    assert_same(_run(idx, Q, 10, L), ref, f"G_bi L={L}")
    idx.close()


def test_projected_graph_search_matches_oracle_tiny(tiny):
    X, pj = tiny["X"], tiny["pj"]
    idx = dev_index(X, pj, tiny["entry"], max_visits=MV)
    from gpu_util import run

    for L in (10, 100):
        ref = oracle.beam_search(X, pj, tiny["entry"], tiny["Q"], 10, L, max_visits=MV)
        assert_same(run(idx, tiny["Q"], 10, L), ref, f"G_pj L={L}")
    idx.close()
