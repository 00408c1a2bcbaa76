"""The builder's dense step (exact kNN, Sec. 4.2.1) and the GPU-assisted construction."""
from collections import deque

import numpy as np
import pytest

import oracle
import roarsynth as rs

pytestmark = pytest.mark.gpu
NONE = 0xFFFFFFFF


def _cuda(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def test_knn_against_fp64_brute_force(tiny):
    """Returned distances are exact fixed-order FP32 values; the returned sets
    agree with FP64 brute force except where two FP64 scores lie within the
    FP32 rounding bound of each other."""
    import torch

    import paper_2408_08933_gb300 as pkg

    X, T = tiny["X"], tiny["T"]
    ids, dist = pkg.knn(_cuda(T), _cuda(X), 100)
    torch.cuda.synchronize()
    ids = ids.cpu().numpy().view(np.uint32)
    dist = dist.cpu().numpy()
    ref = tiny["knn"]                                # oracle FP64, ties to the lower id
    rng = np.random.default_rng(0)
    rows = rng.choice(T.shape[0], 1000, replace=False)
    for r in rows:
        assert np.all(np.diff(dist[r]) >= 0)
        for j in (0, 37, 99):
            assert dist[r, j] == -oracle.dot_fixed(T[r], X[ids[r, j]])
    d64 = -(T[rows].astype(np.float64) @ X.astype(np.float64).T)
    eps = 1e-5
    for i, r in enumerate(rows):
        kth = np.sort(d64[i])[99]
        assert np.all(d64[i][ids[r]] <= kth + eps)
    hits = sum(len(set(ids[r]) & set(ref[r])) for r in rows)
    assert hits / (100 * len(rows)) >= 0.999


def test_knn_small_n_and_ragged():
    import torch

    import paper_2408_08933_gb300 as pkg

    rng = np.random.default_rng(9)
    X = rng.standard_normal((77, 8)).astype(np.float32)
    T = rng.standard_normal((13, 8)).astype(np.float32)
    ids, dist = pkg.knn(_cuda(T), _cuda(X), 77)
    torch.cuda.synchronize()
    ref, _ = oracle.knn_f64(T, X, 77)
    got = ids.cpu().numpy().view(np.uint32)
    for r in range(13):
        assert sorted(got[r].tolist()) == list(range(77))


@pytest.mark.parametrize("d,halves", [(64, "2"), (256, "2"), (256, "1"), (256, ""), (264, ""), (512, "")])
def test_knn_wide_rows(d, halves, monkeypatch):
    """Both CTA shapes of the tensor-core kNN: two 128-row halves of T per CTA
    sharing each X tile (d <= 256; forced here, small launches pick one half)
    and one half, on ragged sizes; returned distances exact in the fixed FP32
    order, sets equal to FP64 brute force up to FP32 near-ties."""
    import torch

    import paper_2408_08933_gb300 as pkg

    monkeypatch.setenv("ROAR_KNN_HALVES", halves)
    rng = np.random.default_rng(d)
    X = rng.standard_normal((2999, d)).astype(np.float32)
    T = rng.standard_normal((517, d)).astype(np.float32)
    ids, dist = pkg.knn(_cuda(T), _cuda(X), 50)
    torch.cuda.synchronize()
    ids = ids.cpu().numpy().view(np.uint32)
    dist = dist.cpu().numpy()
    ref, ref_d = oracle.knn_f64(T, X, 50)
    for r in range(0, T.shape[0], 7):
        assert np.all(np.diff(dist[r]) >= 0)
        for j in (0, 49):
            assert dist[r, j] == -oracle.dot_fixed(T[r], X[ids[r, j]])
        d64 = -(X[ids[r]].astype(np.float64) @ T[r].astype(np.float64))
        assert np.all(d64 <= ref_d[r, 49] + 1e-4)
    hits = sum(len(set(ids[r]) & set(ref[r])) for r in range(T.shape[0]))
    assert hits / (50 * T.shape[0]) >= 0.999


def test_build_invariants_and_recall(tiny):
    import torch

    import paper_2408_08933_gb300 as pkg

    X, T, Q, gt = tiny["X"], tiny["T"], tiny["Q"], tiny["gt"]
    Xd = _cuda(X)
    adj, entry, st = pkg.build_index(Xd, _cuda(T), nq_depth=100, M=32, L_build=500)
    torch.cuda.synchronize()
    A = adj.cpu().numpy().view(np.uint32)
    assert entry == oracle.medoid(X)
    assert A.shape == (X.shape[0], 64)
    seen = np.zeros(X.shape[0], bool)
    seen[entry] = True
    dq = deque([entry])
    for v, row in enumerate(A):
        lst = [int(u) for u in row if u != NONE]
        assert v not in lst and len(set(lst)) == len(lst)
        assert np.all(row[len(lst):] == NONE)
    while dq:
        v = dq.popleft()
        for u in A[v]:
            if u != NONE and not seen[u]:
                seen[u] = True
                dq.append(int(u))
    assert seen.all()
    assert st["pivots"] == len(set(tiny["knn"][:, 0].tolist()))
    assert st["unreachable_after_repair"] == 0
    idx = pkg.Index(Xd, adj, entry)
    ids, *_ = idx.search(_cuda(Q), 10, 100)
    torch.cuda.synchronize()
    rec = oracle.recall_at_k(ids.cpu().numpy().view(np.uint32), gt, 10)
    ref_ids, *_ = oracle.beam_search(X, tiny["adj"], tiny["entry"], Q, 10, 100)
    rec_oracle_graph = oracle.recall_at_k(ref_ids, gt, 10)
    idx.close()
    assert rec >= rec_oracle_graph - 0.05, (rec, rec_oracle_graph)


def test_literal_build_matches_oracle_tiny(tiny):
    """Alg. 1 in its literal order, composed of the library's GPU parts (kNN,
    search, Alg. 3), against the oracle's construction in the same FP32
    fixed-order precision from the same kNN lists: G_pj and the final graph
    identical row for row, the same entry."""
    import torch

    import paper_2408_08933_gb300 as pkg

    X, T = tiny["X"], tiny["T"]
    Xd, Td = _cuda(X), _cuda(T)
    adj, entry, stats, pj = pkg.build_index_literal(Xd, Td, nq_depth=100, M=32, L_build=500)
    kid, _ = pkg.knn(Td, Xd, 100)
    torch.cuda.synchronize()
    knn = kid.cpu().numpy().view(np.uint32)
    assert entry == oracle.medoid(X)
    r_adj, r_pj, r_st = oracle.build_index(X, knn, 32, 500, entry, precision="f32")
    g_pj = pj.cpu().numpy().view(np.uint32)
    g_adj = adj.cpu().numpy().view(np.uint32)
    bad_pj = [v for v in range(len(X)) if not np.array_equal(g_pj[v], r_pj[v])]
    bad_adj = [v for v in range(len(X)) if not np.array_equal(g_adj[v], r_adj[v])]
    assert not bad_pj, (len(bad_pj), bad_pj[:5])
    assert not bad_adj, (len(bad_adj), bad_adj[:5])
    assert (stats["pivots"], stats["repairs"]) == (r_st["pivots"], r_st["repairs"])
