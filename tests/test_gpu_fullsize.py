"""Parity at the benchmark's full size (1M x 200 base rows, 10k OOD queries)
in the launch configuration bench.py times, checked on sampled queries the
oracle computes one by one. The graph is roarsynth.cluster_graph: seeded
structure that comes from neither the oracle nor the CUDA library."""
import numpy as np
import pytest

import oracle
import roarsynth as rs
from gpu_util import dev_index

pytestmark = pytest.mark.gpu
MV = 16384
W = rs.BASE_1M_D200


@pytest.fixture(scope="module")
def full():
    X = rs.base(W)
    Q = rs.test_queries(W)
    adj = rs.cluster_graph(W)
    entry = 0
    return dict(X=X, Q=Q, adj=adj, entry=entry)


def _device(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def _search(idx, Qd, k, L):
    import torch

    ids, dist, visits, hops, st = idx.search(Qd, k, L)
    torch.cuda.synchronize()
    return (ids.cpu().numpy().view(np.uint32), dist.cpu().numpy(), visits.cpu().numpy().view(np.uint32),
            hops.cpu().numpy().view(np.uint32), st.cpu().numpy())


SAMPLE = np.random.default_rng(5).choice(10_000, 12, replace=False)


@pytest.mark.parametrize("L,tw,hash_log2", [(1024, 1, -1), (100, 1, -1), (100, 4, -1), (90, 1, 0), (90, 1, 10)])
def test_fp32_full_batch_sampled_parity(full, L, tw, hash_log2):
    idx = dev_index(full["X"], full["adj"], full["entry"], max_visits=MV)
    idx.set_tuning(L, tw, hash_log2, 0)     # bench-like launch shapes: bitmap, auto, shared table
    got = _search(idx, _device(full["Q"]), 10, L)     # the whole 10k batch in one launch
    idx.close()
    Qs = full["Q"][SAMPLE]
    ref = oracle.beam_search(full["X"], full["adj"], full["entry"], Qs, 10, L, max_visits=MV)
    for g, r in zip(got, ref):
        if g.dtype == np.float32:
            assert np.allclose(g[SAMPLE], r, rtol=1e-6, atol=0)
        else:
            assert np.array_equal(g[SAMPLE], r)


@pytest.mark.parametrize("dtype", ["bf16", "fp8"])
def test_quantized_full_batch_sampled_parity(full, dtype):
    import torch

    import paper_2408_08933_gb300 as pkg

    X = full["X"]
    Xd = _device(X)
    codes_d, sc_d = pkg.quantize(Xd, dtype)
    torch.cuda.synchronize()
    if dtype == "bf16":
        codes = oracle.quant_bf16(X)
        sc = None
        assert np.array_equal(codes_d.cpu().numpy().view(np.uint16)[::997], codes[::997])
    else:
        codes, sc = oracle.quant_e4m3(X)
        assert np.array_equal(codes_d.cpu().numpy()[::997], codes[::997])
        assert np.array_equal(sc_d.cpu().numpy(), sc)
    idx = dev_index(X, full["adj"], full["entry"], dtype=dtype,
                    trav=codes.view(np.int16) if dtype == "bf16" else codes, scales=sc, max_visits=MV)
    got = _search(idx, _device(full["Q"]), 10, 500)
    idx.close()
    Qs = full["Q"][SAMPLE[:6]]
    ref = oracle.beam_search(X, full["adj"], full["entry"], Qs, 10, 500, max_visits=MV, dtype=dtype,
                             Xt=codes, scales=sc)
    assert np.array_equal(got[0][SAMPLE[:6]], ref[0])
    assert np.array_equal(got[2][SAMPLE[:6]], ref[2])
    assert np.allclose(got[1][SAMPLE[:6]], ref[1], rtol=1e-6, atol=0)


def test_knn_full_size_sampled_rows(full):
    """The builder's kNN step (depth 100) on 1,000 training rows, sampled from
    across the 1M-row set, against all 1M base rows, checked against the
    oracle's FP64 brute force (run on the host cores in parallel)."""
    from concurrent.futures import ThreadPoolExecutor
    import os

    import torch

    import paper_2408_08933_gb300 as pkg

    starts = np.sort(np.random.default_rng(8).choice(W.n_train // 100, 100, replace=False)) * 100
    T = np.concatenate([rs.train_queries(W, int(s), int(s) + 10) for s in starts])      # 1,000 rows
    ids, dist = pkg.knn(_device(T), _device(full["X"]), 100)
    torch.cuda.synchronize()
    ids = ids.cpu().numpy().view(np.uint32)
    cores = os.cpu_count() or 1
    parts = [c for c in np.array_split(np.arange(T.shape[0]), 2 * cores) if len(c)]
    with ThreadPoolExecutor(max_workers=cores) as ex:
        res = list(ex.map(lambda ix: oracle.knn_f64(T[ix], full["X"], 100), parts))
    ref_ids = np.concatenate([r[0] for r in res])
    ref_d = np.concatenate([r[1] for r in res])
    overlap = 0
    for r in range(T.shape[0]):
        kth = ref_d[r, 99]
        d64 = -(full["X"][ids[r]].astype(np.float64) @ T[r].astype(np.float64))
        assert np.all(d64 <= kth + 1e-5), r
        overlap += len(set(ids[r]) & set(ref_ids[r]))
    assert overlap / (100 * T.shape[0]) >= 0.999
