"""Uneven batches in one persistent launch, CUDA-graph replay, team sizes and
the launch autotuner: every variant returns exactly the oracle's beam search
(Sec. 4.3) for each query's own (k, L)."""
import numpy as np
import pytest

import oracle
import roarsynth as rs
from gpu_util import dev_index

pytestmark = pytest.mark.gpu
MV = 16384


def _torch(a, dtype=None):
    import torch

    t = torch.from_numpy(np.ascontiguousarray(a))
    return t.to("cuda:0")


def _oracle_per_query(tiny, Q, ks, Ls, dtype="f32", codes=None, scales=None):
    out = []
    for q, k, L in zip(Q, ks, Ls):
        r = oracle.beam_search(tiny["X"], tiny["adj"], tiny["entry"], q[None], int(k), int(L),
                               max_visits=MV, dtype=dtype, Xt=codes, scales=scales)
        out.append(r)
    return out


def _check_uneven(out, ref, ks):
    import torch

    torch.cuda.synchronize()
    off, ids, dist, visits, hops, st = (t.cpu().numpy() for t in out)
    ids = ids.view(np.uint32)
    for i, (r, k) in enumerate(zip(ref, ks)):
        o = off[i]
        assert ids[o:o + k].tolist() == r[0][0].tolist(), f"query {i}"
        assert np.array_equal(dist[o:o + k], r[1][0])
        assert visits[i] == r[2][0] and hops[i] == r[3][0] and st[i] == r[4][0]


@pytest.fixture(scope="module")
def uneven_case(tiny):
    nq = 240
    ks, Ls = rs.uneven_params(nq, seed_tag=31)
    Q = tiny["Q"][:nq]
    ref = _oracle_per_query(tiny, Q, ks, Ls)
    return Q, ks, Ls, ref


def test_uneven_batch_matches_oracle(tiny, uneven_case):
    Q, ks, Ls, ref = uneven_case
    idx = dev_index(tiny["X"], tiny["adj"], tiny["entry"], max_visits=MV)
    out = idx.uneven_outputs(ks)
    idx.search_uneven(_torch(Q), _torch(ks), _torch(Ls), int(Ls.max()), out)
    _check_uneven(out, ref, ks)
    idx.close()


def test_graph_plan_replays_exactly(tiny, uneven_case):
    import torch

    Q, ks, Ls, ref = uneven_case
    idx = dev_index(tiny["X"], tiny["adj"], tiny["entry"], max_visits=MV)
    Qd, kd, Ld = _torch(Q), _torch(ks), _torch(Ls)
    out = idx.uneven_outputs(ks)
    plan = idx.plan_uneven(Qd, kd, Ld, int(Ls.max()), out, longest_first=True)
    for _ in range(3):
        out[1].fill_(0)
        plan.launch()
        _check_uneven(out, ref, ks)
    plan.close()
    idx.close()


@pytest.mark.parametrize("tw", [1, 2, 4, 8])
@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_team_sizes_bit_exact(tiny, tw, dtype):
    X = tiny["X"]
    codes = oracle.quant_bf16(X) if dtype == "bf16" else None
    idx = dev_index(X, tiny["adj"], tiny["entry"], dtype=dtype,
                    trav=None if codes is None else codes.view(np.int16), max_visits=MV)
    Q = tiny["Q"][:150]
    for L in (16, 100, 300):
        idx.set_tuning(L, tw, 0, 0)
        from gpu_util import run
        got = run(idx, Q, 10, L)
        ref = oracle.beam_search(X, tiny["adj"], tiny["entry"], Q, 10, L, max_visits=MV, dtype=dtype,
                                 Xt=codes)
        assert np.array_equal(got[0], ref[0]), (tw, dtype, L)
        assert np.array_equal(got[2], ref[2]) and np.array_equal(got[3], ref[3])
        assert np.array_equal(got[1], ref[1])
    idx.close()


def test_bad_per_query_parameters_are_reported(tiny):
    Q = tiny["Q"][:6]
    ks = np.array([10, 0, 10, 20, 5, 10], np.int32)
    Ls = np.array([50, 50, 5, 20, 2000, 30], np.int32)   # k=0, k>L, L>L_max are invalid
    idx = dev_index(tiny["X"], tiny["adj"], tiny["entry"], max_visits=MV)
    out = idx.uneven_outputs(np.maximum(ks, 1))
    idx.search_uneven(_torch(Q), _torch(ks), _torch(Ls), 64, out)
    import torch

    torch.cuda.synchronize()
    st = out[5].cpu().numpy()
    assert st.tolist() == [0, 1, 1, 0, 1, 0]
    idx.close()


def test_alone_equals_mixed(tiny, uneven_case):
    """Each query's result is the same alone and inside the uneven batch."""
    import torch

    Q, ks, Ls, ref = uneven_case
    idx = dev_index(tiny["X"], tiny["adj"], tiny["entry"], max_visits=MV)
    out = idx.uneven_outputs(ks)
    idx.search_uneven(_torch(Q), _torch(ks), _torch(Ls), int(Ls.max()), out)
    torch.cuda.synchronize()
    mixed = out[1].cpu().numpy().view(np.uint32)
    off = out[0].cpu().numpy()
    for i in (0, 7, 100, 239):
        ids, *_ = idx.search(_torch(Q[i:i + 1]), int(ks[i]), int(Ls[i]))
        torch.cuda.synchronize()
        assert ids.cpu().numpy().view(np.uint32)[0].tolist() == mixed[off[i]:off[i] + ks[i]].tolist()
    idx.close()


def test_autotune_keeps_results(tiny):
    idx = dev_index(tiny["X"], tiny["adj"], tiny["entry"], max_visits=MV)
    Q = tiny["Q"][:400]
    best, res = idx.autotune(_torch(Q), 10, 100, repeats=2)
    assert 0 <= best < 16 and np.isfinite(res[best]) and res[best] < 1e29
    assert res[best] == res[res < 1e29].min()
    from gpu_util import run, assert_same

    ref = oracle.beam_search(tiny["X"], tiny["adj"], tiny["entry"], Q, 10, 100, max_visits=MV)
    assert_same(run(idx, Q, 10, 100), ref, "after autotune")
    idx.close()
