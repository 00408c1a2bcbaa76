"""GPU parity of the FP32 beam search (Sec. 4.3) with the oracle, through the C ABI."""
import numpy as np
import pytest

import oracle
from conftest import path_graph, load_golden
from gpu_util import assert_same, dev_index, run

pytestmark = pytest.mark.gpu
MV = 16384


@pytest.fixture(scope="module")
def tiny_idx(tiny):
    idx = dev_index(tiny["X"], tiny["adj"], tiny["entry"], max_visits=MV)
    yield idx
    idx.close()


@pytest.mark.parametrize("L", [10, 20, 50, 100])
def test_tiny_bit_exact(tiny, tiny_idx, L):
    Q = tiny["Q"]
    ref = oracle.beam_search(tiny["X"], tiny["adj"], tiny["entry"], Q, 10, L, max_visits=MV)
    assert_same(run(tiny_idx, Q, 10, L), ref, f"L={L}")


@pytest.mark.parametrize("k,L", [(1, 1), (7, 33), (64, 64), (200, 257), (1024, 1024)])
def test_tiny_k_and_L_edges(tiny, tiny_idx, k, L):
    Q = tiny["Q"][:37]   # ragged batch: not a multiple of the warps per CTA
    ref = oracle.beam_search(tiny["X"], tiny["adj"], tiny["entry"], Q, k, L, max_visits=MV)
    assert_same(run(tiny_idx, Q, k, L), ref, f"k={k} L={L}")


@pytest.mark.parametrize("L", [320, 321])
def test_staged_and_register_gather_edge(tiny, tiny_idx, L):
    """Pools up to 320 entries gather rows through shared memory, longer ones
    through registers; both give the oracle's trajectory."""
    Q = tiny["Q"][:150]
    ref = oracle.beam_search(tiny["X"], tiny["adj"], tiny["entry"], Q, 10, L, max_visits=MV)
    assert_same(run(tiny_idx, Q, 10, L), ref, f"L={L}")


@pytest.mark.parametrize("nq", [1, 2, 5, 129])
def test_ragged_batches(tiny, tiny_idx, nq):
    Q = tiny["Q"][:nq]
    ref = oracle.beam_search(tiny["X"], tiny["adj"], tiny["entry"], Q, 10, 50, max_visits=MV)
    assert_same(run(tiny_idx, Q, 10, 50), ref, f"nq={nq}")


def test_empty_batch(tiny_idx):
    import torch

    q = torch.empty((0, 64), dtype=torch.float32, device="cuda:0")
    out = tiny_idx.search(q, 10, 10)
    assert out[0].shape == (0, 10)


@pytest.mark.parametrize("log2", [-1, 5, 7, 10])
def test_overflow_visited_table_path(tiny, log2):
    """A tiny shared table forces the global overflow table; results are unchanged."""
    idx = dev_index(tiny["X"], tiny["adj"], tiny["entry"], max_visits=MV)
    idx.set_hash_log2(log2)
    Q = tiny["Q"][:200]
    ref = oracle.beam_search(tiny["X"], tiny["adj"], tiny["entry"], Q, 10, 200, max_visits=MV)
    assert_same(run(idx, Q, 10, 200), ref, f"log2={log2}")
    # the overflow tables are reused by later queries (tagged entries, never cleared)
    assert_same(run(idx, Q, 10, 200), ref, f"log2={log2} again")
    idx.close()


def test_visit_cap(tiny):
    idx = dev_index(tiny["X"], tiny["adj"], tiny["entry"], max_visits=100)
    Q = tiny["Q"][:64]
    ref = oracle.beam_search(tiny["X"], tiny["adj"], tiny["entry"], Q, 10, 100, max_visits=100)
    assert np.all(ref[4] == oracle.ST_EOVERFLOW)
    assert_same(run(idx, Q, 10, 100), ref, "visit cap")
    idx.close()


def test_hand_traced_path_graph():
    g = load_golden("beam_path6.json")
    X, adj = path_graph(g["a"])
    q = np.array([[1, 0, 0, 0]], np.float32)
    for c in g["cases"]:
        idx = dev_index(X, adj, g["entry"], max_visits=c["max_visits"])
        ids, dist, visits, hops, st = run(idx, q, c["L"], c["L"])
        assert ids[0].tolist() == c["pool_ids"]
        assert dist[0].tolist() == c["pool_dist"]
        assert (int(visits[0]), int(hops[0]), int(st[0])) == (c["visits"], c["hops"], c["status"])
        idx.close()


def test_padding_and_bad_ids():
    X, adj = path_graph([0, 1, 3, 2, 5, 4])
    adj[2, :] = 0xFFFFFFFF
    q = np.array([[1, 0, 0, 0]], np.float32)
    idx = dev_index(X, adj, 0)
    ref = oracle.beam_search(X, adj, 0, q, 5, 8, max_visits=MV)
    assert_same(run(idx, q, 5, 8), ref, "padding")
    idx.close()
    adj2 = adj.copy()
    adj2[1, 1] = 77          # an id >= n is skipped and reported
    idx = dev_index(X, adj2, 0)
    ref = oracle.beam_search(X, adj2, 0, q, 5, 8, max_visits=MV)
    assert ref[4][0] == oracle.ST_EINVAL
    assert_same(run(idx, q, 5, 8), ref, "bad id")
    idx.close()


def test_host_buffer_entry_point(tiny, tiny_idx):
    Q = tiny["Q"][:100]
    ref = oracle.beam_search(tiny["X"], tiny["adj"], tiny["entry"], Q, 10, 50, max_visits=MV)
    ids, dist, visits, hops, st = tiny_idx.search_host(np.ascontiguousarray(Q), 10, 50)
    got = (ids.numpy().view(np.uint32), dist.numpy(), visits.numpy().view(np.uint32),
           hops.numpy().view(np.uint32), st.numpy())
    assert_same(got, ref, "host entry point")
