"""Serving loop: continuous batching into one persistent search kernel.

Each query served in a mixed stream is bit-identical to searching it alone
and to the oracle's beam search (Sec. 4.3) with its request's k and L;
admission charges each request the memory its queries need."""
import time

import numpy as np
import pytest

import oracle
import paper_2408_08933_gb300 as pkg
import roarsynth as rs
from gpu_util import dev_index, run

pytestmark = pytest.mark.gpu
MV = 16384


@pytest.fixture(scope="module")
def two_handles(tiny):
    serve = dev_index(tiny["X"], tiny["adj"], tiny["entry"], max_visits=MV)
    ref = dev_index(tiny["X"], tiny["adj"], tiny["entry"], max_visits=MV)
    yield serve, ref
    serve.close()
    ref.close()


def _drain(srv, pending, timeout_s=30.0):
    out = {}
    t_end = time.time() + timeout_s
    while pending and time.time() < t_end:
        for rid in list(pending):
            nq, k = pending[rid]
            r = srv.poll(rid, nq, k, timeout_ms=0)
            if r is not None:
                out[rid] = r
                del pending[rid]
        time.sleep(0.0005)
    assert not pending, f"{len(pending)} requests never completed"
    return out


def test_mixed_stream_equals_alone(tiny, two_handles):
    serve, ref = two_handles
    srv = pkg.Server(serve, k_max=100, L_max=400, ring_capacity=4096, idle_ms=20)
    _, sizes, ks, Ls = rs.poisson_requests(3e5, 0.002, seed_tag=41, size_range=(1, 40))
    Q = tiny["Q"]
    pending, meta, qpos = {}, {}, 0
    for nq, k, L in zip(sizes, ks, Ls):
        nq = int(nq)
        q = Q[qpos % 900: qpos % 900 + nq]
        nq = q.shape[0]
        rid = srv.submit(q, int(k), int(L))
        assert rid is not None
        pending[rid] = (nq, int(k))
        meta[rid] = (q, int(k), int(L))
        qpos += nq
    results = _drain(srv, pending)
    for rid, (lat, ids, dist, vis, st) in results.items():
        q, k, L = meta[rid]
        alone = run(ref, q, k, L)
        assert np.array_equal(ids, alone[0]) and np.array_equal(dist, alone[1])
        assert np.array_equal(vis, alone[2]) and np.array_equal(st, alone[4])
        o_ids, o_dist, o_vis, _, o_st = oracle.beam_search(tiny["X"], tiny["adj"], tiny["entry"], q, k, L,
                                                           max_visits=MV)
        assert np.array_equal(ids, o_ids) and np.array_equal(vis, o_vis) and np.array_equal(st, o_st)
        assert np.allclose(dist, o_dist, rtol=1e-6, atol=0)
        assert lat > 0
    s = srv.stats()
    assert s["completed"] == s["submitted"] == qpos
    srv.close()


def test_admission_refuses_when_ring_is_full(tiny, two_handles):
    serve, _ = two_handles
    srv = pkg.Server(serve, k_max=10, L_max=64, ring_capacity=64, idle_ms=20)
    Q = tiny["Q"]
    with pytest.raises(pkg.RoarError):
        srv.submit(Q[:65], 10, 32)                      # more queries than the ring holds
    a = srv.submit(Q[:64], 10, 32)
    assert a is not None
    assert srv.submit(Q[:1], 10, 32) is None           # no room until released
    r = None
    t_end = time.time() + 10
    while r is None and time.time() < t_end:
        r = srv.poll(a, 64, 10, timeout_ms=50)
    assert r is not None
    assert srv.submit(Q[:1], 10, 32) is not None       # released slots are reused
    with pytest.raises(pkg.RoarError):
        srv.poll(a, 64, 10, timeout_ms=0)              # already released
    with pytest.raises(pkg.RoarError):
        srv.submit(Q[:1], 20, 32)                       # k above k_max
    srv.close()


def test_idle_exit_and_relaunch(tiny, two_handles):
    serve, ref = two_handles
    srv = pkg.Server(serve, k_max=10, L_max=64, ring_capacity=256, idle_ms=5)
    Q = tiny["Q"]
    a = srv.submit(Q[:8], 10, 50)
    r = _drain(srv, {a: (8, 10)})
    time.sleep(0.2)                                     # teams exit after 5 ms idle
    s = srv.stats()
    assert s["running"] == 0.0
    b = srv.submit(Q[8:16], 10, 50)
    r2 = _drain(srv, {b: (8, 10)})
    assert srv.stats()["launches"] >= 2
    assert np.array_equal(r2[b][1], run(ref, Q[8:16], 10, 50)[0])
    srv.close()


def test_poll_timeout_is_bounded(tiny, two_handles):
    serve, _ = two_handles
    srv = pkg.Server(serve, k_max=10, L_max=400, ring_capacity=2048, idle_ms=20)
    rid = srv.submit(tiny["Q"][:1000], 10, 400)
    t0 = time.time()
    first = srv.poll(rid, 1000, 10, timeout_ms=0)      # may or may not be done yet
    assert time.time() - t0 < 1.0
    if first is None:
        assert _drain(srv, {rid: (1000, 10)})
    srv.close()


def test_bf16_serving_matches_oracle(tiny):
    """The serving form the benchmark runs: BF16 traversal + FP32 re-rank,
    mixed (k, L) requests in flight together, each result the oracle's."""
    X = tiny["X"]
    codes = oracle.quant_bf16(X)
    idx = dev_index(X, tiny["adj"], tiny["entry"], dtype="bf16", trav=codes.view(np.int16), max_visits=MV)
    srv = pkg.Server(idx, k_max=100, L_max=400, ring_capacity=2048, idle_ms=20)
    Q = tiny["Q"]
    pending, meta = {}, {}
    rng = np.random.default_rng(43)
    for i in range(24):
        nq = int(rng.integers(1, 30))
        k = int(rng.choice([10, 100]))
        L = int(rng.integers(max(k, 50), 401))
        q = Q[(37 * i) % 900:(37 * i) % 900 + nq]
        rid = srv.submit(q, k, L)
        assert rid is not None
        pending[rid] = (q.shape[0], k)
        meta[rid] = (q, k, L)
    for rid, (lat, ids, dist, vis, st) in _drain(srv, pending).items():
        q, k, L = meta[rid]
        o = oracle.beam_search(X, tiny["adj"], tiny["entry"], q, k, L, max_visits=MV, dtype="bf16", Xt=codes)
        assert np.array_equal(ids, o[0]) and np.array_equal(vis, o[2]) and np.array_equal(st, o[4])
        assert np.allclose(dist, o[1], rtol=1e-6, atol=0)
    srv.close()
    idx.close()


def test_admission_by_memory(tiny, two_handles):
    """Under a memory budget a request is admitted only if its charge (ring
    slot at its k, pool 8L, exact visited table for width L, per query) fits
    beside the requests in flight: with a small-L request in flight a large-L
    one is refused while another small-L one is admitted; once released, the
    large one fits. A request over the whole budget is an error."""
    serve, ref = two_handles
    d = tiny["X"].shape[1]
    small, large = pkg.server_query_charge(d, 10, 50), pkg.server_query_charge(d, 10, 400)
    assert large > 7 * small
    budget = 8 * large
    srv = pkg.Server(serve, k_max=100, L_max=400, memory_budget=budget, idle_ms=20)
    Q = tiny["Q"]
    a = srv.submit(Q[:8], 10, 50)
    assert a is not None
    assert srv.submit(Q[8:16], 10, 400) is None          # 8 small + 8 large > budget
    c = srv.submit(Q[16:24], 10, 50)                      # 16 small fits
    assert c is not None
    assert srv.stats()["inflight_bytes"] == 16 * small
    with pytest.raises(pkg.RoarError):
        srv.submit(Q[:9], 10, 400)                        # 9 large > the whole budget
    got = _drain(srv, {a: (8, 10), c: (8, 10)})
    assert srv.stats()["inflight_bytes"] == 0
    b = srv.submit(Q[8:16], 10, 400)
    assert b is not None
    got.update(_drain(srv, {b: (8, 10)}))
    for rid, (q, L) in {a: (Q[:8], 50), c: (Q[16:24], 50), b: (Q[8:16], 400)}.items():
        assert np.array_equal(got[rid][1], run(ref, q, 10, L)[0])
    srv.close()


def test_ready_lists_completed_requests(tiny, two_handles):
    """ready() names exactly the complete, unpolled requests, oldest first;
    polling them releases them."""
    serve, ref = two_handles
    srv = pkg.Server(serve, k_max=10, L_max=100, ring_capacity=1024, idle_ms=20)
    Q = tiny["Q"]
    rids = [srv.submit(Q[8 * i:8 * i + 8], 10, 50) for i in range(6)]
    assert all(r is not None for r in rids)
    t_end = time.time() + 10
    while time.time() < t_end and len(srv.ready()) < len(rids):
        time.sleep(0.001)
    ready = srv.ready()
    assert ready == sorted(rids)
    for rid in ready[:3]:
        r = srv.poll(rid, 8, 10, timeout_ms=0)
        i = rids.index(rid)
        assert np.array_equal(r[1], run(ref, Q[8 * i:8 * i + 8], 10, 50)[0])
    assert srv.ready() == sorted(rids)[3:]
    assert srv.ready(cap=1) == sorted(rids)[3:4]
    for rid in srv.ready():
        srv.poll(rid, 8, 10, timeout_ms=0)
    assert srv.ready() == []
    srv.close()
