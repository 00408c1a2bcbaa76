"""RoarGraph CPU oracle -- TEST INFRASTRUCTURE ONLY.

A plain, slow restatement of RoarGraph (PVLDB 17(11), 2024) used to check the
CUDA library: index construction (Alg. 1-3) and beam search (Sec. 4.3), in
``roar_oracle.c``, plus the recall metric (Sec. 2.1.1). Only the tests, the
smoke check and the benchmark's CPU-baseline leg use it. It shares no code
with the CUDA library, and the library never imports it.

Parity status of each function:

* ``dot_fixed`` -- pinned (exact on integer inputs, Higham bound, hand case).
* ``knn_f64`` -- pinned (brute force checked against a library sort).
* ``medoid`` -- pinned (closed form).
* ``f32_to_bf16`` / ``f32_to_e4m3`` / decoders -- pinned (library casts).
* ``acquire_neighbors`` (Alg. 3) -- pinned (hand case, property verifier).
* ``beam_search`` (Sec. 4.3), FP32 -- pinned (hand-traced graphs, exact
  special cases); BF16 / FP8 traversal with the FP32 re-rank of the whole
  pool -- pinned (hand-traced case ``quant_search_fan.json``).
* ``build_index`` (Alg. 1-2, connectivity enhancement) -- pinned (hand-traced
  cases ``projection_circle.json``, ``construction_circle.json``) and by
  invariants.
* ``repair`` (reachability repair, an addition) -- pinned (hand-traced case
  ``repair_circle.json``).
* ``insert`` (Sec. 5.7) -- pinned (hand-traced case ``insertion_circle.json``).
* ``bipartite`` / ``beam_search_bi`` (G_bi of Alg. 1, searched through query
  nodes as in Sec. 4.1; the ablation of Sec. 5.4) -- pinned (hand-traced case
  ``bipartite_search.json``, and on a complete bipartite graph the search
  equals brute force).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "roar_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")

NONE_ID = 0xFFFFFFFF
ST_OK, ST_EINVAL, ST_ENOMEM, ST_EOVERFLOW = 0, 1, 2, 4
DTYPES = {"f32": 0, "bf16": 1, "fp8": 2}

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, no FMA contraction)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-Wall",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i32, i64, u32, f32 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_float
        lib.orc_dot_fixed.argtypes = [P, P, i32]
        lib.orc_dot_fixed.restype = f32
        lib.orc_dist_f64.argtypes = [P, P, i32]
        lib.orc_dist_f64.restype = ctypes.c_double
        lib.orc_f32_to_bf16_n.argtypes = [P, i64, P]
        lib.orc_f32_to_e4m3_n.argtypes = [P, i64, P]
        lib.orc_bf16_to_f32.argtypes = [ctypes.c_uint16]
        lib.orc_bf16_to_f32.restype = f32
        lib.orc_e4m3_to_f32.argtypes = [ctypes.c_uint8]
        lib.orc_e4m3_to_f32.restype = f32
        lib.orc_quant_bf16.argtypes = [P, i64, i32, P]
        lib.orc_quant_e4m3.argtypes = [P, i64, i32, P, P]
        lib.orc_beam_search.argtypes = [i32, P, P, P, i64, i32, P, i32, u32, P, i64, i32, i32, u32,
                                        P, P, P, P, P]
        lib.orc_beam_search.restype = ctypes.c_int
        lib.orc_beam_search_tomb.argtypes = [i32, P, P, P, i64, i32, P, i32, u32, P, i64, i32, i32, u32,
                                             P, P, P, P, P, P]
        lib.orc_beam_search_tomb.restype = ctypes.c_int
        lib.orc_beam_search_trace.argtypes = [P, i64, i32, P, i32, u32, P, i32, u32, P, P, P, P, i64,
                                              P, P]
        lib.orc_beam_search_trace.restype = ctypes.c_int
        lib.orc_knn_f64.argtypes = [P, i64, P, i64, i32, i32, P, P]
        lib.orc_knn_f64.restype = ctypes.c_int
        lib.orc_medoid.argtypes = [P, i64, i32]
        lib.orc_medoid.restype = i64
        lib.orc_acquire_neighbors.argtypes = [P, i64, i32, u32, P, i32, i32, i32, P]
        lib.orc_acquire_neighbors.restype = i32
        lib.orc_acquire_neighbors_f32.argtypes = [P, i64, i32, u32, P, i32, i32, i32, P]
        lib.orc_acquire_neighbors_f32.restype = i32
        lib.orc_insert.argtypes = [P, i64, i32, P, i32, u32, i64, P, i64, P, P, P, i32, i32, i32, u32, P]
        lib.orc_insert.restype = i32
        lib.orc_bipartite.argtypes = [P, i64, i32, i64, P, P]
        lib.orc_bipartite.restype = ctypes.c_int
        lib.orc_beam_search_bi.argtypes = [P, i64, i32, P, i64, i32, u32, P, i64, i32, i32, u32, P, P, P, P, P]
        lib.orc_beam_search_bi.restype = ctypes.c_int
        lib.orc_repair.argtypes = [P, i64, i32, P, i32, u32, P]
        lib.orc_repair.restype = i64
        lib.orc_build.argtypes = [P, i64, i64, i32, P, i32, i32, i32, u32, P, P, P]
        lib.orc_build.restype = ctypes.c_int
        lib.orc_build_prec.argtypes = [P, i64, i64, i32, P, i32, i32, i32, u32, P, P, P, i32]
        lib.orc_build_prec.restype = ctypes.c_int
        _lib = lib
        return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float32)


def dot_fixed(q, x) -> np.float32:
    """<q, x> in FP32 in the fixed 32-lane order (see roar_oracle.c)."""
    q, x = _f32(q), _f32(x)
    assert q.shape == x.shape and q.ndim == 1
    return np.float32(_load().orc_dot_fixed(_p(q), _p(x), q.shape[0]))


def dist_f64(a, b) -> float:
    a, b = _f32(a), _f32(b)
    return float(_load().orc_dist_f64(_p(a), _p(b), a.shape[0]))


def f32_to_bf16(a) -> np.ndarray:
    a = _f32(a).ravel()
    out = np.empty(a.shape, dtype=np.uint16)
    _load().orc_f32_to_bf16_n(_p(a), a.size, _p(out))
    return out


def f32_to_e4m3(a) -> np.ndarray:
    a = _f32(a).ravel()
    out = np.empty(a.shape, dtype=np.uint8)
    _load().orc_f32_to_e4m3_n(_p(a), a.size, _p(out))
    return out


def bf16_to_f32(code: int) -> float:
    return float(_load().orc_bf16_to_f32(code))


def e4m3_to_f32(code: int) -> float:
    return float(_load().orc_e4m3_to_f32(code))


def quant_bf16(X) -> np.ndarray:
    X = _f32(X)
    out = np.empty(X.shape, dtype=np.uint16)
    _load().orc_quant_bf16(_p(X), X.shape[0], X.shape[1], _p(out))
    return out


def quant_e4m3(X):
    X = _f32(X)
    out = np.empty(X.shape, dtype=np.uint8)
    sc = np.empty(X.shape[0], dtype=np.float32)
    _load().orc_quant_e4m3(_p(X), X.shape[0], X.shape[1], _p(out), _p(sc))
    return out, sc


def knn_f64(Q, X, k: int):
    """Exact top-k by delta = -<q, x> in FP64, ties to the lower id."""
    Q, X = _f32(Q), _f32(X)
    nq, d = Q.shape
    ids = np.empty((nq, k), dtype=np.uint32)
    dist = np.empty((nq, k), dtype=np.float64)
    rc = _load().orc_knn_f64(_p(Q), nq, _p(X), X.shape[0], d, k, _p(ids), _p(dist))
    if rc != 0:
        raise ValueError(f"orc_knn_f64 failed: {rc}")
    return ids, dist


def medoid(X) -> int:
    X = _f32(X)
    return int(_load().orc_medoid(_p(X), X.shape[0], X.shape[1]))


def acquire_neighbors(X, x: int, cand, M: int, fill: bool):
    """Alg. 3 with ``cand`` already in the caller's order (sorted by delta(x, .))."""
    X = _f32(X)
    cand = np.ascontiguousarray(cand, dtype=np.uint32)
    res = np.empty(max(M, 1), dtype=np.uint32)
    r = _load().orc_acquire_neighbors(_p(X), X.shape[0], X.shape[1], x, _p(cand), cand.size, M,
                                      1 if fill else 0, _p(res))
    if r < 0:
        raise ValueError("orc_acquire_neighbors: bad arguments")
    return res[:r].copy()


def acquire_neighbors_f32(X, x: int, cand, M: int, fill: bool):
    """Alg. 3 with FP32 fixed-order distances (delta = -dot_fixed), ``cand`` in
    the caller's order. Same steps as acquire_neighbors; only the precision of
    the keep / drop comparisons differs."""
    X = _f32(X)
    cand = np.ascontiguousarray(cand, dtype=np.uint32)
    res = np.empty(max(M, 1), dtype=np.uint32)
    r = _load().orc_acquire_neighbors_f32(_p(X), X.shape[0], X.shape[1], x, _p(cand), cand.size, M,
                                          1 if fill else 0, _p(res))
    if r < 0:
        raise ValueError("orc_acquire_neighbors_f32: bad arguments")
    return res[:r].copy()


def insert(X, adj, entry: int, n_old: int, T, pivot, nout, nout_cnt, M: int, L: int, *, max_visits: int):
    """Insertion through the saved bipartite graph (Sec. 5.7) of rows n_old..n-1
    of X into the graph adj [n][R] (rows >= n_old empty). pivot [nt]: each
    training query's nearest base row; nout [nt][cap] / nout_cnt [nt]: N_out
    lists; max_visits: the visit cap of each new row's search. Returns (adj,
    nout, nout_cnt, chosen_q) updated copies."""
    X = _f32(X)
    T = _f32(T)
    adj = np.ascontiguousarray(adj, dtype=np.uint32).copy()
    nout = np.ascontiguousarray(nout, dtype=np.uint32).copy()
    nout_cnt = np.ascontiguousarray(nout_cnt, dtype=np.int32).copy()
    pivot = np.ascontiguousarray(pivot, dtype=np.uint32)
    n, d = X.shape
    chosen = np.full(n - n_old, -1, dtype=np.int32)
    rc = _load().orc_insert(_p(X), n, d, _p(adj), adj.shape[1], entry, n_old, _p(T), T.shape[0], _p(pivot),
                            _p(nout), _p(nout_cnt), nout.shape[1], M, L, max_visits, _p(chosen))
    if rc != 0:
        raise ValueError(f"orc_insert failed: {rc}")
    return adj, nout, nout_cnt, chosen


def repair(X, adj, entry: int):
    """Reachability repair (an addition to Alg. 1; see roar_oracle.c) of a
    graph adj [n][R] with compact rows. Returns (repaired copy, repairs,
    nodes unreachable before the first repair)."""
    X = _f32(X)
    adj = np.ascontiguousarray(adj, dtype=np.uint32).copy()
    n, d = X.shape
    u0 = np.zeros(1, dtype=np.int64)
    r = _load().orc_repair(_p(X), n, d, _p(adj), adj.shape[1], entry, _p(u0))
    if r < 0:
        raise MemoryError("orc_repair")
    return adj, int(r), int(u0[0])


def build_index(X, knn_ids, M: int, L: int, entry: int, precision: str = "f64"):
    """Alg. 1: bipartite graph, projection (Alg. 2), connectivity enhancement,
    then reachability repair. Returns (final adj [n][2M], G_pj [n][M], stats).
    precision "f64": every construction distance in FP64; "f32": the search's
    fixed-order FP32 dot (the precision a GPU construction decides in), same
    steps."""
    X = _f32(X)
    knn_ids = np.ascontiguousarray(knn_ids, dtype=np.uint32)
    n, d = X.shape
    nt, nqd = knn_ids.shape
    adj = np.empty((n, 2 * M), dtype=np.uint32)
    pj = np.empty((n, M), dtype=np.uint32)
    stats = np.zeros(8, dtype=np.int64)
    prec = {"f64": 0, "f32": 1}[precision]
    rc = _load().orc_build_prec(_p(X), n, nt, d, _p(knn_ids), nqd, M, L, entry, _p(pj), _p(adj),
                                _p(stats), prec)
    if rc != 0:
        raise RuntimeError(f"orc_build failed: {rc}")
    keys = ["pivots", "proj_reprunes", "ce_reprunes", "repairs", "pj_edges", "final_edges",
            "isolated_in_pj", "unreachable_before_repair"]
    return adj, pj, dict(zip(keys, (int(s) for s in stats)))


def pack_tombstones(deleted) -> np.ndarray:
    """Bitmap (uint32 words, bit id & 31 of word id >> 5) of a boolean mask."""
    deleted = np.asarray(deleted, dtype=bool)
    words = np.zeros((deleted.size + 31) // 32, dtype=np.uint32)
    idx = np.nonzero(deleted)[0]
    np.bitwise_or.at(words, idx >> 5, (np.uint32(1) << (idx & 31).astype(np.uint32)))
    return words


def beam_search(X32, adj, entry: int, Q, k: int, L: int, max_visits: int = 1 << 20,
                dtype: str = "f32", Xt=None, scales=None, tomb=None):
    """Beam search (Sec. 4.3) for every row of Q.

    dtype "f32": traversal and result on X32. "bf16" / "fp8": traversal on the
    quantised copy ``Xt`` (uint16 / uint8 codes, FP8 with per-row ``scales``),
    then the whole final pool is re-ranked with FP32 distances. ``tomb``: None
    or a deletion bitmap (pack_tombstones); deleted rows route but are not
    answers (Sec. 5.7).
    Returns ids [nq][k] (uint32), dist [nq][k] (float32), visits, hops, status.
    """
    X32 = _f32(X32)
    adj = np.ascontiguousarray(adj, dtype=np.uint32)
    Q = _f32(Q).reshape(-1, X32.shape[1])
    n, d = X32.shape
    nq = Q.shape[0]
    code = DTYPES[dtype]
    if code == 0:
        Xt_arr, sc = X32, None
    else:
        Xt_arr = np.ascontiguousarray(Xt)
        assert Xt_arr.shape == X32.shape
        sc = _f32(scales) if scales is not None else None
    ids = np.empty((nq, k), dtype=np.uint32)
    dist = np.empty((nq, k), dtype=np.float32)
    visits = np.empty(nq, dtype=np.uint32)
    hops = np.empty(nq, dtype=np.uint32)
    status = np.empty(nq, dtype=np.int32)
    tw = None if tomb is None else np.ascontiguousarray(tomb, dtype=np.uint32)
    rc = _load().orc_beam_search_tomb(code, _p(Xt_arr), _p(sc), _p(X32), n, d, _p(adj), adj.shape[1],
                                      entry, _p(Q), nq, k, L, max_visits, _p(tw), _p(ids), _p(dist),
                                      _p(visits), _p(hops), _p(status))
    if rc != 0:
        raise ValueError(f"orc_beam_search failed: {rc}")
    return ids, dist, visits, hops, status


def bipartite(knn_ids, n: int):
    """G_bi of Alg. 1 as CSR: (off [n+1] int64, qids [nt] uint32), B(x) =
    qids[off[x]:off[x+1]] = every training query whose nearest base row is x,
    ascending. N_out(t) is knn_ids[t, 1:]."""
    knn_ids = np.ascontiguousarray(knn_ids, dtype=np.uint32)
    nt, nqd = knn_ids.shape
    off = np.empty(n + 1, dtype=np.int64)
    qids = np.empty(max(nt, 1), dtype=np.uint32)
    rc = _load().orc_bipartite(_p(knn_ids), nt, nqd, n, _p(off), _p(qids))
    if rc != 0:
        raise ValueError(f"orc_bipartite failed: {rc}")
    return off, qids[:nt]


def beam_search_bi(X, knn_ids, entry: int, Q, k: int, L: int, max_visits: int = 1 << 20):
    """Beam search on G_bi (base nodes scored, routed through query nodes; see
    roar_oracle.c). Returns ids, dist, visits, hops, status as beam_search."""
    X = _f32(X)
    knn_ids = np.ascontiguousarray(knn_ids, dtype=np.uint32)
    Q = _f32(Q).reshape(-1, X.shape[1])
    n, d = X.shape
    nt, nqd = knn_ids.shape
    nq = Q.shape[0]
    ids = np.empty((nq, k), dtype=np.uint32)
    dist = np.empty((nq, k), dtype=np.float32)
    visits = np.empty(nq, dtype=np.uint32)
    hops = np.empty(nq, dtype=np.uint32)
    status = np.empty(nq, dtype=np.int32)
    rc = _load().orc_beam_search_bi(_p(X), n, d, _p(knn_ids), nt, nqd, entry, _p(Q), nq, k, L, max_visits,
                                    _p(ids), _p(dist), _p(visits), _p(hops), _p(status))
    if rc != 0:
        raise ValueError(f"orc_beam_search_bi failed: {rc}")
    return ids, dist, visits, hops, status


def beam_search_trace(X32, adj, entry: int, q, L: int, max_visits: int = 1 << 20):
    """One FP32 query; returns (pool ids, pool dists, expansion order, visits, hops, status)."""
    X32 = _f32(X32)
    adj = np.ascontiguousarray(adj, dtype=np.uint32)
    q = _f32(q)
    n, d = X32.shape
    pid = np.empty(L, dtype=np.uint32)
    pdist = np.empty(L, dtype=np.float32)
    psize = np.zeros(1, dtype=np.int32)
    cap = 4 * n + 16
    trace = np.empty(cap, dtype=np.uint32)
    visits = np.zeros(1, dtype=np.uint32)
    hops = np.zeros(1, dtype=np.uint32)
    st = _load().orc_beam_search_trace(_p(X32), n, d, _p(adj), adj.shape[1], entry, _p(q), L,
                                       max_visits, _p(pid), _p(pdist), _p(psize), _p(trace), cap,
                                       _p(visits), _p(hops))
    s = int(psize[0])
    h = int(hops[0])
    return pid[:s].copy(), pdist[:s].copy(), trace[:min(h, cap)].copy(), int(visits[0]), h, st


def recall_at_k(ids, gt_ids, k: int) -> float:
    """Mean of |S intersect KNN(q)| / k over queries (Sec. 2.1.1)."""
    ids = np.asarray(ids)[:, :k]
    gt = np.asarray(gt_ids)[:, :k]
    hits = 0
    for a, b in zip(ids, gt):
        hits += len(set(a.tolist()) & set(b.tolist()))
    return hits / (k * ids.shape[0])
