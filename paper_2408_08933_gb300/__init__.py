"""GB300-native RoarGraph search: Python binding of libroargraph (include/roargraph.h).

The binding only marshals arguments: every step of the search, the build's
dense step and the quantisers run in the library's CUDA kernels. PyTorch
provides device memory and streams. There is no CPU fallback: if the library
is missing, :func:`lib` raises.
"""
from __future__ import annotations

import ctypes
import os

from . import build_ext

NONE_ID = 0xFFFFFFFF
ROAR_OK, ROAR_EINVAL, ROAR_ENOMEM, ROAR_ECUDA, ROAR_EOVERFLOW, ROAR_ETIMEOUT, ROAR_EBUSY = range(7)
ROAR_F32, ROAR_BF16, ROAR_FP8_E4M3 = 0, 1, 2
DTYPE_CODES = {"f32": ROAR_F32, "bf16": ROAR_BF16, "fp8": ROAR_FP8_E4M3}

_lib = None


class ServerCfg(ctypes.Structure):
    """roar_server_cfg (include/roargraph.h)."""
    _fields_ = [("ring_capacity", ctypes.c_int32), ("memory_budget", ctypes.c_int64),
                ("k_max", ctypes.c_int32), ("L_max", ctypes.c_int32), ("team_warps", ctypes.c_int32),
                ("idle_ms", ctypes.c_int32)]


class RoarError(RuntimeError):
    def __init__(self, status: int, where: str):
        lib_ = _lib
        msg = lib_.roar_status_string(status).decode() if lib_ else str(status)
        detail = lib_.roar_last_error().decode() if lib_ else ""
        super().__init__(f"{where}: {msg} ({detail})")
        self.status = status


def lib() -> ctypes.CDLL:
    """Load libroargraph.so (built by ``build_ext.build()``); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(build_ext.LIB):
        raise RuntimeError(f"libroargraph is not built ({build_ext.LIB} missing); "
                           "run __graft_entry__.build() first")
    L = ctypes.CDLL(build_ext.LIB)
    P, i32, i64, u32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
    L.roar_status_string.argtypes = [ctypes.c_int]
    L.roar_status_string.restype = ctypes.c_char_p
    L.roar_last_error.argtypes = []
    L.roar_last_error.restype = ctypes.c_char_p
    L.roar_index_create.argtypes = [i64, i32, P, ctypes.c_int, P, P, P, i32, u32, u32,
                                    ctypes.POINTER(P)]
    L.roar_index_create.restype = ctypes.c_int
    L.roar_index_create_bipartite.argtypes = [i64, i32, P, P, i32, i64, P, P, u32, u32, ctypes.POINTER(P)]
    L.roar_index_create_bipartite.restype = ctypes.c_int
    L.roar_bipartite.argtypes = [P, i64, i32, i64, P, P, P, P, P]
    L.roar_bipartite.restype = ctypes.c_int
    L.roar_index_set_hash_log2.argtypes = [P, i32]
    L.roar_index_set_hash_log2.restype = ctypes.c_int
    L.roar_index_set_tombstones.argtypes = [P, P]
    L.roar_index_set_tombstones.restype = ctypes.c_int
    L.roar_index_destroy.argtypes = [P]
    L.roar_index_destroy.restype = None
    L.roar_search.argtypes = [P, P, i64, i32, i32, P, P, P, P, P, P]
    L.roar_search.restype = ctypes.c_int
    L.roar_search_host.argtypes = [P, P, i64, i32, i32, P, P, P, P, P, P]
    L.roar_search_host.restype = ctypes.c_int
    L.roar_search_uneven.argtypes = [P, P, i64, P, P, P, i32, P, P, P, P, P, P, P]
    L.roar_search_uneven.restype = ctypes.c_int
    L.roar_plan_create.argtypes = [P, P, i64, P, P, P, i32, i32, P, P, P, P, P, P, ctypes.POINTER(P)]
    L.roar_plan_create.restype = ctypes.c_int
    L.roar_plan_launch.argtypes = [P, P]
    L.roar_plan_launch.restype = ctypes.c_int
    L.roar_plan_destroy.argtypes = [P]
    L.roar_plan_destroy.restype = None
    L.roar_index_set_tuning.argtypes = [P, i32, i32, i32, i32]
    L.roar_index_set_tuning.restype = ctypes.c_int
    L.roar_autotune.argtypes = [P, P, i64, i32, i32, i32, P, P, P]
    L.roar_autotune.restype = ctypes.c_int
    L.roar_search_noalloc.argtypes = [i64, i32, P, P, i32, u32, u32, P, i64, i32, i32, P, P, P, P,
                                      P, P]
    L.roar_search_noalloc.restype = ctypes.c_int
    L.roar_server_create.argtypes = [P, ctypes.POINTER(ServerCfg), ctypes.POINTER(P)]
    L.roar_server_create.restype = ctypes.c_int
    L.roar_server_submit.argtypes = [P, P, i32, i32, i32, ctypes.POINTER(ctypes.c_uint64)]
    L.roar_server_submit.restype = ctypes.c_int
    L.roar_server_poll.argtypes = [P, ctypes.c_uint64, i32, P, P, P, P, ctypes.POINTER(ctypes.c_double)]
    L.roar_server_poll.restype = ctypes.c_int
    L.roar_server_stats.argtypes = [P, P]
    L.roar_server_stats.restype = ctypes.c_int
    L.roar_server_ready.argtypes = [P, P, i32, ctypes.POINTER(i32)]
    L.roar_server_ready.restype = ctypes.c_int
    L.roar_server_destroy.argtypes = [P]
    L.roar_server_destroy.restype = None
    L.roar_quantize.argtypes = [P, i64, i32, ctypes.c_int, P, P, P]
    L.roar_quantize.restype = ctypes.c_int
    L.roar_knn.argtypes = [P, i64, P, i64, i32, i32, P, P, P]
    L.roar_knn.restype = ctypes.c_int
    L.roar_knn_set_wait_limit_ns.argtypes = [i64]
    L.roar_knn_set_wait_limit_ns.restype = ctypes.c_int
    L.roar_medoid.argtypes = [P, i64, i32, i32, ctypes.POINTER(u32)]
    L.roar_medoid.restype = ctypes.c_int
    L.roar_acquire.argtypes = [P, i64, i32, P, i64, P, i32, P, i32, i32, P, P, P, P]
    L.roar_acquire.restype = ctypes.c_int
    L.roar_insert.argtypes = [P, i64, i32, P, i32, u32, i64, P, i64, P, P, P, i32, i32, i32, i32, P, P, P]
    L.roar_insert.restype = ctypes.c_int
    L.roar_build_index.argtypes = [P, i64, i32, P, i64, i32, i32, i32, i32, P, P,
                                   ctypes.POINTER(u32), P, P]
    L.roar_build_index.restype = ctypes.c_int
    L.roar_build_index_literal.argtypes = [P, i64, i32, P, i64, i32, i32, i32, P, P, ctypes.POINTER(u32), P, P]
    L.roar_build_index_literal.restype = ctypes.c_int
    _lib = L
    return L


def _check(st: int, where: str):
    if st != ROAR_OK:
        raise RoarError(st, where)


def roar_index_create(n, d, base_f32, trav_dtype, base_trav, scales, adj, rmax, entry,
                      max_visits=0):
    """Raw C-ABI call; pointer arguments are integers (device addresses) or None."""
    h = ctypes.c_void_p()
    _check(lib().roar_index_create(n, d, base_f32, trav_dtype, base_trav, scales, adj, rmax,
                                   entry, max_visits, ctypes.byref(h)), "roar_index_create")
    return h.value


def roar_index_create_bipartite(n, d, base_f32, nout, rn, nt, bi_off, bi_q, entry, max_visits=0):
    """Raw C-ABI call (pointer arguments are device addresses)."""
    h = ctypes.c_void_p()
    _check(lib().roar_index_create_bipartite(n, d, base_f32, nout, rn, nt, bi_off, bi_q, entry, max_visits,
                                             ctypes.byref(h)), "roar_index_create_bipartite")
    return h.value


def roar_bipartite(knn, nt, nqd, n, off, qids, nout, stats=None, stream=None):
    _check(lib().roar_bipartite(knn, nt, nqd, n, off, qids, nout, stats, stream), "roar_bipartite")


def roar_index_set_tombstones(idx, bits):
    _check(lib().roar_index_set_tombstones(idx, bits), "roar_index_set_tombstones")


def roar_index_set_hash_log2(handle, log2):
    _check(lib().roar_index_set_hash_log2(handle, log2), "roar_index_set_hash_log2")


def roar_index_destroy(handle):
    lib().roar_index_destroy(handle)


def roar_search(handle, queries, nq, k, L, ids, dist, visits=None, hops=None, qstatus=None,
                stream=None):
    _check(lib().roar_search(handle, queries, nq, k, L, ids, dist, visits, hops, qstatus, stream),
           "roar_search")


def roar_search_host(handle, queries, nq, k, L, ids, dist, visits=None, hops=None, qstatus=None,
                     stream=None):
    _check(lib().roar_search_host(handle, queries, nq, k, L, ids, dist, visits, hops, qstatus,
                                  stream), "roar_search_host")


def roar_search_uneven(handle, queries, nq, k_dev, L_dev, out_off, L_max, order, ids, dist,
                       visits=None, hops=None, qstatus=None, stream=None):
    _check(lib().roar_search_uneven(handle, queries, nq, k_dev, L_dev, out_off, L_max, order, ids,
                                    dist, visits, hops, qstatus, stream), "roar_search_uneven")


def roar_plan_create(handle, queries, nq, k_dev, L_dev, out_off, L_max, longest_first, ids, dist,
                     visits=None, hops=None, qstatus=None, stream=None):
    p = ctypes.c_void_p()
    _check(lib().roar_plan_create(handle, queries, nq, k_dev, L_dev, out_off, L_max, longest_first,
                                  ids, dist, visits, hops, qstatus, stream, ctypes.byref(p)),
           "roar_plan_create")
    return p.value


def roar_plan_launch(plan, stream=None):
    _check(lib().roar_plan_launch(plan, stream), "roar_plan_launch")


def roar_plan_destroy(plan):
    lib().roar_plan_destroy(plan)


def roar_index_set_tuning(handle, L, team_warps, hash_log2=0, blocks_per_sm_cap=0):
    _check(lib().roar_index_set_tuning(handle, L, team_warps, hash_log2, blocks_per_sm_cap),
           "roar_index_set_tuning")


def roar_autotune(handle, queries, nq, k, L, repeats, results, best, stream=None):
    _check(lib().roar_autotune(handle, queries, nq, k, L, repeats, results, best, stream),
           "roar_autotune")


def roar_search_noalloc(n, d, base_f32, adj, rmax, entry, max_visits, queries, nq, k, L, ids, dist,
                        visits=None, hops=None, qstatus=None, stream=None):
    """Raw C-ABI call of the search that allocates nothing (pointer arguments are integers)."""
    _check(lib().roar_search_noalloc(n, d, base_f32, adj, rmax, entry, max_visits, queries, nq, k,
                                     L, ids, dist, visits, hops, qstatus, stream),
           "roar_search_noalloc")


def roar_server_create(handle, cfg):
    p = ctypes.c_void_p()
    _check(lib().roar_server_create(handle, ctypes.byref(cfg), ctypes.byref(p)), "roar_server_create")
    return p.value


def roar_server_submit(srv, q_host, nq, k, L):
    """Returns the request id, or None when admission refuses it now (ROAR_EBUSY)."""
    rid = ctypes.c_uint64()
    st = lib().roar_server_submit(srv, q_host, nq, k, L, ctypes.byref(rid))
    if st == ROAR_EBUSY:
        return None
    _check(st, "roar_server_submit")
    return rid.value


def server_query_charge(d, k, L):
    """Bytes one query at (k, L) is charged by the serving loop's admission
    (include/roargraph.h, roar_server_create)."""
    lg = 0
    while (1 << lg) < 32 * L:
        lg += 1
    return 4 * d + 8 * k + 24 + 8 * L + (4 << lg)


def roar_server_poll(srv, request_id, timeout_ms, ids=None, dist=None, visits=None, qstatus=None):
    """Returns the latency in seconds when complete, None on ROAR_ETIMEOUT."""
    lat = ctypes.c_double()
    st = lib().roar_server_poll(srv, request_id, timeout_ms, ids, dist, visits, qstatus, ctypes.byref(lat))
    if st == ROAR_ETIMEOUT:
        return None
    _check(st, "roar_server_poll")
    return lat.value


def roar_server_ready(srv, cap=4096):
    """Ids of complete, unreleased requests (oldest first), at most cap."""
    import numpy as np

    ids = np.empty(cap, dtype=np.uint64)
    n = ctypes.c_int32()
    _check(lib().roar_server_ready(srv, ids.ctypes.data, cap, ctypes.byref(n)), "roar_server_ready")
    return ids[:n.value].tolist()


def roar_server_stats(srv):
    import numpy as np

    out = np.zeros(10, dtype=np.float64)
    _check(lib().roar_server_stats(srv, out.ctypes.data), "roar_server_stats")
    return dict(zip(["ring", "submitted", "completed", "released", "launches", "blocks", "team_warps",
                     "running", "inflight_bytes", "memory_budget"], out.tolist()))


def roar_server_destroy(srv):
    lib().roar_server_destroy(srv)


def roar_quantize(X, n, d, dtype, out, scales, stream=None):
    _check(lib().roar_quantize(X, n, d, dtype, out, scales, stream), "roar_quantize")


def roar_knn(T, nt, X, n, d, kk, ids, dist, stream=None):
    _check(lib().roar_knn(T, nt, X, n, d, kk, ids, dist, stream), "roar_knn")


def roar_knn_set_wait_limit_ns(ns):
    """Testing hook: wall-time limit of each bounded wait in roar_knn's kernel
    (ns < 0: the 2 s default; 0: give up at the first incomplete phase)."""
    _check(lib().roar_knn_set_wait_limit_ns(int(ns)), "roar_knn_set_wait_limit_ns")


def roar_acquire(X, n, d, xs, nx, cand, cand_stride, ncand, M, fill, out, out_cnt, sorted_out=None,
                 stream=None):
    _check(lib().roar_acquire(X, n, d, xs, nx, cand, cand_stride, ncand, M, 1 if fill else 0, out, out_cnt,
                              sorted_out, stream), "roar_acquire")


def roar_medoid(X_host, n, d, threads=0):
    e = ctypes.c_uint32()
    _check(lib().roar_medoid(X_host, n, d, threads, ctypes.byref(e)), "roar_medoid")
    return e.value


def roar_build_index(X, n, d, T, nt, nq_depth, M, L_build, threads, adj, stats, stream=None, pj=None):
    e = ctypes.c_uint32()
    _check(lib().roar_build_index(X, n, d, T, nt, nq_depth, M, L_build, threads, adj, pj,
                                  ctypes.byref(e), stats, stream), "roar_build_index")
    return e.value


def _ptr(t):
    return None if t is None else t.data_ptr()


def _stream_ptr(stream):
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


class Index:
    """A resident index over torch CUDA tensors (kept alive by this object).

    base_f32: float32 [n, d]; adj: int32/uint32-compatible [n, rmax] (stored as
    int32 holding uint32 bits, padding -1 == 0xFFFFFFFF); trav: optional BF16
    (int16/uint16 bits or torch.bfloat16) or FP8 (uint8) copy; scales: float32 [n].
    """

    def __init__(self, base_f32, adj, entry, dtype="f32", trav=None, scales=None, max_visits=0):
        import torch

        assert base_f32.is_cuda and base_f32.dtype == torch.float32 and base_f32.is_contiguous()
        assert adj.is_cuda and adj.dtype == torch.int32 and adj.is_contiguous()
        self.base_f32, self.adj, self.trav, self.scales = base_f32, adj, trav, scales
        self.n, self.d = base_f32.shape
        self.rmax = adj.shape[1]
        self.entry = int(entry)
        self.dtype = dtype
        self.handle = roar_index_create(self.n, self.d, _ptr(base_f32), DTYPE_CODES[dtype],
                                        _ptr(trav), _ptr(scales), _ptr(adj), self.rmax, self.entry,
                                        max_visits)

    def set_hash_log2(self, log2: int):
        roar_index_set_hash_log2(self.handle, log2)

    def set_tombstones(self, bits):
        """Deletion bitmap (CUDA int32 [ceil(n/32)] words, bit id & 31 of word
        id >> 5), or None to clear. The tensor is kept alive with the index."""
        self._tomb = bits
        roar_index_set_tombstones(self.handle, _ptr(bits) if bits is not None else None)

    def close(self):
        if getattr(self, "handle", None):
            roar_index_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def search(self, queries, k, L, stream=None, out=None):
        """Search a CUDA float32 [nq, d] batch; returns (ids int32-bits, dist, visits, hops, status)."""
        import torch

        assert queries.is_cuda and queries.dtype == torch.float32 and queries.is_contiguous()
        nq = queries.shape[0]
        dev = queries.device
        if out is None:
            out = (torch.empty((nq, k), dtype=torch.int32, device=dev),
                   torch.empty((nq, k), dtype=torch.float32, device=dev),
                   torch.empty(nq, dtype=torch.int32, device=dev),
                   torch.empty(nq, dtype=torch.int32, device=dev),
                   torch.empty(nq, dtype=torch.int32, device=dev))
        ids, dist, visits, hops, status = out
        roar_search(self.handle, _ptr(queries), nq, k, L, _ptr(ids), _ptr(dist), _ptr(visits),
                    _ptr(hops), _ptr(status), _stream_ptr(stream))
        return out

    def set_tuning(self, L, team_warps, hash_log2=0, blocks_per_sm_cap=0):
        roar_index_set_tuning(self.handle, L, team_warps, hash_log2, blocks_per_sm_cap)

    def autotune(self, queries, k, L, repeats=3, stream=None):
        """Time the 16 launch variants for L's bucket on `queries`; keeps the fastest."""
        import numpy as np

        res = np.zeros(16, dtype=np.float32)
        best = ctypes.c_int32(-1)
        roar_autotune(self.handle, _ptr(queries), queries.shape[0], k, L, repeats, res.ctypes.data,
                      ctypes.byref(best), _stream_ptr(stream))
        return best.value, res

    def uneven_outputs(self, k_host):
        """Output buffers and offsets for per-query k (numpy int32)."""
        import numpy as np
        import torch

        dev = self.base_f32.device
        off = np.zeros(len(k_host), dtype=np.int64)
        off[1:] = np.cumsum(k_host.astype(np.int64))[:-1]
        total = int(k_host.astype(np.int64).sum())
        nq = len(k_host)
        return (torch.from_numpy(off).to(dev), torch.empty(total, dtype=torch.int32, device=dev),
                torch.empty(total, dtype=torch.float32, device=dev),
                torch.empty(nq, dtype=torch.int32, device=dev), torch.empty(nq, dtype=torch.int32, device=dev),
                torch.empty(nq, dtype=torch.int32, device=dev))

    def search_uneven(self, queries, k_dev, L_dev, L_max, out, order=None, stream=None):
        off, ids, dist, visits, hops, status = out
        roar_search_uneven(self.handle, _ptr(queries), queries.shape[0], _ptr(k_dev), _ptr(L_dev),
                           _ptr(off), L_max, _ptr(order), _ptr(ids), _ptr(dist), _ptr(visits),
                           _ptr(hops), _ptr(status), _stream_ptr(stream))
        return out

    def plan_uneven(self, queries, k_dev, L_dev, L_max, out, longest_first=True, stream=None):
        """Capture one uneven search in a CUDA graph; returns a Plan."""
        off, ids, dist, visits, hops, status = out
        h = roar_plan_create(self.handle, _ptr(queries), queries.shape[0], _ptr(k_dev), _ptr(L_dev),
                             _ptr(off), L_max, 1 if longest_first else 0, _ptr(ids), _ptr(dist),
                             _ptr(visits), _ptr(hops), _ptr(status), _stream_ptr(stream))
        return Plan(h, (self, queries, k_dev, L_dev, out))

    def search_host(self, queries, k, L, stream=None, out=None):
        """Host-buffer search (numpy / CPU torch arrays, ideally pinned)."""
        import torch

        q = queries if isinstance(queries, torch.Tensor) else torch.from_numpy(queries)
        assert q.dtype == torch.float32 and q.is_contiguous() and not q.is_cuda
        nq = q.shape[0]
        if out is None:
            out = (torch.empty((nq, k), dtype=torch.int32), torch.empty((nq, k), dtype=torch.float32),
                   torch.empty(nq, dtype=torch.int32), torch.empty(nq, dtype=torch.int32),
                   torch.empty(nq, dtype=torch.int32))
        ids, dist, visits, hops, status = out
        roar_search_host(self.handle, q.data_ptr(), nq, k, L, ids.data_ptr(), dist.data_ptr(),
                         visits.data_ptr(), hops.data_ptr(), status.data_ptr(), _stream_ptr(stream))
        return out


class BipartiteIndex(Index):
    """A search handle over the bipartite graph G_bi (see bipartite()): the
    greedy search through query nodes of Sec. 4.1, for the ablation of
    Sec. 5.4. Searches like Index (FP32, one warp per query)."""

    def __init__(self, base_f32, nout, off, qids, entry, max_visits=0):
        import torch

        assert base_f32.is_cuda and base_f32.dtype == torch.float32 and base_f32.is_contiguous()
        assert nout.is_cuda and nout.dtype == torch.int32 and nout.is_contiguous()
        assert off.dtype == torch.int64 and qids.dtype == torch.int32
        self.base_f32, self.adj, self.trav, self.scales = base_f32, nout, None, None
        self.off, self.qids = off, qids
        self.n, self.d = base_f32.shape
        self.rmax = nout.shape[1]
        self.entry = int(entry)
        self.dtype = "f32"
        self.handle = roar_index_create_bipartite(self.n, self.d, _ptr(base_f32), _ptr(nout), self.rmax,
                                                  nout.shape[0], _ptr(off), _ptr(qids), self.entry, max_visits)


def bipartite(knn, n, stream=None):
    """G_bi of Alg. 1 from CUDA int32 kNN lists [nt, nqd] over n base rows:
    returns (off int64 [n+1], qids int32 [nt], nout int32 [nt, nqd-1], stats)."""
    import numpy as np
    import torch

    assert knn.is_cuda and knn.dtype == torch.int32 and knn.is_contiguous()
    nt, nqd = knn.shape
    dev = knn.device
    off = torch.empty(n + 1, dtype=torch.int64, device=dev)
    qids = torch.empty(nt, dtype=torch.int32, device=dev)
    nout = torch.empty((nt, nqd - 1), dtype=torch.int32, device=dev)
    st = np.zeros(2, dtype=np.int64)
    roar_bipartite(_ptr(knn), nt, nqd, n, _ptr(off), _ptr(qids), _ptr(nout), st.ctypes.data, _stream_ptr(stream))
    return off, qids, nout, {"base_nodes_with_query_edges": int(st[0]), "widest_base_row": int(st[1])}


STAT_KEYS = ["total_s", "knn_s", "projection_s", "enhance_search_s", "reverse_merge_s", "repair_s",
             "pivots", "pj_edges", "final_edges", "unreachable_before_repair", "repairs",
             "unreachable_after_repair"]


def build_index(X, T, nq_depth=100, M=32, L_build=500, threads=0, stream=None, return_pj=False):
    """RoarGraph construction (Alg. 1) of CUDA float32 base rows X [n, d] from
    training queries T [nt, d]. Returns (adj int32 [n, 2M] on X's device, entry,
    stats), and with return_pj also the projected graph G_pj (int32 [n, M])."""
    import numpy as np
    import torch

    assert X.is_cuda and T.is_cuda and X.dtype == torch.float32 and T.dtype == torch.float32
    n, d = X.shape
    adj = torch.empty((n, 2 * M), dtype=torch.int32, device=X.device)
    pj = torch.empty((n, M), dtype=torch.int32, device=X.device) if return_pj else None
    st = np.zeros(16, dtype=np.float64)
    entry = roar_build_index(_ptr(X), n, d, _ptr(T), T.shape[0], nq_depth, M, L_build, threads,
                             _ptr(adj), st.ctypes.data, _stream_ptr(stream),
                             pj=_ptr(pj) if pj is not None else None)
    stats = dict(zip(STAT_KEYS, st.tolist()))
    return (adj, entry, stats, pj) if return_pj else (adj, entry, stats)


def build_index_literal(X, T, nq_depth=100, M=32, L_build=500, stream=None):
    """Alg. 1 in its literal order from the library's GPU parts (see
    roar_build_index_literal): returns (adj int32 [n, 2M], entry, stats,
    G_pj int32 [n, M]). For checking on small inputs."""
    import numpy as np
    import torch

    assert X.is_cuda and T.is_cuda and X.dtype == torch.float32 and T.dtype == torch.float32
    n, d = X.shape
    adj = torch.empty((n, 2 * M), dtype=torch.int32, device=X.device)
    pj = torch.empty((n, M), dtype=torch.int32, device=X.device)
    st = np.zeros(16, dtype=np.float64)
    e = ctypes.c_uint32()
    _check(lib().roar_build_index_literal(_ptr(X), n, d, _ptr(T), T.shape[0], nq_depth, M, L_build, _ptr(adj),
                                          _ptr(pj), ctypes.byref(e), st.ctypes.data, _stream_ptr(stream)),
           "roar_build_index_literal")
    stats = {"total_s": st[0], "pivots": st[6], "pj_edges": st[7], "final_edges": st[8],
             "unreachable_before_repair": st[9], "repairs": st[10]}
    return adj, e.value, stats, pj


def insert(X, adj, entry, n_old, T, pivot, nout, nout_cnt, M, L, window=256, stream=None, return_stats=False):
    """Insert rows n_old.. of CUDA X [n, d] into the CUDA graph adj [n, R]
    (int32, rows >= n_old all -1) through the saved bipartite graph (Sec. 5.7),
    with the result of inserting them one at a time; `window` rows are
    searched per launch (the result does not depend on it). T: host float32
    [nt, d]; pivot: host uint32 [nt]; nout: host uint32 [nt, cap] and
    nout_cnt: host int32 [nt], updated in place. Returns the chosen query per
    new row (numpy int32, -1 when none), and with return_stats a dict of the
    work done."""
    import numpy as np

    n, d = X.shape
    T = np.ascontiguousarray(T, dtype=np.float32)
    pivot = np.ascontiguousarray(pivot, dtype=np.uint32)
    assert nout.dtype == np.uint32 and nout.flags.c_contiguous and nout_cnt.dtype == np.int32
    chosen = np.full(n - n_old, -1, dtype=np.int32)
    st = np.zeros(15, dtype=np.float64)
    _check(lib().roar_insert(_ptr(X), n, d, _ptr(adj), adj.shape[1], entry, n_old, T.ctypes.data, T.shape[0],
                             pivot.ctypes.data, nout.ctypes.data, nout_cnt.ctypes.data, nout.shape[1], M, L,
                             int(window), chosen.ctypes.data, st.ctypes.data, _stream_ptr(stream)), "roar_insert")
    if not return_stats:
        return chosen
    keys = ("windows", "searches", "lists", "lists_redone", "reprune_batches", "rows_repruned", "setup_s",
            "search_s", "lists_s", "apply_s", "reprune_s", "scatter_s", "pick_s", "stops_rewritten",
            "stops_appended")
    return chosen, dict(zip(keys, st.tolist()))


def acquire(X, xs, cand, ncand, M, fill, sorted_out=False, stream=None):
    """Alg. 3 on the GPU for nodes xs [nx] (CUDA int32) with candidate rows
    cand [nx, C] (CUDA int32, -1 = padding) of which ncand [nx] are read.
    Returns (kept [nx, M] int32, counts [nx] int32[, sorted [nx, C] int32])."""
    import torch

    n, d = X.shape
    nx, C = cand.shape
    out = torch.empty((nx, M), dtype=torch.int32, device=X.device)
    cnt = torch.empty(nx, dtype=torch.int32, device=X.device)
    srt = torch.empty((nx, C), dtype=torch.int32, device=X.device) if sorted_out else None
    roar_acquire(_ptr(X), n, d, _ptr(xs), nx, _ptr(cand), C, _ptr(ncand), M, fill, _ptr(out), _ptr(cnt),
                 _ptr(srt) if srt is not None else None, _stream_ptr(stream))
    return (out, cnt, srt) if sorted_out else (out, cnt)


def knn(T, X, kk, stream=None):
    """Exact kNN of CUDA float32 T [nt, d] against X [n, d] (kk <= 128)."""
    import torch

    nt, d = T.shape
    ids = torch.empty((nt, kk), dtype=torch.int32, device=T.device)
    dist = torch.empty((nt, kk), dtype=torch.float32, device=T.device)
    roar_knn(_ptr(T), nt, _ptr(X), X.shape[0], d, kk, _ptr(ids), _ptr(dist), _stream_ptr(stream))
    return ids, dist


def quantize(X, dtype, stream=None):
    """BF16 (returns int16 codes, None) or FP8-E4M3 (uint8 codes, float32 scales) copy of X."""
    import torch

    n, d = X.shape
    if dtype == "bf16":
        out = torch.empty((n, d), dtype=torch.int16, device=X.device)
        roar_quantize(_ptr(X), n, d, ROAR_BF16, _ptr(out), None, _stream_ptr(stream))
        return out, None
    out = torch.empty((n, d), dtype=torch.uint8, device=X.device)
    sc = torch.empty(n, dtype=torch.float32, device=X.device)
    roar_quantize(_ptr(X), n, d, ROAR_FP8_E4M3, _ptr(out), _ptr(sc), _stream_ptr(stream))
    return out, sc


class Plan:
    """A captured uneven search (CUDA graph); keeps its buffers alive."""

    def __init__(self, handle, keep):
        self.handle, self.keep = handle, keep

    def launch(self, stream=None):
        roar_plan_launch(self.handle, _stream_ptr(stream))

    def close(self):
        if self.handle:
            roar_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching search server over an Index (see roar_server_create)."""

    def __init__(self, index, k_max=100, L_max=400, ring_capacity=0, memory_budget=0, team_warps=0,
                 idle_ms=50):
        self.index = index
        cfg = ServerCfg(ring_capacity, memory_budget, k_max, L_max, team_warps, idle_ms)
        self.handle = roar_server_create(index.handle, cfg)
        self.d = index.d

    def submit(self, q, k, L):
        """q: float32 numpy [nq, d]; returns a request id, or None when admission
        refuses it now (no free slots, or its memory charge does not fit)."""
        import numpy as np

        q = np.ascontiguousarray(q, dtype=np.float32)
        return roar_server_submit(self.handle, q.ctypes.data, q.shape[0], k, L)

    def poll(self, rid, nq, k, timeout_ms=0, want_results=True):
        """Returns (latency_s, ids, dist, visits, status) when complete, else None."""
        import numpy as np

        if want_results:
            ids = np.empty((nq, k), np.uint32)
            dist = np.empty((nq, k), np.float32)
            vis = np.empty(nq, np.uint32)
            st = np.empty(nq, np.int32)
            lat = roar_server_poll(self.handle, rid, timeout_ms, ids.ctypes.data, dist.ctypes.data,
                                   vis.ctypes.data, st.ctypes.data)
            return None if lat is None else (lat, ids, dist, vis, st)
        lat = roar_server_poll(self.handle, rid, timeout_ms)
        return None if lat is None else (lat, None, None, None, None)

    def ready(self, cap=4096):
        """Ids of the requests that are complete and not yet polled."""
        return roar_server_ready(self.handle, cap)

    def stats(self):
        return roar_server_stats(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            roar_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
