"""Seeded synthetic inputs shaped like RoarGraph's cross-modal workloads.

This module is the one piece shared by the CPU oracle (``oracle/``) and the
CUDA path (``paper_2408_08933_gb300``): it draws random inputs and nothing
else. It holds none of the method's arithmetic (no distances, no index
construction, no search); its one graph, ``cluster_graph``, is random
structure used as a search input.

The paper evaluates on Text-to-Image (10M x 200, inner product), LAION
(10M x 512, cosine) and WebVid (2.5M x 512, cosine) (Sec. 5.1, Table 1).
None of those datasets is available here, so these generators stand in for
them with the same shapes and the property the paper is about: the queries
come from a different distribution than the base data (Sec. 3, the
"modality gap"). Every vector is L2-normalised, so cosine and inner product
rank identically.

Recipe (all float32):

* ``C`` mixture means ``mu_c ~ N(0, I_d)``;
* one offset ``delta = offset_norm * u`` with ``u`` a random unit vector;
* base row:  ``c ~ U{0..C-1}``, ``x = normalize(mu_c + noise * g)``;
* query row: ``c' ~ U{0..C-1}``, ``q = normalize(mu_c' + delta + noise * g)``;
* ``g ~ N(0, I_d)`` fresh per row.

Training queries (used to build the index, Alg. 1) and test queries (used
to search) are drawn independently from the same query distribution, as the
paper keeps them disjoint (Sec. 5.1). ID queries (``kind="id_queries"``) are
drawn from the base distribution, for in-distribution comparisons (Sec. 5.4).

Rows are generated in fixed chunks of ``CHUNK`` rows, each from its own
``SeedSequence(SEED, spawn_key=(tag, array, chunk))``, so any row range can be
regenerated without generating the rows before it.
"""
from __future__ import annotations

import dataclasses

import numpy as np

SEED = 20240817
CHUNK = 65536

_ARRAYS = {"means": 0, "offset": 1, "base": 2, "train": 3, "test": 4, "id_queries": 5}


@dataclasses.dataclass(frozen=True)
class Workload:
    """Shape of one synthetic cross-modal workload."""

    name: str
    n: int                 # base vectors |X|
    d: int                 # dimension
    n_train: int           # training queries |T| used by index construction
    n_test: int            # test queries |Q| used by search
    n_comp: int            # mixture components C
    offset_norm: float = 1.5
    noise: float = 0.5
    tag: int = 0           # distinguishes the seed streams of different workloads


# The five workload shapes used by the tests and the benchmark.
TINY = Workload("tiny_10k_d64", n=10_000, d=64, n_train=10_000, n_test=1_000, n_comp=32, tag=1)
BASE_1M_D200 = Workload("base_1m_d200", n=1_000_000, d=200, n_train=1_000_000, n_test=10_000,
                        n_comp=256, tag=2)
BASE_10M_D512 = Workload("base_10m_d512", n=10_000_000, d=512, n_train=1_000_000, n_test=10_000,
                         n_comp=1024, tag=3)
BASE_1M_D512 = Workload("base_1m_d512", n=1_000_000, d=512, n_train=1_000_000, n_test=65_536,
                        n_comp=1024, tag=4)
BASE_10M_D200 = Workload("base_10m_d200", n=10_000_000, d=200, n_train=1_000_000, n_test=10_000,
                         n_comp=256, tag=5)

WORKLOADS = {w.name: w for w in (TINY, BASE_1M_D200, BASE_10M_D512, BASE_1M_D512, BASE_10M_D200)}


def scaled(w: Workload, **kw) -> Workload:
    """A copy of ``w`` with some sizes replaced (same seed streams)."""
    return dataclasses.replace(w, **kw)


def _rng(w: Workload, array: str, chunk: int) -> np.random.Generator:
    ss = np.random.SeedSequence(SEED, spawn_key=(w.tag, _ARRAYS[array], chunk))
    return np.random.Generator(np.random.PCG64(ss))


def _normalize_rows(a: np.ndarray) -> np.ndarray:
    a64 = a.astype(np.float64)
    nrm = np.sqrt((a64 * a64).sum(axis=1, keepdims=True))
    nrm[nrm == 0.0] = 1.0
    return (a64 / nrm).astype(np.float32)


def means(w: Workload) -> np.ndarray:
    """Mixture means ``mu_c``, float32 [C, d]."""
    return _rng(w, "means", 0).standard_normal((w.n_comp, w.d), dtype=np.float32)


def offset(w: Workload) -> np.ndarray:
    """The modality-gap offset ``delta``, float32 [d], norm ``offset_norm``."""
    u = _rng(w, "offset", 0).standard_normal(w.d).astype(np.float64)
    u /= np.sqrt((u * u).sum())
    return (w.offset_norm * u).astype(np.float32)


def _rows(w: Workload, array: str, total: int, lo: int, hi: int | None) -> np.ndarray:
    hi = total if hi is None else hi
    if not (0 <= lo <= hi <= total):
        raise ValueError(f"row range [{lo}, {hi}) outside [0, {total})")
    mu = means(w)
    shift = offset(w) if array in ("train", "test") else None
    out = np.empty((hi - lo, w.d), dtype=np.float32)
    c0, c1 = lo // CHUNK, (hi + CHUNK - 1) // CHUNK

    def one(c):
        r0, r1 = c * CHUNK, min(total, (c + 1) * CHUNK)
        rng = _rng(w, array, c)
        comp = rng.integers(0, w.n_comp, size=r1 - r0)
        g = rng.standard_normal((r1 - r0, w.d), dtype=np.float32)
        v = mu[comp] + np.float32(w.noise) * g
        if shift is not None:
            v += shift
        v = _normalize_rows(v)
        a, b = max(lo, r0), min(hi, r1)
        out[a - lo:b - lo] = v[a - r0:b - r0]

    # Chunks are independent streams: generate them on several threads.
    if c1 - c0 > 2:
        from concurrent.futures import ThreadPoolExecutor
        import os

        with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
            list(ex.map(one, range(c0, c1)))
    else:
        for c in range(c0, c1):
            one(c)
    return out


def base_components(w: Workload) -> np.ndarray:
    """Mixture component of every base row (the same draws as base())."""
    out = np.empty(w.n, dtype=np.int32)
    for c in range((w.n + CHUNK - 1) // CHUNK):
        r0, r1 = c * CHUNK, min(w.n, (c + 1) * CHUNK)
        out[r0:r1] = _rng(w, "base", c).integers(0, w.n_comp, size=r1 - r0)
    return out


def cluster_graph(w: Workload, local: int = 24, far: int = 8, rmax: int = 64,
                  seed_tag: int = 9) -> np.ndarray:
    """A seeded graph with the structure of a navigable index but built
    without any distance: every node links to `local` random members of its
    own mixture component and `far` random nodes anywhere. uint32 [n][rmax],
    duplicates and self loops removed, padded with 0xFFFFFFFF. Used as a
    search input that comes from neither the oracle nor the CUDA library."""
    comp = base_components(w)
    order = np.argsort(comp, kind="stable").astype(np.int64)
    starts = np.searchsorted(comp[order], np.arange(w.n_comp + 1))
    ss = np.random.SeedSequence(SEED, spawn_key=(w.tag, 102, seed_tag))
    rng = np.random.Generator(np.random.PCG64(ss))
    n = w.n
    lo = starts[comp]
    size = starts[comp + 1] - lo
    cand = np.empty((n, local + far), dtype=np.int64)
    cand[:, :local] = order[lo[:, None] + (rng.random((n, local)) * size[:, None]).astype(np.int64)]
    cand[:, local:] = rng.integers(0, n, size=(n, far))
    cand[cand == np.arange(n)[:, None]] = -1
    srt = np.sort(cand, axis=1)
    dup = np.zeros_like(srt, dtype=bool)
    dup[:, 1:] = srt[:, 1:] == srt[:, :-1]
    srt[dup] = -1
    srt = -np.sort(-srt, axis=1)              # valid ids first (descending), -1 at the end
    adj = np.full((n, rmax), 0xFFFFFFFF, dtype=np.uint32)
    k = min(rmax, local + far)
    valid = srt[:, :k] >= 0
    adj[:, :k][valid] = srt[:, :k][valid].astype(np.uint32)
    return adj


def base(w: Workload, lo: int = 0, hi: int | None = None) -> np.ndarray:
    """Base vectors X (rows lo..hi), float32 [rows, d], unit norm."""
    return _rows(w, "base", w.n, lo, hi)


def train_queries(w: Workload, lo: int = 0, hi: int | None = None) -> np.ndarray:
    """Training queries T (OOD), float32 [rows, d], unit norm."""
    return _rows(w, "train", w.n_train, lo, hi)


def test_queries(w: Workload, lo: int = 0, hi: int | None = None) -> np.ndarray:
    """Test queries Q (OOD, disjoint draws from T), float32 [rows, d], unit norm."""
    return _rows(w, "test", w.n_test, lo, hi)


def id_queries(w: Workload, count: int) -> np.ndarray:
    """In-distribution queries drawn like base rows (separate stream)."""
    return _rows(w, "id_queries", count, 0, count)


def uneven_params(count: int, seed_tag: int = 7, k_choices=(1, 10, 100), l_max: int = 500):
    """Per-query (k, L) for the uneven batch: k ~ U(k_choices), L ~ U[max(k,10), l_max]."""
    ss = np.random.SeedSequence(SEED, spawn_key=(seed_tag, 100, 0))
    rng = np.random.Generator(np.random.PCG64(ss))
    k = rng.choice(np.asarray(k_choices, dtype=np.int32), size=count)
    lo = np.maximum(k, 10)
    L = (lo + np.floor(rng.random(count) * (l_max - lo + 1))).astype(np.int32)
    return k.astype(np.int32), L


def poisson_requests(rate_qps: float, duration_s: float, seed_tag: int = 8,
                     size_range=(1, 256), k_choices=(10, 100), l_range=(50, 400)):
    """An open-loop request stream: arrival times (s), sizes, k and L per request.

    Requests arrive as a Poisson process whose query rate is ``rate_qps``
    (the request rate is ``rate_qps`` divided by the mean request size).
    """
    ss = np.random.SeedSequence(SEED, spawn_key=(seed_tag, 101, int(rate_qps)))
    rng = np.random.Generator(np.random.PCG64(ss))
    mean_size = 0.5 * (size_range[0] + size_range[1])
    req_rate = rate_qps / mean_size
    n_req = max(1, int(req_rate * duration_s * 1.2) + 16)
    gaps = rng.exponential(1.0 / req_rate, size=n_req)
    t = np.cumsum(gaps)
    t = t[t < duration_s]
    m = len(t)
    size = rng.integers(size_range[0], size_range[1] + 1, size=m).astype(np.int32)
    k = rng.choice(np.asarray(k_choices, dtype=np.int32), size=m).astype(np.int32)
    L = rng.integers(l_range[0], l_range[1] + 1, size=m).astype(np.int32)
    L = np.maximum(L, k)
    return t, size, k, L
