"""Benchmark: batched RoarGraph beam search on one GB300 (plain FP32 and BF16/FP8 + FP32 re-rank).

Workload (default): base 1,000,000 x d=200 FP32, 1,000,000 training queries and
10,000 test queries from the seeded OOD mixture generator (256 components,
offset norm 1.5), index built with kNN depth 100, M = 32, L_build = 500.
The L sweep picks the smallest beam width whose recall@10 reaches 0.90; one
step is one search of the 10,000 test queries at that L (k = 10).

The base rows (800 MB) are far larger than L2 (129 MB), so no L2 flush is
needed between steps. Prints ONE JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

L_SWEEP = [10, 20, 30, 40, 50, 60, 70, 80, 90, 100, 110, 120, 150, 200, 300, 400, 500, 700, 1024]
TARGET_RECALL = 0.90
METRIC = "QPS at recall@10=0.90 (plain FP32 vs BF16/FP8+rerank); serving p50/p99 ms"
CACHE_DIR = os.environ.get("ROAR_BENCH_CACHE", "/tmp/roar_bench_cache")


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = float(p[2])
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(value: float, device=None) -> float:
    """The job's time is the slowest rank's (replicas: no other exchange).
    Without an initialised process group this is the value itself."""
    import torch
    import torch.distributed as tdist

    if not (tdist.is_available() and tdist.is_initialized()) or tdist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device if device is not None else "cpu")
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def _src_hash(paths):
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def _setup(w, torch, pkg, rs, log):
    """Generate the workload, build (or load) the index, ground truth and L sweep."""
    dev = torch.device("cuda", torch.cuda.current_device())
    key = _src_hash(["roarsynth/__init__.py", "paper_2408_08933_gb300/csrc/roar_build.cpp",
                     "paper_2408_08933_gb300/csrc/roar_knn.cu", "paper_2408_08933_gb300/csrc/roar_knn_tc.cu",
                     "paper_2408_08933_gb300/csrc/roar_search_kernel.cuh",
                     "paper_2408_08933_gb300/csrc/roar_search.cu"])
    cache = os.path.join(CACHE_DIR, f"{w.name}_{w.n}_{w.n_train}_{w.n_test}_{w.n_comp}_{w.offset_norm}_{w.noise}_{key}.npz")
    t0 = time.time()
    X = rs.base(w)
    Q = rs.test_queries(w)
    log(f"generated base/test in {time.time() - t0:.1f}s")
    Xd = torch.from_numpy(X).to(dev)
    Qd = torch.from_numpy(Q).to(dev)
    if os.path.exists(cache):
        z = np.load(cache)
        adj = torch.from_numpy(z["adj"]).to(dev)
        entry = int(z["entry"])
        gt = z["gt"]
        stats = json.loads(str(z["stats"]))
        log(f"loaded index from {cache}")
    else:
        t0 = time.time()
        T = rs.train_queries(w)
        Td = torch.from_numpy(T).to(dev)
        log(f"generated training queries in {time.time() - t0:.1f}s")
        adj, entry, stats = pkg.build_index(Xd, Td, nq_depth=100, M=32, L_build=500)
        del Td, T
        log(f"built index: {json.dumps(stats)}")
        gi, _ = pkg.knn(Qd, Xd, 10)
        torch.cuda.synchronize()
        gt = gi.cpu().numpy().view(np.uint32)
        try:
            os.makedirs(CACHE_DIR, exist_ok=True)
            np.savez(cache + ".tmp.npz", adj=adj.cpu().numpy(), entry=entry, gt=gt,
                     stats=json.dumps(stats))
            os.replace(cache + ".tmp.npz", cache)
        except Exception as e:  # cache is an optimisation only
            log(f"cache write failed: {e}")
    return dev, X, Q, Xd, Qd, adj, entry, gt, stats


def _recall(ids, gt, k=10):
    ids = ids[:, :k]
    gt = gt[:, :k]
    hit = (ids[:, :, None] == gt[:, None, :]).any(axis=2).sum()
    return float(hit) / (k * ids.shape[0])


def _sweep(idx, Qd, gt, torch, sweep):
    out = {}
    for L in sweep:
        ids, dist, visits, hops, st = idx.search(Qd, 10, L)
        torch.cuda.synchronize()
        r = _recall(ids.cpu().numpy().view(np.uint32), gt)
        out[L] = dict(recall=r, visits=float(visits.float().mean()), hops=float(hops.float().mean()),
                      overflow=int((st != 0).sum()))
    return out


def _pick_L(sweep):
    """Smallest L reaching the target recall; if none does, the L with the
    highest recall (reported with recall_target_reached = false)."""
    for L in sorted(sweep):
        if sweep[L]["recall"] >= TARGET_RECALL:
            return L, True
    return max(sweep, key=lambda L: (sweep[L]["recall"], -L)), False


def _time_steps(idx, Qd, L, steps, warmup, torch):
    s = torch.cuda.current_stream()
    out = None
    for _ in range(warmup):
        out = idx.search(Qd, 10, L, out=out)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for a, b in ev:
        a.record(s)
        out = idx.search(Qd, 10, L, out=out)
        b.record(s)
    torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in ev]
    return ms, out


def _algorithmic_bytes(visits, hops, deg_mean, d, elem_bytes, scale_bytes, k_rerank_L=None):
    """Bytes the method must move per query: visited rows, adjacency rows read,
    the query; plus the FP32 re-rank rows for the reduced-precision forms."""
    b = visits * (d * elem_bytes + scale_bytes) + hops * deg_mean * 4 + 4 * d
    if k_rerank_L is not None:
        b = b + k_rerank_L * d * 4
    return b


def _cpu_baseline(X, adj_np, entry, Q, L, budget_s=12.0):
    """The oracle's beam search on the host cores over a bounded sample of the
    test queries. Returns (baseline dict, the oracle's results for Q[:n])."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor

    cores = os.cpu_count() or 1
    t0 = time.time()
    oracle.beam_search(X, adj_np, entry, Q[:8], 10, L, max_visits=16384)
    per_q = max(1e-5, (time.time() - t0) / 8)
    n = int(min(len(Q), max(cores * 4, budget_s * cores / per_q)))
    chunks = [c for c in np.array_split(np.arange(n), cores * 4) if len(c)]

    def work(ix):
        return oracle.beam_search(X, adj_np, entry, Q[ix], 10, L, max_visits=16384)

    t0 = time.time()
    with ThreadPoolExecutor(max_workers=cores) as ex:
        parts = list(ex.map(work, chunks))
    dt = time.time() - t0
    ref = tuple(np.concatenate([p[i] for p in parts]) for i in range(5))
    return ({"value": n / dt, "unit": "queries/s", "cores": cores, "kind": "oracle",
             "sample": f"the first {n} of the {len(Q)} test queries at L={L}, k=10, "
                       f"{len(chunks)} chunks on {cores} threads"}, ref)


def _parity(gpu_out, ref):
    """Timed GPU results against the oracle's, query by query: ids, visits,
    hops and status exact, distances within 1e-6 relative."""
    n = ref[0].shape[0]
    ids = gpu_out[0][:n].cpu().numpy().view(np.uint32)
    dist = gpu_out[1][:n].cpu().numpy()
    vis = gpu_out[2][:n].cpu().numpy().view(np.uint32)
    hops = gpu_out[3][:n].cpu().numpy().view(np.uint32)
    st = gpu_out[4][:n].cpu().numpy()
    bad = ~np.all(ids == ref[0], axis=1)
    bad |= (vis != ref[2]) | (hops != ref[3]) | (st != ref[4])
    fin = np.isfinite(ref[1])
    derr = np.where(fin, np.abs(dist.astype(np.float64) - ref[1]) / np.maximum(np.abs(ref[1]), 1e-30), 0.0)
    bad |= np.any(derr > 1e-6, axis=1) | np.any(np.isfinite(dist) != fin, axis=1)
    return {"checked": int(n), "mismatches": int(bad.sum()),
            "compared": "ids, visits, hops, status exact; distances within 1e-6 relative",
            "against": "oracle.beam_search on the timed index and queries", "max_rel_dist_err": float(derr.max())}


def _gt_check(X, Q, gt, n_sample=1000, k=10):
    """The recall ground truth (the library's kNN) against the oracle's FP64
    brute force on sampled test queries. A row passes when every returned id's
    FP64 distance is within 1e-5 of the FP64 k-th best (a different id there
    can only come from a near-tie in FP32)."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor

    rows = np.sort(np.random.default_rng(17).choice(Q.shape[0], min(n_sample, Q.shape[0]), replace=False))
    cores = os.cpu_count() or 1
    chunks = [c for c in np.array_split(rows, cores * 2) if len(c)]
    t0 = time.time()
    with ThreadPoolExecutor(max_workers=cores) as ex:
        parts = list(ex.map(lambda ix: oracle.knn_f64(Q[ix], X, k), chunks))
    ref_ids = np.concatenate([p[0] for p in parts])
    ref_d = np.concatenate([p[1] for p in parts])
    exact = near_tie = bad = 0
    for j, r in enumerate(rows):
        g = gt[r, :k]
        if np.array_equal(np.sort(g), np.sort(ref_ids[j])):
            exact += 1
            continue
        d64 = -(X[g].astype(np.float64) @ Q[r].astype(np.float64))
        if np.all(d64 <= ref_d[j, k - 1] + 1e-5):
            near_tie += 1
        else:
            bad += 1
    return {"checked": int(len(rows)), "same_set": exact, "differ_only_at_near_ties": near_tie,
            "mismatches": bad, "against": f"oracle.knn_f64 (FP64 brute force) top-{k}",
            "seconds": round(time.time() - t0, 1)}


def _serve_rate(srv, Qpool, rate, duration, seed_tag):
    """Open-loop Poisson stream at `rate` queries/s: requests of 1..256 queries,
    k in {10, 100}, L in [50, 400]. Latency = arrival to completion (includes
    any wait for admission)."""
    import roarsynth as rs

    t_arr, sizes, ks, Ls = rs.poisson_requests(rate, duration, seed_tag=seed_tag)
    n = len(t_arr)
    pending = {}
    lats = []
    done_q = 0
    i, qoff = 0, 0
    start = time.perf_counter()
    t_last = start
    deadline = start + duration + 30.0
    while (i < n or pending) and time.perf_counter() < deadline:
        now = time.perf_counter() - start
        while i < n and t_arr[i] <= now:
            nq = int(sizes[i])
            if qoff + nq > len(Qpool):
                qoff = 0
            rid = srv.submit(Qpool[qoff:qoff + nq], int(ks[i]), int(Ls[i]))
            if rid is None:
                break                       # ring full: admission waits
            pending[rid] = (nq, int(ks[i]), t_arr[i], now)
            qoff += nq
            i += 1
        for rid in srv.ready():
            nq, k, ta, tsub = pending[rid]
            r = srv.poll(rid, nq, k, timeout_ms=0, want_results=False)
            lats.append((tsub - ta) + r[0])
            done_q += nq
            t_last = time.perf_counter()
            del pending[rid]
    span = max(1e-9, t_last - start)
    lats = np.asarray(lats)
    return {"offered_qps": rate, "achieved_qps": done_q / span, "requests": int(len(lats)),
            "queries": int(done_q), "p50_ms": float(np.percentile(lats, 50) * 1e3) if len(lats) else None,
            "p99_ms": float(np.percentile(lats, 99) * 1e3) if len(lats) else None,
            "unfinished_requests": int(n - len(lats))}


def _traffic(kernel_file, src_hash):
    """ncu DRAM bytes per launch from the committed profile summary, if it
    was taken on the current kernel source; else None."""
    p = os.path.join(ROOT, "profiles", kernel_file)
    if not os.path.exists(p):
        return None
    vals = {}
    for ln in open(p):
        if ":" in ln:
            k, v = ln.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("kernel_source_sha") != src_hash:
        return None
    try:
        return float(vals["traffic_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def _time_once(fn, torch, reps=3):
    fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def _index_form(pkg, Xd, adj, entry, dtype):
    """A search handle on (Xd, adj) traversing the given form's copy."""
    if dtype == "f32":
        return pkg.Index(Xd, adj, entry, max_visits=16384), None
    codes, sc = pkg.quantize(Xd, dtype)
    return pkg.Index(Xd, adj, entry, dtype=dtype, trav=codes, scales=sc, max_visits=16384), (codes, sc)


def _free(torch):
    import gc

    gc.collect()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()


def _precision_section(torch, pkg, rs, w, log, steps=5, data=None):
    """Precision form: FP32, BF16 and FP8-E4M3 (per-row scale) traversal copies
    of one index, the last two re-ranked in FP32. Per form: the smallest L of
    the sweep reaching recall@10 0.90, its QPS, the recall delta against FP32
    at the same L, and per-result distance errors against FP64 on 200 sampled
    queries (returned FP32 distances, and the traversal distances)."""
    dev, X, Q, Xd, Qd, adj, entry, gt, bstats = data if data is not None else _setup(w, torch, pkg, rs, log)
    nq = Q.shape[0]
    sweepL = [50, 75, 100, 150, 200, 250, 300, 325, 350, 375, 400, 500]
    sample = np.random.default_rng(1).choice(nq, 200, replace=False)
    forms, sweeps = {}, {}
    for dtype in ("f32", "bf16", "fp8"):
        idx, keep = _index_form(pkg, Xd, adj, entry, dtype)
        sw = _sweep(idx, Qd, gt, torch, sweepL)
        sweeps[dtype] = sw
        L, reached = _pick_L(sw)
        idx.autotune(Qd, 10, L, repeats=1)
        ms, out = _time_steps(idx, Qd, L, steps, 3, torch)
        avg = sum(ms) / len(ms)
        ids_h = out[0].cpu().numpy().view(np.uint32)
        dh = out[1].cpu().numpy()[sample].astype(np.float64)
        ih = ids_h[sample]
        ref = -np.einsum("qkd,qd->qk", X[ih].astype(np.float64), Q[sample].astype(np.float64))
        err = np.abs(dh - ref)
        row = {"L": L, "recall_at_10": sw[L]["recall"], "recall_target_reached": reached,
               "qps": nq / (avg / 1e3), "ms_per_step": avg, "visits": sw[L]["visits"],
               "result_dist_err_vs_fp64": {"max": float(err.max()), "mean": float(err.mean())}}
        if keep is not None:
            codes, sc = keep
            sel = torch.from_numpy(ih.ravel().astype(np.int64)).to(dev)
            ch = codes[sel].cpu().numpy()
            if dtype == "bf16":
                dec = (ch.view(np.uint16).astype(np.uint32) << 16).view(np.float32).astype(np.float64)
            else:
                dec = torch.from_numpy(ch).view(torch.float8_e4m3fn).double().numpy()
                dec *= sc[sel].cpu().numpy().astype(np.float64)[:, None]
            trav = -(dec.reshape(len(sample), 10, -1) * Q[sample].astype(np.float64)[:, None, :]).sum(-1)
            terr = np.abs(trav - ref)
            row["traversal_dist_err_vs_fp64"] = {"max": float(terr.max()), "mean": float(terr.mean())}
        forms[dtype] = row
        log(f"precision {dtype}: {row}")
        idx.close()
        del keep, out
        _free(torch)
    for dtype in ("bf16", "fp8"):
        L = forms[dtype]["L"]
        forms[dtype]["recall_delta_vs_f32_at_same_L"] = sweeps[dtype][L]["recall"] - sweeps["f32"][L]["recall"]
    res = {"workload": f"{w.name}: base {w.n}x{w.d}, {w.n_train} training + {nq} test OOD queries, "
                       f"{w.n_comp} components", "build": bstats, "forms": forms,
           "sweep": {k: {str(L): v for L, v in sw.items()} for k, sw in sweeps.items()}}
    del X, Q, Xd, Qd, adj, data
    _free(torch)
    return res


def _uneven_section(torch, pkg, rs, w, dev, Xd, adj, entry, dtype, log):
    """Uneven batch: 65,536 queries with k ~ U{1,10,100} and L ~ U[max(k,10),500]
    in one persistent, CUDA-graph-captured launch (longest beams first)."""
    idx, keep = _index_form(pkg, Xd, adj, entry, dtype)
    nu = 65536
    Qu = rs.test_queries(rs.scaled(w, n_test=nu))
    ku, Lu = rs.uneven_params(nu, seed_tag=7)
    Qud = torch.from_numpy(Qu).to(dev)
    kud, Lud = torch.from_numpy(ku).to(dev), torch.from_numpy(Lu).to(dev)
    uout = idx.uneven_outputs(ku)
    best, _ = idx.autotune(Qud[:8192], 10, int(Lu.max()), repeats=1)   # the launch's pool-size bucket
    plan = idx.plan_uneven(Qud, kud, Lud, int(Lu.max()), uout, longest_first=True)
    for _ in range(2):
        plan.launch()
    torch.cuda.synchronize()
    a_ev, b_ev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a_ev.record()
    reps = 3
    for _ in range(reps):
        plan.launch()
    b_ev.record()
    torch.cuda.synchronize()
    ums = a_ev.elapsed_time(b_ev) / reps
    res = {"index": w.name, "base": f"{w.n}x{w.d}", "form": dtype if dtype == "f32" else f"{dtype} traversal + fp32 re-rank",
           "queries": nu, "k": "U{1,10,100}", "L": "U[max(k,10),500]", "ms_per_launch": ums,
           "qps": nu / (ums / 1e3), "graph_captured": True, "order": "longest L first",
           "autotune_variant": int(best), "mean_visits": float(uout[3].double().mean()),
           "status_nonzero": int((uout[5] != 0).sum())}
    plan.close()
    idx.close()
    del Qud, uout, keep
    _free(torch)
    return res


def _serving_section(torch, pkg, rs, w, dev, Xd, adj, entry, Q, Qd, gt, dtype, log):
    """Continuous batching into the persistent kernel under an open-loop Poisson
    stream (requests of 1..256 queries, k in {10, 100}, L in [50, 400]):
    achieved QPS with p50/p99 latency per offered rate, and the recall of
    served results for the test queries at the form's first L reaching 0.90."""
    sidx, keep = _index_form(pkg, Xd, adj, entry, dtype)
    sw = _sweep(sidx, Qd, gt, torch, [50, 75, 100, 150, 200, 300, 400])
    L90, reached = _pick_L(sw)
    sidx.autotune(Qd, 10, 400, repeats=1)
    Qpool = rs.test_queries(rs.scaled(w, n_test=65536))
    # The device's capacity for the same mix: the queries of a Poisson stream
    # (each with its request's k and L) as one graph-captured uneven batch.
    _, sz, ks, Ls = rs.poisson_requests(1e6, 1.0, seed_tag=299)
    kq = np.repeat(ks, sz)[:len(Qpool)].astype(np.int32)
    Lq = np.repeat(Ls, sz)[:len(Qpool)].astype(np.int32)
    nb = len(kq)
    Qb = torch.from_numpy(Qpool[:nb]).to(dev)
    kbd, Lbd = torch.from_numpy(kq).to(dev), torch.from_numpy(Lq).to(dev)
    bout = sidx.uneven_outputs(kq)
    plan = sidx.plan_uneven(Qb, kbd, Lbd, 400, bout, longest_first=True)
    for _ in range(2):
        plan.launch()
    torch.cuda.synchronize()
    a_ev, b_ev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a_ev.record()
    for _ in range(3):
        plan.launch()
    b_ev.record()
    torch.cuda.synchronize()
    bms = a_ev.elapsed_time(b_ev) / 3
    batched = {"queries": nb, "ms_per_launch": bms, "qps": nb / (bms / 1e3),
               "mean_visits": float(bout[3].double().mean()), "graph_captured": True}
    plan.close()
    del Qb, kbd, Lbd, bout
    log(f"serving mix as one batch: {batched}")
    srv = pkg.Server(sidx, k_max=100, L_max=400, ring_capacity=1 << 16, idle_ms=50)
    res = {"index": w.name, "base": f"{w.n}x{w.d}",
           "form": dtype if dtype == "f32" else f"{dtype} traversal + fp32 re-rank",
           "requests": "Poisson arrivals; 1..256 queries; k in {10,100}; L in [50,400]",
           "same_mix_batched": batched, "rates": []}
    for j, rate in enumerate((1e4, 3e4, 1e5, 3e5, 1e6)):
        res["rates"].append(_serve_rate(srv, Qpool, rate, 1.0, 200 + j))
        log(f"serving {res['rates'][-1]}")
    # served recall: the test queries in requests of 256 at L90
    nq = Q.shape[0]
    rids = []
    for i in range(0, nq, 256):
        rid = None
        while rid is None:
            rid = srv.submit(Q[i:i + 256], 10, L90)
        rids.append((rid, min(256, nq - i)))
    got = []
    for rid, m in rids:
        r = None
        while r is None:
            r = srv.poll(rid, m, 10, timeout_ms=100)
        got.append(r[1])
    res.update({"served_recall_at_10": _recall(np.concatenate(got), gt), "served_recall_L": L90,
                "recall_target_reached": reached, "server": srv.stats()})
    srv.close()
    sidx.close()
    del keep
    _free(torch)
    return res


def _extra_mode(args, w, torch, pkg, rs, dev, X, Q, Xd, Qd, adj, entry, gt, bstats, log):
    """The precision (10M x 512), uneven (1M x 512) and serving (10M x 200) workloads,
    and the OOD-built against ID-built graph comparison (ood)."""
    nq = Q.shape[0]
    res = {"mode": args.mode, "workload": w.name, "n": w.n, "d": w.d, "offset_norm": w.offset_norm, "build": bstats}
    if args.mode == "precision":
        res["precision"] = _precision_section(torch, pkg, rs, w, log,
                                              data=(dev, X, Q, Xd, Qd, adj, entry, gt, bstats))
    elif args.mode == "uneven":
        res["uneven"] = _uneven_section(torch, pkg, rs, w, dev, Xd, adj, entry, "bf16", log)
    elif args.mode == "serving":
        res["serving"] = _serving_section(torch, pkg, rs, w, dev, Xd, adj, entry, Q, Qd, gt, "bf16", log)
    elif args.mode == "ood":
        # The paper's central comparison on synthetic data: a graph built from
        # OOD training queries (RoarGraph as specified) against one built the
        # same way from in-distribution training queries, searched with OOD
        # and with ID test queries.
        idq = rs.id_queries(w, w.n_train + nq)
        Tid = torch.from_numpy(idq[:w.n_train]).to(dev)
        Qid = torch.from_numpy(np.ascontiguousarray(idq[w.n_train:])).to(dev)
        del idq
        gi, _ = pkg.knn(Qid, Xd, 10)
        torch.cuda.synchronize()
        gt_id = gi.cpu().numpy().view(np.uint32)
        t0 = time.time()
        adj_id, entry_id, st_id = pkg.build_index(Xd, Tid, nq_depth=100, M=32, L_build=500)
        torch.cuda.synchronize()
        log(f"ID-built graph in {time.time() - t0:.1f}s")
        del Tid
        sweepL = [10, 20, 30, 50, 75, 100, 150, 200, 300, 500]
        graphs = {"built_from_ood_queries": (adj, entry), "built_from_id_queries": (adj_id, entry_id)}
        qsets = {"ood_queries": (Qd, gt), "id_queries": (Qid, gt_id)}
        table = {}
        for gname, (a_, e_) in graphs.items():
            gidx = pkg.Index(Xd, a_, e_, max_visits=16384)
            for qname, (Qs, gts) in qsets.items():
                rows = {}
                for L in sweepL:
                    ms = _time_once(lambda: gidx.search(Qs, 10, L), torch)
                    ids, dist, visits, hops, st = gidx.search(Qs, 10, L)
                    torch.cuda.synchronize()
                    rows[str(L)] = {"recall_at_10": _recall(ids.cpu().numpy().view(np.uint32), gts),
                                    "visits": float(visits.double().mean()), "hops": float(hops.double().mean()),
                                    "qps": Qs.shape[0] / (ms / 1e3)}
                at = [L for L in sweepL if rows[str(L)]["recall_at_10"] >= TARGET_RECALL]
                table[f"{gname}/{qname}"] = {
                    "sweep": rows,
                    "first_L_at_recall_0.90": at[0] if at else None,
                    "visits_at_that_L": rows[str(at[0])]["visits"] if at else None}
                log(f"{gname}/{qname}: {table[f'{gname}/{qname}']['first_L_at_recall_0.90']}")
            gidx.close()
        res.update({"graphs": table, "build_id_graph": st_id})
    elif args.mode == "ablation":
        # Sec. 5.4: search the bipartite graph G_bi (Alg. 1's bipartite step,
        # every x -> t edge kept, searched through query nodes as in Sec. 4.1),
        # the projected graph G_pj and the final RoarGraph with the same OOD
        # queries.
        t0 = time.time()
        T = rs.train_queries(w)
        Td = torch.from_numpy(T).to(dev)
        del T
        adj_f, entry_f, st_f, pj = pkg.build_index(Xd, Td, nq_depth=100, M=32, L_build=500, return_pj=True)
        kid, _ = pkg.knn(Td, Xd, 100)
        del Td
        off, qids, nout, bst = pkg.bipartite(kid, w.n)
        del kid
        # G_bi's entry: the medoid when it has a query out-neighbour, else the
        # base node with one nearest to it (FP64 inner product, ties by id).
        offh = off.cpu().numpy()
        entry_bi = entry_f
        if offh[entry_f + 1] == offh[entry_f]:
            piv = np.nonzero(np.diff(offh) > 0)[0]
            sc = X[piv].astype(np.float64) @ X[entry_f].astype(np.float64)
            entry_bi = int(piv[np.lexsort((piv, -sc))[0]])
        log(f"graphs ready in {time.time() - t0:.1f}s; G_bi {bst}")
        graphs = {"G_bi": pkg.BipartiteIndex(Xd, nout, off, qids, entry_bi, max_visits=16384),
                  "G_pj": pkg.Index(Xd, pj, entry_f, max_visits=16384),
                  "RoarGraph": pkg.Index(Xd, adj_f, entry_f, max_visits=16384)}
        table = {}
        for gname, gidx in graphs.items():
            rows = {}
            for L in (10, 20, 50, 100, 200, 500):
                ms = _time_once(lambda: gidx.search(Qd, 10, L), torch)
                ids, dist, visits, hops, st = gidx.search(Qd, 10, L)
                torch.cuda.synchronize()
                rows[str(L)] = {"recall_at_10": _recall(ids.cpu().numpy().view(np.uint32), gt),
                                "visits": float(visits.double().mean()), "hops": float(hops.double().mean()),
                                "visits_per_hop": float(visits.double().sum() / max(hops.double().sum(), 1.0)),
                                "capped": int((st == 4).sum()), "qps": nq / (ms / 1e3)}
            gidx.close()
            table[gname] = rows
            log(f"{gname}: {rows}")
        res.update({"graphs": table, "g_bi": {**bst, "entry": entry_bi, "query_nodes": int(qids.shape[0])},
                    "build": st_f})
    elif args.mode == "update":
        # Sec. 5.7: insertion through the saved bipartite graph, and deletion by
        # tombstones. Build on the first 90 % of the rows, insert the rest,
        # compare with the index built over all rows (the cached one).
        n = w.n
        n_old = n - n // 10
        T = rs.train_queries(w)
        Td = torch.from_numpy(T).to(dev)
        t0 = time.time()
        adj_old, entry_old, st_old = pkg.build_index(Xd[:n_old], Td, nq_depth=100, M=32, L_build=500)
        kid, _ = pkg.knn(Td, Xd[:n_old], 100)
        torch.cuda.synchronize()
        build_s = time.time() - t0
        knn_h = kid.cpu().numpy().view(np.uint32)
        del kid, Td
        cap = 99 + 64
        nout = np.full((T.shape[0], cap), 0xFFFFFFFF, dtype=np.uint32)
        nout[:, :99] = knn_h[:, 1:]
        cnt = np.full(T.shape[0], 99, dtype=np.int32)
        R = adj_old.shape[1]
        adj_u = torch.full((n, R), -1, dtype=torch.int32, device=dev)
        adj_u[:n_old] = adj_old
        # The windowed insertion equals the one-row-at-a-time order (window 1):
        # check on the first rows inserted, at the full graph size.
        m_chk = min(2000, n - n_old)
        chk = {}
        for win in (1, args.insert_window):
            a_c = adj_u[:n_old + m_chk].clone()
            no_c, cn_c = nout.copy(), cnt.copy()
            t0 = time.time()
            q_c = pkg.insert(Xd[:n_old + m_chk], a_c, entry_old, n_old, T, knn_h[:, 0], no_c, cn_c, 32, 100,
                             window=win)
            torch.cuda.synchronize()
            chk[win] = (a_c.cpu().numpy(), no_c, cn_c, q_c, time.time() - t0)
            del a_c
        a1, a2 = chk[1], chk[args.insert_window]
        window_check = {"rows": int(m_chk), "identical": bool(np.array_equal(a1[0], a2[0]) and
                                                             np.array_equal(a1[1], a2[1]) and
                                                             np.array_equal(a1[2], a2[2]) and
                                                             np.array_equal(a1[3], a2[3])),
                        "rows_per_s_window_1": m_chk / a1[4],
                        f"rows_per_s_window_{args.insert_window}": m_chk / a2[4]}
        del chk, a1, a2
        log(f"window check {window_check}")
        t0 = time.time()
        chosen, ins_st = pkg.insert(Xd, adj_u, entry_old, n_old, T, knn_h[:, 0], nout, cnt, 32, 100,
                                    window=args.insert_window, return_stats=True)
        torch.cuda.synchronize()
        ins_s = time.time() - t0
        log(f"inserted {n - n_old} rows in {ins_s:.1f}s {ins_st}")
        del T
        table = {}
        for gname, (a_, e_) in {"updated": (adj_u, entry_old), "rebuilt": (adj, entry)}.items():
            gidx = pkg.Index(Xd, a_, e_, max_visits=16384)
            rows = {}
            for L in (50, 90, 100, 150, 200, 300):
                ms = _time_once(lambda: gidx.search(Qd, 10, L), torch)
                ids, dist, visits, hops, st = gidx.search(Qd, 10, L)
                torch.cuda.synchronize()
                rows[str(L)] = {"recall_at_10": _recall(ids.cpu().numpy().view(np.uint32), gt),
                                "visits": float(visits.double().mean()), "qps": nq / (ms / 1e3)}
            table[gname] = rows
            gidx.close()
        # deletion: 10 % of the rows tombstoned; ground truth over the live rows
        dead = np.random.default_rng(5).random(n) < 0.1
        words = np.zeros((n + 31) // 32, dtype=np.uint32)
        di = np.nonzero(dead)[0]
        np.bitwise_or.at(words, di >> 5, (np.uint32(1) << (di & 31).astype(np.uint32)))
        g40, _ = pkg.knn(Qd, Xd, 40)
        torch.cuda.synchronize()
        g40 = g40.cpu().numpy().view(np.uint32)
        gt_live = np.array([[u for u in row if not dead[u]][:10] for row in g40], dtype=np.uint32)
        gidx = pkg.Index(Xd, adj_u, entry_old, max_visits=16384)
        gidx.set_tombstones(torch.from_numpy(words.view(np.int32)).to(dev))
        trows = {}
        for L in (90, 100, 150):
            ms = _time_once(lambda: gidx.search(Qd, 10, L), torch)
            ids, *_ = gidx.search(Qd, 10, L)
            torch.cuda.synchronize()
            ih = ids.cpu().numpy().view(np.uint32)
            trows[str(L)] = {"recall_at_10_live": _recall(ih, gt_live), "qps": nq / (ms / 1e3),
                             "deleted_in_answers": int(dead[ih[ih != 0xFFFFFFFF]].sum())}
        gidx.close()
        res.update({"n_old": int(n_old), "inserted": int(n - n_old), "build_old_s": build_s,
                    "insert_s": ins_s, "inserts_per_s": (n - n_old) / ins_s, "insert_window": args.insert_window,
                    "insert_work": ins_st, "window_check": window_check,
                    "rows_with_a_connected_query": float((chosen >= 0).mean()),
                    "search": table, "tombstones_10pct": trows})
    elif args.mode == "serving":
        codes, sc = pkg.quantize(Xd, "bf16")
        sidx = pkg.Index(Xd, adj, entry, dtype="bf16", trav=codes, scales=None, max_visits=16384)
        sidx.autotune(Qd, 10, 400, repeats=1)
        srv = pkg.Server(sidx, k_max=100, L_max=400, ring_capacity=1 << 16, idle_ms=50)
        Qpool = rs.test_queries(rs.scaled(w, n_test=65536))
        rates = []
        for j, rate in enumerate((1e4, 3e4, 1e5, 3e5, 1e6)):
            rates.append(_serve_rate(srv, Qpool, rate, 1.0, 300 + j))
            log(f"serving {rates[-1]}")
        # recall of served results for the 10k test queries at L = 400
        rids = []
        for i in range(0, nq, 256):
            rid = None
            while rid is None:
                rid = srv.submit(Q[i:i + 256], 10, 400)
            rids.append((rid, min(256, nq - i)))
        got = []
        for rid, m in rids:
            r = None
            while r is None:
                r = srv.poll(rid, m, 10, timeout_ms=100)
            got.append(r[1])
        res.update({"form": "bf16 traversal + fp32 re-rank", "rates": rates,
                    "served_recall_at_10_L400": _recall(np.concatenate(got), gt), "server": srv.stats()})
        srv.close()
        sidx.close()
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="base_1m_d200")
    ap.add_argument("--n", type=int, default=0, help="override base rows (smaller runs)")
    ap.add_argument("--n-train", type=int, default=0, help="override training queries")
    ap.add_argument("--no-forms", action="store_true")
    ap.add_argument("--quick", action="store_true",
                    help="run the uneven batch and the serving loop on the main workload's index and skip "
                         "the 10M x 512 precision workload")
    ap.add_argument("--n-comp", type=int, default=0, help="override the mixture components (small experiments)")
    ap.add_argument("--insert-window", type=int, default=256, help="rows per speculative insertion window (update mode)")
    ap.add_argument("--offset-norm", type=float, default=0.0,
                    help="override the OOD offset norm (ood mode experiments; the workloads use 1.5)")
    ap.add_argument("--mode", default="main", choices=["main", "precision", "uneven", "serving", "ood", "ablation", "update"],
                    help="main: the benchmark line; others: the precision / uneven / serving workloads, "
                         "ood: OOD-built against ID-built graphs with OOD and ID queries, "
                         "ablation: G_bi / G_pj / RoarGraph, update: insertion and tombstones")
    ap.add_argument("--verbose", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    def log(msg):
        if args.verbose and rank == 0:
            print(f"[bench] {msg}", file=sys.stderr, flush=True)

    import torch

    import paper_2408_08933_gb300 as pkg
    import roarsynth as rs

    if args.impl == "reference" and rank != 0:
        return
    torch.cuda.set_device(local)
    dist_on = world > 1 and args.impl == "ours"
    if dist_on:
        import torch.distributed as tdist

        tdist.init_process_group("nccl")
    w = rs.WORKLOADS[args.workload]
    if args.n:
        w = rs.scaled(w, n=args.n, n_train=args.n_train or min(args.n, w.n_train))
    elif args.n_train:
        w = rs.scaled(w, n_train=args.n_train)
    if args.offset_norm > 0:
        w = rs.scaled(w, offset_norm=args.offset_norm)
    if args.n_comp > 0:
        w = rs.scaled(w, n_comp=args.n_comp)
    dev, X, Q, Xd, Qd, adj, entry, gt, bstats = _setup(w, torch, pkg, rs, log)
    if args.mode != "main":
        out = _extra_mode(args, w, torch, pkg, rs, dev, X, Q, Xd, Qd, adj, entry, gt, bstats, log)
        print(json.dumps(out), flush=True)
        return
    idx = pkg.Index(Xd, adj, entry, max_visits=16384)
    sweep = _sweep(idx, Qd, gt, torch, L_SWEEP)
    L, reached = _pick_L(sweep)
    log(f"sweep {json.dumps(sweep)} -> L={L}")
    best, tune_ms = (-1, []) if args.impl == "reference" else idx.autotune(Qd, 10, L, repeats=2)
    log(f"autotune L={L}: best variant {best}, ms {[round(float(x), 3) for x in tune_ms]}")
    nq = Q.shape[0]
    config = {"workload": f"{w.name}: base {w.n}x{w.d} FP32, {w.n_train} training + {nq} test OOD queries, "
                          f"{w.n_comp} components, kNN depth 100, M=32, L_build=500",
              "k": 10, "L": L, "recall_at_10": sweep[L]["recall"], "recall_target": TARGET_RECALL,
              "recall_target_reached": reached, "batch": nq,
              "launch": {"variant": best, "team_warps": [1, 2, 4, 8][best // 4] if best >= 0 else None,
                         "visited_set": ["auto", "bitmap", "2^10 shared + bitmap", "2^12 shared + bitmap"][best % 4] if best >= 0 else None},
              "l2_flush": "not needed: base rows 800 MB > 129 MB L2", "parallelism": f"replicas x{world}"}

    if args.impl == "reference":
        adj_np = adj.cpu().numpy().view(np.uint32)
        step_s = []
        for _ in range(args.warmup + args.steps):
            cb, _ = _cpu_baseline(X, adj_np, entry, Q, L, budget_s=max(1.0, 60.0 / (args.steps + args.warmup)))
            step_s.append(cb)
        vals = [c["value"] for c in step_s[args.warmup:]]
        v = statistics.median(vals)
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "queries/s", "n_gpus": 1,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": None,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic", "config": config,
                "cpu_baseline": {**step_s[-1], "value": v},
                "e2e": {"value": v, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return

    # ---- timed: plain FP32 batch search at L -----------------------------------
    if dist_on:
        tdist.barrier()
    torch.cuda.synchronize()
    # Clocks are sampled from before the warm-up until the end of the
    # end-to-end loop (all of it GPU-busy), so the timed region is inside.
    clk = ClockSampler(local).__enter__()
    time.sleep(0.5)                      # nvidia-smi takes a moment to start sampling
    torch.cuda.nvtx.range_push("timed_f32")
    ms, out = _time_steps(idx, Qd, L, args.steps, args.warmup, torch)
    torch.cuda.nvtx.range_pop()
    if dist_on:
        tdist.barrier()
    total_ms = max_over_ranks(sum(ms), dev if dist_on else None)
    ids, dist, visits, hops, st = out
    value = world * nq * args.steps / (total_ms / 1e3)

    deg_mean = float((adj != -1).sum().item()) / adj.shape[0]
    v_mean = float(visits.double().mean())
    h_mean = float(hops.double().mean())
    bytes_q = _algorithmic_bytes(v_mean, h_mean, deg_mean, w.d, 4, 0)
    avg_ms = total_ms / args.steps
    achieved = bytes_q * nq / (avg_ms / 1e3) / 1e9
    peak, peak_src = _peaks()
    src_hash = _src_hash(["paper_2408_08933_gb300/csrc/roar_search_kernel.cuh",
                          "paper_2408_08933_gb300/csrc/roar_search.cu",
                          "paper_2408_08933_gb300/csrc/roar_internal.cuh",
                          "paper_2408_08933_gb300/csrc/roar_search_f32.cu"])
    traffic = _traffic(f"search_f32_{w.name}.txt", src_hash)

    # ---- e2e: host buffers through roar_search_host -----------------------------
    Qh = torch.from_numpy(Q).pin_memory()
    hout = (torch.empty((nq, 10), dtype=torch.int32).pin_memory(),
            torch.empty((nq, 10), dtype=torch.float32).pin_memory(),
            torch.empty(nq, dtype=torch.int32).pin_memory(), torch.empty(nq, dtype=torch.int32).pin_memory(),
            torch.empty(nq, dtype=torch.int32).pin_memory())
    for _ in range(args.warmup):
        idx.search_host(Qh, 10, L, out=hout)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        idx.search_host(Qh, 10, L, out=hout)
    e2e_s = time.perf_counter() - t0
    clk.__exit__(None, None, None)
    h_ids = hout[0].numpy().view(np.uint32)
    assert np.array_equal(h_ids, ids.cpu().numpy().view(np.uint32)), "host-buffer results differ"

    # ---- reduced-precision forms on the same graph -----------------------------
    forms = {}
    if not args.no_forms:
        for dtype, eb, sb in (("bf16", 2, 0), ("fp8", 1, 4)):
            codes, sc = pkg.quantize(Xd, dtype)
            qidx = pkg.Index(Xd, adj, entry, dtype=dtype, trav=codes, scales=sc, max_visits=16384)
            qs = _sweep(qidx, Qd, gt, torch, L_SWEEP)
            qL, _ = _pick_L(qs)
            qidx.autotune(Qd, 10, qL, repeats=2)
            torch.cuda.nvtx.range_push(f"timed_{dtype}")
            qms, qout = _time_steps(qidx, Qd, qL, max(3, args.steps // 2), 3, torch)
            torch.cuda.nvtx.range_pop()
            qv = float(qout[2].double().mean())
            qh = float(qout[3].double().mean())
            qbytes = _algorithmic_bytes(qv, qh, deg_mean, w.d, eb, sb, k_rerank_L=qL)
            qavg = sum(qms) / len(qms)
            same_L_recall = qs[L]["recall"] if L in qs else None
            forms[dtype] = {"L": qL, "recall_at_10": qs[qL]["recall"], "qps": nq / (qavg / 1e3),
                            "ms_per_step": qavg, "achieved_gbs": qbytes * nq / (qavg / 1e3) / 1e9,
                            "recall_delta_vs_f32_at_same_L": (None if same_L_recall is None
                                                              else same_L_recall - sweep[L]["recall"])}
            qidx.close()
            del codes, sc
        forms["f32"] = {"L": L, "recall_at_10": sweep[L]["recall"], "qps": value / world,
                        "ms_per_step": avg_ms, "achieved_gbs": achieved}

    # ---- the other workloads the metric names ----------------------------------
    # precision form: 10M x 512 (FP32 / BF16 / FP8 + re-rank); uneven batch:
    # 1M x 512 BF16 + re-rank; serving: 10M x 200 BF16 + re-rank. With --quick
    # the uneven batch and the serving loop run on this workload's index.
    precision = uneven = serving = None
    if not args.no_forms:
        if args.quick:
            uneven = _uneven_section(torch, pkg, rs, w, dev, Xd, adj, entry, "bf16", log)
            serving = _serving_section(torch, pkg, rs, w, dev, Xd, adj, entry, Q, Qd, gt, "bf16", log)
        else:
            wu = rs.BASE_1M_D512
            du = _setup(wu, torch, pkg, rs, log)
            uneven = _uneven_section(torch, pkg, rs, wu, du[0], du[3], du[5], du[6], "bf16", log)
            del du
            _free(torch)
            ws = rs.BASE_10M_D200
            ds = _setup(ws, torch, pkg, rs, log)
            serving = _serving_section(torch, pkg, rs, ws, ds[0], ds[3], ds[5], ds[6], ds[2], ds[4], ds[7],
                                       "bf16", log)
            serving["build"] = ds[8]
            del ds
            _free(torch)
            precision = _precision_section(torch, pkg, rs, rs.BASE_10M_D512, log)

    cpu = parity = gt_check = None
    if rank == 0:
        cpu, ref = _cpu_baseline(X, adj.cpu().numpy().view(np.uint32), entry, Q, L)
        parity = _parity(out, ref)
        gt_check = _gt_check(X, Q, gt)

    line = {
        "metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": avg_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded OOD Gaussian mixture)",
        "config": config,
        "e2e": {"value": world * nq * args.steps / e2e_s, "unit": "queries/s",
                "h2d_bytes_per_step": int(Q.nbytes),
                "d2h_bytes_per_step": int(nq * 10 * 8 + nq * 12)},
        "gpu_launches": args.steps,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "peak_source": f"{peak_src} hbm_gbs (burst copy)",
                     "bytes_per_query": bytes_q, "kernel": "beam_search_kernel<f32>"},
        "cpu_baseline": cpu,
        "parity": parity,
        "ground_truth_check": gt_check,
        "clocks": clk.summary(),
        "forms": forms,
        "precision": precision,
        "uneven": uneven,
        "serving": serving,
        "sweep": {str(k): v for k, v in sweep.items()},
        "build": bstats,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    idx.close()
    if dist_on:
        tdist.destroy_process_group()
    if rank == 0 and (parity["mismatches"] or gt_check["mismatches"]):
        print(f"parity failure: {parity['mismatches']} searched queries differ from the oracle, "
              f"{gt_check['mismatches']} ground-truth rows differ from FP64 brute force", file=sys.stderr)
        sys.exit(1)


if __name__ == "__main__":
    main()
