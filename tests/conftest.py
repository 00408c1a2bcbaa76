"""Shared fixtures. GPU tests are marked ``gpu``; everything else runs on CPU."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")


@pytest.fixture(scope="session")
def tiny():
    """The tiny workload (10k x d64, 32 components) with its oracle-built index.

    kNN depth 100, M = 32, L = 500 (Sec. 5.1 parameters, M per the workload).
    """
    import oracle
    import roarsynth as rs

    w = rs.TINY
    X = rs.base(w)
    T = rs.train_queries(w)
    Q = rs.test_queries(w)
    knn, _ = oracle.knn_f64(T, X, 100)
    entry = oracle.medoid(X)
    adj, pj, stats = oracle.build_index(X, knn, 32, 500, entry)
    gt, _ = oracle.knn_f64(Q, X, 100)
    return dict(w=w, X=X, T=T, Q=Q, knn=knn, entry=entry, adj=adj, pj=pj, stats=stats, gt=gt,
                M=32, L_build=500)


def load_golden(name):
    import json

    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def path_graph(a, rmax=4):
    """Path graph 0-1-...-(n-1), both directions, rows padded with 0xFFFFFFFF."""
    n = len(a)
    adj = np.full((n, rmax), 0xFFFFFFFF, dtype=np.uint32)
    for v in range(n):
        nb = [u for u in (v - 1, v + 1) if 0 <= u < n]
        adj[v, :len(nb)] = nb
    X = np.zeros((n, 4), dtype=np.float32)
    X[:, 0] = a
    return X, adj
