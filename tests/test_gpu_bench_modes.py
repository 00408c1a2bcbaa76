"""The paper's qualitative claims, measured by the benchmark's experiment
modes on a small synthetic workload (10k x 64, one mixture component, OOD
offset norm 12) through the product path: GPU construction and GPU search.

- Sec. 5.5 / Sec. 3: for OOD queries, the graph built from OOD training
  queries (RoarGraph) needs fewer visits than one built the same way from
  in-distribution training queries (`bench.py --mode ood`).
- Sec. 5.4: the bipartite graph G_bi visits many more nodes per hop than the
  projected graph G_pj, and the final graph reaches a higher recall than G_pj
  (`bench.py --mode ablation`).
"""
import json
import os
import subprocess
import sys

import pytest

from conftest import ROOT

pytestmark = pytest.mark.gpu
SMALL = ["--workload", "tiny_10k_d64", "--n-comp", "1", "--offset-norm", "12"]


@pytest.fixture(scope="module")
def cache_dir(tmp_path_factory):
    return str(tmp_path_factory.mktemp("bench_cache"))


def _bench(mode, cache_dir):
    env = dict(os.environ, ROAR_BENCH_CACHE=cache_dir)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--mode", mode, *SMALL],
                       capture_output=True, text=True, timeout=900, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_ood_built_graph_needs_fewer_visits_for_ood_queries(cache_dir):
    res = _bench("ood", cache_dir)
    ood = res["graphs"]["built_from_ood_queries/ood_queries"]
    idb = res["graphs"]["built_from_id_queries/ood_queries"]
    assert ood["first_L_at_recall_0.90"] is not None
    if idb["first_L_at_recall_0.90"] is not None:
        assert ood["visits_at_that_L"] < idb["visits_at_that_L"]
    # at every beam width the OOD-built graph is at least as accurate
    for L, row in ood["sweep"].items():
        assert row["recall_at_10"] >= idb["sweep"][L]["recall_at_10"] - 0.01, L


def test_ablation_bipartite_visits_more_per_hop(cache_dir):
    res = _bench("ablation", cache_dir)
    g = res["graphs"]
    for L in ("20", "50", "100"):
        assert g["G_bi"][L]["visits_per_hop"] > 2 * g["G_pj"][L]["visits_per_hop"], L
        assert g["RoarGraph"][L]["recall_at_10"] >= g["G_pj"][L]["recall_at_10"], L
    assert res["g_bi"]["widest_base_row"] >= 1
