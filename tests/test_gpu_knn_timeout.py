"""Failure handling of the tensor-core kNN kernel: a bounded wait that runs out.

The wait limit is set from the host to zero, so every mbarrier wait in the
kernel gives up as soon as its phase is found incomplete. The call must come
back with ROAR_ETIMEOUT through the kernel's abort path (copies and issued
MMAs drained, TMEM freed), and the next call, with the default limit, must
run normally on the same context and give the exact result.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("halves", ["1", "2"])
def test_knn_wait_runs_out_then_recovers(halves, monkeypatch):
    import torch

    import paper_2408_08933_gb300 as pkg

    monkeypatch.setenv("ROAR_KNN_HALVES", halves)   # both CTA shapes' abort paths

    rng = np.random.default_rng(11)
    X = rng.standard_normal((5000, 64)).astype(np.float32)
    T = rng.standard_normal((300, 64)).astype(np.float32)
    Xd = torch.from_numpy(X).to("cuda:0")
    Td = torch.from_numpy(T).to("cuda:0")
    try:
        pkg.roar_knn_set_wait_limit_ns(0)
        for _ in range(2):
            with pytest.raises(pkg.RoarError) as e:
                pkg.knn(Td, Xd, 10)
            assert e.value.status == pkg.ROAR_ETIMEOUT
    finally:
        pkg.roar_knn_set_wait_limit_ns(-1)
    ids, dist = pkg.knn(Td, Xd, 10)
    torch.cuda.synchronize()
    ref, _ = oracle.knn_f64(T, X, 10)
    got = ids.cpu().numpy().view(np.uint32)
    assert np.mean([len(set(got[i]) & set(ref[i])) / 10 for i in range(len(T))]) >= 0.999
    d = dist.cpu().numpy()
    for i in range(0, len(T), 37):
        assert d[i, 0] == -oracle.dot_fixed(T[i], X[got[i, 0]])
