"""The search entry point that allocates nothing (roar_search_noalloc).

Callers that must not allocate device memory (code inside another
framework's memory pool, serving processes that may not allocate once
running) use this call; its scratch is a fixed array inside the library.
Here it must return the same results as the allocating entry point
(roar_search through an index handle), on two calls in a row, since the
fixed array keeps the previous call's contents.
This file sorts last so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest

import paper_2408_08933_gb300 as pkg
from gpu_util import assert_same, dev_index, run

pytestmark = pytest.mark.gpu
MV = 16384


def _noalloc(idx, Q, k, L):
    import torch

    Qd = torch.from_numpy(np.ascontiguousarray(Q, np.float32)).to("cuda:0")
    nq = Q.shape[0]
    ids = torch.empty((nq, k), dtype=torch.int32, device="cuda:0")
    dist = torch.empty((nq, k), dtype=torch.float32, device="cuda:0")
    vis, hops, st = (torch.empty(nq, dtype=torch.int32, device="cuda:0") for _ in range(3))
    s = torch.cuda.current_stream().cuda_stream
    pkg.roar_search_noalloc(idx.n, idx.d, idx.base_f32.data_ptr(), idx.adj.data_ptr(), idx.rmax,
                            idx.entry, MV, Qd.data_ptr(), nq, k, L, ids.data_ptr(),
                            dist.data_ptr(), vis.data_ptr(), hops.data_ptr(), st.data_ptr(), s)
    torch.cuda.synchronize()
    return (ids.cpu().numpy().view(np.uint32), dist.cpu().numpy(), vis.cpu().numpy().view(np.uint32),
            hops.cpu().numpy().view(np.uint32), st.cpu().numpy())


def test_noalloc_matches_allocating_entry_point_twice(tiny):
    idx = dev_index(tiny["X"], tiny["adj"], tiny["entry"], max_visits=MV)
    Q = tiny["Q"]
    for k, L in ((10, 100), (10, 300)):
        ref = run(idx, Q, k, L)
        assert_same(_noalloc(idx, Q, k, L), ref, f"first call k={k} L={L}")
        assert_same(_noalloc(idx, Q, k, L), ref, f"second call k={k} L={L}")
    idx.close()


def test_noalloc_rejects_sizes_beyond_its_scratch(tiny):
    idx = dev_index(tiny["X"], tiny["adj"], tiny["entry"], max_visits=MV)
    with pytest.raises(pkg.RoarError) as e:
        # n far beyond the fixed scratch: rejected before any launch
        pkg.roar_search_noalloc(1 << 30, idx.d, idx.base_f32.data_ptr(), idx.adj.data_ptr(),
                                idx.rmax, 0, MV, idx.base_f32.data_ptr(), 1, 10, 10,
                                idx.adj.data_ptr(), idx.adj.data_ptr())
    assert e.value.status == pkg.ROAR_EINVAL
    assert "64 MiB" in str(e.value)
    idx.close()
