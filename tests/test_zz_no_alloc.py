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


def _buffers(Q, k):
    import torch

    Qd = torch.from_numpy(np.ascontiguousarray(Q, np.float32)).to("cuda:0")
    nq = Q.shape[0]
    ids = torch.empty((nq, k), dtype=torch.int32, device="cuda:0")
    dist = torch.empty((nq, k), dtype=torch.float32, device="cuda:0")
    vis, hops, st = (torch.empty(nq, dtype=torch.int32, device="cuda:0") for _ in range(3))
    return Qd, ids, dist, vis, hops, st


def _call(idx, bufs, k, L, n=None, mv=MV):
    import torch

    Qd, ids, dist, vis, hops, st = bufs
    s = torch.cuda.current_stream().cuda_stream
    pkg.roar_search_noalloc(idx.n if n is None else n, idx.d, idx.base_f32.data_ptr(), idx.adj.data_ptr(),
                            idx.rmax, idx.entry, mv, Qd.data_ptr(), Qd.shape[0], k, L, ids.data_ptr(),
                            dist.data_ptr(), vis.data_ptr(), hops.data_ptr(), st.data_ptr(), s)


def _fetch(bufs):
    import torch

    _, ids, dist, vis, hops, st = bufs
    torch.cuda.synchronize()
    return (ids.cpu().numpy().view(np.uint32), dist.cpu().numpy(), vis.cpu().numpy().view(np.uint32),
            hops.cpu().numpy().view(np.uint32), st.cpu().numpy())


def _noalloc(idx, Q, k, L):
    bufs = _buffers(Q, k)
    _call(idx, bufs, k, L)
    return _fetch(bufs)


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


def test_noalloc_leaves_free_device_memory_unchanged(tiny):
    """The point of the entry point: a call takes no device memory. After a
    first call (which loads the module with its fixed array), free device
    memory is the same before and after another call."""
    import torch

    idx = dev_index(tiny["X"], tiny["adj"], tiny["entry"], max_visits=MV)
    bufs = _buffers(tiny["Q"], 10)
    _call(idx, bufs, 10, 100)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        _call(idx, bufs, 10, 100)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, f"free device memory changed by {free0 - free1} bytes"
    idx.close()


def test_noalloc_at_its_size_limit(tiny):
    """The documented limit: 16 * (ceil(n/32) + max_visits + 128) bytes up to
    64 MiB - 512. At the largest such n the call runs (the rows beyond the
    real index are never reached: the graph only names real rows) and gives
    the allocating entry point's results; one more 32-row word is rejected."""
    Q = tiny["Q"][:200]
    for mv in (MV, 1000, 777):
        idx = dev_index(tiny["X"], tiny["adj"], tiny["entry"], max_visits=mv)
        ref = run(idx, Q, 10, 100)
        words = ((64 << 20) - 512) // 16 - (mv + 128)
        bufs = _buffers(Q, 10)
        _call(idx, bufs, 10, 100, n=32 * words, mv=mv)
        assert_same(_fetch(bufs), ref, f"n at the limit, max_visits {mv}")
        with pytest.raises(pkg.RoarError) as e:
            _call(idx, bufs, 10, 100, n=32 * (words + 1), mv=mv)
        assert e.value.status == pkg.ROAR_EINVAL
        idx.close()
