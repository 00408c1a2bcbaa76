"""Helpers for GPU tests: upload numpy arrays, run the library, fetch results."""
import numpy as np


def dev_index(X, adj, entry, dtype="f32", trav=None, scales=None, max_visits=16384):
    import torch

    import paper_2408_08933_gb300 as pkg

    d = torch.device("cuda:0")
    Xd = torch.from_numpy(np.ascontiguousarray(X, np.float32)).to(d)
    Ad = torch.from_numpy(np.ascontiguousarray(adj, np.uint32).view(np.int32)).to(d)
    Td = None if trav is None else torch.from_numpy(np.ascontiguousarray(trav)).to(d)
    Sd = None if scales is None else torch.from_numpy(np.ascontiguousarray(scales, np.float32)).to(d)
    return pkg.Index(Xd, Ad, entry, dtype=dtype, trav=Td, scales=Sd, max_visits=max_visits)


def run(idx, Q, k, L):
    import torch

    Qd = torch.from_numpy(np.ascontiguousarray(Q, np.float32)).to("cuda:0")
    ids, dist, visits, hops, st = idx.search(Qd, k, L)
    torch.cuda.synchronize()
    return (ids.cpu().numpy().view(np.uint32), dist.cpu().numpy(),
            visits.cpu().numpy().view(np.uint32), hops.cpu().numpy().view(np.uint32),
            st.cpu().numpy())


def assert_same(got, ref, what=""):
    """ids, visits, hops and status bit-exact; distances within 1e-6 relative."""
    gi, gd, gv, gh, gs = got
    ri, rd, rv, rh, rs = ref
    assert np.array_equal(gi, ri), f"{what}: ids differ in {np.sum(np.any(gi != ri, axis=1))} rows"
    assert np.array_equal(gv, rv), f"{what}: visits differ"
    assert np.array_equal(gh, rh), f"{what}: hops differ"
    assert np.array_equal(gs, rs), f"{what}: status differs"
    fin = np.isfinite(rd)
    assert np.array_equal(np.isfinite(gd), fin)
    assert np.all(np.abs(gd[fin] - rd[fin]) <= 1e-6 * np.abs(rd[fin])), f"{what}: dist differs"
