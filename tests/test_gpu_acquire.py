"""GPU AcquireNeighbors (Alg. 3, Sec. 4.2.3) through the C ABI against the
oracle's FP32 form, id for id."""
import numpy as np
import pytest

import oracle
import roarsynth as rs

pytestmark = pytest.mark.gpu
NONE = np.uint32(0xFFFFFFFF)


def _sorted_valid(X, x, cands):
    """The candidates the kernel must consider, in (delta, id) order with
    delta = -dot_fixed (the oracle's FP32 fixed-order dot)."""
    valid = [int(c) for c in cands if c != NONE]
    key = [(-float(oracle.dot_fixed(X[x], X[c])), c) for c in valid]
    return [c for _, c in sorted(key)]


def _case(X, nx, nc_choices, M, fill, seed):
    import torch

    import paper_2408_08933_gb300 as pkg

    n = X.shape[0]
    rng = np.random.default_rng(seed)
    C = max(nc_choices) if max(nc_choices) > 0 else 1
    xs = rng.integers(0, n, nx).astype(np.uint32)
    cand = np.full((nx, C), NONE, dtype=np.uint32)
    ncand = np.zeros(nx, dtype=np.int32)
    for i in range(nx):
        nc = int(rng.choice(nc_choices))
        row = rng.integers(0, n, nc).astype(np.uint32)
        if nc >= 4:
            row[rng.integers(0, nc)] = xs[i]                  # x itself
            row[rng.integers(0, nc)] = row[rng.integers(0, nc)]   # a duplicate
            row[rng.integers(0, nc)] = NONE                   # padding inside the row
        cand[i, :nc] = row
        ncand[i] = nc
    dev = torch.device("cuda:0")
    Xd = torch.from_numpy(X).to(dev)
    out, cnt, srt = pkg.acquire(Xd, torch.from_numpy(xs.view(np.int32)).to(dev),
                                torch.from_numpy(cand.view(np.int32)).to(dev), torch.from_numpy(ncand).to(dev),
                                M, fill, sorted_out=True)
    torch.cuda.synchronize()
    out = out.cpu().numpy().view(np.uint32)
    cnt = cnt.cpu().numpy()
    srt = srt.cpu().numpy().view(np.uint32)
    for i in range(nx):
        order = _sorted_valid(X, int(xs[i]), cand[i, :ncand[i]])
        ref = oracle.acquire_neighbors_f32(X, int(xs[i]), np.asarray(order, np.uint32), M, fill).tolist()
        assert cnt[i] == len(ref), (i, cnt[i], len(ref))
        assert out[i, :cnt[i]].tolist() == ref, i
        assert np.all(out[i, cnt[i]:] == NONE)
        assert srt[i, :len(order)].tolist() == order, i
        assert np.all(srt[i, len(order):] == NONE)


@pytest.mark.parametrize("M,fill", [(1, False), (8, True), (32, False), (32, True), (64, False)])
def test_acquire_matches_oracle_tiny(tiny, M, fill):
    _case(tiny["X"], 96, [0, 1, 37, 300], M, fill, seed=M + (100 if fill else 0))


def test_acquire_full_candidate_rows_d200():
    w = rs.scaled(rs.BASE_1M_D200, n=20_000)
    X = rs.base(w)
    _case(X, 24, [1024, 777], 32, False, seed=5)


def test_acquire_flags_bad_ids(tiny):
    import torch

    import paper_2408_08933_gb300 as pkg

    X = tiny["X"]
    n = X.shape[0]
    dev = torch.device("cuda:0")
    xs = np.array([0, n + 5, 1], dtype=np.uint32)
    cand = np.array([[1, 2, 3], [1, 2, 3], [2, n + 1, 3]], dtype=np.uint32)
    out, cnt = pkg.acquire(torch.from_numpy(X).to(dev), torch.from_numpy(xs.view(np.int32)).to(dev),
                           torch.from_numpy(cand.view(np.int32)).to(dev),
                           torch.tensor([3, 3, 3], dtype=torch.int32, device=dev), 4, False)
    cnt = cnt.cpu().numpy()
    assert cnt[0] >= 1 and cnt[1] == -1 and cnt[2] == -1
    assert np.all(out.cpu().numpy().view(np.uint32)[1:] == NONE)
