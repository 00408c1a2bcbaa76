"""Host-side argument checks of the C ABI: calls with bad sizes return
ROAR_EINVAL (with a message) before any CUDA call, so they run without a GPU."""
import ctypes

import pytest

EINVAL = 1
P = ctypes.c_void_p


@pytest.fixture(scope="module")
def lib():
    import paper_2408_08933_gb300 as pkg

    return pkg.lib()


def _msg(lib):
    return (lib.roar_last_error() or b"").decode()


def test_acquire_rejects_bad_sizes(lib):
    fake = P(16)   # never dereferenced: the checks come first
    for d, M, stride in ((6, 8, 16), (64, 0, 16), (64, 65, 16), (64, 8, 1025), (2048, 8, 16)):
        rc = lib.roar_acquire(fake, 100, d, fake, 4, fake, stride, fake, M, 0, fake, fake, None, None)
        assert rc == EINVAL, (d, M, stride)
        assert "roar_acquire" in _msg(lib)


def test_insert_rejects_bad_sizes(lib):
    fake = P(16)
    cases = [
        dict(n_total=100, d=64, R=8, entry=0, n_old=90, M=9, L=64, cap=64),     # M > R
        dict(n_total=100, d=64, R=8, entry=95, n_old=90, M=4, L=64, cap=64),    # entry not an old row
        dict(n_total=80, d=64, R=8, entry=0, n_old=90, M=4, L=64, cap=64),      # fewer rows than before
        dict(n_total=100, d=64, R=8, entry=0, n_old=90, M=4, L=64, cap=2000),   # N_out capacity
        dict(n_total=100, d=66, R=8, entry=0, n_old=90, M=4, L=64, cap=64),     # d % 4
        dict(n_total=100, d=64, R=8, entry=0, n_old=90, M=4, L=64, cap=64, win=0),     # window
        dict(n_total=100, d=64, R=8, entry=0, n_old=90, M=4, L=64, cap=64, win=5000),  # window
    ]
    for c in cases:
        rc = lib.roar_insert(fake, c["n_total"], c["d"], fake, c["R"], c["entry"], c["n_old"], fake, 10, fake,
                             fake, fake, c["cap"], c["M"], c["L"], c.get("win", 64), fake, None, None)
        assert rc == EINVAL, c
        assert "roar_insert" in _msg(lib)


def test_knn_rejects_bad_sizes(lib):
    fake = P(16)
    for d, kk, n in ((60, 10, 1000), (64, 129, 1000), (64, 50, 20), (1024, 10, 1000)):
        assert lib.roar_knn(fake, 10, fake, n, d, kk, fake, fake, None) == EINVAL, (d, kk, n)


def test_build_rejects_bad_sizes(lib):
    fake = P(16)
    st = (ctypes.c_double * 16)()
    entry = ctypes.c_uint32()
    for M, L, nqd in ((0, 100, 10), (80, 500, 10), (32, 16, 10), (32, 500, 1)):
        rc = lib.roar_build_index(fake, 1000, 64, fake, 100, nqd, M, L, 1, fake, None, ctypes.byref(entry), st, None)
        assert rc == EINVAL, (M, L, nqd)


def test_tombstones_need_a_handle(lib):
    assert lib.roar_index_set_tombstones(None, None) == EINVAL
