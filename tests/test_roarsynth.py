"""The seeded input generator shared by the oracle and the CUDA path: row
ranges regenerate exactly, rows are unit-norm, streams are distinct."""
import numpy as np

import roarsynth as rs


def test_row_ranges_regenerate_exactly():
    w = rs.scaled(rs.BASE_1M_D200, n=200_000, n_train=70_000, n_test=1_000)
    full = rs.base(w, 60_000, 140_000)                  # spans chunk boundaries
    part = rs.base(w, 100_000, 131_073)
    assert np.array_equal(full[40_000:71_073], part)
    assert np.array_equal(rs.train_queries(w, 0, 10), rs.train_queries(w)[:10])


def test_rows_are_unit_norm():
    w = rs.TINY
    for rows in (rs.base(w, 0, 500), rs.train_queries(w, 0, 500), rs.test_queries(w), rs.id_queries(w, 300)):
        nrm = np.linalg.norm(rows.astype(np.float64), axis=1)
        assert np.allclose(nrm, 1.0, atol=1e-6)


def test_streams_are_distinct():
    w = rs.TINY
    a, b, c = rs.base(w, 0, 50), rs.train_queries(w, 0, 50), rs.test_queries(w)[:50]
    assert not np.array_equal(a, b) and not np.array_equal(b, c)
    w2 = rs.scaled(rs.TINY, tag=99)
    assert not np.array_equal(rs.base(w2, 0, 50), a)


def test_queries_carry_the_offset():
    """The OOD offset moves the query mean along delta (the modality gap)."""
    w = rs.TINY
    u = rs.offset(w).astype(np.float64)
    u /= np.linalg.norm(u)
    shift_q = float((rs.train_queries(w, 0, 4000).astype(np.float64) @ u).mean())
    shift_x = float((rs.base(w, 0, 4000).astype(np.float64) @ u).mean())
    assert shift_q - shift_x > 0.05


def test_uneven_and_poisson_parameters_are_in_range():
    k, L = rs.uneven_params(5000)
    assert set(np.unique(k)) <= {1, 10, 100}
    assert np.all(L >= np.maximum(k, 10)) and np.all(L <= 500)
    t, size, kk, LL = rs.poisson_requests(1e5, 0.5)
    assert np.all(np.diff(t) > 0) and t.max() < 0.5
    assert np.all((size >= 1) & (size <= 256)) and np.all(LL >= kk)
