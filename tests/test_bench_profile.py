"""The bench's roofline `traffic` comes from the committed ncu summary of the
FP32 search kernel, keyed by a hash of the kernel's source: the summary must
be of the current source (else the bench reports traffic null), and its
figures must parse. No GPU needed."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

SEARCH_SOURCES = ["paper_2408_08933_gb300/csrc/roar_search_kernel.cuh",
                  "paper_2408_08933_gb300/csrc/roar_search.cu",
                  "paper_2408_08933_gb300/csrc/roar_internal.cuh",
                  "paper_2408_08933_gb300/csrc/roar_search_f32.cu"]


def test_search_profile_matches_kernel_source():
    h = bench._src_hash(SEARCH_SOURCES)
    t = bench._traffic("search_f32_base_1m_d200.txt", h)
    assert t is not None, "profiles/search_f32_base_1m_d200.txt was not captured on the current kernel source"
    # DRAM bytes of one 10k-query launch: above the algorithmic 19.78 GB, far below 2x.
    assert 19.78e9 < t < 2 * 19.78e9


def test_traffic_ignores_a_stale_summary():
    assert bench._traffic("search_f32_base_1m_d200.txt", "0" * 16) is None
    assert bench._traffic("no_such_summary.txt", bench._src_hash(SEARCH_SOURCES)) is None


def test_algorithmic_bytes_formula():
    # V*d*b + H*R*4 + 4d per query (the bench's roofline numerator)
    got = bench._algorithmic_bytes(2453.5, 110.84, 31.86, 200, 4, 0)
    assert abs(got - (2453.5 * 800 + 110.84 * 31.86 * 4 + 800)) < 1e-6 * got
