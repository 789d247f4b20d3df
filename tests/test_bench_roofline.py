"""Arithmetic of bench.py's rooflines, on hand-computed cases: the build's
sector-model and random-access rooflines, and the algorithmic bytes of the
kernels that the bench line's `roofline` divides by the measured time."""
import os
import sys
from types import SimpleNamespace

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    sys.path.insert(0, ROOT)
    import bench as b
    return b


def test_build_rooflines_by_hand(bench):
    st = {"n_pairs": 100, "n_locations": 100}
    r = bench.build_rooflines(1000, st, read32_gbs=1000.0, copy_gbs=5000.0, achieved_gbps=10.0)
    # sector model: 1 B per base + 64 B per pair + 16 B per location, all at the copy peak
    assert r["sector_model"]["bytes_per_bp"] == pytest.approx(9.0)
    assert r["sector_model"]["roofline_gbps"] == pytest.approx(5000.0 / 9.0, abs=0.05)
    assert r["sector_model"]["frac"] == pytest.approx(10.0 / (5000.0 / 9.0), abs=1e-4)
    # random-access model: the 64 pair bytes per pair at the random rate, the rest streamed
    ra = r["random_access_model"]
    assert ra["random_bytes_per_bp"] == pytest.approx(6.4)
    assert ra["stream_bytes_per_bp"] == pytest.approx(2.6)
    assert ra["roofline_gbps"] == pytest.approx(1.0 / (6.4 / 1000e9 + 2.6 / 5000e9) / 1e9, abs=0.05)
    # a random read is never faster than a copy, so this roofline is the lower one
    assert ra["roofline_gbps"] <= r["sector_model"]["roofline_gbps"]


def test_algorithmic_bytes_of_the_kernels(bench):
    s = 16
    w = SimpleNamespace(db_params={"sketch_size": s}, n_bp=5000, roffs=np.array([0, 150, 300, 450, 600], np.uint64),
                        n_seq=4, n_queries=2)
    st = {"n_windows": 40, "n_pairs": 500, "n_locations": 480, "n_keys": 60}
    slots = 40 * s
    assert bench.algorithmic_bytes("sketch_emit", w, st, None) == 5000 + 8.0 * slots
    assert bench.algorithmic_bytes("radix_pass", w, st, None) == (slots + 3 * 500) * 8.0 + 4 * 500 * 8.0
    assert bench.algorithmic_bytes("fin_emit", w, st, None) == 500 * 8.0 + 480 * 8.0 + 60 * 20.0
    ctr = np.zeros(28, np.int64)
    ctr[0], ctr[4] = 64, 39  # features looked up, buckets found
    k = bench.SCORE_KERNELS["classify_sort512"]
    ctr[7 + 3 * k: 10 + 3 * k] = (2, 39, 84)  # queries, found buckets, sectors
    assert bench.algorithmic_bytes("classify_sort512", w, st, ctr) == 28.0 * 2 + 8.0 * 39 + 32.0 * 84
    reads_in = 600 + 8 * 5 + 4 * 3
    assert bench.algorithmic_bytes("classify_lookup", w, st, ctr) == reads_in + 32.0 * 64 + 8.0 * 39 + 16.0 * 2
    # every scoring kernel has its own counter block
    blocks = sorted(bench.SCORE_KERNELS.values())
    assert blocks == list(range(len(blocks))) and 7 + 3 * max(blocks) + 2 < 28
