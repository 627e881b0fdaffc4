"""Host-side pieces of bench.py that need no GPU: the guard around the extra
measurements and the single-process max over ranks."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

pytest.importorskip("torch")
import bench  # noqa: E402


def test_extra_records_a_failure_in_place():
    assert bench.extra(lambda a, b: {"sum": a + b}, 2, 3) == {"sum": 5}
    err = bench.extra(lambda: 1 // 0)
    assert set(err) == {"error"} and err["error"].startswith("ZeroDivisionError")


def test_max_over_ranks_single_process():
    assert bench.max_over_ranks(3.25) == 3.25
