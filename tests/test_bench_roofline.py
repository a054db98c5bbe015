"""The roofline bookkeeping of bench.py on CPU: the stage kernel's algorithmic
bytes per element-stage equal the itemised list of what an element must move, and
a recorded ncu traffic figure that matches the current kernel sources lies just
above those bytes (more would mean re-reads)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _itemised(N, ts):
    Np = (N + 1) * (N + 2) // 2
    words = {"read Q (h, hu, hv)": 3 * Np, "read B": Np, "read two older R slots": 6 * Np,
             "read geometry": 4, "write R": 3 * Np, "write Q": 3 * Np, "write means": 3,
             "write P1 vertex values": 9}
    return sum(words.values()) * ts + 4 * 4 + 1      # + connectivity (4 int32) + dry byte


@pytest.mark.parametrize("ts", [4, 8])
@pytest.mark.parametrize("N", [1, 2, 3, 4, 5])
def test_stage_bytes_match_the_itemised_list(N, ts):
    import bench
    assert bench.stage_bytes_per_element(N, ts) == _itemised(N, ts)


def test_benchmark_order_figure():
    import bench
    assert bench.stage_bytes_per_element(4, 4) == 1041      # N = 4, FP32
    assert bench.stage_bytes_per_element(4, 8) == 2065      # N = 4, FP64


def test_recorded_traffic_is_close_to_the_algorithmic_bytes():
    import bench
    t = bench.recorded_traffic(4, "fp32tc")
    if t is None:
        pytest.skip("no ncu traffic recorded for the current kernel sources")
    ratio = t / bench.stage_bytes_per_element(4, 4)
    assert 1.0 <= ratio <= 1.15, ratio
