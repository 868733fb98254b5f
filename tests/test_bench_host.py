"""Host-side logic of bench.py that needs no GPU: which roof the roofline
line states, and the shard plan's cover of the instance range."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402

HBM = {"achieved": 2478.4, "peak": 6778.0, "unit": "GB/s", "frac": 0.3657, "peak_source": "measured"}
ISSUE = {"inst_per_output": 52.61, "achieved_tinst_s": 31.4, "peak_tinst_s": 40.27, "frac": 0.78,
         "peak_source": "152 SMs x 4 schedulers x 32 threads x 2070 MHz"}


def test_issue_roof_binds_when_closer():
    r = bench.binding_roof(HBM, ISSUE)
    assert r["bound"] == "alu" and r["frac"] == 0.78 and r["peak"] == 40.27
    assert r["unit"] == "T thread-instructions/s"
    assert abs(r["achieved"] / r["peak"] - r["frac"]) < 0.01


def test_hbm_roof_binds_for_streaming_kernels_and_without_counts():
    streaming = dict(HBM, achieved=7038.4, frac=1.038)
    assert bench.binding_roof(streaming, dict(ISSUE, frac=0.33))["bound"] == "hbm"
    r = bench.binding_roof(HBM, None)
    assert r["bound"] == "hbm" and r["frac"] == HBM["frac"] and r["unit"] == "GB/s"


def test_shard_ranges_cover_the_instances_once():
    for world in (1, 2, 3, 8):
        covered = []
        for rank in range(world):
            first, count, total = bench.shard_range(rank, world, 1000)
            assert total == 1000 * world
            covered += list(range(first, first + count))
        assert covered == list(range(1000 * world))
