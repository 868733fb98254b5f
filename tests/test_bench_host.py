"""Host-side logic of bench.py that needs no GPU: which roof the roofline
line states, the algorithmic bytes of a call, and the shard plan's cover of
the instance range."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402

HBM = {"achieved": 2478.4, "peak": 6778.0, "unit": "GB/s", "frac": 0.3657, "peak_source": "measured"}
ALG = {"achieved": 30.2, "peak": 40.27, "unit": "T integer ops/s", "frac": 0.75, "ops_per_number": 8.0}


def test_write_calls_are_stated_against_hbm_whatever_the_issue_rate():
    # a call that writes its numbers is bound by the bytes it must move
    for form in ("u32", "f32", "normal"):
        r = bench.roof_of(form, HBM, ALG)
        assert r["bound"] == "hbm" and r["frac"] == HBM["frac"] and r["unit"] == "GB/s"


def test_consume_in_register_calls_are_stated_against_their_algorithmic_ops():
    r = bench.roof_of("u32_xor", HBM, ALG)
    assert r["bound"] == "alu" and r["frac"] == 0.75 and r["unit"] == "T integer ops/s"


def test_algorithmic_bytes_of_a_call():
    class FakeBulk:
        algorithmic_bytes = bench.Bulk.algorithmic_bytes
    b = FakeBulk()
    n, K = 1 << 20, 1024
    # output words plus the state's load and store (XORWOW: six words each way)
    assert b.algorithmic_bytes(("x", 3, "u32", None, n, K, 0)) == n * K * 4 + 48 * n
    assert b.algorithmic_bytes(("x", 3, "u32_xor", None, n, K, 0)) == n * 4 + 48 * n
    assert set(bench.ALG_OPS) == set(range(bench.N_KINDS))


def test_shard_ranges_cover_the_instances_once():
    for world in (1, 2, 3, 8):
        covered = []
        for rank in range(world):
            first, count, total = bench.shard_range(rank, world, 1000)
            assert total == 1000 * world
            covered += list(range(first, first + count))
        assert covered == list(range(1000 * world))
