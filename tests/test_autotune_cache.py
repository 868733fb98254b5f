"""The cache of tuned launch shapes (ising_autotune_cached): host logic on
CPU with the library's calls replaced by fakes, and the real path on the
GPU."""
import json
import os

import numpy as np
import pytest

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture
def R():
    if not os.path.exists(os.path.join(ROOT, "paper_1204_6193_gb300", "_build", "librng_gb300.so")):
        pytest.fail("librng_gb300.so is not built (run __graft_entry__.build())")
    import paper_1204_6193_gb300 as R
    return R


def test_cache_hit_miss_and_keys_without_gpu(R, tmp_path, monkeypatch):
    lattices = {1: [(64, 0, 3)], 2: [(64, 0, 3), (128, 0, 5)]}
    calls = {"tune": 0, "set": []}
    monkeypatch.setattr(R, "ising_info", lambda h, i=0: {"n_lattices": len(lattices[h]), "L": lattices[h][i][0],
                                                          "layout": lattices[h][i][1], "kind": lattices[h][i][2],
                                                          "sweeps": 0})

    def tune(h, probe):
        calls["tune"] += 1

    monkeypatch.setattr(R, "ising_autotune", tune)
    monkeypatch.setattr(R, "ising_get_launch", lambda h: {"threads": 256 * h, "ctas_per_sm": h, "min_sites": 1024})
    monkeypatch.setattr(R, "ising_set_launch", lambda h, t, c, m: calls["set"].append((h, t, c, m)))
    monkeypatch.setattr(R, "ising_get_halo_depth", lambda h: 2)
    monkeypatch.setattr(R, "ising_set_halo_depth", lambda h, d: calls["set"].append((h, "depth", d)))
    path = str(tmp_path / "sub" / "autotune.json")
    a = R.ising_autotune_cached(1, path=path, device="fake/152")
    assert a == {"threads": 256, "ctas_per_sm": 1, "min_sites": 1024, "halo_depth": 2, "cached": False}
    assert calls["tune"] == 1
    b = R.ising_autotune_cached(1, path=path, device="fake/152")
    assert b["cached"] and calls["tune"] == 1 and calls["set"] == [(1, 256, 1, 1024), (1, "depth", 2)]
    # other lattices or another device: a miss, stored beside the first entry
    c = R.ising_autotune_cached(2, path=path, device="fake/152")
    d = R.ising_autotune_cached(1, path=path, device="other/76")
    assert not c["cached"] and not d["cached"] and calls["tune"] == 3
    with open(path) as f:
        assert len(json.load(f)) == 3
    # a damaged cache file is rebuilt, not fatal
    with open(path, "w") as f:
        f.write("{not json")
    assert not R.ising_autotune_cached(1, path=path, device="fake/152")["cached"]


@pytest.mark.gpu
def test_cached_shape_is_reused_on_the_gpu(R, tmp_path):
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    path = str(tmp_path / "autotune.json")
    seed = 0x0123456789ABCDEF
    ref, _, _ = O.ising_run(128, 0.42, O.XORWOW, seed, 20)
    shapes = []
    for _ in range(2):
        h = R.ising_create(128, 0.42, 0, O.XORWOW, 0, seed, 2)
        try:
            shapes.append(R.ising_autotune_cached(h, 8, path=path))
            assert R.ising_get_launch(h) == {k: shapes[-1][k] for k in ("threads", "ctas_per_sm", "min_sites")}
            R.ising_sweep(h, 20)
            assert np.array_equal(R.ising_get_spins(h), ref)
        finally:
            R.ising_destroy(h)
    assert not shapes[0]["cached"] and shapes[1]["cached"]
