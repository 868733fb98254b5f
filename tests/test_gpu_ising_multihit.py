"""Parity of the multi-hit (double checkerboard) Ising update, Sec. 2 and the
k = 100 column of Table 1, with the CPU oracle: spins bit-exact after the
same rounds from the same seeds, accumulators exactly equal; and the
physics of the chain (e, C_V against the exact finite-lattice values)."""
import json
import os
import time

import numpy as np
import pytest

import oracle as O
from ising_stats import binned_library_run, jackknife_e_cv

pytestmark = pytest.mark.gpu

SEED = 0x0123456789ABCDEF
BETA_C = float(np.log(1 + np.sqrt(2)) / 2)
KINDS = [O.LCG32, O.LCG64, O.MWC, O.XORWOW, O.PHILOX4X32_10, O.XS1024W, O.PHILOX4X32_7]
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def R():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1204_6193_gb300 as R
    return R


def gpu_multihit(R, L, beta, kind, rounds, *, k, n_strips, layout=0, G=2, flags=0, measure_every=0,
                 calls=None):
    h = R.ising_create(L, beta, layout, kind, flags, SEED, G)
    try:
        for n in (calls or [rounds]):
            R.ising_sweep_multihit(h, n, k, n_strips, measure_every)
        return R.ising_get_spins(h), R.ising_observables(h)
    finally:
        R.ising_destroy(h)


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("layout", [0, 1])
def test_L64_k3_bit_exact(R, kind, layout):
    ref, acc, nm = O.ising_run_multihit(64, BETA_C, kind, SEED, 10, k=3, n_strips=4, measure_every=2)
    spins, obs = gpu_multihit(R, 64, BETA_C, kind, 10, k=3, n_strips=4, layout=layout, measure_every=2)
    assert np.array_equal(spins, ref)
    assert obs["acc"] == acc.tolist() and obs["n_meas"] == nm
    assert (obs["E"], obs["M"]) == O.ising_energy(ref)


@pytest.mark.parametrize("n_strips", [2, 8, 32])
@pytest.mark.parametrize("k", [1, 100])
def test_L64_strip_counts_and_hits(R, n_strips, k):
    rounds = 3 if k == 100 else 20
    ref, acc, nm = O.ising_run_multihit(64, 0.4, O.XS1024W, SEED, rounds, k=k, n_strips=n_strips, measure_every=1)
    spins, obs = gpu_multihit(R, 64, 0.4, O.XS1024W, rounds, k=k, n_strips=n_strips, measure_every=1)
    assert np.array_equal(spins, ref)
    assert obs["acc"] == acc.tolist() and obs["n_meas"] == nm


@pytest.mark.parametrize("kind", [O.XORWOW, O.XS1024W, O.PHILOX4X32_10])
@pytest.mark.parametrize("layout", [0, 1])
@pytest.mark.parametrize("n_strips", [256, 16])  # register-resident states; states streamed through L2
def test_L1024_bit_exact(R, kind, layout, n_strips):
    ref, acc, nm = O.ising_run_multihit(1024, BETA_C, kind, SEED, 2, k=5, n_strips=n_strips, measure_every=1)
    spins, obs = gpu_multihit(R, 1024, BETA_C, kind, 2, k=5, n_strips=n_strips, layout=layout, measure_every=1)
    assert np.array_equal(spins, ref)
    assert obs["acc"] == acc.tolist() and obs["n_meas"] == nm


@pytest.mark.parametrize("layout", [0, 1])
def test_k2_intrinsic_philox7_L1024(R, layout):
    # the k = 2 configuration of Sec. 7 with Philox4x32-7 and intrinsic keys:
    # a strip phase of two sweeps consumes two whole 4-word blocks per stream
    flags = O.PHILOX_INTRINSIC_KEY
    ref, acc, nm = O.ising_run_multihit(1024, BETA_C, O.PHILOX4X32_7, SEED, 3, k=2, n_strips=256, flags=flags,
                                        measure_every=1)
    spins, obs = gpu_multihit(R, 1024, BETA_C, O.PHILOX4X32_7, 3, k=2, n_strips=256, layout=layout, flags=flags,
                              measure_every=1)
    assert np.array_equal(spins, ref)
    assert obs["acc"] == acc.tolist() and obs["n_meas"] == nm


def test_other_G_and_seeding_flags(R):
    for L, G, kind, flags, layout in [(128, 4, O.XORWOW, 0, 1), (96, 3, O.MWC, O.MWC_SAME_A, 0),
                                      (64, 1, O.XS1024W, O.SEED_SUBSTREAM, 0), (128, 2, O.LCG32, O.SEED_LEAPFROG, 1)]:
        n_strips = 4 if L != 96 else 6
        ref, _, _ = O.ising_run_multihit(L, 0.42, kind, SEED, 4, k=4, n_strips=n_strips, G=G, flags=flags)
        spins, _ = gpu_multihit(R, L, 0.42, kind, 4, k=4, n_strips=n_strips, G=G, flags=flags, layout=layout)
        assert np.array_equal(spins, ref), (L, G, kind)


def test_launch_chunks_and_split_calls(R):
    # k = 1000 holds 4 rounds per launch: 6 rounds take two launches, the
    # measurements (every 4th round) straddle them, and calls compose
    ref, acc, nm = O.ising_run_multihit(64, 0.44, O.XORWOW, SEED, 6, k=1000, n_strips=2, measure_every=4)
    for calls in ([6], [1, 2, 3]):
        spins, obs = gpu_multihit(R, 64, 0.44, O.XORWOW, 6, k=1000, n_strips=2, measure_every=4, calls=calls)
        assert np.array_equal(spins, ref), calls
        if calls == [6]:
            assert obs["acc"] == acc.tolist() and obs["n_meas"] == nm


@pytest.mark.parametrize("kind", [O.XORWOW, O.XS1024W, O.PHILOX4X32_7])
@pytest.mark.parametrize("layout", [0, 1])
def test_fixed_slot_and_general_phase_loops_agree(R, kind, layout):
    # the usual plan (one stream of each coarse colour per thread: 16 strips
    # of 1024 streams, two per block) runs the fixed-slot phase loop; a set
    # launch shape of 256 threads runs the general loop, its states streamed
    # through L2: same spins and accumulators as the oracle
    L, k, n_strips = 256, 5, 16
    ref, acc, nm = O.ising_run_multihit(L, 0.43, kind, SEED, 3, k=k, n_strips=n_strips, measure_every=1)
    for shape in (None, (256, 1, 0)):
        h = R.ising_create(L, 0.43, layout, kind, 0, SEED, 2)
        try:
            if shape:
                R.ising_set_launch(h, *shape)
            R.ising_sweep_multihit(h, 3, k, n_strips, 1)
            obs = R.ising_observables(h)
            assert np.array_equal(R.ising_get_spins(h), ref), shape
            assert obs["acc"] == acc.tolist() and obs["n_meas"] == nm, shape
        finally:
            R.ising_destroy(h)


def test_degenerate_temperatures(R):
    # beta = 0 accepts every proposal: a round of odd k flips every site
    spins, _ = gpu_multihit(R, 64, 0.0, O.XORWOW, 1, k=3, n_strips=4, layout=1)
    assert np.array_equal(spins, -O.ising_init_spins(64, SEED))
    ref, _, _ = O.ising_run_multihit(64, 50.0, O.PHILOX4X32_10, SEED, 3, k=7, n_strips=8)
    spins, _ = gpu_multihit(R, 64, 50.0, O.PHILOX4X32_10, 3, k=7, n_strips=8)
    assert np.array_equal(spins, ref)


def test_plain_plan_unaffected_after_multihit(R):
    # the multi-hit plan is cached beside the plain one: a plain sweep after
    # multi-hit rounds continues every stream where the rounds left it
    h = R.ising_create(64, 0.4, 0, O.XORWOW, 0, SEED, 2)
    h2 = R.ising_create(64, 0.4, 0, O.XORWOW, 0, SEED, 2)
    try:
        R.ising_sweep_multihit(h, 2, 5, 4)
        R.ising_sweep(h, 7)
        R.ising_sweep_multihit(h2, 2, 5, 4)
        R.ising_sweep_plain(h2, 7)
        assert np.array_equal(R.ising_get_spins(h), R.ising_get_spins(h2))
        # 2 rounds of k = 5 plus 7 sweeps: 17 sweeps' worth of draws per stream
        assert R.ising_info(h)["sweeps"] == 17
    finally:
        R.ising_destroy(h)
        R.ising_destroy(h2)


def test_strip_that_stops_publishing_times_out_without_hanging(R):
    h = R.ising_create(256, 0.4, 0, O.XORWOW, 0, SEED, 2)
    try:
        R.ising_debug_mute_strip(h, 1, 20_000_000)  # 20 ms budget
        t0 = time.time()
        R.ising_sweep_multihit(h, 5, 4, 8)
        with pytest.raises(R.RngError) as e:
            R.ising_observables(h)
        assert e.value.status == R.RNG_ETIMEOUT
        assert time.time() - t0 < 30
    finally:
        R.ising_destroy(h)
    ref, _, _ = O.ising_run_multihit(64, 0.4, O.XORWOW, SEED, 2, k=2, n_strips=2)
    spins, _ = gpu_multihit(R, 64, 0.4, O.XORWOW, 2, k=2, n_strips=2)
    assert np.array_equal(spins, ref)


def test_argument_errors(R):
    h = R.ising_create(64, 0.4, 0, O.XORWOW, 0, SEED, 2)
    try:
        for k, n_strips in [(0, 4), (3, 3), (3, 6), (3, 0), (70000, 4),
                            (3, 64)]:  # 64 strips of one row: 16 streams, not whole warps
            with pytest.raises(R.RngError) as e:
                R.ising_sweep_multihit(h, 1, k, n_strips)
            assert e.value.status == R.RNG_EINVAL, (k, n_strips)
        R.ising_sweep_multihit(h, 0, 3, 4)  # zero rounds: nothing to do
    finally:
        R.ising_destroy(h)
    hb = R.ising_batch_create([64, 64], [0.4, 0.4], [O.XORWOW, O.XORWOW], SEED, 2)
    try:
        with pytest.raises(R.RngError) as e:
            R.ising_sweep_multihit(hb, 1, 3, 4)
        assert e.value.status == R.RNG_EUNSUPPORTED
    finally:
        R.ising_destroy(hb)


def _exact(L, beta):
    with open(os.path.join(HERE, "golden", "exact_ising.json")) as f:
        for c in json.load(f)["cases"]:
            if c["L"] == L and abs(c["beta"] - beta) < 1e-12:
                return c["e"], c["C_V"]
    raise KeyError((L, beta))


@pytest.mark.parametrize("k,n_strips,kind", [(100, 4, O.XS1024W), (1, 8, O.XORWOW)])
def test_multihit_chain_samples_the_ising_distribution(R, k, n_strips, kind):
    # each flip is a Metropolis step against the current neighbours (the
    # other coarse colour is frozen during a phase), so the chain keeps the
    # Boltzmann distribution: e and C_V match the exact L = 64 values
    L, beta, N = 64, 0.4, 64 * 64
    # k = 100: 200 rounds per bin, measurements 100 sweeps apart; e and C_V
    # from the pooled accumulators, jackknife errors over the bins
    bins, per_bin = 40, 200 if k > 1 else 2500
    h = R.ising_create(L, beta, 0, kind, 0, SEED, 2)
    try:
        R.ising_sweep_multihit(h, max(1, 2000 // k), k, n_strips)
        sE, sE2, nb = binned_library_run(R, h, bins, lambda h: R.ising_sweep_multihit(h, per_bin, k, n_strips, 1))
    finally:
        R.ising_destroy(h)
    (e, de), (cv, dcv) = jackknife_e_cv(sE, sE2, nb, N, beta)
    e_ex, cv_ex = _exact(L, beta)
    print(f"multi-hit k={k} strips={n_strips}: e={e:.6f}({de:.1e}) exact {e_ex:.6f} Delta_rel={(e - e_ex) / de:+.2f}; "
          f"C_V={cv:.5f}({dcv:.1e}) exact {cv_ex:.5f}")
    assert abs(e - e_ex) < 4.5 * de
    assert abs(cv - cv_ex) < 4.5 * dcv
