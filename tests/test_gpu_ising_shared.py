"""The block-shared generators in the application test (Sec. 4 and 5,
Table 1's lagged Fibonacci rows): MT19937 and the lagged Fibonacci
generators (521, 353) and (1279, 861), one generator per 32 streams feeding
them in lane order, through the C ABI, against the CPU oracle -- spins
bit-exact, integer observables and accumulators equal -- and the chain's e
and C_V against the exact L = 64 values."""
import numpy as np
import pytest

import oracle as O
from ising_stats import binned_library_run, jackknife_e_cv

pytestmark = pytest.mark.gpu

SEED = 0x0123456789ABCDEF
BETA_C = float(np.log(1 + np.sqrt(2)) / 2)
SHARED = [O.MT19937_SHARED, O.LFIB521, O.LFIB1279]


@pytest.fixture(scope="module")
def R():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1204_6193_gb300 as R
    return R


def gpu_run(R, L, beta, kind, n, *, layout=0, G=2, measure_every=0, plain=False, split=None):
    h = R.ising_create(L, beta, layout, kind, 0, SEED, G)
    try:
        for m in (split or [n]):
            (R.ising_sweep_plain if plain else R.ising_sweep)(h, m, measure_every)
        return R.ising_get_spins(h), R.ising_observables(h)
    finally:
        R.ising_destroy(h)


@pytest.mark.parametrize("kind", SHARED)
@pytest.mark.parametrize("layout", [0, 1])
@pytest.mark.parametrize("L", [64, 1024])
def test_100_sweeps_bit_exact(R, kind, layout, L):
    ref, acc, nm = O.ising_run(L, BETA_C, kind, SEED, 100, measure_every=10)
    spins, obs = gpu_run(R, L, BETA_C, kind, 100, layout=layout, measure_every=10)
    assert np.array_equal(spins, ref)
    assert obs["acc"] == acc.tolist() and obs["n_meas"] == nm
    assert (obs["E"], obs["M"]) == O.ising_energy(ref)


@pytest.mark.parametrize("kind", SHARED)
def test_ragged_generators_and_split_calls(R, kind):
    # 48^2 / 2 / 3 = 384 streams (12 generators), G = 3; L = 12: 36 streams,
    # a second generator with 4 used lanes; calls split mid-run (measure_every
    # counts the sweeps of each call, so every sweep is measured here)
    for L, G in ((48, 3), (12, 2), (96, 6)):
        ref, acc, nm = O.ising_run(L, 0.4, kind, SEED, 30, G=G, measure_every=1)
        spins, obs = gpu_run(R, L, 0.4, kind, 30, G=G, measure_every=1, split=[7, 1, 22])
        assert np.array_equal(spins, ref), (L, G)
        assert obs["acc"] == acc.tolist() and obs["n_meas"] == nm


@pytest.mark.parametrize("kind", SHARED)
def test_plain_entry_point_and_limits(R, kind):
    ref, _, _ = O.ising_run(64, 0.0, kind, SEED, 3)
    spins, _ = gpu_run(R, 64, 0.0, kind, 3, plain=True)
    assert np.array_equal(spins, ref)
    assert np.array_equal(spins, -O.ising_init_spins(64, SEED))  # beta = 0: every site flips each sweep
    h = R.ising_create(64, 0.4, 0, kind, 0, SEED, 2)
    try:
        assert R.ising_autotune(h, 8)["threads"] == 256  # nothing to tune
        with pytest.raises(R.RngError) as e:
            R.ising_sweep_multihit(h, 1, 2, 4)
        assert e.value.status == R.RNG_EUNSUPPORTED
    finally:
        R.ising_destroy(h)


@pytest.mark.parametrize("kind", SHARED)
def test_chain_samples_the_ising_distribution(R, kind):
    L, beta = 64, 0.4
    h = R.ising_create(L, beta, 0, kind, 0, SEED, 2)
    try:
        R.ising_sweep(h, 1000)
        sE, sE2, nb = binned_library_run(R, h, 40, lambda h: R.ising_sweep(h, 500, 1))
    finally:
        R.ising_destroy(h)
    (e, de), (cv, dcv) = jackknife_e_cv(sE, sE2, nb, L * L, beta)
    import json, os
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "exact_ising.json")) as f:
        ex = [c for c in json.load(f)["cases"] if c["L"] == L and abs(c["beta"] - beta) < 1e-12][0]
    print(f"kind {kind}: e={e:.6f}({de:.1e}) exact {ex['e']:.6f}; C_V={cv:.5f}({dcv:.1e}) exact {ex['C_V']:.5f}")
    assert abs(e - ex["e"]) < 4.5 * de
    assert abs(cv - ex["C_V"]) < 4.5 * dcv
