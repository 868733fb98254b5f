"""Largest sizes: instance indices past 2^31 and 2^32 (64-bit index and
seed-word arithmetic), the intrinsic Philox key at its 2^32 limit, and
lattices too large for a plan of co-resident strips (the per-half-sweep
fallback) or large enough that the strips stream their generator states
through L2.  Outputs are checked on sampled instances and rows against the
oracle, or through properties that hold at any size."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu
SEED = 0x0123456789ABCDEF


@pytest.fixture(scope="module")
def R():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1204_6193_gb300 as R
    return R


def sampled_generation(R, kind, n, K, samples, flags=0):
    import torch
    h = R.rng_create(kind, n, flags)
    try:
        R.rng_seed(h, SEED)
        out = torch.empty(n * K, dtype=torch.int32, device="cuda")
        R.rng_generate_u32(h, out.data_ptr(), K, R.RNG_STEP_MAJOR)
        torch.cuda.synchronize()
        view = out.view(K, n)
        for i in samples:
            got = view[:, i].cpu().numpy().view(np.uint32)
            ref = O.generate(kind, SEED, n, K, flags=flags, i_lo=i, i_hi=i + 1)[0]
            assert np.array_equal(got, ref), (kind, i)
        del out, view
    finally:
        R.rng_destroy(h)
        torch.cuda.synchronize()
        torch.cuda.empty_cache()


def test_lcg32_past_2_32_instances(R):
    n = (1 << 32) + 96
    sampled_generation(R, O.LCG32, n, 2, [0, (1 << 31) - 1, 1 << 31, (1 << 32) - 1, 1 << 32, n - 1])


def test_xorwow_past_2_31_instances(R):
    n = (1 << 31) + 64
    sampled_generation(R, O.XORWOW, n, 1, [0, (1 << 31) - 1, 1 << 31, n - 1])


def test_intrinsic_philox_keys_at_2_32(R):
    n = 1 << 32
    sampled_generation(R, O.PHILOX4X32_7, n, 1, [0, (1 << 31) + 5, n - 1], flags=O.PHILOX_INTRINSIC_KEY)


@pytest.mark.parametrize("layout", [0, 1])
def test_8192_lattice_bit_exact(R, layout):
    # int8: no plan of co-resident strips fits, so the sweep runs the
    # per-half-sweep kernels; multispin: 43 strips whose generator states
    # stream through L2
    ref, acc, nm = O.ising_run(8192, 0.44, O.XORWOW, SEED, 2, measure_every=1)
    h = R.ising_create(8192, 0.44, layout, O.XORWOW, 0, SEED, 2)
    try:
        R.ising_sweep(h, 2, 1)
        obs = R.ising_observables(h)
        assert np.array_equal(R.ising_get_spins(h), ref)
        assert obs["acc"] == acc.tolist() and obs["n_meas"] == nm
    finally:
        R.ising_destroy(h)


def test_16384_lattice_infinite_temperature(R):
    # beta = 0 accepts every proposal: one sweep flips all 2^28 spins
    L = 16384
    init = O.ising_init_spins(L, SEED)
    E0, M0 = O.ising_energy(init)
    h = R.ising_create(L, 0.0, 0, O.XS1024W, 0, SEED, 2)
    try:
        R.ising_sweep(h, 1)
        obs = R.ising_observables(h)
        assert (obs["E"], obs["M"]) == (E0, -M0)
        got = R.ising_get_spins(h)
        for y in (0, 1, L // 2, L - 1):
            assert np.array_equal(got[y], -init[y])
        assert np.array_equal(got, -init)
    finally:
        R.ising_destroy(h)
