"""Parity of the CUDA checkerboard Metropolis path (through the C ABI) with
the CPU oracle: spins bit-exact after the same sweeps from the same seeds,
integer observables and accumulators exactly equal."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

SEED = 0x0123456789ABCDEF
BETA_C = float(np.log(1 + np.sqrt(2)) / 2)
KINDS = [O.LCG32, O.LCG64, O.MWC, O.XORWOW, O.PHILOX4X32_10, O.XS1024W, O.PHILOX4X32_7]


@pytest.fixture(scope="module")
def R():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1204_6193_gb300 as R
    return R


def gpu_run(R, L, beta, kind, n, *, layout=0, G=2, flags=0, seed=SEED, mode="persist", measure_every=0):
    h = R.ising_create(L, beta, layout, kind, flags, seed, G)
    try:
        if mode == "persist":
            R.ising_sweep(h, n, measure_every)
        else:
            R.ising_sweep_plain(h, n, measure_every)
        return R.ising_get_spins(h), R.ising_observables(h)
    finally:
        R.ising_destroy(h)


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("layout", [0, 1])
@pytest.mark.parametrize("mode", ["persist", "plain"])
def test_100_sweeps_L64_bit_exact(R, kind, layout, mode):
    ref, acc, nm = O.ising_run(64, BETA_C, kind, SEED, 100, measure_every=10)
    spins, obs = gpu_run(R, 64, BETA_C, kind, 100, layout=layout, mode=mode, measure_every=10)
    assert np.array_equal(spins, ref)
    assert obs["acc"] == acc.tolist() and obs["n_meas"] == nm
    assert (obs["E"], obs["M"]) == O.ising_energy(ref)


@pytest.mark.parametrize("kind", [O.XORWOW, O.XS1024W])
@pytest.mark.parametrize("layout", [0, 1])
def test_100_sweeps_L1024_bit_exact(R, kind, layout):
    ref, acc, nm = O.ising_run(1024, BETA_C, kind, SEED, 100, measure_every=25)
    spins, obs = gpu_run(R, 1024, BETA_C, kind, 100, layout=layout, measure_every=25)
    assert np.array_equal(spins, ref)
    assert obs["acc"] == acc.tolist() and obs["n_meas"] == nm


@pytest.mark.parametrize("L,G,kind", [(16, 2, O.XORWOW), (16, 1, O.XS1024W), (48, 3, O.PHILOX4X32_10),
                                      (40, 4, O.MWC), (12, 2, O.LCG64), (256, 8, O.XS1024W),
                                      (192, 6, O.LCG32), (8, 4, O.XORWOW)])
def test_small_and_ragged_lattices(R, L, G, kind):
    ref, _, _ = O.ising_run(L, 0.4, kind, SEED, 60, G=G)
    for mode in ["persist", "plain"]:
        spins, _ = gpu_run(R, L, 0.4, kind, 60, G=G, mode=mode)
        assert np.array_equal(spins, ref), mode


def test_multispin_other_G(R):
    for L, G in [(128, 4), (192, 2), (128, 32)]:
        ref, _, _ = O.ising_run(L, 0.3, O.XORWOW, SEED, 40, G=G)
        for mode in ["persist", "plain"]:
            spins, _ = gpu_run(R, L, 0.3, O.XORWOW, 40, layout=1, G=G, mode=mode)
            assert np.array_equal(spins, ref), (L, G, mode)


@pytest.mark.parametrize("flags,kind", [(O.SEED_LEAPFROG, O.LCG32), (O.SEED_SUBSTREAM, O.XS1024W),
                                        (O.MWC_SAME_A, O.MWC), (O.PHILOX_INTRINSIC_KEY, O.PHILOX4X32_10),
                                        (O.PHILOX_INTRINSIC_KEY, O.PHILOX4X32_7)])
def test_seeding_flags(R, flags, kind):
    ref, _, _ = O.ising_run(64, 0.4, kind, SEED, 30, flags=flags)
    spins, _ = gpu_run(R, 64, 0.4, kind, 30, flags=flags)
    assert np.array_equal(spins, ref)


@pytest.mark.parametrize("layout", [0, 1])
def test_intrinsic_philox_keys_L1024(R, layout):
    # Sec. 7: key = (site-pair number, run word), counter = sweep number
    # (two sites per stream: a sweep draws exactly one 4-word block)
    flags = O.PHILOX_INTRINSIC_KEY
    ref, acc, nm = O.ising_run(1024, BETA_C, O.PHILOX4X32_7, SEED, 100, flags=flags, measure_every=20)
    spins, obs = gpu_run(R, 1024, BETA_C, O.PHILOX4X32_7, 100, layout=layout, flags=flags, measure_every=20)
    assert np.array_equal(spins, ref)
    assert obs["acc"] == acc.tolist() and obs["n_meas"] == nm
    # the keys take the seed's low half only: from the same start, a seed
    # that differs above bit 31 gives the same run
    h = R.ising_create(1024, BETA_C, layout, O.PHILOX4X32_7, flags, SEED ^ (0xABCD << 40), 2)
    try:
        R.ising_set_spins(h, O.ising_init_spins(1024, SEED))
        R.ising_sweep(h, 100)
        assert np.array_equal(R.ising_get_spins(h), ref)
    finally:
        R.ising_destroy(h)


def test_degenerate_temperatures(R):
    # beta = 0: every proposal accepted; beta = 50: zero-temperature quench
    for beta in [0.0, 50.0]:
        ref, _, _ = O.ising_run(64, beta, O.PHILOX4X32_10, SEED, 20)
        spins, _ = gpu_run(R, 64, beta, O.PHILOX4X32_10, 20)
        assert np.array_equal(spins, ref)
    # beta = 0 accepts every proposal: one sweep flips every site once
    spins, _ = gpu_run(R, 64, 0.0, O.XORWOW, 1, layout=1)
    assert np.array_equal(spins, -O.ising_init_spins(64, SEED))


def test_chunk_boundary_and_measurement_phase(R):
    # more sweeps than one persistent launch holds, measurements straddling it
    ref, acc, nm = O.ising_run(32, 0.44, O.XS1024W, SEED, 5000, measure_every=7)
    spins, obs = gpu_run(R, 32, 0.44, O.XS1024W, 5000, measure_every=7)
    assert np.array_equal(spins, ref)
    assert obs["acc"] == acc.tolist() and obs["n_meas"] == nm


@pytest.mark.parametrize("layout", [0, 1])
def test_many_short_launches(R, layout):
    # one-sweep launches back to back: each launch restarts its halo tags;
    # odd sweep counts per launch (the int8 two-row-halo loop takes two
    # sweeps per pass)
    ref, _, _ = O.ising_run(1024, 0.44, O.XORWOW, SEED, 6)
    h = R.ising_create(1024, 0.44, layout, O.XORWOW, 0, SEED, 2)
    try:
        for n in (1, 1, 1, 3):
            R.ising_sweep(h, n)
        assert np.array_equal(R.ising_get_spins(h), ref)
    finally:
        R.ising_destroy(h)


def test_calls_compose_and_checkpoint_restores(R):
    L, beta, kind = 128, 0.42, O.XORWOW
    ref, _, _ = O.ising_run(L, beta, kind, SEED, 100)
    h = R.ising_create(L, beta, 0, kind, 0, SEED, 2)
    try:
        R.ising_sweep(h, 50)
        spins50 = R.ising_get_spins(h)
        blob = R.rng_get_state(R.ising_get_rng(h))
        R.ising_sweep_plain(h, 30)
        R.ising_sweep(h, 20)
        assert np.array_equal(R.ising_get_spins(h), ref)
    finally:
        R.ising_destroy(h)
    h2 = R.ising_create(L, beta, 0, kind, 0, SEED + 1, 2)  # different seed, then restored
    try:
        R.ising_set_spins(h2, spins50)
        R.rng_set_state(R.ising_get_rng(h2), blob)
        R.ising_sweep(h2, 50)
        assert np.array_equal(R.ising_get_spins(h2), ref)
    finally:
        R.ising_destroy(h2)


def test_launch_shape_does_not_change_results(R):
    L, kind = 512, O.XS1024W
    ref, _, _ = O.ising_run(L, 0.4, kind, SEED, 20)
    for threads, per_sm, mins in [(256, 1, 0), (1024, 1, 0), (512, 4, 0), (0, 0, 0), (256, 1, 1 << 20)]:
        h = R.ising_create(L, 0.4, 0, kind, 0, SEED, 2)
        try:
            R.ising_set_launch(h, threads, per_sm, mins)
            R.ising_sweep(h, 20)
            assert np.array_equal(R.ising_get_spins(h), ref), (threads, per_sm)
        finally:
            R.ising_destroy(h)
    h = R.ising_create(L, 0.4, 1, kind, 0, SEED, 2)
    try:
        cfg = R.ising_autotune(h, 16)
        assert cfg["threads"] in (256, 512, 1024)
        R.ising_sweep(h, 20)
        assert np.array_equal(R.ising_get_spins(h), ref)
    finally:
        R.ising_destroy(h)


@pytest.mark.parametrize("L,layout", [(64, 0), (64, 1), (32, 0), (128, 1)])
@pytest.mark.parametrize("kind", [O.XORWOW, O.XS1024W, O.LCG64])
def test_whole_lattice_in_one_block(R, L, layout, kind):
    # one block holds the whole lattice, one stream per thread: a half-sweep
    # is one pass and one barrier, the edge rows also writing their halo
    # copies (as does the default shape wherever the streams fit one block);
    # 256 threads with 1024 sites per block split it into strips instead
    ref, acc, nm = O.ising_run(L, 0.43, kind, SEED, 40, measure_every=4)
    for shape in ((1024, 1, 1 << 16), (0, 0, 0), (256, 1, 1024)):
        h = R.ising_create(L, 0.43, layout, kind, 0, SEED, 2)
        try:
            R.ising_set_launch(h, *shape)
            R.ising_sweep(h, 40, 4)
            obs = R.ising_observables(h)
            assert np.array_equal(R.ising_get_spins(h), ref), shape
            assert obs["acc"] == acc.tolist() and obs["n_meas"] == nm, shape
        finally:
            R.ising_destroy(h)


@pytest.mark.parametrize("L", [1024, 512])
@pytest.mark.parametrize("layout", [0, 1])
@pytest.mark.parametrize("kind,flags", [(O.XORWOW, 0), (O.XS1024W, 0), (O.PHILOX4X32_7, O.PHILOX_INTRINSIC_KEY)])
def test_fixed_slot_exact_checkerboard(R, L, layout, kind, flags):
    # two blocks of 512 per SM: one strip of 2 to 4 rows per block, whose
    # first and last rows fill every thread's slot 0 and the rows between its
    # slot 1 (the fixed-slot kernel); one block of 1024 per SM with its roles
    # split by warp and a polling warp (the default shape at L = 1024); one
    # block of 512 per SM runs the general loop with up to four slots per thread
    ref, acc, nm = O.ising_run(L, BETA_C, kind, SEED, 30, flags=flags, measure_every=3)
    for shape in ((512, 2, 0), (0, 0, 0), (1024, 1, 0), (512, 1, 0)):
        h = R.ising_create(L, BETA_C, layout, kind, flags, SEED, 2)
        try:
            R.ising_set_launch(h, *shape)
            R.ising_sweep(h, 30, 3)
            obs = R.ising_observables(h)
            assert np.array_equal(R.ising_get_spins(h), ref), shape
            assert obs["acc"] == acc.tolist() and obs["n_meas"] == nm, shape
        finally:
            R.ising_destroy(h)


@pytest.mark.parametrize("L,G,kind,layout", [(1024, 2, O.XORWOW, 0), (1024, 2, O.XS1024W, 1), (768, 2, O.PHILOX4X32_10, 0),
                                             (768, 2, O.LCG64, 1), (1024, 4, O.MWC, 0), (512, 1, O.LCG32, 0),
                                             (1024, 2, O.PHILOX4X32_7, 1)])
def test_split_role_exact_checkerboard(R, L, G, kind, layout):
    # one block of 1024 threads per SM, one strip of R rows each (R = 3 .. 7
    # here, uneven): the first 2 L/(2G) threads hold the first and last rows
    # in slot 0, the other compute threads the first rows between, slot 1 the
    # rest, and the last warp polls the neighbours' rows
    ref, acc, nm = O.ising_run(L, BETA_C, kind, SEED, 30, G=G, measure_every=3)
    h = R.ising_create(L, BETA_C, layout, kind, 0, SEED, G)
    try:
        R.ising_set_launch(h, 1024, 1, 0)
        info = R.ising_plan_info(h)
        assert info["threads"] == 1024 and info["blocks"] == info["strips"] >= 2
        R.ising_sweep(h, 30, 3)
        obs = R.ising_observables(h)
        assert np.array_equal(R.ising_get_spins(h), ref)
        assert obs["acc"] == acc.tolist() and obs["n_meas"] == nm
    finally:
        R.ising_destroy(h)


def test_default_shape_at_L1024_is_one_strip_per_sm(R):
    # one strip of 6 or 7 rows per SM, 1024 threads (a halo of two rows: one
    # exchange per sweep)
    import torch
    h = R.ising_create(1024, BETA_C, 0, O.XORWOW, 0, SEED, 2)
    try:
        info = R.ising_plan_info(h)
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        assert info == {"groups": 1, "blocks": sms, "strips": sms, "threads": 1024}
    finally:
        R.ising_destroy(h)


@pytest.mark.parametrize("layout", [0, 1])
def test_streamed_generator_state(R, layout):
    # 256 threads x 4 slots per block cannot hold a 1024^2 strip's streams:
    # the kernel streams generator states through L2 every half-sweep
    L, kind = 1024, O.PHILOX4X32_10
    ref, acc, nm = O.ising_run(L, 0.42, kind, SEED, 12, measure_every=4)
    h = R.ising_create(L, 0.42, layout, kind, 0, SEED, 2)
    try:
        R.ising_set_launch(h, 256, 1)
        R.ising_sweep(h, 12, 4)
        assert np.array_equal(R.ising_get_spins(h), ref)
        assert R.ising_observables(h)["acc"] == acc.tolist()
    finally:
        R.ising_destroy(h)


def test_batch_streamed_state_matches_alone(R):
    Ls = [512, 256, 128, 64, 32, 16] * 2
    betas = [0.3 + 0.025 * b for b in range(len(Ls))]
    kinds = [O.XS1024W if b % 2 else O.XORWOW for b in range(len(Ls))]
    h = R.ising_batch_create(Ls, betas, kinds, SEED + 5, 2)
    try:
        R.ising_set_launch(h, 128, 1)
        R.ising_batch_sweep(h, 15)
        for b, L in enumerate(Ls):
            ref, _, _ = O.ising_run(L, betas[b], kinds[b], O.seed_word(SEED + 5, b), 15)
            assert np.array_equal(R.ising_batch_get_spins(h, b), ref), b
    finally:
        R.ising_destroy(h)


def test_batch_matches_lattices_alone(R):
    rng = np.random.default_rng(4)
    Ls = [16, 32, 64, 128, 256, 512, 16, 64, 32, 128, 256, 48]
    betas = rng.uniform(0.30, 0.60, len(Ls)).tolist()
    kinds = [O.XORWOW if b % 2 == 0 else O.XS1024W for b in range(len(Ls))]
    h = R.ising_batch_create(Ls, betas, kinds, SEED, 2)
    try:
        R.ising_batch_sweep(h, 30, 10)
        R.ising_batch_sweep(h, 30, 10)  # graph replay
        for b, L in enumerate(Ls):
            wb = O.seed_word(SEED, b)
            ref, acc, nm = O.ising_run(L, betas[b], kinds[b], wb, 60, measure_every=10)
            # two calls of 30: measurements after sweeps 10, 20, 30 of each call
            assert np.array_equal(R.ising_batch_get_spins(h, b), ref), b
            obs = R.ising_batch_observables(h, b)
            assert obs["n_meas"] == nm
            assert obs["acc"] == acc.tolist(), b
    finally:
        R.ising_destroy(h)


def test_batch_in_several_waves_matches_lattices_alone(R):
    # more streams of one kind than the device keeps in registers at once
    # (2048 per SM): that kind group runs as two waves of launches
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    cap = sms * 2048
    n512 = cap // (512 * 512 // 4) + 1
    Ls = [512] * n512 + [256, 64, 16] + [512, 512, 128, 32]
    kinds = [O.XORWOW] * (n512 + 3) + [O.XS1024W] * 4
    betas = [0.30 + 0.02 * b for b in range(len(Ls))]
    h = R.ising_batch_create(Ls, betas, kinds, SEED + 9, 2)
    try:
        info = R.ising_plan_info(h)
        assert info["groups"] == 3, info
        R.ising_batch_sweep(h, 12, 4)
        for b, L in enumerate(Ls):
            ref, acc, nm = O.ising_run(L, betas[b], kinds[b], O.seed_word(SEED + 9, b), 12, measure_every=4)
            assert np.array_equal(R.ising_batch_get_spins(h, b), ref), b
            obs = R.ising_batch_observables(h, b)
            assert obs["n_meas"] == nm and obs["acc"] == acc.tolist(), b
    finally:
        R.ising_destroy(h)


@pytest.mark.parametrize("L,G", [(1024, 2), (768, 2), (1024, 4)])
@pytest.mark.parametrize("layout", [0, 1])
@pytest.mark.parametrize("kind,flags", [(O.XORWOW, 0), (O.XS1024W, 0), (O.LCG32, 0), (O.PHILOX4X32_10, 0),
                                        (O.PHILOX4X32_7, O.PHILOX_INTRINSIC_KEY)])
def test_halo_depths_give_the_same_chain(R, L, G, layout, kind, flags):
    # one strip of 5 .. 7 rows per SM: boundary rows exchanged after every
    # half-sweep (depth 1) or once per sweep with the rows just outside each
    # strip updated from copies of the neighbours' streams (depth 2); both
    # equal the oracle, measurements included
    ref, acc, nm = O.ising_run(L, BETA_C, kind, SEED, 40, G=G, flags=flags, measure_every=3)
    for depth in (1, 2, 0):
        h = R.ising_create(L, BETA_C, layout, kind, flags, SEED, G)
        try:
            R.ising_set_launch(h, 1024, 1, 0)
            R.ising_set_halo_depth(h, depth)
            info = R.ising_plan_info(h)
            assert info["threads"] == 1024 and info["blocks"] == info["strips"] >= 2
            R.ising_sweep(h, 40, 3)
            obs = R.ising_observables(h)
            assert np.array_equal(R.ising_get_spins(h), ref), depth
            assert obs["acc"] == acc.tolist() and obs["n_meas"] == nm, depth
        finally:
            R.ising_destroy(h)
    with pytest.raises(R.RngError):
        h = R.ising_create(64, BETA_C, 0, O.XORWOW, 0, SEED, 2)
        try:
            R.ising_set_halo_depth(h, 3)
        finally:
            R.ising_destroy(h)


@pytest.mark.parametrize("depth", [1, 2])
def test_strip_that_stops_publishing_times_out_without_hanging(R, depth):
    import time
    h = R.ising_create(1024, 0.4, 0, O.XORWOW, 0, SEED, 2)
    try:
        R.ising_set_halo_depth(h, depth)
        info = R.ising_plan_info(h)
        assert info["strips"] >= 2
        R.ising_debug_mute_strip(h, 1, 20_000_000)  # 20 ms budget
        t0 = time.time()
        R.ising_sweep(h, 10)
        with pytest.raises(R.RngError) as e:
            R.ising_observables(h)
        assert e.value.status == R.RNG_ETIMEOUT
        assert time.time() - t0 < 30
    finally:
        R.ising_destroy(h)
    # the context is still usable
    ref, _, _ = O.ising_run(64, 0.4, O.XORWOW, SEED, 5)
    spins, _ = gpu_run(R, 64, 0.4, O.XORWOW, 5)
    assert np.array_equal(spins, ref)


def test_argument_errors(R):
    for args in [(63, 0.4, 0), (66, 0.4, 1), (64, -1.0, 0), (2, 0.4, 0)]:
        with pytest.raises(R.RngError):
            R.ising_create(args[0], args[1], args[2], O.XORWOW, 0, 1, 2)
    with pytest.raises(R.RngError) as e:  # block-shared kinds: one lattice per handle
        R.ising_batch_create([64, 32], [0.4, 0.4], [O.XORWOW, O.MT19937_SHARED], 1, 2)
    assert e.value.status == R.RNG_EUNSUPPORTED
    with pytest.raises(R.RngError):
        R.ising_create(64, 0.4, 0, O.XORWOW, 0, 1, 3)  # G does not divide L/2
