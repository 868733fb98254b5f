"""Pins of the CPU oracle's Ising application test (CPU only): the exact
finite-lattice solution against brute force, the paper's printed exact row
and Onsager's infinite-lattice result; the checkerboard Metropolis chain
against the exact moments."""
import numpy as np
import pytest

import oracle as O
from ising_stats import jackknife_e_cv
from oracle import ising_exact as X

mp = pytest.importorskip("mpmath")
BETA_C = float(np.log(1 + np.sqrt(2)) / 2)


@pytest.mark.parametrize("beta", [0.2, 0.4, BETA_C, 0.6])
def test_kaufman_matches_brute_force_4x4(beta):
    lz, mE, mE2 = X.brute_force_moments(4, beta)
    lz2, mE_, mE2_ = X.exact_moments(4, beta)
    assert abs(lz - lz2) < 1e-10
    assert abs(mE - mE_) < 1e-9
    assert abs(mE2 - mE2_) < 1e-7


def test_exact_row_of_table_1(golden):
    # Table 1, row "exact": e = 1.106079207, C_V = 0.8616983594 (L = 1024,
    # beta = 0.4).  The closed form evaluated at 40 digits gives
    # 1.1060792037 and 0.8616983568: both within 4e-9 of the printed values,
    # three orders of magnitude below the table's smallest statistical error
    # (1.4e-6), so the printed row is read as carrying ~3e-9 numerical error.
    g = golden["ising_exact_1024_beta04"]
    e, cv = X.exact_e_cv(g["L"], g["beta"])
    assert abs(e - g["e"]) < 5e-9
    assert abs(cv - g["C_V"]) < 5e-9


def test_finite_lattice_agrees_with_onsager_at_beta_04():
    # Independent formula: Onsager's infinite-lattice free energy
    # -beta f = ln(2 cosh 2K) + (1/2pi) int_0^pi ln[(1 + sqrt(1 - k^2 sin^2 t))/2] dt,
    # k = 2 sinh 2K / cosh^2 2K.  At beta = 0.4 the correlation length is a
    # few sites, so the L = 1024 torus equals the infinite lattice to 1e-12.
    with mp.workdps(30):
        def f(K):
            k = 2 * mp.sinh(2 * K) / mp.cosh(2 * K) ** 2
            return mp.log(2 * mp.cosh(2 * K)) + mp.quad(
                lambda t: mp.log((1 + mp.sqrt(1 - k**2 * mp.sin(t) ** 2)) / 2), [0, mp.pi]) / (2 * mp.pi)
        K = mp.mpf("0.4")
        e_inf = float(mp.diff(f, K, 1))
        cv_inf = float(K**2 * mp.diff(f, K, 2))
    e, cv = X.exact_e_cv(1024, 0.4)
    assert abs(e - e_inf) < 1e-12
    assert abs(cv - cv_inf) < 1e-10


def test_threshold_is_floor_of_2_32_boltzmann_factor():
    with mp.workdps(50):
        for beta in [0.1, 0.3, 0.4, BETA_C, 0.6, 2.0]:
            for dE in (4, 8):
                exact = int(mp.floor(mp.mpf(2) ** 32 * mp.exp(-mp.mpf(beta) * dE)))
                assert O.ising_threshold(beta, dE) == exact
    assert O.ising_threshold(50.0, 4) == 0


def test_observables_of_simple_configurations():
    L = 8
    up = np.ones((L, L), dtype=np.int8)
    assert O.ising_energy(up) == (-2 * L * L, L * L)
    neel = np.fromfunction(lambda y, x: 1 - 2 * ((x + y) % 2), (L, L)).astype(np.int8)
    assert O.ising_energy(neel) == (2 * L * L, 0)


def test_initial_spins_are_balanced():
    s = O.ising_init_spins(256, 99)
    n = s.size
    assert set(np.unique(s)) == {-1, 1}
    assert abs(int(s.astype(np.int64).sum())) < 5 * np.sqrt(n)


@pytest.mark.parametrize("kind,flags", [(O.XORWOW, 0), (O.XS1024W, 0), (O.PHILOX4X32_10, 0), (O.LCG64, 0),
                                        (O.PHILOX4X32_7, O.PHILOX_INTRINSIC_KEY)])
@pytest.mark.parametrize("beta", [0.3, 0.4])
def test_checkerboard_chain_reproduces_exact_energy(kind, flags, beta):
    # Application test of Sec. 2 on a lattice whose exact values are cheap:
    # e and C_V of an 8x8 torus from 50 independent chains, pooled, with
    # jackknife errors over the chains
    L, chunks, per = 8, 50, 2000
    sE, sE2, nb = [], [], []
    for c in range(chunks):
        s0, _, _ = O.ising_run(L, beta, kind, 5000 + c, 200, flags=flags)  # equilibration
        s, acc, nm = O.ising_run(L, beta, kind, 9000 + c, per, measure_every=1, spins=s0, flags=flags)
        sE.append(acc[0])
        sE2.append(acc[1])
        nb.append(nm)
    (e_est, e_err), (cv_est, cv_err) = jackknife_e_cv(sE, sE2, nb, L * L, beta)
    e_ex, cv_ex = X.exact_e_cv(L, beta)
    assert abs(e_est - e_ex) < 4.5 * e_err, (e_est, e_ex, e_err)
    assert abs(cv_est - cv_ex) < 4.5 * cv_err, (cv_est, cv_ex, cv_err)


def test_zero_temperature_energy_never_increases():
    L = 16
    s = O.ising_init_spins(L, 3)
    E_prev = O.ising_energy(s)[0]
    for t in range(20):
        s, _, _ = O.ising_run(L, 50.0, O.XORWOW, 3 + t, 1, spins=s)
        E = O.ising_energy(s)[0]
        assert E <= E_prev
        E_prev = E


def test_isolated_flipped_spin_is_restored_at_zero_temperature():
    L = 8
    s = np.ones((L, L), dtype=np.int8)
    s[3, 4] = -1  # colour (4 + 3) & 1 = 1; neighbours all +1, dE = -8
    out, _, _ = O.ising_run(L, 50.0, O.PHILOX4X32_10, 1, 1, spins=s)
    assert np.all(out == 1)


def test_measurement_accumulators():
    L = 8
    s, acc, nm = O.ising_run(L, 0.4, O.XORWOW, 7, 10, measure_every=5)
    assert nm == 2
    s1, _, _ = O.ising_run(L, 0.4, O.XORWOW, 7, 5)
    E1, M1 = O.ising_energy(s1)
    E2, M2 = O.ising_energy(s)
    assert acc.tolist() == [E1 + E2, E1 * E1 + E2 * E2, M1 * M1 + M2 * M2, abs(M1) + abs(M2)]


def test_runs_are_deterministic_and_seeded():
    a = O.ising_run(16, 0.4, O.MWC, 11, 7)[0]
    b = O.ising_run(16, 0.4, O.MWC, 11, 7)[0]
    c = O.ising_run(16, 0.4, O.MWC, 12, 7)[0]
    assert np.array_equal(a, b) and not np.array_equal(a, c)


def test_infinite_temperature_flips_every_site_once_per_sweep():
    # beta = 0: T = 2^32 exceeds every 32-bit draw, so every proposal is accepted
    init = O.ising_init_spins(32, 5)
    out, _, _ = O.ising_run(32, 0.0, O.LCG64, 5, 1)
    assert np.array_equal(out, -init)
    out2, _, _ = O.ising_run(32, 0.0, O.LCG64, 5, 2)
    assert np.array_equal(out2, init)


# ------------------------------------------- multi-hit (double checkerboard)
def test_multihit_infinite_temperature_flips_k_times_per_round():
    init = O.ising_init_spins(16, 4)
    for k in (1, 2, 3):
        out, _, _ = O.ising_run_multihit(16, 0.0, O.XORWOW, 4, 1, k=k, n_strips=4)
        assert np.array_equal(out, init if k % 2 == 0 else -init)


def test_multihit_zero_temperature_energy_never_increases():
    s = O.ising_init_spins(16, 9)
    E_prev = O.ising_energy(s)[0]
    for t in range(10):
        s, _, _ = O.ising_run_multihit(16, 50.0, O.PHILOX4X32_10, 9 + t, 1, k=3, n_strips=2, spins=s)
        E = O.ising_energy(s)[0]
        assert E <= E_prev
        E_prev = E


@pytest.mark.parametrize("k,strips", [(1, 2), (5, 4)])
@pytest.mark.parametrize("beta", [0.3, 0.4])
def test_multihit_chain_reproduces_exact_energy(k, strips, beta):
    # single-site Metropolis steps in any order keep the Boltzmann weights:
    # e and C_V of an 8x8 torus from 50 independent chains, pooled, with
    # jackknife errors over the chains
    L, chunks, rounds = 8, 50, 2000 // k
    sE, sE2, nb = [], [], []
    for c in range(chunks):
        s0, _, _ = O.ising_run_multihit(L, beta, O.XORWOW, 300 + c, 100, k=k, n_strips=strips)
        _, acc, nm = O.ising_run_multihit(L, beta, O.XORWOW, 700 + c, rounds, k=k, n_strips=strips,
                                          measure_every=1, spins=s0)
        sE.append(acc[0])
        sE2.append(acc[1])
        nb.append(nm)
    (e_est, e_err), (cv_est, cv_err) = jackknife_e_cv(sE, sE2, nb, L * L, beta)
    e_ex, cv_ex = X.exact_e_cv(L, beta)
    assert abs(e_est - e_ex) < 4.5 * e_err, (e_est, e_ex, e_err)
    assert abs(cv_est - cv_ex) < 4.5 * cv_err, (cv_est, cv_ex, cv_err)


# ------------------------------- block-shared generators in the application test
SHARED = [O.MT19937_SHARED, O.LFIB521, O.LFIB1279]


@pytest.mark.parametrize("kind", SHARED)
def test_shared_generator_feeds_its_32_streams_in_lane_order(kind):
    # generator j serves streams 32j .. 32j+31; the d-th number of stream
    # 32j + l is word 32d + l of generator j's stream (seeded as generator j
    # of a generation call with ceil(streams / 32) generators)
    L, G, beta, seed = 16, 2, 0.44, 77
    nst = L * L // 2 // G              # 64 streams: 2 generators
    ngen = (nst + 31) // 32
    words = O.generate(kind, seed, ngen, 32 * 2 * G)  # one sweep: 2G numbers per stream
    draws = np.zeros((nst, 2 * G), dtype=np.uint32)
    for s in range(nst):
        j, l = divmod(s, 32)
        draws[s] = words[j, l::32][: 2 * G]
    s0 = O.ising_init_spins(L, seed)
    want = O.ising_sweep_given(s0[None], beta, draws[None], G=G)[0]
    got, _, _ = O.ising_run(L, beta, kind, seed, 1, G=G)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("kind", SHARED)
def test_shared_generator_infinite_and_zero_temperature(kind):
    init = O.ising_init_spins(32, 5)
    out, _, _ = O.ising_run(32, 0.0, kind, 5, 1)
    assert np.array_equal(out, -init)
    s = init
    E_prev = O.ising_energy(s)[0]
    for t in range(8):
        s, _, _ = O.ising_run(32, 50.0, kind, 5 + t, 1, spins=s)
        E = O.ising_energy(s)[0]
        assert E <= E_prev
        E_prev = E


@pytest.mark.parametrize("kind", SHARED)
def test_shared_generator_chain_reproduces_exact_energy(kind):
    # e and C_V of an 8x8 torus at beta = 0.4 from 50 independent chains
    L, beta, chunks, per = 8, 0.4, 50, 2000
    sE, sE2, nb = [], [], []
    for c in range(chunks):
        s0, _, _ = O.ising_run(L, beta, kind, 5000 + c, 200)
        _, acc, nm = O.ising_run(L, beta, kind, 9000 + c, per, measure_every=1, spins=s0)
        sE.append(acc[0])
        sE2.append(acc[1])
        nb.append(nm)
    (e_est, e_err), (cv_est, cv_err) = jackknife_e_cv(sE, sE2, nb, L * L, beta)
    e_ex, cv_ex = X.exact_e_cv(L, beta)
    assert abs(e_est - e_ex) < 4.5 * e_err, (e_est, e_ex, e_err)
    assert abs(cv_est - cv_ex) < 4.5 * cv_err, (cv_est, cv_ex, cv_err)


def test_shared_generator_multihit_needs_whole_warps_per_strip():
    # a warp's generator must lie within one strip: 8 x 8 with 4 strips has
    # 8 streams per strip
    with pytest.raises(O.OracleError):
        O.ising_run_multihit(8, 0.4, O.MT19937_SHARED, 1, 1, k=1, n_strips=4)
    out, _, _ = O.ising_run_multihit(32, 0.0, O.LFIB521, 3, 1, k=1, n_strips=2)
    assert np.array_equal(out, -O.ising_init_spins(32, 3))
