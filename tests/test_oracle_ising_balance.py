"""Exact transition matrix of the oracle's checkerboard Metropolis update
(Sec. 2, application test) on 2x2 and 4x4 tori, and its stationary
distribution against the Boltzmann weights.

The oracle's own sweep code runs on every configuration with numbers the
test chooses.  An acceptance test compares a 32-bit draw r with the
thresholds T[4], T[8], so the draws fall into three classes, [0, T8), [T8,
T4) and [T4, 2^32); each class is entered at both of its edges, and both
edges must give the same result (an off-by-one such as r <= T fails here).
Weighting the classes by their widths gives the exact probability of every
transition as a fraction over 2^32.  The tests then check, with no tolerance,
that a site's acceptance probability is 1 for dE <= 0 and T[dE] / 2^32
otherwise, dE taken from the energy function itself; that the sites of a
half-sweep move independently (random draw vectors); that a sweep is the
colour-0 half-sweep followed by the colour-1 one and a multi-hit round the
documented sequence of strip half-sweeps; and that the Boltzmann weights
are stationary under every half-sweep to within what the integer thresholds
allow (|T/2^32 - e^(-beta dE)| < 2^-32).  On the 2x2 torus the whole
sweep's matrix is built in exact rationals and the Boltzmann vector checked
against it."""
from fractions import Fraction

import numpy as np
import pytest

import oracle as O

mp = pytest.importorskip("mpmath")
TWO32 = 1 << 32
BETA_C = float(np.log(1 + np.sqrt(2)) / 2)


def exact_threshold(beta, dE):
    # floor(2^32 exp(-beta dE)), evaluated to 50 digits
    with mp.workdps(50):
        return int(mp.floor(mp.mpf(2) ** 32 * mp.exp(-mp.mpf(beta) * dE)))


def all_configs(L):
    n = L * L
    idx = np.arange(1 << n, dtype=np.int64)
    bits = (idx[:, None] >> np.arange(n)) & 1  # site j = y L + x <-> bit j
    return (1 - 2 * bits).astype(np.int8).reshape(-1, L, L)


def config_index(spins):
    L = spins.shape[-1]
    b = (spins.reshape(spins.shape[0], L * L) < 0).astype(np.int64)
    return (b << np.arange(L * L)).sum(axis=1)


def energy(spins):
    # E = -sum over the bonds of the torus (each site's right and lower bond)
    s = spins.astype(np.int64)
    return -(s * np.roll(s, -1, axis=2) + s * np.roll(s, -1, axis=1)).sum(axis=(1, 2))


def colour_sites(L, c):
    return [y * L + x for y in range(L) for x in range(L) if (x + y) & 1 == c]


def classes(beta):
    """(lower edge, upper edge, width) of the draw classes that the two
    thresholds cut [0, 2^32) into (empty classes dropped)."""
    t4, t8 = exact_threshold(beta, 4), exact_threshold(beta, 8)
    assert O.ising_threshold(beta, 4) == t4 and O.ising_threshold(beta, 8) == t8
    cuts = sorted({0, min(t8, TWO32), min(t4, TWO32), TWO32})
    return [(a, b - 1, b - a) for a, b in zip(cuts, cuts[1:]) if b > a], t4, t8


def per_site_numerators(L, beta, c, G, cfg, rows=None):
    """A[sigma, j]: 2^32 x the probability that colour-c site j flips in one
    half-sweep of the oracle from configuration sigma (0 for sites the
    half-sweep does not touch).  Asserts that the draw classes are
    homogeneous and that nothing outside colour c changes."""
    n_cfg = cfg.shape[0]
    sites = colour_sites(L, c)
    if rows is not None:
        sites = [j for j in sites if rows[0] <= j // L < rows[1]]
    cls, _, _ = classes(beta)
    A = np.zeros((n_cfg, L * L), dtype=object)
    flips_of_class = []
    for lo, hi, width in cls:
        outs = []
        for r in (lo, hi):
            draws = np.full((n_cfg, L * L // 2), r, dtype=np.uint32)
            outs.append(O.ising_half_sweep_given(cfg, beta, c, draws, G=G, rows=rows))
        assert np.array_equal(outs[0], outs[1]), f"class [{lo}, {hi}] is not homogeneous"
        flipped = (outs[0] != cfg).reshape(n_cfg, L * L)
        untouched = [j for j in range(L * L) if j not in sites]
        assert not flipped[:, untouched].any(), "a site outside the half-sweep changed"
        flips_of_class.append(flipped)
        A[:, sites] += flipped[:, sites].astype(object) * width
    return A, sites, cls, flips_of_class


def flip_energy_change(cfg, j):
    L = cfg.shape[-1]
    other = cfg.copy().reshape(cfg.shape[0], L * L)
    other[:, j] = -other[:, j]
    return energy(other.reshape(cfg.shape)) - energy(cfg)


# (L, G) pairs with G dividing L/2, as the library requires
@pytest.mark.parametrize("L,G", [(2, 1), (4, 1), (4, 2)])
@pytest.mark.parametrize("beta", [0.0, 0.3, BETA_C, 2.0])
def test_acceptance_is_exactly_the_quantised_metropolis_rule(L, G, beta):
    cfg = all_configs(L)
    _, t4, t8 = classes(beta)
    T = {4: min(t4, TWO32), 8: min(t8, TWO32)}
    for c in (0, 1):
        A, sites, _, _ = per_site_numerators(L, beta, c, G, cfg)
        for j in sites:
            dE = flip_energy_change(cfg, j)
            want = np.array([TWO32 if d <= 0 else T[int(d)] for d in dE], dtype=object)
            assert (A[:, j] == want).all(), (c, j)


@pytest.mark.parametrize("G", [1, 2])
def test_sites_of_a_half_sweep_move_independently(G):
    # random draw vectors: every site does what its own draw's class says
    L, beta = 4, 0.35
    rng = np.random.default_rng(11 + G)
    cfg = all_configs(L)
    for c in (0, 1):
        _, sites, cls, flips = per_site_numerators(L, beta, c, G, cfg)
        edges = np.array([lo for lo, _, _ in cls[1:]], dtype=np.uint64)
        for _ in range(3):
            draws = rng.integers(0, TWO32, size=(cfg.shape[0], L * L // 2), dtype=np.uint64)
            # a quarter of the draws sit on a class edge
            on_edge = rng.random(draws.shape) < 0.25
            pick = np.array([lo for lo, _, _ in cls] + [hi for _, hi, _ in cls], dtype=np.uint64)
            draws[on_edge] = rng.choice(pick, size=int(on_edge.sum()))
            out = O.ising_half_sweep_given(cfg, beta, c, draws.astype(np.uint32), G=G)
            got = (out != cfg).reshape(cfg.shape[0], L * L)
            # stream sidx's draw g drives colour-c site q = sidx G + g
            for j in sites:
                y, x = divmod(j, L)
                q = y * (L // 2) + (x >> 1)
                d = draws[:, q]
                k = np.searchsorted(edges, d, side="right")
                want = np.choose(k, [f[:, j] for f in flips])
                assert np.array_equal(got[:, j], want), (c, j)


def stationarity_defect(L, beta, c, G, rows=None):
    """max over sigma' of |(pi P_c)(sigma') - pi(sigma')| / pi(sigma') for the
    Boltzmann weights pi and the oracle's exact half-sweep matrix P_c."""
    cfg = all_configs(L)
    A, sites, _, _ = per_site_numerators(L, beta, c, G, cfg, rows=rows)
    a = (A[:, sites].astype(np.float64)) / TWO32
    E = energy(cfg).astype(np.float64)
    pi = np.exp(-beta * (E - E.min()))
    pi /= pi.sum()
    idx = np.arange(cfg.shape[0])
    masks = [1 << j for j in sites]
    out = np.zeros_like(pi)
    for sub in range(1 << len(sites)):
        m = 0
        prob = np.ones_like(pi)
        for k, mk in enumerate(masks):
            if sub >> k & 1:
                m |= mk
        src = idx ^ m
        for k in range(len(sites)):
            p_src = a[src, k]
            prob *= p_src if sub >> k & 1 else 1.0 - p_src
        out += pi[src] * prob
    return float(np.max(np.abs(out - pi) / pi))


@pytest.mark.parametrize("beta", [0.3, 0.4, BETA_C])
@pytest.mark.parametrize("c", [0, 1])
def test_boltzmann_weights_are_stationary_under_each_half_sweep(beta, c):
    # each accepted uphill move has probability T/2^32 = e^(-beta dE) - d,
    # 0 <= d < 2^-32; over the 8 sites of a half-sweep that moves
    # (pi P)(sigma') from pi(sigma') by less than 8 e^(8 beta) 2^-32
    bound = 8 * np.exp(8 * beta) * 2.0**-32
    defect = stationarity_defect(4, beta, c, 2)
    assert defect < bound, (defect, bound)


@pytest.mark.parametrize("rows", [(0, 2), (2, 4), (1, 3)])
def test_strip_half_sweeps_keep_the_boltzmann_weights(rows):
    # the half-sweeps of a multi-hit phase touch the rows of one strip only
    beta = 0.4
    bound = 8 * np.exp(8 * beta) * 2.0**-32
    for c in (0, 1):
        assert stationarity_defect(4, beta, c, 2, rows=rows) < bound


def test_a_sweep_is_colour_0_then_colour_1():
    L, G, beta = 4, 2, 0.4
    rng = np.random.default_rng(5)
    cfg = all_configs(L)
    draws = rng.integers(0, TWO32, size=(cfg.shape[0], L * L // 2 // G, 2 * G), dtype=np.uint64).astype(np.uint32)
    got = O.ising_sweep_given(cfg, beta, draws, G=G)
    half0 = O.ising_half_sweep_given(cfg, beta, 0, np.ascontiguousarray(draws[:, :, :G]), G=G)
    want = O.ising_half_sweep_given(half0, beta, 1, np.ascontiguousarray(draws[:, :, G:]), G=G)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("k,strips", [(1, 2), (2, 2), (2, 4)])
def test_a_multihit_round_is_its_strip_half_sweeps_in_order(k, strips):
    # phase C = 0, 1; in each, k hits of (colour 0, colour 1) over the strips
    # of coarse colour C; stream sidx takes its next G numbers each time
    L, G, beta = 8, 2, 0.4
    rng = np.random.default_rng(100 + k + strips)
    n = 4096
    cfg = rng.choice(np.array([-1, 1], dtype=np.int8), size=(n, L, L))
    nst = L * L // 2 // G
    draws = rng.integers(0, TWO32, size=(n, nst, 2 * k * G), dtype=np.uint64).astype(np.uint32)
    got = O.ising_multihit_round_given(cfg, beta, draws, k=k, n_strips=strips, G=G)
    rows = L // strips
    used = 0 * np.arange(nst)
    want = cfg.copy()
    for C in (0, 1):
        for _ in range(k):
            for c in (0, 1):
                for b in range(C, strips, 2):
                    r0, r1 = b * rows, (b + 1) * rows
                    s0, s1 = r0 * (L // 2) // G, r1 * (L // 2) // G
                    d = np.zeros((n, nst, G), dtype=np.uint32)
                    for g in range(G):
                        d[:, s0:s1, g] = draws[np.arange(n)[:, None], np.arange(s0, s1)[None, :],
                                               used[s0:s1][None, :] + g]
                    used[s0:s1] += G
                    want = O.ising_half_sweep_given(want, beta, c, d, G=G, rows=(r0, r1))
    assert (used == 2 * k * G).all()
    assert np.array_equal(got, want)


def test_2x2_sweep_keeps_the_boltzmann_weights_exactly_up_to_quantisation():
    # The whole sweep's matrix, P = P_0 P_1 in exact rationals.  On the 2x2
    # torus the two stripe configurations have dE = 0 at every site, so
    # Metropolis flips them into each other with certainty: the chain is
    # reducible and its stationary vector is not unique (the null space of
    # P^T - I is 3-dimensional).  The Boltzmann vector must be one of them.
    sympy = pytest.importorskip("sympy")
    L, G, beta = 2, 1, 0.3
    cfg = all_configs(L)
    n = cfg.shape[0]
    mats = []
    for c in (0, 1):
        A, sites, _, _ = per_site_numerators(L, beta, c, G, cfg)
        P = [[Fraction(0)] * n for _ in range(n)]
        for i in range(n):
            for sub in range(1 << len(sites)):
                p = Fraction(1)
                dst = i
                for k, j in enumerate(sites):
                    aj = Fraction(int(A[i, j]), TWO32)
                    if sub >> k & 1:
                        p *= aj
                        dst ^= 1 << j
                    else:
                        p *= 1 - aj
                P[i][dst] += p
        mats.append(sympy.Matrix(n, n, lambda i, j, P=P: sympy.Rational(P[i][j].numerator, P[i][j].denominator)))
    P = mats[0] * mats[1]  # a sweep: colour 0, then colour 1 (row vectors)
    assert all(sum(P.row(i)) == 1 for i in range(n))
    stripes = [int(config_index(np.array([[[-1, 1], [-1, 1]]], dtype=np.int8))[0]),
               int(config_index(np.array([[[1, -1], [1, -1]]], dtype=np.int8))[0])]
    assert P[stripes[0], stripes[1]] == 1 and P[stripes[1], stripes[0]] == 1
    E = energy(cfg)
    w = np.exp(-beta * (E - E.min()).astype(np.float64))
    w /= w.sum()
    Pf = np.array(P.evalf(30).tolist(), dtype=np.float64)
    defect = np.max(np.abs(w @ Pf - w) / w)
    assert defect < 4 * np.exp(8 * beta) * 2.0**-32, defect
