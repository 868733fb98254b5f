"""Pins of the CPU oracle's generators against facts fixed by the paper, by
mathematics or by independent implementations (CPU only)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle as O

SEED = 0x0123456789ABCDEF
M64 = 2**64 - 1


def _bm_gf2(bits):
    """Berlekamp-Massey over GF(2): (connection polynomial as int, length)."""
    C, B, L, m = 1, 1, 0, 1
    for n, s in enumerate(bits):
        d = s
        for i in range(1, L + 1):
            if (C >> i) & 1:
                d ^= bits[n - i]
        if d == 0:
            m += 1
        elif 2 * L <= n:
            T = C
            C ^= B << m
            L, B, m = n + 1 - L, T, 1
        else:
            C ^= B << m
            m += 1
    return C, L


# --------------------------------------------------------------------- seeds
def test_mix64_is_a_bijection_by_inversion():
    # The inverse of each xorshift-multiply stage, derived independently: an
    # odd multiplier is inverted mod 2^64, x ^ (x >> s) by iterated unshifting.
    def unxorshift(x, s):
        y = x
        for _ in range(64 // s + 1):
            y = x ^ (y >> s)
        return y & M64

    inv1 = pow(0xBF58476D1CE4E5B9, -1, 2**64)
    inv2 = pow(0x94D049BB133111EB, -1, 2**64)
    rng = np.random.default_rng(7)
    for z in [0, 1, M64, *rng.integers(0, 2**63, 200, dtype=np.uint64).tolist()]:
        h = O.mix64(int(z))
        x = unxorshift(h, 31)
        x = (x * inv2) & M64
        x = unxorshift(x, 27)
        x = (x * inv1) & M64
        x = unxorshift(x, 30)
        assert x == int(z)


def test_seed_words_distinct():
    w = [O.seed_word(SEED, k) for k in range(100000)]
    assert len(set(w)) == len(w)


# ---------------------------------------------------------------------- LCG
@pytest.mark.parametrize("kind", [O.LCG32, O.LCG64])
def test_lcg_constants_are_the_papers(golden, kind):
    g = golden["lcg32" if kind == O.LCG32 else "lcg64"]
    m = 2 ** g["m_log2"]
    x = O.seed_word(SEED, 5) % m
    out = O.generate(kind, SEED, 8, 6, i_lo=5, i_hi=6)[0]
    for k in range(6):
        x = (g["a"] * x + g["c"]) % m  # Sec. 2, Eq. (1); output = new state
        expect = x if kind == O.LCG32 else x >> 32
        assert int(out[k]) == expect


@pytest.mark.parametrize("kind", [O.LCG32, O.LCG64])
@pytest.mark.parametrize("flags", [O.SEED_RANDOM, O.SEED_LEAPFROG])
def test_lcg_skip_ahead_matches_stepping(kind, flags):
    # Eq. (2) against the definition Eq. (1)
    for t in [1, 2, 3, 17, 1000, 4097]:
        a = O.generate(kind, SEED, 64, 8, flags=flags, skip=t, jump=True)
        b = O.generate(kind, SEED, 64, 8, flags=flags, skip=t, jump=False)
        assert np.array_equal(a, b), t


def test_lcg_jump_coefficient_reading():
    # c_t = sum_{i<t} a^i c satisfies Eq. (2) for t = 1: (a_1, c_1) = (a, c)
    assert O.lcg_jump_coeffs(False, 1) == (1664525, 1013904223)
    assert O.lcg_jump_coeffs(True, 1) == (2862933555777941757, 1442695040888963407)
    assert O.lcg_jump_coeffs(False, 0) == (1, 0)


def test_lcg_full_periods():
    # Every cycle length of an affine bijection mod 2^k is a power of two,
    # so "period 2^k" <=> the 2^(k-1)-step map is not the identity while
    # the 2^k-step map is (Sec. 2: p = m for suitable a, c).
    assert O.lcg_jump_coeffs(False, 2**32) == (1, 0)
    assert O.lcg_jump_coeffs(False, 2**31) != (1, 0)
    at, ct = O.lcg_jump_coeffs(True, 2**63)
    assert (at, ct) != (1, 0)
    # Hull-Dobell for m = 2^64: c odd, a = 1 mod 4
    assert 1442695040888963407 % 2 == 1 and 2862933555777941757 % 4 == 1


def test_lcg32_low_bit_periods(golden):
    # Sec. 2: the k-th least significant bit (1-based) has period 2^k
    s = O.generate(O.LCG32, SEED, 1, 1 << 14)[0].astype(np.int64)
    for b in range(12):
        bit = (s >> b) & 1
        p = 2 ** (b + 1)
        assert np.array_equal(bit[p:], bit[:-p]), b
        assert not np.array_equal(bit[p // 2:], bit[:-p // 2]), b


def test_lcg_leapfrog_is_the_serial_sequence():
    # Sec. 2: with t = number of instances, all instances together produce
    # the one global sequence; the step-major order is the serial order.
    n, K = 96, 20
    lf = O.generate(O.LCG32, SEED, n, K, flags=O.SEED_LEAPFROG)
    serial = O.generate(O.LCG32, SEED, 1, n * K, flags=O.SEED_LEAPFROG)[0]
    assert np.array_equal(lf.T.ravel(), serial)
    x = O.seed_word(SEED, 0) & 0xFFFFFFFF
    for k in range(5):
        x = (1664525 * x + 1013904223) % 2**32
        assert int(serial[k]) == x
    lf64 = O.generate(O.LCG64, SEED, n, K, flags=O.SEED_LEAPFROG)
    serial64 = O.generate(O.LCG64, SEED, 1, n * K, flags=O.SEED_LEAPFROG)[0]
    assert np.array_equal(lf64.T.ravel(), serial64)


# ---------------------------------------------------------------------- MWC
def test_mwc_first_multiplier_is_the_papers(golden):
    sympy = pytest.importorskip("sympy")
    a0 = golden["mwc"]["first_multiplier"]
    tab = O.mwc_multipliers(64)
    assert int(tab[0]) == a0
    # it is the largest: no a in (a0, 2^32) has both a 2^32 - 1, a 2^31 - 1 prime
    for a in range(a0 + 1, 2**32):
        assert not (sympy.isprime(a * 2**32 - 1) and sympy.isprime(a * 2**31 - 1))
    # the table is exactly the descending list of such a (no gaps)
    hits = [a for a in range(a0, int(tab[-1]) - 1, -1)
            if sympy.isprime(a * 2**32 - 1) and sympy.isprime(a * 2**31 - 1)]
    assert hits == [int(a) for a in tab]


def test_miller_rabin_against_sympy():
    sympy = pytest.importorskip("sympy")
    rng = np.random.default_rng(3)
    cands = [int(x) | 1 for x in rng.integers(2**40, 2**63, 3000, dtype=np.uint64)]
    cands += [2**61 - 1, 3825123056546413051, 318665857834031151167461 % 2**64, 2**64 - 59]
    for c in cands:
        assert O.is_prime_u64(c) == sympy.isprime(c), c


@pytest.mark.slow
def test_mwc_more_than_a_million_multipliers(golden):
    tab = O.mwc_multipliers(1 << 20)
    assert len(tab) == 1 << 20 >= golden["mwc"]["min_count"]
    assert np.all(np.diff(tab.astype(np.int64)) < 0)


@pytest.mark.parametrize("flags", [0, O.MWC_SAME_A])
def test_mwc_skip_ahead_matches_stepping(flags):
    for t in [1, 5, 999, 4096]:
        a = O.generate(O.MWC, SEED, 40, 6, flags=flags, skip=t, jump=True)
        b = O.generate(O.MWC, SEED, 40, 6, flags=flags, skip=t, jump=False)
        assert np.array_equal(a, b), t


def test_mwc_period_is_half_of_am_minus_2():
    # p = a 2^32 - 1 = 7 (mod 8), so 2 and hence a = 2^(-32) (mod p) are
    # quadratic residues: the order of a divides (p-1)/2, which is prime.
    # The period is therefore (a m - 2)/2, not the a m - 2 of Sec. 3.
    a = 4294967118
    p = a * 2**32 - 1
    q = (p - 1) // 2
    assert pow(a, q, p) == 1 and pow(a, 2, p) != 1
    s0 = O.generate(O.MWC, SEED, 1, 4, flags=O.MWC_SAME_A)
    sq = O.generate(O.MWC, SEED, 1, 4, flags=O.MWC_SAME_A, skip=q, jump=True)
    assert np.array_equal(s0, sq)
    sh = O.generate(O.MWC, SEED, 1, 4, flags=O.MWC_SAME_A, skip=q // 3, jump=True)
    assert not np.array_equal(s0, sh)


# ------------------------------------------------------------------- XORWOW
def test_xorwow_skip_ahead_matches_stepping():
    for t in [1, 2, 160, 3001]:
        a = O.generate(O.XORWOW, SEED, 32, 7, skip=t, jump=True)
        b = O.generate(O.XORWOW, SEED, 32, 7, skip=t, jump=False)
        assert np.array_equal(a, b), t


def test_xorwow_xorshift_order_divides_2_160_minus_1():
    # Sec. 6: period 2^192 - 2^32 = (2^160 - 1) 2^32; the xorshift part has
    # order dividing 2^160 - 1, i.e. T^(2^160) = T.
    assert np.array_equal(O.matrix_pow2k("xorwow", 160), O.xorwow_matrix())
    assert not np.array_equal(O.matrix_pow2k("xorwow", 80), O.xorwow_matrix())


# --------------------------------------------------------- paper's generator
def test_xs1024_charpoly_degree_1024_weight_475(golden):
    rng = np.random.default_rng(1)
    x = rng.integers(0, 2**32, 32, dtype=np.uint32)
    bits = []
    for _ in range(2200):
        x = O.xs1024_shift_step(x)
        bits.append(int(x[17] >> 5) & 1)
    C, L = _bm_gf2(bits)
    assert L == golden["xs1024"]["charpoly_degree"]
    assert bin(C).count("1") == golden["xs1024"]["charpoly_weight"]


def test_xs1024_matches_three_shift_equation_on_1024_bit_integers(golden):
    # Eq. (threeshift) with x (I + L^a) = x ^ (x << a) on a w = 1024 bit word;
    # Listing 1: lane 0 holds the most significant 32 bits.
    g = golden["xs1024"]
    mask = 2**1024 - 1
    rng = np.random.default_rng(11)
    for _ in range(20):
        w = rng.integers(0, 2**32, 32, dtype=np.uint32)
        X = 0
        for i in range(32):
            X |= int(w[i]) << (32 * (31 - i))
        X ^= (X << g["a"]) & mask
        X ^= X >> g["b"]
        X ^= (X << g["c"]) & mask
        expect = [(X >> (32 * (31 - i))) & 0xFFFFFFFF for i in range(32)]
        assert [int(v) for v in O.xs1024_shift_step(w)] == expect


def test_xs1024_listing_word_shifts(golden):
    g = golden["xs1024"]
    assert g["a"] == 32 * g["wordshift"] + g["rand_a"]
    assert g["b"] == 32 * g["wordshift"] + g["rand_b"]
    assert g["c"] == 32 * g["wordshift"] + g["rand_c"]


def test_xs1024w_weyl_output(golden):
    # Sec. 6: output = y_n (I + R^16) + x_n mod 2^32, y_n = n c (y_0 = 0)
    c, gam = golden["weyl"]["c"], golden["weyl"]["gamma"]
    out = O.generate(O.XS1024W, SEED, 32, 5)
    x = np.array([O.seed_word(SEED, l) & 0xFFFFFFFF for l in range(32)], dtype=np.uint32)
    for n in range(1, 6):
        x = O.xs1024_shift_step(x)
        y = (n * c) % 2**32
        assert np.array_equal(out[:, n - 1], (x.astype(np.uint64) + (y ^ (y >> gam))) % 2**32)


@pytest.mark.parametrize("flags", [O.SEED_RANDOM, O.SEED_SUBSTREAM])
def test_xs1024w_skip_ahead_matches_stepping(flags):
    for t in [1, 31, 1000]:
        a = O.generate(O.XS1024W, SEED, 64, 5, flags=flags, skip=t, jump=True)
        b = O.generate(O.XS1024W, SEED, 64, 5, flags=flags, skip=t, jump=False)
        assert np.array_equal(a, b), t


def test_xs1024w_substream_warps_are_2_137_apart():
    # warp 1 = warp 0 advanced by 2^137 steps: 2^137 = (2^68)(2^69), applied
    # as 2^69 squarings of the 2^68-step matrix would be the same product;
    # here the block matrix is checked to be the 137-fold square of the
    # one-step matrix by applying it to warp 0's state and comparing with
    # warp 1's seeded state.
    P = O.matrix_pow2k("xs1024", 137)
    n = 64
    w0 = O.generate(O.XS1024W, SEED, n, 1, flags=O.SEED_SUBSTREAM, i_lo=0, i_hi=32)
    w1 = O.generate(O.XS1024W, SEED, n, 1, flags=O.SEED_SUBSTREAM, i_lo=32, i_hi=64)
    base = []
    for m in range(16):
        w = O.seed_word(SEED, m)
        base += [w >> 32, w & 0xFFFFFFFF]
    bvec = 0
    for i, v in enumerate(base):
        bvec |= v << (32 * i)
    out = 0
    for i in range(1024):
        if (bvec >> i) & 1:
            row = 0
            for k in range(16):
                row |= int(P[i, k]) << (64 * k)
            out ^= row
    x1 = np.array([(out >> (32 * i)) & 0xFFFFFFFF for i in range(32)], dtype=np.uint32)
    x1 = O.xs1024_shift_step(x1)
    y = 362437
    assert np.array_equal(w1[:, 0], (x1.astype(np.uint64) + (y ^ (y >> 16))) % 2**32)
    assert not np.array_equal(w0, w1)


@pytest.mark.slow
def test_xs1024_order_divides_2_1024_minus_1():
    assert np.array_equal(O.matrix_pow2k("xs1024", 1024), O.xs_matrix())


# ------------------------------------------------------------------- Philox
_PHILOX_SRC = r"""
#include <ATen/core/PhiloxRNGEngine.h>
#include <cstdio>
#include <cstdlib>
int main(int argc, char** argv) {
  unsigned long long key, off; int rounds;
  while (std::scanf("%llu %llu %d", &key, &off, &rounds) == 3) {
    at::philox_engine e(key, 0, off);
    for (int i = 0; i < 4; i++) std::printf("%u ", e(rounds));
    std::printf("\n");
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def torch_philox(tmp_path_factory):
    torch = pytest.importorskip("torch")
    if shutil.which("g++") is None:
        pytest.skip("no g++")
    inc = os.path.join(os.path.dirname(torch.__file__), "include")
    if not os.path.exists(os.path.join(inc, "ATen", "core", "PhiloxRNGEngine.h")):
        pytest.skip("torch headers without PhiloxRNGEngine.h")
    d = tmp_path_factory.mktemp("philox")
    src = d / "p.cpp"
    src.write_text(_PHILOX_SRC)
    exe = d / "p"
    subprocess.check_call(["g++", "-std=c++17", "-O1", f"-I{inc}", str(src), "-o", str(exe)])
    return str(exe)


@pytest.mark.parametrize("rounds", [7, 10])
def test_philox_against_torch_engine(torch_philox, rounds):
    # An independent open-source Philox4x32 (torch's PhiloxRNGEngine.h):
    # key = seed, counter = (offset, subsequence) -> words 0..3 of a block.
    rng = np.random.default_rng(5)
    cases = [(0, 0), (M64, M64 >> 1)] + [(int(k), int(o)) for k, o in
                                        zip(rng.integers(0, 2**63, 40, dtype=np.uint64),
                                            rng.integers(0, 2**40, 40, dtype=np.uint64))]
    inp = "".join(f"{k} {o} {rounds}\n" for k, o in cases)
    res = subprocess.run([torch_philox], input=inp, capture_output=True, text=True, check=True)
    lines = res.stdout.strip().split("\n")
    for (k, o), line in zip(cases, lines):
        ref = [int(v) for v in line.split()]
        got = O.philox4x32([o & 0xFFFFFFFF, o >> 32, 0, 0], k & 0xFFFFFFFF, k >> 32, rounds)
        assert [int(v) for v in got] == ref


def test_philox_stream_is_counter_blocks():
    s = O.generate(O.PHILOX4X32_10, SEED, 4, 12, i_lo=2, i_hi=3)[0]
    w = O.seed_word(SEED, 2)
    for j in range(3):
        blk = O.philox4x32([j, 0, 0, 0], w & 0xFFFFFFFF, w >> 32, 10)
        assert np.array_equal(s[4 * j:4 * j + 4], blk)
    a = O.generate(O.PHILOX4X32_10, SEED, 16, 9, skip=123457, jump=True)
    b = O.generate(O.PHILOX4X32_10, SEED, 16, 9, skip=123457, jump=False)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("kind,rounds", [(O.PHILOX4X32_7, 7), (O.PHILOX4X32_10, 10)])
@pytest.mark.parametrize("flags", [0, O.PHILOX_INTRINSIC_KEY])
def test_philox_streams_against_torch_engine(torch_philox, kind, rounds, flags):
    # Whole streams, key mapping and counter layout included, against the
    # independent engine: draw d of instance i is word d % 4 of the block at
    # counter d / 4, under key w_i or, with intrinsic keys (Sec. 7), under
    # key (i, low half of the seed)
    seed, n, K = 0xDEADBEEF00C0FFEE, 1 << 20, 11
    idx = [0, 1, 77, n - 1]
    got = np.concatenate([O.generate(kind, seed, n, K, flags=flags, i_lo=i, i_hi=i + 1, skip=5) for i in idx])
    lines = []
    for i in idx:
        key = ((seed & 0xFFFFFFFF) << 32 | i) if flags else O.seed_word(seed, i)
        lines += [f"{key} {j} {rounds}\n" for j in range(1, 5)]  # draws 5..15 lie in blocks 1..3
    res = subprocess.run([torch_philox], input="".join(lines), capture_output=True, text=True, check=True)
    words = np.array([[int(v) for v in ln.split()] for ln in res.stdout.strip().split("\n")], dtype=np.uint64)
    words = words.reshape(len(idx), -1)
    assert np.array_equal(got, words[:, 1:1 + K].astype(np.uint32))


def test_philox_intrinsic_keys_do_not_depend_on_the_instance_count():
    # a stream is named by its own index and the run word only: any shard or
    # launch split of the instances reproduces it
    a = O.generate(O.PHILOX4X32_7, SEED, 64, 20, flags=O.PHILOX_INTRINSIC_KEY, i_lo=10, i_hi=14)
    b = O.generate(O.PHILOX4X32_7, SEED, 1 << 30, 20, flags=O.PHILOX_INTRINSIC_KEY, i_lo=10, i_hi=14)
    assert np.array_equal(a, b)
    # the run word is the low half of the seed
    c = O.generate(O.PHILOX4X32_7, SEED ^ (1 << 40), 64, 20, flags=O.PHILOX_INTRINSIC_KEY, i_lo=10, i_hi=14)
    assert np.array_equal(a, c)
    d = O.generate(O.PHILOX4X32_7, SEED, 64, 20, i_lo=10, i_hi=14)
    assert not np.array_equal(a, d)
    with pytest.raises(O.OracleError):
        O.generate(O.XORWOW, SEED, 64, 4, flags=O.PHILOX_INTRINSIC_KEY)
    with pytest.raises(O.OracleError):  # instance indices past 2^32 do not fit the key word
        O.generate(O.PHILOX4X32_7, SEED, (1 << 32) + 1, 4, flags=O.PHILOX_INTRINSIC_KEY, i_lo=0, i_hi=1)


# ---------------------------------------------------- lagged Fibonacci (Sec. 4)
def _gf2_mulmod(a, b, P, deg):
    r = 0
    while b:
        if b & 1:
            r ^= a
        b >>= 1
        a <<= 1
        if (a >> deg) & 1:
            a ^= P
    return r


@pytest.mark.parametrize("lags", [(521, 353), (1279, 861)])
def test_lfib_trinomials_are_primitive(golden, lags):
    # x^r + x^s + 1 over GF(2): with r prime, Rabin's test reduces to
    # x^(2^r) = x (mod P) and P having no root in GF(2); as 2^r - 1 is then
    # a (Mersenne) prime, irreducible means primitive, so the low bits have
    # period 2^r - 1 and the words 2^31 (2^r - 1) (Brent's bound, Sec. 4)
    assert list(lags) in golden["lfib"]["lags"]
    r, s = lags
    P = (1 << r) | (1 << s) | 1
    x = 2
    for _ in range(r):
        x = _gf2_mulmod(x, x, P, r)
    assert x == 2
    assert P & 1 and bin(P).count("1") % 2 == 1  # P(0) = P(1) = 1


@pytest.mark.parametrize("kind", [O.LFIB521, O.LFIB1279])
def test_lfib_low_bits_follow_the_papers_lags(kind):
    # Berlekamp-Massey on the low bit of the oracle's words must return the
    # trinomial 1 + x^s + x^r of the lags printed in Sec. 4: a wrong lag, a
    # wrong ring index or a subtraction for the addition all fail here
    r, s = O.LFIB_LAGS[kind]
    out = O.generate(kind, SEED, 3, 3 * r, i_lo=2, i_hi=3)[0]
    C, L = _bm_gf2([int(v) & 1 for v in out])
    assert L == r
    assert C == (1 | (1 << s) | (1 << r))


def _period(seq, r):
    """Least P > 0 with the r-word state after P outputs equal to the start."""
    start = seq[:r]
    for P in range(1, len(seq) - r):
        if seq[P] == start[0] and np.array_equal(seq[P:P + r], start):
            return P
    return None


@pytest.mark.parametrize("r,s", [(5, 2), (5, 3), (7, 3), (7, 1)])
@pytest.mark.parametrize("bits", [1, 3, 6])
def test_lfib_small_lag_periods(r, s, bits):
    # additive lagged Fibonacci mod 2^m on a primitive trinomial: period
    # 2^(m-1) (2^r - 1) when a seed is odd (Sec. 4, after Brent); the ring
    # arithmetic of the oracle is the one the production lags use
    rng = np.random.default_rng(r * 100 + s * 10 + bits)
    seeds = rng.integers(0, 1 << bits, r, dtype=np.uint32)
    seeds[0] |= 1
    expect = (1 << (bits - 1)) * ((1 << r) - 1)
    seq = O.lfib_raw(r, s, bits, seeds, 2 * expect + r + 1)
    assert _period(seq, r) == expect
    if bits > 1:  # all seeds even: the words never leave the even residues
        ev = O.lfib_raw(r, s, bits, seeds & ~np.uint32(1), 2 * expect + r + 1)
        assert np.all(ev & 1 == 0)
        assert _period(ev, r) <= expect // 2


@pytest.mark.parametrize("kind", [O.LFIB521, O.LFIB1279])
def test_lfib_streams_start_from_their_seed_words(kind):
    r, s = O.LFIB_LAGS[kind]
    i = 5
    seeds = np.array([O.seed_word(SEED, r * i + j) & 0xFFFFFFFF for j in range(r)], dtype=np.uint32)
    if not np.any(seeds & 1):
        seeds[0] |= 1
    got = O.generate(kind, SEED, 8, 2000, i_lo=i, i_hi=i + 1)[0]
    assert np.array_equal(got, O.lfib_raw(r, s, 32, seeds, 2000))
    # the first outputs are the recurrence on the seeds themselves
    assert got[0] == (int(seeds[0]) + int(seeds[r - s])) & 0xFFFFFFFF
    with pytest.raises(O.OracleError):
        O.generate(kind, SEED, 8, 4, skip=10, jump=True)  # no skip-ahead for the ring generators


# ----------------------------------------------------------------------- MT
def test_mt19937_cxx_standard_value():
    # The C++ standard ([rand.predef]) fixes the 10000th output of
    # mt19937 seeded with its default seed 5489 at 4123659995.
    assert int(O.mt19937_raw(5489, 10000)[-1]) == 4123659995


def test_mt19937_against_numpy():
    for s in [0, 1, 5489, 0xDEADBEEF]:
        bg = np.random.MT19937()
        bg._legacy_seeding(s)
        assert np.array_equal(bg.random_raw(2000).astype(np.uint32), O.mt19937_raw(s, 2000))


def test_mt_generator_streams_use_seed_words():
    s = O.generate(O.MT19937_SHARED, SEED, 3, 700, i_lo=1, i_hi=2)[0]
    assert np.array_equal(s, O.mt19937_raw(O.seed_word(SEED, 1) & 0xFFFFFFFF, 700))


# -------------------------------------------------------------- conversions
def test_f32_conversion_exact_in_single_precision():
    r = np.array([0, 1, 255, 256, 0x7FFFFFFF, 0xFFFFFF00, 0xFFFFFFFF], dtype=np.uint32)
    r = np.concatenate([r, np.random.default_rng(0).integers(0, 2**32, 10000, dtype=np.uint32)])
    u = O.to_f32(r)
    f = (r >> 8).astype(np.float32) * np.float32(2.0**-24)
    assert np.array_equal(u, f.astype(np.float64))
    assert u.min() >= 0.0 and u.max() < 1.0


def test_box_muller_moments_and_endpoints():
    r = O.generate(O.PHILOX4X32_10, SEED, 4096, 4096).ravel()
    z = O.box_muller(r)
    n = z.size
    assert abs(z.mean()) < 5 / np.sqrt(n)
    assert abs(z.var() - 1) < 5 * np.sqrt(2 / n)
    kurt = (z**4).mean() / z.var() ** 2
    assert abs(kurt - 3) < 5 * np.sqrt(24 / n)
    # u1 = 1 (r0 >> 8 = 2^24 - 1) gives z = 0; u1 = 2^-24 the largest radius
    e = O.box_muller(np.array([0xFFFFFFFF, 12345, 0, 0], dtype=np.uint32))
    assert e[0] == 0.0 and e[1] == 0.0
    assert abs(e[2] - np.sqrt(2 * 24 * np.log(2))) < 1e-12 and e[3] == 0.0
