/*
 * oracle.c -- plain, slow, serial CPU oracle for the per-thread random
 * number streams and the checkerboard Ising update of Manssen, Weigel and
 * Hartmann, "Random number generators for massively parallel simulations on
 * GPU" (arXiv:1204.6193).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library includes, links
 * or calls this file; only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark load it (through oracle/__init__.py).  It shares no
 * header, helper, table or constant generator with the CUDA path: every
 * constant below is retyped from the paper or from the published definition
 * it names.
 *
 * Conventions (the paper is silent on seeding; these readings are the
 * library's contract and are recorded with the design notes):
 *   - master seed -> words w_k = mix64(seed + (k+1)*0x9E3779B97F4A7C15),
 *     mix64 being SplitMix64's finaliser (Steele, Lea, Flood 2014);
 *   - a "stream" s_i[0], s_i[1], ... is the sequence of uint32 outputs of
 *     instance i; the canonical result of a generation call is s_i[k].
 *
 * Everything is written for clarity, not speed: generators are stepped one
 * draw at a time, matrices over GF(2) are multiplied row by row, and the
 * Ising update visits sites in plain loops.
 *
 * Parity unpinned: the conventions the paper leaves open have no value in
 * the paper to check them against, and the tests can only confirm that they
 * are applied consistently -- the seed-word mapping of every kind (including
 * the lagged Fibonacci rings and the intrinsic Philox key (i, low half of
 * the seed)), the XS1024W Weyl reading (y_0 = 0, one value for all lanes),
 * the initial spins, the Ising draw order (stream s owns sites sG..sG+G-1
 * of both colours) and the multi-hit strip and phase order.  Everything
 * built on them (recurrences, skip-ahead, the Metropolis step, the exact
 * Ising values) is pinned by the tests.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

enum { K_LCG32 = 0, K_LCG64 = 1, K_MWC = 2, K_XORWOW = 3, K_PHILOX = 4, K_XS1024W = 5, K_MT = 6, K_PHILOX7 = 7,
       K_LFIB521 = 8, K_LFIB1279 = 9 };
enum { F_LEAPFROG = 1, F_SUBSTREAM = 2, F_MWC_SAME_A = 4, F_PHILOX_INTRINSIC = 8 };
enum { ORC_OK = 0, ORC_EINVAL = 1, ORC_ENOMEM = 2, ORC_EUNSUPPORTED = 3 };

/* ------------------------------------------------------------------------ */
/* Seed expansion: SplitMix64 (Steele, Lea, Flood 2014), counter form.       */
/* ------------------------------------------------------------------------ */
static uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

uint64_t orc_mix64(uint64_t z) { return mix64(z); }

/* w_k: the k-th SplitMix64 output for the master seed. */
uint64_t orc_seed_word(uint64_t seed, uint64_t k)
{
    return mix64(seed + (k + 1) * 0x9E3779B97F4A7C15ULL);
}

/* ------------------------------------------------------------------------ */
/* Linear congruential generators, Sec. 2, Eq. (1).                          */
/* 32-bit: a = 1664525, c = 1013904223; 64-bit: a = 2862933555777941757,     */
/* c = 1442695040888963407 (both printed in Sec. 2).  The output of a step   */
/* is the new state; the 64-bit generator outputs its 32 most significant   */
/* bits (Sec. 2, performance discussion).                                    */
/* ------------------------------------------------------------------------ */
#define LCG32_A 1664525u
#define LCG32_C 1013904223u
#define LCG64_A 2862933555777941757ULL
#define LCG64_C 1442695040888963407ULL

/* Skip-ahead, Sec. 2, Eq. (2): x_{n+t} = a_t x_n + c_t with a_t = a^t and
 * c_t the sum of a^i c for i = 0..t-1 (the paper prints the sum from 1 to t;
 * the form that satisfies Eq. (2) for t = 1 is the sum from 0 to t-1).
 * Computed by composing the affine map x -> a x + c with itself, by binary
 * powering, modulo 2^64 (the 32-bit modulus is its low half). */
static void lcg_jump_coeffs(uint64_t a, uint64_t c, uint64_t t, uint64_t *at, uint64_t *ct)
{
    uint64_t A = 1, C = 0;        /* accumulated map: identity */
    uint64_t pa = a, pc = c;      /* map for 2^bit steps */
    while (t) {
        if (t & 1) {              /* apply accumulated, then the 2^bit map */
            C = pa * C + pc;
            A = pa * A;
        }
        pc = pa * pc + pc;        /* square the 2^bit map */
        pa = pa * pa;
        t >>= 1;
    }
    *at = A;
    *ct = C;
}

void orc_lcg_jump_coeffs(int is64, uint64_t t, uint64_t *at, uint64_t *ct)
{
    if (is64) lcg_jump_coeffs(LCG64_A, LCG64_C, t, at, ct);
    else {
        lcg_jump_coeffs(LCG32_A, LCG32_C, t, at, ct);
        *at &= 0xffffffffULL;
        *ct &= 0xffffffffULL;
    }
}

/* ------------------------------------------------------------------------ */
/* Multiply-with-carry, Sec. 3.  State v = c*2^32 + x.  One step:            */
/*   x' = (a x + c) mod 2^32,  c' = floor((a x + c) / 2^32),                 */
/* i.e. v' = a*(v mod 2^32) + floor(v / 2^32); the output is x'.             */
/* Multipliers: a < 2^32 with a*2^32 - 1 and (a*2^32 - 2)/2 both prime,      */
/* taken in descending order from the largest (Sec. 3: 4294967118).         */
/* ------------------------------------------------------------------------ */
static uint64_t mulmod64(uint64_t a, uint64_t b, uint64_t m)
{
    return (uint64_t)(((u128)a * b) % m);
}

static uint64_t powmod64(uint64_t b, uint64_t e, uint64_t m)
{
    uint64_t r = 1 % m;
    b %= m;
    while (e) {
        if (e & 1) r = mulmod64(r, b, m);
        b = mulmod64(b, b, m);
        e >>= 1;
    }
    return r;
}

/* Miller-Rabin with the first twelve primes as bases: deterministic for
 * every n below 3.3e24, hence for every 64-bit n. */
static int is_prime_u64(uint64_t n)
{
    static const uint64_t bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return 0;
    for (int i = 0; i < 12; i++) {
        if (n == bases[i]) return 1;
        if (n % bases[i] == 0) return 0;
    }
    uint64_t d = n - 1;
    int s = 0;
    while ((d & 1) == 0) { d >>= 1; s++; }
    for (int i = 0; i < 12; i++) {
        uint64_t x = powmod64(bases[i], d, n);
        if (x == 1 || x == n - 1) continue;
        int witness = 1;
        for (int r = 1; r < s; r++) {
            x = mulmod64(x, x, n);
            if (x == n - 1) { witness = 0; break; }
        }
        if (witness) return 0;
    }
    return 1;
}

int orc_is_prime_u64(uint64_t n) { return is_prime_u64(n); }

static uint32_t *g_mwc_table = NULL;
static uint64_t g_mwc_count = 0;       /* entries found so far */
static uint64_t g_mwc_next_a = 0xffffffffULL; /* next candidate to test */

/* Extends the descending multiplier table to at least `count` entries.  The
 * candidates are first sieved by the odd primes below 2^16 (a candidate whose
 * p = a*2^32-1 or q = a*2^31-1 has such a factor is composite, since both
 * exceed 2^16), then both p and q go through Miller-Rabin. */
static int mwc_extend(uint64_t count)
{
    if (count <= g_mwc_count) return ORC_OK;
    /* the table is a cache of a fixed list: grow it geometrically so that
     * callers asking for one more entry at a time do not rescan */
    if (count < 2 * g_mwc_count) count = 2 * g_mwc_count;
    if (count < 4096) count = 4096;
    uint32_t *t = (uint32_t *)realloc(g_mwc_table, count * sizeof(uint32_t));
    if (!t) return ORC_ENOMEM;
    g_mwc_table = t;

    enum { SIEVE_LIMIT = 65536, SEG = 1 << 20 };
    static uint32_t primes[8192];
    static uint32_t inv_p[8192], inv_q[8192];  /* a with p or q = 0 mod prime */
    static int nprimes = 0;
    if (nprimes == 0) {
        char *comp = (char *)calloc(SIEVE_LIMIT, 1);
        if (!comp) return ORC_ENOMEM;
        for (uint32_t i = 3; i < SIEVE_LIMIT; i += 2) {
            if (comp[i]) continue;
            primes[nprimes] = i;
            /* p = a 2^32 - 1 = 0 mod l  <=>  a = (2^32)^(-1) mod l, likewise q */
            uint64_t two32 = powmod64(2, 32, i), two31 = powmod64(2, 31, i);
            inv_p[nprimes] = (uint32_t)powmod64(two32, i - 2, i);
            inv_q[nprimes] = (uint32_t)powmod64(two31, i - 2, i);
            nprimes++;
            for (uint32_t j = i * 3; j < SIEVE_LIMIT; j += 2 * i) comp[j] = 1;
        }
        free(comp);
    }
    char *mark = (char *)malloc(SEG);
    if (!mark) return ORC_ENOMEM;
    while (g_mwc_count < count && g_mwc_next_a >= 2) {
        uint64_t hi = g_mwc_next_a;
        uint64_t lo = hi >= SEG - 1 + 2 ? hi - (SEG - 1) : 2;
        uint64_t len = hi - lo + 1;
        memset(mark, 0, len);
        for (int k = 0; k < nprimes; k++) {
            uint64_t l = primes[k];
            uint64_t r0 = inv_p[k], r1 = inv_q[k];
            /* first a >= lo with a = r (mod l) */
            uint64_t s0 = lo + ((r0 + l - lo % l) % l);
            uint64_t s1 = lo + ((r1 + l - lo % l) % l);
            for (uint64_t a = s0; a <= hi; a += l) mark[a - lo] = 1;
            for (uint64_t a = s1; a <= hi; a += l) mark[a - lo] = 1;
        }
        for (uint64_t a = hi;; a--) {
            if (!mark[a - lo]) {
                uint64_t p = (a << 32) - 1, q = (a << 31) - 1;
                if (is_prime_u64(q) && is_prime_u64(p)) {
                    g_mwc_table[g_mwc_count++] = (uint32_t)a;
                    if (g_mwc_count == count) { g_mwc_next_a = a - 1; break; }
                }
            }
            if (a == lo) { g_mwc_next_a = lo - 1; break; }
        }
    }
    free(mark);
    return g_mwc_count >= count ? ORC_OK : ORC_EINVAL;
}

/* Copies the first `count` multipliers (descending) into out. */
int orc_mwc_multipliers(uint64_t count, uint32_t *out)
{
    int st = mwc_extend(count);
    if (st != ORC_OK) return st;
    memcpy(out, g_mwc_table, count * sizeof(uint32_t));
    return ORC_OK;
}

static uint32_t mwc_step(uint64_t *v, uint32_t a)
{
    *v = (uint64_t)a * (*v & 0xffffffffULL) + (*v >> 32);
    return (uint32_t)*v;
}

/* Skip-ahead for MWC.  With b = 2^32 and p = a b - 1, a step maps v to
 * v' = a x + c, and b v' = a b x + b c = x + b c = v (mod p); hence
 * v' = v b^(-1) = v a (mod p), and t steps multiply v by a^t mod p. */
static uint64_t mwc_jump(uint64_t v, uint32_t a, uint64_t t)
{
    uint64_t p = ((uint64_t)a << 32) - 1;
    return mulmod64(v % p, powmod64(a, t, p), p);
}

/* ------------------------------------------------------------------------ */
/* XORWOW (Marsaglia 2003, "Xorshift RNGs", the xorwow listing): a five-word */
/* xorshift with a Weyl sequence d += 362437, output d + v (Sec. 6).         */
/* ------------------------------------------------------------------------ */
typedef struct { uint32_t x, y, z, w, v, d; } xorwow_t;

static void xorwow_shift(xorwow_t *s)
{
    uint32_t t = s->x ^ (s->x >> 2);
    s->x = s->y;
    s->y = s->z;
    s->z = s->w;
    s->w = s->v;
    s->v = (s->v ^ (s->v << 4)) ^ (t ^ (t << 1));
}

static uint32_t xorwow_next(xorwow_t *s)
{
    xorwow_shift(s);
    s->d += 362437u;
    return s->d + s->v;
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-r (Salmon, Moraes, Dror, Shaw 2011), Sec. 7: two S-boxes per   */
/* round, L' = mullo(R, M), R' = mulhi(R, M) ^ k ^ L, followed by the        */
/* published 4-word permutation; the key is bumped by the Weyl constants     */
/* between rounds.                                                           */
/* ------------------------------------------------------------------------ */
void orc_philox4x32(const uint32_t ctr_in[4], uint32_t k0, uint32_t k1, int rounds, uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    for (int r = 0; r < rounds; r++) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ------------------------------------------------------------------------ */
/* The paper's generator, Sec. 6: a three-shift xorshift on w = 1024 bits,   */
/*   X_n = X_{n-1} (I + L^329)(I + R^347)(I + L^344),                        */
/* held as 32 words, one per lane of a warp, lane 0 the most significant     */
/* word (the bits reaching lane i on a left shift by 329 come from lanes     */
/* i+10 and i+11).  Shifts are logical: bits shifted past either end are    */
/* dropped and zeros enter (the zero padding of the shared array).  The      */
/* output of lane i at step n is (y_n ^ (y_n >> 16)) + X_n[i] mod 2^32 with  */
/* the Weyl sequence y_n = n*362437 mod 2^32, the same for every lane and    */
/* warp (y_0 = 0).                                                           */
/* ------------------------------------------------------------------------ */
#define XS_WORDS 32

/* out = X << s as a 1024-bit integer (lane 0 most significant). */
static void shl1024(const uint32_t *x, int s, uint32_t *out)
{
    int q = s / 32, r = s % 32;
    for (int i = 0; i < XS_WORDS; i++) {
        uint32_t a = (i + q < XS_WORDS) ? x[i + q] : 0;         /* same significance - q */
        uint32_t b = (i + q + 1 < XS_WORDS) ? x[i + q + 1] : 0; /* next lower word */
        out[i] = r ? (a << r) | (b >> (32 - r)) : a;
    }
}

/* out = X >> s as a 1024-bit integer. */
static void shr1024(const uint32_t *x, int s, uint32_t *out)
{
    int q = s / 32, r = s % 32;
    for (int i = 0; i < XS_WORDS; i++) {
        uint32_t a = (i - q >= 0) ? x[i - q] : 0;         /* same significance + q */
        uint32_t b = (i - q - 1 >= 0) ? x[i - q - 1] : 0; /* next higher word */
        out[i] = r ? (a >> r) | (b << (32 - r)) : a;
    }
}

static void xs_shift_step(uint32_t *x)
{
    uint32_t t[XS_WORDS];
    shl1024(x, 329, t);
    for (int i = 0; i < XS_WORDS; i++) x[i] ^= t[i];
    shr1024(x, 347, t);
    for (int i = 0; i < XS_WORDS; i++) x[i] ^= t[i];
    shl1024(x, 344, t);
    for (int i = 0; i < XS_WORDS; i++) x[i] ^= t[i];
}

/* One step of one warp: x updated in place; n is the step count after the
 * step; out receives the 32 lane outputs. */
static void xs_step(uint32_t *x, uint64_t n, uint32_t *out)
{
    xs_shift_step(x);
    uint32_t y = (uint32_t)(n * 362437u);
    uint32_t yy = y ^ (y >> 16);
    for (int i = 0; i < XS_WORDS; i++) out[i] = yy + x[i];
}

/* Exposed for tests: one raw xorshift step of a 1024-bit state. */
void orc_xs1024_shift_step(uint32_t *x) { xs_shift_step(x); }

/* ------------------------------------------------------------------------ */
/* MT19937 (Matsumoto and Nishimura 1998), Sec. 5: N = 624, M = 397,         */
/* r = 31, twist constant 0x9908B0DF, standard tempering and the standard    */
/* 32-bit seeding recurrence with multiplier 1812433253.                     */
/* ------------------------------------------------------------------------ */
typedef struct { uint32_t mt[624]; int mti; } mt_t;

static void mt_seed(mt_t *g, uint32_t s)
{
    g->mt[0] = s;
    for (int i = 1; i < 624; i++)
        g->mt[i] = 1812433253u * (g->mt[i - 1] ^ (g->mt[i - 1] >> 30)) + (uint32_t)i;
    g->mti = 624;
}

static uint32_t mt_next(mt_t *g)
{
    if (g->mti >= 624) {
        for (int i = 0; i < 624; i++) {
            uint32_t y = (g->mt[i] & 0x80000000u) | (g->mt[(i + 1) % 624] & 0x7fffffffu);
            g->mt[i] = g->mt[(i + 397) % 624] ^ (y >> 1) ^ ((y & 1u) ? 0x9908B0DFu : 0u);
        }
        g->mti = 0;
    }
    uint32_t y = g->mt[g->mti++];
    y ^= y >> 11;
    y ^= (y << 7) & 0x9D2C5680u;
    y ^= (y << 15) & 0xEFC60000u;
    y ^= y >> 18;
    return y;
}

/* ------------------------------------------------------------------------ */
/* Additive lagged Fibonacci generators, Sec. 4, Eq. (used_fibonacci):       */
/* u_n = u_(n-r) + u_(n-s) (mod 1) with (r, s) = (521, 353) or (1279, 861).  */
/* Written on the 32-bit words x_n = 2^32 u_n, where the same recurrence is  */
/* x_n = x_(n-r) + x_(n-s) mod 2^32 (m = 2^32, the modulus the section      */
/* fixes).  The ring `hist` holds the last r values: x_m sits in slot m mod  */
/* r.  The generic width `bits` (1..32) serves the small-lag period checks.  */
/* ------------------------------------------------------------------------ */
typedef struct { uint32_t r, s, mask; uint64_t n; uint32_t *hist; } lfib_t;

/* hist[j] = x_(j-r) for j < r: the r seed values, oldest first */
static int lfib_init(lfib_t *g, uint32_t r, uint32_t s, int bits, const uint32_t *seeds)
{
    g->r = r;
    g->s = s;
    g->mask = bits >= 32 ? 0xffffffffu : ((1u << bits) - 1u);
    g->n = 0;
    g->hist = (uint32_t *)malloc(r * sizeof(uint32_t));
    if (!g->hist) return ORC_ENOMEM;
    for (uint32_t j = 0; j < r; j++) g->hist[j] = seeds[j] & g->mask;
    return ORC_OK;
}

static uint32_t lfib_next(lfib_t *g)
{
    uint32_t old_r = g->hist[g->n % g->r];                   /* x_(n-r) */
    uint32_t old_s = g->hist[(g->n + g->r - g->s) % g->r];   /* x_(n-s) */
    uint32_t x = (old_r + old_s) & g->mask;
    g->hist[g->n % g->r] = x;
    g->n++;
    return x;
}

/* Seeds of generator i ("seed the ring buffers ... with an independent RNG",
 * Sec. 4): x_(j-r) = low half of w_(r i + j); if all r are even, the low bit
 * of the first is set (an all-even start never reaches an odd value and
 * misses the full period 2^31 (2^r - 1)). */
static void lfib_seeds(uint64_t seed, uint32_t r, uint64_t i, uint32_t *out)
{
    uint32_t odd = 0;
    for (uint32_t j = 0; j < r; j++) {
        out[j] = (uint32_t)orc_seed_word(seed, (uint64_t)r * i + j);
        odd |= out[j] & 1u;
    }
    if (!odd) out[0] |= 1u;
}

/* Generic small-width form for the tests: K outputs of the (r, s) generator
 * on `bits`-bit words from the given r seed values. */
int orc_lfib_raw(uint32_t r, uint32_t s, int bits, const uint32_t *seeds, uint64_t K, uint32_t *out)
{
    if (r < 2 || s < 1 || s >= r || bits < 1 || bits > 32) return ORC_EINVAL;
    lfib_t g;
    if (lfib_init(&g, r, s, bits, seeds)) return ORC_ENOMEM;
    for (uint64_t k = 0; k < K; k++) out[k] = lfib_next(&g);
    free(g.hist);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Bit matrices over GF(2) (Sec. 6, Eq. threeshift): states are row vectors  */
/* and x' = x M, so row i of M is the image of the unit vector e_i.          */
/* ------------------------------------------------------------------------ */
typedef struct { int n, nw; uint64_t *r; } bm_t;

static int bm_alloc(bm_t *m, int n)
{
    m->n = n;
    m->nw = (n + 63) / 64;
    m->r = (uint64_t *)calloc((size_t)n * m->nw, sizeof(uint64_t));
    return m->r ? ORC_OK : ORC_ENOMEM;
}

static void bm_free(bm_t *m) { free(m->r); m->r = NULL; }

/* y = x M */
static void bm_vecmul(const bm_t *m, const uint64_t *x, uint64_t *y)
{
    uint64_t t[16];
    memset(t, 0, sizeof(t));
    for (int i = 0; i < m->n; i++)
        if ((x[i / 64] >> (i % 64)) & 1)
            for (int w = 0; w < m->nw; w++) t[w] ^= m->r[(size_t)i * m->nw + w];
    memcpy(y, t, m->nw * sizeof(uint64_t));
}

/* C = A B (C may alias neither) */
static void bm_mul(const bm_t *a, const bm_t *b, bm_t *c)
{
    for (int i = 0; i < a->n; i++) bm_vecmul(b, a->r + (size_t)i * a->nw, c->r + (size_t)i * c->nw);
}

static void bm_copy(bm_t *dst, const bm_t *src)
{
    memcpy(dst->r, src->r, (size_t)src->n * src->nw * sizeof(uint64_t));
}

static void bm_identity(bm_t *m)
{
    memset(m->r, 0, (size_t)m->n * m->nw * sizeof(uint64_t));
    for (int i = 0; i < m->n; i++) m->r[(size_t)i * m->nw + i / 64] |= 1ULL << (i % 64);
}

/* r = m^(2^k) by k squarings */
static int bm_pow2k(const bm_t *m, int k, bm_t *r)
{
    bm_t t;
    if (bm_alloc(&t, m->n)) return ORC_ENOMEM;
    bm_copy(r, m);
    for (int i = 0; i < k; i++) {
        bm_mul(r, r, &t);
        bm_copy(r, &t);
    }
    bm_free(&t);
    return ORC_OK;
}

/* r = m^e by binary powering */
static int bm_pow(const bm_t *m, uint64_t e, bm_t *r)
{
    bm_t sq, t;
    if (bm_alloc(&sq, m->n)) return ORC_ENOMEM;
    if (bm_alloc(&t, m->n)) { bm_free(&sq); return ORC_ENOMEM; }
    bm_identity(r);
    bm_copy(&sq, m);
    while (e) {
        if (e & 1) { bm_mul(r, &sq, &t); bm_copy(r, &t); }
        e >>= 1;
        if (e) { bm_mul(&sq, &sq, &t); bm_copy(&sq, &t); }
    }
    bm_free(&sq);
    bm_free(&t);
    return ORC_OK;
}

/* State <-> bit vector: bit j = bit (j % 32) of word (j / 32). */
static void words_to_bits(const uint32_t *w, int nwords, uint64_t *b)
{
    memset(b, 0, ((nwords * 32 + 63) / 64) * sizeof(uint64_t));
    for (int i = 0; i < nwords; i++) b[i / 2] |= (uint64_t)w[i] << (32 * (i % 2));
}

static void bits_to_words(const uint64_t *b, int nwords, uint32_t *w)
{
    for (int i = 0; i < nwords; i++) w[i] = (uint32_t)(b[i / 2] >> (32 * (i % 2)));
}

/* One-step matrix of the 1024-bit xorshift, built from the step itself. */
static int xs_matrix(bm_t *m)
{
    if (bm_alloc(m, 1024)) return ORC_ENOMEM;
    for (int i = 0; i < 1024; i++) {
        uint32_t x[XS_WORDS];
        memset(x, 0, sizeof(x));
        x[i / 32] = 1u << (i % 32);
        xs_shift_step(x);
        words_to_bits(x, XS_WORDS, m->r + (size_t)i * m->nw);
    }
    return ORC_OK;
}

/* One-step matrix of the 160-bit xorshift part of XORWOW (x, y, z, w, v). */
static int xorwow_matrix(bm_t *m)
{
    if (bm_alloc(m, 160)) return ORC_ENOMEM;
    for (int i = 0; i < 160; i++) {
        uint32_t w5[5] = {0, 0, 0, 0, 0};
        w5[i / 32] = 1u << (i % 32);
        xorwow_t s = {w5[0], w5[1], w5[2], w5[3], w5[4], 0};
        xorwow_shift(&s);
        uint32_t o[5] = {s.x, s.y, s.z, s.w, s.v};
        words_to_bits(o, 5, m->r + (size_t)i * m->nw);
    }
    return ORC_OK;
}

/* Exposed for tests: the dense one-step matrices (row-major u64 words). */
int orc_xs_matrix(uint64_t *out /* 1024*16 */)
{
    bm_t m;
    if (xs_matrix(&m)) return ORC_ENOMEM;
    memcpy(out, m.r, 1024 * 16 * sizeof(uint64_t));
    bm_free(&m);
    return ORC_OK;
}

int orc_xorwow_matrix(uint64_t *out /* 160*3 */)
{
    bm_t m;
    if (xorwow_matrix(&m)) return ORC_ENOMEM;
    memcpy(out, m.r, 160 * 3 * sizeof(uint64_t));
    bm_free(&m);
    return ORC_OK;
}

/* out = m^(2^k) for the chosen one-step matrix (0: 1024-bit, 1: XORWOW). */
int orc_matrix_pow2k(int which, int k, uint64_t *out)
{
    bm_t m, r;
    int st = which ? xorwow_matrix(&m) : xs_matrix(&m);
    if (st) return st;
    if (bm_alloc(&r, m.n)) { bm_free(&m); return ORC_ENOMEM; }
    st = bm_pow2k(&m, k, &r);
    if (!st) memcpy(out, r.r, (size_t)r.n * r.nw * sizeof(uint64_t));
    bm_free(&m);
    bm_free(&r);
    return st;
}

/* Substream jump matrix P = M^(2^137) (Sec. 6: blocks of 2^137 numbers). */
static bm_t g_xs_P = {0, 0, NULL};

static int xs_substream_matrix(void)
{
    if (g_xs_P.r) return ORC_OK;
    bm_t m;
    if (xs_matrix(&m)) return ORC_ENOMEM;
    if (bm_alloc(&g_xs_P, 1024)) { bm_free(&m); return ORC_ENOMEM; }
    int st = bm_pow2k(&m, 137, &g_xs_P);
    bm_free(&m);
    return st;
}

/* ------------------------------------------------------------------------ */
/* Instances: seeding (the mapping from master seed words) and one draw.     */
/* ------------------------------------------------------------------------ */
typedef struct {
    int kind;
    uint32_t flags;
    /* LCG32/LCG64 */
    uint64_t x, A, C;     /* state and per-draw map (a, c), or (a_n, c_n) */
    /* MWC */
    uint64_t v;
    uint32_t a;
    /* XORWOW */
    xorwow_t xw;
    /* Philox */
    uint32_t k0, k1;
    uint64_t pos;         /* draws consumed */
    /* MT */
    mt_t *mt;
    /* lagged Fibonacci */
    lfib_t lf;
} inst_t;

/* Seeds per-thread instance i of n (not XS1024W, whose unit is a warp). */
static int inst_init(inst_t *s, int kind, uint32_t flags, uint64_t seed, uint64_t n, uint64_t i)
{
    memset(s, 0, sizeof(*s));
    s->kind = kind;
    s->flags = flags;
    switch (kind) {
    case K_LCG32:
    case K_LCG64: {
        int is64 = kind == K_LCG64;
        uint64_t a = is64 ? LCG64_A : LCG32_A, c = is64 ? LCG64_C : LCG32_C;
        uint64_t mask = is64 ? ~0ULL : 0xffffffffULL;
        if (flags & F_LEAPFROG) {
            /* Sec. 2: all instances share one serial sequence x_0, x_1, ...
             * seeded by w_0; instance i starts at x_(i+1-n) (mod the
             * period) and steps with (a_n, c_n), so that draw k of instance
             * i is x_(k n + i + 1). */
            uint64_t x0 = orc_seed_word(seed, 0) & mask;
            uint64_t at, ct;
            lcg_jump_coeffs(a, c, i + 1 - n, &at, &ct);  /* wraps mod 2^64 */
            s->x = (at * x0 + ct) & mask;
            lcg_jump_coeffs(a, c, n, &s->A, &s->C);
            s->A &= mask;
            s->C &= mask;
        } else {
            s->x = orc_seed_word(seed, i) & mask;
            s->A = a;
            s->C = c;
        }
        return ORC_OK;
    }
    case K_MWC: {
        uint32_t a;
        if (flags & F_MWC_SAME_A) {
            if (mwc_extend(1)) return ORC_ENOMEM;
            a = g_mwc_table[0];
        } else {
            int st = mwc_extend(i + 1);
            if (st) return st;
            a = g_mwc_table[i];
        }
        uint64_t w = orc_seed_word(seed, i);
        uint64_t x = w & 0xffffffffULL, c = (w >> 32) % a;
        /* (0, 0) and (2^32-1, a-1) are fixed points of the step */
        if ((x == 0 && c == 0) || (x == 0xffffffffULL && c == a - 1)) x = 1;
        s->v = (c << 32) | x;
        s->a = a;
        return ORC_OK;
    }
    case K_XORWOW: {
        uint64_t w0 = orc_seed_word(seed, 3 * i), w1 = orc_seed_word(seed, 3 * i + 1),
                 w2 = orc_seed_word(seed, 3 * i + 2);
        s->xw.x = (uint32_t)w0;
        s->xw.y = (uint32_t)(w0 >> 32);
        s->xw.z = (uint32_t)w1;
        s->xw.w = (uint32_t)(w1 >> 32);
        s->xw.v = (uint32_t)w2;
        s->xw.d = (uint32_t)(w2 >> 32);
        if (!(s->xw.x | s->xw.y | s->xw.z | s->xw.w | s->xw.v)) s->xw.x = 1;
        return ORC_OK;
    }
    case K_PHILOX:
    case K_PHILOX7: {
        if (flags & F_PHILOX_INTRINSIC) {
            /* Sec. 7, intrinsic variables: the key is the instance (site)
             * number and a word naming the run, here the low half of the
             * seed; the counter (the block index) is the draw position */
            s->k0 = (uint32_t)i;
            s->k1 = (uint32_t)seed;
        } else {
            uint64_t w = orc_seed_word(seed, i);
            s->k0 = (uint32_t)w;
            s->k1 = (uint32_t)(w >> 32);
        }
        s->pos = 0;
        return ORC_OK;
    }
    case K_MT: {
        s->mt = (mt_t *)malloc(sizeof(mt_t));
        if (!s->mt) return ORC_ENOMEM;
        mt_seed(s->mt, (uint32_t)orc_seed_word(seed, i));
        return ORC_OK;
    }
    case K_LFIB521:
    case K_LFIB1279: {
        uint32_t r = kind == K_LFIB521 ? 521 : 1279, sl = kind == K_LFIB521 ? 353 : 861;
        uint32_t *seeds = (uint32_t *)malloc(r * sizeof(uint32_t));
        if (!seeds) return ORC_ENOMEM;
        lfib_seeds(seed, r, i, seeds);
        int st = lfib_init(&s->lf, r, sl, 32, seeds);
        free(seeds);
        return st;
    }
    }
    return ORC_EINVAL;
}

static void inst_free(inst_t *s)
{
    free(s->mt);
    s->mt = NULL;
    free(s->lf.hist);
    s->lf.hist = NULL;
}

static uint32_t inst_next(inst_t *s, int philox_rounds)
{
    switch (s->kind) {
    case K_LCG32:
        s->x = (s->A * s->x + s->C) & 0xffffffffULL;
        return (uint32_t)s->x;
    case K_LCG64:
        s->x = s->A * s->x + s->C;
        return (uint32_t)(s->x >> 32);
    case K_MWC:
        return mwc_step(&s->v, s->a);
    case K_XORWOW:
        return xorwow_next(&s->xw);
    case K_PHILOX:
    case K_PHILOX7: {
        /* draw d is word d % 4 of block d / 4; counter = (block, 0);
         * Philox4x32-7 (Sec. 7) always takes 7 rounds */
        uint64_t j = s->pos / 4;
        uint32_t ctr[4] = {(uint32_t)j, (uint32_t)(j >> 32), 0, 0}, o[4];
        orc_philox4x32(ctr, s->k0, s->k1, s->kind == K_PHILOX7 ? 7 : philox_rounds, o);
        return o[s->pos++ % 4];
    }
    case K_MT:
        return mt_next(s->mt);
    case K_LFIB521:
    case K_LFIB1279:
        return lfib_next(&s->lf);
    }
    return 0;
}

/* Advances an instance by t draws with the generator's skip-ahead (Sec. 2
 * Eq. (2) for LCGs, the modular power for MWC, the GF(2) matrix power for
 * XORWOW, a counter add for Philox). */
static int inst_jump(inst_t *s, uint64_t t)
{
    switch (s->kind) {
    case K_LCG32:
    case K_LCG64: {
        uint64_t mask = s->kind == K_LCG64 ? ~0ULL : 0xffffffffULL;
        uint64_t at, ct;
        lcg_jump_coeffs(s->A, s->C, t, &at, &ct);
        s->x = (at * s->x + ct) & mask;
        return ORC_OK;
    }
    case K_MWC:
        s->v = mwc_jump(s->v, s->a, t);
        return ORC_OK;
    case K_XORWOW: {
        bm_t m, mt;
        if (xorwow_matrix(&m)) return ORC_ENOMEM;
        if (bm_alloc(&mt, 160)) { bm_free(&m); return ORC_ENOMEM; }
        bm_pow(&m, t, &mt);
        uint32_t w5[5] = {s->xw.x, s->xw.y, s->xw.z, s->xw.w, s->xw.v};
        uint64_t b[3];
        words_to_bits(w5, 5, b);
        bm_vecmul(&mt, b, b);
        bits_to_words(b, 5, w5);
        s->xw.x = w5[0]; s->xw.y = w5[1]; s->xw.z = w5[2]; s->xw.w = w5[3]; s->xw.v = w5[4];
        s->xw.d += (uint32_t)(t * 362437u);
        bm_free(&m);
        bm_free(&mt);
        return ORC_OK;
    }
    case K_PHILOX:
    case K_PHILOX7:
        s->pos += t;
        return ORC_OK;
    }
    return ORC_EUNSUPPORTED;
}

/* Warp j of the 1024-bit generator: x = its 32 words. */
static int xs_warp_init(uint32_t flags, uint64_t seed, uint64_t j, uint32_t *x)
{
    if (flags & F_SUBSTREAM) {
        /* Sec. 6: all warps start from one base state; warp j skips j blocks
         * of 2^137 steps, i.e. x_j = base P^j with P = M^(2^137). */
        for (int m = 0; m < 16; m++) {
            uint64_t w = orc_seed_word(seed, m);
            x[2 * m] = (uint32_t)(w >> 32);
            x[2 * m + 1] = (uint32_t)w;
        }
        int nz = 0;
        for (int i = 0; i < XS_WORDS; i++) nz |= x[i] != 0;
        if (!nz) x[XS_WORDS - 1] = 1;
        if (j == 0) return ORC_OK;
        if (xs_substream_matrix()) return ORC_ENOMEM;
        uint64_t b[16];
        words_to_bits(x, XS_WORDS, b);
        for (uint64_t k = 0; k < j; k++) bm_vecmul(&g_xs_P, b, b);
        bits_to_words(b, XS_WORDS, x);
    } else {
        /* seeding "with another RNG" (Sec. 6): lane l <- low half of w_(32j+l) */
        int nz = 0;
        for (int l = 0; l < XS_WORDS; l++) {
            x[l] = (uint32_t)orc_seed_word(seed, 32 * j + l);
            nz |= x[l] != 0;
        }
        if (!nz) x[XS_WORDS - 1] = 1;
    }
    return ORC_OK;
}

static int xs_warp_jump(uint32_t *x, uint64_t t)
{
    bm_t m, mt;
    if (xs_matrix(&m)) return ORC_ENOMEM;
    if (bm_alloc(&mt, 1024)) { bm_free(&m); return ORC_ENOMEM; }
    bm_pow(&m, t, &mt);
    uint64_t b[16];
    words_to_bits(x, XS_WORDS, b);
    bm_vecmul(&mt, b, b);
    bits_to_words(b, XS_WORDS, x);
    bm_free(&m);
    bm_free(&mt);
    return ORC_OK;
}

static int check_kind_flags(int kind, uint32_t flags, uint64_t n)
{
    if (kind < 0 || kind > K_LFIB1279 || n == 0) return ORC_EINVAL;
    if ((flags & F_PHILOX_INTRINSIC) && kind != K_PHILOX && kind != K_PHILOX7) return ORC_EUNSUPPORTED;
    if ((flags & F_PHILOX_INTRINSIC) && n > (1ULL << 32)) return ORC_EINVAL;  /* a 32-bit key word */
    if ((flags & F_LEAPFROG) && kind != K_LCG32 && kind != K_LCG64) return ORC_EUNSUPPORTED;
    if ((flags & F_SUBSTREAM) && kind != K_XS1024W) return ORC_EUNSUPPORTED;
    if ((flags & F_MWC_SAME_A) && kind != K_MWC) return ORC_EUNSUPPORTED;
    if (kind == K_XS1024W && n % 32) return ORC_EINVAL;
    return ORC_OK;
}

/*
 * Streams of instances [i_lo, i_hi) of an n-instance generator seeded with
 * `seed`, starting after `skip` draws, K draws each:
 *   out[(i - i_lo) * K + k] = s_i[skip + k].
 * jump = 0 reaches the start by stepping, jump = 1 by the skip-ahead method.
 * philox_rounds selects Philox4x32-r (10 by default in the library).
 */
int orc_generate(int kind, uint32_t flags, uint64_t seed, uint64_t n, uint64_t skip, int jump,
                 uint64_t i_lo, uint64_t i_hi, uint64_t K, int philox_rounds, uint32_t *out)
{
    int st = check_kind_flags(kind, flags, n);
    if (st) return st;
    if (i_lo > i_hi || i_hi > n) return ORC_EINVAL;
    if ((kind == K_MT || kind == K_LFIB521 || kind == K_LFIB1279) && jump && skip) return ORC_EUNSUPPORTED;
    if (kind == K_XS1024W) {
        for (uint64_t j = i_lo / 32; j * 32 < i_hi; j++) {
            uint32_t x[XS_WORDS], o[XS_WORDS];
            if ((st = xs_warp_init(flags, seed, j, x))) return st;
            uint64_t steps = 0;
            if (jump) {
                if (skip && (st = xs_warp_jump(x, skip))) return st;
                steps = skip;
            } else {
                for (; steps < skip; steps++) xs_shift_step(x);
            }
            for (uint64_t k = 0; k < K; k++) {
                xs_step(x, steps + k + 1, o);
                for (int l = 0; l < XS_WORDS; l++) {
                    uint64_t i = 32 * j + l;
                    if (i >= i_lo && i < i_hi) out[(i - i_lo) * K + k] = o[l];
                }
            }
        }
        return ORC_OK;
    }
    for (uint64_t i = i_lo; i < i_hi; i++) {
        inst_t s;
        if ((st = inst_init(&s, kind, flags, seed, n, i))) return st;
        if (jump) {
            if (skip && (st = inst_jump(&s, skip))) { inst_free(&s); return st; }
        } else {
            for (uint64_t t = 0; t < skip; t++) inst_next(&s, philox_rounds);
        }
        for (uint64_t k = 0; k < K; k++) out[(i - i_lo) * K + k] = inst_next(&s, philox_rounds);
        inst_free(&s);
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Output conversions (Sec. 2: u = x/m).  f32: the 24 high bits scaled by    */
/* 2^-24, exact in single precision.  Normal deviates: Box-Muller on         */
/* consecutive pairs (r0, r1) of one stream with u1 = (hi24(r0) + 1) 2^-24   */
/* in (0, 1] and u2 = hi24(r1) 2^-24; computed here in double.               */
/* ------------------------------------------------------------------------ */
void orc_to_f32(const uint32_t *r, uint64_t count, double *u)
{
    for (uint64_t i = 0; i < count; i++) u[i] = (double)(r[i] >> 8) * 0x1p-24;
}

void orc_box_muller(const uint32_t *r, uint64_t pairs, double *z)
{
    const double two_pi = 6.283185307179586476925286766559;
    for (uint64_t i = 0; i < pairs; i++) {
        double u1 = ((double)(r[2 * i] >> 8) + 1.0) * 0x1p-24;
        double u2 = (double)(r[2 * i + 1] >> 8) * 0x1p-24;
        double rad = sqrt(-2.0 * log(u1));
        z[2 * i] = rad * cos(two_pi * u2);
        z[2 * i + 1] = rad * sin(two_pi * u2);
    }
}

/* ------------------------------------------------------------------------ */
/* 2D Ising ferromagnet, J = 1, zero field, periodic L x L (Sec. 2,          */
/* application test): checkerboard Metropolis.                               */
/*   colour of (x, y) = (x + y) & 1;                                         */
/*   colour-compressed index of a colour-c site: q = y (L/2) + (x >> 1);     */
/*   stream s owns q in [s G, (s+1) G) of both colours;                      */
/*   a sweep is colour 0 then colour 1; in a half-sweep every stream draws   */
/*   one number per owned site, in increasing q, whatever the energy change; */
/*   the flip is accepted iff dE <= 0 or r < T[dE],                          */
/*   T[dE] = floor(2^32 exp(-beta dE)) for dE = 4, 8.                        */
/* Spins are int8 +-1, row-major (index y L + x).                            */
/* ------------------------------------------------------------------------ */
uint64_t orc_ising_threshold(double beta, int dE)
{
    return (uint64_t)floor(4294967296.0 * exp(-beta * (double)dE));
}

/* Initial spins: spin j = +1 iff bit (j mod 64) of w_(j/64) is set, the
 * words drawn from the master seed XOR 0x5350494E. */
void orc_ising_init_spins(uint32_t L, uint64_t seed, int8_t *s)
{
    uint64_t seed2 = seed ^ 0x5350494EULL;
    for (uint64_t j = 0; j < (uint64_t)L * L; j++)
        s[j] = ((orc_seed_word(seed2, j / 64) >> (j % 64)) & 1) ? 1 : -1;
}

void orc_ising_energy(uint32_t L, const int8_t *s, int64_t *E, int64_t *M)
{
    int64_t e = 0, m = 0;
    for (uint32_t y = 0; y < L; y++)
        for (uint32_t x = 0; x < L; x++) {
            int si = s[y * L + x];
            e -= si * s[y * L + (x + 1) % L];       /* bond to the right */
            e -= si * s[((y + 1) % L) * L + x];     /* bond below */
            m += si;
        }
    *E = e;
    *M = m;
}

static void ising_site(uint32_t L, int8_t *s, uint64_t q, int colour, uint32_t r, const uint64_t T[9])
{
    uint32_t half = L / 2;
    uint32_t y = (uint32_t)(q / half);
    uint32_t x = 2 * (uint32_t)(q % half) + ((colour + y) & 1);
    int nn = s[y * L + (x + L - 1) % L] + s[y * L + (x + 1) % L] + s[((y + L - 1) % L) * L + x] +
             s[((y + 1) % L) * L + x];
    int dE = 2 * s[y * L + x] * nn;
    if (dE <= 0 || (uint64_t)r < T[dE]) s[y * L + x] = (int8_t)-s[y * L + x];
}

/*
 * One half-sweep of colour c over the sites owned by streams [s0, s1):
 * stream sidx's site number g (q = sidx G + g) takes draws[(sidx - s0) G +
 * g], the g-th number that stream drew for this half-sweep.  Sites of one
 * colour have no bond between them, so the order of the visits does not
 * matter.
 */
static void ising_half_sweep(uint32_t L, int8_t *s, int c, uint32_t G, uint64_t s0, uint64_t s1,
                             const uint32_t *draws, const uint64_t T[9])
{
    for (uint64_t sidx = s0; sidx < s1; sidx++)
        for (uint32_t g = 0; g < G; g++) ising_site(L, s, sidx * G + g, c, draws[(sidx - s0) * G + g], T);
}

/*
 * Where a half-sweep's numbers come from: fill(ctx, G, s0, s1, draws) puts
 * the next G numbers of every stream sidx in [s0, s1) at draws[(sidx - s0) G
 * + g], g = 0 .. G-1, in the order the stream produces them.
 */
typedef void (*ising_fill_fn)(void *ctx, uint32_t G, uint64_t s0, uint64_t s1, uint32_t *draws);

/* The streams of an Ising run: per-thread instances, or one state per warp
 * of 32 streams -- the 1024-bit generator (Sec. 6), and the block-shared
 * generators MT19937 (Sec. 5) and lagged Fibonacci (Sec. 4), of which
 * generator j is seeded as generator j of a generation call with
 * ceil(streams / 32) generators.  In a warp-shared draw round the 32
 * streams 32j .. 32j+31 each take one word: stream 32j + l takes word l of
 * the round, so its d-th number is word 32d + l of generator j's stream.
 * Lanes beyond the last stream draw but are unused. */
static int warp_shared(int kind) { return kind == K_XS1024W || kind == K_MT || kind == K_LFIB521 || kind == K_LFIB1279; }

typedef struct {
    int kind;
    int philox_rounds;
    uint64_t nstreams;
    inst_t *inst;
    uint32_t *xs;
    uint64_t *xs_steps;   /* the Weyl step count of each warp state */
} ising_streams_t;

static void ising_fill_streams(void *ctx, uint32_t G, uint64_t s0, uint64_t s1, uint32_t *draws)
{
    ising_streams_t *st = (ising_streams_t *)ctx;
    if (warp_shared(st->kind)) {
        /* every lane of warp j draws once per round of the warp's generator */
        for (uint32_t g = 0; g < G; g++)
            for (uint64_t j = s0 / 32; j < (s1 + 31) / 32; j++) {
                uint32_t o[32];
                if (st->kind == K_XS1024W) {
                    st->xs_steps[j]++;
                    xs_step(st->xs + j * XS_WORDS, st->xs_steps[j], o);
                } else {
                    for (int l = 0; l < 32; l++) o[l] = inst_next(&st->inst[j], st->philox_rounds);
                }
                for (int l = 0; l < 32; l++) {
                    uint64_t sidx = 32 * j + l;
                    if (sidx >= s0 && sidx < s1) draws[(sidx - s0) * G + g] = o[l];
                }
            }
        return;
    }
    for (uint64_t sidx = s0; sidx < s1; sidx++)
        for (uint32_t g = 0; g < G; g++) draws[(sidx - s0) * G + g] = inst_next(&st->inst[sidx], st->philox_rounds);
}

static void ising_streams_free(ising_streams_t *st)
{
    uint64_t n_inst = warp_shared(st->kind) ? (st->nstreams + 31) / 32 : st->nstreams;
    if (st->inst)
        for (uint64_t i = 0; i < n_inst; i++) inst_free(&st->inst[i]);
    free(st->inst);
    free(st->xs);
    free(st->xs_steps);
    st->inst = NULL;
    st->xs = NULL;
    st->xs_steps = NULL;
}

/* Seeds the streams of an L x L lattice at G sites per stream. */
static int ising_streams_init(ising_streams_t *st, uint32_t L, int kind, uint32_t flags, uint64_t seed, uint32_t G,
                              int philox_rounds)
{
    memset(st, 0, sizeof(*st));
    st->kind = kind;
    st->philox_rounds = philox_rounds;
    st->nstreams = (uint64_t)L * L / 2 / G;
    uint64_t n = kind == K_XS1024W ? (st->nstreams + 31) / 32 * 32
               : warp_shared(kind) ? (st->nstreams + 31) / 32 : st->nstreams;  /* instances */
    int rc = check_kind_flags(kind, flags, n);
    if (rc) return rc;
    if (kind == K_XS1024W) {
        uint64_t nwarps = n / 32;
        st->xs = (uint32_t *)malloc(nwarps * XS_WORDS * sizeof(uint32_t));
        st->xs_steps = (uint64_t *)calloc(nwarps, sizeof(uint64_t));
        if (!st->xs || !st->xs_steps) { ising_streams_free(st); return ORC_ENOMEM; }
        for (uint64_t j = 0; j < nwarps; j++)
            if ((rc = xs_warp_init(flags, seed, j, st->xs + j * XS_WORDS))) { ising_streams_free(st); return rc; }
        return ORC_OK;
    }
    st->inst = (inst_t *)calloc(n, sizeof(inst_t));
    if (!st->inst) return ORC_ENOMEM;
    for (uint64_t i = 0; i < n; i++)
        if ((rc = inst_init(&st->inst[i], kind, flags, seed, n, i))) { ising_streams_free(st); return rc; }
    return ORC_OK;
}

/* One sweep: colour 0, then colour 1; every stream draws G numbers per
 * half-sweep.  draws: scratch of nstreams G words. */
static void ising_sweep(uint32_t L, int8_t *s, uint32_t G, uint64_t nstreams, ising_fill_fn fill, void *ctx,
                        uint32_t *draws, const uint64_t T[9])
{
    for (int c = 0; c < 2; c++) {
        fill(ctx, G, 0, nstreams, draws);
        ising_half_sweep(L, s, c, G, 0, nstreams, draws, T);
    }
}

static void ising_measure(uint32_t L, const int8_t *s, int64_t acc[4], uint64_t *n_meas)
{
    int64_t E, M;
    orc_ising_energy(L, s, &E, &M);
    acc[0] += E;
    acc[1] += E * E;
    acc[2] += M * M;
    acc[3] += M < 0 ? -M : M;
    (*n_meas)++;
}

static void ising_thresholds(double beta, uint64_t T[9])
{
    memset(T, 0, 9 * sizeof(uint64_t));
    T[4] = orc_ising_threshold(beta, 4);
    T[8] = orc_ising_threshold(beta, 8);
}

/*
 * n_sweeps sweeps from the spins in s (updated in place) with freshly seeded
 * streams (n = L^2 / (2G) instances, rounded up to a multiple of 32 for the
 * 1024-bit generator, whose lanes beyond the last stream draw but are
 * unused).  If measure_every > 0, after every measure_every-th sweep E and M
 * are measured and acc[0..3] += E, E^2, M^2, |M|.
 */
int orc_ising_run(uint32_t L, double beta, int kind, uint32_t flags, uint64_t seed, uint32_t G,
                  uint64_t n_sweeps, uint32_t measure_every, int philox_rounds, int8_t *s,
                  int64_t acc[4], uint64_t *n_meas)
{
    if (L < 2 || L % 2 || G == 0 || ((uint64_t)L * L / 2) % G) return ORC_EINVAL;
    ising_streams_t st;
    int rc = ising_streams_init(&st, L, kind, flags, seed, G, philox_rounds);
    if (rc) return rc;
    uint32_t *draws = (uint32_t *)malloc(st.nstreams * G * sizeof(uint32_t));
    if (!draws) { ising_streams_free(&st); return ORC_ENOMEM; }
    uint64_t T[9];
    ising_thresholds(beta, T);
    for (uint64_t t = 1; t <= n_sweeps; t++) {
        ising_sweep(L, s, G, st.nstreams, ising_fill_streams, &st, draws, T);
        if (measure_every && t % measure_every == 0) ising_measure(L, s, acc, n_meas);
    }
    free(draws);
    ising_streams_free(&st);
    return ORC_OK;
}

/*
 * Multi-hit updates with a double checkerboard (Sec. 2: "k hits" per tile
 * load, with k = 1 and k = 100 in Table 1).  The lattice is cut into
 * n_strips strips of L / n_strips rows (n_strips even); strip b has coarse
 * colour b & 1.  A round is: for coarse colour C = 0, 1 in turn, k sweeps
 * (colour 0 then colour 1 sites) over the rows of every strip of coarse
 * colour C, while the strips of the other coarse colour -- the only
 * neighbours of those rows outside the strip -- stay fixed.  In each
 * half-sweep every stream of an updated strip draws one number per owned
 * site, in increasing q, as in orc_ising_run.  Every step is a single-site
 * Metropolis update, so the Boltzmann distribution is left invariant.
 * Measurements (if measure_every > 0) follow every measure_every-th round.
 */
static void ising_multihit_round(uint32_t L, int8_t *s, uint32_t G, uint32_t n_strips, uint32_t k_hits,
                                 uint64_t per_strip, ising_fill_fn fill, void *ctx, uint32_t *draws,
                                 const uint64_t T[9])
{
    for (uint32_t C = 0; C < 2; C++)
        for (uint32_t hit = 0; hit < k_hits; hit++)
            for (int c = 0; c < 2; c++)
                for (uint32_t b = C; b < n_strips; b += 2) {
                    uint64_t s0 = b * per_strip, s1 = s0 + per_strip;
                    fill(ctx, G, s0, s1, draws);
                    ising_half_sweep(L, s, c, G, s0, s1, draws, T);
                }
}

static int multihit_args_ok(uint32_t L, uint32_t G, uint32_t n_strips, uint32_t k_hits)
{
    return L >= 2 && L % 2 == 0 && G != 0 && (L / 2) % G == 0 && n_strips >= 2 && n_strips % 2 == 0 &&
           L % n_strips == 0 && k_hits != 0;
}

int orc_ising_run_multihit(uint32_t L, double beta, int kind, uint32_t flags, uint64_t seed, uint32_t G,
                           uint32_t n_strips, uint32_t k_hits, uint64_t n_rounds, uint32_t measure_every,
                           int philox_rounds, int8_t *s, int64_t acc[4], uint64_t *n_meas)
{
    if (!multihit_args_ok(L, G, n_strips, k_hits)) return ORC_EINVAL;
    uint64_t per_strip = (uint64_t)(L / n_strips) * ((L / 2) / G);  /* streams per strip */
    if (warp_shared(kind) && per_strip % 32) return ORC_EINVAL;     /* a warp's generator within one strip */
    ising_streams_t st;
    int rc = ising_streams_init(&st, L, kind, flags, seed, G, philox_rounds);
    if (rc) return rc;
    uint32_t *draws = (uint32_t *)malloc(per_strip * G * sizeof(uint32_t));
    if (!draws) { ising_streams_free(&st); return ORC_ENOMEM; }
    uint64_t T[9];
    ising_thresholds(beta, T);
    for (uint64_t t = 1; t <= n_rounds; t++) {
        ising_multihit_round(L, s, G, n_strips, k_hits, per_strip, ising_fill_streams, &st, draws, T);
        if (measure_every && t % measure_every == 0) ising_measure(L, s, acc, n_meas);
    }
    free(draws);
    ising_streams_free(&st);
    return ORC_OK;
}

/*
 * The same updates driven by numbers the caller gives, for tests that
 * enumerate the draws (the exact transition matrix of the update): stream
 * sidx's d-th draw of the call is given[sidx * per_stream + d].  Each of
 * n_lattices lattices (spins: n_lattices L x L arrays, updated in place)
 * takes its own block of nstreams * per_stream words.
 */
typedef struct {
    const uint32_t *given;
    uint64_t per_stream;
    uint64_t *used;       /* draws taken so far by each stream */
} ising_given_t;

static void ising_fill_given(void *ctx, uint32_t G, uint64_t s0, uint64_t s1, uint32_t *draws)
{
    ising_given_t *gv = (ising_given_t *)ctx;
    for (uint64_t sidx = s0; sidx < s1; sidx++)
        for (uint32_t g = 0; g < G; g++) {
            uint64_t d = gv->used[sidx]++;
            draws[(sidx - s0) * G + g] = d < gv->per_stream ? gv->given[sidx * gv->per_stream + d] : 0;
        }
}

/* One half-sweep of colour c over the rows [row0, row1) (the streams that
 * own them: G numbers each). */
int orc_ising_half_sweep_given(uint32_t L, double beta, uint32_t G, int colour, uint32_t row0, uint32_t row1,
                               uint64_t n_lattices, const uint32_t *given, int8_t *spins)
{
    if (L < 2 || L % 2 || G == 0 || (L / 2) % G || colour < 0 || colour > 1 || row0 >= row1 || row1 > L)
        return ORC_EINVAL;
    uint64_t spr = (L / 2) / G, nstreams = (uint64_t)L * L / 2 / G;
    uint64_t s0 = row0 * spr, s1 = row1 * spr;
    uint64_t T[9];
    ising_thresholds(beta, T);
    for (uint64_t b = 0; b < n_lattices; b++)
        ising_half_sweep(L, spins + b * L * L, colour, G, s0, s1, given + b * nstreams * G + s0 * G, T);
    return ORC_OK;
}

/* One sweep (both colours, 2G numbers per stream), as in orc_ising_run. */
int orc_ising_sweep_given(uint32_t L, double beta, uint32_t G, uint64_t n_lattices, const uint32_t *given,
                          int8_t *spins)
{
    if (L < 2 || L % 2 || G == 0 || ((uint64_t)L * L / 2) % G) return ORC_EINVAL;
    uint64_t nstreams = (uint64_t)L * L / 2 / G;
    uint32_t *draws = (uint32_t *)malloc(nstreams * G * sizeof(uint32_t));
    uint64_t *used = (uint64_t *)calloc(nstreams, sizeof(uint64_t));
    if (!draws || !used) { free(draws); free(used); return ORC_ENOMEM; }
    uint64_t T[9];
    ising_thresholds(beta, T);
    for (uint64_t b = 0; b < n_lattices; b++) {
        ising_given_t gv = {given + b * nstreams * 2 * G, 2 * (uint64_t)G, used};
        memset(used, 0, nstreams * sizeof(uint64_t));
        ising_sweep(L, spins + b * L * L, G, nstreams, ising_fill_given, &gv, draws, T);
    }
    free(draws);
    free(used);
    return ORC_OK;
}

/* One multi-hit round (2 k G numbers per stream), as in orc_ising_run_multihit. */
int orc_ising_multihit_round_given(uint32_t L, double beta, uint32_t G, uint32_t n_strips, uint32_t k_hits,
                                   uint64_t n_lattices, const uint32_t *given, int8_t *spins)
{
    if (!multihit_args_ok(L, G, n_strips, k_hits)) return ORC_EINVAL;
    uint64_t nstreams = (uint64_t)L * L / 2 / G;
    uint64_t per_strip = (uint64_t)(L / n_strips) * ((L / 2) / G);
    uint64_t per_stream = 2 * (uint64_t)k_hits * G;
    uint32_t *draws = (uint32_t *)malloc(per_strip * G * sizeof(uint32_t));
    uint64_t *used = (uint64_t *)calloc(nstreams, sizeof(uint64_t));
    if (!draws || !used) { free(draws); free(used); return ORC_ENOMEM; }
    uint64_t T[9];
    ising_thresholds(beta, T);
    for (uint64_t b = 0; b < n_lattices; b++) {
        ising_given_t gv = {given + b * nstreams * per_stream, per_stream, used};
        memset(used, 0, nstreams * sizeof(uint64_t));
        ising_multihit_round(L, spins + b * L * L, G, n_strips, k_hits, per_strip, ising_fill_given, &gv, draws, T);
    }
    free(draws);
    free(used);
    return ORC_OK;
}

/* The MT19937 generator alone, for the standard-library comparison:
 * out[k] = k-th output after seeding with the 32-bit seed s. */
void orc_mt19937_raw(uint32_t s, uint64_t K, uint32_t *out)
{
    mt_t g;
    mt_seed(&g, s);
    for (uint64_t k = 0; k < K; k++) out[k] = mt_next(&g);
}
