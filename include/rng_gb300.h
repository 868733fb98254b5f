/*
 * rng_gb300.h -- C ABI of librng_gb300.so: per-thread pseudo-random streams
 * for massively parallel simulations and their consumption by a
 * checkerboard Metropolis update of the 2D Ising ferromagnet, after
 * Manssen, Weigel and Hartmann, "Random number generators for massively
 * parallel simulations on GPU" (arXiv:1204.6193).
 *
 * Problem statement (Sec. 1): many generator instances, one per thread,
 * each producing its own stream, set up so that the streams are independent
 * (by random seeding, by skip-ahead into sub-streams of one sequence, or by
 * distinct keys), then consumed in place by the threads of a simulation.
 *
 * General conventions
 *  - Every function returns a status (RNG_OK = 0 or an RNG_E* code).  No
 *    function exits, throws or prints.  rng_last_error() gives a
 *    thread-local one-line description of the last failure.
 *  - Device pointers (d_*) are CUDA global-memory pointers owned by the
 *    caller; host pointers (host_*) are ordinary host memory owned by the
 *    caller.  Generator state, lattices and scratch buffers are owned by the
 *    library and live on the device that was current at creation.
 *  - cuda_stream is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Generation and sweep calls are asynchronous on that stream;
 *    calls that return host data (observables, get_state, get_spins)
 *    synchronise it.
 *  - Handles are not thread-safe: one host thread at a time per handle.
 *  - A "stream" s_i[0], s_i[1], ... is the uint32 output sequence of
 *    instance i.  A generation call with n_per_instance = K emits draws
 *    s_i[p], ..., s_i[p+K-1] of every instance, p being the number of draws
 *    already consumed, and advances every instance by K.
 */
#ifndef RNG_GB300_H
#define RNG_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rng_s *rng_t;
typedef struct ising_s *ising_t;

/* Status codes. */
enum {
    RNG_OK = 0,
    RNG_EINVAL = 1,       /* bad argument (null pointer, size, combination) */
    RNG_ENOMEM = 2,       /* device or host allocation failed */
    RNG_EUNSUPPORTED = 3, /* operation not defined for this generator */
    RNG_ECUDA = 4,        /* a CUDA call failed (detail in rng_last_error) */
    RNG_ETIMEOUT = 5,     /* a bounded device-side wait gave up */
    RNG_EBUSY = 6         /* no free slot or memory to admit a request */
};

/* Generator kinds (Sec. 2-7). */
enum {
    RNG_LCG32 = 0,          /* Sec. 2, Eq. (1): a = 1664525, c = 1013904223, m = 2^32 */
    RNG_LCG64 = 1,          /* Sec. 2: a = 2862933555777941757, c = 1442695040888963407, m = 2^64; top 32 bits */
    RNG_MWC = 2,            /* Sec. 3: multiply-with-carry, base 2^32, safe-prime multipliers */
    RNG_XORWOW = 3,         /* Sec. 6: Marsaglia's 160-bit xorshift plus Weyl sequence */
    RNG_PHILOX4X32_10 = 4,  /* Sec. 7: counter-based Philox4x32, 10 rounds */
    RNG_XS1024W = 5,        /* Sec. 6, Listing 1: the paper's 1024-bit warp-shared xorshift plus Weyl */
    RNG_MT19937_SHARED = 6, /* Sec. 5: MT19937, one block-shared state per generator */
    RNG_PHILOX4X32_7 = 7,   /* Sec. 7: Philox4x32 with 7 rounds (the fewest the Philox authors found
                               Crush-resistant); streams laid out as RNG_PHILOX4X32_10 */
    RNG_LFIB521 = 8,        /* Sec. 4, Eq. (used_fibonacci): additive lagged Fibonacci, lags (521, 353),
                               one ring shared by a warp; x_n = x_(n-521) + x_(n-353) mod 2^32 */
    RNG_LFIB1279 = 9        /* Sec. 4: the same with lags (1279, 861) */
};

/* Seeding flags (rng_create). */
enum {
    RNG_SEED_RANDOM = 0,    /* each instance seeded from its own SplitMix64 words */
    RNG_SEED_LEAPFROG = 1,  /* LCGs only, Sec. 2 Eq. (2): instances interleave one serial sequence */
    RNG_SEED_SUBSTREAM = 2, /* XS1024W only, Sec. 6: warp j starts 2^137 j steps into one sequence */
    RNG_MWC_SAME_A = 4,     /* MWC only, Sec. 3: one shared multiplier instead of one per instance */
    RNG_PHILOX_INTRINSIC_KEY = 8 /* Philox kinds only, Sec. 7: intrinsic-variable keys -- instance i
                                    (an Ising stream: its site-pair number) has key (k0, k1) =
                                    (i, low 32 bits of the seed), the run word; counter = draw
                                    block index, which for two sites per stream is the sweep
                                    number.  Needs n_total <= 2^32. */
};

/* Output layouts (rng_generate_*). */
enum {
    RNG_STEP_MAJOR = 0,     /* d_out[k * n + i] = draw k of instance i ("warp order", Sec. 6) */
    RNG_INSTANCE_MAJOR = 1, /* d_out[i * K + k] ("single-thread order", Sec. 6) */
    RNG_XOR_REDUCE = 2      /* consume in registers: d_out[i] = XOR of the K output words
                               (u32 and f32 bit patterns); for normals the float sum */
};

/* Ising lattice layouts. */
enum {
    ISING_INT8 = 0,         /* one int8 (+1 or -1) per site */
    ISING_MULTISPIN32 = 1   /* 32 same-colour sites per uint32, bit set = spin -1; L % 64 == 0 */
};

/* ---------------------------------------------------------------- streams */

/* Creates n_instances generator instances of `kind` on the current device
 * (Sec. 1: one instance per thread; for RNG_XS1024W an instance is one lane
 * of a warp-shared 1024-bit state, Sec. 6, so n_instances must be a multiple
 * of 32; for RNG_MT19937_SHARED an instance is one MT19937 generator whose
 * 624-word state a thread block shares, Sec. 5; for RNG_LFIB521/1279 one
 * lagged Fibonacci generator whose r-word ring a warp shares, Sec. 4).  `flags` is an OR of the
 * RNG_SEED_* / RNG_MWC_SAME_A / RNG_PHILOX_INTRINSIC_KEY values valid for
 * the kind, else RNG_EUNSUPPORTED.  The instances are unseeded until rng_seed.
 * RNG_MWC without RNG_MWC_SAME_A needs n_instances distinct multipliers
 * (more than 10^6 exist below 2^32, Sec. 3); beyond the table, RNG_EINVAL. */
int rng_create(rng_t *out, int kind, uint64_t n_instances, uint32_t flags, void *cuda_stream);

/* Like rng_create, but the handle holds instances [first, first + count) of
 * an n_total-instance generator: seeding, leapfrog and sub-stream positions
 * use the global instance index, so shards on several devices together give
 * exactly the streams of one n_total handle.  XS1024W: first and count
 * multiples of 32. */
int rng_create_shard(rng_t *out, int kind, uint64_t n_total, uint64_t first, uint64_t count,
                     uint32_t flags, void *cuda_stream);

int rng_destroy(rng_t h);

/* Seeds every instance from one 64-bit master seed, expanded by SplitMix64
 * into words w_k = mix64(seed + (k+1) 0x9E3779B97F4A7C15) (the paper seeds
 * instances "with an independent RNG", Sec. 4 and 6).  Per kind: LCG32 x_0 =
 * low32(w_i); LCG64 x_0 = w_i; LEAPFROG: instance i starts at x_(i+1-n) of
 * the serial sequence from w_0 and steps by (a_n, c_n), Eq. (2); MWC x =
 * low32(w_i), c = high32(w_i) mod a_i; XORWOW (x,y),(z,w),(v,d) from
 * w_3i..w_3i+2; Philox key = w_i, counter = block index; XS1024W lane l of
 * warp j = low32(w_(32j+l)), or with SUBSTREAM base words from w_0..w_15 and
 * warp j advanced by j 2^137 steps; MT generator g seeded with low32(w_g);
 * lagged Fibonacci generator g (lags r, s) starts from x_(j-r) =
 * low32(w_(r g + j)), j < r, with the low bit of x_(-r) set if all r words
 * are even.  Resets the draw position to 0. */
int rng_seed(rng_t h, uint64_t seed);

/* Advances every instance by n draws without producing them (Sec. 2 Eq. (2)
 * for LCGs; v <- v a^n mod (a 2^32 - 1) for MWC; the n-th power of the
 * GF(2) transition matrix for XORWOW and XS1024W, Sec. 6; a counter add for
 * Philox, Sec. 7).  Block-shared kinds (RNG_MT19937_SHARED, RNG_LFIB521,
 * RNG_LFIB1279): RNG_EUNSUPPORTED.  Allocates and
 * frees device scratch on the handle's stream for the matrix kinds. */
int rng_skipahead(rng_t h, uint64_t n);

/* Same advance as rng_skipahead for RNG_XORWOW and RNG_XS1024W, on a state
 * array the caller owns, with no device allocation of any kind: for callers
 * that cannot allocate device memory (code inside a framework that owns
 * every device allocation, or that must not let an allocation synchronise
 * the device mid-sequence).  The paper has no counterpart.
 *  d_state: device array in the library's state layout, advanced in place:
 *    RNG_XORWOW   6 consecutive arrays of n_instances words (x, y, z, w, v, d);
 *    RNG_XS1024W  n_instances words, 32 consecutive words per warp state
 *                 (n_instances a multiple of 32); the Weyl step count is the
 *                 caller's and is not touched.
 *  Scratch: one file-scope device array of 384 KiB (three 1024 x 1024-bit
 *  matrices), held by every GPU that loads the library until the process
 *  exits.  States wider than 1024 bits (RNG_MT19937_SHARED, RNG_LFIB*) are rejected
 *  with RNG_EINVAL; kinds that skip without matrices (LCGs, MWC, Philox)
 *  with RNG_EUNSUPPORTED; more than (2^31 - 1) * 256 instances (one launch
 *  of 256-thread blocks) with RNG_EINVAL.  Every call looks up the array's
 *  device address with the calling device current; the first call on a
 *  device also loads the library's module there (make it before any stream
 *  capture).  Every call on a device shares the one array: calls whose work
 *  overlaps on the GPU (different streams, no ordering) race and give wrong
 *  results; order them on one stream or synchronise between them.
 *  Asynchronous on cuda_stream. */
int rng_skipahead_noalloc(int kind, void *d_state, uint64_t n_instances, uint64_t n, void *cuda_stream);

/* Raw 32-bit draws.  d_out holds n * n_per_instance words (n for
 * RNG_XOR_REDUCE) in the chosen layout. */
int rng_generate_u32(rng_t h, uint32_t *d_out, uint64_t n_per_instance, int layout, void *cuda_stream);

/* Uniform floats u = (r >> 8) 2^-24 in [0, 1), exact in single precision
 * (Sec. 2: u_n = x_n / m, here on the 24 high bits). */
int rng_generate_f32(rng_t h, float *d_out, uint64_t n_per_instance, int layout, void *cuda_stream);

/* Standard normal deviates by Box-Muller on consecutive pairs (r0, r1) of a
 * stream: u1 = ((r0 >> 8) + 1) 2^-24, u2 = (r1 >> 8) 2^-24,
 * z0 = sqrt(-2 ln u1) cos(2 pi u2), z1 = sqrt(-2 ln u1) sin(2 pi u2), in
 * single precision (within 2e-6 of the exact values).  n_per_instance must
 * be even.  The paper has no normal deviates; this is the conventional
 * transform of its uniform output. */
int rng_generate_normal(rng_t h, float *d_out, uint64_t n_per_instance, int layout, void *cuda_stream);

/* The same Box-Muller transform on caller-provided words: pair i of
 * d_in (words 2i, 2i+1, as r0, r1 above) becomes normals d_out[2i],
 * d_out[2i+1].  d_in, d_out: device arrays of 2 n_pairs elements, 16-byte
 * aligned (else RNG_EINVAL), owned by the caller.  Asynchronous.  (The
 * paper has no normal deviates; this exposes the conversion of
 * rng_generate_normal for streams produced elsewhere.) */
int rng_u32_to_normal(const uint32_t *d_in, float *d_out, uint64_t n_pairs, void *cuda_stream);

/* Checkpoint: copies the full generator state (plus kind, sizes, flags and
 * draw position) into host_buf.  With host_buf == NULL only *bytes is set
 * to the required size.  rng_set_state restores a blob taken from a handle
 * of the same kind, size and flags.  Counter-based and Weyl parts need no
 * stored state beyond the position (Sec. 6 and 7). */
int rng_get_state(rng_t h, void *host_buf, size_t *bytes);
int rng_set_state(rng_t h, const void *host_buf, size_t bytes);

/* Kind, number of instances held, first global instance, and draws consumed. */
int rng_info(rng_t h, int *kind, uint64_t *n_instances, uint64_t *first, uint64_t *position);

/* The MWC multipliers in use: the descending list of a < 2^32 with a 2^32 - 1
 * and a 2^31 - 1 prime (Sec. 3), entries [first, first + count) copied to
 * host_out.  Found on the device by Miller-Rabin; cached per device. */
int rng_mwc_multipliers(uint64_t first, uint64_t count, uint32_t *host_out);

/* ------------------------------------------------------------------ Ising */

/* Creates an L x L periodic 2D Ising ferromagnet (J = 1, zero field) at
 * inverse temperature beta >= 0, updated by checkerboard Metropolis (Sec. 2,
 * application test).  Colour of site (x, y) = (x + y) & 1; the colour-c
 * sites are numbered q = y (L/2) + (x >> 1); stream s owns q in
 * [sG, (s+1)G) of both colours, giving L^2/(2G) streams of generator
 * `rng_kind` seeded by rng_seed(seed) semantics with `rng_flags`.  The
 * block-shared kinds (RNG_MT19937_SHARED, Sec. 5; RNG_LFIB521 and
 * RNG_LFIB1279, Sec. 4 and Table 1) share one generator among 32 streams:
 * generator j of ceil(streams / 32), seeded as generator j of a generation
 * handle, feeds streams 32j .. 32j+31 in lane order, so the d-th number of
 * stream 32j + l is word 32d + l of generator j's stream (as the 1024-bit
 * generator feeds its lanes).  Their states are too large to stay on chip
 * for a whole lattice, so their sweeps run the per-half-sweep path: each
 * half-sweep the generators write their 32 G words per generator to an
 * L2-resident buffer (the generation kernels), and one kernel consumes
 * them; ising_batch_create and ising_sweep_multihit do not take them
 * (RNG_EUNSUPPORTED).  Initial spins: site j = y L + x is +1 iff bit j % 64 of
 * SplitMix64 word j / 64 of (seed XOR 0x5350494E) is set.  Requires L even,
 * 4 <= L <= 65536, G dividing L/2 (each stream's sites lie in one row), and
 * L % 64 == 0 for ISING_MULTISPIN32. */
int ising_create(ising_t *out, uint32_t L, double beta, int layout, int rng_kind, uint32_t rng_flags,
                 uint64_t seed, uint32_t G, void *cuda_stream);

/* n_sweeps sweeps (colour 0 then colour 1).  In a half-sweep every stream
 * draws one number per owned site in increasing q, whatever the energy
 * change dE = 2 s_i sum_nn s_j, and the flip is accepted iff dE <= 0 or
 * r < T[dE], T[dE] = floor(2^32 exp(-beta dE)) computed once in double.
 * With measure_every > 0 the energy E and magnetisation M are measured
 * after every measure_every-th sweep and accumulated (see
 * ising_observables).  Persistent fused kernel: random numbers never leave
 * registers and the lattice stays on chip between half-sweeps.  A lattice
 * too large for any plan of co-resident row strips (beyond about 4096^2
 * int8 or 8192^2 multispin on a GB300) runs the per-half-sweep kernels of
 * ising_sweep_plain instead, with the same result.  Asynchronous: a
 * timed-out wait between row strips (RNG_ETIMEOUT) is reported by the next
 * ising_observables / ising_get_spins. */
int ising_sweep(ising_t h, uint64_t n_sweeps, uint32_t measure_every, void *cuda_stream);

/* n_rounds rounds of the multi-hit (double checkerboard) update, Sec. 2
 * (the t_up^{k=100} column of Table 1: k hits per tile load).  The rows
 * are cut into n_strips equal strips (n_strips even, dividing L); strip b
 * has coarse colour b & 1.  A round is two phases C = 0, 1: in phase C the
 * strips of coarse colour C each take k full checkerboard sweeps of their
 * own rows (colour 0 then colour 1, k times) while the other strips stay
 * fixed, so a strip's updates see its neighbours' boundary rows as they
 * were at the start of the phase.  Each stream draws its G numbers per
 * half-sweep in the same order as in ising_sweep, so a round advances every
 * stream by 2kG draws; k = 1 is a legal Markov chain with a different
 * update order than ising_sweep, and no round equals a plain sweep.
 * measure_every counts rounds (E, M measured after the round).  Requires
 * one lattice per handle of a per-thread kind or the 1024-bit generator
 * (else RNG_EUNSUPPORTED), 1 <= k <= 65536, each
 * strip's streams a multiple of 32 (whole warps), L % 8 == 0 for
 * ISING_INT8, two strips per block fitting in shared memory and n_strips/2
 * co-resident blocks (else RNG_EINVAL / RNG_EUNSUPPORTED).  Asynchronous
 * like ising_sweep. */
int ising_sweep_multihit(ising_t h, uint64_t n_rounds, uint32_t k, uint32_t n_strips, uint32_t measure_every,
                         void *cuda_stream);

/* Same result as ising_sweep, one kernel launch per half-sweep with the
 * generator state and lattice in global memory (the baseline the
 * persistent kernel is compared with). */
int ising_sweep_plain(ising_t h, uint64_t n_sweeps, uint32_t measure_every, void *cuda_stream);

/* Current E = -sum_bonds s_i s_j and M = sum_i s_i, and the accumulators
 * acc = {sum E, sum E^2, sum M^2, sum |M|} over n_meas measurements (the
 * quantities of Table 1: e = -<E>/N, C_V = beta^2 (<E^2> - <E>^2)/N).
 * Synchronises the handle's stream.  Any output pointer may be NULL. */
int ising_observables(ising_t h, int64_t *E, int64_t *M, int64_t acc[4], uint64_t *n_meas);

/* Launch shape of the persistent kernel: threads per block (multiple of 32,
 * <= 1024; 0 = heuristic), blocks per SM the row-strip plan aims for (0 =
 * heuristic), and the fewest sites a block takes before lattices are split
 * into more strips (0 = 1024).  With all three 0, a single lattice whose
 * streams fit one block (at most 1024) runs whole in one block with one
 * stream per thread, and one needing 1024 to 2048 streams per SM runs two
 * blocks of 512 threads per SM; everything else aims for one block per SM.
 * Results do not depend on the shape: the draw order is fixed by the site
 * numbering alone. */
int ising_set_launch(ising_t h, uint32_t threads, int ctas_per_sm, uint32_t min_sites_per_block);

/* How far the strips of the exact checkerboard exchange boundary rows
 * (Sec. 2 application test; the exchange itself is this library's):
 * depth 1, after every half-sweep, each strip updating only its own rows;
 * depth 2, once per sweep, each strip also updating colour 0 of the row just
 * outside it on either side with copies of the neighbours' streams, which
 * draw exactly as their owners do (the spins are the same either way).
 * Depth 2 needs a plan of one strip of 4 to 10 rows per block of 1024
 * threads whose rows hold at most 256 streams (else depth 1 runs).  0 (the
 * default) takes depth 2 there for every generator but Philox4x32-10 on
 * int8 spins; ising_autotune times both.  Other values:
 * RNG_EINVAL.  Takes effect at the next sweep (replans). */
int ising_set_halo_depth(ising_t h, uint32_t depth);

/* The depth last set by ising_set_halo_depth or chosen by ising_autotune
 * (0: automatic). */
int ising_get_halo_depth(ising_t h, uint32_t *depth);

/* The launch shape last set by ising_set_launch or chosen by
 * ising_autotune (zeros: heuristic), so that a tuned shape can be stored
 * and set again on a handle of the same lattices.  Any pointer may be
 * NULL. */
int ising_get_launch(ising_t h, uint32_t *threads, int *ctas_per_sm, uint32_t *min_sites_per_block);

/* Times the persistent kernel on a clone of the handle (same lattices and
 * seeds; the handle itself does not advance) for a few launch shapes,
 * probe_sweeps sweeps each, and applies the fastest (reported through the
 * optional outputs).  The block-shared kinds have no persistent shape to
 * tune: RNG_OK with *threads = 256 and *ctas_per_sm = 0. */
int ising_autotune(ising_t h, uint32_t probe_sweeps, uint32_t *threads, int *ctas_per_sm);

/* The current persistent launch plan: launches per chunk of sweeps (one per
 * wave of each kind group: lattices of one generator kind whose streams fit
 * the registers of the device together, at most 2048 per SM), thread blocks
 * and row strips summed over them, and the largest threads per block.
 * Plans on first use. */
int ising_plan_info(ising_t h, uint32_t *groups, uint32_t *blocks, uint32_t *strips, uint32_t *threads);

/* Failure-detection hook for tests: row strip `strip` (-1: none) of the
 * plan stops publishing its boundary rows, so the strips next to it wait
 * until wait_budget_ns (0: the default of 2 s) runs out, record
 * RNG_ETIMEOUT and end the launch; the next ising_observables or
 * ising_get_spins returns RNG_ETIMEOUT and the handle's lattice is then
 * undefined.  The device context stays usable. */
int ising_debug_mute_strip(ising_t h, int32_t strip, uint64_t wait_budget_ns);

/* Bounds-check build.  The library compiled with -DRNG_BOUNDS_CHECK (a
 * separate shared object, see build.py) checks the shared- and
 * global-memory indices of the generation kernels, the lagged Fibonacci
 * kernels and the persistent Ising kernel: an index out of range is
 * recorded and the access skipped, so that it becomes an error status
 * instead of a memory fault.  This call synchronises the device and reports
 * the first recorded access (*site = file code * 10000 + source line; 0:
 * none), clearing the records when reset != 0.  A library built without
 * the checks returns RNG_EUNSUPPORTED. */
int rng_debug_bounds_status(int *site, int reset);

/* Spins as int8 +-1, row-major y L + x (host_LxL holds L*L bytes). */
int ising_get_spins(ising_t h, int8_t *host_LxL);
int ising_set_spins(ising_t h, const int8_t *host_LxL);

/* Generator state of the lattice's streams (see rng_get_state). */
int ising_get_rng(ising_t h, rng_t *rng);

int ising_destroy(ising_t h);

/* Number of lattices of the handle, and lattice idx's size, layout,
 * generator kind and sweeps done since creation.  Any output may be NULL. */
int ising_info(ising_t h, uint32_t idx, uint32_t *n_lattices, uint32_t *L, int *layout, int *rng_kind,
               uint64_t *sweeps_done);

/* ---------------------------------------------------------------- batched */

/* n independent lattices of sizes L[b], inverse temperatures beta[b] and
 * generator kinds rng_kind[b] (RNG_XORWOW or RNG_XS1024W or any per-thread
 * kind; the block-shared kinds: RNG_EUNSUPPORTED), lattice b seeded with
 * w_b of the master seed; int8 layout.
 * Batching is not in the paper: it packs many application-test lattices
 * into persistent launches over work lists of (lattice, row strip) items. */
int ising_batch_create(ising_t *out, uint32_t n, const uint32_t *L, const double *beta,
                       const int *rng_kind, uint64_t seed, uint32_t G, void *cuda_stream);

/* All lattices advance n_sweeps sweeps, as one CUDA graph (captured once and
 * replayed when the same n_sweeps is requested again).  Lattices of one
 * generator kind run in waves whose streams fit the device's registers
 * together; per chunk of 4096 sweeps each wave is one persistent launch.
 * Each lattice's result equals ising_sweep on that lattice alone. */
int ising_batch_sweep(ising_t h, uint64_t n_sweeps, uint32_t measure_every, void *cuda_stream);

/* Lattice `idx` of a batch: observables and spins as for single lattices. */
int ising_batch_observables(ising_t h, uint32_t idx, int64_t *E, int64_t *M, int64_t acc[4],
                            uint64_t *n_meas);
int ising_batch_get_spins(ising_t h, uint32_t idx, int8_t *host_LxL);

/* ---------------------------------------------------------------- serving */

/* A request loop with continuous batching (not in the paper): generator
 * states stay resident on the device as "stream sets", and requests that
 * arrive while others run are admitted as soon as a slot (one of n_slots
 * CUDA streams for draws, plus four for sweeps) and device memory (a byte
 * budget for outputs and lattices) are free, in arrival order within each
 * request type (a request waiting for a slot of its type holds back only
 * later requests of that type); their GPU work overlaps.  The lattices of fetched sweep requests are kept (a few
 * per slot, size and kind) and reset for the next request of that shape
 * instead of being created again.  A host worker thread owns all of the
 * server's CUDA calls; submit, wait and fetch may be called from any host
 * thread. */
typedef struct rng_server_s *rng_server_t;

enum { RNG_REQ_DRAW = 0, RNG_REQ_SWEEP = 1 };
enum { RNG_OUT_U32 = 0, RNG_OUT_F32 = 1, RNG_OUT_NORMAL = 2 };

typedef struct {
    int32_t type;      /* RNG_REQ_DRAW or RNG_REQ_SWEEP */
    int32_t kind;      /* generator kind, any per-thread kind (not a block-shared one) */
    uint64_t seed;     /* draw: stream-set seed; sweep: lattice seed */
    uint64_t offset;   /* draw: draws skipped in every instance of the set */
    uint64_t count;    /* draw: numbers returned (even for normals) */
    int32_t out;       /* draw: RNG_OUT_U32, RNG_OUT_F32 or RNG_OUT_NORMAL */
    uint32_t L;        /* sweep: lattice size (even, 4..16384) */
    double beta;       /* sweep: inverse temperature */
    uint64_t sweeps;   /* sweep: number of sweeps */
} rng_request_t;

typedef struct {
    int32_t status;    /* RNG_OK or the request's error */
    int32_t done;
    uint64_t bytes;    /* result size: draw count*4, sweep L*L */
    uint64_t t_submit_ns, t_start_ns, t_done_ns;  /* host steady clock */
    int64_t E, M;      /* sweep: energy and magnetisation after the sweeps */
} rng_result_t;

/* A draw request returns, in step-major order, the first `count` numbers of
 * the n = instances_per_set instances of stream set (kind, seed) -- seeded
 * as rng_seed(seed) -- advanced by `offset` draws:
 * result[j] = s_(j mod n)[offset + j div n].  A sweep request returns the
 * int8 spins of ising_create(L, beta, ISING_INT8, kind, 0, seed, 2) after
 * `sweeps` sweeps, with E and M.  Each result is a pure function of its
 * request, whatever else is in flight.  Up to n_sets stream sets stay
 * resident (least recently used evicted). */
int rng_server_create(rng_server_t *out, uint32_t n_sets, uint32_t instances_per_set, uint32_t n_slots,
                      uint64_t mem_budget_bytes);
/* Queues a request; RNG_EBUSY if the queue is full, RNG_ENOMEM if the
 * request alone exceeds the memory budget. */
int rng_server_submit(rng_server_t s, const rng_request_t *req, uint64_t *ticket);
/* Waits (timeout_s < 0: forever) until the request is done; fills *res. */
int rng_server_wait(rng_server_t s, uint64_t ticket, double timeout_s, rng_result_t *res);
/* Copies a finished request's result to host memory (host_dst may be NULL
 * to discard it) and releases the request and its device memory. */
int rng_server_fetch(rng_server_t s, uint64_t ticket, void *host_dst, uint64_t bytes);
int rng_server_stats(rng_server_t s, uint64_t *submitted, uint64_t *completed, uint64_t *mem_in_use,
                     uint32_t *max_concurrent);
int rng_server_destroy(rng_server_t s);

/* ----------------------------------------------------------- measurement */

/* Throughput of the SM pipes on the current device, in thread-instructions
 * per second over the whole GPU: 32-bit logic (LOP3), integer multiply-add
 * (IMAD), warp shuffle (SHFL) and float FMA (FFMA; its full rate equals the
 * issue rate of one warp-instruction per scheduler and cycle).  Each is
 * timed on eight independent chains per thread at full occupancy, best of
 * three runs with CUDA events on cuda_stream (synchronises it).  Any output
 * pointer may be NULL.  Not part of the paper: the denominators of the
 * instruction-issue rooflines of the consume-in-register and normal modes. */
int rng_issue_peaks(double *lop3, double *imad, double *shfl, double *ffma, void *cuda_stream);

/* ------------------------------------------------------------- allocator */

/* Device memory the library owns for its handles (generator state,
 * lattices, plans, scratch, server request buffers) comes from
 * cudaMallocAsync / cudaFreeAsync on the handle's stream unless an
 * allocator is installed here, e.g. a framework's caching allocator
 * (process-lifetime tables -- MWC multipliers, GF(2) sub-stream matrices,
 * the server's skip ladders -- stay on cudaMalloc).  alloc: *ptr = `bytes` of device memory on the current
 * device, usable on `cuda_stream` (stream-ordered), returns 0 on success and
 * nonzero on failure (reported as RNG_ENOMEM); free: releases a pointer from
 * alloc, ordered after work on `cuda_stream`.  The hooks may be called from
 * the request server's worker thread.  Process-wide; alloc = free = NULL
 * restores the default.  Returns RNG_EBUSY while any memory from the
 * previous allocator is outstanding (install it before creating handles and
 * change it only after destroying them), RNG_EINVAL if exactly one hook is
 * NULL.  Not part of the paper: an integration point for the caller's
 * memory management. */
typedef int (*rng_alloc_fn)(void **ptr, size_t bytes, void *cuda_stream, void *ctx);
typedef void (*rng_free_fn)(void *ptr, void *cuda_stream, void *ctx);
int rng_set_allocator(rng_alloc_fn alloc, rng_free_fn free, void *ctx);

/* ----------------------------------------------------------------- errors */

const char *rng_strerror(int status);
const char *rng_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* RNG_GB300_H */
