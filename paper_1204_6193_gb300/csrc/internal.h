// internal.h -- shared declarations of the library's translation units
// (handles, error reporting, device allocation, launchers).  Not installed.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include "../../include/rng_gb300.h"

namespace rngx {

constexpr int MT_N_WORDS = 624;  // MT19937 state words (Sec. 5: N = 624)
constexpr int kNumKinds = RNG_LFIB1279 + 1;  // generator kinds 0 .. kNumKinds-1

// Block-shared generators: an instance is one generator whose state a
// group of threads shares (no per-thread stream, no Ising consumer).
constexpr bool is_block_shared(int kind)
{
    return kind == RNG_MT19937_SHARED || kind == RNG_LFIB521 || kind == RNG_LFIB1279;
}

// ------------------------------------------------------------- errors
void set_error(const char *fmt, ...);
int cuda_fail(cudaError_t e, const char *what);

#define RNGX_CHECK_CUDA(expr)                                   \
    do {                                                        \
        cudaError_t _e = (expr);                                \
        if (_e != cudaSuccess) return ::rngx::cuda_fail(_e, #expr); \
    } while (0)

#define RNGX_CHECK(expr)              \
    do {                              \
        int _s = (expr);              \
        if (_s != RNG_OK) return _s;  \
    } while (0)

// ---------------------------------------------------- fault injection
// Host-side failures for testing error paths without any GPU fault, chosen
// by the environment variable RNG_FAULT (read at every check, so a process
// may change it): "oom" fails every library allocation with RNG_ENOMEM,
// "oom:N" only the N-th from now; "launch" reports every kernel launch as
// failed (RNG_ECUDA) after it was issued; "timeout" makes the next status
// check of an Ising handle report a timed-out neighbour wait (RNG_ETIMEOUT).
bool fault_oom();
bool fault_launch();
bool fault_timeout();
int injected(const char *what, int status);

#define RNGX_CHECK_LAUNCH()                                                          \
    do {                                                                             \
        if (::rngx::fault_launch()) return ::rngx::injected("kernel launch", RNG_ECUDA); \
        RNGX_CHECK_CUDA(cudaGetLastError());                                         \
    } while (0)

// ---------------------------------------------------- device allocation
// Stream-ordered device memory owned by the library.
int dalloc(void **p, size_t bytes, cudaStream_t s);
void dfree(void *p, cudaStream_t s);

// ------------------------------------------------------ generator state
// Per-instance state arrays, structure of arrays so that consecutive
// instances are consecutive words (coalesced loads and stores).
struct GenState {
    int kind;
    uint32_t flags;
    uint64_t n;          // instances held
    uint64_t first;      // global index of the first instance
    uint64_t n_total;    // instances of the whole (sharded) generator
    void *s[6];          // state arrays (meaning depends on kind)
    const uint32_t *mwc_a;  // per-instance multipliers (MWC without SAME_A)
    uint32_t mwc_a0;     // shared multiplier (MWC_SAME_A)
    uint64_t A, C;       // LCG map applied per draw: (a, c), or (a_n, c_n) when leapfrogging
    uint64_t pos;        // draws consumed since seeding (uniform over instances)
    int philox_rounds;
};

}  // namespace rngx

struct rng_s {
    rngx::GenState g;
    int device;
    cudaStream_t stream;     // stream used for allocation and host-side setup
    size_t state_bytes;      // bytes of state arrays
    void *state;             // one allocation holding all arrays
    bool seeded;
    uint64_t seed;
};

namespace rngx {

// Device kernels launched by the handle code (gen.cu, init.cu, gf2.cu, mwc.cu).
int launch_generate(const GenState &g, void *d_out, uint64_t K, int out_kind, int layout, cudaStream_t s);
int launch_seed(GenState &g, uint64_t seed, cudaStream_t s);
int launch_skipahead(GenState &g, uint64_t t, cudaStream_t s);
int launch_u32_to_normal(const uint32_t *in, float *out, uint64_t n_pairs, cudaStream_t s);
int launch_generate_lfib(const GenState &g, void *d_out, uint64_t K, int out_kind, int layout, cudaStream_t s);
int launch_seed_lfib(GenState &g, uint64_t seed, cudaStream_t s);

// Output kinds of the generation kernels.
enum { OUT_U32 = 0, OUT_F32 = 1, OUT_NORMAL = 2 };

// MWC multipliers: device table with at least `count` entries, cached per device.
int mwc_table(uint64_t count, const uint32_t **d_table, cudaStream_t s);

// GF(2) matrices of the xorshift kinds: one-step matrix and its powers.
// n = 1024 (XS1024W) or 160 (XORWOW); rows of n/32 words; x' = x M.
int gf2_one_step(int kind, uint32_t *d_m, cudaStream_t s);
int gf2_mul(int n, const uint32_t *d_a, const uint32_t *d_b, uint32_t *d_c, cudaStream_t s);
int gf2_pow(int kind, uint64_t t, uint32_t *d_out, uint32_t *d_tmp1, uint32_t *d_tmp2, cudaStream_t s);
int xs_substream_matrices(int levels, const uint32_t **d_P, cudaStream_t s);  // P_k = M^(2^(137+k))

struct DevParams;
int launch_matrix_apply(int kind, const DevParams &p, const uint32_t *M, uint64_t t, cudaStream_t s);

// Single-lattice Ising handle back to its state after ising_create with
// (beta, seed), keeping memory and plan (the server's lattice pool).
int ising_reset_lattice(ising_t h, double beta, uint64_t seed);

// Bounds-check build (bounds.cuh): each module's first recorded site.
#define RNGX_BOUNDS_READER(name) int bounds_site_##name(int *site, bool reset);
RNGX_BOUNDS_READER(gen)
RNGX_BOUNDS_READER(lfib)
RNGX_BOUNDS_READER(persist_RNG_LCG32)
RNGX_BOUNDS_READER(persist_RNG_LCG64)
RNGX_BOUNDS_READER(persist_RNG_MWC)
RNGX_BOUNDS_READER(persist_RNG_XORWOW)
RNGX_BOUNDS_READER(persist_RNG_PHILOX4X32_10)
RNGX_BOUNDS_READER(persist_RNG_PHILOX4X32_7)
RNGX_BOUNDS_READER(persist_RNG_XS1024W)
#undef RNGX_BOUNDS_READER

}  // namespace rngx
