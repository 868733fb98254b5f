// init.cu -- seeding and skip-ahead kernels.  Seeding expands one master
// seed into SplitMix64 words indexed by the global instance number, so a
// shard of instances [first, first + n) seeds exactly like the same range
// of one large handle.
#include <vector>

#include "gen_device.cuh"
#include "modarith.cuh"

namespace rngx {
namespace {

constexpr int kBlock = 256;

inline unsigned blocks_for(uint64_t n) { return static_cast<unsigned>((n + kBlock - 1) / kBlock); }

constexpr uint64_t kLcg32A = 1664525ull, kLcg32C = 1013904223ull;
constexpr uint64_t kLcg64A = 2862933555777941757ull, kLcg64C = 1442695040888963407ull;

__global__ void k_seed_lcg(DevParams p, uint64_t seed, uint64_t first, uint64_t n_total, int is64, int leapfrog)
{
    const uint64_t li = static_cast<uint64_t>(blockIdx.x) * kBlock + threadIdx.x;
    if (li >= p.n) return;
    const uint64_t i = first + li;
    const uint64_t mask = is64 ? ~0ull : 0xffffffffull;
    uint64_t x;
    if (leapfrog) {
        // one serial sequence from w_0; instance i starts at x_(i+1-n)
        const uint64_t x0 = d_seed_word(seed, 0) & mask;
        uint64_t at, ct;
        affine_pow(is64 ? kLcg64A : kLcg32A, is64 ? kLcg64C : kLcg32C, i + 1 - n_total, at, ct);
        x = (at * x0 + ct) & mask;
    } else {
        x = d_seed_word(seed, i) & mask;
    }
    if (is64) static_cast<uint64_t *>(p.s[0])[li] = x;
    else static_cast<uint32_t *>(p.s[0])[li] = static_cast<uint32_t>(x);
}

__global__ void k_seed_mwc(DevParams p, uint64_t seed, uint64_t first)
{
    const uint64_t li = static_cast<uint64_t>(blockIdx.x) * kBlock + threadIdx.x;
    if (li >= p.n) return;
    const uint32_t a = p.mwc_a ? p.mwc_a[li] : p.mwc_a0;
    const uint64_t w = d_seed_word(seed, first + li);
    uint64_t x = w & 0xffffffffull;
    const uint64_t c = (w >> 32) % a;
    if ((x == 0 && c == 0) || (x == 0xffffffffull && c == a - 1)) x = 1;  // fixed points
    static_cast<uint64_t *>(p.s[0])[li] = (c << 32) | x;
}

__global__ void k_seed_xorwow(DevParams p, uint64_t seed, uint64_t first)
{
    const uint64_t li = static_cast<uint64_t>(blockIdx.x) * kBlock + threadIdx.x;
    if (li >= p.n) return;
    const uint64_t i = first + li;
    const uint64_t w0 = d_seed_word(seed, 3 * i), w1 = d_seed_word(seed, 3 * i + 1), w2 = d_seed_word(seed, 3 * i + 2);
    uint32_t v[6] = {static_cast<uint32_t>(w0), static_cast<uint32_t>(w0 >> 32), static_cast<uint32_t>(w1),
                     static_cast<uint32_t>(w1 >> 32), static_cast<uint32_t>(w2), static_cast<uint32_t>(w2 >> 32)};
    if ((v[0] | v[1] | v[2] | v[3] | v[4]) == 0) v[0] = 1;
    for (int k = 0; k < 6; k++) static_cast<uint32_t *>(p.s[k])[li] = v[k];
}

// Philox keys: the instance's seed word, or the intrinsic key (global
// instance index, low half of the seed) -- Sec. 7.
__global__ void k_seed_philox(DevParams p, uint64_t seed, uint64_t first, bool intrinsic)
{
    const uint64_t li = static_cast<uint64_t>(blockIdx.x) * kBlock + threadIdx.x;
    if (li >= p.n) return;
    const uint64_t i = first + li;
    static_cast<uint64_t *>(p.s[0])[li] =
        intrinsic ? ((seed & 0xFFFFFFFFull) << 32) | (i & 0xFFFFFFFFull) : d_seed_word(seed, i);
}

// Random seeding of the 1024-bit generator: lane l of global warp J takes
// the low half of w_(32J + l) (= w of the global instance index).
__global__ void k_seed_xs_random(DevParams p, uint64_t seed, uint64_t first)
{
    const uint64_t li = static_cast<uint64_t>(blockIdx.x) * kBlock + threadIdx.x;
    if ((li & ~31ull) >= p.n) return;
    uint32_t x = static_cast<uint32_t>(d_seed_word(seed, first + li));
    const unsigned nz = __ballot_sync(0xffffffffu, x != 0);
    if (nz == 0 && (threadIdx.x & 31) == 31) x = 1;
    static_cast<uint32_t *>(p.s[0])[li] = x;
}

// x <- x P for one warp's 1024-bit state (lane l holds word l, bit j of the
// vector = bit j % 32 of word j / 32); P has 1024 rows of 32 words.
__device__ __forceinline__ uint32_t warp_vecmul1024(uint32_t x, const uint32_t *__restrict__ P)
{
    const int lane = threadIdx.x & 31;
    uint32_t acc = 0;
    for (int wi = 0; wi < 32; wi++) {
        uint32_t bits = __shfl_sync(0xffffffffu, x, wi);
        while (bits) {
            const int b = __ffs(bits) - 1;
            bits &= bits - 1;
            acc ^= __ldg(P + (static_cast<size_t>(wi) * 32 + b) * 32 + lane);
        }
    }
    return acc;
}

// Sub-stream seeding (Sec. 6): every warp starts from the base state (words
// from w_0..w_15, lane 2m = high half and lane 2m+1 = low half of w_m) and
// global warp J advances J * 2^137 steps: x_J = base prod_{bit k of J} P_k
// with P_k = M^(2^(137+k)).
__global__ void k_seed_xs_substream(DevParams p, uint64_t seed, uint64_t first, const uint32_t *P, int levels)
{
    const uint64_t li = static_cast<uint64_t>(blockIdx.x) * kBlock + threadIdx.x;
    if ((li & ~31ull) >= p.n) return;
    const int lane = threadIdx.x & 31;
    const uint64_t w = d_seed_word(seed, lane >> 1);
    uint32_t x = (lane & 1) ? static_cast<uint32_t>(w) : static_cast<uint32_t>(w >> 32);
    const unsigned nz = __ballot_sync(0xffffffffu, x != 0);
    if (nz == 0 && lane == 31) x = 1;
    const uint64_t J = (first + li) >> 5;
    for (int k = 0; k < levels; k++)
        if ((J >> k) & 1) x = warp_vecmul1024(x, P + static_cast<size_t>(k) * 1024 * 32);
    static_cast<uint32_t *>(p.s[0])[li] = x;
}

// MT19937 standard 32-bit seeding recurrence, one thread per generator.
__global__ void k_seed_mt(DevParams p, uint64_t seed, uint64_t first)
{
    const uint64_t g = static_cast<uint64_t>(blockIdx.x) * kBlock + threadIdx.x;
    if (g >= p.n) return;
    uint32_t *mt = static_cast<uint32_t *>(p.s[0]) + g * MT_N;
    uint32_t v = static_cast<uint32_t>(d_seed_word(seed, first + g));
    mt[0] = v;
    for (int i = 1; i < MT_N; i++) {
        v = 1812433253u * (v ^ (v >> 30)) + static_cast<uint32_t>(i);
        mt[i] = v;
    }
}

// ------------------------------------------------------------ skip-ahead
__global__ void k_skip_lcg(DevParams p, uint64_t t, int is64)
{
    const uint64_t li = static_cast<uint64_t>(blockIdx.x) * kBlock + threadIdx.x;
    if (li >= p.n) return;
    uint64_t at, ct;
    affine_pow(p.A, p.C, t, at, ct);
    if (is64) {
        uint64_t *x = static_cast<uint64_t *>(p.s[0]) + li;
        *x = at * *x + ct;
    } else {
        uint32_t *x = static_cast<uint32_t *>(p.s[0]) + li;
        *x = static_cast<uint32_t>(at) * *x + static_cast<uint32_t>(ct);
    }
}

// MWC: v_t = v_0 a^t mod (a 2^32 - 1) (a step divides v by 2^32 = a^(-1)).
__global__ void k_skip_mwc(DevParams p, uint64_t t)
{
    const uint64_t li = static_cast<uint64_t>(blockIdx.x) * kBlock + threadIdx.x;
    if (li >= p.n) return;
    const uint32_t a = p.mwc_a ? p.mwc_a[li] : p.mwc_a0;
    const uint64_t mod = (static_cast<uint64_t>(a) << 32) - 1;
    const Mont m = mont_setup(mod);
    uint64_t *v = static_cast<uint64_t *>(p.s[0]) + li;
    const uint64_t am = mont_pow(to_mont(a, m), t, m);
    *v = from_mont(mont_mul(to_mont(*v, m), am, m), m);
}

__global__ void k_skip_xorwow(DevParams p, const uint32_t *__restrict__ T, uint64_t t)
{
    const uint64_t li = static_cast<uint64_t>(blockIdx.x) * kBlock + threadIdx.x;
    if (li >= p.n) return;
    uint32_t in[5], out[5] = {0, 0, 0, 0, 0};
    for (int k = 0; k < 5; k++) in[k] = static_cast<uint32_t *>(p.s[k])[li];
    for (int wi = 0; wi < 5; wi++) {
        uint32_t bits = in[wi];
        while (bits) {
            const int b = __ffs(bits) - 1;
            bits &= bits - 1;
            const uint32_t *row = T + (wi * 32 + b) * 5;
#pragma unroll
            for (int k = 0; k < 5; k++) out[k] ^= __ldg(row + k);
        }
    }
    for (int k = 0; k < 5; k++) static_cast<uint32_t *>(p.s[k])[li] = out[k];
    static_cast<uint32_t *>(p.s[5])[li] += static_cast<uint32_t>(t) * 362437u;
}

__global__ void k_skip_xs(DevParams p, const uint32_t *M)
{
    const uint64_t li = static_cast<uint64_t>(blockIdx.x) * kBlock + threadIdx.x;
    if ((li & ~31ull) >= p.n) return;
    uint32_t *x = static_cast<uint32_t *>(p.s[0]) + li;
    *x = warp_vecmul1024(*x, M);
}

}  // namespace

int launch_seed(GenState &g, uint64_t seed, cudaStream_t s)
{
    const DevParams p = dev_params(g);
    const unsigned nb = blocks_for(g.n);
    switch (g.kind) {
    case RNG_LCG32:
    case RNG_LCG64:
        k_seed_lcg<<<nb, kBlock, 0, s>>>(p, seed, g.first, g.n_total, g.kind == RNG_LCG64,
                                          (g.flags & RNG_SEED_LEAPFROG) != 0);
        break;
    case RNG_MWC: k_seed_mwc<<<nb, kBlock, 0, s>>>(p, seed, g.first); break;
    case RNG_XORWOW: k_seed_xorwow<<<nb, kBlock, 0, s>>>(p, seed, g.first); break;
    case RNG_PHILOX4X32_10:
    case RNG_PHILOX4X32_7:
        k_seed_philox<<<nb, kBlock, 0, s>>>(p, seed, g.first, (g.flags & RNG_PHILOX_INTRINSIC_KEY) != 0);
        break;
    case RNG_XS1024W:
        if (g.flags & RNG_SEED_SUBSTREAM) {
            int levels = 0;
            const uint64_t last_warp = (g.first + g.n - 1) >> 5;
            while (levels < 64 && (last_warp >> levels) != 0) levels++;
            const uint32_t *P = nullptr;
            if (levels > 0) RNGX_CHECK(xs_substream_matrices(levels, &P, s));
            k_seed_xs_substream<<<nb, kBlock, 0, s>>>(p, seed, g.first, P, levels);
        } else {
            k_seed_xs_random<<<nb, kBlock, 0, s>>>(p, seed, g.first);
        }
        break;
    case RNG_MT19937_SHARED: k_seed_mt<<<nb, kBlock, 0, s>>>(p, seed, g.first); break;
    case RNG_LFIB521:
    case RNG_LFIB1279: return launch_seed_lfib(g, seed, s);
    default: set_error("launch_seed: unknown kind %d", g.kind); return RNG_EINVAL;
    }
    RNGX_CHECK_LAUNCH();
    return RNG_OK;
}

// Applies a precomputed t-step GF(2) matrix to every instance of an
// xorshift kind (and advances XORWOW's Weyl word by t steps).
int launch_matrix_apply(int kind, const DevParams &p, const uint32_t *M, uint64_t t, cudaStream_t s)
{
    const unsigned nb = blocks_for(p.n);
    if (kind == RNG_XS1024W) k_skip_xs<<<nb, kBlock, 0, s>>>(p, M);
    else k_skip_xorwow<<<nb, kBlock, 0, s>>>(p, M, t);
    RNGX_CHECK_LAUNCH();
    return RNG_OK;
}

int launch_skipahead(GenState &g, uint64_t t, cudaStream_t s)
{
    if (t == 0) return RNG_OK;
    const DevParams p = dev_params(g);
    const unsigned nb = blocks_for(g.n);
    switch (g.kind) {
    case RNG_LCG32:
    case RNG_LCG64:
        k_skip_lcg<<<nb, kBlock, 0, s>>>(p, t, g.kind == RNG_LCG64);
        break;
    case RNG_MWC: k_skip_mwc<<<nb, kBlock, 0, s>>>(p, t); break;
    case RNG_PHILOX4X32_10:
    case RNG_PHILOX4X32_7: break;  // counter-based: the position alone moves
    case RNG_XORWOW:
    case RNG_XS1024W: {
        const int n = g.kind == RNG_XS1024W ? 1024 : 160;
        const size_t mbytes = static_cast<size_t>(n) * (n / 32) * sizeof(uint32_t);
        void *buf = nullptr;
        RNGX_CHECK(dalloc(&buf, 3 * mbytes, s));
        uint32_t *m0 = static_cast<uint32_t *>(buf);
        uint32_t *m1 = m0 + mbytes / 4, *m2 = m1 + mbytes / 4;
        int st = gf2_pow(g.kind, t, m0, m1, m2, s);
        if (st == RNG_OK) {
            if (g.kind == RNG_XS1024W) k_skip_xs<<<nb, kBlock, 0, s>>>(p, m0);
            else k_skip_xorwow<<<nb, kBlock, 0, s>>>(p, m0, t);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) st = cuda_fail(e, "skip-ahead kernel");
        }
        dfree(buf, s);
        RNGX_CHECK(st);
        break;
    }
    default:
        set_error("rng_skipahead: not defined for the block-shared generators (MT19937, lagged Fibonacci)");
        return RNG_EUNSUPPORTED;
    }
    RNGX_CHECK_LAUNCH();
    g.pos += t;
    return RNG_OK;
}

}  // namespace rngx
