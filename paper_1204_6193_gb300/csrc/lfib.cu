// lfib.cu -- the additive lagged Fibonacci generators of Sec. 4,
// Eq. (used_fibonacci): u_n = u_(n-r) + u_(n-s) (mod 1), (r, s) = (521, 353)
// and (1279, 861), run on the 32-bit words x_n = 2^32 u_n, where the
// recurrence is x_n = x_(n-r) + x_(n-s) mod 2^32 and is exact.
//
// An instance is one generator whose state (the last r words) a group of
// threads shares.  Here that group is one warp: the ring of r + s words
// sits in shared memory and the warp computes s new words per step in
// parallel (word n+j needs x_(n+j-r) and x_(n+j-s), both older than n for
// j < s, Sec. 4).  With r + s slots the s new words never overwrite a word
// another lane still reads in the same step, so a step needs no barrier
// beyond the warp sync between steps.  When the position is a multiple of
// 32 a chunked form of the same recurrence runs instead (below): the same
// words, fewer instructions per word.
//
// State in HBM: r words per generator, x_m in slot m mod r for the r most
// recent m; the handle's position counts the words produced.
#include "gen_device.cuh"
#include "internal.h"

namespace rngx {

namespace {

template <int R, int S>
struct Lfib {
    static constexpr int kRing = R + S;                                   // shared ring words
    static constexpr int kWarps = kRing * 4 * 8 <= 40 * 1024 ? 8 : 4;     // generators per block
    static constexpr int kBlock = 32 * kWarps;
};

// Seeds: x_(j-r) = low half of w_(r g + j) for global generator g; an
// all-even ring gets its low bit set (it could never become odd).
template <int R>
__global__ void k_seed_lfib(DevParams p, uint64_t seed, uint64_t first)
{
    const uint64_t g = (static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (g >= p.n) return;  // whole warps
    uint32_t *st = static_cast<uint32_t *>(p.s[0]) + g * R;
    uint32_t odd = 0;
    for (int j = lane; j < R; j += 32) {
        const uint32_t v = static_cast<uint32_t>(d_seed_word(seed, static_cast<uint64_t>(R) * (first + g) + j));
        st[j] = v;
        odd |= v & 1u;
    }
    if (!__any_sync(0xffffffffu, odd != 0) && lane == 0) st[0] |= 1u;
}

template <int R, int S, int OUT, int LAYOUT>
__global__ void __launch_bounds__(Lfib<R, S>::kBlock) k_generate_lfib(DevParams p, void *out_, uint64_t K)
{
    constexpr int RS = Lfib<R, S>::kRing;
    constexpr int W = Lfib<R, S>::kWarps;
    // a normal pair never straddles two steps: even steps from the call start
    constexpr int STEP = OUT == OUT_NORMAL ? (S & ~1) : S;
    __shared__ uint32_t ring_s[W][RS];
    BmTables bt{};
    if constexpr (OUT == OUT_NORMAL) bt = bm_stage();  // every thread, before any leaves
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint64_t g = static_cast<uint64_t>(blockIdx.x) * W + w;
    const uint64_t n = p.n;
    if (g >= n) return;  // whole warps only: no block-wide barriers below
    uint32_t *ring = ring_s[w];
    uint32_t *st = static_cast<uint32_t *>(p.s[0]) + g * R;

    // x_m, m in [pos - r, pos), goes to ring slot m mod (r + s); with
    // head = pos mod (r + s), x_(pos-r+t) sits at head + s + t (mod r + s)
    // and comes from state slot (pos + t) mod r
    const uint32_t head0 = static_cast<uint32_t>(p.pos % RS);
    const uint32_t sr0 = static_cast<uint32_t>(p.pos % R);
    for (int t = lane; t < R; t += 32) {
        uint32_t a = head0 + S + t;
        a = a >= RS ? a - RS : a;
        uint32_t b = sr0 + t;
        b = b >= R ? b - R : b;
        ring[a] = st[b];
    }
    __syncwarp();

    auto out_index = [&](uint64_t d) -> uint64_t {
        return LAYOUT == RNG_INSTANCE_MAJOR ? g * K + d : d * n + g;
    };
    uint32_t xacc = 0;
    float facc = 0.0f;
    uint32_t head = head0;
    const bool out_even = (reinterpret_cast<uintptr_t>(out_) & 7) == 0;
    for (uint64_t k = 0; k < K;) {
        const int cnt = static_cast<int>(K - k < static_cast<uint64_t>(STEP) ? K - k : STEP);
        // word pos+k+j (slot head+j) = word -r (slot head+j+s) + word -s (slot head+j+r)
        for (int j = lane; j < cnt; j += 32) {
            uint32_t a = head + j + S, b = head + j + R, c = head + j;
            a = a >= RS ? a - RS : a;
            b = b >= RS ? b - RS : b;
            c = c >= RS ? c - RS : c;
            if (!RNGX_IDX_OK(a, RS, kSiteLfib + __LINE__) || !RNGX_IDX_OK(b, RS, kSiteLfib + __LINE__) ||
                !RNGX_IDX_OK(c, RS, kSiteLfib + __LINE__))
                continue;
            const uint32_t v = ring[a] + ring[b];
            ring[c] = v;
            if (OUT != OUT_NORMAL) {
                const uint32_t bits = OUT == OUT_U32 ? v : __float_as_uint(u32_to_unit(v));
                if (LAYOUT == RNG_XOR_REDUCE) xacc ^= bits;
                else if (RNGX_IDX_OK(out_index(k + j), n * K, kSiteLfib + __LINE__))
                    __stcs(static_cast<uint32_t *>(out_) + out_index(k + j), bits);
            }
        }
        if (OUT == OUT_NORMAL) {
            __syncwarp();
            for (int t = lane; 2 * t < cnt; t += 32) {
                uint32_t c0 = head + 2 * t, c1 = head + 2 * t + 1;
                c0 = c0 >= RS ? c0 - RS : c0;
                c1 = c1 >= RS ? c1 - RS : c1;
                float z0, z1;
                box_muller(ring[c0], ring[c1], z0, z1, bt);
                if (LAYOUT == RNG_XOR_REDUCE) {
                    facc += z0;
                    facc += z1;
                } else if (LAYOUT == RNG_INSTANCE_MAJOR && out_even) {
                    // g K + k + 2t is even (K and the step even): one 8-byte store
                    __stcs(reinterpret_cast<float2 *>(static_cast<float *>(out_) + out_index(k + 2 * t)),
                           make_float2(z0, z1));
                } else {
                    float *out = static_cast<float *>(out_);
                    __stcs(out + out_index(k + 2 * t), z0);
                    __stcs(out + out_index(k + 2 * t + 1), z1);
                }
            }
        }
        __syncwarp();
        head += cnt;
        head = head >= RS ? head - RS : head;
        k += cnt;
    }
    if (LAYOUT == RNG_XOR_REDUCE) {
        if (OUT == OUT_NORMAL) {
            for (int o = 16; o > 0; o >>= 1) facc += __shfl_down_sync(0xffffffffu, facc, o);
            if (lane == 0) static_cast<float *>(out_)[g] = facc;
        } else {
            for (int o = 16; o > 0; o >>= 1) xacc ^= __shfl_down_sync(0xffffffffu, xacc, o);
            if (lane == 0) static_cast<uint32_t *>(out_)[g] = xacc;
        }
    }
    // the r newest words back to their state slots: x_(pos+K-r+t) at
    // ring head + s + t, state slot (pos + K + t) mod r
    const uint32_t srK = static_cast<uint32_t>((p.pos + K) % R);
    for (int t = lane; t < R; t += 32) {
        uint32_t a = head + S + t;
        a = a >= RS ? a - RS : a;
        uint32_t b = srK + t;
        b = b >= R ? b - R : b;
        st[b] = ring[a];
    }
}

// ----------------------------------------------------------- chunked form
// The same recurrence computed in chunks of 32 consecutive words, one word
// per lane: word m + j (j < 32) reads x_(m+j-r) and x_(m+j-s), made at least
// s - 31 words earlier, so chunks need no step structure, and the U chunks
// of a group (32U <= s) are mutually independent.  The ring has RS = 2^k >=
// r + 32U slots (x_m at slot m mod RS) followed by a mirror of its first
// 32U slots, written together with them: a group starting at a slot that
// is a multiple of 32U then reads both operand windows and writes its words
// with immediate offsets from three bases, without modular indices.  The
// words it writes replace x_(m-RS), older than every word it reads (RS >=
// r + 32U).  Used when the position is a multiple of 32; otherwise the
// step form above runs.
template <int R, int S>
struct LfibChunked {
    static constexpr int kU = 8;                       // chunks per group
    static constexpr int kG = 32 * kU;                 // words per group
    static_assert(kG <= S, "the chunks of a group must be independent");
    static constexpr int kRS = R + kG <= 1024 ? 1024 : (R + kG <= 2048 ? 2048 : 4096);
    static constexpr int kBuf = kRS + kG;              // ring and mirror
    static constexpr int kWarps = 4;                   // generators per block
    static constexpr int kBlock = 32 * kWarps;
};

template <int R, int S, int OUT, int LAYOUT>
__global__ void __launch_bounds__(LfibChunked<R, S>::kBlock) k_generate_lfib_chunked(DevParams p, void *out_,
                                                                                    uint64_t K)
{
    using F = LfibChunked<R, S>;
    constexpr int RS = F::kRS, G = F::kG, U = F::kU, W = F::kWarps;
    constexpr uint32_t MASK = RS - 1;
    __shared__ __align__(16) uint32_t ring_s[W][F::kBuf];
    BmTables bt{};
    if constexpr (OUT == OUT_NORMAL) bt = bm_stage();  // every thread, before any leaves
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint64_t g = static_cast<uint64_t>(blockIdx.x) * W + w;
    const uint64_t n = p.n;
    if (g >= n) return;  // whole warps only
    uint32_t *ring = ring_s[w];
    uint32_t *st = static_cast<uint32_t *>(p.s[0]) + g * R;

    // x_(pos-r+t) from state slot (pos + t) mod r to ring slot (pos - r + t) mod RS
    const uint32_t q0 = static_cast<uint32_t>((p.pos + RS - R) & MASK);
    const uint32_t sr0 = static_cast<uint32_t>(p.pos % R);
    for (int t = lane; t < R; t += 32) {
        const uint32_t q = (q0 + t) & MASK;
        uint32_t b = sr0 + t;
        b = b >= R ? b - R : b;
        const uint32_t v = st[b];
        ring[q] = v;
        if (q < G) ring[q + RS] = v;
    }
    __syncwarp();

    auto out_index = [&](uint64_t d) -> uint64_t {
        return LAYOUT == RNG_INSTANCE_MAJOR ? g * K + d : d * n + g;
    };
    uint32_t xacc = 0;
    float facc = 0.0f;
    const bool out_even = (reinterpret_cast<uintptr_t>(out_) & 7) == 0;
    auto put = [&](uint64_t d, uint32_t v) {
        const uint32_t bits = OUT == OUT_U32 ? v : __float_as_uint(u32_to_unit(v));
        if (LAYOUT == RNG_XOR_REDUCE) xacc ^= bits;
        else if (RNGX_IDX_OK(out_index(d), n * K, kSiteLfib + __LINE__))
            __stcs(static_cast<uint32_t *>(out_) + out_index(d), bits);
    };
    // normal pair t of the words just written at slots pc.. (call index k..)
    auto put_pair = [&](uint32_t pc, uint64_t k, int t) {
        if (!RNGX_IDX_OK(pc + 2 * t + 1, F::kBuf, kSiteLfib + __LINE__) ||
            (LAYOUT != RNG_XOR_REDUCE && !RNGX_IDX_OK(out_index(k + 2 * t + 1), n * K, kSiteLfib + __LINE__)))
            return;
        const uint2 pr = *reinterpret_cast<const uint2 *>(ring + pc + 2 * t);
        float z0, z1;
        box_muller(pr.x, pr.y, z0, z1, bt);
        if (LAYOUT == RNG_XOR_REDUCE) {
            facc += z0;
            facc += z1;
        } else if (LAYOUT == RNG_INSTANCE_MAJOR && out_even) {
            __stcs(reinterpret_cast<float2 *>(static_cast<float *>(out_) + out_index(k + 2 * t)), make_float2(z0, z1));
        } else {
            float *out = static_cast<float *>(out_);
            __stcs(out + out_index(k + 2 * t), z0);
            __stcs(out + out_index(k + 2 * t + 1), z1);
        }
    };

    uint32_t pc = static_cast<uint32_t>(p.pos & MASK);  // slot of the next word, a multiple of 32
    uint64_t k = 0;
    while (k < K) {
        if ((pc & (G - 1)) == 0 && K - k >= static_cast<uint64_t>(G)) {
            const uint32_t *ra = ring + ((pc + RS - R) & MASK) + lane;
            const uint32_t *rb = ring + ((pc + RS - S) & MASK) + lane;
            // warp-uniform checks (the last lane's words): the whole warp leaves
            // the loop together, before its next warp sync
            if (!RNGX_IDX_OK(((pc + RS - R) & MASK) + 31 + 32 * (U - 1), F::kBuf, kSiteLfib + __LINE__) ||
                !RNGX_IDX_OK(((pc + RS - S) & MASK) + 31 + 32 * (U - 1), F::kBuf, kSiteLfib + __LINE__) ||
                !RNGX_IDX_OK(pc + 31 + 32 * (U - 1) + (pc == 0 ? RS : 0), F::kBuf, kSiteLfib + __LINE__))
                break;
            uint32_t v[U];
#pragma unroll
            for (int u = 0; u < U; u++) v[u] = ra[32 * u] + rb[32 * u];
            uint32_t *rc = ring + pc + lane;
#pragma unroll
            for (int u = 0; u < U; u++) rc[32 * u] = v[u];
            if (pc == 0) {
#pragma unroll
                for (int u = 0; u < U; u++) rc[RS + 32 * u] = v[u];
            }
            if (OUT != OUT_NORMAL) {
#pragma unroll
                for (int u = 0; u < U; u++) put(k + 32 * u + lane, v[u]);
            }
            __syncwarp();
            if (OUT == OUT_NORMAL) {
#pragma unroll
                for (int u = 0; u < U / 2; u++) put_pair(pc, k, 32 * u + lane);
            }
            pc = (pc + G) & MASK;
            k += G;
        } else {  // one chunk: aligning the slot to a group, or the tail
            const int cnt = K - k < 32 ? static_cast<int>(K - k) : 32;
            if (!RNGX_IDX_OK(pc + 31 + (pc < G ? RS : 0), F::kBuf, kSiteLfib + __LINE__)) break;
            const uint32_t v = ring[((pc + RS - R) & MASK) + lane] + ring[((pc + RS - S) & MASK) + lane];
            if (lane < cnt) {
                ring[pc + lane] = v;
                if (pc < G) ring[RS + pc + lane] = v;
                if (OUT != OUT_NORMAL) put(k + lane, v);
            }
            __syncwarp();
            if (OUT == OUT_NORMAL && 2 * lane < cnt) put_pair(pc, k, lane);  // cnt is even for normals
            pc = (pc + 32) & MASK;
            k += cnt;
        }
    }
    __syncwarp();
    if (LAYOUT == RNG_XOR_REDUCE) {
        if (OUT == OUT_NORMAL) {
            for (int o = 16; o > 0; o >>= 1) facc += __shfl_down_sync(0xffffffffu, facc, o);
            if (lane == 0) static_cast<float *>(out_)[g] = facc;
        } else {
            for (int o = 16; o > 0; o >>= 1) xacc ^= __shfl_down_sync(0xffffffffu, xacc, o);
            if (lane == 0) static_cast<uint32_t *>(out_)[g] = xacc;
        }
    }
    // x_(pos+K-r+t) from ring slot (pos + K - r + t) mod RS to state slot (pos + K + t) mod r
    const uint32_t qK = static_cast<uint32_t>((p.pos + K + RS - R) & MASK);
    const uint32_t srK = static_cast<uint32_t>((p.pos + K) % R);
    for (int t = lane; t < R; t += 32) {
        uint32_t b = srK + t;
        b = b >= R ? b - R : b;
        st[b] = ring[(qK + t) & MASK];
    }
}

template <int OUT, auto KERN>
int launch_lfib_kernel(dim3 grid, int block, cudaStream_t s, const DevParams &p, void *out, uint64_t K)
{
    size_t smem = 0;
    if constexpr (OUT == OUT_NORMAL) {  // the Box-Muller tables
        RNGX_CHECK_CUDA(bm_allow_smem<KERN>());
        smem = kBmSmemBytes;
    }
    KERN<<<grid, block, smem, s>>>(p, out, K);
    RNGX_CHECK_LAUNCH();
    return RNG_OK;
}

template <int R, int S, int OUT>
int launch_out(const GenState &g, void *out, uint64_t K, int layout, cudaStream_t s)
{
    const DevParams p = dev_params(g);
    if ((g.pos & 31) == 0) {
        using F = LfibChunked<R, S>;
        const dim3 grid(static_cast<unsigned>((g.n + F::kWarps - 1) / F::kWarps));
        switch (layout) {
        case RNG_STEP_MAJOR:
            return launch_lfib_kernel<OUT, k_generate_lfib_chunked<R, S, OUT, RNG_STEP_MAJOR>>(grid, F::kBlock, s, p,
                                                                                              out, K);
        case RNG_INSTANCE_MAJOR:
            return launch_lfib_kernel<OUT, k_generate_lfib_chunked<R, S, OUT, RNG_INSTANCE_MAJOR>>(grid, F::kBlock, s,
                                                                                                  p, out, K);
        default:
            return launch_lfib_kernel<OUT, k_generate_lfib_chunked<R, S, OUT, RNG_XOR_REDUCE>>(grid, F::kBlock, s, p,
                                                                                              out, K);
        }
    }
    constexpr int W = Lfib<R, S>::kWarps, B = Lfib<R, S>::kBlock;
    const dim3 grid(static_cast<unsigned>((g.n + W - 1) / W));
    switch (layout) {
    case RNG_STEP_MAJOR: return launch_lfib_kernel<OUT, k_generate_lfib<R, S, OUT, RNG_STEP_MAJOR>>(grid, B, s, p, out, K);
    case RNG_INSTANCE_MAJOR:
        return launch_lfib_kernel<OUT, k_generate_lfib<R, S, OUT, RNG_INSTANCE_MAJOR>>(grid, B, s, p, out, K);
    default: return launch_lfib_kernel<OUT, k_generate_lfib<R, S, OUT, RNG_XOR_REDUCE>>(grid, B, s, p, out, K);
    }
}

template <int R, int S>
int launch_lags(const GenState &g, void *out, uint64_t K, int out_kind, int layout, cudaStream_t s)
{
    switch (out_kind) {
    case OUT_U32: return launch_out<R, S, OUT_U32>(g, out, K, layout, s);
    case OUT_F32: return launch_out<R, S, OUT_F32>(g, out, K, layout, s);
    default: return launch_out<R, S, OUT_NORMAL>(g, out, K, layout, s);
    }
}

}  // namespace

RNGX_BOUNDS_MODULE(lfib)

int launch_generate_lfib(const GenState &g, void *d_out, uint64_t K, int out_kind, int layout, cudaStream_t s)
{
    if (g.kind == RNG_LFIB521) return launch_lags<521, 353>(g, d_out, K, out_kind, layout, s);
    return launch_lags<1279, 861>(g, d_out, K, out_kind, layout, s);
}

int launch_seed_lfib(GenState &g, uint64_t seed, cudaStream_t s)
{
    const DevParams p = dev_params(g);
    const unsigned threads = 256;
    const unsigned blocks = static_cast<unsigned>((g.n * 32 + threads - 1) / threads);
    if (g.kind == RNG_LFIB521) k_seed_lfib<521><<<blocks, threads, 0, s>>>(p, seed, g.first);
    else k_seed_lfib<1279><<<blocks, threads, 0, s>>>(p, seed, g.first);
    RNGX_CHECK_LAUNCH();
    return RNG_OK;
}

}  // namespace rngx
