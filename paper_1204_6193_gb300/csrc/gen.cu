// gen.cu -- generation kernels: every instance emits K draws as u32, exact
// uniform f32 or Box-Muller normals, in step-major, instance-major or
// consume-in-register (XOR / sum) form.  The state is loaded into
// registers once, stepped K times and stored once (the paper's concern
// about state load/store overhead, Sec. 2 and the caption of Table 2).
#include <algorithm>
#include <type_traits>

#include "gen_device.cuh"
#include "modarith.cuh"

namespace rngx {
namespace {

constexpr int kBlock = 256;
constexpr int kWarps = kBlock / 32;

__device__ __forceinline__ void st_stream(uint32_t *p, uint32_t v) { __stcs(p, v); }
__device__ __forceinline__ void st_stream(float *p, float v) { __stcs(p, v); }

// Per-thread generators (LCG32/64, MWC, XORWOW, Philox) and the warp-shared
// 1024-bit generator, whose lanes are instances.  One thread per instance.
template <int KIND, int OUT, int LAYOUT>
__global__ void __launch_bounds__(kBlock) k_generate(DevParams p, void *out_, uint64_t K)
{
    __shared__ uint32_t tile[LAYOUT == RNG_INSTANCE_MAJOR ? kWarps : 1][32][33];
    BmTables bt{};
    if constexpr (OUT == OUT_NORMAL) bt = bm_stage();  // every thread, before any leaves
    const uint64_t n = p.n;
    const uint64_t i = static_cast<uint64_t>(blockIdx.x) * kBlock + threadIdx.x;
    const bool active = i < n;
    // Warps entirely past the end leave; partial warps keep every lane for
    // the warp-level transpose (per-thread kinds only: n % 32 == 0 for XS1024W).
    if ((i & ~static_cast<uint64_t>(31)) >= n) return;
    Gen<KIND> g;
    if (active) g.load(p, i);
    else g.load(p, n - 1);  // dummy state, output discarded

    if constexpr (is_philox(KIND)) {
        // block-aligned calls: one block evaluation yields draws k..k+3
        if (LAYOUT != RNG_INSTANCE_MAJOR && (p.pos & 3) == 0 && (K & 3) == 0) {
            constexpr int RR = Gen<KIND>::kRounds;
            const uint64_t blk0 = p.pos >> 2;
            const PhiloxKeys<RR> keys(g.k0, g.k1);
            uint32_t xacc = 0;
            float facc = 0.0f;
#pragma unroll 2
            for (uint64_t k = 0; k < K; k += 4) {
                const uint64_t blk = blk0 + (k >> 2);
                uint32_t o[4];
                philox_keys<RR>(static_cast<uint32_t>(blk), static_cast<uint32_t>(blk >> 32), 0u, 0u, keys, o[0],
                                o[1], o[2], o[3]);
                if (OUT == OUT_NORMAL) {
                    float z[4];
                    box_muller(o[0], o[1], z[0], z[1], bt);
                    box_muller(o[2], o[3], z[2], z[3], bt);
                    if (LAYOUT == RNG_XOR_REDUCE) {
#pragma unroll
                        for (int j = 0; j < 4; j++) facc += z[j];
                    } else if (active) {
#pragma unroll
                        for (int j = 0; j < 4; j++)
                            if (RNGX_IDX_OK((k + j) * n + i, n * K, kSiteGen + __LINE__))
                                st_stream(static_cast<float *>(out_) + (k + j) * n + i, z[j]);
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < 4; j++) {
                        const uint32_t bits = OUT == OUT_U32 ? o[j] : __float_as_uint(u32_to_unit(o[j]));
                        if (LAYOUT == RNG_XOR_REDUCE) xacc ^= bits;
                        else if (active && RNGX_IDX_OK((k + j) * n + i, n * K, kSiteGen + __LINE__))
                            __stcs(static_cast<uint32_t *>(out_) + (k + j) * n + i, bits);
                    }
                }
            }
            if (LAYOUT == RNG_XOR_REDUCE && active) {
                if (OUT == OUT_NORMAL) static_cast<float *>(out_)[i] = facc;
                else static_cast<uint32_t *>(out_)[i] = xacc;
            }
            return;  // Philox keeps no state beyond the handle's position
        }
    }

    if (LAYOUT == RNG_STEP_MAJOR) {
        if (OUT == OUT_NORMAL) {
            float *out = static_cast<float *>(out_);
#pragma unroll 2
            for (uint64_t k = 0; k < K; k += 2) {
                const uint32_t r0 = g.next(), r1 = g.next();
                float z0, z1;
                box_muller(r0, r1, z0, z1, bt);
                if (active && RNGX_IDX_OK((k + 1) * n + i, n * K, kSiteGen + __LINE__)) {
                    st_stream(out + k * n + i, z0);
                    st_stream(out + (k + 1) * n + i, z1);
                }
            }
        } else {
            for (uint64_t k = 0; k < K; k++) {
                const uint32_t r = g.next();
                if (!active || !RNGX_IDX_OK(k * n + i, n * K, kSiteGen + __LINE__)) continue;
                if (OUT == OUT_U32) st_stream(static_cast<uint32_t *>(out_) + k * n + i, r);
                else st_stream(static_cast<float *>(out_) + k * n + i, u32_to_unit(r));
            }
        }
    } else if (LAYOUT == RNG_INSTANCE_MAJOR) {
        // 32 instances x 32 draws per warp staged in shared memory, so that
        // every store instruction writes 128 contiguous bytes of one row.
        const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
        const uint64_t i0 = i - lane;
        for (uint64_t k0 = 0; k0 < K; k0 += 32) {
            const int cnt = static_cast<int>(K - k0 < 32 ? K - k0 : 32);
            if (OUT == OUT_NORMAL) {
                for (int j = 0; j < cnt; j += 2) {
                    const uint32_t r0 = g.next(), r1 = g.next();
                    float z0, z1;
                    box_muller(r0, r1, z0, z1, bt);
                    tile[w][lane][j] = __float_as_uint(z0);
                    tile[w][lane][j + 1] = __float_as_uint(z1);
                }
            } else {
                for (int j = 0; j < cnt; j++) {
                    const uint32_t r = g.next();
                    tile[w][lane][j] = OUT == OUT_U32 ? r : __float_as_uint(u32_to_unit(r));
                }
            }
            __syncwarp();
            if (lane < cnt) {
                uint32_t *out = static_cast<uint32_t *>(out_);
                for (int r = 0; r < 32; r++)
                    if (i0 + r < n && RNGX_IDX_OK((i0 + r) * K + k0 + lane, n * K, kSiteGen + __LINE__))
                        __stcs(out + (i0 + r) * K + k0 + lane, tile[w][r][lane]);
            }
            __syncwarp();
        }
    } else {  // RNG_XOR_REDUCE: consume in registers
        if (OUT == OUT_NORMAL) {
            float acc = 0.0f;
            for (uint64_t k = 0; k < K; k += 2) {
                const uint32_t r0 = g.next(), r1 = g.next();
                float z0, z1;
                box_muller(r0, r1, z0, z1, bt);
                acc += z0;
                acc += z1;
            }
            if (active) static_cast<float *>(out_)[i] = acc;
        } else {
            uint32_t acc = 0;
            for (uint64_t k = 0; k < K; k++) {
                const uint32_t r = g.next();
                acc ^= OUT == OUT_U32 ? r : __float_as_uint(u32_to_unit(r));
            }
            if (active) static_cast<uint32_t *>(out_)[i] = acc;
        }
    }
    if (active) g.store(p, i);
}

// ------------------------------------------------- long streams, few instances
// Step-major output of a handle with too few instances to fill the GPU:
// each instance's K draws are cut into ranges of Kc (a multiple of 4), one
// thread per (instance, range).  Thread (i, c) jumps its copy of instance
// i's state over c Kc draws -- Eq. (2) for the LCGs, v a^t mod (a 2^32 - 1)
// for MWC, the counter for Philox -- and makes draws [c Kc, min(K, (c+1)
// Kc)); the last range stores the state.  The draws are those of the
// one-thread-per-instance kernel.
template <int KIND>
__device__ __forceinline__ void jump_draws(Gen<KIND> &g, const DevParams &p, uint64_t t)
{
    if constexpr (KIND == RNG_LCG32 || KIND == RNG_LCG64) {
        uint64_t at, ct;
        affine_pow(p.A, p.C, t, at, ct);
        if constexpr (KIND == RNG_LCG32) g.x = static_cast<uint32_t>(at) * g.x + static_cast<uint32_t>(ct);
        else g.x = at * g.x + ct;
    } else if constexpr (KIND == RNG_MWC) {
        const uint64_t mod = (static_cast<uint64_t>(g.a) << 32) - 1;
        const Mont m = mont_setup(mod);
        g.v = from_mont(mont_mul(to_mont(g.v, m), mont_pow(to_mont(g.a, m), t, m), m), m);
    } else {
        g.pos += t;  // Philox: the counter
    }
}

template <int KIND, int OUT>
__global__ void __launch_bounds__(kBlock) k_generate_split(DevParams p, void *out_, uint64_t K, uint64_t Kc)
{
    BmTables bt{};
    if constexpr (OUT == OUT_NORMAL) bt = bm_stage();  // every thread, before any leaves
    const uint64_t n = p.n;
    const uint64_t i = static_cast<uint64_t>(blockIdx.x) * kBlock + threadIdx.x;
    if (i >= n) return;
    const uint64_t k0 = blockIdx.y * Kc, k1 = k0 + Kc < K ? k0 + Kc : K;
    Gen<KIND> g;
    g.load(p, i);
    jump_draws<KIND>(g, p, k0);
    if constexpr (is_philox(KIND)) {
        if ((g.pos & 3) == 0) {  // whole counter blocks: the round keys once
            constexpr int RR = Gen<KIND>::kRounds;
            const PhiloxKeys<RR> keys(g.k0, g.k1);
            for (uint64_t k = k0; k < k1; k += 4) {
                const uint64_t blk = (g.pos + (k - k0)) >> 2;
                uint32_t o[4];
                philox_keys<RR>(static_cast<uint32_t>(blk), static_cast<uint32_t>(blk >> 32), 0u, 0u, keys, o[0],
                                o[1], o[2], o[3]);
                if (OUT == OUT_NORMAL) {
                    float z[4];
                    box_muller(o[0], o[1], z[0], z[1], bt);
                    box_muller(o[2], o[3], z[2], z[3], bt);
#pragma unroll
                    for (int j = 0; j < 4; j++)
                        if (k + j < k1 && RNGX_IDX_OK((k + j) * n + i, n * K, kSiteGen + __LINE__))
                            st_stream(static_cast<float *>(out_) + (k + j) * n + i, z[j]);
                } else {
#pragma unroll
                    for (int j = 0; j < 4; j++) {
                        const uint32_t bits = OUT == OUT_U32 ? o[j] : __float_as_uint(u32_to_unit(o[j]));
                        if (k + j < k1 && RNGX_IDX_OK((k + j) * n + i, n * K, kSiteGen + __LINE__))
                            __stcs(static_cast<uint32_t *>(out_) + (k + j) * n + i, bits);
                    }
                }
            }
            return;  // Philox keeps no state beyond the handle's position
        }
    }
    if (OUT == OUT_NORMAL) {
        float *out = static_cast<float *>(out_);
        for (uint64_t k = k0; k < k1; k += 2) {  // k0 and K are even
            const uint32_t r0 = g.next(), r1 = g.next();
            float z0, z1;
            box_muller(r0, r1, z0, z1, bt);
            if (RNGX_IDX_OK((k + 1) * n + i, n * K, kSiteGen + __LINE__)) {
                st_stream(out + k * n + i, z0);
                st_stream(out + (k + 1) * n + i, z1);
            }
        }
    } else {
        for (uint64_t k = k0; k < k1; k++) {
            const uint32_t r = g.next();
            if (!RNGX_IDX_OK(k * n + i, n * K, kSiteGen + __LINE__)) continue;
            if (OUT == OUT_U32) st_stream(static_cast<uint32_t *>(out_) + k * n + i, r);
            else st_stream(static_cast<float *>(out_) + k * n + i, u32_to_unit(r));
        }
    }
    if (k1 == K) g.store(p, i);
}

// ------------------------------------------------------------- MT19937
// One generator per warp (Sec. 5: one state shared by the threads that
// refill it).  The warp keeps the 624-word state in registers: lane l holds
// word 32j + l in x[j] (j < 20; x[19] only in lanes 0..15).  A refill is 20
// chunks of 32 words, chunk j making words 32j .. 32j+31 at once.  In the
// sequential recurrence word i reads word i+1 (not yet rewritten; for i =
// 623 the new word 0) and word i+397 mod 624, which for i < 227 is not yet
// rewritten and for i >= 227 is the new word i-227, made in an earlier
// chunk.  Both come by one warp shuffle each: the sending lane picks the
// register the receiving lane needs (the two receivers of a sender never
// need different registers, except in the chunk that crosses i = 227).
// Uniform outputs are tempered and stored as they are made; normals stage
// the tempered words of a block in shared memory and pair them from there.
constexpr int kMtWarps = 8;
constexpr int kMtBlock = 32 * kMtWarps;
constexpr int kMtRegs = (MT_N + 31) / 32;  // 20

// Powers of two for the left shifts of the tempering, read from constant
// memory so that the compiler keeps them as integer multiplies (y << b = y
// 2^b), which issue to the FMA pipe: the refill and the tempering are
// otherwise all shifts and logic operations on the ALU pipe, which they
// saturate.  (Right shifts as high words of products measured slower.)
__constant__ uint32_t c_mt_pow2[2] = {1u << 7, 1u << 15};

__device__ __forceinline__ uint32_t mt_mix(uint32_t cur, uint32_t nxt, uint32_t far)
{
    const uint32_t y = (cur & 0x80000000u) | (nxt & 0x7fffffffu);
    return far ^ (y >> 1) ^ ((nxt & 1u) * 0x9908B0DFu);  // far ^ (y >> 1) ^ mag01[y & 1]
}

// MT19937 tempering (the left shifts as multiplies, see above).
__device__ __forceinline__ uint32_t mt_temper_mul(uint32_t y)
{
    y ^= y >> 11;
    y ^= (y * c_mt_pow2[0]) & 0x9D2C5680u;  // (y << 7) & b
    y ^= (y * c_mt_pow2[1]) & 0xEFC60000u;  // (y << 15) & c
    y ^= y >> 18;
    return y;
}

// One refill of the register-resident state (all 32 lanes call it).
__device__ __forceinline__ void mt_twist_regs(uint32_t (&x)[kMtRegs], int lane)
{
    constexpr unsigned FULL = 0xffffffffu;
#pragma unroll
    for (int j = 0; j < kMtRegs; j++) {
        // word i + 1: lane l + 1 of the same register; lane 31 takes lane 0's
        // next register; word 623 (lane 15 of x[19]) the new word 0
        uint32_t nxt;
        if (j < kMtRegs - 1) nxt = __shfl_sync(FULL, lane == 0 ? x[j + 1] : x[j], (lane + 1) & 31);
        else nxt = __shfl_sync(FULL, lane == 0 ? x[0] : x[j], lane == 15 ? 0 : (lane + 1) & 31);
        // word i + 397 = 32(j + 12) + l + 13 (old), or the new word i - 227 =
        // 32(j - 8) + l + 29
        uint32_t far;
        if (j < 7) {
            far = __shfl_sync(FULL, lane >= 13 ? x[j + 12] : x[j + 13], (lane + 13) & 31);
        } else if (j == 7) {
            const uint32_t fo = __shfl_sync(FULL, x[19], (lane + 13) & 31);  // i = 224..226: words 621..623
            const uint32_t fn = __shfl_sync(FULL, x[0], (lane + 29) & 31);   // i >= 227: new words 0..28
            far = lane < 3 ? fo : fn;
        } else {
            far = __shfl_sync(FULL, lane >= 29 ? x[j - 8] : x[j - 7], (lane + 29) & 31);
        }
        x[j] = mt_mix(x[j], nxt, far);
    }
}

template <int OUT, int LAYOUT>
__global__ void __launch_bounds__(kMtBlock) k_generate_mt(DevParams p, void *out_, uint64_t K)
{
    // normals: tempered words, pair-aligned (rows of a multiple of 4 words,
    // so that every row starts on a 16-byte boundary)
    __shared__ __align__(16) uint32_t tb_s[OUT == OUT_NORMAL ? kMtWarps : 1][MT_N + 4];
    BmTables bt{};
    if constexpr (OUT == OUT_NORMAL) bt = bm_stage();  // every thread, before any leaves
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint64_t gidx = static_cast<uint64_t>(blockIdx.x) * kMtWarps + w;
    const uint64_t n = p.n;
    if (gidx >= n) return;  // whole warps only: no block-wide barriers below
    uint32_t *st = static_cast<uint32_t *>(p.s[0]) + gidx * MT_N;
    const uint64_t n_out = LAYOUT == RNG_XOR_REDUCE ? n : n * K;  // words of the output
    uint32_t x[kMtRegs];
#pragma unroll
    for (int j = 0; j < kMtRegs - 1; j++) x[j] = st[32 * j + lane];
    x[kMtRegs - 1] = lane < MT_N - 32 * (kMtRegs - 1) ? st[32 * (kMtRegs - 1) + lane] : 0u;
    // words of the current block already consumed (MT_N: refill first)
    const int mti = p.pos == 0 ? MT_N : static_cast<int>((p.pos - 1) % MT_N) + 1;

    auto out_index = [&](uint64_t d) -> uint64_t {
        return LAYOUT == RNG_INSTANCE_MAJOR ? gidx * K + d : d * n + gidx;
    };
    uint32_t xacc = 0;
    float facc = 0.0f;
    uint32_t *tb = tb_s[OUT == OUT_NORMAL ? w : 0];
    uint32_t pending = 0;  // normals: tempered word waiting for its partner (odd call index)
    const bool out_even = (reinterpret_cast<uintptr_t>(out_) & 7) == 0;
    const bool out_quad = (reinterpret_cast<uintptr_t>(out_) & 15) == 0 && (K & 3) == 0;

    // Hands the words lo .. hi-1 of the state (call index kb for word lo) to
    // the output.  FULL: the whole block (lo = 0, hi = MT_N).
    auto emit = [&](auto full, int lo, int hi, uint64_t kb) {
        constexpr bool FULLB = decltype(full)::value;
        if (OUT != OUT_NORMAL) {
#pragma unroll
            for (int j = 0; j < kMtRegs; j++) {
                const int wd = 32 * j + lane;
                const bool in = FULLB ? (j < kMtRegs - 1 || wd < MT_N) : (wd >= lo && wd < hi);
                if (in) {
                    const uint32_t r = mt_temper_mul(x[j]);
                    const uint32_t bits = OUT == OUT_U32 ? r : __float_as_uint(u32_to_unit(r));
                    if (LAYOUT == RNG_XOR_REDUCE) xacc ^= bits;
                    else if (RNGX_IDX_OK(out_index(kb + (wd - lo)), n_out, kSiteGen + __LINE__))
                        __stcs(static_cast<uint32_t *>(out_) + out_index(kb + (wd - lo)), bits);
                }
            }
        } else {
            if constexpr (FULLB && LAYOUT == RNG_INSTANCE_MAJOR) {
                if (out_quad && (kb & 3) == 0) {
                    // a whole block at a 16-byte aligned place of the row:
                    // lane l takes words 4q .. 4q+3 (q = l + 32 i) in one
                    // 16-byte read, makes their two pairs and writes the four
                    // normals with one 16-byte store; no word is left over
#pragma unroll
                    for (int j = 0; j < kMtRegs; j++)
                        if (j < kMtRegs - 1 || 32 * j + lane < MT_N) tb[32 * j + lane] = mt_temper_mul(x[j]);
                    __syncwarp();
                    const uint4 *tq = reinterpret_cast<const uint4 *>(tb);
                    float4 *oq = reinterpret_cast<float4 *>(static_cast<float *>(out_) + gidx * K + kb);
#pragma unroll
                    for (int i = 0; i < (MT_N / 4 + 31) / 32; i++) {
                        const int q = lane + 32 * i;
                        if (q < MT_N / 4 && RNGX_IDX_OK(gidx * K + kb + 4 * q + 3, n_out, kSiteGen + __LINE__)) {
                            const uint4 w = tq[q];
                            float4 z;
                            box_muller(w.x, w.y, z.x, z.y, bt);
                            box_muller(w.z, w.w, z.z, z.w, bt);
                            __stcs(oq + q, z);
                        }
                    }
                    __syncwarp();
                    return;
                }
            }
            // pairs start at even call indices: an odd kb continues the pending word
            const int off = static_cast<int>(kb & 1);
            if (off && lane == 0) tb[0] = pending;
#pragma unroll
            for (int j = 0; j < kMtRegs; j++) {
                const int wd = 32 * j + lane;
                const bool in = FULLB ? (j < kMtRegs - 1 || wd < MT_N) : (wd >= lo && wd < hi);
                if (in && RNGX_IDX_OK(off + wd - lo, MT_N + 2, kSiteGen + __LINE__)) tb[off + wd - lo] = mt_temper_mul(x[j]);
            }
            __syncwarp();
            const int avail = off + hi - lo;
            const uint64_t d0 = kb - off;  // call index of tb[0]
            for (int t = lane; t < avail / 2; t += 32) {
                const uint2 pr = reinterpret_cast<const uint2 *>(tb)[t];
                float z0, z1;
                box_muller(pr.x, pr.y, z0, z1, bt);
                if (LAYOUT == RNG_XOR_REDUCE) {
                    facc += z0;
                    facc += z1;
                } else if (!RNGX_IDX_OK(out_index(d0 + 2 * t + 1), n_out, kSiteGen + __LINE__) ||
                           !RNGX_IDX_OK(out_index(d0 + 2 * t), n_out, kSiteGen + __LINE__)) {
                } else if (LAYOUT == RNG_INSTANCE_MAJOR && out_even) {
                    // gidx K + d0 + 2t is even (K and d0 even): one 8-byte store
                    __stcs(reinterpret_cast<float2 *>(static_cast<float *>(out_) + out_index(d0 + 2 * t)),
                           make_float2(z0, z1));
                } else {
                    float *out = static_cast<float *>(out_);
                    __stcs(out + out_index(d0 + 2 * t), z0);
                    __stcs(out + out_index(d0 + 2 * t + 1), z1);
                }
            }
            if (avail & 1) pending = tb[avail - 1];  // the same value in every lane
            __syncwarp();
        }
    };

    uint64_t k = 0;
    bool twisted = false;
    if (K > 0 && mti < MT_N) {  // the rest of the current block
        const int cnt = K < static_cast<uint64_t>(MT_N - mti) ? static_cast<int>(K) : MT_N - mti;
        emit(std::false_type{}, mti, mti + cnt, 0);
        k = cnt;
    }
#pragma unroll 1
    while (K - k >= static_cast<uint64_t>(MT_N)) {
        mt_twist_regs(x, lane);
        twisted = true;
        emit(std::true_type{}, 0, MT_N, k);
        k += MT_N;
    }
    if (k < K) {
        mt_twist_regs(x, lane);
        twisted = true;
        emit(std::false_type{}, 0, static_cast<int>(K - k), k);
    }
    if (LAYOUT == RNG_XOR_REDUCE) {
        if (OUT == OUT_NORMAL) {
            for (int o = 16; o > 0; o >>= 1) facc += __shfl_down_sync(0xffffffffu, facc, o);
            if (lane == 0) static_cast<float *>(out_)[gidx] = facc;
        } else {
            for (int o = 16; o > 0; o >>= 1) xacc ^= __shfl_down_sync(0xffffffffu, xacc, o);
            if (lane == 0) static_cast<uint32_t *>(out_)[gidx] = xacc;
        }
    }
    if (twisted) {
#pragma unroll
        for (int j = 0; j < kMtRegs - 1; j++) st[32 * j + lane] = x[j];
        if (lane < MT_N - 32 * (kMtRegs - 1)) st[32 * (kMtRegs - 1) + lane] = x[kMtRegs - 1];
    }
}

// ------------------------------------------- the 1024-bit generator, by thread
// For step-major and consume-in-register output one thread holds a whole
// 1024-bit state (its 32 lanes' words) in registers and applies the three
// shifts with funnel shifts: identical draws to the warp-shuffle form, at
// about seven instructions per output instead of six shuffles and a dozen
// selects per lane.  Step-major output is then 32 consecutive words per
// thread and step (eight 16-byte stores).
constexpr int kXsBlock = 64;

// Writes the 32 x 32 words a warp produced for one step (lane o holds the
// words of state j0 + o) as 4 KiB of contiguous output: staged through
// shared memory so that each 16-byte store instruction covers 512
// consecutive bytes.
__device__ __forceinline__ void xs_store_step(uint32_t (*tile)[33], const uint32_t (&v)[32], uint32_t *row,
                                              uint64_t j0, uint64_t nstates, int lane, const uint32_t *row_base,
                                              uint64_t row_len)
{
#pragma unroll
    for (int l = 0; l < 32; l++) tile[lane][l] = v[l];
    __syncwarp();
#pragma unroll
    for (int m = 0; m < 8; m++) {
        const int c = m * 32 + lane;  // 16-byte chunk of the warp's 4 KiB
        const int o = c >> 3, wo = (c & 7) * 4;
        if (j0 + o < nstates && RNGX_IDX_OK(static_cast<uint64_t>(row + 32 * j0 + 4 * c + 3 - row_base), row_len, kSiteGen + __LINE__))
            __stcs(reinterpret_cast<uint4 *>(row + 32 * j0) + c,
                   make_uint4(tile[o][wo], tile[o][wo + 1], tile[o][wo + 2], tile[o][wo + 3]));
    }
    __syncwarp();
}

template <int OUT, int LAYOUT>
__global__ void __launch_bounds__(kXsBlock) k_generate_xs_reg(DevParams p, void *out_, uint64_t K)
{
    __shared__ uint32_t tile_s[kXsBlock / 32][32][33];
    BmTables bt{};
    if constexpr (OUT == OUT_NORMAL) bt = bm_stage();  // every thread, before any leaves
    const uint64_t n = p.n, nstates = n / 32;
    const uint64_t j = static_cast<uint64_t>(blockIdx.x) * kXsBlock + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const uint64_t j0 = j - lane;
    if (j0 >= nstates) return;  // whole warps leave together
    const bool active = j < nstates;
    uint32_t(*tile)[33] = tile_s[threadIdx.x >> 5];
    uint32_t *state = static_cast<uint32_t *>(p.s[0]) + 32 * (active ? j : j0);
    uint32_t x[32];
#pragma unroll
    for (int m = 0; m < 8; m++) {
        const uint4 v = reinterpret_cast<const uint4 *>(state)[m];
        x[4 * m] = v.x;
        x[4 * m + 1] = v.y;
        x[4 * m + 2] = v.z;
        x[4 * m + 3] = v.w;
    }
    uint64_t step = p.pos;
    auto shift_step = [&]() {
#pragma unroll
        for (int i = 0; i <= 21; i++)  // X ^= X << 329: words i+10, i+11 (zero past the end)
            x[i] ^= __funnelshift_l(i + 11 < 32 ? x[i + 11 < 32 ? i + 11 : 31] : 0u, x[i + 10], 9);
#pragma unroll
        for (int i = 31; i >= 10; i--)  // X ^= X >> 347: words i-10, i-11 (zero before the start)
            x[i] ^= __funnelshift_r(x[i - 10], i - 11 >= 0 ? x[i - 11 >= 0 ? i - 11 : 0] : 0u, 27);
#pragma unroll
        for (int i = 0; i <= 21; i++)  // X ^= X << 344
            x[i] ^= __funnelshift_l(i + 11 < 32 ? x[i + 11 < 32 ? i + 11 : 31] : 0u, x[i + 10], 24);
    };
    auto weyl = [&]() -> uint32_t {
        step++;
        const uint32_t y = static_cast<uint32_t>(step) * 362437u;
        return y ^ (y >> 16);
    };
    if (LAYOUT == RNG_XOR_REDUCE) {
        uint32_t acc[32];
        float facc[32];
#pragma unroll
        for (int l = 0; l < 32; l++) {
            acc[l] = 0;
            facc[l] = 0.0f;
        }
        if (OUT == OUT_NORMAL) {
            for (uint64_t k = 0; k < K; k += 2) {
                shift_step();
                const uint32_t y0 = weyl();
                uint32_t a[32];
#pragma unroll
                for (int l = 0; l < 32; l++) a[l] = x[l] + y0;
                shift_step();
                const uint32_t y1 = weyl();
#pragma unroll
                for (int l = 0; l < 32; l++) {
                    float z0, z1;
                    box_muller(a[l], x[l] + y1, z0, z1, bt);
                    facc[l] += z0;
                    facc[l] += z1;
                }
            }
        } else {
            for (uint64_t k = 0; k < K; k++) {
                shift_step();
                const uint32_t yy = weyl();
#pragma unroll
                for (int l = 0; l < 32; l++) {
                    const uint32_t r = x[l] + yy;
                    acc[l] ^= OUT == OUT_U32 ? r : __float_as_uint(u32_to_unit(r));
                }
            }
        }
        if (active && RNGX_IDX_OK(32 * j + 31, n, kSiteGen + __LINE__)) {
            uint4 *dst = reinterpret_cast<uint4 *>(static_cast<uint32_t *>(out_) + 32 * j);
#pragma unroll
            for (int m = 0; m < 8; m++) {
                uint4 v;
                if (OUT == OUT_NORMAL) {
                    v = make_uint4(__float_as_uint(facc[4 * m]), __float_as_uint(facc[4 * m + 1]),
                                   __float_as_uint(facc[4 * m + 2]), __float_as_uint(facc[4 * m + 3]));
                } else {
                    v = make_uint4(acc[4 * m], acc[4 * m + 1], acc[4 * m + 2], acc[4 * m + 3]);
                }
                dst[m] = v;
            }
        }
    } else {  // RNG_STEP_MAJOR
        uint32_t *out = static_cast<uint32_t *>(out_);
        if (OUT == OUT_NORMAL) {
            for (uint64_t k = 0; k < K; k += 2) {
                shift_step();
                const uint32_t y0 = weyl();
                uint32_t a[32];
#pragma unroll
                for (int l = 0; l < 32; l++) a[l] = x[l] + y0;
                shift_step();
                const uint32_t y1 = weyl();
                uint32_t z1b[32];
#pragma unroll
                for (int l = 0; l < 32; l++) {
                    float z0, z1;
                    box_muller(a[l], x[l] + y1, z0, z1, bt);
                    a[l] = __float_as_uint(z0);
                    z1b[l] = __float_as_uint(z1);
                }
                xs_store_step(tile, a, out + k * n, j0, nstates, lane, out, n * K);
                xs_store_step(tile, z1b, out + (k + 1) * n, j0, nstates, lane, out, n * K);
            }
        } else {
            for (uint64_t k = 0; k < K; k++) {
                shift_step();
                const uint32_t yy = weyl();
                uint32_t v[32];
#pragma unroll
                for (int l = 0; l < 32; l++) {
                    const uint32_t r = x[l] + yy;
                    v[l] = OUT == OUT_U32 ? r : __float_as_uint(u32_to_unit(r));
                }
                xs_store_step(tile, v, out + k * n, j0, nstates, lane, out, n * K);
            }
        }
    }
    if (active) {
#pragma unroll
        for (int m = 0; m < 8; m++)
            reinterpret_cast<uint4 *>(state)[m] = make_uint4(x[4 * m], x[4 * m + 1], x[4 * m + 2], x[4 * m + 3]);
    }
}

// Normals of the 1024-bit generator take the one-thread-per-state form only
// when there are states enough for about 200 per SM (6 warps): each thread
// then has 32 independent Box-Muller pairs per two steps, which costs less
// than the six shuffles per word of the lane-per-instance form; with fewer
// threads that form's parallelism wins (measured on GB300: 2^20 instances,
// 1.66 against 1.83 ms per 2^30 normals; 2^18 instances, 4.8 against 1.8
// ms per 2^30).
inline bool xs_reg_normals(uint64_t n)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return false;
    return n / 32 >= 200ull * static_cast<uint64_t>(sms);
}

// SMs of the current device (0 if unknown).
inline int device_sms()
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 0;
    return sms;
}

// Whether a step-major call of n instances x K draws takes the split form,
// and its range length Kc: when the instances fill less than a quarter of
// the device's thread slots (2048 per SM) and each range keeps at least 256
// draws, the ranges bring the threads up to about the device's slots.
inline bool split_draws(uint64_t n, uint64_t K, uint64_t *Kc)
{
    const uint64_t slots = static_cast<uint64_t>(device_sms()) * 2048;
    if (slots == 0 || 4 * n >= slots || K < 512) return false;
    uint64_t ranges = (slots + n - 1) / n;
    ranges = ranges < K / 256 ? ranges : K / 256;
    if (ranges < 2) return false;
    uint64_t kc = (K + ranges - 1) / ranges;
    kc = (kc + 3) & ~3ull;  // whole Philox blocks and normal pairs
    if (kc >= K) return false;
    *Kc = kc;
    return true;
}

// The one-thread-per-state form of the 1024-bit generator needs states
// enough to occupy the device (one thread each): at least 16 per SM.
inline bool xs_reg_uniform(uint64_t n) { return n / 32 >= 16ull * static_cast<uint64_t>(device_sms()); }

// Launches KERN with the Box-Muller tables' dynamic shared memory when it
// makes normals.
template <int OUT, auto KERN>
int launch_gen(dim3 grid, int block, cudaStream_t s, const DevParams &p, void *out, uint64_t K)
{
    size_t smem = 0;
    if constexpr (OUT == OUT_NORMAL) {
        RNGX_CHECK_CUDA(bm_allow_smem<KERN>());
        smem = kBmSmemBytes;
    }
    KERN<<<grid, block, smem, s>>>(p, out, K);
    RNGX_CHECK_LAUNCH();
    return RNG_OK;
}

template <int KIND, int OUT>
int launch_kind_out(const GenState &g, void *out, uint64_t K, int layout, cudaStream_t s)
{
    const DevParams p = dev_params(g);
    if constexpr (KIND == RNG_MT19937_SHARED) {
        const dim3 grid(static_cast<unsigned>((g.n + kMtWarps - 1) / kMtWarps));
        switch (layout) {
        case RNG_STEP_MAJOR: return launch_gen<OUT, k_generate_mt<OUT, RNG_STEP_MAJOR>>(grid, kMtBlock, s, p, out, K);
        case RNG_INSTANCE_MAJOR:
            return launch_gen<OUT, k_generate_mt<OUT, RNG_INSTANCE_MAJOR>>(grid, kMtBlock, s, p, out, K);
        default: return launch_gen<OUT, k_generate_mt<OUT, RNG_XOR_REDUCE>>(grid, kMtBlock, s, p, out, K);
        }
    } else if (KIND == RNG_XS1024W && layout != RNG_INSTANCE_MAJOR &&
               (reinterpret_cast<uintptr_t>(out) & 15) == 0 &&
               (OUT != OUT_NORMAL ? xs_reg_uniform(g.n) : xs_reg_normals(g.n))) {
        const dim3 grid(static_cast<unsigned>((g.n / 32 + kXsBlock - 1) / kXsBlock));
        if (layout == RNG_STEP_MAJOR)
            return launch_gen<OUT, k_generate_xs_reg<OUT, RNG_STEP_MAJOR>>(grid, kXsBlock, s, p, out, K);
        return launch_gen<OUT, k_generate_xs_reg<OUT, RNG_XOR_REDUCE>>(grid, kXsBlock, s, p, out, K);
    } else {
        if constexpr (KIND == RNG_LCG32 || KIND == RNG_LCG64 || KIND == RNG_MWC || is_philox(KIND)) {
            uint64_t Kc = 0;
            if (layout == RNG_STEP_MAJOR && split_draws(g.n, K, &Kc)) {
                const dim3 grid(static_cast<unsigned>((g.n + kBlock - 1) / kBlock),
                                static_cast<unsigned>((K + Kc - 1) / Kc));
                size_t smem = 0;
                if constexpr (OUT == OUT_NORMAL) {
                    RNGX_CHECK_CUDA((bm_allow_smem<k_generate_split<KIND, OUT>>()));
                    smem = kBmSmemBytes;
                }
                k_generate_split<KIND, OUT><<<grid, kBlock, smem, s>>>(p, out, K, Kc);
                RNGX_CHECK_LAUNCH();
                return RNG_OK;
            }
        }
        const dim3 grid(static_cast<unsigned>((g.n + kBlock - 1) / kBlock));
        switch (layout) {
        case RNG_STEP_MAJOR: return launch_gen<OUT, k_generate<KIND, OUT, RNG_STEP_MAJOR>>(grid, kBlock, s, p, out, K);
        case RNG_INSTANCE_MAJOR:
            return launch_gen<OUT, k_generate<KIND, OUT, RNG_INSTANCE_MAJOR>>(grid, kBlock, s, p, out, K);
        default: return launch_gen<OUT, k_generate<KIND, OUT, RNG_XOR_REDUCE>>(grid, kBlock, s, p, out, K);
        }
    }
}

template <int KIND>
int launch_kind(const GenState &g, void *out, uint64_t K, int out_kind, int layout, cudaStream_t s)
{
    switch (out_kind) {
    case OUT_U32: return launch_kind_out<KIND, OUT_U32>(g, out, K, layout, s);
    case OUT_F32: return launch_kind_out<KIND, OUT_F32>(g, out, K, layout, s);
    default: return launch_kind_out<KIND, OUT_NORMAL>(g, out, K, layout, s);
    }
}

}  // namespace

namespace {
// Word pairs -> normal pairs, 16-byte loads and stores for four words.
__global__ void k_u32_to_normal(const uint32_t *in, float *out, uint64_t n_pairs)
{
    const BmTables bt = bm_stage();
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
    for (uint64_t q = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; 2 * q < n_pairs; q += stride) {
        if (2 * q + 1 < n_pairs) {
            const uint4 w = reinterpret_cast<const uint4 *>(in)[q];
            float4 z;
            box_muller(w.x, w.y, z.x, z.y, bt);
            box_muller(w.z, w.w, z.z, z.w, bt);
            reinterpret_cast<float4 *>(out)[q] = z;
        } else {
            float z0, z1;
            if (!RNGX_IDX_OK(4 * q + 1, 2 * n_pairs, kSiteGen + __LINE__)) continue;
            box_muller(in[4 * q], in[4 * q + 1], z0, z1, bt);
            out[4 * q] = z0;
            out[4 * q + 1] = z1;
        }
    }
}
}  // namespace

RNGX_BOUNDS_MODULE(gen)

int launch_u32_to_normal(const uint32_t *in, float *out, uint64_t n_pairs, cudaStream_t s)
{
    if (n_pairs == 0) return RNG_OK;
    int dev = 0, sms = 0;
    RNGX_CHECK_CUDA(cudaGetDevice(&dev));
    RNGX_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const uint64_t quads = (n_pairs + 1) / 2;
    const unsigned blocks = static_cast<unsigned>(std::min<uint64_t>((quads + 255) / 256, static_cast<uint64_t>(sms) * 8));
    RNGX_CHECK_CUDA(bm_allow_smem<k_u32_to_normal>());
    k_u32_to_normal<<<blocks, 256, kBmSmemBytes, s>>>(in, out, n_pairs);
    RNGX_CHECK_LAUNCH();
    return RNG_OK;
}

int launch_generate(const GenState &g, void *d_out, uint64_t K, int out_kind, int layout, cudaStream_t s)
{
    if (K == 0) return RNG_OK;
    switch (g.kind) {
    case RNG_LCG32: return launch_kind<RNG_LCG32>(g, d_out, K, out_kind, layout, s);
    case RNG_LCG64: return launch_kind<RNG_LCG64>(g, d_out, K, out_kind, layout, s);
    case RNG_MWC: return launch_kind<RNG_MWC>(g, d_out, K, out_kind, layout, s);
    case RNG_XORWOW: return launch_kind<RNG_XORWOW>(g, d_out, K, out_kind, layout, s);
    case RNG_PHILOX4X32_10: return launch_kind<RNG_PHILOX4X32_10>(g, d_out, K, out_kind, layout, s);
    case RNG_PHILOX4X32_7: return launch_kind<RNG_PHILOX4X32_7>(g, d_out, K, out_kind, layout, s);
    case RNG_XS1024W: return launch_kind<RNG_XS1024W>(g, d_out, K, out_kind, layout, s);
    case RNG_MT19937_SHARED: return launch_kind<RNG_MT19937_SHARED>(g, d_out, K, out_kind, layout, s);
    case RNG_LFIB521:
    case RNG_LFIB1279: return launch_generate_lfib(g, d_out, K, out_kind, layout, s);
    }
    set_error("launch_generate: unknown kind %d", g.kind);
    return RNG_EINVAL;
}

}  // namespace rngx
