// gen.cu -- generation kernels: every instance emits K draws as u32, exact
// uniform f32 or Box-Muller normals, in step-major, instance-major or
// consume-in-register (XOR / sum) form.  The state is loaded into
// registers once, stepped K times and stored once (the paper's concern
// about state load/store overhead, Sec. 2 and the caption of Table 2).
#include "gen_device.cuh"

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
    const uint64_t n = p.n;
    const uint64_t i = static_cast<uint64_t>(blockIdx.x) * kBlock + threadIdx.x;
    const bool active = i < n;
    // Warps entirely past the end leave; partial warps keep every lane for
    // the warp-level transpose (per-thread kinds only: n % 32 == 0 for XS1024W).
    if ((i & ~static_cast<uint64_t>(31)) >= n) return;
    Gen<KIND> g;
    if (active) g.load(p, i);
    else g.load(p, n - 1);  // dummy state, output discarded

    if (LAYOUT == RNG_STEP_MAJOR) {
        if (OUT == OUT_NORMAL) {
            float *out = static_cast<float *>(out_);
            for (uint64_t k = 0; k < K; k += 2) {
                const uint32_t r0 = g.next(), r1 = g.next();
                float z0, z1;
                box_muller(r0, r1, z0, z1);
                if (active) {
                    st_stream(out + k * n + i, z0);
                    st_stream(out + (k + 1) * n + i, z1);
                }
            }
        } else {
            for (uint64_t k = 0; k < K; k++) {
                const uint32_t r = g.next();
                if (!active) continue;
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
                    box_muller(r0, r1, z0, z1);
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
                    if (i0 + r < n) __stcs(out + (i0 + r) * K + k0 + lane, tile[w][r][lane]);
            }
            __syncwarp();
        }
    } else {  // RNG_XOR_REDUCE: consume in registers
        if (OUT == OUT_NORMAL) {
            float acc = 0.0f;
            for (uint64_t k = 0; k < K; k += 2) {
                const uint32_t r0 = g.next(), r1 = g.next();
                float z0, z1;
                box_muller(r0, r1, z0, z1);
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

// ------------------------------------------------------------- MT19937
// One generator per thread block: the 624-word state lives in shared
// memory and is refilled cooperatively in three barrier-separated phases
// whose ranges [0,227), [227,454), [454,624) only read words that are
// either not yet rewritten or rewritten by an earlier phase (Sec. 5; the
// block-wise vectorisation of the paper's GPU Mersenne twister variants).
constexpr int kMtBlock = 256;

__device__ __forceinline__ uint32_t mt_mix(uint32_t cur, uint32_t nxt, uint32_t far)
{
    const uint32_t y = (cur & 0x80000000u) | (nxt & 0x7fffffffu);
    return far ^ (y >> 1) ^ ((y & 1u) ? 0x9908B0DFu : 0u);
}

__device__ void mt_twist(uint32_t *mt)
{
    const int t = threadIdx.x;
    uint32_t v = 0;
    // phase 1: i in [0, 227), far word i + 397 not yet rewritten
    if (t < MT_N - MT_M) v = mt_mix(mt[t], mt[t + 1], mt[t + MT_M]);
    __syncthreads();
    if (t < MT_N - MT_M) mt[t] = v;
    __syncthreads();
    // phase 2: i in [227, 454), far word i - 227 rewritten in phase 1
    if (t < MT_N - MT_M) {
        const int i = t + (MT_N - MT_M);
        v = mt_mix(mt[i], mt[i + 1], mt[i - (MT_N - MT_M)]);
    }
    __syncthreads();
    if (t < MT_N - MT_M) mt[t + (MT_N - MT_M)] = v;
    __syncthreads();
    // phase 3: i in [454, 624), far word i - 227 rewritten in phase 2; the
    // last word pairs with the new word 0
    const int base = 2 * (MT_N - MT_M);
    if (t < MT_N - base) {
        const int i = t + base;
        v = mt_mix(mt[i], mt[(i + 1) % MT_N], mt[i - (MT_N - MT_M)]);
    }
    __syncthreads();
    if (t < MT_N - base) mt[t + base] = v;
    __syncthreads();
}

template <int OUT, int LAYOUT>
__global__ void __launch_bounds__(kMtBlock) k_generate_mt(DevParams p, void *out_, uint64_t K)
{
    __shared__ uint32_t mt[MT_N];
    __shared__ uint32_t buf[MT_N + 1];
    __shared__ uint32_t red[kMtBlock];
    const uint64_t gidx = blockIdx.x;
    const uint64_t n = p.n;
    uint32_t *st = static_cast<uint32_t *>(p.s[0]) + gidx * MT_N;
    for (int t = threadIdx.x; t < MT_N; t += kMtBlock) mt[t] = st[t];
    int mti = p.pos == 0 ? MT_N : static_cast<int>((p.pos - 1) % MT_N) + 1;
    __syncthreads();

    auto out_index = [&](uint64_t d) -> uint64_t {
        return LAYOUT == RNG_INSTANCE_MAJOR ? gidx * K + d : d * n + gidx;
    };
    uint32_t xacc = 0;
    float facc = 0.0f;
    uint32_t pending = 0;  // first word of a normal pair split across refills
    bool twisted = false;
    uint64_t k = 0;
    while (k < K) {
        if (mti == MT_N) {
            mt_twist(mt);
            mti = 0;
            twisted = true;
        }
        const int cnt = static_cast<int>(K - k < static_cast<uint64_t>(MT_N - mti) ? K - k : MT_N - mti);
        if (OUT != OUT_NORMAL) {
            for (int t = threadIdx.x; t < cnt; t += kMtBlock) {
                const uint32_t r = mt_temper(mt[mti + t]);
                const uint32_t bits = OUT == OUT_U32 ? r : __float_as_uint(u32_to_unit(r));
                if (LAYOUT == RNG_XOR_REDUCE) xacc ^= bits;
                else __stcs(static_cast<uint32_t *>(out_) + out_index(k + t), bits);
            }
        } else {
            // buf[0] = pending word when k is odd, then the chunk
            const int off = static_cast<int>(k & 1);
            for (int t = threadIdx.x; t < cnt; t += kMtBlock) buf[off + t] = mt_temper(mt[mti + t]);
            if (threadIdx.x == 0 && off) buf[0] = pending;
            __syncthreads();
            const uint64_t d0 = k - off;           // draw index of buf[0], even
            const int avail = cnt + off;
            const int pairs = avail / 2;
            for (int t = threadIdx.x; t < pairs; t += kMtBlock) {
                float z0, z1;
                box_muller(buf[2 * t], buf[2 * t + 1], z0, z1);
                if (LAYOUT == RNG_XOR_REDUCE) {
                    facc += z0;
                    facc += z1;
                } else {
                    float *out = static_cast<float *>(out_);
                    __stcs(out + out_index(d0 + 2 * t), z0);
                    __stcs(out + out_index(d0 + 2 * t + 1), z1);
                }
            }
            if (avail & 1) pending = buf[avail - 1];  // uniform across threads
        }
        k += cnt;
        mti += cnt;
        __syncthreads();
    }
    if (LAYOUT == RNG_XOR_REDUCE) {
        if (OUT == OUT_NORMAL) red[threadIdx.x] = __float_as_uint(facc);
        else red[threadIdx.x] = xacc;
        __syncthreads();
        for (int s = kMtBlock / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s) {
                if (OUT == OUT_NORMAL)
                    red[threadIdx.x] = __float_as_uint(__uint_as_float(red[threadIdx.x]) +
                                                       __uint_as_float(red[threadIdx.x + s]));
                else red[threadIdx.x] ^= red[threadIdx.x + s];
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) static_cast<uint32_t *>(out_)[gidx] = red[0];
    }
    if (twisted)
        for (int t = threadIdx.x; t < MT_N; t += kMtBlock) st[t] = mt[t];
}

template <int KIND, int OUT>
int launch_kind_out(const GenState &g, void *out, uint64_t K, int layout, cudaStream_t s)
{
    const DevParams p = dev_params(g);
    if constexpr (KIND == RNG_MT19937_SHARED) {
        const dim3 grid(static_cast<unsigned>(g.n));
        switch (layout) {
        case RNG_STEP_MAJOR: k_generate_mt<OUT, RNG_STEP_MAJOR><<<grid, kMtBlock, 0, s>>>(p, out, K); break;
        case RNG_INSTANCE_MAJOR: k_generate_mt<OUT, RNG_INSTANCE_MAJOR><<<grid, kMtBlock, 0, s>>>(p, out, K); break;
        default: k_generate_mt<OUT, RNG_XOR_REDUCE><<<grid, kMtBlock, 0, s>>>(p, out, K); break;
        }
    } else {
        const dim3 grid(static_cast<unsigned>((g.n + kBlock - 1) / kBlock));
        switch (layout) {
        case RNG_STEP_MAJOR: k_generate<KIND, OUT, RNG_STEP_MAJOR><<<grid, kBlock, 0, s>>>(p, out, K); break;
        case RNG_INSTANCE_MAJOR: k_generate<KIND, OUT, RNG_INSTANCE_MAJOR><<<grid, kBlock, 0, s>>>(p, out, K); break;
        default: k_generate<KIND, OUT, RNG_XOR_REDUCE><<<grid, kBlock, 0, s>>>(p, out, K); break;
        }
    }
    RNGX_CHECK_CUDA(cudaGetLastError());
    return RNG_OK;
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

int launch_generate(const GenState &g, void *d_out, uint64_t K, int out_kind, int layout, cudaStream_t s)
{
    if (K == 0) return RNG_OK;
    switch (g.kind) {
    case RNG_LCG32: return launch_kind<RNG_LCG32>(g, d_out, K, out_kind, layout, s);
    case RNG_LCG64: return launch_kind<RNG_LCG64>(g, d_out, K, out_kind, layout, s);
    case RNG_MWC: return launch_kind<RNG_MWC>(g, d_out, K, out_kind, layout, s);
    case RNG_XORWOW: return launch_kind<RNG_XORWOW>(g, d_out, K, out_kind, layout, s);
    case RNG_PHILOX4X32_10: return launch_kind<RNG_PHILOX4X32_10>(g, d_out, K, out_kind, layout, s);
    case RNG_XS1024W: return launch_kind<RNG_XS1024W>(g, d_out, K, out_kind, layout, s);
    case RNG_MT19937_SHARED: return launch_kind<RNG_MT19937_SHARED>(g, d_out, K, out_kind, layout, s);
    }
    set_error("launch_generate: unknown kind %d", g.kind);
    return RNG_EINVAL;
}

}  // namespace rngx
