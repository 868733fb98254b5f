// gf2.cu -- matrices over GF(2) for the xorshift generators (Sec. 6, Eq.
// (threeshift): x_n = x_{n-1} M).  States are row vectors, row i of M is
// the image of unit vector e_i, bit j of a vector is bit j % 32 of word
// j / 32.  The one-step matrix is built by running the device step on the
// unit vectors, so it matches the generator by construction; powers come
// from repeated squaring (one warp per output row).
#include <mutex>
#include <vector>

#include "gen_device.cuh"

namespace rngx {
namespace {

// Row i of the 1024-bit one-step matrix: warp i steps e_i once.
__global__ void k_one_step_xs(uint32_t *M)
{
    const int row = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const uint32_t lane = threadIdx.x & 31;
    if (row >= 1024) return;
    Gen<RNG_XS1024W> g;
    g.lane = lane;
    g.step = 0;
    g.x = (static_cast<uint32_t>(row >> 5) == lane) ? (1u << (row & 31)) : 0u;
    g.shift_step();
    M[row * 32 + lane] = g.x;
}

// Row i of the 160-bit xorshift part of XORWOW (words x, y, z, w, v).
__global__ void k_one_step_xorwow(uint32_t *M)
{
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= 160) return;
    uint32_t w[5] = {0, 0, 0, 0, 0};
    w[row >> 5] = 1u << (row & 31);
    Gen<RNG_XORWOW> g;
    g.x = w[0];
    g.y = w[1];
    g.z = w[2];
    g.w = w[3];
    g.v = w[4];
    g.d = 0;
    g.shift();
    const uint32_t o[5] = {g.x, g.y, g.z, g.w, g.v};
    for (int k = 0; k < 5; k++) M[row * 5 + k] = o[k];
}

__global__ void k_identity(uint32_t *M, int n)
{
    const int nw = n / 32;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * nw) return;
    const int row = idx / nw, w = idx % nw;
    M[idx] = (row >> 5) == w ? (1u << (row & 31)) : 0u;
}

// C = A B: warp per row of C; row i = XOR of rows k of B with A[i][k] = 1.
__global__ void k_mul(int n, const uint32_t *__restrict__ A, const uint32_t *__restrict__ B, uint32_t *__restrict__ C)
{
    const int nw = n / 32;
    const int row = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    uint32_t acc = 0;
    for (int wi = 0; wi < nw; wi++) {
        uint32_t bits = A[row * nw + wi];
        while (bits) {
            const int b = __ffs(bits) - 1;
            bits &= bits - 1;
            if (lane < nw) acc ^= B[(wi * 32 + b) * nw + lane];
        }
    }
    if (lane < nw) C[row * nw + lane] = acc;
}

struct SubstreamCache {
    std::mutex mu;
    int levels = 0;
    uint32_t *d = nullptr;  // levels matrices of 1024 x 32 words
};

SubstreamCache g_sub[64];

}  // namespace

int gf2_one_step(int kind, uint32_t *d_m, cudaStream_t s)
{
    if (kind == RNG_XS1024W) k_one_step_xs<<<128, 256, 0, s>>>(d_m);
    else k_one_step_xorwow<<<1, 160, 0, s>>>(d_m);
    RNGX_CHECK_LAUNCH();
    return RNG_OK;
}

int gf2_mul(int n, const uint32_t *d_a, const uint32_t *d_b, uint32_t *d_c, cudaStream_t s)
{
    const int warps_per_block = 8;
    k_mul<<<(n + warps_per_block - 1) / warps_per_block, 32 * warps_per_block, 0, s>>>(n, d_a, d_b, d_c);
    RNGX_CHECK_LAUNCH();
    return RNG_OK;
}

// d_out = M^t with two temporaries of the same size.
int gf2_pow(int kind, uint64_t t, uint32_t *d_out, uint32_t *d_sq, uint32_t *d_tmp, cudaStream_t s)
{
    const int n = kind == RNG_XS1024W ? 1024 : 160;
    const int words = n * (n / 32);
    k_identity<<<(words + 255) / 256, 256, 0, s>>>(d_out, n);
    RNGX_CHECK_LAUNCH();
    RNGX_CHECK(gf2_one_step(kind, d_sq, s));
    while (t) {
        if (t & 1) {
            RNGX_CHECK(gf2_mul(n, d_out, d_sq, d_tmp, s));
            RNGX_CHECK_CUDA(cudaMemcpyAsync(d_out, d_tmp, words * 4, cudaMemcpyDeviceToDevice, s));
        }
        t >>= 1;
        if (t) {
            RNGX_CHECK(gf2_mul(n, d_sq, d_sq, d_tmp, s));
            RNGX_CHECK_CUDA(cudaMemcpyAsync(d_sq, d_tmp, words * 4, cudaMemcpyDeviceToDevice, s));
        }
    }
    return RNG_OK;
}

// P_k = M^(2^(137+k)), k < levels, cached per device for the process.
int xs_substream_matrices(int levels, const uint32_t **d_P, cudaStream_t s)
{
    int dev = 0;
    RNGX_CHECK_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) {
        set_error("device index %d out of range", dev);
        return RNG_EINVAL;
    }
    SubstreamCache &c = g_sub[dev];
    std::lock_guard<std::mutex> lock(c.mu);
    if (c.levels < levels) {
        const int want = levels < 20 ? 20 : levels;
        const size_t mw = 1024 * 32;
        uint32_t *d = nullptr, *tmp = nullptr;
        RNGX_CHECK_CUDA(cudaMalloc(&d, want * mw * 4));
        cudaError_t e = cudaMalloc(&tmp, 2 * mw * 4);
        if (e != cudaSuccess) {
            cudaFree(d);
            return cuda_fail(e, "cudaMalloc");
        }
        uint32_t *a = tmp, *b = tmp + mw;
        int st = gf2_one_step(RNG_XS1024W, a, s);
        for (int i = 0; i < 137 && st == RNG_OK; i++) {  // M^(2^137)
            st = gf2_mul(1024, a, a, b, s);
            uint32_t *t = a;
            a = b;
            b = t;
        }
        if (st == RNG_OK) st = cudaMemcpyAsync(d, a, mw * 4, cudaMemcpyDeviceToDevice, s) == cudaSuccess
                                   ? RNG_OK : RNG_ECUDA;
        for (int k = 1; k < want && st == RNG_OK; k++) st = gf2_mul(1024, d + (k - 1) * mw, d + (k - 1) * mw, d + k * mw, s);
        e = cudaStreamSynchronize(s);
        cudaFree(tmp);
        if (st != RNG_OK || e != cudaSuccess) {
            cudaFree(d);
            return st != RNG_OK ? st : cuda_fail(e, "substream matrices");
        }
        if (c.d) cudaFree(c.d);
        c.d = d;
        c.levels = want;
    }
    *d_P = c.d;
    return RNG_OK;
}

}  // namespace rngx
