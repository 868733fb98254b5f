// peaks.cu -- throughput microbenchmark of the SM pipes the generators and
// the Ising update run on: 32-bit logic (LOP3, the integer ALU pipe),
// integer multiply-add (IMAD), warp shuffles (SHFL) and float FMA (FFMA,
// whose full rate equals the issue rate of one instruction per scheduler
// and cycle).  Every thread runs eight independent dependency chains of one
// instruction kind, in inline PTX so that none is folded away; the rate is
// thread-instructions per second over the whole GPU.  Not part of the
// paper: it supplies the denominators of the instruction-issue rooflines.
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"

namespace rngx {

namespace {

constexpr int kChains = 8;
constexpr int kPeakBlock = 256;

enum { P_LOP3 = 0, P_IMAD = 1, P_SHFL = 2, P_FFMA = 3 };

template <int OP>
__global__ void __launch_bounds__(kPeakBlock) k_peak(uint32_t *sink, int iters)
{
    const uint32_t b = threadIdx.x * 0x9E3779B9u + 1u, c = blockIdx.x * 0x85EBCA6Bu + 3u;
    uint32_t a[kChains];
    float f[kChains];
#pragma unroll
    for (int j = 0; j < kChains; j++) {
        a[j] = b + j * 0x27D4EB2Fu;
        f[j] = 1.0f + 1e-3f * static_cast<float>(j + threadIdx.x % 7);
    }
    const float fb = 0.999999f, fc = 1e-7f;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int j = 0; j < kChains; j++) {
            if (OP == P_LOP3) asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(a[j]) : "r"(b), "r"(c));
            if (OP == P_IMAD) asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(a[j]) : "r"(b), "r"(c));
            if (OP == P_SHFL) asm volatile("shfl.sync.bfly.b32 %0, %0, 1, 0x1f, 0xffffffff;" : "+r"(a[j]));
            if (OP == P_FFMA) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(f[j]) : "f"(fb), "f"(fc));
        }
    }
    uint32_t acc = 0;
#pragma unroll
    for (int j = 0; j < kChains; j++) acc ^= a[j] ^ __float_as_uint(f[j]);
    if (acc == 0x12345678u) sink[0] = acc;  // keeps the chains live
}

template <int OP>
int time_peak(uint32_t *sink, int blocks, int iters, cudaStream_t s, double *ops_per_s)
{
    cudaEvent_t e0, e1;
    RNGX_CHECK_CUDA(cudaEventCreate(&e0));
    RNGX_CHECK_CUDA(cudaEventCreate(&e1));
    k_peak<OP><<<blocks, kPeakBlock, 0, s>>>(sink, iters / 8);  // warm-up
    float best = 1e30f;
    for (int rep = 0; rep < 3; rep++) {
        cudaEventRecord(e0, s);
        k_peak<OP><<<blocks, kPeakBlock, 0, s>>>(sink, iters);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        best = std::min(best, ms);
    }
    cudaError_t e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(e, "issue-peak kernel");
    *ops_per_s = static_cast<double>(blocks) * kPeakBlock * iters * kChains / (best * 1e-3);
    return RNG_OK;
}

}  // namespace

}  // namespace rngx

extern "C" int rng_issue_peaks(double *lop3, double *imad, double *shfl, double *ffma, void *cuda_stream)
{
    using namespace rngx;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0, sms = 0;
    RNGX_CHECK_CUDA(cudaGetDevice(&dev));
    RNGX_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = sms * 8;  // 2048 threads per SM: full occupancy
    uint32_t *sink = nullptr;
    RNGX_CHECK(dalloc(reinterpret_cast<void **>(&sink), sizeof(uint32_t), s));
    double v[4] = {0, 0, 0, 0};
    int st = time_peak<P_LOP3>(sink, blocks, 4096, s, &v[0]);
    if (st == RNG_OK) st = time_peak<P_IMAD>(sink, blocks, 4096, s, &v[1]);
    if (st == RNG_OK) st = time_peak<P_SHFL>(sink, blocks, 2048, s, &v[2]);
    if (st == RNG_OK) st = time_peak<P_FFMA>(sink, blocks, 4096, s, &v[3]);
    dfree(sink, s);
    if (st != RNG_OK) return st;
    if (lop3) *lop3 = v[0];
    if (imad) *imad = v[1];
    if (shfl) *shfl = v[2];
    if (ffma) *ffma = v[3];
    return RNG_OK;
}
