// mwc.cu -- the multiply-with-carry multiplier table (Sec. 3): the
// descending list of a < 2^32 for which p = a 2^32 - 1 and q = (p - 1)/2 =
// a 2^31 - 1 are both prime (p a safe prime), starting from 4294967118.
// Candidates are tested in parallel on the device (trial division by small
// primes, then Miller-Rabin on q and p) and compacted in descending order.
#include <mutex>
#include <vector>

#include "modarith.cuh"
#include "internal.h"

namespace rngx {
namespace {

constexpr int kBlock = 256;
constexpr int kNumSmall = 96;  // odd primes 3 .. 503

// For each small odd prime l: the residues of a that make l divide p or q,
// i.e. a = (2^32)^(-1) and a = (2^31)^(-1) (mod l); computed on the host.
struct SmallPrimes {
    uint32_t l[kNumSmall], rp[kNumSmall], rq[kNumSmall];
};
__constant__ SmallPrimes c_small;

__global__ void k_flags(uint64_t a_hi, uint64_t count, uint32_t *flags, uint32_t *block_counts)
{
    const uint64_t c = static_cast<uint64_t>(blockIdx.x) * kBlock + threadIdx.x;
    bool hit = false;
    if (c < count && a_hi >= c + 2) {
        const uint32_t a = static_cast<uint32_t>(a_hi - c);
        bool ok = true;
        for (int k = 0; k < kNumSmall && ok; k++) {
            const uint32_t r = a % c_small.l[k];
            ok = r != c_small.rp[k] && r != c_small.rq[k];
        }
        if (ok) {
            const uint64_t p = (static_cast<uint64_t>(a) << 32) - 1, q = (static_cast<uint64_t>(a) << 31) - 1;
            hit = is_prime_odd64(q) && is_prime_odd64(p);
        }
    }
    const unsigned ballot = __ballot_sync(0xffffffffu, hit);
    __shared__ uint32_t warp_counts[kBlock / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
        flags[blockIdx.x * (kBlock / 32) + w] = ballot;
        warp_counts[w] = __popc(ballot);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t s = 0;
        for (int i = 0; i < kBlock / 32; i++) s += warp_counts[i];
        block_counts[blockIdx.x] = s;
    }
}

__global__ void k_scatter(uint64_t a_hi, uint64_t count, const uint32_t *flags, const uint64_t *block_offsets,
                          uint32_t *table, uint64_t base, uint64_t cap)
{
    const uint64_t c = static_cast<uint64_t>(blockIdx.x) * kBlock + threadIdx.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t ballot = flags[blockIdx.x * (kBlock / 32) + w];
    if (c >= count || !((ballot >> lane) & 1)) return;
    uint64_t rank = block_offsets[blockIdx.x];
    for (int i = 0; i < w; i++) rank += __popc(flags[blockIdx.x * (kBlock / 32) + i]);
    rank += __popc(ballot & ((1u << lane) - 1));
    if (base + rank < cap) table[base + rank] = static_cast<uint32_t>(a_hi - c);
}

uint64_t host_powmod(uint64_t b, uint64_t e, uint64_t m)
{
    uint64_t r = 1 % m;
    b %= m;
    while (e) {
        if (e & 1) r = r * b % m;  // m < 2^10: no overflow
        b = b * b % m;
        e >>= 1;
    }
    return r;
}

struct Table {
    std::mutex mu;
    uint32_t *d = nullptr;
    uint64_t cap = 0, count = 0;
    uint64_t next_a = 0xffffffffull;  // next candidate to test
    bool consts = false;
};
Table g_tab[64];

}  // namespace

int mwc_table(uint64_t need, const uint32_t **d_table, cudaStream_t s)
{
    int dev = 0;
    RNGX_CHECK_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) {
        set_error("device index %d out of range", dev);
        return RNG_EINVAL;
    }
    Table &t = g_tab[dev];
    std::lock_guard<std::mutex> lock(t.mu);
    if (!t.consts) {
        SmallPrimes sp;
        int k = 0;
        for (uint32_t l = 3; k < kNumSmall; l += 2) {
            bool prime = true;
            for (uint32_t d = 3; d * d <= l; d += 2)
                if (l % d == 0) prime = false;
            if (!prime) continue;
            const uint64_t inv32 = host_powmod(host_powmod(2, 32, l), l - 2, l);
            const uint64_t inv31 = host_powmod(host_powmod(2, 31, l), l - 2, l);
            sp.l[k] = l;
            sp.rp[k] = static_cast<uint32_t>(inv32);
            sp.rq[k] = static_cast<uint32_t>(inv31);
            k++;
        }
        RNGX_CHECK_CUDA(cudaMemcpyToSymbol(c_small, &sp, sizeof(sp)));
        t.consts = true;
    }
    if (t.count < need) {
        // room for the request plus one chunk's worth of hits (a chunk of
        // 2^26 candidates holds far fewer than 2^20 multipliers)
        uint64_t cap = t.cap ? t.cap : (1ull << 21);
        while (cap < need + (1ull << 20)) cap *= 2;
        if (cap != t.cap) {
            uint32_t *d = nullptr;
            RNGX_CHECK_CUDA(cudaMalloc(&d, cap * 4));
            if (t.count) {
                cudaError_t e = cudaMemcpy(d, t.d, t.count * 4, cudaMemcpyDeviceToDevice);
                if (e != cudaSuccess) {
                    cudaFree(d);
                    return cuda_fail(e, "cudaMemcpy");
                }
            }
            if (t.d) cudaFree(t.d);
            t.d = d;
            t.cap = cap;
        }
        const uint64_t chunk = 1ull << 26;
        const uint64_t nblocks = chunk / kBlock;
        uint32_t *flags = nullptr, *counts = nullptr;
        uint64_t *offs = nullptr;
        RNGX_CHECK_CUDA(cudaMalloc(&flags, chunk / 8));
        RNGX_CHECK_CUDA(cudaMalloc(&counts, nblocks * 4));
        RNGX_CHECK_CUDA(cudaMalloc(&offs, nblocks * 8));
        std::vector<uint32_t> h_counts(nblocks);
        std::vector<uint64_t> h_offs(nblocks);
        int st = RNG_OK;
        while (t.count < need && st == RNG_OK) {
            if (t.next_a < 2) {
                set_error("MWC multiplier table exhausted below %llu entries", (unsigned long long)need);
                st = RNG_EINVAL;
                break;
            }
            const uint64_t cnt = t.next_a - 1 < chunk ? t.next_a - 1 : chunk;
            k_flags<<<static_cast<unsigned>(nblocks), kBlock, 0, s>>>(t.next_a, cnt, flags, counts);
            cudaError_t e = cudaMemcpyAsync(h_counts.data(), counts, nblocks * 4, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) {
                st = cuda_fail(e, "MWC multiplier search");
                break;
            }
            uint64_t acc = 0;
            for (uint64_t b = 0; b < nblocks; b++) {
                h_offs[b] = acc;
                acc += h_counts[b];
            }
            e = cudaMemcpyAsync(offs, h_offs.data(), nblocks * 8, cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess) {
                k_scatter<<<static_cast<unsigned>(nblocks), kBlock, 0, s>>>(t.next_a, cnt, flags, offs, t.d, t.count,
                                                                              t.cap);
                e = cudaGetLastError();
            }
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) {
                st = cuda_fail(e, "MWC multiplier scatter");
                break;
            }
            t.count = t.count + acc < t.cap ? t.count + acc : t.cap;
            t.next_a -= cnt;
            if (t.count >= t.cap && t.count < need) {
                set_error("MWC table capacity");
                st = RNG_ENOMEM;
            }
        }
        cudaFree(flags);
        cudaFree(counts);
        cudaFree(offs);
        RNGX_CHECK(st);
    }
    *d_table = t.d;
    return RNG_OK;
}

}  // namespace rngx

extern "C" int rng_mwc_multipliers(uint64_t first, uint64_t count, uint32_t *host_out)
{
    if (!host_out && count) {
        rngx::set_error("rng_mwc_multipliers: null output");
        return RNG_EINVAL;
    }
    const uint32_t *d = nullptr;
    RNGX_CHECK(rngx::mwc_table(first + count, &d, 0));
    RNGX_CHECK_CUDA(cudaMemcpy(host_out, d + first, count * 4, cudaMemcpyDeviceToHost));
    return RNG_OK;
}
