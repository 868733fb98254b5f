// mwc.cu -- the multiply-with-carry multiplier table (Sec. 3): the
// descending list of a < 2^32 for which p = a 2^32 - 1 and q = (p - 1)/2 =
// a 2^31 - 1 are both prime (p a safe prime), starting from 4294967118.
// Candidates are sieved in shared memory by the odd primes below 2^16, the
// survivors tested by Miller-Rabin on q and p, and the hits compacted in
// descending order of a.
#include <mutex>
#include <vector>

#include "modarith.cuh"
#include "internal.h"

namespace rngx {
namespace {

constexpr int kBlock = 256;
constexpr int kSeg = 1 << 16;           // candidates sieved by one block
constexpr uint32_t kSieveLimit = 1 << 16;  // odd primes below this sieve the candidates
constexpr uint32_t kSmall = 1024;          // primes below this are marked by the whole block

// One block sieves kSeg consecutive candidates c (multiplier a = a_hi - c):
// a candidate is composite when an odd prime l < 2^16 divides p = a 2^32 - 1
// or q = a 2^31 - 1, i.e. when a = (2^32)^(-1) or (2^31)^(-1) (mod l).  The
// survivors (about 1%) then go through Miller-Rabin for q and p; flags get
// one bit per candidate, block_counts the hits of the block.
__global__ void __launch_bounds__(kBlock) k_flags(uint64_t a_hi, uint64_t count, const uint32_t *primes,
                                                  const uint32_t *rp, const uint32_t *rq, int nprimes,
                                                  uint32_t *flags, uint32_t *block_counts)
{
    __shared__ uint32_t comp[kSeg / 32];
    __shared__ uint32_t warp_hits[kBlock / 32];
    const uint64_t c0 = static_cast<uint64_t>(blockIdx.x) * kSeg;
    for (int w = threadIdx.x; w < kSeg / 32; w += kBlock) {
        uint32_t m = 0;
        for (int b = 0; b < 32; b++) {
            const uint64_t c = c0 + 32 * w + b;
            if (c >= count || a_hi < c + 2) m |= 1u << b;  // past the chunk, or a < 2
        }
        comp[w] = m;
    }
    __syncthreads();
    // primes below kSmall mark many candidates each: all threads share their
    // marks; the larger primes are spread one per thread
    int k = 0;
    for (; k < nprimes && primes[k] < kSmall; k++) {
        const uint32_t l = primes[k];
        const uint32_t ah = static_cast<uint32_t>(a_hi % l), cm = static_cast<uint32_t>(c0 % l);
        for (int j = 0; j < 2; j++) {
            // a_hi - c = r (mod l)  <=>  c = a_hi - r (mod l)
            const uint32_t t = (ah + l - (j ? rq[k] : rp[k])) % l;
            const uint32_t start = (t + l - cm) % l;
            for (uint32_t c = start + threadIdx.x * l; c < static_cast<uint32_t>(kSeg); c += kBlock * l)
                atomicOr(&comp[c >> 5], 1u << (c & 31));
        }
    }
    for (k += threadIdx.x; k < nprimes; k += kBlock) {
        const uint32_t l = primes[k];
        const uint32_t ah = static_cast<uint32_t>(a_hi % l), cm = static_cast<uint32_t>(c0 % l);
        for (int j = 0; j < 2; j++) {
            const uint32_t t = (ah + l - (j ? rq[k] : rp[k])) % l;
            for (uint32_t c = (t + l - cm) % l; c < static_cast<uint32_t>(kSeg); c += l)
                atomicOr(&comp[c >> 5], 1u << (c & 31));
        }
    }
    __syncthreads();
    // each thread tests the survivors of 8 consecutive words (256 candidates)
    uint32_t hits = 0;
    const int w0 = threadIdx.x * (kSeg / 32 / kBlock);
    for (int w = w0; w < w0 + kSeg / 32 / kBlock; w++) {
        uint32_t live = ~comp[w], out = 0;
        while (live) {
            const int b = __ffs(live) - 1;
            live &= live - 1;
            const uint32_t a = static_cast<uint32_t>(a_hi - (c0 + 32 * w + b));
            const uint64_t p = (static_cast<uint64_t>(a) << 32) - 1, q = (static_cast<uint64_t>(a) << 31) - 1;
            if (is_prime_odd64(q) && is_prime_odd64(p)) out |= 1u << b;
        }
        flags[(c0 >> 5) + w] = out;
        hits += __popc(out);
    }
    for (int o = 16; o > 0; o >>= 1) hits += __shfl_down_sync(0xffffffffu, hits, o);
    if ((threadIdx.x & 31) == 0) warp_hits[threadIdx.x >> 5] = hits;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int i = 0; i < kBlock / 32; i++) t += warp_hits[i];
        block_counts[blockIdx.x] = t;
    }
}

// Writes the hits of each block in candidate order (descending a) at the
// block's offset of the running table.
__global__ void __launch_bounds__(kBlock) k_scatter(uint64_t a_hi, const uint32_t *flags, const uint64_t *block_offsets,
                                                    uint32_t *table, uint64_t base, uint64_t cap)
{
    __shared__ uint32_t scan[kBlock];
    const uint64_t c0 = static_cast<uint64_t>(blockIdx.x) * kSeg;
    const int per = kSeg / 32 / kBlock;
    const int w0 = threadIdx.x * per;
    uint32_t mine = 0;
    for (int w = w0; w < w0 + per; w++) mine += __popc(flags[(c0 >> 5) + w]);
    scan[threadIdx.x] = mine;
    __syncthreads();
    for (int o = 1; o < kBlock; o <<= 1) {  // inclusive scan
        const uint32_t v = threadIdx.x >= o ? scan[threadIdx.x - o] : 0;
        __syncthreads();
        scan[threadIdx.x] += v;
        __syncthreads();
    }
    uint64_t pos = base + block_offsets[blockIdx.x] + scan[threadIdx.x] - mine;
    for (int w = w0; w < w0 + per; w++) {
        uint32_t f = flags[(c0 >> 5) + w];
        while (f) {
            const int b = __ffs(f) - 1;
            f &= f - 1;
            if (pos < cap) table[pos] = static_cast<uint32_t>(a_hi - (c0 + 32 * w + b));
            pos++;
        }
    }
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
    uint32_t *d_primes = nullptr;     // odd primes below 2^16 and their residues
    uint32_t *d_rp = nullptr, *d_rq = nullptr;
    int nprimes = 0;
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
    if (!t.d_primes) {
        std::vector<uint32_t> pr, rp, rq;
        std::vector<char> compo(kSieveLimit, 0);
        for (uint32_t l = 3; l < kSieveLimit; l += 2) {
            if (compo[l]) continue;
            for (uint64_t m = static_cast<uint64_t>(l) * l; m < kSieveLimit; m += 2 * l) compo[m] = 1;
            pr.push_back(l);
            // the a that make l divide a 2^32 - 1 (resp. a 2^31 - 1)
            rp.push_back(static_cast<uint32_t>(host_powmod(host_powmod(2, 32, l), l - 2, l)));
            rq.push_back(static_cast<uint32_t>(host_powmod(host_powmod(2, 31, l), l - 2, l)));
        }
        const size_t nb = pr.size() * 4;
        RNGX_CHECK_CUDA(cudaMalloc(&t.d_primes, 3 * nb));
        t.d_rp = t.d_primes + pr.size();
        t.d_rq = t.d_rp + pr.size();
        RNGX_CHECK_CUDA(cudaMemcpy(t.d_primes, pr.data(), nb, cudaMemcpyHostToDevice));
        RNGX_CHECK_CUDA(cudaMemcpy(t.d_rp, rp.data(), nb, cudaMemcpyHostToDevice));
        RNGX_CHECK_CUDA(cudaMemcpy(t.d_rq, rq.data(), nb, cudaMemcpyHostToDevice));
        t.nprimes = static_cast<int>(pr.size());
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
        const uint64_t nblocks = chunk / kSeg;
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
            k_flags<<<static_cast<unsigned>(nblocks), kBlock, 0, s>>>(t.next_a, cnt, t.d_primes, t.d_rp, t.d_rq,
                                                                     t.nprimes, flags, counts);
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
                k_scatter<<<static_cast<unsigned>(nblocks), kBlock, 0, s>>>(t.next_a, flags, offs, t.d, t.count,
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
