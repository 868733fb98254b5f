// ising_kernels.cuh -- per-kind kernel templates of the Ising path: the
// one-launch-per-half-sweep kernel (generator state and lattice in global
// memory) and the launcher of the persistent kernel.  Instantiated once per
// generator kind in ising_k*.cu so that the kinds compile in parallel.
#pragma once

#include "ising_persist.cuh"

namespace rngx {

// One half-sweep, one thread per stream (warps of 32 consecutive streams).
template <int KIND, int LAYOUT>
__global__ void __launch_bounds__(256) k_ising_half(LatDev lat, int c)
{
    const uint64_t s = static_cast<uint64_t>(blockIdx.x) * 256 + threadIdx.x;
    const uint64_t n_inst = lat.rng.n;
    if ((s & ~31ull) >= n_inst) return;
    const bool valid = s < lat.nstreams;
    Gen<KIND> gen;
    gen.load(lat.rng, s < n_inst ? s : n_inst - 1);
    const uint32_t G = lat.G, half = lat.half, L = lat.L;
    const uint64_t q0 = s * G;
    const uint32_t y = valid ? static_cast<uint32_t>(q0 / half) : 0;
    const uint32_t xh0 = valid ? static_cast<uint32_t>(q0 - static_cast<uint64_t>(y) * half) : 0;
    const uint32_t p = (c + y) & 1u;
    const uint32_t yu = y == 0 ? L - 1 : y - 1, yd = y + 1 == L ? 0 : y + 1;
    if (LAYOUT == ISING_INT8) {
        int8_t *sp = static_cast<int8_t *>(lat.spins);
        for (uint32_t g = 0; g < G; g++) {
            const uint32_t rr = gen.next();
            if (!valid) continue;
            const uint32_t x = 2 * (xh0 + g) + p;
            const uint32_t xl = x == 0 ? L - 1 : x - 1, xr = x + 1 == L ? 0 : x + 1;
            const size_t row = static_cast<size_t>(y) * L;
            const int nn = sp[row + xl] + sp[row + xr] + sp[static_cast<size_t>(yu) * L + x] +
                           sp[static_cast<size_t>(yd) * L + x];
            const int si = sp[row + x];
            if (accept_flip(2 * si * nn, rr, lat.T4, lat.T8)) sp[row + x] = static_cast<int8_t>(-si);
        }
    } else {
        const uint32_t W = lat.W;
        uint32_t *pc = static_cast<uint32_t *>(lat.spins) + static_cast<size_t>(c) * L * W;
        const uint32_t *po = static_cast<const uint32_t *>(lat.spins) + static_cast<size_t>(1 - c) * L * W;
        const uint32_t *o = po + static_cast<size_t>(y) * W;
        const uint32_t *ou = po + static_cast<size_t>(yu) * W;
        const uint32_t *od = po + static_cast<size_t>(yd) * W;
        const uint32_t *own = pc + static_cast<size_t>(y) * W;
        const int lane = threadIdx.x & 31;
        const uint32_t lq0 = lane * G;
        uint32_t c_lo = 0, c_hi = 0;
        for (uint32_t g = 0; g < G; g++) {
            const uint32_t rr = gen.next();
            if (!valid) continue;
            const uint32_t xh = xh0 + g;
            const int nn = bit_spin(o, col_left(xh, p, half)) + bit_spin(o, col_right(xh, p, half)) + bit_spin(ou, xh) +
                           bit_spin(od, xh);
            const int si = bit_spin(own, xh);
            if (accept_flip(2 * si * nn, rr, lat.T4, lat.T8)) {
                const uint32_t lq = lq0 + g;
                if ((lq >> 5) == (lq0 >> 5)) c_lo |= 1u << (lq & 31);
                else c_hi |= 1u << (lq & 31);
            }
        }
        const uint64_t first_word = ((s & ~31ull) * G) >> 5;
        const uint64_t words = static_cast<uint64_t>(L) * W;
        for (uint32_t m = 0; m < G; m++) {
            const uint32_t mine = ((lq0 >> 5) == m ? c_lo : 0u) | ((lq0 >> 5) + 1 == m ? c_hi : 0u);
            const uint32_t word = __reduce_or_sync(0xffffffffu, mine);
            if (lane == 0 && word && first_word + m < words) pc[first_word + m] ^= word;
        }
    }
    if (s < n_inst) gen.store(lat.rng, s);
}

template <int KIND>
int launch_half(const LatDev &lat, int c, cudaStream_t s)
{
    const unsigned nb = static_cast<unsigned>((lat.rng.n + 255) / 256);
    if (lat.layout == ISING_INT8) k_ising_half<KIND, ISING_INT8><<<nb, 256, 0, s>>>(lat, c);
    else k_ising_half<KIND, ISING_MULTISPIN32><<<nb, 256, 0, s>>>(lat, c);
    RNGX_CHECK_CUDA(cudaGetLastError());
    return RNG_OK;
}

template <int KIND, int LAYOUT, int SMAX>
int launch_persist_t(const PersistArgs &a, unsigned nblocks, unsigned threads, size_t smem, cudaStream_t s,
                     int *max_blocks)
{
    // kernel modes: 0 exact, 1 multi-hit, 2 / 3 the same with fixed slot roles
    // (SMAX = 2), 4 exact with one whole resident lattice per block (SMAX = 1),
    // 5 exact with roles split by warp and a polling warp (SMAX = 2), 6 exact
    // with a halo of two rows and one exchange per sweep (SMAX = 3, only)
    void (*kern)(PersistArgs);
    if constexpr (SMAX == 3) {
        if (a.k_hits || a.fixed_slots != 4) {
            set_error("persistent Ising: three slots per thread are the two-row-halo kernel's only");
            return RNG_EINVAL;
        }
        kern = k_ising_persist<KIND, LAYOUT, 3, 6>;
    } else {
        const bool fixed = SMAX == 2 && a.fixed_slots == 1, whole = SMAX == 1 && a.fixed_slots == 2;
        const bool split = SMAX == 2 && a.fixed_slots == 3 && !a.k_hits;
        kern = a.k_hits ? (fixed ? k_ising_persist<KIND, LAYOUT, SMAX, SMAX == 2 ? 2 : 1>
                                 : k_ising_persist<KIND, LAYOUT, SMAX, 1>)
                        : (fixed ? k_ising_persist<KIND, LAYOUT, SMAX, SMAX == 2 ? 3 : 0>
                                 : (whole ? k_ising_persist<KIND, LAYOUT, SMAX, SMAX == 1 ? 4 : 0>
                                          : (split ? k_ising_persist<KIND, LAYOUT, SMAX, SMAX == 2 ? 5 : 0>
                                                   : k_ising_persist<KIND, LAYOUT, SMAX, 0>)));
    }
    RNGX_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
    int per_sm = 0, dev = 0, sms = 0;
    RNGX_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
    RNGX_CHECK_CUDA(cudaGetDevice(&dev));
    RNGX_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (max_blocks) *max_blocks = per_sm * sms;
    if (nblocks == 0) return RNG_OK;  // occupancy query only
    if (static_cast<long>(nblocks) > static_cast<long>(per_sm) * sms) {
        set_error("persistent Ising launch needs %u co-resident blocks, the device holds %d", nblocks, per_sm * sms);
        return RNG_EINVAL;
    }
    PersistArgs args = a;
    void *params[] = {&args};
    RNGX_CHECK_CUDA(cudaLaunchCooperativeKernel(reinterpret_cast<void *>(kern), dim3(nblocks), dim3(threads), params,
                                                smem, s));
    return RNG_OK;
}

template <int KIND>
int launch_persist(int layout, int smax, const PersistArgs &a, unsigned nblocks, unsigned threads, size_t smem,
                   cudaStream_t s, int *max_blocks)
{
    if (layout == ISING_INT8) {
        switch (smax) {
        case 1: return launch_persist_t<KIND, ISING_INT8, 1>(a, nblocks, threads, smem, s, max_blocks);
        case 2: return launch_persist_t<KIND, ISING_INT8, 2>(a, nblocks, threads, smem, s, max_blocks);
        case 3: return launch_persist_t<KIND, ISING_INT8, 3>(a, nblocks, threads, smem, s, max_blocks);
        default: return launch_persist_t<KIND, ISING_INT8, 4>(a, nblocks, threads, smem, s, max_blocks);
        }
    }
    switch (smax) {
    case 1: return launch_persist_t<KIND, ISING_MULTISPIN32, 1>(a, nblocks, threads, smem, s, max_blocks);
    case 2: return launch_persist_t<KIND, ISING_MULTISPIN32, 2>(a, nblocks, threads, smem, s, max_blocks);
    case 3: return launch_persist_t<KIND, ISING_MULTISPIN32, 3>(a, nblocks, threads, smem, s, max_blocks);
    default: return launch_persist_t<KIND, ISING_MULTISPIN32, 4>(a, nblocks, threads, smem, s, max_blocks);
    }
}

#define RNGX_ISING_INSTANTIATE(KIND)                                                                          \
    template int launch_half<KIND>(const LatDev &, int, cudaStream_t);                                        \
    template int launch_persist<KIND>(int, int, const PersistArgs &, unsigned, unsigned, size_t, cudaStream_t, \
                                      int *);                                                                 \
    RNGX_BOUNDS_MODULE(persist_##KIND)

}  // namespace rngx
