// ising_common.cuh -- shared definitions of the checkerboard Metropolis
// kernels (application test of Sec. 2: 2D Ising ferromagnet, J = 1, zero
// field, periodic L x L, checkerboard update).
//
// Site numbering: colour c of (x, y) is (x + y) & 1; the colour-c sites of
// row y are x = 2 xh + p with p = (c + y) & 1, xh < L/2, numbered
// q = y (L/2) + xh.  Stream s owns q in [sG, (s+1)G) of both colours and
// draws one number per owned site per half-sweep, in increasing q, whatever
// the energy change; a flip is accepted iff dE <= 0 or r < T[dE].
// Neighbours of colour-c site (xh, y) are colour (1-c) sites (xh+p-1, y),
// (xh+p, y) (mod L/2) and (xh, y-1), (xh, y+1) (mod L).
#pragma once

#include "gen_device.cuh"

namespace rngx {

// One lattice as the kernels see it.
struct LatDev {
    uint32_t L, G, layout, half;   // half = L/2
    uint32_t W;                    // multispin words per plane row (L/64)
    uint32_t pad;
    uint64_t T4, T8;               // acceptance thresholds (64-bit: 2^32 at beta = 0)
    uint64_t nstreams;
    DevParams rng;                 // generator state of the lattice's streams
    void *spins;                   // int8 row-major L*L, or 2 bit planes of L*W words
    int64_t *meas;                 // per launch: (E, M) of each measurement
    int64_t *acc;                  // sum E, sum E^2, sum M^2, sum |M|, n_meas, E, M
    uint64_t *pos_dev;             // draws consumed per stream (device copy of the position)
};

// A row strip [y0, y1) of one lattice held by one thread block.
struct SegDev {
    uint32_t lat;                  // lattice index
    uint32_t coarse;               // strip index parity (multi-hit phases)
    uint32_t y0, y1;
    uint32_t smem_off;             // bytes into the block's dynamic shared memory
    int32_t up, down;              // segments holding rows y0-1 and y1; -1: this one (whole lattice)
    uint64_t s0, s1;               // streams [s0, s1) owned by the strip
};

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(uint32_t *p, uint32_t v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ bool accept_flip(int dE, uint32_t r, uint64_t T4, uint64_t T8)
{
    return dE <= 0 || static_cast<uint64_t>(r) < (dE == 4 ? T4 : T8);
}

// Column helpers for the neighbours in the other colour (wrap at L/2).
__device__ __forceinline__ uint32_t col_left(uint32_t xh, uint32_t p, uint32_t half)
{
    return (xh + p == 0) ? half - 1 : xh + p - 1;
}
__device__ __forceinline__ uint32_t col_right(uint32_t xh, uint32_t p, uint32_t half)
{
    return (xh + p == half) ? 0 : xh + p;
}

__device__ __forceinline__ int bit_spin(const uint32_t *row, uint32_t xh)
{
    return 1 - 2 * static_cast<int>((row[xh >> 5] >> (xh & 31)) & 1u);
}

}  // namespace rngx
