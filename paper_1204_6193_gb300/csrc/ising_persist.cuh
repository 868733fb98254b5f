// ising_persist.cuh -- the persistent fused checkerboard kernel.
//
// One cooperative launch runs many sweeps.  The grid works through a list
// of row strips ("segments") of one or more lattices; each thread block
// keeps its strips, plus one halo row above and below, in shared memory as
// two colour planes, and each thread keeps the generator state of its
// streams in registers for the whole launch: random numbers are consumed
// where they are drawn and never touch memory (the state load/store per
// tile that Sec. 2 identifies as the cost of the application test happens
// once per launch).  After each half-sweep a strip publishes its two
// boundary rows of the colour just updated and waits (bounded) only for
// the strips above and below it; a strip that holds a whole lattice
// refreshes its halo from itself.  In multi-hit mode (k_hits > 0) the
// strips of one coarse colour take k sweeps of their own rows between two
// exchanges, which then carry both colours of the boundary rows.
#pragma once

#include "ising_common.cuh"

namespace rngx {

constexpr int kPersistMaxSegs = 32;   // segments per thread block
constexpr uint64_t kWaitBudgetNs = 2000000000ull;  // default: 2 s per neighbour wait

struct PersistArgs {
    const LatDev *lats;
    const SegDev *segs;
    const uint32_t *cta_seg;   // segments of block b: [cta_seg[b], cta_seg[b+1])
    uint8_t *halo;             // per segment: 2 slots x 2 rows (first, last) x 2 colours x halo_row_bytes
    uint32_t halo_row_bytes;
    uint64_t halo_bytes;       // size of the halo buffer (bounds-check build)
    int *err;
    uint64_t n_sweeps;
    uint64_t sweep0;           // sweeps of the same call before this launch
    uint32_t measure_every;    // measure after sweeps sweep0+t+1 that are multiples
    int32_t mute_seg;          // test hook: this segment never publishes (-1: none)
    uint64_t wait_budget_ns;   // limit of one neighbour wait
    uint32_t k_hits;           // 0: exact checkerboard; k > 0: multi-hit rounds of k sweeps per strip phase
    uint32_t fixed_slots;      // 1: the plan fixes each slot's role (kernel modes 2, 3); 2: one whole lattice per block
                               // (mode 4); 3: one strip per block of split roles with a polling warp (mode 5)
};

struct alignas(16) SegLocal {  // per-segment constants held in shared memory
    // the site update's constants first, as two 16-byte words (one shared
    // load each): half, G, pstride, W and t4, t8, a_max, R
    uint32_t half, G, pstride, W;
    uint32_t t4, t8;           // T4, T8 below 2^32 (beta > 0)
    int32_t a_max;             // flips with a <= a_max always: 0, or 2 / 4 where T4 / T8 = 2^32
    uint32_t R;
    uint32_t L, y0, off, lat, coarse;
    uint32_t hd;               // halo rows above and below the strip (1; 2 in kernel mode 6)
    int32_t up, down, gid;
    uint64_t s0, prefix, T4, T8;
    uint64_t n_valid, n_inst;  // streams with sites; generator instances
    DevParams rng;             // the lattice's generator (position at launch start)
};

template <int LAYOUT>
__device__ __forceinline__ uint32_t row_bytes(const SegLocal &S)
{
    return LAYOUT == ISING_INT8 ? S.half : S.W * 4u;
}

// Address of plane c, local row r (r in [-hd, R + hd - 1]) of a segment.
template <int LAYOUT>
__device__ __forceinline__ uint8_t *plane_row(uint8_t *smem, const SegLocal &S, int c, int r)
{
    const uint32_t rb = row_bytes<LAYOUT>(S);
    return smem + S.off + (static_cast<uint32_t>(c) * (S.R + 2 * S.hd) + static_cast<uint32_t>(r + static_cast<int>(S.hd))) * rb;
}

// Global spins -> shared planes for rows y0-hd .. y0+R+hd-1 (all threads).
template <int LAYOUT>
__device__ void load_segment(uint8_t *smem, const SegLocal &S, const void *spins)
{
    const int rows = static_cast<int>(S.R + 2 * S.hd);
    if (LAYOUT == ISING_INT8) {
        const int8_t *g = static_cast<const int8_t *>(spins);
        const uint32_t total = rows * S.L;
        for (uint32_t idx = threadIdx.x; idx < total; idx += blockDim.x) {
            const int r = static_cast<int>(idx / S.L) - static_cast<int>(S.hd);
            const uint32_t x = idx % S.L;
            const uint32_t y = (S.y0 + S.L + r) % S.L;
            const int c = (x + y) & 1;
            int8_t *dst = reinterpret_cast<int8_t *>(plane_row<LAYOUT>(smem, S, c, r)) + (x >> 1);
            if (RNGX_IDX_OK(static_cast<size_t>(y) * S.L + x, static_cast<uint64_t>(S.L) * S.L, kSitePersist + __LINE__) &&
                RNGX_SMEM_OK(dst, smem, 1, kSitePersist + __LINE__))
                *dst = g[static_cast<size_t>(y) * S.L + x];
        }
    } else {
        const uint32_t *g = static_cast<const uint32_t *>(spins);
        const uint32_t total = 2 * rows * S.W;
        for (uint32_t idx = threadIdx.x; idx < total; idx += blockDim.x) {
            const int c = idx / (rows * S.W);
            const uint32_t rem = idx % (rows * S.W);
            const int r = static_cast<int>(rem / S.W) - static_cast<int>(S.hd);
            const uint32_t w = rem % S.W;
            const uint32_t y = (S.y0 + S.L + r) % S.L;
            uint32_t *dst = reinterpret_cast<uint32_t *>(plane_row<LAYOUT>(smem, S, c, r)) + w;
            const size_t gi = static_cast<size_t>(c) * S.L * S.W + static_cast<size_t>(y) * S.W + w;
            if (RNGX_IDX_OK(gi, 2ull * S.L * S.W, kSitePersist + __LINE__) && RNGX_SMEM_OK(dst, smem, 4, kSitePersist + __LINE__))
                *dst = g[gi];
        }
    }
}

template <int LAYOUT>
__device__ void store_segment(uint8_t *smem, const SegLocal &S, void *spins)
{
    if (LAYOUT == ISING_INT8) {
        int8_t *g = static_cast<int8_t *>(spins);
        const uint32_t total = S.R * S.L;
        for (uint32_t idx = threadIdx.x; idx < total; idx += blockDim.x) {
            const int r = static_cast<int>(idx / S.L);
            const uint32_t x = idx % S.L;
            const uint32_t y = S.y0 + r;
            const int c = (x + y) & 1;
            const int8_t *src = reinterpret_cast<int8_t *>(plane_row<LAYOUT>(smem, S, c, r)) + (x >> 1);
            if (RNGX_IDX_OK(static_cast<size_t>(y) * S.L + x, static_cast<uint64_t>(S.L) * S.L, kSitePersist + __LINE__) &&
                RNGX_SMEM_OK(src, smem, 1, kSitePersist + __LINE__))
                g[static_cast<size_t>(y) * S.L + x] = *src;
        }
    } else {
        uint32_t *g = static_cast<uint32_t *>(spins);
        const uint32_t total = 2 * S.R * S.W;
        for (uint32_t idx = threadIdx.x; idx < total; idx += blockDim.x) {
            const int c = idx / (S.R * S.W);
            const uint32_t rem = idx % (S.R * S.W);
            const int r = static_cast<int>(rem / S.W);
            const uint32_t w = rem % S.W;
            const uint32_t *src = reinterpret_cast<uint32_t *>(plane_row<LAYOUT>(smem, S, c, r)) + w;
            const size_t gi = static_cast<size_t>(c) * S.L * S.W + static_cast<size_t>(S.y0 + r) * S.W + w;
            if (RNGX_IDX_OK(gi, 2ull * S.L * S.W, kSitePersist + __LINE__) && RNGX_SMEM_OK(src, smem, 4, kSitePersist + __LINE__))
                g[gi] = *src;
        }
    }
}

// Partial E (bonds with a colour-0 endpoint in the strip's rows) and M.
template <int LAYOUT>
__device__ void strip_energy(uint8_t *smem, const SegLocal &S, long long &E, long long &M)
{
    E = 0;
    M = 0;
    if (LAYOUT == ISING_INT8) {
        const uint32_t total = S.R * S.half;
        for (uint32_t idx = threadIdx.x; idx < total; idx += blockDim.x) {
            const int r = static_cast<int>(idx / S.half);
            const uint32_t xh = idx % S.half;
            const uint32_t y = S.y0 + r;
            const uint32_t p = y & 1u;  // colour 0
            const int8_t *o = reinterpret_cast<const int8_t *>(plane_row<LAYOUT>(smem, S, 1, r));
            const int s0 = reinterpret_cast<const int8_t *>(plane_row<LAYOUT>(smem, S, 0, r))[xh];
            const int s1 = o[xh];
            const int nn = o[col_left(xh, p, S.half)] + o[col_right(xh, p, S.half)] +
                           reinterpret_cast<const int8_t *>(plane_row<LAYOUT>(smem, S, 1, r - 1))[xh] +
                           reinterpret_cast<const int8_t *>(plane_row<LAYOUT>(smem, S, 1, r + 1))[xh];
            E -= s0 * nn;
            M += s0 + s1;
        }
    } else {
        const uint32_t total = S.R * S.W;
        for (uint32_t idx = threadIdx.x; idx < total; idx += blockDim.x) {
            const int r = static_cast<int>(idx / S.W);
            const uint32_t w = idx % S.W;
            const uint32_t y = S.y0 + r;
            const uint32_t *o = reinterpret_cast<const uint32_t *>(plane_row<LAYOUT>(smem, S, 1, r));
            const uint32_t own = reinterpret_cast<const uint32_t *>(plane_row<LAYOUT>(smem, S, 0, r))[w];
            const uint32_t up = reinterpret_cast<const uint32_t *>(plane_row<LAYOUT>(smem, S, 1, r - 1))[w];
            const uint32_t dn = reinterpret_cast<const uint32_t *>(plane_row<LAYOUT>(smem, S, 1, r + 1))[w];
            uint32_t lft, rgt;
            if ((y & 1u) == 0) {  // p = 0: left = xh - 1, right = xh
                lft = (o[w] << 1) | (o[w == 0 ? S.W - 1 : w - 1] >> 31);
                rgt = o[w];
            } else {              // p = 1: left = xh, right = xh + 1
                lft = o[w];
                rgt = (o[w] >> 1) | (o[w + 1 == S.W ? 0 : w + 1] << 31);
            }
            const int U = __popc(own ^ lft) + __popc(own ^ rgt) + __popc(own ^ up) + __popc(own ^ dn);
            E += 2 * U - 4 * 32;
            M += 64 - 2 * (__popc(own) + __popc(o[w]));
        }
    }
}

__device__ __forceinline__ long long block_sum(long long v, long long *red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    long long s = 0;
    if (threadIdx.x == 0)
        for (int i = 0; i < static_cast<int>(blockDim.x >> 5); i++) s += red[i];
    return s;  // valid in thread 0
}

// One stream slot of a thread: which strip, which stream, where its sites
// are, and the warp-uniform flags the passes select on (all fixed for a
// launch, so computed once).
struct StreamSlot {
    uint32_t seg;            // strip index in the block
    uint32_t xh0;            // first column of its sites
    uint32_t base;           // shared-memory offset of the slot's row in plane 0
    uint32_t s;              // stream (instance) index in its lattice (s G < L^2/2 <= 2^31)
    uint32_t flags;          // SL_* bits
    __device__ __forceinline__ bool in() const { return flags & 1u; }
    __device__ __forceinline__ bool val() const { return flags & 2u; }
};
enum : uint32_t {
    SL_IN = 1u,         // inside the block's stream range
    SL_VAL = 2u,        // owns sites
    SL_WARP_IN = 4u,    // some lane of the warp is inside
    SL_WARP_BND = 8u,   // some lane of the warp holds a first or last row of the strip
    SL_COARSE = 16u,    // the strip's coarse colour is 1 (multi-hit phases)
    SL_ODD_ROW = 32u,   // the sites' row is odd
    SL_ROW_FIRST = 64u, // the slot's sites start its row (left neighbour wraps)
    SL_ROW_LAST = 128u, // the slot's sites end its row (right neighbour wraps)
    SL_DUP_DOWN = 256u, // whole lattice, first row: its flips also go to the halo row below the last
    SL_DUP_UP = 512u,   // whole lattice, last row: its flips also go to the halo row above the first
    SL_MS_PAIR = 1024u, // multispin, G = 2: lanes 16h .. 16h+15 hold the 16 streams of one word, in bit order
    // kernel mode 6 (halo of two rows, one exchange per sweep): the phases a slot takes part in
    SL_PH_A = 2048u,    // colour 0, the rows between the first and the last (no halo needed)
    SL_PH_B = 4096u,    // colour 0, the first and last rows and the halo rows -1 and R (after the poll)
    SL_PH_C = 8192u,    // colour 1, rows 0, 1, R-2, R-1 (the rows published)
    SL_PH_D = 16384u,   // colour 1, rows 2 .. R-3
    SL_REPLICA = 32768u // a copy of a neighbour's stream (halo row -1 or R): never stored
};

template <int LAYOUT>
__device__ __forceinline__ void finish_slot(const SegLocal &sg, bool in, bool val, StreamSlot &o)
{
    const uint32_t q0 = o.s * sg.G;
    const uint32_t row = q0 / sg.half;
    o.xh0 = q0 - row * sg.half;
    o.base = sg.off + (row - sg.y0 + sg.hd) * row_bytes<LAYOUT>(sg);
    const bool wi = __any_sync(0xffffffffu, in);
    const bool wb = __any_sync(0xffffffffu, in && (row == sg.y0 || row + 1 == sg.y0 + sg.R));
    // multispin with two sites per stream: every lane inside the block holds
    // sites 2l, 2l + 1 (l = lane mod 16) of its word
    const bool pair = LAYOUT != ISING_INT8 && sg.G == 2 &&
                      __all_sync(0xffffffffu, !in || (o.xh0 & 31u) == 2u * (threadIdx.x & 15u));
    o.flags = (in ? SL_IN : 0u) | (val ? SL_VAL : 0u) | (wi ? SL_WARP_IN : 0u) | (wb ? SL_WARP_BND : 0u) |
              (pair ? SL_MS_PAIR : 0u) |
              (sg.coarse ? SL_COARSE : 0u) | ((row & 1u) ? SL_ODD_ROW : 0u) | (o.xh0 == 0 ? SL_ROW_FIRST : 0u) |
              (o.xh0 + sg.G == sg.half ? SL_ROW_LAST : 0u) | (sg.up < 0 && row == sg.y0 ? SL_DUP_DOWN : 0u) |
              (sg.up < 0 && row + 1 == sg.y0 + sg.R ? SL_DUP_UP : 0u);
}

template <int LAYOUT>
__device__ __forceinline__ void setup_slot(const SegLocal *S, uint32_t nseg, uint64_t prefix_end, uint64_t f,
                                           StreamSlot &o)
{
    const bool in = f < prefix_end;
    uint32_t j = 0;
    while (j + 1 < nseg && f >= S[j + 1].prefix) j++;
    o.seg = j;
    o.s = static_cast<uint32_t>(S[j].s0 + (in ? f - S[j].prefix : 0));
    finish_slot<LAYOUT>(S[j], in, in && o.s < S[j].n_valid, o);
}

// Metropolis acceptance of a site whose aligned-neighbour sum is
// a = s_i sum_nn s_j (dE = 2a): always for a <= 0, else iff r < T[2a].
__device__ __forceinline__ bool accept_a(int a, uint32_t r, uint64_t T4, uint64_t T8)
{
    return a <= 0 || static_cast<uint64_t>(r) < (a == 2 ? T4 : T8);
}

// Draws G numbers from the slot's generator and updates its G colour-c
// sites in shared memory (all 32 lanes of the warp call this together).
// DUP: a whole lattice's edge rows also write their flips into the halo
// rows (the other edge's copy), so that no copy pass is needed.
template <int KIND, int LAYOUT, bool DUP = false>
__device__ __forceinline__ void update_slot(uint8_t *smem, const SegLocal &sg, const StreamSlot &sl, Gen<KIND> &gen,
                                            int c, int lane)
{
    const uint32_t p = (c + ((sl.flags & SL_ODD_ROW) ? 1u : 0u)) & 1u;
    // (the field order of SegLocal makes these two 16-byte shared loads)
    const uint4 q0 = *reinterpret_cast<const uint4 *>(&sg.half), q1 = *reinterpret_cast<const uint4 *>(&sg.t4);
    const uint32_t half = q0.x, G = q0.y, pstride = q0.z, W_ = q0.w;
    const uint32_t t4_ = q1.x, t8_ = q1.y;
    const int a_max_ = static_cast<int>(q1.z);
    const uint64_t T4 = sg.T4, T8 = sg.T8;
    uint8_t *own_row = smem + sl.base + (c ? pstride : 0u);
    uint8_t *o_row = smem + sl.base + (c ? 0u : pstride);
    if (LAYOUT == ISING_INT8) {
        int8_t *own = reinterpret_cast<int8_t *>(own_row);
        const int8_t *o = reinterpret_cast<const int8_t *>(o_row);
        const int8_t *ou = o - half, *od = o + half;
        if (G == 2) {
            // the two sites xh, xh + 1 (xh even) as one 16-bit word, and so
            // their neighbours above, below and in the row (xh and every row
            // offset are even).  Per byte, (s ^ n) & 2 is 2 when n is
            // anti-aligned with s (+1 = 0x01, -1 = 0xff), so one sum of four
            // masked words gives 2k, k the anti-aligned neighbours, of both
            // sites at once (2k <= 8: no carries); s_i sum_nn s_j = 4 - 2k.
            // Draws are taken in site order before either update.
            const uint32_t r0 = gen.next(), r1 = gen.next();
            if (!sl.val()) return;
            const int8_t *ox = o + sl.xh0;
            int8_t *ow = own + sl.xh0;
            const int hf = static_cast<int>(half);
            // the row neighbour outside the pair: left of xh (p = 0) or right
            // of xh + 1 (p = 1), wrapped at the row's ends
            const int eo = p ? ((sl.flags & SL_ROW_LAST) ? 2 - hf : 2) : ((sl.flags & SL_ROW_FIRST) ? hf - 1 : -1);
            if (!RNGX_SMEM_OK(ow, smem, 2, kSitePersist + __LINE__) || !RNGX_SMEM_OK(ox, smem, 2, kSitePersist + __LINE__) ||
                !RNGX_SMEM_OK(ox + eo, smem, 1, kSitePersist + __LINE__) ||
                !RNGX_SMEM_OK(ox - hf, smem, 2, kSitePersist + __LINE__) || !RNGX_SMEM_OK(ox + hf, smem, 2, kSitePersist + __LINE__))
                return;
            if constexpr (DUP) {
                if ((sl.flags & (SL_DUP_DOWN | SL_DUP_UP)) &&
                    !RNGX_SMEM_OK(ow + static_cast<int>(sg.R * half) * ((sl.flags & SL_DUP_DOWN) ? 1 : -1), smem, 2,
                                  kSitePersist + __LINE__))
                    return;
            }
            const uint32_t o2 = *reinterpret_cast<const uint16_t *>(ow);
            const uint32_t m2 = *reinterpret_cast<const uint16_t *>(ox);
            const uint32_t u2 = *reinterpret_cast<const uint16_t *>(ox - hf);
            const uint32_t d2 = *reinterpret_cast<const uint16_t *>(ox + hf);
            const uint32_t e = static_cast<uint8_t>(ox[eo]);
            // row neighbours of (xh, xh + 1) in the (low, high) bytes:
            // p = 0: (e, m.lo) and (m.lo, m.hi); p = 1: (m.lo, m.hi) and (m.hi, e)
            const uint32_t na = p ? m2 : (((m2 << 8) | e) & 0xffffu);
            const uint32_t nb = p ? ((m2 >> 8) | (e << 8)) : m2;
            const uint32_t k2 = ((o2 ^ u2) & 0x0202u) + ((o2 ^ d2) & 0x0202u) + ((o2 ^ na) & 0x0202u) +
                                ((o2 ^ nb) & 0x0202u);
            const uint32_t k0 = k2 & 0xffu, k1 = k2 >> 8;
            // flip when 4 - 2k <= a_max (every k >= 2, and every k where
            // T = 2^32), else iff r < T(4 - 2k): T8 for k = 0, T4 for k = 1
            const uint32_t kf = static_cast<uint32_t>(4 - a_max_);
            const uint32_t t4 = t4_, t8 = t8_;
            const bool f0 = k0 >= kf || r0 < (k0 ? t4 : t8), f1 = k1 >= kf || r1 < (k1 ? t4 : t8);
            if (f0 || f1) {
                // -s = s ^ 0xfe for s = 0x01, 0xff
                const uint16_t n2 = static_cast<uint16_t>(o2 ^ ((f0 ? 0x00feu : 0u) | (f1 ? 0xfe00u : 0u)));
                *reinterpret_cast<uint16_t *>(ow) = n2;
                if constexpr (DUP) {
                    if (sl.flags & (SL_DUP_DOWN | SL_DUP_UP))
                        *reinterpret_cast<uint16_t *>(ow + static_cast<int>(sg.R * half) *
                                                                ((sl.flags & SL_DUP_DOWN) ? 1 : -1)) = n2;
                }
            }
            return;
        }
        for (uint32_t g = 0; g < G; g++) {
            const uint32_t rr = gen.next();
            if (!sl.val()) continue;
            const uint32_t xh = sl.xh0 + g;
            if (!RNGX_IDX_OK(xh, half, kSitePersist + __LINE__) || !RNGX_SMEM_OK(ou + xh, smem, 1, kSitePersist + __LINE__) ||
                !RNGX_SMEM_OK(od + xh, smem, 1, kSitePersist + __LINE__) || !RNGX_SMEM_OK(own + xh, smem, 1, kSitePersist + __LINE__))
                continue;
            const int nn = o[col_left(xh, p, half)] + o[col_right(xh, p, half)] + ou[xh] + od[xh];
            const int sp = own[xh];
            if (accept_a(sp * nn, rr, T4, T8)) {
                own[xh] = static_cast<int8_t>(-sp);
                if constexpr (DUP) {
                    if (sl.flags & (SL_DUP_DOWN | SL_DUP_UP))
                        own[xh + static_cast<int>(sg.R * half) * ((sl.flags & SL_DUP_DOWN) ? 1 : -1)] =
                            static_cast<int8_t>(-sp);
                }
            }
        }
    } else if (G == 2 && (sl.flags & SL_MS_PAIR)) {
        // Two sites per stream, and the 16 streams of a word in 16 lanes in
        // bit order (half-warp h holds word h of the warp's two).  The
        // anti-aligned neighbours k of all 32 sites of the word are counted
        // at once, bit-sliced, from the word, its row neighbours (shifted by
        // one site, the carry bit from the next or previous word) and the
        // words above and below, and kept as three masks: k >= 2 (always
        // flips, s_i sum_nn s_j = 4 - 2k <= 0), k = 1 (flips iff r < T4) and
        // k = 0 (iff r < T8).  Each lane sets its two draws' acceptance bits
        // at its sites' positions; one OR-reduction per half-warp then gives
        // the word's flips, which its first lane applies.
        const uint32_t W = W_;
        uint32_t *own = reinterpret_cast<uint32_t *>(own_row);
        const uint32_t *o = reinterpret_cast<const uint32_t *>(o_row);
        const uint32_t r0 = gen.next(), r1 = gen.next();
        const uint32_t wi = sl.xh0 >> 5, b0 = sl.xh0 & 31u;
        const bool ok = sl.val() && RNGX_IDX_OK(wi, W, kSitePersist + __LINE__) &&
                        RNGX_SMEM_OK(o - W + wi, smem, 4, kSitePersist + __LINE__) &&
                        RNGX_SMEM_OK(o + W + wi, smem, 4, kSitePersist + __LINE__) &&
                        RNGX_SMEM_OK(own + wi, smem, 4, kSitePersist + __LINE__);
        uint32_t fl = 0, ow = 0, ge2 = 0;
        if (ok) {
            ow = own[wi];
            const uint32_t mw = o[wi];
            // the row neighbours' word: the next one (p = 1) or the previous
            // one (p = 0), wrapped; its edge bit enters the shifted word
            const uint32_t nwi = p ? (wi + 1 == W ? 0u : wi + 1) : (wi == 0 ? W - 1 : wi - 1);
            const uint32_t nw = o[nwi];
            const uint32_t n2 = p ? __funnelshift_r(mw, nw, 1) : __funnelshift_l(nw, mw, 1);
            const uint32_t up = o[wi - W], dn = o[wi + W];
            // anti-aligned indicators a1..a4 = ow ^ (mw, n2, up, dn), added
            // as two half adders: s = a1 ^ a2 (ow cancels), c = a1 & a2
            const uint32_t s1 = mw ^ n2, c1 = (ow ^ mw) & (ow ^ n2);
            const uint32_t s2 = up ^ dn, c2 = (ow ^ up) & (ow ^ dn);
            const uint32_t k0 = s1 ^ s2;  // the low bit of k
            // k >= 2: c1 c2 | (c1 ^ c2) t | (c1 ^ c2 ^ t) = c1 | c2 | t, t = s1 s2
            ge2 = c1 | c2 | (s1 & s2);
            // below k = 2 a site flips iff r < T4 (k = 1: k0 set) or r < T8
            // (k = 0); T = 2^32 (a_max) accepts every draw
            const bool f4 = a_max_ >= 2, f8 = a_max_ >= 4;
            const uint32_t kb = k0 >> b0;
            const bool p0 = (kb & 1u) ? (f4 || r0 < t4_) : (f8 || r0 < t8_);
            const bool p1 = (kb & 2u) ? (f4 || r1 < t4_) : (f8 || r1 < t8_);
            fl = ((p0 ? 1u : 0u) | (p1 ? 2u : 0u)) << b0;
        }
        // the word's flips: k >= 2 (the same in all its lanes) and the
        // lanes' accepted draws
        const uint32_t fa = __reduce_or_sync(0xffffffffu, lane < 16 ? fl : 0u);
        const uint32_t fb = __reduce_or_sync(0xffffffffu, lane < 16 ? 0u : fl);
        const uint32_t fw = (lane < 16 ? fa : fb) | ge2;
        if (ok && (lane & 15) == 0 && fw) {
            own[wi] = ow ^ fw;
            if constexpr (DUP) {  // the halo copy of a whole lattice's edge row
                if (sl.flags & (SL_DUP_DOWN | SL_DUP_UP)) {
                    uint32_t *cp = own + wi + static_cast<int>(sg.R * W) * ((sl.flags & SL_DUP_DOWN) ? 1 : -1);
                    if (RNGX_SMEM_OK(cp, smem, 4, kSitePersist + __LINE__)) *cp = ow ^ fw;
                }
            }
        }
    } else {
        // any G, site by site: the warp's 32 G sites are G consecutive words
        // of plane c, assembled by one OR-reduction each
        const uint32_t W = W_;
        const uint32_t *own = reinterpret_cast<const uint32_t *>(own_row);
        const uint32_t *o = reinterpret_cast<const uint32_t *>(o_row);
        const uint32_t *ou = o - W, *od = o + W;
        const uint32_t lq0 = lane * G;
        uint32_t c_lo = 0, c_hi = 0;
        for (uint32_t g = 0; g < G; g++) {
            const uint32_t rr = gen.next();
            if (!sl.val()) continue;
            const uint32_t xh = sl.xh0 + g;
            const int nn = bit_spin(o, col_left(xh, p, half)) + bit_spin(o, col_right(xh, p, half)) +
                           bit_spin(ou, xh) + bit_spin(od, xh);
            const int sp = bit_spin(own, xh);
            if (accept_a(sp * nn, rr, T4, T8)) {
                const uint32_t lq = lq0 + g;
                if ((lq >> 5) == (lq0 >> 5)) c_lo |= 1u << (lq & 31);
                else c_hi |= 1u << (lq & 31);
            }
        }
        // the warp's first word, counted from row 0 of plane c (rows are
        // contiguous; a halo copy's row -1 gives a negative count)
        const uint32_t base0 = __shfl_sync(0xffffffffu, sl.base, 0), x0 = __shfl_sync(0xffffffffu, sl.xh0, 0);
        uint32_t *plane_c = reinterpret_cast<uint32_t *>(plane_row<LAYOUT>(smem, sg, c, 0));
        const int wbase = static_cast<int>(reinterpret_cast<uint32_t *>(smem + base0 + (c ? pstride : 0u)) - plane_c) +
                          static_cast<int>(x0 >> 5);
        const int own_words = static_cast<int>(sg.R * W), lo = -static_cast<int>(sg.hd - 1) * static_cast<int>(W),
                  hi = own_words + static_cast<int>(sg.hd - 1) * static_cast<int>(W);
        for (uint32_t m = 0; m < G; m++) {
            const uint32_t mine = ((lq0 >> 5) == m ? c_lo : 0u) | ((lq0 >> 5) + 1 == m ? c_hi : 0u);
            const uint32_t word = __reduce_or_sync(0xffffffffu, mine);
            const int wm = wbase + static_cast<int>(m);
            if (lane == 0 && word && wm >= lo && wm < hi && RNGX_SMEM_OK(plane_c + wm, smem, 4, kSitePersist + __LINE__)) {
                plane_c[wm] ^= word;
                if constexpr (DUP) {  // the halo copies of the whole lattice's edge rows
                    if (wm < static_cast<int>(W)) plane_c[wm + own_words] ^= word;
                    if (wm >= own_words - static_cast<int>(W)) plane_c[wm - own_words] ^= word;
                }
            }
        }
    }
}

__device__ __forceinline__ void st_relaxed_u64(uint64_t *p, uint64_t v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t *p)
{
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Which warps a pass updates: those holding a first or last row of their
// strip, the others, or all warps of the strips of one coarse colour
// (multi-hit phases).  A warp is classified as a whole, so warp-wide steps
// see all 32 lanes.
// SEL_ALL: every warp (blocks that hold whole lattices only).
enum { SEL_BOUNDARY = 0, SEL_INTERIOR = 1, SEL_COARSE0 = 2, SEL_COARSE1 = 3, SEL_ALL = 4 };

__device__ __forceinline__ bool warp_selected(const StreamSlot &sl, int sel)
{
    if (!(sl.flags & SL_WARP_IN)) return false;
    if (sel == SEL_ALL) return true;
    if (sel >= SEL_COARSE0) return ((sl.flags & SL_COARSE) != 0) == (sel == SEL_COARSE1);
    return ((sl.flags & SL_WARP_BND) != 0) == (sel == SEL_BOUNDARY);
}

// Updates the colour-c sites of the selected warps.  pos_off is the number
// of draws every updated stream made earlier in this launch (streamed
// states reload their position from it).
template <int KIND, int LAYOUT, int SMAX>
__device__ __forceinline__ void update_pass(uint8_t *smem, const SegLocal *S, uint32_t nseg, uint64_t prefix_end,
                                            bool resident, Gen<KIND> (&gen)[SMAX], const StreamSlot (&slot)[SMAX],
                                            uint64_t pos_off, int c, int lane, int sel)
{
    if (resident) {
#pragma unroll
        for (int k = 0; k < SMAX; k++) {
            if (!warp_selected(slot[k], sel)) continue;
            update_slot<KIND, LAYOUT>(smem, S[slot[k].seg], slot[k], gen[k], c, lane);
        }
        return;
    }
    // streamed states: strip by strip, one stream per thread per step (the
    // strips' stream counts are multiples of 32, so warps never straddle two)
    for (uint32_t j = 0; j < nseg; j++) {
        const SegLocal &sg = S[j];
        if ((sel == SEL_COARSE0 || sel == SEL_COARSE1) && sg.coarse != static_cast<uint32_t>(sel - SEL_COARSE0))
            continue;
        const uint64_t count = (j + 1 < nseg ? S[j + 1].prefix : prefix_end) - sg.prefix;
        for (uint64_t base = 0; base < count; base += blockDim.x) {
            const uint64_t f = base + threadIdx.x;
            StreamSlot sl;
            sl.seg = j;
            const bool in = f < count;
            sl.s = static_cast<uint32_t>(sg.s0 + (in ? f : 0));
            finish_slot<LAYOUT>(sg, in, in && sl.s < sg.n_valid, sl);
            if (!warp_selected(sl, sel)) continue;
            DevParams rp = sg.rng;
            rp.pos += pos_off;
            Gen<KIND> g;
            g.load(rp, sl.s < sg.n_inst ? sl.s : sg.n_inst - 1);
            update_slot<KIND, LAYOUT>(smem, sg, sl, g, c, lane);
            if (sl.in() && sl.s < sg.n_inst) g.store(rp, sl.s);
        }
    }
}

// Resident states: a pass updates the slots whose warp it selects (sel as
// in warp_selected).
template <int KIND, int LAYOUT, int SMAX>
__device__ __forceinline__ void update_resident(uint8_t *smem, const SegLocal *S, Gen<KIND> (&gen)[SMAX],
                                                const StreamSlot (&slot)[SMAX], int c, int lane, int sel)
{
#pragma unroll
    for (int k = 0; k < SMAX; k++)
        if (warp_selected(slot[k], sel)) update_slot<KIND, LAYOUT>(smem, S[slot[k].seg], slot[k], gen[k], c, lane);
}

// Halo buffer: per strip, 2 slots x 2 rows (first, last) x 2 colours.
__device__ __forceinline__ uint64_t *halo_row(const PersistArgs &a, int gid, uint32_t slot, int row, int colour)
{
    return reinterpret_cast<uint64_t *>(
        a.halo + ((((static_cast<size_t>(gid) * 2 + slot) * 2 + row) * 2 + colour)) * a.halo_row_bytes);
}

// Publishes the first and last rows of colour c of strip sg as 64-bit
// (tag, 32 data bits) words: one relaxed atomic store each, no fence.
// Threads tid = 0 .. nthr-1 share the stores.
template <int LAYOUT>
__device__ __forceinline__ void publish_rows_by(uint8_t *smem, const SegLocal &sg, const PersistArgs &a, uint32_t slot,
                                                uint32_t tag, int c, uint32_t tid, uint32_t nthr)
{
    if (sg.gid == a.mute_seg) return;  // test hook: a strip that never publishes
    const uint32_t words = row_bytes<LAYOUT>(sg) / 4;
    const uint32_t *row0 = reinterpret_cast<const uint32_t *>(plane_row<LAYOUT>(smem, sg, c, 0));
    const uint32_t *rowl = reinterpret_cast<const uint32_t *>(plane_row<LAYOUT>(smem, sg, c, sg.R - 1));
    uint64_t *d0 = halo_row(a, sg.gid, slot, 0, c), *d1 = halo_row(a, sg.gid, slot, 1, c);
    const uint64_t t = static_cast<uint64_t>(tag) << 32;
    [[maybe_unused]] const uint64_t *hb = reinterpret_cast<const uint64_t *>(a.halo);
    for (uint32_t i = tid; i < words; i += nthr) {
        if (!RNGX_IDX_OK(d0 + i - hb, a.halo_bytes / 8, kSitePersist + __LINE__) ||
            !RNGX_IDX_OK(d1 + i - hb, a.halo_bytes / 8, kSitePersist + __LINE__) ||
            !RNGX_SMEM_OK(row0 + i, smem, 4, kSitePersist + __LINE__) || !RNGX_SMEM_OK(rowl + i, smem, 4, kSitePersist + __LINE__))
            continue;
        st_relaxed_u64(d0 + i, t | row0[i]);
        st_relaxed_u64(d1 + i, t | rowl[i]);
    }
}

template <int LAYOUT>
__device__ __forceinline__ void publish_rows(uint8_t *smem, const SegLocal &sg, const PersistArgs &a, uint32_t slot,
                                             uint32_t tag, int c)
{
    publish_rows_by<LAYOUT>(smem, sg, a, slot, tag, c, threadIdx.x, blockDim.x);
}

// Polls the neighbours' rows of colour c into strip sg's halo rows (the up
// neighbour's last row above, the down neighbour's first row below) until
// their words carry `tag`; the wait is bounded by two clocks (the global ns
// timer and the SM cycle counter, at most 4 cycles per ns of budget).
template <int LAYOUT>
__device__ __forceinline__ bool poll_rows(uint8_t *smem, const SegLocal &sg, const PersistArgs &a, uint32_t slot,
                                          uint32_t tag, int c, uint64_t t0, long long c0)
{
    const uint32_t words = row_bytes<LAYOUT>(sg) / 4;
    const uint64_t *up_last = halo_row(a, sg.up, slot, 1, c), *dn_first = halo_row(a, sg.down, slot, 0, c);
    uint32_t *top = reinterpret_cast<uint32_t *>(plane_row<LAYOUT>(smem, sg, c, -1));
    uint32_t *bot = reinterpret_cast<uint32_t *>(plane_row<LAYOUT>(smem, sg, c, sg.R));
    [[maybe_unused]] const uint64_t *hb = reinterpret_cast<const uint64_t *>(a.halo);
    for (uint32_t i = threadIdx.x; i < 2 * words; i += blockDim.x) {
        const uint64_t *src = i < words ? up_last + i : dn_first + (i - words);
        // an index outside the halo buffer or the halo rows is recorded
        // and skipped, never waited on
        if (!RNGX_IDX_OK(src - hb, a.halo_bytes / 8, kSitePersist + __LINE__) ||
            !RNGX_SMEM_OK(i < words ? top + i : bot + (i - words), smem, 4, kSitePersist + __LINE__))
            continue;
        uint64_t v;
        uint32_t spins = 0;
        while (((v = ld_relaxed_u64(src)) >> 32) != tag) {
            // tight re-reads first (the word is usually one L2 round trip
            // away); every 32nd miss checks the clocks and the abort flag
            // and backs off briefly
            if ((++spins & 31u) == 0) {
                if (global_ns() - t0 > a.wait_budget_ns ||
                    static_cast<uint64_t>(clock64() - c0) > 4 * a.wait_budget_ns ||
                    ld_acquire(reinterpret_cast<const uint32_t *>(a.err)) != 0) {
                    atomicCAS(a.err, 0, RNG_ETIMEOUT);
                    return false;
                }
                __nanosleep(32);
            }
        }
        (i < words ? top[i] : bot[i - words]) = static_cast<uint32_t>(v);
    }
    return true;
}

// The same poll by one warp (lane = its lane) that does nothing else while
// the block's other warps update their rows: each lane keeps up to eight
// independent loads in flight and re-reads only the words whose tag is not
// there yet.  The wait is bounded like poll_rows', and ends early when
// another block has recorded an error.
template <int LAYOUT>
__device__ __forceinline__ bool poll_rows_warp(uint8_t *smem, const SegLocal &sg, const PersistArgs &a, uint32_t slot,
                                               uint32_t tag, int c, int lane)
{
    constexpr int K = 8;
    const uint32_t words = row_bytes<LAYOUT>(sg) / 4, total = 2 * words;
    const uint64_t *up_last = halo_row(a, sg.up, slot, 1, c), *dn_first = halo_row(a, sg.down, slot, 0, c);
    uint32_t *top = reinterpret_cast<uint32_t *>(plane_row<LAYOUT>(smem, sg, c, -1));
    uint32_t *bot = reinterpret_cast<uint32_t *>(plane_row<LAYOUT>(smem, sg, c, sg.R));
    [[maybe_unused]] const uint64_t *hb = reinterpret_cast<const uint64_t *>(a.halo);
    const uint64_t t0 = global_ns();
    const long long c0 = clock64();
    for (uint32_t base = 0; base < total; base += 32 * K) {
        uint32_t pend = 0;
#pragma unroll
        for (int k = 0; k < K; k++) {
            const uint32_t i = base + lane + 32 * k;
            // an index outside the halo buffer or the halo rows is recorded
            // and skipped, never waited on
            if (i < total &&
                RNGX_IDX_OK((i < words ? up_last + i : dn_first + (i - words)) - hb, a.halo_bytes / 8,
                            kSitePersist + __LINE__) &&
                RNGX_SMEM_OK(i < words ? top + i : bot + (i - words), smem, 4, kSitePersist + __LINE__))
                pend |= 1u << k;
        }
        uint32_t spins = 0;
        while (pend) {
            uint64_t v[K];
#pragma unroll
            for (int k = 0; k < K; k++) {
                const uint32_t i = base + lane + 32 * k;
                v[k] = ((pend >> k) & 1u) ? ld_relaxed_u64(i < words ? up_last + i : dn_first + (i - words)) : 0;
            }
#pragma unroll
            for (int k = 0; k < K; k++) {
                const uint32_t i = base + lane + 32 * k;
                if (((pend >> k) & 1u) && (v[k] >> 32) == tag) {
                    (i < words ? top[i] : bot[i - words]) = static_cast<uint32_t>(v[k]);
                    pend &= ~(1u << k);
                }
            }
            if (pend && (++spins & 7u) == 0 &&
                (global_ns() - t0 > a.wait_budget_ns || static_cast<uint64_t>(clock64() - c0) > 4 * a.wait_budget_ns ||
                 ld_acquire(reinterpret_cast<const uint32_t *>(a.err)) != 0)) {
                atomicCAS(a.err, 0, RNG_ETIMEOUT);
                return false;
            }
        }
    }
    return true;
}

// ---- kernel mode 6: a halo of two rows, one exchange per sweep.
// Each strip also updates colour 0 of the rows just outside it (-1 and R),
// with copies of the neighbours' streams that draw exactly as the owners
// do, so that colour 1 of its own rows needs nothing from outside; after
// colour 1 of its rows it publishes six half-rows (rows 0, 1, R-2, R-1),
// which the neighbours take into rows -2 .. -1 and R .. R+1 before their
// next sweep's edge rows.
constexpr int kNoRow = -1000;

// Local row held by slot k, cell `cell` (cell = thread / streams per row) of
// a strip of R rows (4 <= R <= 10): the edge rows and the halo copies each
// fill one cell of different warps, so that each phase spreads over the
// block.  slot 0: rows 0, R-1, D2, D3; slot 1: D0, D1, 1, R-2; slot 2: D4,
// D5, -1, R; D_i = 2 + i, the rows 2 .. R-3.
__device__ __forceinline__ int mode6_row(int k, uint32_t cell, int R)
{
    auto D = [&](int i) { return 2 + i <= R - 3 ? 2 + i : kNoRow; };
    if (cell >= 4) return kNoRow;
    if (k == 0) return cell == 0 ? 0 : (cell == 1 ? R - 1 : D(static_cast<int>(cell)));
    if (k == 1) return cell == 0 ? D(0) : (cell == 1 ? D(1) : (cell == 2 ? 1 : R - 2));
    return cell == 0 ? D(4) : (cell == 1 ? D(5) : (cell == 2 ? -1 : R));
}

// Mode 6 halo buffer: per strip, 2 parities x 6 half-rows: the first row
// (colours 0, 1), the second row (colour 1), the last row (colours 0, 1), the
// second-last row (colour 1).
__device__ __forceinline__ uint64_t *halo_row6(const PersistArgs &a, int gid, uint32_t par, uint32_t which)
{
    return reinterpret_cast<uint64_t *>(a.halo + ((static_cast<size_t>(gid) * 2 + par) * 6 + which) * a.halo_row_bytes);
}

__device__ __forceinline__ void mode6_half_row(const SegLocal &sg, uint32_t which, int &row, int &colour)
{
    row = which <= 1 ? 0 : (which == 2 ? 1 : (which == 5 ? static_cast<int>(sg.R) - 2 : static_cast<int>(sg.R) - 1));
    colour = (which == 0 || which == 3) ? 0 : 1;
}

// Each thread publishes at most one word and polls at most one (6 half-rows
// of at most blockDim / 6 words): its addresses are worked out once per
// launch into shared tables (parity 0; parity 1 lies 6 half-rows further).
struct Mode6Tab {
    uint64_t *pub_dst;         // halo buffer word this thread publishes
    const uint64_t *poll_src;  // halo buffer word this thread polls
    uint32_t pub_src, poll_dst;  // shared-memory byte offsets of the word published / filled
};

template <int LAYOUT>
__device__ __forceinline__ void mode6_table(uint8_t *smem, const SegLocal &sg, const PersistArgs &a, Mode6Tab *tab)
{
    const uint32_t words = row_bytes<LAYOUT>(sg) / 4, i = threadIdx.x;
    Mode6Tab e{nullptr, nullptr, 0u, 0u};
    if (i < 6 * words) {
        const uint32_t which = i / words, w = i - which * words;
        int row, colour;
        mode6_half_row(sg, which, row, colour);
        e.pub_src = static_cast<uint32_t>(plane_row<LAYOUT>(smem, sg, colour, row) - smem) + 4 * w;
        e.pub_dst = halo_row6(a, sg.gid, 0, which) + w;
        // which 0..2: the upper neighbour's half-rows 3..5 into rows -1, -1, -2;
        // 3..5: the lower neighbour's 0..2 into rows R, R, R+1
        e.poll_src = which < 3 ? halo_row6(a, sg.up, 0, which + 3) + w : halo_row6(a, sg.down, 0, which - 3) + w;
        const int prow = which <= 1 ? -1 : (which == 2 ? -2 : (which == 5 ? static_cast<int>(sg.R) + 1 : static_cast<int>(sg.R)));
        const int pcol = (which == 0 || which == 3) ? 0 : 1;
        e.poll_dst = static_cast<uint32_t>(plane_row<LAYOUT>(smem, sg, pcol, prow) - smem) + 4 * w;
    }
    tab[threadIdx.x] = e;
}

// Publishes this thread's word as (tag, 32 data bits), one relaxed store.
__device__ __forceinline__ void publish6(uint8_t *smem, const SegLocal &sg, const PersistArgs &a, const Mode6Tab &e,
                                         uint32_t par, uint32_t tag)
{
    if (e.pub_dst == nullptr || sg.gid == a.mute_seg) return;  // mute_seg: test hook, a strip that never publishes
    uint64_t *dst = e.pub_dst + par * (6 * a.halo_row_bytes / 8);
    [[maybe_unused]] const uint64_t *hb = reinterpret_cast<const uint64_t *>(a.halo);
    const uint32_t *src = reinterpret_cast<const uint32_t *>(smem + e.pub_src);
    if (!RNGX_IDX_OK(dst - hb, a.halo_bytes / 8, kSitePersist + __LINE__) || !RNGX_SMEM_OK(src, smem, 4, kSitePersist + __LINE__))
        return;
    st_relaxed_u64(dst, (static_cast<uint64_t>(tag) << 32) | *src);
}

// Waits (bounded like poll_rows) for this thread's word to carry `tag` and
// puts its data into the halo; false when the wait ran out or another block
// recorded an error.
__device__ __forceinline__ bool poll6(uint8_t *smem, const PersistArgs &a, const Mode6Tab &e, uint32_t par,
                                      uint32_t tag)
{
    if (e.poll_src == nullptr) return true;
    const uint64_t *src = e.poll_src + par * (6 * a.halo_row_bytes / 8);
    [[maybe_unused]] const uint64_t *hb = reinterpret_cast<const uint64_t *>(a.halo);
    uint32_t *dst = reinterpret_cast<uint32_t *>(smem + e.poll_dst);
    if (!RNGX_IDX_OK(src - hb, a.halo_bytes / 8, kSitePersist + __LINE__) || !RNGX_SMEM_OK(dst, smem, 4, kSitePersist + __LINE__))
        return true;
    uint64_t v;
    uint32_t spins = 0;
    uint64_t t0 = 0;
    long long c0 = 0;
    while (((v = ld_relaxed_u64(src)) >> 32) != tag) {
        if (spins == 0) {
            t0 = global_ns();
            c0 = clock64();
        }
        if ((++spins & 31u) == 0) {
            if (global_ns() - t0 > a.wait_budget_ns || static_cast<uint64_t>(clock64() - c0) > 4 * a.wait_budget_ns ||
                ld_acquire(reinterpret_cast<const uint32_t *>(a.err)) != 0) {
                atomicCAS(a.err, 0, RNG_ETIMEOUT);
                return false;
            }
            __nanosleep(32);
        }
    }
    *dst = static_cast<uint32_t>(v);
    return true;
}

// Barrier 1 among the first nthr threads of the block (a multiple of 32).
__device__ __forceinline__ void bar_sync_first(uint32_t nthr)
{
    asm volatile("bar.sync 1, %0;" ::"r"(nthr) : "memory");
}

template <int LAYOUT>
__device__ void measure_strips(uint8_t *smem, const SegLocal *S, uint32_t nseg, const PersistArgs &a,
                               uint64_t meas_idx, long long *red)
{
    for (uint32_t j = 0; j < nseg; j++) {
        long long E, M;
        strip_energy<LAYOUT>(smem, S[j], E, M);
        const long long Es = block_sum(E, red);
        __syncthreads();
        const long long Ms = block_sum(M, red);
        if (threadIdx.x == 0) {
            int64_t *meas = a.lats[S[j].lat].meas;
            atomicAdd(reinterpret_cast<unsigned long long *>(meas + 2 * meas_idx), static_cast<unsigned long long>(Es));
            atomicAdd(reinterpret_cast<unsigned long long *>(meas + 2 * meas_idx + 1),
                      static_cast<unsigned long long>(Ms));
        }
        __syncthreads();
    }
}

// MODE selects the loop at compile time, so that each keeps its own
// register allocation: 0 the exact checkerboard and 1 the multi-hit rounds
// (a.k_hits > 0), both for any slot layout; 2 and 3 (SMAX = 2 only) the same
// for plans that fix each slot's role, so that a pass updates one slot with
// no per-slot selection (with 1024 threads, or two blocks of 512 per SM, the
// general loops do not fit the 64 registers a thread has):
//   2: multi-hit, thread slot 0 a stream of coarse colour 0, slot 1 one of
//      coarse colour 1 (block = a coarse-0 strip and a coarse-1 strip);
//   3: exact checkerboard, one strip per block, slot 0 the streams of its
//      first and last rows (the boundary pass), slot 1 those of the rows
//      between (the interior pass);
//   4: (SMAX = 1 only) exact checkerboard, every block one whole lattice
//      with resident states: a half-sweep is one pass and one barrier, the
//      edge rows writing their flips into the halo rows as well;
//   5: (SMAX = 2 only) exact checkerboard, one strip per block of roles
//      split by warp: the warps of the first and last rows update them and
//      publish them first, then all but the last warp update the rows
//      between, and the last warp holds no stream: it polls the
//      neighbours' rows for the whole half-sweep, so that their arrival
//      overlaps the interior work (one block of 1024 threads per SM).
//   6: (SMAX = 3 only) exact checkerboard, one strip of 4 .. 10 rows per
//      block with a halo of two rows: the strip also updates colour 0 of
//      rows -1 and R with copies of the neighbours' streams, so that rows are
//      exchanged once per sweep (the phases A .. D of the mode-6 loop below).
// Launch bounds: the exact-checkerboard kernel runs multi-slot shapes with
// at most 512 threads, except modes 5 and 6; the multi-hit kernel also runs
// two slots with up to 1024 threads.
template <int KIND, int LAYOUT, int SMAX, int MODE>
__global__ void __launch_bounds__(MODE >= 5 ? 1024 : (SMAX >= ((MODE == 1 || MODE == 2) ? 4 : 2) ? 512 : 1024),
                                  ((MODE == 0 || MODE == 3 || MODE == 4) && SMAX == 2) ? 2 : 1)
    k_ising_persist(PersistArgs a)
{
    static_assert(MODE != 5 || SMAX == 2, "mode 5 holds two stream slots per thread");
    static_assert(MODE != 6 || SMAX == 3, "mode 6 holds three stream slots per thread");
    constexpr bool MH = MODE == 1 || MODE == 2;
    constexpr bool EXACT_LOOPS = MODE == 0 || MODE == 3;
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ SegLocal S[kPersistMaxSegs];
    __shared__ Mode6Tab m6tab[MODE == 6 ? 1024 : 1];
    __shared__ uint64_t prefix_end;
    __shared__ int s_abort;
    __shared__ long long red[32];
    const uint32_t sb = a.cta_seg[blockIdx.x], nseg = a.cta_seg[blockIdx.x + 1] - sb;
    if (threadIdx.x < nseg) {
        const SegDev d = a.segs[sb + threadIdx.x];
        const LatDev &l = a.lats[d.lat];
        SegLocal s;
        s.L = l.L;
        s.half = l.half;
        s.W = l.W;
        s.G = l.G;
        s.y0 = d.y0;
        s.R = d.y1 - d.y0;
        s.off = d.smem_off;
        s.lat = d.lat;
        s.coarse = d.coarse;
        s.hd = MODE == 6 ? 2u : 1u;
        s.pstride = (s.R + 2 * s.hd) * (l.layout == ISING_INT8 ? l.half : l.W * 4u);
        s.up = d.up;
        s.down = d.down;
        s.gid = static_cast<int32_t>(sb + threadIdx.x);
        s.s0 = d.s0;
        s.T4 = l.T4;
        s.T8 = l.T8;
        s.t4 = static_cast<uint32_t>(l.T4 > 0xffffffffull ? 0xffffffffull : l.T4);
        s.t8 = static_cast<uint32_t>(l.T8 > 0xffffffffull ? 0xffffffffull : l.T8);
        s.a_max = l.T8 > 0xffffffffull ? 4 : (l.T4 > 0xffffffffull ? 2 : 0);
        s.n_valid = l.nstreams;
        s.n_inst = l.rng.n;
        s.rng = l.rng;
        s.rng.pos = *l.pos_dev;
        S[threadIdx.x] = s;
    }
    if (threadIdx.x == 0) s_abort = 0;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint64_t pre = 0;
        for (uint32_t j = 0; j < nseg; j++) {
            S[j].prefix = pre;
            const SegDev d = a.segs[sb + j];
            pre += d.s1 - d.s0;
        }
        prefix_end = pre;
    }
    __syncthreads();
    for (uint32_t j = 0; j < nseg; j++) load_segment<LAYOUT>(smem, S[j], a.lats[S[j].lat].spins);

    // Streams of this thread: flat indices f = tid + k * blockDim over the
    // block's strips.  When they all fit (k < SMAX), the generator states
    // stay in registers for the whole launch; otherwise each half-sweep
    // walks the streams in passes of SMAX * blockDim, loading and storing
    // the states (L2-resident) around their draws.
    const bool resident = prefix_end <= static_cast<uint64_t>(SMAX) * blockDim.x;
    Gen<KIND> gen[SMAX];
    StreamSlot slot[SMAX];
    if (resident) {
#pragma unroll
        for (int k = 0; k < SMAX; k++) {
            if constexpr (MODE == 3) {
                // slot 0: rows 0 and R-1 of the block's strip; slot 1: rows 1 .. R-2
                const SegLocal &sg = S[0];
                const uint32_t spr = sg.half / sg.G, t = threadIdx.x;
                bool in;
                uint64_t f;
                if (k == 0) {
                    in = t < 2 * spr;
                    f = t < spr ? t : static_cast<uint64_t>(sg.R - 1) * spr + (t - spr);
                } else {
                    in = t < (sg.R - 2) * spr;
                    f = spr + static_cast<uint64_t>(t);
                }
                slot[k].seg = 0;
                slot[k].s = static_cast<uint32_t>(sg.s0 + (in ? f : 0));
                finish_slot<LAYOUT>(sg, in, in && slot[k].s < sg.n_valid, slot[k]);
            } else if constexpr (MODE == 5) {
                // compute threads t < nc = blockDim - 32.  Slot 0: rows 0
                // and R-1 for t < 2 spr, then the first interior streams;
                // slot 1: the remaining interior streams.  The last warp
                // holds none.
                const SegLocal &sg = S[0];
                const uint32_t spr = sg.half / sg.G, t = threadIdx.x, nc = blockDim.x - 32;
                const int64_t ni = sg.R >= 2 ? static_cast<int64_t>(sg.R - 2) * spr : 0;
                bool in = false;
                uint64_t f = 0;
                if (t < nc) {
                    if (k == 0 && t < 2 * spr) {
                        in = true;
                        f = t < spr ? t : static_cast<uint64_t>(sg.R - 1) * spr + (t - spr);
                    } else {
                        const int64_t i = k == 0 ? static_cast<int64_t>(t) - 2 * static_cast<int64_t>(spr)
                                                 : static_cast<int64_t>(nc) - 2 * static_cast<int64_t>(spr) + t;
                        in = i >= 0 && i < ni;
                        f = in ? spr + static_cast<uint64_t>(i) : 0;
                    }
                }
                slot[k].seg = 0;
                slot[k].s = static_cast<uint32_t>(sg.s0 + (in ? f : 0));
                finish_slot<LAYOUT>(sg, in, in && slot[k].s < sg.n_valid, slot[k]);
            } else if constexpr (MODE == 6) {
                // the rows of (slot, cell) as mode6_row lays them out; the
                // halo rows -1 and R hold copies of the neighbours' streams
                const SegLocal &sg = S[0];
                const uint32_t spr = sg.half / sg.G, cell = threadIdx.x / spr, j = threadIdx.x - cell * spr;
                const int R = static_cast<int>(sg.R);
                const int lr = mode6_row(k, cell, R);
                const bool in = lr != kNoRow;
                const uint32_t grow = in ? static_cast<uint32_t>((static_cast<int>(sg.y0 + sg.L) + lr) % static_cast<int>(sg.L)) : 0u;
                StreamSlot &o = slot[k];
                o.seg = 0;
                o.s = in ? static_cast<uint32_t>(static_cast<uint64_t>(grow) * spr + j) : static_cast<uint32_t>(sg.s0);
                o.xh0 = j * sg.G;
                o.base = sg.off + static_cast<uint32_t>((in ? lr : 0) + static_cast<int>(sg.hd)) * row_bytes<LAYOUT>(sg);
                uint32_t f = 0;
                if (in) {
                    f = SL_IN | SL_VAL | ((grow & 1u) ? SL_ODD_ROW : 0u) | (o.xh0 == 0 ? SL_ROW_FIRST : 0u) |
                        (o.xh0 + sg.G == sg.half ? SL_ROW_LAST : 0u);
                    if (lr == -1 || lr == R) {
                        f |= SL_PH_B | SL_REPLICA;
                    } else {
                        if (lr >= 1 && lr <= R - 2) f |= SL_PH_A;
                        if (lr == 0 || lr == R - 1) f |= SL_PH_B;
                        if (lr <= 1 || lr >= R - 2) f |= SL_PH_C;
                        if (lr >= 2 && lr <= R - 3) f |= SL_PH_D;
                    }
                }
                if (__any_sync(0xffffffffu, in)) f |= SL_WARP_IN;
                if (LAYOUT != ISING_INT8 && sg.G == 2 &&
                    __all_sync(0xffffffffu, !in || (o.xh0 & 31u) == 2u * (threadIdx.x & 15u)))
                    f |= SL_MS_PAIR;
                o.flags = f;
            } else {
                setup_slot<LAYOUT>(S, nseg, prefix_end, threadIdx.x + static_cast<uint64_t>(k) * blockDim.x, slot[k]);
            }
            const SegLocal &sg = S[slot[k].seg];
            gen[k].load(sg.rng, slot[k].s < sg.n_inst ? slot[k].s : sg.n_inst - 1);
        }
    }
    __syncthreads();

    uint64_t meas_idx = 0;
    const int lane = threadIdx.x & 31;
    if constexpr (MODE == 4) {
        // the host chose this kernel for blocks of one whole resident lattice
        const bool ok = resident && nseg == 1 && S[0].up < 0;
        if (!__syncthreads_and(ok)) {
            if (threadIdx.x == 0) atomicCAS(a.err, 0, RNG_EINVAL);
            goto done;
        }
        for (uint64_t t = 0; t < a.n_sweeps; t++) {
            for (int c = 0; c < 2; c++) {
                if (slot[0].flags & SL_WARP_IN) update_slot<KIND, LAYOUT, true>(smem, S[0], slot[0], gen[0], c, lane);
                __syncthreads();
            }
            if (a.measure_every && (a.sweep0 + t + 1) % a.measure_every == 0) {
                measure_strips<LAYOUT>(smem, S, nseg, a, meas_idx, red);
                meas_idx++;
            }
        }
    }
    if constexpr (MODE == 3) {
        // the host chose this kernel for one strip per block whose boundary
        // rows fill at most slot 0 and whose interior rows slot 1: check it
        const uint32_t spr = S[0].half / S[0].G;
        const bool ok = resident && nseg == 1 && S[0].R >= 2 && spr % 32 == 0 && 2 * spr <= blockDim.x &&
                        (S[0].R - 2) * spr <= blockDim.x && prefix_end == static_cast<uint64_t>(S[0].R) * spr;
        if (!__syncthreads_and(ok)) {
            if (threadIdx.x == 0) atomicCAS(a.err, 0, RNG_EINVAL);
            goto done;
        }
    }
    if constexpr (MODE == 5) {
        // the host chose this kernel for one strip per block whose first and
        // last rows fill slot 0 of the first 2 spr threads and whose rows
        // between fit the rest of the compute threads' two slots
        const SegLocal &sg = S[0];
        const uint32_t spr = sg.half / sg.G, nc = blockDim.x - 32;
        const bool ok = resident && nseg == 1 && sg.up >= 0 && sg.R >= 2 && spr % 32 == 0 && blockDim.x % 32 == 0 &&
                        blockDim.x >= 64 && 2 * spr <= nc && prefix_end == static_cast<uint64_t>(sg.R) * spr &&
                        prefix_end <= 2ull * nc;
        if (!__syncthreads_and(ok)) {
            if (threadIdx.x == 0) atomicCAS(a.err, 0, RNG_EINVAL);
            goto done;
        }
        const bool poller = threadIdx.x >= nc;
        const bool bnd = threadIdx.x < 2 * spr;  // warp-uniform: 2 spr is a multiple of 32
        for (uint64_t t = 0; t < a.n_sweeps; t++) {
            for (int c = 0; c < 2; c++) {
                const uint32_t h = static_cast<uint32_t>(2 * t + c);
                if (poller) {
                    // the neighbours' rows of colour c go to the halo rows of
                    // plane c, which no update of colour c reads
                    if (!poll_rows_warp<LAYOUT>(smem, sg, a, h & 1, h + 1, c, lane)) s_abort = 1;
                } else {
                    // the strip's first and last rows first, then published;
                    // the other compute warps wait, so that these rows are
                    // ready as early as possible
                    if (bnd) update_slot<KIND, LAYOUT>(smem, sg, slot[0], gen[0], c, lane);
                    bar_sync_first(nc);
                    publish_rows_by<LAYOUT>(smem, sg, a, h & 1, h + 1, c, threadIdx.x, nc);
                    if (!bnd && (slot[0].flags & SL_WARP_IN)) update_slot<KIND, LAYOUT>(smem, sg, slot[0], gen[0], c, lane);
                    if (slot[1].flags & SL_WARP_IN) update_slot<KIND, LAYOUT>(smem, sg, slot[1], gen[1], c, lane);
                }
                __syncthreads();
                if (s_abort) goto done;
            }
            if (a.measure_every && (a.sweep0 + t + 1) % a.measure_every == 0) {
                measure_strips<LAYOUT>(smem, S, nseg, a, meas_idx, red);
                meas_idx++;
            }
        }
    }
    if constexpr (MODE == 6) {
        // the host chose this kernel for one strip of 4 .. 10 rows per block
        // whose rows and halo copies fit the cells of mode6_row
        const SegLocal &sg = S[0];
        const uint32_t spr = sg.half / sg.G;
        const bool ok = resident && nseg == 1 && sg.up >= 0 && sg.R >= 4 && sg.R <= 10 && spr % 32 == 0 &&
                        4 * spr <= blockDim.x && 6 * (row_bytes<LAYOUT>(sg) / 4) <= blockDim.x &&
                        prefix_end == static_cast<uint64_t>(sg.R) * spr;
        if (!__syncthreads_and(ok)) {
            if (threadIdx.x == 0) atomicCAS(a.err, 0, RNG_EINVAL);
            goto done;
        }
        mode6_table<LAYOUT>(smem, sg, a, m6tab);
        __syncthreads();
        const Mode6Tab &e6 = m6tab[threadIdx.x];
        bool polled = false;  // the halo already holds the neighbours' rows of the last sweep
        // two sweeps per loop body for int8 (measured 1-2.5% faster; for
        // multispin no faster, and five sweeps slower for both)
#pragma unroll(LAYOUT == ISING_INT8 ? 2 : 1)
        for (uint64_t t = 0; t < a.n_sweeps; t++) {
            // colour 0 of the rows between the edges: own rows only
#pragma unroll
            for (int k = 0; k < SMAX; k++)
                if (slot[k].flags & SL_PH_A) update_slot<KIND, LAYOUT>(smem, sg, slot[k], gen[k], 0, lane);
            // the neighbours' rows after the last sweep (the first sweep of a
            // launch has them from the lattice itself)
            if (t > 0 && !polled && !poll6(smem, a, e6, static_cast<uint32_t>((t - 1) & 1), static_cast<uint32_t>(t)))
                s_abort = 1;
            polled = false;
            __syncthreads();
            if (s_abort) goto done;
            // colour 0 of the edge rows and of the halo rows -1 and R
#pragma unroll
            for (int k = 0; k < SMAX; k++)
                if (slot[k].flags & SL_PH_B) update_slot<KIND, LAYOUT>(smem, sg, slot[k], gen[k], 0, lane);
            __syncthreads();
            // colour 1 of all rows in one pass; the halo copies draw the
            // numbers their owners take now and update nothing (colour 1 of
            // the halo comes with the next exchange).  Publishing after the
            // whole pass costs one barrier less per sweep than publishing
            // rows 0, 1, R-2, R-1 first (measured faster); the words then
            // travel while the next sweep's rows between the edges update
            // (they read none of the published rows' colour-0 sites).
#pragma unroll
            for (int k = 0; k < SMAX; k++) {
                if (slot[k].flags & (SL_PH_C | SL_PH_D)) {
                    update_slot<KIND, LAYOUT>(smem, sg, slot[k], gen[k], 1, lane);
                } else if (slot[k].flags & SL_REPLICA) {
                    for (uint32_t g = 0; g < sg.G; g++) (void)gen[k].next();
                }
            }
            __syncthreads();
            publish6(smem, sg, a, e6, static_cast<uint32_t>(t & 1), static_cast<uint32_t>(t + 1));
            if (a.measure_every && (a.sweep0 + t + 1) % a.measure_every == 0) {
                // the energy reads colour 1 of the halo rows: take this
                // sweep's rows first
                if (!poll6(smem, a, e6, static_cast<uint32_t>(t & 1), static_cast<uint32_t>(t + 1))) s_abort = 1;
                polled = true;
                __syncthreads();
                if (s_abort) goto done;
                measure_strips<LAYOUT>(smem, S, nseg, a, meas_idx, red);
                meas_idx++;
            }
        }
    }
    if constexpr (EXACT_LOOPS) {
        // ---------------- exact checkerboard: all strips, every half-sweep
        // A block of whole lattices exchanges nothing with other blocks: a
        // half-sweep is one pass over all its warps, then the halo rows are
        // copied from the edge rows (no boundary-first pass).
        bool all_whole = MODE == 0;
        for (uint32_t j = 0; j < nseg; j++) all_whole = all_whole && S[j].up < 0;
        for (uint64_t t = 0; t < a.n_sweeps && all_whole; t++) {
            for (int c = 0; c < 2; c++) {
                if (resident) {
                    update_resident<KIND, LAYOUT, SMAX>(smem, S, gen, slot, c, lane, SEL_ALL);
                } else {
                    update_pass<KIND, LAYOUT, SMAX>(smem, S, nseg, prefix_end, false, gen, slot,
                                                    (2 * t + c) * static_cast<uint64_t>(S[0].G), c, lane, SEL_ALL);
                }
                __syncthreads();
                for (uint32_t j = 0; j < nseg; j++) {
                    const SegLocal &sg = S[j];
                    const uint32_t rb = row_bytes<LAYOUT>(sg);
                    uint8_t *top = plane_row<LAYOUT>(smem, sg, c, -1), *bot = plane_row<LAYOUT>(smem, sg, c, sg.R);
                    const uint8_t *last = plane_row<LAYOUT>(smem, sg, c, sg.R - 1);
                    const uint8_t *first = plane_row<LAYOUT>(smem, sg, c, 0);
                    for (uint32_t i = threadIdx.x; i < rb; i += blockDim.x) {
                        top[i] = last[i];
                        bot[i] = first[i];
                    }
                }
                __syncthreads();
            }
            if (a.measure_every && (a.sweep0 + t + 1) % a.measure_every == 0) {
                measure_strips<LAYOUT>(smem, S, nseg, a, meas_idx, red);
                meas_idx++;
            }
        }
        for (uint64_t t = 0; t < a.n_sweeps && !all_whole; t++) {
            for (int c = 0; c < 2; c++) {
                const uint32_t h = static_cast<uint32_t>(2 * t + c);
                const uint64_t pos_off = (2 * t + c) * static_cast<uint64_t>(S[0].G);
                // warps that hold a strip's first or last row go first ...
                if constexpr (MODE == 3) {
                    if (slot[0].flags & SL_WARP_IN) update_slot<KIND, LAYOUT>(smem, S[0], slot[0], gen[0], c, lane);
                } else if (resident) {
                    update_resident<KIND, LAYOUT, SMAX>(smem, S, gen, slot, c, lane, SEL_BOUNDARY);
                } else {
                    update_pass<KIND, LAYOUT, SMAX>(smem, S, nseg, prefix_end, false, gen, slot, pos_off, c, lane,
                                                    SEL_BOUNDARY);
                }
                __syncthreads();
                // ... their rows are published (a whole lattice copies them into
                // its own halo rows) ...
                bool any_split = false;
                for (uint32_t j = 0; j < nseg; j++) {
                    const SegLocal &sg = S[j];
                    if (sg.up < 0) {
                        // byte copies: an int8 row of L/2 bytes need not be word aligned
                        const uint32_t rb = row_bytes<LAYOUT>(sg);
                        uint8_t *top = plane_row<LAYOUT>(smem, sg, c, -1), *bot = plane_row<LAYOUT>(smem, sg, c, sg.R);
                        const uint8_t *last = plane_row<LAYOUT>(smem, sg, c, sg.R - 1);
                        const uint8_t *first = plane_row<LAYOUT>(smem, sg, c, 0);
                        for (uint32_t i = threadIdx.x; i < rb; i += blockDim.x) {
                            top[i] = last[i];
                            bot[i] = first[i];
                        }
                    } else {
                        any_split = true;
                        publish_rows<LAYOUT>(smem, sg, a, h & 1, h + 1, c);
                    }
                }
                // ... the interior rows are updated while those words travel ...
                if constexpr (MODE == 3) {
                    if (slot[SMAX - 1].flags & SL_WARP_IN)
                        update_slot<KIND, LAYOUT>(smem, S[0], slot[SMAX - 1], gen[SMAX - 1], c, lane);
                } else if (resident) {
                    update_resident<KIND, LAYOUT, SMAX>(smem, S, gen, slot, c, lane, SEL_INTERIOR);
                } else {
                    update_pass<KIND, LAYOUT, SMAX>(smem, S, nseg, prefix_end, false, gen, slot, pos_off, c, lane,
                                                    SEL_INTERIOR);
                }
                // ... and the neighbours' rows are polled into the halo rows
                if (any_split) {
                    const uint64_t t0 = global_ns();
                    const long long c0 = clock64();
                    bool ok = true;
                    for (uint32_t j = 0; j < nseg && ok; j++)
                        if (S[j].up >= 0) ok = poll_rows<LAYOUT>(smem, S[j], a, h & 1, h + 1, c, t0, c0);
                    if (!ok) s_abort = 1;
                }
                __syncthreads();
                if (s_abort) goto done;
            }
            if (a.measure_every && (a.sweep0 + t + 1) % a.measure_every == 0) {
                measure_strips<LAYOUT>(smem, S, nseg, a, meas_idx, red);
                meas_idx++;
            }
        }
    } else if constexpr (MH) {
        // ---------------- multi-hit rounds (double checkerboard): the strips
        // of coarse colour C take k sweeps of their own rows while the other
        // strips stay fixed; then they publish both colours of their first
        // and last rows, which the other strips poll before their phase
        const uint32_t k = a.k_hits;
        if constexpr (MODE == 2) {
            // the host chose this kernel for a plan with one resident slot of
            // each coarse colour per thread, slot 0 in colour 0: check it
            bool ok = resident;
#pragma unroll
            for (int kk = 0; kk < SMAX; kk++)
                if ((slot[kk].flags & SL_IN) && ((slot[kk].flags & SL_COARSE) != 0) != (kk == 1)) ok = false;
            if (!__syncthreads_and(ok)) {
                if (threadIdx.x == 0) atomicCAS(a.err, 0, RNG_EINVAL);
                goto done;
            }
        }
        for (uint64_t t = 0; t < a.n_sweeps; t++) {
            for (int C = 0; C < 2; C++) {
                const uint32_t ph = static_cast<uint32_t>(2 * t + C);
                if (ph > 0) {  // the other coarse colour published at the end of phase ph - 1
                    const uint64_t t0 = global_ns();
                    const long long c0 = clock64();
                    bool ok = true;
                    for (uint32_t j = 0; j < nseg && ok; j++)
                        if (S[j].coarse == static_cast<uint32_t>(C))
                            for (int cc = 0; cc < 2 && ok; cc++)
                                ok = poll_rows<LAYOUT>(smem, S[j], a, ((ph - 1) >> 1) & 1, ph, cc, t0, c0);
                    if (!ok) s_abort = 1;
                    __syncthreads();
                    if (s_abort) goto done;
                }
                if constexpr (MODE == 2) {
                    // slot C is the thread's stream of coarse colour C
                    if (C == 0) {
                        const bool act = (slot[0].flags & SL_WARP_IN) != 0;
                        const SegLocal &sg = S[slot[0].seg];
                        for (uint32_t hit = 0; hit < k; hit++) {
                            if (act) update_slot<KIND, LAYOUT>(smem, sg, slot[0], gen[0], 0, lane);
                            __syncthreads();
                            if (act) update_slot<KIND, LAYOUT>(smem, sg, slot[0], gen[0], 1, lane);
                            __syncthreads();
                        }
                    } else {
                        const bool act = (slot[SMAX - 1].flags & SL_WARP_IN) != 0;
                        const SegLocal &sg = S[slot[SMAX - 1].seg];
                        for (uint32_t hit = 0; hit < k; hit++) {
                            if (act) update_slot<KIND, LAYOUT>(smem, sg, slot[SMAX - 1], gen[SMAX - 1], 0, lane);
                            __syncthreads();
                            if (act) update_slot<KIND, LAYOUT>(smem, sg, slot[SMAX - 1], gen[SMAX - 1], 1, lane);
                            __syncthreads();
                        }
                    }
                } else {
                    for (uint32_t hit = 0; hit < k; hit++) {
                        for (int c = 0; c < 2; c++) {
                            const uint64_t pos_off = (2 * (t * k + hit) + c) * static_cast<uint64_t>(S[0].G);
                            if (resident)
                                update_resident<KIND, LAYOUT, SMAX>(smem, S, gen, slot, c, lane, SEL_COARSE0 + C);
                            else
                                update_pass<KIND, LAYOUT, SMAX>(smem, S, nseg, prefix_end, false, gen, slot, pos_off,
                                                                c, lane, SEL_COARSE0 + C);
                            __syncthreads();
                        }
                    }
                }
                for (uint32_t j = 0; j < nseg; j++)
                    if (S[j].coarse == static_cast<uint32_t>(C))
                        for (int cc = 0; cc < 2; cc++) publish_rows<LAYOUT>(smem, S[j], a, (ph >> 1) & 1, ph + 1, cc);
            }
            if (a.measure_every && (a.sweep0 + t + 1) % a.measure_every == 0) {
                // the coarse-0 strips first take the rows the coarse-1 strips just published
                const uint32_t ph = static_cast<uint32_t>(2 * t + 1);
                const uint64_t t0 = global_ns();
                const long long c0 = clock64();
                bool ok = true;
                for (uint32_t j = 0; j < nseg && ok; j++)
                    if (S[j].coarse == 0)
                        for (int cc = 0; cc < 2 && ok; cc++)
                            ok = poll_rows<LAYOUT>(smem, S[j], a, (ph >> 1) & 1, ph + 1, cc, t0, c0);
                if (!ok) s_abort = 1;
                __syncthreads();
                if (s_abort) goto done;
                measure_strips<LAYOUT>(smem, S, nseg, a, meas_idx, red);
                meas_idx++;
            }
        }
    }
done:
    __syncthreads();
    for (uint32_t j = 0; j < nseg; j++) store_segment<LAYOUT>(smem, S[j], a.lats[S[j].lat].spins);
    if (resident) {
#pragma unroll
        for (int k = 0; k < SMAX; k++)
            if (slot[k].in() && !(slot[k].flags & SL_REPLICA) && slot[k].s < S[slot[k].seg].n_inst)
                gen[k].store(a.lats[S[slot[k].seg].lat].rng, slot[k].s);
    }
}

}  // namespace rngx
