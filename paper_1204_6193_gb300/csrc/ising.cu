// ising.cu -- C ABI of the Ising application test: lattice handles, the
// tile plan of the persistent kernel, chunked persistent launches, the
// one-launch-per-half-sweep baseline, observables, batches of lattices
// replayed from a CUDA graph, and the launch-shape autotuner.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "ising_persist.cuh"

namespace rngx {

template <int KIND> int launch_half(const LatDev &, int, cudaStream_t);
template <int KIND>
int launch_persist(int, int, const PersistArgs &, unsigned, unsigned, size_t, cudaStream_t, int *);

namespace {

constexpr uint64_t kChunkSweeps = 4096;  // sweeps per persistent launch
constexpr uint32_t kMaxHits = 65536;      // multi-hit sweeps per strip phase
constexpr size_t kSmemCap = 200 * 1024;  // dynamic shared memory per block we plan for
constexpr uint64_t kWaveStreamsPerSm = 2048;  // streams per SM that one persistent launch keeps in registers

int dispatch_half(int kind, const LatDev &lat, int c, cudaStream_t s)
{
    switch (kind) {
    case RNG_LCG32: return launch_half<RNG_LCG32>(lat, c, s);
    case RNG_LCG64: return launch_half<RNG_LCG64>(lat, c, s);
    case RNG_MWC: return launch_half<RNG_MWC>(lat, c, s);
    case RNG_XORWOW: return launch_half<RNG_XORWOW>(lat, c, s);
    case RNG_PHILOX4X32_10: return launch_half<RNG_PHILOX4X32_10>(lat, c, s);
    case RNG_PHILOX4X32_7: return launch_half<RNG_PHILOX4X32_7>(lat, c, s);
    case RNG_XS1024W: return launch_half<RNG_XS1024W>(lat, c, s);
    }
    set_error("Ising: generator kind %d not supported", kind);
    return RNG_EUNSUPPORTED;
}

int dispatch_persist(int kind, int layout, int smax, const PersistArgs &a, unsigned nb, unsigned th, size_t smem,
                     cudaStream_t s, int *max_blocks)
{
    switch (kind) {
    case RNG_LCG32: return launch_persist<RNG_LCG32>(layout, smax, a, nb, th, smem, s, max_blocks);
    case RNG_LCG64: return launch_persist<RNG_LCG64>(layout, smax, a, nb, th, smem, s, max_blocks);
    case RNG_MWC: return launch_persist<RNG_MWC>(layout, smax, a, nb, th, smem, s, max_blocks);
    case RNG_XORWOW: return launch_persist<RNG_XORWOW>(layout, smax, a, nb, th, smem, s, max_blocks);
    case RNG_PHILOX4X32_10: return launch_persist<RNG_PHILOX4X32_10>(layout, smax, a, nb, th, smem, s, max_blocks);
    case RNG_PHILOX4X32_7: return launch_persist<RNG_PHILOX4X32_7>(layout, smax, a, nb, th, smem, s, max_blocks);
    case RNG_XS1024W: return launch_persist<RNG_XS1024W>(layout, smax, a, nb, th, smem, s, max_blocks);
    }
    set_error("Ising: generator kind %d not supported", kind);
    return RNG_EUNSUPPORTED;
}

// ------------------------------------------------------------- kernels
// Initial spins: site j = y L + x is +1 iff bit j % 64 of the SplitMix64
// word j / 64 of (seed ^ 0x5350494E) is set.
__device__ __forceinline__ int init_spin(uint64_t seed2, uint64_t j)
{
    return ((d_seed_word(seed2, j >> 6) >> (j & 63)) & 1) ? 1 : -1;
}

__global__ void k_init_int8(int8_t *sp, uint32_t L, uint64_t seed2)
{
    const uint64_t j = static_cast<uint64_t>(blockIdx.x) * 256 + threadIdx.x;
    if (j < static_cast<uint64_t>(L) * L) sp[j] = static_cast<int8_t>(init_spin(seed2, j));
}

__global__ void k_init_ms(uint32_t *planes, uint32_t L, uint32_t W, uint64_t seed2)
{
    const uint64_t idx = static_cast<uint64_t>(blockIdx.x) * 256 + threadIdx.x;
    if (idx >= 2ull * L * W) return;
    const uint32_t c = static_cast<uint32_t>(idx / (static_cast<uint64_t>(L) * W));
    const uint32_t rem = static_cast<uint32_t>(idx % (static_cast<uint64_t>(L) * W));
    const uint32_t y = rem / W, wi = rem % W;
    uint32_t word = 0;
    for (int b = 0; b < 32; b++) {
        const uint32_t xh = 32 * wi + b;
        const uint32_t x = 2 * xh + ((c + y) & 1);
        if (init_spin(seed2, static_cast<uint64_t>(y) * L + x) < 0) word |= 1u << b;
    }
    planes[idx] = word;
}

__device__ __forceinline__ void add_i64(int64_t *p, long long v)
{
    atomicAdd(reinterpret_cast<unsigned long long *>(p), static_cast<unsigned long long>(v));
}

// E = -sum_bonds s_i s_j and M over the whole lattice into acc[5], acc[6].
__global__ void k_energy(LatDev lat)
{
    __shared__ long long red[2][8];
    long long E = 0, M = 0;
    const uint64_t tid = static_cast<uint64_t>(blockIdx.x) * 256 + threadIdx.x;
    const uint32_t L = lat.L;
    if (lat.layout == ISING_INT8) {
        const int8_t *sp = static_cast<const int8_t *>(lat.spins);
        if (tid < static_cast<uint64_t>(L) * L) {
            const uint32_t y = static_cast<uint32_t>(tid / L), x = static_cast<uint32_t>(tid % L);
            const int s = sp[tid];
            E = -s * (sp[static_cast<size_t>(y) * L + (x + 1 == L ? 0 : x + 1)] +
                      sp[static_cast<size_t>(y + 1 == L ? 0 : y + 1) * L + x]);
            M = s;
        }
    } else {
        const uint32_t W = lat.W;
        if (tid < static_cast<uint64_t>(L) * W) {
            const uint32_t y = static_cast<uint32_t>(tid / W), w = static_cast<uint32_t>(tid % W);
            const uint32_t *p0 = static_cast<const uint32_t *>(lat.spins);
            const uint32_t *p1 = p0 + static_cast<size_t>(L) * W;
            const uint32_t *o = p1 + static_cast<size_t>(y) * W;
            const uint32_t own = p0[static_cast<size_t>(y) * W + w];
            const uint32_t up = p1[static_cast<size_t>(y == 0 ? L - 1 : y - 1) * W + w];
            const uint32_t dn = p1[static_cast<size_t>(y + 1 == L ? 0 : y + 1) * W + w];
            uint32_t lft, rgt;
            if ((y & 1u) == 0) {
                lft = (o[w] << 1) | (o[w == 0 ? W - 1 : w - 1] >> 31);
                rgt = o[w];
            } else {
                lft = o[w];
                rgt = (o[w] >> 1) | (o[w + 1 == W ? 0 : w + 1] << 31);
            }
            const int U = __popc(own ^ lft) + __popc(own ^ rgt) + __popc(own ^ up) + __popc(own ^ dn);
            E = 2 * U - 128;
            M = 64 - 2 * (__popc(own) + __popc(o[w]));
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        E += __shfl_down_sync(0xffffffffu, E, o);
        M += __shfl_down_sync(0xffffffffu, M, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = E;
        red[1][threadIdx.x >> 5] = M;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long e = 0, m = 0;
        for (int i = 0; i < 8; i++) {
            e += red[0][i];
            m += red[1][i];
        }
        add_i64(lat.acc + 5, e);
        add_i64(lat.acc + 6, m);
    }
}

// acc[0..4] += E, E^2, M^2, |M|, 1 from the current E, M in acc[5], acc[6].
__global__ void k_accumulate_now(int64_t *acc)
{
    const long long E = acc[5], M = acc[6];
    acc[0] += E;
    acc[1] += E * E;
    acc[2] += M * M;
    acc[3] += M < 0 ? -M : M;
    acc[4] += 1;
}

// acc[0..4] += the n measurements (E, M) recorded by a persistent launch.
__global__ void k_meas_finalize(const int64_t *meas, uint32_t n, int64_t *acc)
{
    __shared__ long long red[4][32];
    long long s[4] = {0, 0, 0, 0};
    for (uint32_t m = threadIdx.x; m < n; m += blockDim.x) {
        const long long E = meas[2 * m], M = meas[2 * m + 1];
        s[0] += E;
        s[1] += E * E;
        s[2] += M * M;
        s[3] += M < 0 ? -M : M;
    }
    for (int k = 0; k < 4; k++) {
        for (int o = 16; o > 0; o >>= 1) s[k] += __shfl_down_sync(0xffffffffu, s[k], o);
        if ((threadIdx.x & 31) == 0) red[k][threadIdx.x >> 5] = s[k];
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        long long t = 0;
        for (int i = 0; i < static_cast<int>(blockDim.x >> 5); i++) t += red[threadIdx.x][i];
        acc[threadIdx.x] += t;
    }
    if (threadIdx.x == 0) acc[4] += n;
}

__global__ void k_add_u64(uint64_t *p, uint64_t v) { *p += v; }
__global__ void k_set_u64(uint64_t *p, uint64_t v) { *p = v; }

// One half-sweep with warp-shared generators (MT19937, lagged Fibonacci):
// their numbers for this half-sweep were generated into `draws`, generator
// j's 32 G words at draws[j 32 G ..], so that the g-th number of stream s =
// 32 j + l is draws[j 32 G + 32 g + l].  One thread per stream.
template <int LAYOUT>
__global__ void __launch_bounds__(256) k_ising_half_given(LatDev lat, int c, const uint32_t *__restrict__ draws)
{
    const uint64_t s = static_cast<uint64_t>(blockIdx.x) * 256 + threadIdx.x;
    if ((s & ~31ull) >= lat.nstreams) return;  // whole warps
    const bool valid = s < lat.nstreams;
    const uint32_t G = lat.G, half = lat.half, L = lat.L;
    const uint32_t *dr = draws + (s >> 5) * 32ull * G + (s & 31u);
    const uint64_t q0 = s * G;
    const uint32_t y = valid ? static_cast<uint32_t>(q0 / half) : 0;
    const uint32_t xh0 = valid ? static_cast<uint32_t>(q0 - static_cast<uint64_t>(y) * half) : 0;
    const uint32_t p = (c + y) & 1u;
    const uint32_t yu = y == 0 ? L - 1 : y - 1, yd = y + 1 == L ? 0 : y + 1;
    if (LAYOUT == ISING_INT8) {
        int8_t *sp = static_cast<int8_t *>(lat.spins);
        for (uint32_t g = 0; g < G && valid; g++) {
            const uint32_t rr = dr[32u * g];
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
        for (uint32_t g = 0; g < G && valid; g++) {
            const uint32_t rr = dr[32u * g];
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
        // the warp's 32 G sites are G consecutive words of plane c
        const uint64_t first_word = ((s & ~31ull) * G) >> 5;
        const uint64_t words = static_cast<uint64_t>(L) * W;
        for (uint32_t m = 0; m < G; m++) {
            const uint32_t mine = ((lq0 >> 5) == m ? c_lo : 0u) | ((lq0 >> 5) + 1 == m ? c_hi : 0u);
            const uint32_t word = __reduce_or_sync(0xffffffffu, mine);
            if (lane == 0 && word && first_word + m < words) pc[first_word + m] ^= word;
        }
    }
}

}  // namespace
}  // namespace rngx

using namespace rngx;

// One lattice: parameters, its streams, spins and accumulators.
struct IsingLat {
    uint32_t L = 0, G = 0, W = 0;
    int layout = 0, kind = 0;
    uint32_t flags = 0;
    double beta = 0;
    uint64_t seed = 0, T4 = 0, T8 = 0, nstreams = 0;
    rng_t rng = nullptr;
    void *spins = nullptr;
    size_t spin_bytes = 0;
    int64_t *acc = nullptr;      // device [8]
    uint64_t *pos_dev = nullptr; // device [1]
    int64_t *meas = nullptr;     // device [2 * meas_cap]
    uint64_t meas_cap = 0;
    uint32_t *draws = nullptr;   // warp-shared generators: one half-sweep's numbers, 32 G per generator
};

// Persistent launch plan of one group of lattices of one generator kind.
struct Plan {
    int kind = 0, layout = 0, smax = 1;
    int fixed_slots = 0;  // 1: each thread slot has a fixed role (kernel modes 2, 3); 2: whole lattices (mode 4);
                          // 3: one strip per block, roles split by warp, a polling warp (mode 5);
                          // 4: one strip per block with a halo of two rows, one exchange per sweep (mode 6)
    unsigned nblocks = 0, threads = 0;
    size_t smem = 0;
    uint32_t nsegs = 0, halo_row_bytes = 0;
    SegDev *d_segs = nullptr;
    uint32_t *d_cta = nullptr;
    uint8_t *d_halo = nullptr;
    // per strip: 2 slots x 2 rows x 2 colours of (tag, data) words (mode 6:
    // 2 parities x 6 half-rows)
    size_t halo_bytes() const { return static_cast<size_t>(nsegs) * (fixed_slots == 4 ? 12 : 8) * halo_row_bytes; }
};

struct ising_s {
    std::vector<IsingLat> lats;
    bool batch = false;
    uint64_t master_seed = 0;  // batch: lattice b is seeded with w_b of this seed
    cudaStream_t stream = nullptr;
    LatDev *d_lats = nullptr;
    int *d_err = nullptr;
    std::vector<Plan> plans;
    bool planned = false;
    bool plan_unfit = false;     // no persistent plan fits: sweeps run the per-half-sweep kernels
    std::vector<Plan> mh_plans;  // the multi-hit plan (one lattice) and its strip count
    uint32_t mh_strips = 0;
    unsigned cfg_threads = 0;    // 0: heuristic
    int cfg_ctas_per_sm = 0;     // 0: heuristic
    uint32_t cfg_min_sites = 0;  // 0: heuristic (1024)
    uint32_t cfg_halo_depth = 0; // 0: two-row halo where a plan fits it, 1: one row
    cudaGraphExec_t gexec = nullptr;
    cudaGraph_t graph = nullptr;
    int32_t mute_seg = -1;                  // test hook (see ising_debug_mute_strip)
    uint64_t wait_budget_ns = kWaitBudgetNs;
    uint64_t g_sweeps = 0;
    uint32_t g_meas = 0;
    LatDev host_lat{};  // staging of an asynchronous parameter upload (ising_reset_lattice)
};

namespace {

int lat_create(IsingLat &t, uint32_t L, double beta, int layout, int kind, uint32_t flags, uint64_t seed, uint32_t G,
               cudaStream_t s)
{
    if (L < 4 || L % 2 || L > 65536) {
        set_error("Ising: L must be even, 4 <= L <= 65536 (got %u)", L);
        return RNG_EINVAL;
    }
    if (!(beta >= 0.0) || !std::isfinite(beta)) {
        set_error("Ising: beta must be finite and >= 0");
        return RNG_EINVAL;
    }
    if (layout != ISING_INT8 && layout != ISING_MULTISPIN32) {
        set_error("Ising: unknown layout %d", layout);
        return RNG_EINVAL;
    }
    if (layout == ISING_MULTISPIN32 && L % 64) {
        set_error("Ising: the multispin layout packs 32 same-colour sites per word and needs L %% 64 == 0");
        return RNG_EINVAL;
    }
    if (G == 0 || (L / 2) % G) {
        set_error("Ising: G (sites per stream per colour) must divide L/2");
        return RNG_EINVAL;
    }
    if (kind < RNG_LCG32 || kind >= kNumKinds) {
        set_error("Ising: generator kind %d is not supported by the application test", kind);
        return RNG_EUNSUPPORTED;
    }
    t.L = L;
    t.G = G;
    t.W = L / 64;
    t.layout = layout;
    t.kind = kind;
    t.flags = flags;
    t.beta = beta;
    t.seed = seed;
    // T[dE] = floor(2^32 exp(-beta dE)), once, in double
    t.T4 = static_cast<uint64_t>(std::floor(4294967296.0 * std::exp(-beta * 4.0)));
    t.T8 = static_cast<uint64_t>(std::floor(4294967296.0 * std::exp(-beta * 8.0)));
    t.nstreams = static_cast<uint64_t>(L) * L / 2 / G;
    // the 1024-bit generator: a lane per stream, whole warps; the block-shared
    // generators: one per 32 streams, feeding them in lane order
    const uint64_t n_inst = kind == RNG_XS1024W ? (t.nstreams + 31) / 32 * 32
                            : is_block_shared(kind) ? (t.nstreams + 31) / 32 : t.nstreams;
    RNGX_CHECK(rng_create(&t.rng, kind, n_inst, flags, s));
    RNGX_CHECK(rng_seed(t.rng, seed));
    if (is_block_shared(kind))
        RNGX_CHECK(dalloc(reinterpret_cast<void **>(&t.draws), n_inst * 32 * G * sizeof(uint32_t), s));
    t.spin_bytes = layout == ISING_INT8 ? static_cast<size_t>(L) * L : 2ull * L * t.W * 4;
    RNGX_CHECK(dalloc(&t.spins, t.spin_bytes, s));
    RNGX_CHECK(dalloc(reinterpret_cast<void **>(&t.acc), 8 * sizeof(int64_t), s));
    RNGX_CHECK(dalloc(reinterpret_cast<void **>(&t.pos_dev), sizeof(uint64_t), s));
    RNGX_CHECK_CUDA(cudaMemsetAsync(t.acc, 0, 8 * sizeof(int64_t), s));
    RNGX_CHECK_CUDA(cudaMemsetAsync(t.pos_dev, 0, sizeof(uint64_t), s));
    const uint64_t seed2 = seed ^ 0x5350494EULL;
    if (layout == ISING_INT8) {
        const uint64_t n = static_cast<uint64_t>(L) * L;
        k_init_int8<<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(static_cast<int8_t *>(t.spins), L, seed2);
    } else {
        const uint64_t n = 2ull * L * t.W;
        k_init_ms<<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(static_cast<uint32_t *>(t.spins), L, t.W,
                                                                          seed2);
    }
    RNGX_CHECK_LAUNCH();
    return RNG_OK;
}

void lat_free(IsingLat &t, cudaStream_t s)
{
    if (t.rng) rng_destroy(t.rng);
    dfree(t.spins, s);
    dfree(t.acc, s);
    dfree(t.pos_dev, s);
    dfree(t.meas, s);
    dfree(t.draws, s);
    t = IsingLat();
}

LatDev lat_dev(const IsingLat &t)
{
    LatDev d;
    memset(&d, 0, sizeof(d));
    d.L = t.L;
    d.G = t.G;
    d.layout = static_cast<uint32_t>(t.layout);
    d.half = t.L / 2;
    d.W = t.W;
    d.T4 = t.T4;
    d.T8 = t.T8;
    d.nstreams = t.nstreams;
    d.rng = dev_params(t.rng->g);
    d.spins = t.spins;
    d.meas = t.meas;
    d.acc = t.acc;
    d.pos_dev = t.pos_dev;
    return d;
}

int upload_lats(ising_t h)
{
    std::vector<LatDev> v;
    for (auto &t : h->lats) v.push_back(lat_dev(t));
    if (!h->d_lats) RNGX_CHECK(dalloc(reinterpret_cast<void **>(&h->d_lats), v.size() * sizeof(LatDev), h->stream));
    RNGX_CHECK_CUDA(cudaStreamSynchronize(h->stream));
    RNGX_CHECK_CUDA(cudaMemcpy(h->d_lats, v.data(), v.size() * sizeof(LatDev), cudaMemcpyHostToDevice));
    return RNG_OK;
}

void free_plans(ising_t h)
{
    for (auto *v : {&h->plans, &h->mh_plans})
        for (auto &p : *v) {
            dfree(p.d_segs, h->stream);
            dfree(p.d_cta, h->stream);
            dfree(p.d_halo, h->stream);
        }
    h->plans.clear();
    h->mh_plans.clear();
    h->planned = false;
    h->mh_strips = 0;
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    if (h->graph) cudaGraphDestroy(h->graph);
    h->gexec = nullptr;
    h->graph = nullptr;
}

uint32_t gcd32(uint32_t a, uint32_t b) { return b ? gcd32(b, a % b) : a; }

// Rows a strip boundary must be a multiple of, so that every strip starts
// at a stream index that is a multiple of 32 (whole warps per strip).
uint32_t align_rows(const IsingLat &t)
{
    const uint32_t spr = t.L / 2 / t.G;
    return 32 / gcd32(spr, 32);
}

size_t seg_smem(const IsingLat &t, uint32_t rows, uint32_t hd = 1)
{
    const size_t rb = t.layout == ISING_INT8 ? t.L / 2 : t.W * 4;
    return (2 * (rows + 2 * hd) * rb + 15) / 16 * 16;
}

struct SegPlan {
    uint32_t lat, y0, y1;
};

int materialize_plan(ising_t h, int kind, int layout, const std::vector<std::vector<SegPlan>> &blocks, Plan &P,
                     bool multihit, unsigned cfg_threads);
int plan_blocks(ising_t h, const std::vector<uint32_t> &ids, double target, std::vector<std::vector<SegPlan>> &blocks);

// Plans one kind group: splits big lattices into aligned row strips, packs
// small whole lattices into shared blocks, and picks the block shape.
int build_plan(ising_t h, int kind, int layout, const std::vector<uint32_t> &ids, Plan &P)
{
    int dev = 0, sms = 0;
    RNGX_CHECK_CUDA(cudaGetDevice(&dev));
    RNGX_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int per_sm = h->cfg_ctas_per_sm > 0 ? h->cfg_ctas_per_sm : 1;
    unsigned cfg_threads = h->cfg_threads;
    uint64_t total_sites = 0;
    for (uint32_t id : ids) total_sites += static_cast<uint64_t>(h->lats[id].L) * h->lats[id].L;
    // about one block per SM (or per_sm), but no fewer than 1024 sites per
    // block: smaller strips spend their time waiting on their neighbours
    double min_sites = h->cfg_min_sites ? static_cast<double>(h->cfg_min_sites) : 1024.0;
    if (!h->batch && ids.size() == 1 && !h->cfg_threads && !h->cfg_ctas_per_sm && !h->cfg_min_sites) {
        // a single lattice without a tuned shape takes the shapes the
        // autotuner finds: one block with one stream per thread when its
        // streams fit (no exchange at all); when one block per SM needs
        // more than 1024 streams, one block of 1024 threads per SM (a halo
        // of two rows, kernel mode 6, or a polling last warp, mode 5; see
        // materialize_plan) if its strips fit those layouts, else two blocks
        // of 512 threads with two resident streams each per SM (all of these
        // fit the device)
        const IsingLat &t = h->lats[ids[0]];
        const uint64_t n = t.nstreams;
        if (n <= 1024) {
            min_sites = static_cast<double>(total_sites);
            cfg_threads = static_cast<unsigned>(std::max<uint64_t>(32, (n + 31) / 32 * 32));
        } else if (n > static_cast<uint64_t>(sms) * 1024 && n <= static_cast<uint64_t>(sms) * 2048) {
            const uint64_t spr = t.L / 2 / t.G, rmax = (t.L + sms - 1) / sms;
            if (spr % 32 == 0 && 2 * spr <= 1024 - 32 && rmax * spr <= 2 * (1024 - 32) && t.L >= 2 * sms) {
                cfg_threads = 1024;
            } else {
                per_sm = 2;
                cfg_threads = 512;
            }
        }
    }
    const uint64_t target_blocks = static_cast<uint64_t>(sms) * per_sm;
    double target = std::max(min_sites, static_cast<double>(total_sites) / target_blocks);
    std::vector<std::vector<SegPlan>> blocks;
    // each lattice's strip count is rounded on its own, so the blocks can
    // outnumber target_blocks; a larger target per block then brings them
    // back within what the device holds at once
    for (int attempt = 0; attempt < 16; attempt++) {
        int st = plan_blocks(h, ids, target, blocks);
        if (st != RNG_OK) return st;
        if (blocks.size() <= target_blocks) break;
        target *= 1.02 * static_cast<double>(blocks.size()) / static_cast<double>(target_blocks);
    }
    return materialize_plan(h, kind, layout, blocks, P, false, cfg_threads);
}

// Strips and packed whole lattices of about `target` sites each, one list
// per thread block.
int plan_blocks(ising_t h, const std::vector<uint32_t> &ids, double target, std::vector<std::vector<SegPlan>> &blocks)
{
    blocks.clear();
    std::vector<std::pair<uint64_t, uint32_t>> whole;  // (sites, lattice) packed later
    for (uint32_t id : ids) {
        const IsingLat &t = h->lats[id];
        const uint64_t sites = static_cast<uint64_t>(t.L) * t.L;
        const uint32_t ar = align_rows(t);
        const bool splittable = t.L % ar == 0 && (t.layout == ISING_MULTISPIN32 || t.L % 8 == 0) && t.L >= 2 * ar;
        uint64_t k = static_cast<uint64_t>(std::llround(static_cast<double>(sites) / target));
        const uint32_t units = splittable ? t.L / ar : 1;
        k = std::min<uint64_t>(std::max<uint64_t>(k, 1), units);
        // a strip must fit in shared memory
        while (k < units && seg_smem(t, static_cast<uint32_t>((units + k - 1) / k) * ar) > kSmemCap) k++;
        if (k <= 1 || !splittable) {
            if (seg_smem(t, t.L) > kSmemCap) {
                set_error("Ising: lattice L=%u cannot be split for the persistent kernel", t.L);
                return RNG_EUNSUPPORTED;
            }
            whole.push_back({sites, id});
            continue;
        }
        for (uint64_t b = 0; b < k; b++) {
            const uint32_t u0 = static_cast<uint32_t>(b * units / k), u1 = static_cast<uint32_t>((b + 1) * units / k);
            blocks.push_back({{id, u0 * ar, u1 * ar}});
        }
    }
    // first-fit decreasing of whole lattices into blocks of about `target` sites
    std::sort(whole.begin(), whole.end(), [](auto &a, auto &b) { return a.first > b.first; });
    std::vector<std::pair<uint64_t, size_t>> bins;  // (sites, smem)
    std::vector<std::vector<SegPlan>> wb;
    for (auto &w : whole) {
        const IsingLat &t = h->lats[w.second];
        const size_t sm = seg_smem(t, t.L);
        bool placed = false;
        for (size_t b = 0; b < bins.size() && !placed; b++) {
            if (bins[b].first + w.first <= target * 1.05 && bins[b].second + sm <= kSmemCap &&
                wb[b].size() < static_cast<size_t>(kPersistMaxSegs)) {
                bins[b].first += w.first;
                bins[b].second += sm;
                wb[b].push_back({w.second, 0, t.L});
                placed = true;
            }
        }
        if (!placed) {
            bins.push_back({w.first, sm});
            wb.push_back({{w.second, 0, t.L}});
        }
    }
    for (auto &b : wb) blocks.push_back(b);
    return RNG_OK;
}

// Segments, ring links, block shape and device buffers of a list of blocks
// (each a list of strips).  Strips of one lattice are linked into a ring in
// list order; a strip's coarse colour is its position in that ring mod 2.
int materialize_plan(ising_t h, int kind, int layout, const std::vector<std::vector<SegPlan>> &blocks, Plan &P,
                     bool multihit, unsigned cfg_threads)
{
    std::vector<SegDev> segs;
    std::vector<uint32_t> cta(1, 0);
    std::vector<std::vector<uint32_t>> lat_strips(h->lats.size());
    size_t smem_max = 0;
    uint64_t max_streams = 0;
    uint32_t halo_rb = 4;
    for (auto &blk : blocks) {
        size_t off = 0;
        uint64_t streams = 0;
        for (auto &sp : blk) {
            const IsingLat &t = h->lats[sp.lat];
            SegDev d;
            d.lat = sp.lat;
            d.coarse = static_cast<uint32_t>(lat_strips[sp.lat].size() & 1);
            d.y0 = sp.y0;
            d.y1 = sp.y1;
            d.smem_off = static_cast<uint32_t>(off);
            d.up = d.down = -1;
            const uint64_t spr = t.L / 2 / t.G;
            d.s0 = static_cast<uint64_t>(sp.y0) * spr;
            d.s1 = static_cast<uint64_t>(sp.y1) * spr;
            if (sp.y0 == 0 && sp.y1 == t.L) d.s1 = (t.nstreams + 31) / 32 * 32;  // whole warps
            off += seg_smem(t, sp.y1 - sp.y0);
            streams += d.s1 - d.s0;
            lat_strips[sp.lat].push_back(static_cast<uint32_t>(segs.size()));
            halo_rb = std::max<uint32_t>(halo_rb, t.layout == ISING_INT8 ? t.L / 2 : t.W * 4);
            segs.push_back(d);
        }
        smem_max = std::max(smem_max, off);
        max_streams = std::max(max_streams, streams);
        cta.push_back(static_cast<uint32_t>(segs.size()));
    }
    for (auto &ls : lat_strips) {
        if (ls.size() <= 1) continue;
        const size_t n = ls.size();
        for (size_t i = 0; i < n; i++) {
            segs[ls[i]].up = static_cast<int32_t>(ls[(i + n - 1) % n]);
            segs[ls[i]].down = static_cast<int32_t>(ls[(i + 1) % n]);
        }
    }
    // block shape: up to 4 streams per thread keep their state in registers;
    // beyond that the kernel streams the states through L2 each half-sweep
    unsigned threads = cfg_threads ? cfg_threads : 256;
    while (!cfg_threads && threads < 1024 && (max_streams + threads - 1) / threads > 4) threads *= 2;
    uint64_t spt = std::min<uint64_t>(4, std::max<uint64_t>(1, (max_streams + threads - 1) / threads));
    // exact checkerboard at 1024 threads: one strip per block with roles
    // split by warp (kernel mode 5) when every block's strip fits: its
    // first and last rows in slot 0 of the first threads, all its streams
    // in two slots of the threads other than the polling last warp
    bool split = !multihit && threads == 1024 && !blocks.empty();
    for (size_t b = 0; b < blocks.size() && split; b++) {
        if (blocks[b].size() != 1) {
            split = false;
            break;
        }
        const SegDev &d = segs[cta[b]];
        const IsingLat &t = h->lats[d.lat];
        const uint64_t spr = t.L / 2 / t.G, R = d.y1 - d.y0, nc = threads - 32;
        if (d.up < 0 || R < 2 || spr % 32 || 2 * spr > nc || d.s1 - d.s0 != R * spr || R * spr > 2 * nc) split = false;
    }
    // the same with a halo of two rows (kernel mode 6): every block one
    // strip of 4 .. 10 rows whose rows and the two halo copies fill the
    // cells of the kernel's layout (four cells of one row's streams per slot)
    // (automatic choice: every generator but Philox4x32-10 on int8 spins,
    // whose copies' extra ten-round draws cost more than the exchanges they
    // save, measured on GB300)
    const bool deep_auto = !(kind == RNG_PHILOX4X32_10 && layout == ISING_INT8);
    bool deep = !multihit && threads == 1024 && !blocks.empty() &&
                (h->cfg_halo_depth == 2 || (h->cfg_halo_depth == 0 && deep_auto));
    size_t deep_smem = 0;
    for (size_t b = 0; b < blocks.size() && deep; b++) {
        if (blocks[b].size() != 1) {
            deep = false;
            break;
        }
        const SegDev &d = segs[cta[b]];
        const IsingLat &t = h->lats[d.lat];
        const uint64_t spr = t.L / 2 / t.G, R = d.y1 - d.y0;
        const uint64_t row_words = (t.layout == ISING_INT8 ? t.L / 2 : t.W * 4) / 4;
        if (d.up < 0 || R < 4 || R > 10 || spr % 32 || 4 * spr > threads || 6 * row_words > threads ||
            d.s1 - d.s0 != R * spr || seg_smem(t, static_cast<uint32_t>(R), 2) > kSmemCap)
            deep = false;
        else
            deep_smem = std::max(deep_smem, seg_smem(t, static_cast<uint32_t>(R), 2));
    }
    if (deep) split = false;
    if (split) spt = 2;
    if (spt >= 2 && threads > 512 && !split && !deep) {  // other multi-slot kernels are built for at most 512 threads
        threads = 512;
        spt = std::min<uint64_t>(4, (max_streams + threads - 1) / threads);
    }
    // plans whose largest blocks stream their states anyway keep one slot
    // per thread: the kernel then needs fewer registers, so more blocks fit
    // an SM to hide the L2 loads of the states (1.2x on a batch of 256
    // lattices of 16 .. 512)
    if (!multihit && max_streams > 4ull * threads) spt = 1;
    bool fixed = false;  // fixed slot roles (the kernel's modes 2 and 3)
    if (multihit && !cfg_threads && max_streams <= 2048) {
        // one stream of each coarse colour per thread: every thread works
        // in both phases (the multi-hit kernel runs two slots at up to 1024)
        threads = static_cast<unsigned>(std::max<uint64_t>(32, max_streams / 2));
        spt = 2;
        // blocks hold a coarse-0 strip then a coarse-1 strip of `threads`
        // streams each: slot 0 and slot 1 of every thread, in that order
        fixed = true;
        for (size_t b = 0; b < blocks.size() && fixed; b++) {
            const auto &blk = blocks[b];
            if (blk.size() != 2) fixed = false;
            for (size_t i = 0; i < blk.size() && fixed; i++) {
                const SegDev &d = segs[cta[b] + i];
                if (d.coarse != i || d.s1 - d.s0 != threads) fixed = false;
            }
        }
    }
    P.kind = kind;
    P.layout = layout;
    P.smax = spt <= 1 ? 1 : (spt <= 2 ? 2 : 4);
    if (deep) {
        P.smax = 3;
        smem_max = deep_smem;  // one strip per block at offset 0
    }
    if (!multihit && P.smax == 2) {
        // exact checkerboard: one strip per block whose first and last rows
        // fill at most one slot of every thread and the rows between another
        fixed = true;
        for (size_t b = 0; b < blocks.size() && fixed; b++) {
            if (blocks[b].size() != 1) {
                fixed = false;
                break;
            }
            const SegDev &d = segs[cta[b]];
            const IsingLat &t = h->lats[d.lat];
            const uint64_t spr = t.L / 2 / t.G, R = d.y1 - d.y0;
            if (R < 2 || spr % 32 || 2 * spr > threads || (R - 2) * spr > threads || d.s1 - d.s0 != R * spr)
                fixed = false;
        }
    }
    P.fixed_slots = fixed && P.smax == 2 ? 1 : 0;
    if (split) P.fixed_slots = 3;
    if (deep) P.fixed_slots = 4;
    if (!multihit && P.smax == 1 && max_streams <= threads) {
        // every block one whole lattice whose streams fit one slot per thread
        bool whole = true;
        for (size_t b = 0; b < blocks.size() && whole; b++)
            if (blocks[b].size() != 1 || segs[cta[b]].up >= 0) whole = false;
        if (whole) P.fixed_slots = 2;
    }
    P.threads = threads;
    P.nblocks = static_cast<unsigned>(blocks.size());
    P.smem = std::max<size_t>(smem_max, 16);
    P.nsegs = static_cast<uint32_t>(segs.size());
    P.halo_row_bytes = (2 * halo_rb + 15) / 16 * 16;  // one 64-bit (tag, data) word per 32 data bits
    RNGX_CHECK(dalloc(reinterpret_cast<void **>(&P.d_segs), segs.size() * sizeof(SegDev), h->stream));
    RNGX_CHECK(dalloc(reinterpret_cast<void **>(&P.d_cta), cta.size() * sizeof(uint32_t), h->stream));
    RNGX_CHECK(dalloc(reinterpret_cast<void **>(&P.d_halo), P.halo_bytes(), h->stream));
    RNGX_CHECK_CUDA(cudaStreamSynchronize(h->stream));
    RNGX_CHECK_CUDA(cudaMemcpy(P.d_segs, segs.data(), segs.size() * sizeof(SegDev), cudaMemcpyHostToDevice));
    RNGX_CHECK_CUDA(cudaMemcpy(P.d_cta, cta.data(), cta.size() * sizeof(uint32_t), cudaMemcpyHostToDevice));
    int max_blocks = 0;
    PersistArgs dummy;
    memset(&dummy, 0, sizeof(dummy));
    dummy.k_hits = multihit ? 1 : 0;  // selects the kernel whose occupancy is asked
    dummy.fixed_slots = static_cast<uint32_t>(P.fixed_slots);
    RNGX_CHECK(dispatch_persist(kind, layout, P.smax, dummy, 0, P.threads, P.smem, h->stream, &max_blocks));
    if (static_cast<int>(P.nblocks) > max_blocks) {
        set_error("Ising: plan needs %u co-resident blocks, device holds %d", P.nblocks, max_blocks);
        return RNG_EUNSUPPORTED;
    }
    return RNG_OK;
}

// The multi-hit plan of a single lattice: n_strips equal row strips, block
// m holding strips 2m (coarse colour 0) and 2m + 1 (coarse colour 1), so
// that every thread has streams in both and works in both phases.
int build_multihit_plan(ising_t h, uint32_t n_strips, Plan &P)
{
    const IsingLat &t = h->lats[0];
    const uint32_t R = t.L / n_strips;
    const uint64_t per_strip = static_cast<uint64_t>(R) * (t.L / 2 / t.G);
    if (per_strip % 32) {
        set_error("Ising multi-hit: a strip's %llu streams must be whole warps (a multiple of 32)",
                  static_cast<unsigned long long>(per_strip));
        return RNG_EINVAL;
    }
    if (t.layout == ISING_INT8 && t.L % 8) {
        set_error("Ising multi-hit: the int8 layout exchanges rows as 32-bit words and needs L %% 8 == 0");
        return RNG_EINVAL;
    }
    if (2 * seg_smem(t, R) > kSmemCap) {
        set_error("Ising multi-hit: two strips of %u rows exceed the shared memory of a block", R);
        return RNG_EUNSUPPORTED;
    }
    std::vector<std::vector<SegPlan>> blocks;
    for (uint32_t m = 0; m < n_strips / 2; m++)
        blocks.push_back({{0, 2 * m * R, (2 * m + 1) * R}, {0, (2 * m + 1) * R, (2 * m + 2) * R}});
    return materialize_plan(h, t.kind, t.layout, blocks, P, true, h->cfg_threads);
}

// Splits the lattices of one kind group into waves whose streams fit the
// device's registers (kWaveStreamsPerSm per SM: two blocks of 512 threads
// with two resident streams each), first fit in decreasing size; a lattice
// larger than that is a wave of its own.  Each wave is one persistent launch
// per chunk of sweeps, its generator states in registers for the whole
// launch; lattices are independent, so running them in waves changes no
// result, while one launch over all of them would stream every state
// through L2 in every half-sweep.
std::vector<std::vector<uint32_t>> split_waves(const ising_t h, std::vector<uint32_t> ids, uint64_t cap_streams)
{
    std::stable_sort(ids.begin(), ids.end(),
                     [&](uint32_t a, uint32_t b) { return h->lats[a].nstreams > h->lats[b].nstreams; });
    std::vector<std::vector<uint32_t>> waves;
    std::vector<uint64_t> used;
    for (uint32_t id : ids) {
        const uint64_t n = h->lats[id].nstreams;
        size_t w = 0;
        while (w < waves.size() && used[w] + n > cap_streams) w++;
        if (w == waves.size()) {
            waves.emplace_back();
            used.push_back(0);
        }
        waves[w].push_back(id);
        used[w] += n;
    }
    for (auto &w : waves) std::sort(w.begin(), w.end());
    return waves;
}

int ensure_plan(ising_t h)
{
    if (h->planned) return RNG_OK;
    int dev = 0, sms = 0;
    RNGX_CHECK_CUDA(cudaGetDevice(&dev));
    RNGX_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const uint64_t cap_streams = static_cast<uint64_t>(sms) * kWaveStreamsPerSm;
    // one group per (kind, layout), each in waves of register-resident size
    std::vector<std::pair<int, int>> keys;
    for (auto &t : h->lats)
        if (std::find(keys.begin(), keys.end(), std::make_pair(t.kind, t.layout)) == keys.end())
            keys.push_back({t.kind, t.layout});
    for (auto &k : keys) {
        std::vector<uint32_t> ids;
        for (uint32_t i = 0; i < h->lats.size(); i++)
            if (h->lats[i].kind == k.first && h->lats[i].layout == k.second) ids.push_back(i);
        for (auto &wave : split_waves(h, ids, cap_streams)) {
            Plan P;
            int st = build_plan(h, k.first, k.second, wave, P);
            h->plans.push_back(P);
            if (st != RNG_OK) {
                free_plans(h);
                return st;
            }
        }
    }
    h->planned = true;
    return RNG_OK;
}

int ensure_meas(ising_t h, uint64_t need)
{
    bool changed = false;
    for (auto &t : h->lats) {
        if (t.meas_cap >= need) continue;
        dfree(t.meas, h->stream);
        t.meas = nullptr;
        RNGX_CHECK(dalloc(reinterpret_cast<void **>(&t.meas), 2 * need * sizeof(int64_t), h->stream));
        t.meas_cap = need;
        changed = true;
    }
    if (changed || !h->d_lats) RNGX_CHECK(upload_lats(h));
    return RNG_OK;
}

// Sweeps (k_hits = 0) or multi-hit rounds (k_hits = k) per persistent launch.
uint64_t chunk_units(uint32_t k_hits) { return k_hits ? std::max<uint64_t>(1, kChunkSweeps / k_hits) : kChunkSweeps; }

// Enqueues n_units persistent sweeps (k_hits = 0) or multi-hit rounds of k
// sweeps per strip phase (k_hits = k) of every lattice (no host sync).
int enqueue_persistent(ising_t h, std::vector<Plan> &plans, uint64_t n_units, uint32_t k_hits,
                       uint32_t measure_every, cudaStream_t s)
{
    const uint64_t per_launch = chunk_units(k_hits);
    const uint64_t sweeps_per_unit = k_hits ? k_hits : 1;
    uint64_t done = 0;
    while (done < n_units) {
        const uint64_t chunk = std::min(per_launch, n_units - done);
        const uint64_t n_meas = measure_every ? (chunk + (done % measure_every)) / measure_every : 0;
        for (auto &t : h->lats)
            if (n_meas) RNGX_CHECK_CUDA(cudaMemsetAsync(t.meas, 0, 2 * n_meas * sizeof(int64_t), s));
        for (auto &P : plans) {
            // halo words carry phase tags that restart at every launch
            RNGX_CHECK_CUDA(cudaMemsetAsync(P.d_halo, 0, P.halo_bytes(), s));
            PersistArgs a;
            a.lats = h->d_lats;
            a.segs = P.d_segs;
            a.cta_seg = P.d_cta;
            a.halo = P.d_halo;
            a.halo_row_bytes = P.halo_row_bytes;
            a.halo_bytes = P.halo_bytes();
            a.err = h->d_err;
            a.n_sweeps = chunk;
            a.measure_every = measure_every;
            a.sweep0 = done;
            a.mute_seg = h->mute_seg;
            a.wait_budget_ns = h->wait_budget_ns;
            a.k_hits = k_hits;
            a.fixed_slots = static_cast<uint32_t>(P.fixed_slots);
            RNGX_CHECK(dispatch_persist(P.kind, P.layout, P.smax, a, P.nblocks, P.threads, P.smem, s, nullptr));
        }
        for (auto &t : h->lats) {
            if (n_meas) k_meas_finalize<<<1, 256, 0, s>>>(t.meas, static_cast<uint32_t>(n_meas), t.acc);
            k_add_u64<<<1, 1, 0, s>>>(t.pos_dev, 2 * t.G * sweeps_per_unit * chunk);
        }
        RNGX_CHECK_LAUNCH();
        done += chunk;
    }
    return RNG_OK;
}

int enqueue_persistent(ising_t h, uint64_t n_sweeps, uint32_t measure_every, cudaStream_t s)
{
    return enqueue_persistent(h, h->plans, n_sweeps, 0, measure_every, s);
}

void advance_host_pos(ising_t h, uint64_t n_sweeps)
{
    for (auto &t : h->lats) t.rng->g.pos += 2 * t.G * n_sweeps;
}

int check_err(ising_t h)
{
    int err = 0;
    RNGX_CHECK_CUDA(cudaStreamSynchronize(h->stream));
    if (fault_timeout()) return injected("a neighbour wait of the persistent sweep", RNG_ETIMEOUT);
    RNGX_CHECK_CUDA(cudaMemcpy(&err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (err) {
        set_error("Ising: a persistent sweep gave up waiting for a neighbouring strip (status %d)", err);
        cudaMemset(h->d_err, 0, sizeof(int));
        return RNG_ETIMEOUT;
    }
    return RNG_OK;
}

int valid(ising_t h)
{
    if (!h) {
        set_error("null Ising handle");
        return RNG_EINVAL;
    }
    return RNG_OK;
}

int observe(ising_t h, uint32_t idx, int64_t *E, int64_t *M, int64_t acc[4], uint64_t *n_meas)
{
    RNGX_CHECK(valid(h));
    if (idx >= h->lats.size()) {
        set_error("Ising: lattice index %u out of range", idx);
        return RNG_EINVAL;
    }
    RNGX_CHECK(check_err(h));
    IsingLat &t = h->lats[idx];
    RNGX_CHECK_CUDA(cudaMemsetAsync(t.acc + 5, 0, 2 * sizeof(int64_t), h->stream));
    const uint64_t n = t.layout == ISING_INT8 ? static_cast<uint64_t>(t.L) * t.L : static_cast<uint64_t>(t.L) * t.W;
    k_energy<<<static_cast<unsigned>((n + 255) / 256), 256, 0, h->stream>>>(lat_dev(t));
    RNGX_CHECK_LAUNCH();
    int64_t host[8];
    RNGX_CHECK_CUDA(cudaStreamSynchronize(h->stream));
    RNGX_CHECK_CUDA(cudaMemcpy(host, t.acc, sizeof(host), cudaMemcpyDeviceToHost));
    if (E) *E = host[5];
    if (M) *M = host[6];
    if (acc)
        for (int i = 0; i < 4; i++) acc[i] = host[i];
    if (n_meas) *n_meas = static_cast<uint64_t>(host[4]);
    return RNG_OK;
}

int get_spins(ising_t h, uint32_t idx, int8_t *out)
{
    RNGX_CHECK(valid(h));
    if (!out || idx >= h->lats.size()) {
        set_error("Ising: null output or bad lattice index");
        return RNG_EINVAL;
    }
    RNGX_CHECK(check_err(h));
    IsingLat &t = h->lats[idx];
    if (t.layout == ISING_INT8) {
        RNGX_CHECK_CUDA(cudaMemcpy(out, t.spins, t.spin_bytes, cudaMemcpyDeviceToHost));
        return RNG_OK;
    }
    std::vector<uint32_t> planes(t.spin_bytes / 4);
    RNGX_CHECK_CUDA(cudaMemcpy(planes.data(), t.spins, t.spin_bytes, cudaMemcpyDeviceToHost));
    for (uint32_t y = 0; y < t.L; y++)
        for (uint32_t x = 0; x < t.L; x++) {
            const uint32_t c = (x + y) & 1, xh = x >> 1;
            const uint32_t w = planes[static_cast<size_t>(c) * t.L * t.W + static_cast<size_t>(y) * t.W + xh / 32];
            out[static_cast<size_t>(y) * t.L + x] = ((w >> (xh % 32)) & 1) ? -1 : 1;
        }
    return RNG_OK;
}

}  // namespace

namespace rngx {

// Puts a single-lattice handle back in the state ising_create(L, beta,
// layout, kind, flags, seed, G) leaves, keeping its memory and launch plan
// (for the server's pool of lattices): new thresholds, reseeded streams,
// initial spins, zeroed accumulators, all on the handle's stream.
int ising_reset_lattice(ising_t h, double beta, uint64_t seed)
{
    RNGX_CHECK(valid(h));
    if (h->lats.size() != 1 || !(beta >= 0.0) || !std::isfinite(beta)) {
        set_error("ising_reset_lattice: one lattice per handle and a finite beta >= 0");
        return RNG_EINVAL;
    }
    IsingLat &t = h->lats[0];
    cudaStream_t s = h->stream;
    t.beta = beta;
    t.seed = seed;
    t.T4 = static_cast<uint64_t>(std::floor(4294967296.0 * std::exp(-beta * 4.0)));
    t.T8 = static_cast<uint64_t>(std::floor(4294967296.0 * std::exp(-beta * 8.0)));
    RNGX_CHECK(rng_seed(t.rng, seed));
    const uint64_t seed2 = seed ^ 0x5350494EULL;
    if (t.layout == ISING_INT8) {
        const uint64_t n = static_cast<uint64_t>(t.L) * t.L;
        k_init_int8<<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(static_cast<int8_t *>(t.spins), t.L, seed2);
    } else {
        const uint64_t n = 2ull * t.L * t.W;
        k_init_ms<<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(static_cast<uint32_t *>(t.spins), t.L, t.W,
                                                                          seed2);
    }
    RNGX_CHECK_LAUNCH();
    RNGX_CHECK_CUDA(cudaMemsetAsync(t.acc, 0, 8 * sizeof(int64_t), s));
    RNGX_CHECK_CUDA(cudaMemsetAsync(t.pos_dev, 0, sizeof(uint64_t), s));
    RNGX_CHECK_CUDA(cudaMemsetAsync(h->d_err, 0, sizeof(int), s));
    // the device copy of the lattice's parameters (thresholds, generator
    // position), staged from the handle so that the copy stays ordered
    h->host_lat = lat_dev(t);
    RNGX_CHECK_CUDA(cudaMemcpyAsync(h->d_lats, &h->host_lat, sizeof(LatDev), cudaMemcpyHostToDevice, s));
    return RNG_OK;
}

}  // namespace rngx

extern "C" {

int ising_create(ising_t *out, uint32_t L, double beta, int layout, int rng_kind, uint32_t rng_flags, uint64_t seed,
                 uint32_t G, void *cuda_stream)
{
    if (!out) {
        set_error("null output handle pointer");
        return RNG_EINVAL;
    }
    *out = nullptr;
    ising_s *h = new (std::nothrow) ising_s();
    if (!h) return RNG_ENOMEM;
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    h->lats.resize(1);
    int st = lat_create(h->lats[0], L, beta, layout, rng_kind, rng_flags, seed, G, h->stream);
    if (st == RNG_OK) st = dalloc(reinterpret_cast<void **>(&h->d_err), sizeof(int), h->stream);
    if (st == RNG_OK) st = cudaMemsetAsync(h->d_err, 0, sizeof(int), h->stream) == cudaSuccess ? RNG_OK : RNG_ECUDA;
    if (st == RNG_OK) st = upload_lats(h);
    if (st != RNG_OK) {
        ising_destroy(h);
        return st;
    }
    *out = h;
    return RNG_OK;
}

int ising_batch_create(ising_t *out, uint32_t n, const uint32_t *L, const double *beta, const int *rng_kind,
                       uint64_t seed, uint32_t G, void *cuda_stream)
{
    if (!out || !L || !beta || !rng_kind || n == 0) {
        set_error("ising_batch_create: null argument or empty batch");
        return RNG_EINVAL;
    }
    *out = nullptr;
    ising_s *h = new (std::nothrow) ising_s();
    if (!h) return RNG_ENOMEM;
    h->batch = true;
    h->master_seed = seed;
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    for (uint32_t b = 0; b < n; b++)
        if (is_block_shared(rng_kind[b])) {
            delete h;
            set_error("ising_batch_create: the block-shared generators (kind %d) sweep one lattice per handle",
                      rng_kind[b]);
            return RNG_EUNSUPPORTED;
        }
    h->lats.resize(n);
    int st = RNG_OK;
    for (uint32_t b = 0; b < n && st == RNG_OK; b++) {
        // lattice b is seeded with the master seed's SplitMix64 word w_b
        uint64_t z = seed + (static_cast<uint64_t>(b) + 1) * 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        st = lat_create(h->lats[b], L[b], beta[b], ISING_INT8, rng_kind[b], 0, z, G, h->stream);
    }
    if (st == RNG_OK) st = dalloc(reinterpret_cast<void **>(&h->d_err), sizeof(int), h->stream);
    if (st == RNG_OK) st = cudaMemsetAsync(h->d_err, 0, sizeof(int), h->stream) == cudaSuccess ? RNG_OK : RNG_ECUDA;
    if (st == RNG_OK) st = upload_lats(h);
    if (st != RNG_OK) {
        ising_destroy(h);
        return st;
    }
    *out = h;
    return RNG_OK;
}

int ising_destroy(ising_t h)
{
    if (!h) return RNG_OK;
    free_plans(h);
    for (auto &t : h->lats) lat_free(t, h->stream);
    dfree(h->d_lats, h->stream);
    dfree(h->d_err, h->stream);
    cudaError_t e = cudaStreamSynchronize(h->stream);
    delete h;
    return e == cudaSuccess ? RNG_OK : cuda_fail(e, "ising_destroy");
}

int ising_sweep(ising_t h, uint64_t n_sweeps, uint32_t measure_every, void *cuda_stream)
{
    RNGX_CHECK(valid(h));
    if (n_sweeps == 0) return RNG_OK;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    // warp-shared generators stream their states each half-sweep: they run
    // the per-half-sweep path
    if (h->plan_unfit || is_block_shared(h->lats[0].kind)) return ising_sweep_plain(h, n_sweeps, measure_every, cuda_stream);
    if (!h->batch && !h->planned) {
        const int st = ensure_plan(h);
        if (st == RNG_EUNSUPPORTED) {
            h->plan_unfit = true;
            // no row-strip plan fits the device (a lattice too large for
            // co-resident blocks): the per-half-sweep kernels give the same
            // result
            return ising_sweep_plain(h, n_sweeps, measure_every, cuda_stream);
        }
        RNGX_CHECK(st);
    }
    RNGX_CHECK(ensure_plan(h));
    RNGX_CHECK(ensure_meas(h, measure_every ? std::max<uint64_t>(1, kChunkSweeps / measure_every + 1) : 1));
    // the device copy of the draw position follows the host's (which a
    // restored generator state may have moved)
    for (auto &t : h->lats) k_set_u64<<<1, 1, 0, s>>>(t.pos_dev, t.rng->g.pos);
    RNGX_CHECK(enqueue_persistent(h, n_sweeps, measure_every, s));
    advance_host_pos(h, n_sweeps);
    return RNG_OK;
}

int ising_sweep_multihit(ising_t h, uint64_t n_rounds, uint32_t k, uint32_t n_strips, uint32_t measure_every,
                         void *cuda_stream)
{
    RNGX_CHECK(valid(h));
    if (h->lats.size() != 1) {
        set_error("Ising multi-hit: one lattice per handle (batch handles sweep with ising_batch_sweep)");
        return RNG_EUNSUPPORTED;
    }
    const IsingLat &t = h->lats[0];
    if (is_block_shared(t.kind)) {
        set_error("Ising multi-hit: not built for the block-shared generators (kind %d)", t.kind);
        return RNG_EUNSUPPORTED;
    }
    if (k == 0 || k > kMaxHits || n_strips < 2 || n_strips % 2 || t.L % n_strips) {
        set_error("Ising multi-hit: need 1 <= k <= %u and an even strip count >= 2 that divides L=%u (got k=%u, "
                  "n_strips=%u)",
                  kMaxHits, t.L, k, n_strips);
        return RNG_EINVAL;
    }
    if (n_rounds == 0) return RNG_OK;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    if (h->mh_strips != n_strips) {
        for (auto &p : h->mh_plans) {
            dfree(p.d_segs, h->stream);
            dfree(p.d_cta, h->stream);
            dfree(p.d_halo, h->stream);
        }
        h->mh_plans.clear();
        h->mh_strips = 0;
        Plan P;
        const int st = build_multihit_plan(h, n_strips, P);
        h->mh_plans.push_back(P);
        if (st != RNG_OK) {
            free_plans(h);
            return st;
        }
        h->mh_strips = n_strips;
    }
    RNGX_CHECK(ensure_meas(h, measure_every ? std::max<uint64_t>(1, chunk_units(k) / measure_every + 1) : 1));
    for (auto &l : h->lats) k_set_u64<<<1, 1, 0, s>>>(l.pos_dev, l.rng->g.pos);
    RNGX_CHECK(enqueue_persistent(h, h->mh_plans, n_rounds, k, measure_every, s));
    advance_host_pos(h, n_rounds * k);
    return RNG_OK;
}

int ising_sweep_plain(ising_t h, uint64_t n_sweeps, uint32_t measure_every, void *cuda_stream)
{
    RNGX_CHECK(valid(h));
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    for (auto &t : h->lats) {
        LatDev d = lat_dev(t);
        const uint64_t n = t.layout == ISING_INT8 ? static_cast<uint64_t>(t.L) * t.L : static_cast<uint64_t>(t.L) * t.W;
        const bool shared = is_block_shared(t.kind);
        for (uint64_t sw = 0; sw < n_sweeps; sw++) {
            for (int c = 0; c < 2; c++) {
                if (shared) {
                    // this half-sweep's 32 G words of every generator (the
                    // generator advances its own position), then the sites
                    RNGX_CHECK(rng_generate_u32(t.rng, t.draws, 32ull * t.G, RNG_INSTANCE_MAJOR, s));
                    const unsigned nb = static_cast<unsigned>((t.nstreams + 255) / 256);
                    if (t.layout == ISING_INT8) k_ising_half_given<ISING_INT8><<<nb, 256, 0, s>>>(d, c, t.draws);
                    else k_ising_half_given<ISING_MULTISPIN32><<<nb, 256, 0, s>>>(d, c, t.draws);
                    RNGX_CHECK_LAUNCH();
                    continue;
                }
                d.rng.pos = t.rng->g.pos;
                RNGX_CHECK(dispatch_half(t.kind, d, c, s));
                t.rng->g.pos += t.G;
            }
            if (measure_every && (sw + 1) % measure_every == 0) {
                RNGX_CHECK_CUDA(cudaMemsetAsync(t.acc + 5, 0, 2 * sizeof(int64_t), s));
                k_energy<<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(d);
                k_accumulate_now<<<1, 1, 0, s>>>(t.acc);
            }
        }
        k_set_u64<<<1, 1, 0, s>>>(t.pos_dev, t.rng->g.pos);
        RNGX_CHECK_LAUNCH();
    }
    return RNG_OK;
}

int ising_observables(ising_t h, int64_t *E, int64_t *M, int64_t acc[4], uint64_t *n_meas)
{
    return observe(h, 0, E, M, acc, n_meas);
}

int ising_batch_observables(ising_t h, uint32_t idx, int64_t *E, int64_t *M, int64_t acc[4], uint64_t *n_meas)
{
    return observe(h, idx, E, M, acc, n_meas);
}

int ising_get_spins(ising_t h, int8_t *host_LxL) { return get_spins(h, 0, host_LxL); }

int ising_batch_get_spins(ising_t h, uint32_t idx, int8_t *host_LxL) { return get_spins(h, idx, host_LxL); }

int ising_set_spins(ising_t h, const int8_t *host_LxL)
{
    RNGX_CHECK(valid(h));
    if (!host_LxL) {
        set_error("null spins");
        return RNG_EINVAL;
    }
    IsingLat &t = h->lats[0];
    const uint64_t n = static_cast<uint64_t>(t.L) * t.L;
    for (uint64_t j = 0; j < n; j++)
        if (host_LxL[j] != 1 && host_LxL[j] != -1) {
            set_error("spins must be +1 or -1");
            return RNG_EINVAL;
        }
    RNGX_CHECK_CUDA(cudaStreamSynchronize(h->stream));
    if (t.layout == ISING_INT8) {
        RNGX_CHECK_CUDA(cudaMemcpy(t.spins, host_LxL, t.spin_bytes, cudaMemcpyHostToDevice));
        return RNG_OK;
    }
    std::vector<uint32_t> planes(t.spin_bytes / 4, 0);
    for (uint32_t y = 0; y < t.L; y++)
        for (uint32_t x = 0; x < t.L; x++) {
            if (host_LxL[static_cast<size_t>(y) * t.L + x] > 0) continue;
            const uint32_t c = (x + y) & 1, xh = x >> 1;
            planes[static_cast<size_t>(c) * t.L * t.W + static_cast<size_t>(y) * t.W + xh / 32] |= 1u << (xh % 32);
        }
    RNGX_CHECK_CUDA(cudaMemcpy(t.spins, planes.data(), t.spin_bytes, cudaMemcpyHostToDevice));
    return RNG_OK;
}

int ising_get_rng(ising_t h, rng_t *rng)
{
    RNGX_CHECK(valid(h));
    if (!rng) {
        set_error("null output");
        return RNG_EINVAL;
    }
    *rng = h->lats[0].rng;
    return RNG_OK;
}

int ising_get_launch(ising_t h, uint32_t *threads, int *ctas_per_sm, uint32_t *min_sites_per_block)
{
    RNGX_CHECK(valid(h));
    if (threads) *threads = h->cfg_threads;
    if (ctas_per_sm) *ctas_per_sm = h->cfg_ctas_per_sm;
    if (min_sites_per_block) *min_sites_per_block = h->cfg_min_sites;
    return RNG_OK;
}

int ising_set_launch(ising_t h, uint32_t threads, int ctas_per_sm, uint32_t min_sites_per_block)
{
    RNGX_CHECK(valid(h));
    if (threads && (threads % 32 || threads > 1024)) {
        set_error("threads per block must be a multiple of 32 up to 1024");
        return RNG_EINVAL;
    }
    if (ctas_per_sm < 0 || ctas_per_sm > 8) {
        set_error("blocks per SM must be in 0..8");
        return RNG_EINVAL;
    }
    RNGX_CHECK_CUDA(cudaStreamSynchronize(h->stream));
    free_plans(h);
    h->plan_unfit = false;
    h->cfg_threads = threads;
    h->cfg_ctas_per_sm = ctas_per_sm;
    h->cfg_min_sites = min_sites_per_block;
    return RNG_OK;
}

int ising_set_halo_depth(ising_t h, uint32_t depth)
{
    RNGX_CHECK(valid(h));
    if (depth > 2) {
        set_error("halo depth must be 0 (automatic), 1 or 2");
        return RNG_EINVAL;
    }
    RNGX_CHECK_CUDA(cudaStreamSynchronize(h->stream));
    free_plans(h);
    h->plan_unfit = false;
    h->cfg_halo_depth = depth;
    return RNG_OK;
}

int ising_get_halo_depth(ising_t h, uint32_t *depth)
{
    RNGX_CHECK(valid(h));
    if (depth) *depth = h->cfg_halo_depth;
    return RNG_OK;
}

int ising_batch_sweep(ising_t h, uint64_t n_sweeps, uint32_t measure_every, void *cuda_stream)
{
    RNGX_CHECK(valid(h));
    if (n_sweeps == 0) return RNG_OK;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    RNGX_CHECK(ensure_plan(h));
    RNGX_CHECK(ensure_meas(h, measure_every ? std::max<uint64_t>(1, kChunkSweeps / measure_every + 1) : 1));
    if (!h->gexec || h->g_sweeps != n_sweeps || h->g_meas != measure_every) {
        if (h->gexec) cudaGraphExecDestroy(h->gexec);
        if (h->graph) cudaGraphDestroy(h->graph);
        h->gexec = nullptr;
        h->graph = nullptr;
        cudaStream_t cs;
        RNGX_CHECK_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        int st = e == cudaSuccess ? enqueue_persistent(h, n_sweeps, measure_every, cs) : cuda_fail(e, "capture");
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(cs, &g);
        if (st == RNG_OK && e != cudaSuccess) st = cuda_fail(e, "cudaStreamEndCapture");
        if (st == RNG_OK) {
            e = cudaGraphInstantiate(&h->gexec, g, 0);
            if (e != cudaSuccess) st = cuda_fail(e, "cudaGraphInstantiate");
        }
        cudaStreamDestroy(cs);
        if (st != RNG_OK) {
            if (g) cudaGraphDestroy(g);
            h->gexec = nullptr;
            return st;
        }
        h->graph = g;
        h->g_sweeps = n_sweeps;
        h->g_meas = measure_every;
    }
    RNGX_CHECK_CUDA(cudaGraphLaunch(h->gexec, s));
    advance_host_pos(h, n_sweeps);
    return RNG_OK;
}

}  // extern "C"

extern "C" int ising_autotune(ising_t h, uint32_t probe_sweeps, uint32_t *threads_out, int *ctas_per_sm_out)
{
    RNGX_CHECK(valid(h));
    if (!h->batch && is_block_shared(h->lats[0].kind)) {
        // the per-half-sweep path of the block-shared generators has no
        // persistent launch shape to tune
        if (threads_out) *threads_out = 256;
        if (ctas_per_sm_out) *ctas_per_sm_out = 0;
        return RNG_OK;
    }
    if (probe_sweeps == 0) probe_sweeps = 64;
    static const uint32_t kThreads[] = {256, 512, 1024};
    static const int kPerSm[] = {1, 2, 4};
    static const uint32_t kMinSites[] = {1024, 8192, 65536};
    float best = -1.0f;
    uint32_t best_t = 0, best_m = 0, best_d = 0;
    int best_c = 0;
    cudaEvent_t e0, e1;
    RNGX_CHECK_CUDA(cudaEventCreate(&e0));
    RNGX_CHECK_CUDA(cudaEventCreate(&e1));
    uint64_t total_sites = 0;
    for (auto &t : h->lats) total_sites += static_cast<uint64_t>(t.L) * t.L;
    for (uint32_t ms : kMinSites) {
        if (ms > 1024 && ms / 8 > total_sites) continue;  // same plan as a smaller minimum
        for (uint32_t th : kThreads) {
          for (int pc : kPerSm) {
            // a single lattice in blocks of 1024 threads: both halo depths
            for (uint32_t hd = (th == 1024 && !h->batch) ? 1 : 0; hd <= ((th == 1024 && !h->batch) ? 2u : 0u); hd++) {
                // probe a clone: the launch shape never changes results, and
                // the handle itself must not advance
                ising_t c = nullptr;
                int st;
                if (h->batch) {
                    std::vector<uint32_t> L;
                    std::vector<double> beta;
                    std::vector<int> kind;
                    for (auto &t : h->lats) {
                        L.push_back(t.L);
                        beta.push_back(t.beta);
                        kind.push_back(t.kind);
                    }
                    st = ising_batch_create(&c, static_cast<uint32_t>(L.size()), L.data(), beta.data(), kind.data(),
                                            h->master_seed, h->lats[0].G, h->stream);
                } else {
                    const IsingLat &t = h->lats[0];
                    st = ising_create(&c, t.L, t.beta, t.layout, t.kind, t.flags, t.seed, t.G, h->stream);
                }
                if (st != RNG_OK) continue;
                c->cfg_threads = th;
                c->cfg_ctas_per_sm = pc;
                c->cfg_min_sites = ms;
                c->cfg_halo_depth = hd;
                st = ising_sweep(c, std::max<uint32_t>(1, probe_sweeps / 4), 0, h->stream);
                float msec = 0.0f;
                if (st == RNG_OK) {
                    cudaEventRecord(e0, h->stream);
                    st = ising_sweep(c, probe_sweeps, 0, h->stream);
                    cudaEventRecord(e1, h->stream);
                    if (st == RNG_OK && cudaEventSynchronize(e1) == cudaSuccess) cudaEventElapsedTime(&msec, e0, e1);
                    if (st == RNG_OK) st = check_err(c);
                }
                cudaGetLastError();
                ising_destroy(c);
                if (st == RNG_OK && msec > 0.0f && (best < 0.0f || msec < best)) {
                    best = msec;
                    best_t = th;
                    best_c = pc;
                    best_m = ms;
                    best_d = hd;
                }
            }
          }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best < 0.0f) {
        set_error("ising_autotune: no launch shape ran");
        return RNG_EUNSUPPORTED;
    }
    RNGX_CHECK(ising_set_launch(h, best_t, best_c, best_m));
    RNGX_CHECK(ising_set_halo_depth(h, best_d));
    if (threads_out) *threads_out = best_t;
    if (ctas_per_sm_out) *ctas_per_sm_out = best_c;
    return RNG_OK;
}
extern "C" int ising_info(ising_t h, uint32_t idx, uint32_t *n_lattices, uint32_t *L, int *layout, int *rng_kind,
                          uint64_t *sweeps_position)
{
    RNGX_CHECK(valid(h));
    if (idx >= h->lats.size()) {
        set_error("Ising: lattice index %u out of range", idx);
        return RNG_EINVAL;
    }
    const IsingLat &t = h->lats[idx];
    if (n_lattices) *n_lattices = static_cast<uint32_t>(h->lats.size());
    if (L) *L = t.L;
    if (layout) *layout = t.layout;
    if (rng_kind) *rng_kind = t.kind;
    if (sweeps_position) *sweeps_position = t.rng->g.pos / (2 * t.G);
    return RNG_OK;
}

extern "C" int ising_debug_mute_strip(ising_t h, int32_t strip, uint64_t wait_budget_ns)
{
    RNGX_CHECK(valid(h));
    h->mute_seg = strip;
    h->wait_budget_ns = wait_budget_ns ? wait_budget_ns : kWaitBudgetNs;
    return RNG_OK;
}

extern "C" int ising_plan_info(ising_t h, uint32_t *groups, uint32_t *blocks, uint32_t *strips, uint32_t *threads)
{
    RNGX_CHECK(valid(h));
    RNGX_CHECK(ensure_plan(h));
    uint32_t b = 0, s = 0, t = 0;
    for (auto &P : h->plans) {
        b += P.nblocks;
        s += P.nsegs;
        t = std::max(t, P.threads);
    }
    if (groups) *groups = static_cast<uint32_t>(h->plans.size());
    if (blocks) *blocks = b;
    if (strips) *strips = s;
    if (threads) *threads = t;
    return RNG_OK;
}
