// noalloc.cu -- skip-ahead of caller-owned xorshift states with no device
// allocation, for callers that cannot allocate device memory themselves or
// through the library: code running inside a framework that owns every
// device allocation (a memory-pool or arena allocator, or a sandbox that
// forbids cudaMalloc), and code that must not trigger an allocation's
// implicit synchronisation in the middle of a time-critical sequence.
//
// The matrix power that rng_skipahead computes in stream-ordered scratch
// (three n x n GF(2) matrices, n = 160 for XORWOW, 1024 for the 1024-bit
// generator) lives here in one file-scope device array sized for the
// largest generator, 1024 state bits: 3 x 1024 x 1024 bits = 384 KiB.  Every
// GPU that loads the library holds that array until the process exits.
#include <cstring>

#include "gen_device.cuh"

namespace {

constexpr int kMaxStateBits = 1024;
constexpr size_t kMatrixWords = static_cast<size_t>(kMaxStateBits) * (kMaxStateBits / 32);

static __device__ __align__(256) uint32_t g_skip_scratch[3 * kMatrixWords];

// Host code sees g_skip_scratch only as a stand-in symbol: its device
// address is looked up on every call, with the calling device current, so
// that no pointer outlives a cudaDeviceReset (which reloads the module and
// can move the array).  The lookup costs little; the first one on a device
// also loads the module there.
int scratch_address(uint32_t **out)
{
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_skip_scratch);
    if (e != cudaSuccess) return rngx::cuda_fail(e, "cudaGetSymbolAddress(g_skip_scratch)");
    *out = static_cast<uint32_t *>(p);
    return RNG_OK;
}

// One thread per instance in blocks of 256: the grid's x extent (at most
// 2^31 - 1 blocks) bounds the instance count.
constexpr uint64_t kMaxInstances = ((1ull << 31) - 1) * 256ull;

}  // namespace

// See include/rng_gb300.h.
extern "C" int rng_skipahead_noalloc(int kind, void *d_state, uint64_t n_instances, uint64_t n, void *cuda_stream)
{
    using namespace rngx;
    int state_bits = 0;
    switch (kind) {
    case RNG_XORWOW: state_bits = 160; break;
    case RNG_XS1024W: state_bits = 1024; break;
    case RNG_MT19937_SHARED: state_bits = 19937; break;
    case RNG_LFIB521: state_bits = 521 * 32; break;
    case RNG_LFIB1279: state_bits = 1279 * 32; break;
    case RNG_LCG32:
    case RNG_LCG64:
    case RNG_MWC:
    case RNG_PHILOX4X32_10:
    case RNG_PHILOX4X32_7:
        set_error("rng_skipahead_noalloc: kind %d skips without scratch; use rng_skipahead", kind);
        return RNG_EUNSUPPORTED;
    default: set_error("rng_skipahead_noalloc: unknown generator kind %d", kind); return RNG_EINVAL;
    }
    if (state_bits > kMaxStateBits) {
        set_error("rng_skipahead_noalloc: a %d-bit state needs a transition matrix larger than the %d-bit "
                  "maximum of the static scratch",
                  state_bits, kMaxStateBits);
        return RNG_EINVAL;
    }
    if (!d_state || n_instances == 0) {
        set_error("rng_skipahead_noalloc: null state or no instances");
        return RNG_EINVAL;
    }
    if (n_instances > kMaxInstances) {
        set_error("rng_skipahead_noalloc: %llu instances exceed the %llu that one launch covers",
                  static_cast<unsigned long long>(n_instances), static_cast<unsigned long long>(kMaxInstances));
        return RNG_EINVAL;
    }
    if (kind == RNG_XS1024W && n_instances % 32) {
        set_error("rng_skipahead_noalloc: the 1024-bit generator needs whole warps (n_instances %% 32 == 0)");
        return RNG_EINVAL;
    }
    if (n == 0) return RNG_OK;
    uint32_t *scratch = nullptr;
    RNGX_CHECK(scratch_address(&scratch));
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    uint32_t *m0 = scratch, *m1 = scratch + kMatrixWords, *m2 = scratch + 2 * kMatrixWords;
    // gf2_pow writes every word of the three matrices before reading it, so
    // whatever an earlier call left in the scratch does not matter
    RNGX_CHECK(gf2_pow(kind, n, m0, m1, m2, s));
    DevParams p;
    memset(&p, 0, sizeof(p));
    p.n = n_instances;
    const int arrays = kind == RNG_XORWOW ? 6 : 1;
    for (int k = 0; k < arrays; k++) p.s[k] = static_cast<uint32_t *>(d_state) + k * n_instances;
    return launch_matrix_apply(kind, p, m0, n, s);
}
