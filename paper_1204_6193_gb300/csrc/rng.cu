// rng.cu -- the C ABI for generator handles: creation, seeding, skip-ahead,
// generation, checkpoint and errors.
#include <atomic>
#include <cstdarg>
#include <cstdlib>
#include <string>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>

#include "internal.h"

namespace rngx {

namespace {
thread_local char t_err[512] = "";
}

void set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(t_err, sizeof(t_err), fmt, ap);
    va_end(ap);
}

int cuda_fail(cudaError_t e, const char *what)
{
    set_error("%s: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? RNG_ENOMEM : RNG_ECUDA;
}

namespace {
// The installed allocator (none: cudaMallocAsync) and the number of
// library allocations it still has outstanding.
struct Allocator {
    rng_alloc_fn alloc = nullptr;
    rng_free_fn free = nullptr;
    void *ctx = nullptr;
};
std::mutex g_alloc_mu;
Allocator g_alloc;
std::atomic<int64_t> g_outstanding{0};

Allocator current_allocator()
{
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    return g_alloc;
}
}  // namespace

namespace {
std::mutex g_fault_mu;
std::string g_fault_seen;   // the RNG_FAULT value the countdown belongs to
long long g_fault_left = 0;  // "oom:N": allocations left before the failing one

std::string fault_env()
{
    const char *v = std::getenv("RNG_FAULT");
    return v ? std::string(v) : std::string();
}
}  // namespace

bool fault_oom()
{
    const std::string v = fault_env();
    if (v == "oom") return true;
    if (v.rfind("oom:", 0) != 0) return false;
    std::lock_guard<std::mutex> lk(g_fault_mu);
    if (v != g_fault_seen) {  // a new setting restarts the countdown
        g_fault_seen = v;
        g_fault_left = std::atoll(v.c_str() + 4);
    }
    return g_fault_left > 0 && --g_fault_left == 0;
}

bool fault_launch() { return fault_env() == "launch"; }
bool fault_timeout() { return fault_env() == "timeout"; }

int injected(const char *what, int status)
{
    set_error("%s failed (injected by RNG_FAULT=%s)", what, fault_env().c_str());
    return status;
}

int dalloc(void **p, size_t bytes, cudaStream_t s)
{
    *p = nullptr;
    if (bytes == 0) return RNG_OK;
    if (fault_oom()) return injected("device allocation", RNG_ENOMEM);
    const Allocator a = current_allocator();
    if (a.alloc) {
        if (a.alloc(p, bytes, s, a.ctx) != 0 || !*p) {
            *p = nullptr;
            set_error("the installed allocator failed to provide %zu bytes", bytes);
            return RNG_ENOMEM;
        }
    } else {
        cudaError_t e = cudaMallocAsync(p, bytes, s);
        if (e != cudaSuccess) {
            cudaGetLastError();
            *p = nullptr;
            return cuda_fail(e, "cudaMallocAsync");
        }
    }
    g_outstanding.fetch_add(1);
    return RNG_OK;
}

void dfree(void *p, cudaStream_t s)
{
    if (!p) return;
    const Allocator a = current_allocator();
    if (a.free) a.free(p, s, a.ctx);
    else cudaFreeAsync(p, s);
    g_outstanding.fetch_sub(1);
}

namespace {

// Bytes of state per instance and the number of arrays (SoA).
void state_layout(int kind, size_t &bytes_per, int &arrays, size_t &elem)
{
    switch (kind) {
    case RNG_LCG32: bytes_per = 4; arrays = 1; elem = 4; break;
    case RNG_LCG64: bytes_per = 8; arrays = 1; elem = 8; break;
    case RNG_MWC: bytes_per = 8; arrays = 1; elem = 8; break;
    case RNG_XORWOW: bytes_per = 24; arrays = 6; elem = 4; break;
    case RNG_PHILOX4X32_10:
    case RNG_PHILOX4X32_7: bytes_per = 8; arrays = 1; elem = 8; break;
    case RNG_XS1024W: bytes_per = 4; arrays = 1; elem = 4; break;
    case RNG_MT19937_SHARED: bytes_per = 4 * MT_N_WORDS; arrays = 1; elem = 4 * MT_N_WORDS; break;
    case RNG_LFIB521: bytes_per = 4 * 521; arrays = 1; elem = 4 * 521; break;
    case RNG_LFIB1279: bytes_per = 4 * 1279; arrays = 1; elem = 4 * 1279; break;
    default: bytes_per = 0; arrays = 0; elem = 0;
    }
}

int check_flags(int kind, uint32_t flags)
{
    if (flags & ~static_cast<uint32_t>(RNG_SEED_LEAPFROG | RNG_SEED_SUBSTREAM | RNG_MWC_SAME_A |
                                       RNG_PHILOX_INTRINSIC_KEY)) {
        set_error("unknown flag bits 0x%x", flags);
        return RNG_EINVAL;
    }
    if ((flags & RNG_SEED_LEAPFROG) && kind != RNG_LCG32 && kind != RNG_LCG64) {
        set_error("RNG_SEED_LEAPFROG is defined for the LCGs only");
        return RNG_EUNSUPPORTED;
    }
    if ((flags & RNG_SEED_SUBSTREAM) && kind != RNG_XS1024W) {
        set_error("RNG_SEED_SUBSTREAM is defined for RNG_XS1024W only");
        return RNG_EUNSUPPORTED;
    }
    if ((flags & RNG_MWC_SAME_A) && kind != RNG_MWC) {
        set_error("RNG_MWC_SAME_A is defined for RNG_MWC only");
        return RNG_EUNSUPPORTED;
    }
    if ((flags & RNG_PHILOX_INTRINSIC_KEY) && kind != RNG_PHILOX4X32_10 && kind != RNG_PHILOX4X32_7) {
        set_error("RNG_PHILOX_INTRINSIC_KEY is defined for the Philox kinds only");
        return RNG_EUNSUPPORTED;
    }
    return RNG_OK;
}

// LCG per-draw map: (a, c), or (a_n, c_n) for leapfrogging over n instances.
void lcg_map(int kind, uint32_t flags, uint64_t n_total, uint64_t &A, uint64_t &C)
{
    const bool is64 = kind == RNG_LCG64;
    uint64_t a = is64 ? 2862933555777941757ull : 1664525ull;
    uint64_t c = is64 ? 1442695040888963407ull : 1013904223ull;
    if (!(flags & RNG_SEED_LEAPFROG)) {
        A = a;
        C = c;
        return;
    }
    uint64_t ra = 1, rc = 0, t = n_total;
    while (t) {
        if (t & 1) {
            rc = a * rc + c;
            ra = a * ra;
        }
        c = a * c + c;
        a = a * a;
        t >>= 1;
    }
    const uint64_t mask = is64 ? ~0ull : 0xffffffffull;
    A = ra & mask;
    C = rc & mask;
}

struct StateHeader {
    uint32_t magic, version;
    int32_t kind;
    uint32_t flags;
    uint64_t n, first, n_total, pos, seed, state_bytes;
};
constexpr uint32_t kMagic = 0x52474233;  // "RGB3"

int valid(rng_t h)
{
    if (!h) {
        set_error("null rng handle");
        return RNG_EINVAL;
    }
    return RNG_OK;
}

int generate(rng_t h, void *d_out, uint64_t K, int out_kind, int layout, void *stream)
{
    RNGX_CHECK(valid(h));
    if (!h->seeded) {
        set_error("rng handle used before rng_seed");
        return RNG_EINVAL;
    }
    if (!d_out && K) {
        set_error("null output pointer");
        return RNG_EINVAL;
    }
    if (layout < RNG_STEP_MAJOR || layout > RNG_XOR_REDUCE) {
        set_error("unknown layout %d", layout);
        return RNG_EINVAL;
    }
    if (out_kind == OUT_NORMAL && (K & 1)) {
        set_error("normal deviates come in pairs: n_per_instance must be even");
        return RNG_EINVAL;
    }
    if (K && h->g.n > (~0ull) / K) {
        set_error("output size overflows");
        return RNG_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    RNGX_CHECK(launch_generate(h->g, d_out, K, out_kind, layout, s));
    h->g.pos += K;
    return RNG_OK;
}

}  // namespace
}  // namespace rngx

using namespace rngx;

extern "C" {

int rng_create_shard(rng_t *out, int kind, uint64_t n_total, uint64_t first, uint64_t count, uint32_t flags,
                     void *cuda_stream)
{
    if (!out) {
        set_error("null output handle pointer");
        return RNG_EINVAL;
    }
    *out = nullptr;
    if (kind < RNG_LCG32 || kind >= kNumKinds) {
        set_error("unknown generator kind %d", kind);
        return RNG_EINVAL;
    }
    if (count == 0 || n_total == 0 || first > n_total || count > n_total - first) {
        set_error("bad instance range [%llu, +%llu) of %llu", (unsigned long long)first, (unsigned long long)count,
                  (unsigned long long)n_total);
        return RNG_EINVAL;
    }
    RNGX_CHECK(check_flags(kind, flags));
    if (kind == RNG_XS1024W && (count % 32 || first % 32 || n_total % 32)) {
        set_error("RNG_XS1024W shares one 1024-bit state per 32 lanes: sizes must be multiples of 32");
        return RNG_EINVAL;
    }
    if (is_block_shared(kind) && count > 0x7fffffffull) {
        set_error("too many block-shared generators");
        return RNG_EINVAL;
    }
    if ((flags & RNG_PHILOX_INTRINSIC_KEY) && n_total > (1ull << 32)) {
        set_error("intrinsic Philox keys hold the instance index in 32 bits: at most 2^32 instances");
        return RNG_EINVAL;
    }
    if (count > (1ull << 34)) {
        set_error("too many instances");
        return RNG_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    rng_s *h = new (std::nothrow) rng_s();
    if (!h) {
        set_error("host allocation failed");
        return RNG_ENOMEM;
    }
    RNGX_CHECK_CUDA(cudaGetDevice(&h->device));
    h->stream = s;
    GenState &g = h->g;
    g.kind = kind;
    g.flags = flags;
    g.n = count;
    g.first = first;
    g.n_total = n_total;
    g.pos = 0;
    g.philox_rounds = kind == RNG_PHILOX4X32_7 ? 7 : 10;
    g.mwc_a = nullptr;
    g.mwc_a0 = 0;
    for (int i = 0; i < 6; i++) g.s[i] = nullptr;
    size_t per = 0, elem = 0;
    int arrays = 0;
    state_layout(kind, per, arrays, elem);
    h->state_bytes = per * count;
    int st = dalloc(&h->state, h->state_bytes, s);
    if (st != RNG_OK) {
        delete h;
        return st;
    }
    for (int k = 0; k < arrays; k++) g.s[k] = static_cast<char *>(h->state) + k * elem * count;
    if (kind == RNG_LCG32 || kind == RNG_LCG64) lcg_map(kind, flags, n_total, g.A, g.C);
    if (kind == RNG_MWC) {
        const uint32_t *tab = nullptr;
        st = mwc_table((flags & RNG_MWC_SAME_A) ? 1 : first + count, &tab, s);
        if (st == RNG_OK) {
            if (flags & RNG_MWC_SAME_A) {
                cudaError_t e = cudaMemcpy(&g.mwc_a0, tab, 4, cudaMemcpyDeviceToHost);
                if (e != cudaSuccess) st = cuda_fail(e, "cudaMemcpy");
            } else {
                g.mwc_a = tab + first;
            }
        }
        if (st != RNG_OK) {
            dfree(h->state, s);
            delete h;
            return st;
        }
    }
    *out = h;
    return RNG_OK;
}

int rng_create(rng_t *out, int kind, uint64_t n_instances, uint32_t flags, void *cuda_stream)
{
    return rng_create_shard(out, kind, n_instances, 0, n_instances, flags, cuda_stream);
}

int rng_destroy(rng_t h)
{
    if (!h) return RNG_OK;
    dfree(h->state, h->stream);
    cudaError_t e = cudaStreamSynchronize(h->stream);
    delete h;
    if (e != cudaSuccess) return cuda_fail(e, "rng_destroy");
    return RNG_OK;
}

int rng_seed(rng_t h, uint64_t seed)
{
    RNGX_CHECK(valid(h));
    RNGX_CHECK(launch_seed(h->g, seed, h->stream));
    h->g.pos = 0;
    h->seeded = true;
    h->seed = seed;
    return RNG_OK;
}

int rng_skipahead(rng_t h, uint64_t n)
{
    RNGX_CHECK(valid(h));
    if (!h->seeded) {
        set_error("rng handle used before rng_seed");
        return RNG_EINVAL;
    }
    return launch_skipahead(h->g, n, h->stream);
}

int rng_generate_u32(rng_t h, uint32_t *d_out, uint64_t n_per_instance, int layout, void *cuda_stream)
{
    return generate(h, d_out, n_per_instance, OUT_U32, layout, cuda_stream);
}

int rng_generate_f32(rng_t h, float *d_out, uint64_t n_per_instance, int layout, void *cuda_stream)
{
    return generate(h, d_out, n_per_instance, OUT_F32, layout, cuda_stream);
}

int rng_generate_normal(rng_t h, float *d_out, uint64_t n_per_instance, int layout, void *cuda_stream)
{
    return generate(h, d_out, n_per_instance, OUT_NORMAL, layout, cuda_stream);
}

int rng_u32_to_normal(const uint32_t *d_in, float *d_out, uint64_t n_pairs, void *cuda_stream)
{
    if (n_pairs == 0) return RNG_OK;
    if (!d_in || !d_out || (reinterpret_cast<uintptr_t>(d_in) & 15) || (reinterpret_cast<uintptr_t>(d_out) & 15)) {
        set_error("rng_u32_to_normal: input and output must be non-null and 16-byte aligned");
        return RNG_EINVAL;
    }
    return launch_u32_to_normal(d_in, d_out, n_pairs, static_cast<cudaStream_t>(cuda_stream));
}

int rng_get_state(rng_t h, void *host_buf, size_t *bytes)
{
    RNGX_CHECK(valid(h));
    if (!bytes) {
        set_error("null size pointer");
        return RNG_EINVAL;
    }
    const size_t need = sizeof(StateHeader) + h->state_bytes;
    if (!host_buf) {
        *bytes = need;
        return RNG_OK;
    }
    if (*bytes < need) {
        set_error("state buffer too small: %zu < %zu", *bytes, need);
        *bytes = need;
        return RNG_EINVAL;
    }
    StateHeader hd;
    hd.magic = kMagic;
    hd.version = 1;
    hd.kind = h->g.kind;
    hd.flags = h->g.flags;
    hd.n = h->g.n;
    hd.first = h->g.first;
    hd.n_total = h->g.n_total;
    hd.pos = h->g.pos;
    hd.seed = h->seed;
    hd.state_bytes = h->state_bytes;
    memcpy(host_buf, &hd, sizeof(hd));
    RNGX_CHECK_CUDA(cudaStreamSynchronize(h->stream));
    RNGX_CHECK_CUDA(cudaMemcpy(static_cast<char *>(host_buf) + sizeof(hd), h->state, h->state_bytes,
                               cudaMemcpyDeviceToHost));
    *bytes = need;
    return RNG_OK;
}

int rng_set_state(rng_t h, const void *host_buf, size_t bytes)
{
    RNGX_CHECK(valid(h));
    if (!host_buf || bytes < sizeof(StateHeader)) {
        set_error("state blob missing or truncated");
        return RNG_EINVAL;
    }
    StateHeader hd;
    memcpy(&hd, host_buf, sizeof(hd));
    if (hd.magic != kMagic || hd.version != 1 || hd.kind != h->g.kind || hd.flags != h->g.flags ||
        hd.n != h->g.n || hd.first != h->g.first || hd.n_total != h->g.n_total || hd.state_bytes != h->state_bytes ||
        bytes != sizeof(hd) + h->state_bytes) {
        set_error("state blob does not match this handle");
        return RNG_EINVAL;
    }
    RNGX_CHECK_CUDA(cudaStreamSynchronize(h->stream));
    RNGX_CHECK_CUDA(cudaMemcpy(h->state, static_cast<const char *>(host_buf) + sizeof(hd), h->state_bytes,
                               cudaMemcpyHostToDevice));
    h->g.pos = hd.pos;
    h->seed = hd.seed;
    h->seeded = true;
    return RNG_OK;
}

int rng_info(rng_t h, int *kind, uint64_t *n_instances, uint64_t *first, uint64_t *position)
{
    RNGX_CHECK(valid(h));
    if (kind) *kind = h->g.kind;
    if (n_instances) *n_instances = h->g.n;
    if (first) *first = h->g.first;
    if (position) *position = h->g.pos;
    return RNG_OK;
}

int rng_set_allocator(rng_alloc_fn alloc, rng_free_fn free_fn, void *ctx)
{
    if ((alloc == nullptr) != (free_fn == nullptr)) {
        set_error("rng_set_allocator: give both hooks or neither");
        return RNG_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    if (g_outstanding.load() != 0) {
        set_error("rng_set_allocator: %lld allocations of the current allocator are still live",
                  static_cast<long long>(g_outstanding.load()));
        return RNG_EBUSY;
    }
    g_alloc.alloc = alloc;
    g_alloc.free = free_fn;
    g_alloc.ctx = ctx;
    return RNG_OK;
}

const char *rng_strerror(int status)
{
    switch (status) {
    case RNG_OK: return "ok";
    case RNG_EINVAL: return "invalid argument";
    case RNG_ENOMEM: return "out of memory";
    case RNG_EUNSUPPORTED: return "operation not supported for this generator";
    case RNG_ECUDA: return "CUDA error";
    case RNG_ETIMEOUT: return "device-side wait timed out";
    case RNG_EBUSY: return "busy";
    default: return "unknown status";
    }
}

const char *rng_last_error(void) { return t_err; }

}  // extern "C"

// See include/rng_gb300.h.
extern "C" int rng_debug_bounds_status(int *site, int reset)
{
    using namespace rngx;
    if (!site) {
        set_error("rng_debug_bounds_status: null output");
        return RNG_EINVAL;
    }
    *site = 0;
#ifdef RNG_BOUNDS_CHECK
    int (*readers[])(int *, bool) = {bounds_site_gen,
                                     bounds_site_lfib,
                                     bounds_site_persist_RNG_LCG32,
                                     bounds_site_persist_RNG_LCG64,
                                     bounds_site_persist_RNG_MWC,
                                     bounds_site_persist_RNG_XORWOW,
                                     bounds_site_persist_RNG_PHILOX4X32_10,
                                     bounds_site_persist_RNG_PHILOX4X32_7,
                                     bounds_site_persist_RNG_XS1024W};
    RNGX_CHECK_CUDA(cudaDeviceSynchronize());
    for (auto rd : readers) {
        int v = 0;
        RNGX_CHECK(rd(&v, reset != 0));
        if (v && !*site) *site = v;
    }
    return RNG_OK;
#else
    (void)reset;
    set_error("rng_debug_bounds_status: this library was built without RNG_BOUNDS_CHECK");
    return RNG_EUNSUPPORTED;
#endif
}
