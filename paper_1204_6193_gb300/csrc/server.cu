// server.cu -- request serving with continuous batching.  A host worker
// thread owns every CUDA call of the server: it admits queued requests
// whenever a slot (a CUDA stream) and device memory are free, so that work
// of requests that arrive while others run overlaps on the device, and it
// retires requests when their completion events fire.  Generator states
// stay resident on the device as "stream sets" keyed by (kind, seed), so a
// draw request costs a state copy, a skip-ahead and one generation launch.
//
// A draw request (kind, seed, offset, count, out) returns the first `count`
// numbers, in step-major order, of the stream set (kind, seed) -- n_set
// instances seeded by rng_seed(seed) -- advanced by `offset` draws:
//   result[j] = s_(j mod n_set)[offset + j div n_set].
// A sweep request (kind, seed, L, beta, sweeps) returns the int8 spins of an
// L x L lattice created by ising_create(L, beta, ISING_INT8, kind, 0, seed,
// 2) after `sweeps` sweeps, plus its E and M.  Both are pure functions of
// the request, whatever else is in flight.
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <thread>
#include <unordered_map>
#include <vector>

#include "gen_device.cuh"

namespace rngx {
namespace {

uint64_t now_ns()
{
    return static_cast<uint64_t>(
        std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
            .count());
}

// ---------------------------------------------- skip-ahead by matrix ladder
// x <- x prod_{bit k of t} M^(2^k), with the 64 powers M^(2^k) precomputed
// once per server: one launch per skip instead of a chain of matrix products.
__device__ __forceinline__ uint32_t warp_mul1024(uint32_t x, const uint32_t *__restrict__ P)
{
    const int lane = threadIdx.x & 31;
    uint32_t acc = 0;
    for (int wi = 0; wi < 32; wi++) {
        uint32_t bits = __shfl_sync(0xffffffffu, x, wi);
        while (bits) {
            const int b = __ffs(bits) - 1;
            bits &= bits - 1;
            acc ^= __ldg(P + (static_cast<size_t>(wi) * 32 + b) * 32 + lane);
        }
    }
    return acc;
}

__global__ void k_ladder_xs(uint32_t *state, uint64_t n, const uint32_t *ladder, uint64_t t)
{
    const uint64_t i = static_cast<uint64_t>(blockIdx.x) * 256 + threadIdx.x;
    if ((i & ~31ull) >= n) return;
    uint32_t x = state[i];
    for (int k = 0; k < 64; k++)
        if ((t >> k) & 1) x = warp_mul1024(x, ladder + static_cast<size_t>(k) * 1024 * 32);
    state[i] = x;
}

__global__ void k_ladder_xorwow(uint32_t *state, uint64_t n, const uint32_t *ladder, uint64_t t)
{
    const uint64_t i = static_cast<uint64_t>(blockIdx.x) * 256 + threadIdx.x;
    if (i >= n) return;
    uint32_t v[5];
    for (int k = 0; k < 5; k++) v[k] = state[k * n + i];
    for (int k = 0; k < 64; k++) {
        if (!((t >> k) & 1)) continue;
        const uint32_t *M = ladder + static_cast<size_t>(k) * 160 * 5;
        uint32_t o[5] = {0, 0, 0, 0, 0};
        for (int wi = 0; wi < 5; wi++) {
            uint32_t bits = v[wi];
            while (bits) {
                const int b = __ffs(bits) - 1;
                bits &= bits - 1;
                for (int j = 0; j < 5; j++) o[j] ^= __ldg(M + (wi * 32 + b) * 5 + j);
            }
        }
        for (int j = 0; j < 5; j++) v[j] = o[j];
    }
    for (int k = 0; k < 5; k++) state[k * n + i] = v[k];
    state[5 * n + i] += static_cast<uint32_t>(t) * 362437u;
}

}  // namespace
}  // namespace rngx

using namespace rngx;

struct ServerReq {
    rng_request_t r;
    uint64_t ticket = 0;
    int state = 0;  // 0 queued, 1 running, 2 done
    int slot = -1;
    void *d_out = nullptr;
    uint64_t out_bytes = 0, charged = 0;  // device bytes counted against the budget
    ising_t ising = nullptr;
    rng_result_t res;
    cudaEvent_t ev = nullptr;
    struct SetEntry *set = nullptr;
};

struct SetEntry {
    int kind = 0;
    uint64_t seed = 0;
    rng_t base = nullptr;
    cudaEvent_t ready = nullptr;
    uint64_t last_use = 0;
    int in_use = 0;
};

// Sweep requests run on the last kSweepSlots slots.
constexpr uint32_t kSweepSlots = 4;

struct rng_server_s {
    uint32_t n_sets = 0, n_set_inst = 0, n_slots = 0;
    uint64_t budget = 0, in_use = 0;
    int device = 0;
    std::vector<cudaStream_t> slots;          // draw slots, then kSweepSlots sweep slots
    // lattices of finished sweep requests, by (slot, L, kind), reset and
    // reused instead of created again (a handle stays on the slot whose
    // stream it was created on)
    std::map<std::tuple<int, uint32_t, int>, std::vector<ising_t>> lattice_pool;
    std::vector<ServerReq *> slot_req;
    std::vector<std::vector<rng_t>> work;     // [slot][kind] working generator
    std::map<std::pair<int, uint64_t>, SetEntry *> sets;
    uint32_t *ladder_xs = nullptr, *ladder_xw = nullptr;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<ServerReq *> queue;
    std::unordered_map<uint64_t, ServerReq *> reqs;
    uint64_t next_ticket = 1, submitted = 0, completed = 0, tick = 0;
    uint32_t max_conc = 0;
    bool stop = false;
    int fatal = RNG_OK;
    std::thread worker;
};

namespace {

constexpr size_t kQueueMax = 1 << 16;

int build_ladders(rng_server_s *S, cudaStream_t s)
{
    const size_t xs_words = 1024 * 32, xw_words = 160 * 5;
    RNGX_CHECK_CUDA(cudaMalloc(&S->ladder_xs, 64 * xs_words * 4));
    RNGX_CHECK_CUDA(cudaMalloc(&S->ladder_xw, 64 * xw_words * 4));
    RNGX_CHECK(gf2_one_step(RNG_XS1024W, S->ladder_xs, s));
    RNGX_CHECK(gf2_one_step(RNG_XORWOW, S->ladder_xw, s));
    for (int k = 1; k < 64; k++) {
        RNGX_CHECK(gf2_mul(1024, S->ladder_xs + (k - 1) * xs_words, S->ladder_xs + (k - 1) * xs_words,
                           S->ladder_xs + k * xs_words, s));
        RNGX_CHECK(gf2_mul(160, S->ladder_xw + (k - 1) * xw_words, S->ladder_xw + (k - 1) * xw_words,
                           S->ladder_xw + k * xw_words, s));
    }
    RNGX_CHECK_CUDA(cudaStreamSynchronize(s));
    return RNG_OK;
}

// Stream set (kind, seed): created and seeded on the slot that first needs
// it; other slots wait for its ready event.  Least recently used sets that
// no running request holds are evicted beyond n_sets.
int get_set(rng_server_s *S, int kind, uint64_t seed, cudaStream_t s, SetEntry **out)
{
    auto key = std::make_pair(kind, seed);
    auto it = S->sets.find(key);
    if (it == S->sets.end()) {
        while (S->sets.size() >= S->n_sets) {
            SetEntry *victim = nullptr;
            for (auto &kv : S->sets)
                if (kv.second->in_use == 0 && (!victim || kv.second->last_use < victim->last_use)) victim = kv.second;
            if (!victim) break;
            cudaEventSynchronize(victim->ready);
            rng_destroy(victim->base);
            cudaEventDestroy(victim->ready);
            S->sets.erase(std::make_pair(victim->kind, victim->seed));
            delete victim;
        }
        SetEntry *e = new (std::nothrow) SetEntry();
        if (!e) return RNG_ENOMEM;
        e->kind = kind;
        e->seed = seed;
        int st = rng_create(&e->base, kind, S->n_set_inst, 0, s);
        if (st == RNG_OK) st = rng_seed(e->base, seed);
        if (st == RNG_OK && cudaEventCreateWithFlags(&e->ready, cudaEventDisableTiming) != cudaSuccess) st = RNG_ECUDA;
        if (st == RNG_OK && cudaEventRecord(e->ready, s) != cudaSuccess) st = RNG_ECUDA;
        if (st != RNG_OK) {
            if (e->base) rng_destroy(e->base);
            delete e;
            return st;
        }
        it = S->sets.emplace(key, e).first;
    }
    *out = it->second;
    return RNG_OK;
}

// Enqueues the GPU work of a draw request on its slot.
int launch_draw(rng_server_s *S, ServerReq *q)
{
    const int slot = q->slot;
    cudaStream_t s = S->slots[slot];
    const rng_request_t &r = q->r;
    SetEntry *set = nullptr;
    RNGX_CHECK(get_set(S, r.kind, r.seed, s, &set));
    set->in_use++;
    set->last_use = ++S->tick;
    q->set = set;
    rng_t &w = S->work[slot][r.kind];
    if (!w) RNGX_CHECK(rng_create(&w, r.kind, S->n_set_inst, 0, s));
    RNGX_CHECK_CUDA(cudaStreamWaitEvent(s, set->ready, 0));
    RNGX_CHECK_CUDA(cudaMemcpyAsync(w->state, set->base->state, w->state_bytes, cudaMemcpyDeviceToDevice, s));
    w->seeded = true;
    w->g.pos = 0;
    if (r.offset) {
        if (r.kind == RNG_XS1024W || r.kind == RNG_XORWOW) {
            const unsigned nb = static_cast<unsigned>((w->g.n + 255) / 256);
            if (r.kind == RNG_XS1024W)
                k_ladder_xs<<<nb, 256, 0, s>>>(static_cast<uint32_t *>(w->state), w->g.n, S->ladder_xs, r.offset);
            else k_ladder_xorwow<<<nb, 256, 0, s>>>(static_cast<uint32_t *>(w->state), w->g.n, S->ladder_xw, r.offset);
            RNGX_CHECK_LAUNCH();
            w->g.pos = r.offset;
        } else {
            RNGX_CHECK(launch_skipahead(w->g, r.offset, s));
        }
    }
    const uint64_t n = S->n_set_inst;
    uint64_t K = (r.count + n - 1) / n;
    if (r.out == RNG_OUT_NORMAL) K = (K + 1) / 2 * 2;
    RNGX_CHECK(launch_generate(w->g, q->d_out, K, r.out, RNG_STEP_MAJOR, s));
    return RNG_OK;
}

int launch_sweep(rng_server_s *S, ServerReq *q)
{
    cudaStream_t s = S->slots[q->slot];
    const rng_request_t &r = q->r;
    auto &pool = S->lattice_pool[std::make_tuple(q->slot, r.L, r.kind)];
    if (!pool.empty()) {
        q->ising = pool.back();
        pool.pop_back();
        RNGX_CHECK(ising_reset_lattice(q->ising, r.beta, r.seed));
    } else {
        RNGX_CHECK(ising_create(&q->ising, r.L, r.beta, ISING_INT8, r.kind, 0, r.seed, 2, s));
    }
    return ising_sweep(q->ising, r.sweeps, 0, s);
}

uint64_t out_bytes(const rng_server_s *S, const rng_request_t &r)
{
    if (r.type == RNG_REQ_SWEEP) return 0;  // the lattice handle owns its memory
    const uint64_t n = S->n_set_inst;
    uint64_t K = (r.count + n - 1) / n;
    if (r.out == RNG_OUT_NORMAL) K = (K + 1) / 2 * 2;
    return K * n * 4;
}

uint64_t req_mem(const rng_server_s *S, const rng_request_t &r)
{
    if (r.type == RNG_REQ_SWEEP) return 3ull * r.L * r.L + (1 << 20);  // spins, streams, plan
    return out_bytes(S, r);
}

void finish(rng_server_s *S, ServerReq *q, int status)
{
    q->res.status = status;
    q->res.done = 1;
    q->res.t_done_ns = now_ns();
    q->state = 2;
    if (q->set) q->set->in_use--;
    S->completed++;
}

void worker_main(rng_server_s *S)
{
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    while (true) {
        bool progress = false;
        // retire finished slots
        for (size_t i = 0; i < S->slots.size(); i++) {
            ServerReq *q = S->slot_req[i];
            if (!q) continue;
            const cudaError_t e = cudaEventQuery(q->ev);
            if (e == cudaErrorNotReady) continue;
            int st = e == cudaSuccess ? RNG_OK : cuda_fail(e, "server request");
            if (st == RNG_OK && q->r.type == RNG_REQ_SWEEP) {
                int64_t E = 0, M = 0;
                st = ising_observables(q->ising, &E, &M, nullptr, nullptr);
                q->res.E = E;
                q->res.M = M;
            }
            finish(S, q, st);
            S->slot_req[i] = nullptr;
            progress = true;
        }
        if (progress) S->cv_done.notify_all();
        // admit while a slot and memory are free, in arrival order within
        // each request type: a request that waits for a slot of its type (or
        // for memory) holds back the later requests of its type only, so a
        // sweep waiting for a sweep slot does not keep draws from idle draw
        // slots, nor the other way round
        for (int type = 0; type < 2; type++) {
            const bool sweep = type == 1;
            const size_t first_sweep = S->slots.size() - kSweepSlots;
            while (true) {
                auto it = S->queue.begin();
                while (it != S->queue.end() && ((*it)->r.type == RNG_REQ_SWEEP) != sweep) ++it;
                if (it == S->queue.end()) break;
                ServerReq *q = *it;
                int slot = -1;
                for (size_t i = sweep ? first_sweep : 0; i < (sweep ? S->slots.size() : first_sweep); i++)
                    if (!S->slot_req[i]) {
                        slot = static_cast<int>(i);
                        break;
                    }
                const uint64_t need = req_mem(S, q->r);
                if (slot < 0 || S->in_use + need > S->budget) break;
                S->queue.erase(it);
                q->slot = slot;
                q->state = 1;
                q->res.t_start_ns = now_ns();
                int st = RNG_OK;
                q->out_bytes = out_bytes(S, q->r);
                if (q->out_bytes) st = dalloc(&q->d_out, q->out_bytes, S->slots[slot]);
                if (st == RNG_OK) {
                    S->in_use += need;
                    q->charged = need;
                    st = sweep ? launch_sweep(S, q) : launch_draw(S, q);
                }
                if (st == RNG_OK && cudaEventRecord(q->ev, S->slots[slot]) != cudaSuccess) st = RNG_ECUDA;
                if (st != RNG_OK) {
                    finish(S, q, st);
                    S->cv_done.notify_all();
                    continue;
                }
                S->slot_req[slot] = q;
                uint32_t busy = 0;
                for (auto *x : S->slot_req) busy += x != nullptr;
                if (busy > S->max_conc) S->max_conc = busy;
                progress = true;
            }
        }
        bool any_running = false;
        for (auto *x : S->slot_req) any_running |= x != nullptr;
        if (S->stop && S->queue.empty() && !any_running) break;
        if (!progress) {
            if (any_running) {
                lk.unlock();
                std::this_thread::yield();
                lk.lock();
            } else {
                S->cv_work.wait_for(lk, std::chrono::milliseconds(5));
            }
        }
    }
}

int find_req(rng_server_s *S, uint64_t ticket, ServerReq **q)
{
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) {
        set_error("unknown or already fetched ticket %llu", static_cast<unsigned long long>(ticket));
        return RNG_EINVAL;
    }
    *q = it->second;
    return RNG_OK;
}

void release(rng_server_s *S, ServerReq *q)
{
    cudaStream_t s = q->slot >= 0 ? S->slots[q->slot] : nullptr;
    if (q->d_out) dfree(q->d_out, s);
    if (q->ising) {
        // a finished lattice goes back to its slot's pool (a few per size)
        auto &pool = S->lattice_pool[std::make_tuple(q->slot, q->r.L, q->r.kind)];
        if (q->res.status == RNG_OK && pool.size() < 2) pool.push_back(q->ising);
        else ising_destroy(q->ising);
    }
    S->in_use -= q->charged;
    if (q->ev) cudaEventDestroy(q->ev);
    S->reqs.erase(q->ticket);
    delete q;
}

}  // namespace

extern "C" {

int rng_server_create(rng_server_t *out, uint32_t n_sets, uint32_t instances_per_set, uint32_t n_slots,
                      uint64_t mem_budget_bytes)
{
    if (!out || n_sets == 0 || instances_per_set == 0 || instances_per_set % 32 || n_slots == 0 || n_slots > 64 ||
        mem_budget_bytes == 0) {
        set_error("rng_server_create: need n_sets > 0, instances_per_set a positive multiple of 32, "
                  "1 <= n_slots <= 64, a memory budget");
        return RNG_EINVAL;
    }
    *out = nullptr;
    rng_server_s *S = new (std::nothrow) rng_server_s();
    if (!S) return RNG_ENOMEM;
    S->n_sets = n_sets;
    S->n_set_inst = instances_per_set;
    S->n_slots = n_slots;
    S->budget = mem_budget_bytes;
    int st = cudaGetDevice(&S->device) == cudaSuccess ? RNG_OK : RNG_ECUDA;
    S->slots.resize(n_slots + kSweepSlots, nullptr);
    S->slot_req.resize(n_slots + kSweepSlots, nullptr);
    S->work.assign(n_slots + kSweepSlots, std::vector<rng_t>(kNumKinds, nullptr));
    for (auto &s : S->slots)
        if (st == RNG_OK && cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) st = RNG_ECUDA;
    if (st == RNG_OK) st = build_ladders(S, S->slots[0]);
    if (st != RNG_OK) {
        rng_server_destroy(S);
        return st;
    }
    S->worker = std::thread(worker_main, S);
    *out = S;
    return RNG_OK;
}

int rng_server_submit(rng_server_t S, const rng_request_t *req, uint64_t *ticket)
{
    if (!S || !req || !ticket) {
        set_error("rng_server_submit: null argument");
        return RNG_EINVAL;
    }
    const rng_request_t &r = *req;
    if (r.type == RNG_REQ_DRAW) {
        if (r.kind < RNG_LCG32 || r.kind >= kNumKinds || is_block_shared(r.kind) || r.count == 0 ||
            r.out < RNG_OUT_U32 ||
            r.out > RNG_OUT_NORMAL || (r.out == RNG_OUT_NORMAL && (r.count & 1))) {
            set_error("rng_server_submit: bad draw request (kind, count, output form)");
            return RNG_EINVAL;
        }
    } else if (r.type == RNG_REQ_SWEEP) {
        if (r.L < 4 || r.L % 2 || r.L > 16384 || r.kind < RNG_LCG32 || r.kind >= kNumKinds ||
            is_block_shared(r.kind)) {
            set_error("rng_server_submit: bad sweep request");
            return RNG_EINVAL;
        }
    } else {
        set_error("rng_server_submit: unknown request type %d", r.type);
        return RNG_EINVAL;
    }
    ServerReq *q = new (std::nothrow) ServerReq();
    if (!q) return RNG_ENOMEM;
    q->r = r;
    memset(&q->res, 0, sizeof(q->res));
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (req_mem(S, r) > S->budget) {
            delete q;
            set_error("rng_server_submit: request needs more device memory than the whole budget");
            return RNG_ENOMEM;
        }
        if (S->queue.size() >= kQueueMax) {
            delete q;
            set_error("rng_server_submit: queue full");
            return RNG_EBUSY;
        }
        if (cudaEventCreateWithFlags(&q->ev, cudaEventDisableTiming) != cudaSuccess) {
            delete q;
            set_error("rng_server_submit: cudaEventCreate failed");
            return RNG_ECUDA;
        }
        q->ticket = S->next_ticket++;
        q->res.t_submit_ns = now_ns();
        q->res.bytes = r.type == RNG_REQ_SWEEP ? static_cast<uint64_t>(r.L) * r.L : r.count * 4;
        S->reqs[q->ticket] = q;
        S->queue.push_back(q);
        S->submitted++;
        *ticket = q->ticket;
    }
    S->cv_work.notify_one();
    return RNG_OK;
}

int rng_server_wait(rng_server_t S, uint64_t ticket, double timeout_s, rng_result_t *res)
{
    if (!S) {
        set_error("null server");
        return RNG_EINVAL;
    }
    std::unique_lock<std::mutex> lk(S->mu);
    ServerReq *q = nullptr;
    RNGX_CHECK(find_req(S, ticket, &q));
    const auto until = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
    while (q->state != 2) {
        if (timeout_s >= 0 && std::chrono::steady_clock::now() >= until) {
            set_error("rng_server_wait: timed out");
            return RNG_ETIMEOUT;
        }
        S->cv_done.wait_for(lk, std::chrono::milliseconds(1));
    }
    if (res) *res = q->res;
    return q->res.status;
}

int rng_server_fetch(rng_server_t S, uint64_t ticket, void *host_dst, uint64_t bytes)
{
    if (!S) {
        set_error("null server");
        return RNG_EINVAL;
    }
    std::unique_lock<std::mutex> lk(S->mu);
    ServerReq *q = nullptr;
    RNGX_CHECK(find_req(S, ticket, &q));
    if (q->state != 2) {
        set_error("rng_server_fetch: request not finished (wait first)");
        return RNG_EBUSY;
    }
    int st = q->res.status;
    if (st == RNG_OK && host_dst) {
        if (bytes < q->res.bytes) {
            set_error("rng_server_fetch: destination holds %llu bytes, result has %llu",
                      static_cast<unsigned long long>(bytes), static_cast<unsigned long long>(q->res.bytes));
            return RNG_EINVAL;
        }
        if (q->r.type == RNG_REQ_SWEEP) {
            st = ising_get_spins(q->ising, static_cast<int8_t *>(host_dst));
        } else {
            // the completion event has fired: the output is final
            cudaError_t e = cudaMemcpy(host_dst, q->d_out, q->res.bytes, cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) st = cuda_fail(e, "rng_server_fetch");
        }
    }
    release(S, q);
    lk.unlock();
    S->cv_work.notify_one();
    return st;
}

int rng_server_stats(rng_server_t S, uint64_t *submitted, uint64_t *completed, uint64_t *mem_in_use,
                     uint32_t *max_concurrent)
{
    if (!S) {
        set_error("null server");
        return RNG_EINVAL;
    }
    std::lock_guard<std::mutex> lk(S->mu);
    if (submitted) *submitted = S->submitted;
    if (completed) *completed = S->completed;
    if (mem_in_use) *mem_in_use = S->in_use;
    if (max_concurrent) *max_concurrent = S->max_conc;
    return RNG_OK;
}

int rng_server_destroy(rng_server_t S)
{
    if (!S) return RNG_OK;
    if (S->worker.joinable()) {
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->stop = true;
        }
        S->cv_work.notify_all();
        S->worker.join();
    }
    std::vector<ServerReq *> left;
    for (auto &kv : S->reqs) left.push_back(kv.second);
    for (auto *q : left) release(S, q);
    for (auto &kv : S->sets) {
        if (kv.second->ready) cudaEventSynchronize(kv.second->ready);
        rng_destroy(kv.second->base);
        if (kv.second->ready) cudaEventDestroy(kv.second->ready);
        delete kv.second;
    }
    for (auto &row : S->work)
        for (auto w : row)
            if (w) rng_destroy(w);
    for (auto &kv : S->lattice_pool)
        for (auto h : kv.second) ising_destroy(h);
    for (auto s : S->slots)
        if (s) {
            cudaStreamSynchronize(s);
            cudaStreamDestroy(s);
        }
    cudaFree(S->ladder_xs);
    cudaFree(S->ladder_xw);
    delete S;
    return RNG_OK;
}

}  // extern "C"
