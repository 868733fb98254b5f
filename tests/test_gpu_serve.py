"""The serving loop: every result in a mix of concurrent requests equals the
same request run alone (plain calls through the C ABI, and the CPU oracle),
admission respects the memory budget, and evicted stream sets come back
identical."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

N_SET = 1024


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1204_6193_gb300 as R
    return R, torch


def draw_req(R, kind, seed, offset, count, out):
    r = R.rng_request_t()
    r.type, r.kind, r.seed, r.offset, r.count, r.out = R.RNG_REQ_DRAW, kind, seed, offset, count, out
    return r


def sweep_req(R, kind, seed, L, beta, sweeps):
    r = R.rng_request_t()
    r.type, r.kind, r.seed, r.L, r.beta, r.sweeps = R.RNG_REQ_SWEEP, kind, seed, L, beta, sweeps
    return r


def alone_draw(R, torch, r):
    """The request by plain calls: create, seed, skip, generate step-major."""
    h = R.rng_create(r.kind, N_SET)
    try:
        R.rng_seed(h, r.seed)
        if r.offset:
            R.rng_skipahead(h, r.offset)
        K = -(-r.count // N_SET)
        if r.out == R.RNG_OUT_NORMAL:
            K += K % 2
        buf = torch.empty(N_SET * K, dtype=torch.int32, device="cuda")
        fn = {R.RNG_OUT_U32: R.rng_generate_u32, R.RNG_OUT_F32: R.rng_generate_f32,
              R.RNG_OUT_NORMAL: R.rng_generate_normal}[r.out]
        fn(h, buf.data_ptr(), K, R.RNG_STEP_MAJOR)
        torch.cuda.synchronize()
        return buf.cpu().numpy().view(np.uint32)[: r.count].copy()
    finally:
        R.rng_destroy(h)


def fetch(R, srv, ticket, nbytes):
    out = np.zeros(nbytes, dtype=np.uint8)
    R.rng_server_fetch(srv, ticket, out.ctypes.data, nbytes)
    return out


def test_mixed_requests_equal_alone(env):
    R, torch = env
    rng = np.random.default_rng(11)
    srv = R.rng_server_create(16, N_SET, 4, 1 << 30)
    try:
        reqs = []
        for i in range(48):
            kind = int(rng.integers(0, 6))
            out = int(rng.integers(0, 3))
            count = int(2 ** rng.uniform(10, 18)) // 2 * 2
            offset = int(rng.integers(0, 2**34)) if i % 3 else 0
            reqs.append(draw_req(R, kind, int(rng.integers(0, 6)), offset, count, out))
        for i, (L, sw) in enumerate([(64, 20), (128, 10), (64, 33), (256, 5)]):
            reqs.insert(7 * i + 3, sweep_req(R, [3, 5, 4, 0][i], 100 + i, L, 0.44, sw))
        tickets = [R.rng_server_submit(srv, r) for r in reqs]
        results = []
        for r, t in zip(reqs, tickets):
            res = R.rng_server_wait(srv, t, 60.0)
            assert res.status == 0 and res.done == 1
            assert res.t_done_ns >= res.t_start_ns >= res.t_submit_ns
            results.append((res, fetch(R, srv, t, res.bytes)))
        st = R.rng_server_stats(srv)
        assert st["completed"] == len(reqs) and st["mem_in_use"] == 0
        assert st["max_concurrent"] >= 2  # work of different requests overlapped
    finally:
        R.rng_server_destroy(srv)
    for r, (res, data) in zip(reqs, results):
        if r.type == R.RNG_REQ_SWEEP:
            spins = data.view(np.int8).reshape(r.L, r.L)
            ref, _, _ = O.ising_run(r.L, r.beta, r.kind, r.seed, r.sweeps)
            assert np.array_equal(spins, ref)
            assert (res.E, res.M) == O.ising_energy(ref)
        else:
            got = data.view(np.uint32)
            assert np.array_equal(got, alone_draw(R, torch, r))


def test_draw_result_definition_against_oracle(env):
    R, torch = env
    srv = R.rng_server_create(4, N_SET, 2, 1 << 28)
    try:
        for kind in [O.XORWOW, O.XS1024W, O.PHILOX4X32_10, O.MWC]:
            r = draw_req(R, kind, 77, 123457, 5000, R.RNG_OUT_U32)
            t = R.rng_server_submit(srv, r)
            res = R.rng_server_wait(srv, t, 60.0)
            got = fetch(R, srv, t, res.bytes).view(np.uint32)
            K = -(-5000 // N_SET)
            o = O.generate(kind, 77, N_SET, K, skip=123457, jump=True)  # [instance, draw]
            assert np.array_equal(got, o.T.ravel()[:5000])
    finally:
        R.rng_server_destroy(srv)


def test_admission_by_memory_and_eviction(env):
    R, torch = env
    # each request's output is 64 KiB; the budget admits two at a time
    srv = R.rng_server_create(2, N_SET, 8, 128 << 10)
    try:
        reqs = [draw_req(R, O.XORWOW, s % 5, 0, N_SET * 16, R.RNG_OUT_U32) for s in range(12)]
        tickets = [R.rng_server_submit(srv, r) for r in reqs]
        for r, t in zip(reqs, tickets):
            res = R.rng_server_wait(srv, t, 60.0)
            assert res.status == 0
            got = fetch(R, srv, t, res.bytes).view(np.uint32)
            assert np.array_equal(got, alone_draw(R, torch, r))
        assert R.rng_server_stats(srv)["max_concurrent"] <= 2
        with pytest.raises(R.RngError) as e:
            R.rng_server_submit(srv, draw_req(R, O.XORWOW, 1, 0, N_SET * 64, R.RNG_OUT_U32))
        assert e.value.status == R.RNG_ENOMEM
        with pytest.raises(R.RngError):
            R.rng_server_submit(srv, draw_req(R, O.MT19937_SHARED, 1, 0, 64, R.RNG_OUT_U32))
        with pytest.raises(R.RngError):
            R.rng_server_submit(srv, draw_req(R, O.XORWOW, 1, 0, 63, R.RNG_OUT_NORMAL))
    finally:
        R.rng_server_destroy(srv)


def test_reused_lattices_equal_fresh_ones(env):
    """Sweep requests of one shape in a row: after the first ones are
    fetched, their lattices are reset and reused (new seed, temperature,
    initial spins and streams); each result equals the oracle's, and so does
    a concurrent mix of such requests on the sweep slots."""
    R, torch = env
    srv = R.rng_server_create(4, N_SET, 2, 1 << 30)
    try:
        cases = [(O.XORWOW, 64, 0.30 + 0.02 * i, 500 + i, 7 + i) for i in range(6)] + \
                [(O.XS1024W, 128, 0.44, 900 + i, 5) for i in range(4)]
        # one at a time: every request after the first of its shape reuses a lattice
        for kind, L, beta, seed, sweeps in cases:
            t = R.rng_server_submit(srv, sweep_req(R, kind, seed, L, beta, sweeps))
            res = R.rng_server_wait(srv, t, 60.0)
            assert res.status == 0
            spins = fetch(R, srv, t, res.bytes).view(np.int8).reshape(L, L)
            ref, _, _ = O.ising_run(L, beta, kind, seed, sweeps)
            assert np.array_equal(spins, ref), (kind, L, seed)
            assert (res.E, res.M) == O.ising_energy(ref)
        # all at once: every sweep slot busy, pooled lattices in use
        tickets = [R.rng_server_submit(srv, sweep_req(R, k, s + 50, L, b, w)) for k, L, b, s, w in cases]
        for (kind, L, beta, seed, sweeps), t in zip(cases, tickets):
            res = R.rng_server_wait(srv, t, 60.0)
            spins = fetch(R, srv, t, res.bytes).view(np.int8).reshape(L, L)
            ref, _, _ = O.ising_run(L, beta, kind, seed + 50, sweeps)
            assert np.array_equal(spins, ref), (kind, L, seed)
    finally:
        R.rng_server_destroy(srv)
