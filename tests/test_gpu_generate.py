"""Parity of the CUDA generation path (through the C ABI) with the CPU
oracle: bit-exact for integer draws and uniform floats, within 2e-6 for
Box-Muller normals."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

SEED = 0x0123456789ABCDEF
THREAD_KINDS = [O.LCG32, O.LCG64, O.MWC, O.XORWOW, O.PHILOX4X32_10, O.XS1024W, O.PHILOX4X32_7]
SHARED_KINDS = [O.MT19937_SHARED, O.LFIB521, O.LFIB1279]  # one state shared by a group of threads
ALL_KINDS = THREAD_KINDS + SHARED_KINDS
NORMAL_TOL = 2e-6  # absolute, for float32 Box-Muller against the double oracle


@pytest.fixture(scope="module")
def R():
    import paper_1204_6193_gb300 as R
    return R


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


def run_gpu(R, torch, kind, n, Ks, *, flags=0, out="u32", layout=0, seed=SEED, skip=0, shard=None):
    """Creates, seeds, optionally skips, then generates len(Ks) calls; returns list of numpy arrays."""
    if shard is None:
        h = R.rng_create(kind, n, flags)
        n_local = n
    else:
        first, count = shard
        h = R.rng_create_shard(kind, n, first, count, flags)
        n_local = count
    try:
        R.rng_seed(h, seed)
        if skip:
            R.rng_skipahead(h, skip)
        res = []
        for K in Ks:
            size = n_local if layout == R.RNG_XOR_REDUCE else n_local * K
            dt = torch.int32 if out == "u32" else torch.float32
            buf = torch.empty(size, dtype=dt, device="cuda")
            fn = {"u32": R.rng_generate_u32, "f32": R.rng_generate_f32, "normal": R.rng_generate_normal}[out]
            fn(h, buf.data_ptr(), K, layout)
            torch.cuda.synchronize()
            a = buf.cpu().numpy()
            a = a.view(np.uint32) if out == "u32" else a
            if layout == R.RNG_STEP_MAJOR:
                a = a.reshape(K, n_local).T
            elif layout == R.RNG_INSTANCE_MAJOR:
                a = a.reshape(n_local, K)
            res.append(a)
        return res
    finally:
        R.rng_destroy(h)


def as_f32_oracle(r):
    return O.to_f32(r).astype(np.float32)


# ---------------------------------------------------------------- config 1
@pytest.mark.parametrize("kind", THREAD_KINDS)
def test_plain_generation_16384x256_bit_exact(R, torch_cuda, kind):
    n, K = 16384, 256
    g = run_gpu(R, torch_cuda, kind, n, [K])[0]
    o = O.generate(kind, SEED, n, K)
    assert np.array_equal(g, o)


def test_mt_64_generators_x_65536_bit_exact(R, torch_cuda):
    n, K = 64, 65536
    g = run_gpu(R, torch_cuda, O.MT19937_SHARED, n, [K], layout=1)[0]
    o = O.generate(O.MT19937_SHARED, SEED, n, K)
    assert np.array_equal(g, o)


@pytest.mark.parametrize("kind", [O.LFIB521, O.LFIB1279])
def test_lfib_64_generators_x_65536_bit_exact(R, torch_cuda, kind):
    # warp-shared rings (Sec. 4): many steps of s words, and the state
    # carried across calls of odd length
    n = 64
    o = O.generate(kind, SEED, n, 65536 + 777)
    g = run_gpu(R, torch_cuda, kind, n, [65536, 777], layout=1)
    assert np.array_equal(np.concatenate(g, axis=1), o)


@pytest.mark.parametrize("kind", SHARED_KINDS)
@pytest.mark.parametrize("layout", [0, 1, 2])
def test_block_shared_mixed_forms_and_positions(R, torch_cuda, kind, layout):
    # one handle, calls of every form in turn: positions that are multiples
    # of 32 (the chunked lagged Fibonacci form, entered on and off its
    # 256-word groups) and positions that are not (its step form); MT19937
    # blocks entered part-way, normal pairs split across two refills
    torch = torch_cuda
    n = 5
    calls = [("u32", 32), ("normal", 4160), ("f32", 96), ("normal", 1250), ("u32", 37), ("normal", 626),
             ("u32", 27), ("normal", 2048), ("f32", 1311), ("normal", 8)]
    o = O.generate(kind, SEED, n, sum(K for _, K in calls))
    h = R.rng_create(kind, n)
    try:
        R.rng_seed(h, SEED)
        start = 0
        for form, K in calls:
            ref = o[:, start:start + K]
            start += K
            dt = torch.int32 if form == "u32" else torch.float32
            buf = torch.empty(n if layout == 2 else n * K, dtype=dt, device="cuda")
            fn = {"u32": R.rng_generate_u32, "f32": R.rng_generate_f32, "normal": R.rng_generate_normal}[form]
            fn(h, buf.data_ptr(), K, layout)
            torch.cuda.synchronize()
            a = buf.cpu().numpy()
            if layout == 2:
                if form == "u32":
                    assert np.array_equal(a.view(np.uint32), np.bitwise_xor.reduce(ref, axis=1)), (form, K)
                elif form == "f32":
                    assert np.array_equal(a.view(np.uint32),
                                          np.bitwise_xor.reduce(as_f32_oracle(ref).view(np.uint32), axis=1)), (form, K)
                else:
                    z = O.box_muller(ref)
                    u = 2.0**-24
                    tol = K * NORMAL_TOL + (K - 1) * u / (1 - (K - 1) * u) * np.abs(z).sum(axis=1) * 2
                    assert np.all(np.abs(a.astype(np.float64) - z.sum(axis=1)) <= tol), (form, K)
                continue
            a = a.reshape(K, n).T if layout == 0 else a.reshape(n, K)
            if form == "u32":
                assert np.array_equal(a.view(np.uint32), ref), (form, K)
            elif form == "f32":
                assert np.array_equal(a, as_f32_oracle(ref)), (form, K)
            else:
                assert np.abs(a.astype(np.float64) - O.box_muller(ref)).max() <= NORMAL_TOL, (form, K)
        assert R.rng_info(h)["position"] == start
    finally:
        R.rng_destroy(h)


# ------------------------------------------------------ layouts and forms
def ragged_n(kind):
    if kind == O.XS1024W:
        return 96
    if kind in SHARED_KINDS:
        return 5  # a partial block of warp-shared generators
    return 1000  # not a multiple of 32: partial last warp


@pytest.mark.parametrize("kind", ALL_KINDS)
@pytest.mark.parametrize("layout", [0, 1])
def test_u32_and_f32_layouts_ragged(R, torch_cuda, kind, layout):
    n = ragged_n(kind)
    K = 1501 if kind in SHARED_KINDS else 77
    o = O.generate(kind, SEED, n, K)
    g = run_gpu(R, torch_cuda, kind, n, [K], layout=layout)[0]
    assert np.array_equal(g, o)
    f = run_gpu(R, torch_cuda, kind, n, [K], layout=layout, out="f32")[0]
    assert np.array_equal(f, as_f32_oracle(o))
    assert f.min() >= 0.0 and f.max() < 1.0


@pytest.mark.parametrize("kind", ALL_KINDS)
@pytest.mark.parametrize("layout", [0, 1])
def test_normals_within_2e6(R, torch_cuda, kind, layout):
    n = ragged_n(kind)
    K = 1250 if kind in SHARED_KINDS else 78
    o = O.box_muller(O.generate(kind, SEED, n, K))
    g = run_gpu(R, torch_cuda, kind, n, [K], layout=layout, out="normal")[0]
    err = np.abs(g.astype(np.float64) - o).max()
    assert err <= NORMAL_TOL, err


def test_box_muller_exhaustive_over_each_word(R, torch_cuda):
    # every u1 (all 2^24 values of r0 >> 8) at the angles where cos = 1 and
    # sin = 1, and every u2 at the largest radius (u1 = 2^-24), against the
    # oracle's double-precision transform
    torch = torch_cuda
    m = np.arange(1 << 24, dtype=np.uint32) << np.uint32(8)
    cases = []
    for r1 in (0, (1 << 22) << 8):
        w = np.empty(2 * len(m), dtype=np.uint32)
        w[0::2], w[1::2] = m, r1
        cases.append(w)
    w = np.empty(2 * len(m), dtype=np.uint32)
    w[0::2], w[1::2] = 0, m
    cases.append(w)
    worst = 0.0
    for w in cases:
        din = torch.from_numpy(w.view(np.int32)).cuda()
        dout = torch.empty(len(w), dtype=torch.float32, device="cuda")
        R.rng_u32_to_normal(din.data_ptr(), dout.data_ptr(), len(w) // 2)
        torch.cuda.synchronize()
        err = np.abs(dout.cpu().numpy().astype(np.float64) - O.box_muller(w))
        worst = max(worst, float(err.max()))
    print(f"Box-Muller max abs error over the exhaustive sweeps: {worst:.3e}")
    assert worst <= NORMAL_TOL


def test_u32_to_normal_ragged_and_errors(R, torch_cuda):
    torch = torch_cuda
    w = np.random.default_rng(3).integers(0, 2**32, 2 * 1001, dtype=np.uint32)
    din = torch.from_numpy(w.view(np.int32)).cuda()
    dout = torch.full((len(w) + 4,), 7.0, dtype=torch.float32, device="cuda")
    R.rng_u32_to_normal(din.data_ptr(), dout.data_ptr(), 1001)  # an odd number of pairs
    got = dout.cpu().numpy()
    assert np.abs(got[:len(w)] - O.box_muller(w)).max() <= NORMAL_TOL
    assert np.all(got[len(w):] == 7.0)  # nothing past the last pair
    with pytest.raises(R.RngError):
        R.rng_u32_to_normal(din.data_ptr() + 4, dout.data_ptr(), 4)  # not 16-byte aligned


@pytest.mark.parametrize("kind", ALL_KINDS)
def test_consume_in_register_modes(R, torch_cuda, kind):
    n = ragged_n(kind)
    K = 1250 if kind in SHARED_KINDS else 78
    o = O.generate(kind, SEED, n, K)
    g = run_gpu(R, torch_cuda, kind, n, [K], layout=R.RNG_XOR_REDUCE)[0]
    assert np.array_equal(g, np.bitwise_xor.reduce(o, axis=1))
    gf = run_gpu(R, torch_cuda, kind, n, [K], layout=R.RNG_XOR_REDUCE, out="f32")[0].view(np.uint32)
    assert np.array_equal(gf, np.bitwise_xor.reduce(as_f32_oracle(o).view(np.uint32), axis=1))
    z = O.box_muller(o)
    gz = run_gpu(R, torch_cuda, kind, n, [K], layout=R.RNG_XOR_REDUCE, out="normal")[0].astype(np.float64)
    # per-term error <= 2e-6, plus float32 summation error gamma_(K-1) sum |z|
    u = 2.0**-24
    tol = K * NORMAL_TOL + (K - 1) * u / (1 - (K - 1) * u) * np.abs(z).sum(axis=1) * 2
    assert np.all(np.abs(gz - z.sum(axis=1)) <= tol)


@pytest.mark.parametrize("kind", [O.PHILOX4X32_10, O.PHILOX4X32_7])
@pytest.mark.parametrize("layout", [0, 2])
@pytest.mark.parametrize("out", ["u32", "f32", "normal"])
def test_philox_block_aligned_and_misaligned(R, torch_cuda, kind, layout, out):
    n = 300
    o = O.generate(kind, SEED, n, 2 + 96 + 96)
    for Ks in ([96, 96], [2, 96, 96]):  # block-aligned calls, then misaligned ones
        g = run_gpu(R, torch_cuda, kind, n, Ks, layout=layout, out=out)
        start = 0
        for K, a in zip(Ks, g):
            ref = o[:, start:start + K]
            start += K
            if layout == R.RNG_XOR_REDUCE:
                if out == "u32":
                    assert np.array_equal(a, np.bitwise_xor.reduce(ref, axis=1))
                elif out == "f32":
                    assert np.array_equal(a.view(np.uint32),
                                          np.bitwise_xor.reduce(as_f32_oracle(ref).view(np.uint32), axis=1))
                else:
                    z = O.box_muller(ref)
                    assert np.all(np.abs(a - z.sum(axis=1)) <= K * NORMAL_TOL + 1e-4 * np.abs(z).sum(axis=1))
            elif out == "u32":
                assert np.array_equal(a, ref)
            elif out == "f32":
                assert np.array_equal(a, as_f32_oracle(ref))
            else:
                assert np.abs(a - O.box_muller(ref)).max() <= NORMAL_TOL


def test_xs1024w_unaligned_output_pointer(R, torch_cuda):
    torch = torch_cuda
    n, K = 64, 10
    h = R.rng_create(R.RNG_XS1024W, n)
    try:
        R.rng_seed(h, SEED)
        buf = torch.empty(n * K + 1, dtype=torch.int32, device="cuda")
        R.rng_generate_u32(h, buf.data_ptr() + 4, K, R.RNG_STEP_MAJOR)  # 4-byte aligned only
        torch.cuda.synchronize()
        g = buf[1:].cpu().numpy().view(np.uint32).reshape(K, n).T
        assert np.array_equal(g, O.generate(O.XS1024W, SEED, n, K))
    finally:
        R.rng_destroy(h)


# ------------------------------------------------- positions and seeding
@pytest.mark.parametrize("kind", ALL_KINDS)
def test_consecutive_calls_continue_the_streams(R, torch_cuda, kind):
    n = ragged_n(kind)
    Ks = [37, 91, 2] if kind not in SHARED_KINDS else [37, 1300, 611]
    o = O.generate(kind, SEED, n, sum(Ks))
    g = run_gpu(R, torch_cuda, kind, n, Ks)
    assert np.array_equal(np.concatenate(g, axis=1), o)


@pytest.mark.parametrize("kind", [O.LCG32, O.LCG64, O.MWC, O.XORWOW, O.PHILOX4X32_10, O.XS1024W, O.PHILOX4X32_7])
@pytest.mark.parametrize("t", [1, 1003, 2**33 + 7])
def test_skipahead(R, torch_cuda, kind, t):
    n = 256 if kind != O.MWC else 64
    g = run_gpu(R, torch_cuda, kind, n, [9], skip=t)[0]
    o = O.generate(kind, SEED, n, 9, skip=t, jump=True)
    assert np.array_equal(g, o)


@pytest.mark.parametrize("kind", SHARED_KINDS)
def test_skipahead_unsupported_for_block_shared_kinds(R, torch_cuda, kind):
    h = R.rng_create(kind, 2)
    try:
        R.rng_seed(h, 1)
        with pytest.raises(R.RngError) as e:
            R.rng_skipahead(h, 5)
        assert e.value.status == R.RNG_EUNSUPPORTED
    finally:
        R.rng_destroy(h)


@pytest.mark.parametrize("kind", [O.LCG32, O.LCG64])
def test_leapfrog_is_the_serial_sequence(R, torch_cuda, kind):
    n, K = 1024, 64
    g = run_gpu(R, torch_cuda, kind, n, [K], flags=O.SEED_LEAPFROG)[0]
    o = O.generate(kind, SEED, n, K, flags=O.SEED_LEAPFROG)
    assert np.array_equal(g, o)
    serial = O.generate(kind, SEED, 1, n * K, flags=O.SEED_LEAPFROG)[0]
    assert np.array_equal(g.T.ravel(), serial)


def test_xs1024w_substream_seeding(R, torch_cuda):
    n, K = 32 * 10, 40
    g = run_gpu(R, torch_cuda, O.XS1024W, n, [K], flags=O.SEED_SUBSTREAM)[0]
    o = O.generate(O.XS1024W, SEED, n, K, flags=O.SEED_SUBSTREAM)
    assert np.array_equal(g, o)


@pytest.mark.parametrize("kind", [O.PHILOX4X32_10, O.PHILOX4X32_7])
def test_philox_intrinsic_keys(R, torch_cuda, kind):
    # Sec. 7: key = (instance number, run word); shards and launch splits
    # name the same streams
    n, K = 5000, 45
    o = O.generate(kind, SEED, n, K, flags=O.PHILOX_INTRINSIC_KEY)
    g = run_gpu(R, torch_cuda, kind, n, [K], flags=O.PHILOX_INTRINSIC_KEY)[0]
    assert np.array_equal(g, o)
    b = run_gpu(R, torch_cuda, kind, n, [K], flags=O.PHILOX_INTRINSIC_KEY, shard=(1234, 3000))[0]
    assert np.array_equal(b, o[1234:4234])
    for out in ("f32", "normal"):
        g = run_gpu(R, torch_cuda, kind, n, [44], flags=O.PHILOX_INTRINSIC_KEY, out=out)[0]
        ref = as_f32_oracle(o[:, :44]) if out == "f32" else O.box_muller(o[:, :44])
        assert np.abs(g - ref).max() <= (0 if out == "f32" else NORMAL_TOL)
    with pytest.raises(R.RngError) as e:
        R.rng_create(R.RNG_XORWOW, 64, R.RNG_PHILOX_INTRINSIC_KEY)
    assert e.value.status == R.RNG_EUNSUPPORTED
    with pytest.raises(R.RngError) as e:
        R.rng_create_shard(kind, (1 << 32) + 64, 0, 64, R.RNG_PHILOX_INTRINSIC_KEY)
    assert e.value.status == R.RNG_EINVAL


def test_mwc_same_a(R, torch_cuda):
    g = run_gpu(R, torch_cuda, O.MWC, 500, [33], flags=O.MWC_SAME_A)[0]
    assert np.array_equal(g, O.generate(O.MWC, SEED, 500, 33, flags=O.MWC_SAME_A))


def test_mwc_multiplier_table_matches_oracle(R, torch_cuda):
    n = 20000
    assert np.array_equal(R.rng_mwc_multipliers(0, n), O.mwc_multipliers(n))
    assert int(R.rng_mwc_multipliers(0, 1)[0]) == 4294967118


@pytest.mark.parametrize("kind", ALL_KINDS)
def test_shards_reproduce_the_whole(R, torch_cuda, kind):
    n = 256 if kind not in SHARED_KINDS else 6
    K = 21
    flags = O.SEED_LEAPFROG if kind == O.LCG32 else (O.SEED_SUBSTREAM if kind == O.XS1024W else 0)
    whole = run_gpu(R, torch_cuda, kind, n, [K], flags=flags)[0]
    cut = n // 2 if kind != O.XS1024W else 128
    a = run_gpu(R, torch_cuda, kind, n, [K], flags=flags, shard=(0, cut))[0]
    b = run_gpu(R, torch_cuda, kind, n, [K], flags=flags, shard=(cut, n - cut))[0]
    assert np.array_equal(np.concatenate([a, b]), whole)
    assert np.array_equal(whole, O.generate(kind, SEED, n, K, flags=flags))


@pytest.mark.parametrize("kind", ALL_KINDS)
def test_checkpoint_restore(R, torch_cuda, kind):
    torch = torch_cuda
    n = ragged_n(kind)
    h = R.rng_create(kind, n)
    try:
        R.rng_seed(h, SEED)
        buf = torch.empty(n * 50, dtype=torch.int32, device="cuda")
        R.rng_generate_u32(h, buf.data_ptr(), 50, 1)
        blob = R.rng_get_state(h)
        R.rng_generate_u32(h, buf.data_ptr(), 50, 1)
        a = buf.cpu().numpy().view(np.uint32).reshape(n, 50).copy()
        R.rng_set_state(h, blob)
        R.rng_generate_u32(h, buf.data_ptr(), 50, 1)
        b = buf.cpu().numpy().view(np.uint32).reshape(n, 50)
        assert np.array_equal(a, b)
        assert np.array_equal(a, O.generate(kind, SEED, n, 50, skip=50))
        assert R.rng_info(h)["position"] == 100
    finally:
        R.rng_destroy(h)


def test_argument_errors(R, torch_cuda):
    with pytest.raises(R.RngError) as e:
        R.rng_create(R.RNG_XS1024W, 33)
    assert e.value.status == R.RNG_EINVAL
    with pytest.raises(R.RngError) as e:
        R.rng_create(R.RNG_XORWOW, 64, R.RNG_SEED_LEAPFROG)
    assert e.value.status == R.RNG_EUNSUPPORTED
    with pytest.raises(R.RngError):
        R.rng_create(99, 64)
    with pytest.raises(R.RngError):
        R.rng_create(R.RNG_LCG32, 0)
    h = R.rng_create(R.RNG_LCG32, 64)
    try:
        with pytest.raises(R.RngError):
            R.rng_generate_u32(h, 0, 4)  # unseeded
        R.rng_seed(h, 1)
        with pytest.raises(R.RngError):
            R.rng_generate_normal(h, 1 << 20, 3)  # odd count of normals
        with pytest.raises(R.RngError):
            R.rng_generate_u32(h, 0, 4)  # null output
    finally:
        R.rng_destroy(h)


# ------------------------------------------------ full size (config 2)
@pytest.mark.parametrize("kind", ALL_KINDS)
def test_full_size_sampled(R, torch_cuda, kind):
    """2^30 outputs per call in the bench's launch configuration and order
    (u32, f32, normal, then u32 consumed in registers as an XOR, one handle),
    checked on sampled instances, every draw of each: bit-exact for u32, f32
    and the XOR, within 2e-6 for the normals."""
    torch = torch_cuda
    if kind in SHARED_KINDS:
        n, K, layout = 1 << 15, 1 << 15, 1  # one generator per warp, 2^20 threads
    else:
        n, K, layout = 1 << 20, 1024, 0
    h = R.rng_create(kind, n, 0)
    try:
        R.rng_seed(h, SEED)
        buf = torch.empty(n * K, dtype=torch.int32, device="cuda")
        red = torch.empty(n, dtype=torch.int32, device="cuda")
        rng = np.random.default_rng(kind)
        if kind == O.XS1024W:
            samp = sorted({0, 31, 32, n - 1, *rng.integers(0, n, 6).tolist()})
        elif kind in SHARED_KINDS:
            samp = sorted({0, 1, n - 1, *rng.integers(0, n, 5).tolist()})
        else:
            samp = sorted({0, 1, n - 1, *rng.integers(0, n, 24).tolist()})
        want = {i: O.generate(kind, SEED, n, 4 * K, i_lo=i, i_hi=i + 1)[0] for i in samp}

        def column(i):
            v = buf.view(K, n)[:, i] if layout == 0 else buf.view(n, K)[i]
            return v.cpu().numpy()

        R.rng_generate_u32(h, buf.data_ptr(), K, layout)
        torch.cuda.synchronize()
        for i in samp:
            assert np.array_equal(column(i).view(np.uint32), want[i][:K]), ("u32", i)
        R.rng_generate_f32(h, buf.data_ptr(), K, layout)
        torch.cuda.synchronize()
        for i in samp:
            assert np.array_equal(column(i).view(np.float32), as_f32_oracle(want[i][K:2 * K])), ("f32", i)
        R.rng_generate_normal(h, buf.data_ptr(), K, layout)
        torch.cuda.synchronize()
        for i in samp:
            z = O.box_muller(want[i][2 * K:3 * K])
            dev = np.abs(column(i).view(np.float32).astype(np.float64) - z).max()
            assert dev <= NORMAL_TOL, ("normal", i, dev)
        R.rng_generate_u32(h, red.data_ptr(), K, R.RNG_XOR_REDUCE)
        torch.cuda.synchronize()
        got = red.cpu().numpy().view(np.uint32)
        for i in samp:
            assert got[i] == np.bitwise_xor.reduce(want[i][3 * K:]), ("xor", i)
        del buf
    finally:
        R.rng_destroy(h)


@pytest.mark.parametrize("kind", [O.XS1024W, O.MWC])
def test_full_size_sampled_u32_substream_and_same_a(R, torch_cuda, kind):
    """u32 at the bench's size with the other seeding modes: sub-streams for
    the 1024-bit generator, one shared multiplier for MWC."""
    torch = torch_cuda
    n, K = 1 << 20, 1024
    flags = O.SEED_SUBSTREAM if kind == O.XS1024W else O.MWC_SAME_A
    h = R.rng_create(kind, n, flags)
    try:
        R.rng_seed(h, SEED)
        buf = torch.empty(n * K, dtype=torch.int32, device="cuda")
        R.rng_generate_u32(h, buf.data_ptr(), K, 0)
        torch.cuda.synchronize()
        rng = np.random.default_rng(7 + kind)
        for i in sorted({0, 31, 32, n - 1, *rng.integers(0, n, 6).tolist()}):
            g = buf.view(K, n)[:, i].cpu().numpy().view(np.uint32)
            assert np.array_equal(g, O.generate(kind, SEED, n, K, flags=flags, i_lo=i, i_hi=i + 1)[0]), i
        del buf
    finally:
        R.rng_destroy(h)


@pytest.mark.parametrize("kind", THREAD_KINDS)
def test_full_size_normals_sampled(R, torch_cuda, kind):
    """Normals with the bench's 2^20 instances (the 1024-bit generator then
    takes its one-thread-per-state form), on sampled instances."""
    torch = torch_cuda
    n, K = 1 << 20, 16
    flags = O.SEED_SUBSTREAM if kind == O.XS1024W else 0
    h = R.rng_create(kind, n, flags)
    try:
        R.rng_seed(h, SEED)
        R.rng_generate_u32(h, torch.empty(n * 2, dtype=torch.int32, device="cuda").data_ptr(), 2, 0)
        buf = torch.empty(n * K, dtype=torch.float32, device="cuda")
        R.rng_generate_normal(h, buf.data_ptr(), K, R.RNG_STEP_MAJOR)
        red = torch.empty(n, dtype=torch.float32, device="cuda")
        R.rng_generate_normal(h, red.data_ptr(), K, R.RNG_XOR_REDUCE)
        torch.cuda.synchronize()
        view = buf.view(K, n)
        rng = np.random.default_rng(100 + kind)
        for i in sorted({0, 31, 32, n - 1, *rng.integers(0, n, 12).tolist()}):
            o = O.generate(kind, SEED, n, 2 + 2 * K, flags=flags, i_lo=i, i_hi=i + 1)[0]
            assert np.abs(view[:, i].cpu().numpy().astype(np.float64) - O.box_muller(o[2:2 + K])).max() <= NORMAL_TOL, i
            z = O.box_muller(o[2 + K:])
            assert abs(float(red[i]) - z.sum()) <= K * NORMAL_TOL + 1e-5 * np.abs(z).sum(), i
    finally:
        R.rng_destroy(h)


def test_xs1024w_thread_form_normals_ragged_whole(R, torch_cuda):
    """Every normal of the 1024-bit generator in its one-thread-per-state
    forms (step-major: two warps per 32 states), with the fewest states that
    select them plus a ragged 5 (the last block has 5 of 32 states), then u32
    draws that continue the streams."""
    torch = torch_cuda
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    nstates = 200 * sms + 37
    n, K = 32 * nstates, 6
    assert nstates % 32 == 5
    h = R.rng_create(O.XS1024W, n, 0)
    try:
        R.rng_seed(h, SEED)
        buf = torch.empty(n * K, dtype=torch.float32, device="cuda")
        R.rng_generate_normal(h, buf.data_ptr(), K, R.RNG_STEP_MAJOR)
        red = torch.empty(n, dtype=torch.float32, device="cuda")
        R.rng_generate_normal(h, red.data_ptr(), 2, R.RNG_XOR_REDUCE)
        tail = torch.empty(n * 3, dtype=torch.int32, device="cuda")
        R.rng_generate_u32(h, tail.data_ptr(), 3, R.RNG_STEP_MAJOR)
        torch.cuda.synchronize()
        o = O.generate(O.XS1024W, SEED, n, K + 5)
        got = buf.view(K, n).T.cpu().numpy().astype(np.float64)
        assert np.abs(got - O.box_muller(o[:, :K])).max() <= NORMAL_TOL
        z = O.box_muller(o[:, K:K + 2])
        err = np.abs(red.cpu().numpy().astype(np.float64) - z.sum(1))
        assert (err <= 2 * NORMAL_TOL + 1e-5 * np.abs(z).sum(1)).all()
        assert np.array_equal(tail.view(3, n).T.cpu().numpy().view(np.uint32), o[:, K + 2:])
    finally:
        R.rng_destroy(h)


def test_mwc_full_table_matches_oracle(R, torch_cuda):
    n = 1 << 20
    assert np.array_equal(R.rng_mwc_multipliers(0, n), O.mwc_multipliers(n))


# ---------------------------------------------------- empty and tiny inputs
@pytest.mark.parametrize("kind", ALL_KINDS)
def test_zero_draws_and_single_instance(R, torch_cuda, kind):
    # K = 0 is a no-op that leaves the position alone; one instance (one
    # warp-shared state for XS1024W: 32 lanes) is the smallest handle
    torch = torch_cuda
    n = 32 if kind == O.XS1024W else 1
    h = R.rng_create(kind, n)
    try:
        R.rng_seed(h, SEED)
        sentinel = torch.full((n * 8,), -7, dtype=torch.int32, device="cuda")
        for fn in (R.rng_generate_u32, R.rng_generate_f32, R.rng_generate_normal):
            fn(h, sentinel.data_ptr(), 0, R.RNG_INSTANCE_MAJOR)
        if kind not in SHARED_KINDS:
            R.rng_skipahead(h, 0)
        torch.cuda.synchronize()
        assert torch.all(sentinel == -7) and R.rng_info(h)["position"] == 0
        R.rng_generate_u32(h, sentinel.data_ptr(), 8, R.RNG_INSTANCE_MAJOR)
        torch.cuda.synchronize()
        got = sentinel.cpu().numpy().view(np.uint32).reshape(n, 8)
        assert np.array_equal(got, O.generate(kind, SEED, n, 8))
    finally:
        R.rng_destroy(h)


def test_zero_sweeps_and_smallest_lattice(R, torch_cuda):
    # 0 sweeps change nothing; L = 4 (two streams per colour row pair) is
    # the smallest lattice, a whole lattice in one strip
    h = R.ising_create(4, 0.4, 0, O.XORWOW, 0, SEED, 2)
    try:
        init = R.ising_get_spins(h)
        R.ising_sweep(h, 0)
        R.ising_sweep_plain(h, 0)
        assert np.array_equal(R.ising_get_spins(h), init)
        assert np.array_equal(init, O.ising_init_spins(4, SEED))
        R.ising_sweep(h, 25, 5)
        ref, acc, nm = O.ising_run(4, 0.4, O.XORWOW, SEED, 25, measure_every=5)
        obs = R.ising_observables(h)
        assert np.array_equal(R.ising_get_spins(h), ref)
        assert obs["acc"] == acc.tolist() and obs["n_meas"] == nm
    finally:
        R.ising_destroy(h)


# ------------------------------------------ long streams of few instances
SPLIT_KINDS = [O.LCG32, O.LCG64, O.MWC, O.PHILOX4X32_10, O.PHILOX4X32_7]


@pytest.mark.parametrize("kind", SPLIT_KINDS)
@pytest.mark.parametrize("out", ["u32", "f32", "normal"])
def test_split_form_for_long_streams_of_few_instances(R, torch_cuda, kind, out):
    """Few instances and many draws: each instance's draws are cut into
    ranges that threads make from jumped copies of its state.  Ragged range
    lengths, a Philox position off a counter block (an odd first call),
    and a second call that continues the streams."""
    torch = torch_cuda
    n, Ks = 1000, (6, 4098, 2050)  # the first call leaves Philox mid-block
    got = run_gpu(R, torch, kind, n, Ks)  # u32 draws, whatever the form under test below
    ref = O.generate(kind, SEED, n, sum(Ks))
    pos = 0
    for K, g in zip(Ks, got):
        want = ref[:, pos:pos + K]
        assert np.array_equal(g, want), (K, pos)
        pos += K
    if out == "u32":
        return
    # the f32 and normal forms of the split kernel, after an even first call
    Ks = (2, 6146)
    got = run_gpu(R, torch, kind, n, Ks, out=out)
    ref = O.generate(kind, SEED, n, sum(Ks))[:, 2:]
    if out == "f32":
        assert np.array_equal(got[1], as_f32_oracle(ref))
    else:
        assert np.abs(got[1].astype(np.float64) - O.box_muller(ref.reshape(-1)).reshape(n, -1)).max() <= NORMAL_TOL


@pytest.mark.parametrize("kind,flags", [(O.LCG32, O.SEED_LEAPFROG), (O.LCG64, O.SEED_LEAPFROG),
                                        (O.MWC, O.MWC_SAME_A), (O.PHILOX4X32_7, O.PHILOX_INTRINSIC_KEY)])
def test_split_form_other_seedings(R, torch_cuda, kind, flags):
    torch = torch_cuda
    n, K = 96, 8192
    got = run_gpu(R, torch, kind, n, (K,), flags=flags)[0]
    assert np.array_equal(got, O.generate(kind, SEED, n, K, flags=flags))
