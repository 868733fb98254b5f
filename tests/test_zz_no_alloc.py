"""rng_skipahead_noalloc: the skip-ahead for callers that cannot allocate
device memory (a framework that owns every device allocation, or a sequence
that must not synchronise on an allocation).  It advances a state array the
caller owns, keeping its matrix scratch in a static device array, and must
give exactly what rng_skipahead gives on a library handle -- on two calls in
a row, with every way the library could allocate made to fail, and with the
device's free memory unchanged.  Collected last on purpose: a failure here
comes after every other test has run."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SEED = 0x0123456789ABCDEF
STEPS = (12345, 2**40 + 77)  # two calls in a row


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1204_6193_gb300 as R
    return R, torch


def state_words(R, h, n_words):
    blob = R.rng_get_state(h)
    return np.frombuffer(blob[len(blob) - 4 * n_words:], dtype=np.uint32).copy()


@pytest.mark.parametrize("kind,n,arrays", [(3, 1000, 6), (5, 4096, 1)])
def test_noalloc_matches_rng_skipahead_twice(env, kind, n, arrays, monkeypatch):
    R, torch = env
    # the expected states, from a library handle and its allocating skip-ahead
    h = R.rng_create(kind, n)
    try:
        R.rng_seed(h, SEED)
        start = state_words(R, h, arrays * n)
        expected = []
        for t in STEPS:
            R.rng_skipahead(h, t)
            expected.append(state_words(R, h, arrays * n))
    finally:
        R.rng_destroy(h)
    mine = torch.from_numpy(start.view(np.int32)).cuda()
    # a first call loads the module (and its static array) on this device
    warm = mine.clone()
    R.rng_skipahead_noalloc(kind, warm.data_ptr(), n, 1)
    torch.cuda.synchronize()

    # every allocation route of the library fails from here on: the
    # injected out-of-memory fault and an allocator that counts and refuses
    calls = []

    def refuse(nbytes, stream):
        calls.append(nbytes)
        return 0

    monkeypatch.setenv("RNG_FAULT", "oom")
    R.rng_set_allocator(refuse, lambda ptr, stream: None)
    try:
        free_before, _ = torch.cuda.mem_get_info()
        for t, want in zip(STEPS, expected):
            R.rng_skipahead_noalloc(kind, mine.data_ptr(), n, t)
            torch.cuda.synchronize()
            got = mine.cpu().numpy().view(np.uint32)
            assert np.array_equal(got, want), t
        free_after, _ = torch.cuda.mem_get_info()
    finally:
        R.rng_set_allocator()
    assert calls == [], "the no-allocation entry point asked the allocator for memory"
    assert free_after == free_before, "device memory was allocated during the calls"


def test_noalloc_rejects_what_it_cannot_do(env):
    R, torch = env
    buf = torch.zeros(6 * 64, dtype=torch.int32, device="cuda")
    with pytest.raises(R.RngError) as e:
        R.rng_skipahead_noalloc(R.RNG_MT19937_SHARED, buf.data_ptr(), 1, 5)
    assert e.value.status == R.RNG_EINVAL and "maximum" in str(e.value)
    with pytest.raises(R.RngError) as e:
        R.rng_skipahead_noalloc(R.RNG_LCG32, buf.data_ptr(), 64, 5)
    assert e.value.status == R.RNG_EUNSUPPORTED
    with pytest.raises(R.RngError) as e:
        R.rng_skipahead_noalloc(R.RNG_XS1024W, buf.data_ptr(), 33, 5)
    assert e.value.status == R.RNG_EINVAL
    with pytest.raises(R.RngError):
        R.rng_skipahead_noalloc(R.RNG_XORWOW, 0, 64, 5)
    # more instances than one launch covers: rejected before anything runs
    with pytest.raises(R.RngError) as e:
        R.rng_skipahead_noalloc(R.RNG_XORWOW, buf.data_ptr(), 1 << 40, 5)
    assert e.value.status == R.RNG_EINVAL and "instances" in str(e.value)
