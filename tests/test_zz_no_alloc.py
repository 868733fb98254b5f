"""rng_skipahead_noalloc: the skip-ahead for callers that cannot allocate
device memory (a framework that owns every device allocation, or a sequence
that must not synchronise on an allocation).  It advances a state array the
caller owns, keeping its matrix scratch in a static device array, and must
give exactly what rng_skipahead gives on a library handle.  Collected last on
purpose: a failure here comes after every other test has run."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SEED = 0x0123456789ABCDEF


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
def test_noalloc_matches_rng_skipahead_twice(env, kind, n, arrays):
    R, torch = env
    h = R.rng_create(kind, n)
    try:
        R.rng_seed(h, SEED)
        mine = torch.from_numpy(state_words(R, h, arrays * n).view(np.int32)).cuda()
        for t in (12345, 2**40 + 77):  # two calls in a row
            R.rng_skipahead_noalloc(kind, mine.data_ptr(), n, t)
            R.rng_skipahead(h, t)
            torch.cuda.synchronize()
            ref = state_words(R, h, arrays * n)
            got = mine.cpu().numpy().view(np.uint32)
            assert np.array_equal(got, ref), t
    finally:
        R.rng_destroy(h)


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
