"""The allocator hook of the C ABI (rng_set_allocator): the library's
handle memory comes from the installed allocator -- here PyTorch's caching
allocator -- with results unchanged, and the allocator cannot change while
its memory is live."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu
SEED = 0x0123456789ABCDEF


@pytest.fixture(scope="module")
def R():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1204_6193_gb300 as R
    return R


def test_torch_caching_allocator_backs_handles(R):
    import torch
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    R.use_torch_allocator()
    try:
        n, K = 1 << 20, 64
        h = R.rng_create(R.RNG_XORWOW, n)
        try:
            held = torch.cuda.memory_allocated() - base
            assert held >= 24 * n  # six 32-bit words of state per instance
            R.rng_seed(h, SEED)
            out = torch.empty(n * K, dtype=torch.int32, device="cuda")
            R.rng_generate_u32(h, out.data_ptr(), K, R.RNG_INSTANCE_MAJOR)
            torch.cuda.synchronize()
            got = out.view(n, K)[:300].cpu().numpy().view(np.uint32)
            assert np.array_equal(got, O.generate(O.XORWOW, SEED, n, K, i_lo=0, i_hi=300))
            with pytest.raises(R.RngError) as e:  # memory of the installed allocator is live
                R.use_torch_allocator(False)
            assert e.value.status == R.RNG_EBUSY
            del out
        finally:
            R.rng_destroy(h)
        torch.cuda.synchronize()
        assert torch.cuda.memory_allocated() - base <= 0
        # an Ising handle (lattice, plan, halo buffers) through the same hooks
        ref, _, _ = O.ising_run(128, 0.42, O.XS1024W, SEED, 30)
        hi = R.ising_create(128, 0.42, 0, O.XS1024W, 0, SEED, 2)
        try:
            R.ising_sweep(hi, 30)
            assert np.array_equal(R.ising_get_spins(hi), ref)
        finally:
            R.ising_destroy(hi)
    finally:
        torch.cuda.synchronize()
        R.use_torch_allocator(False)


def test_failing_allocator_reports_out_of_memory(R):
    calls = []

    def alloc(nbytes, stream):
        calls.append(nbytes)
        return 0  # no memory

    R.rng_set_allocator(alloc, lambda ptr, stream: None)
    try:
        with pytest.raises(R.RngError) as e:
            R.rng_create(R.RNG_LCG32, 1024)
        assert e.value.status == R.RNG_ENOMEM
        assert calls
    finally:
        R.rng_set_allocator()
    h = R.rng_create(R.RNG_LCG32, 1024)  # the default allocator is back
    R.rng_destroy(h)


def test_hooks_come_in_pairs(R):
    lib = R.library()
    assert lib.rng_set_allocator(R.RNG_ALLOC_FN(lambda *a: 1), R.RNG_FREE_FN(), None) == R.RNG_EINVAL
