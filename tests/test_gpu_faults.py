"""Failure paths driven by host-side fault injection (RNG_FAULT): injected
allocation failures at every allocation of a handle's construction and
first sweep, injected launch failures and an injected neighbour-wait
timeout.  No GPU fault is made: the failures are fakes of the failing host
calls, and every test checks that the library leaks nothing and keeps
working once the fault is gone."""
import os

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


@pytest.fixture
def fault():
    def set_fault(v):
        if v is None:
            os.environ.pop("RNG_FAULT", None)
        else:
            os.environ["RNG_FAULT"] = v
    yield set_fault
    os.environ.pop("RNG_FAULT", None)


def no_live_allocations(R):
    # the allocator can only be (re)set when none of its memory is live
    try:
        R.rng_set_allocator()
        return True
    except R.RngError as e:
        assert e.status == R.RNG_EBUSY
        return False


def test_every_allocation_of_an_ising_handle_can_fail_cleanly(R, fault):
    import torch
    assert no_live_allocations(R)
    failures = 0
    for nth in range(1, 40):
        fault(f"oom:{nth}")
        h = None
        try:
            h = R.ising_create(256, 0.4, 0, O.XORWOW, 0, SEED, 2)
            R.ising_sweep(h, 3, 1)
            R.ising_observables(h)
        except R.RngError as e:
            assert e.status == R.RNG_ENOMEM, e
            assert "RNG_FAULT" in R.rng_last_error()
            failures += 1
        finally:
            fault(None)
            if h is not None:
                R.ising_destroy(h)
        torch.cuda.synchronize()
        assert no_live_allocations(R), f"allocation {nth}: memory leaked after the failure"
        if failures < nth:  # the countdown passed every allocation: all were covered
            break
    assert failures >= 5
    # and the library still works
    ref, _, _ = O.ising_run(64, 0.4, O.XORWOW, SEED, 10)
    h = R.ising_create(64, 0.4, 0, O.XORWOW, 0, SEED, 2)
    try:
        R.ising_sweep(h, 10)
        assert np.array_equal(R.ising_get_spins(h), ref)
    finally:
        R.ising_destroy(h)


def test_allocation_failure_of_generators(R, fault):
    fault("oom")
    for kind in (O.LCG32, O.MWC, O.XS1024W, O.MT19937_SHARED, O.LFIB521):
        with pytest.raises(R.RngError) as e:
            R.rng_create(kind, 64)
        assert e.value.status == R.RNG_ENOMEM
    fault(None)
    assert no_live_allocations(R)


def test_launch_failure_is_reported_and_the_handle_recovers(R, fault):
    import torch
    n, K = 1000, 33
    h = R.rng_create(O.XORWOW, n)
    try:
        fault("launch")
        with pytest.raises(R.RngError) as e:
            R.rng_seed(h, SEED)
        assert e.value.status == R.RNG_ECUDA
        buf = torch.empty(n * K, dtype=torch.int32, device="cuda")
        with pytest.raises(R.RngError):
            R.rng_generate_u32(h, buf.data_ptr(), K, R.RNG_INSTANCE_MAJOR)
        fault(None)
        R.rng_seed(h, SEED)  # a fresh seed defines the streams again
        R.rng_generate_u32(h, buf.data_ptr(), K, R.RNG_INSTANCE_MAJOR)
        torch.cuda.synchronize()
        got = buf.cpu().numpy().view(np.uint32).reshape(n, K)
        assert np.array_equal(got, O.generate(O.XORWOW, SEED, n, K))
    finally:
        R.rng_destroy(h)


def test_timeout_is_reported_then_cleared(R, fault):
    h = R.ising_create(128, 0.4, 1, O.PHILOX4X32_10, 0, SEED, 2)
    try:
        R.ising_sweep(h, 5)
        fault("timeout")
        with pytest.raises(R.RngError) as e:
            R.ising_observables(h)
        assert e.value.status == R.RNG_ETIMEOUT
        fault(None)
        obs = R.ising_observables(h)
        ref, _, _ = O.ising_run(128, 0.4, O.PHILOX4X32_10, SEED, 5)
        assert (obs["E"], obs["M"]) == O.ising_energy(ref)
    finally:
        R.ising_destroy(h)
