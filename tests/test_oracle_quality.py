"""Self-written frequency and serial checks of the oracle's streams (the
paper's equidistribution test, Sec. 6, divides [0,1) into 2^l cells and
t-dimensional cubes; these are the l = 8, t = 1 and l = 4, t = 2 cases), in
single-instance order and in step-major ("warp") order.  The low bits of the
32-bit LCG, whose bit k has period 2^k (Sec. 2), are the negative control."""
import numpy as np
import pytest

import oracle as O

SEED = 0x0123456789ABCDEF
KINDS = [O.LCG32, O.LCG64, O.MWC, O.XORWOW, O.PHILOX4X32_10, O.XS1024W, O.MT19937_SHARED, O.PHILOX4X32_7,
         O.LFIB521, O.LFIB1279]


def chi2_cells(cells, ncells):
    h = np.bincount(cells, minlength=ncells).astype(np.float64)
    e = len(cells) / ncells
    return ((h - e) ** 2 / e).sum()


def bound(dof, sig=7.0):
    return dof + sig * np.sqrt(2 * dof)


def streams(kind):
    if kind in (O.MT19937_SHARED, O.LFIB521, O.LFIB1279):  # block-shared states: few long streams
        return O.generate(kind, SEED, 4, 1 << 18)
    return O.generate(kind, SEED, 1024, 1024)


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("order", ["instance", "step"])
def test_frequency_and_serial(kind, order):
    s = streams(kind)
    seq = (s.ravel() if order == "instance" else s.T.ravel()).astype(np.uint64)
    assert chi2_cells((seq >> 24).astype(np.int64), 256) < bound(255)
    pairs = ((seq[:-1:2] >> 28) << 4) | (seq[1::2] >> 28)
    assert chi2_cells(pairs.astype(np.int64), 256) < bound(255)
    u = seq.astype(np.float64)
    rho = np.corrcoef(u[:-1], u[1:])[0, 1]
    assert abs(rho) < 7 / np.sqrt(len(u))


def test_lcg32_low_bits_fail_the_serial_test():
    s = O.generate(O.LCG32, SEED, 1, 1 << 16)[0].astype(np.uint64)
    pairs = ((s[:-1:2] & 15) << 4) | (s[1::2] & 15)
    assert chi2_cells(pairs.astype(np.int64), 256) > 10 * bound(255)
