"""Exact finite-lattice results for the 2D Ising ferromagnet (J = 1, zero
field, periodic L x L), the reference values of the paper's application test
(Sec. 2 and Table 1: e and C_V of a 1024^2 lattice at beta = 0.4, computed
from the exact finite-size solution of Ferdinand and Fisher).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Partition function (Kaufman 1949; Ferdinand and Fisher 1969) of an L x L
torus with coupling K = beta J:

    Z = 1/2 (2 sinh 2K)^(L^2/2) (Z1 + Z2 + Z3 + Z4),
    Z1 = prod_{r<L} 2 cosh(L g_{2r+1} / 2),  Z2 = prod 2 sinh(L g_{2r+1} / 2),
    Z3 = prod_{r<L} 2 cosh(L g_{2r} / 2),    Z4 = prod 2 sinh(L g_{2r} / 2),
    cosh g_k = cosh 2K coth 2K - cos(pi k / L)  (g_k > 0 for k != 0),
    g_0 = 2K + ln tanh K  (signed).

The paper's e is -<E>/N (positive) and C_V = beta^2 (<E^2> - <E>^2) / N with
N = L^2; with K = beta these are (1/N) d lnZ/dK and (K^2/N) d^2 lnZ/dK^2.
mpmath carries arbitrary exponents, so the products are formed directly and
differentiated numerically at high working precision.
"""
from __future__ import annotations

import numpy as np

try:
    import mpmath as mp
except ImportError:  # pragma: no cover - the GPU image has no mpmath
    mp = None


def _gammas(K, L):
    c = mp.cosh(2 * K) * mp.coth(2 * K)
    g = [None] * (2 * L)
    g[0] = 2 * K + mp.log(mp.tanh(K))
    for k in range(1, 2 * L):
        g[k] = mp.acosh(c - mp.cos(mp.pi * k / L))
    return g


def log_z(K, L: int):
    """ln Z of the L x L periodic lattice at coupling K (mpmath number)."""
    K = mp.mpf(K)
    g = _gammas(K, L)
    z1 = z2 = z3 = z4 = mp.mpf(1)
    for r in range(L):
        a = L * g[2 * r + 1] / 2
        b = L * g[2 * r] / 2
        z1 *= 2 * mp.cosh(a)
        z2 *= 2 * mp.sinh(a)
        z3 *= 2 * mp.cosh(b)
        z4 *= 2 * mp.sinh(b)
    return mp.log(mp.mpf(1) / 2) + mp.mpf(L * L) / 2 * mp.log(2 * mp.sinh(2 * K)) + mp.log(z1 + z2 + z3 + z4)


def exact_e_cv(L: int, beta: float, dps: int = 40) -> tuple[float, float]:
    """(e, C_V) per spin, e = -<E>/N, C_V = beta^2 var(E) / N."""
    if mp is None:
        raise RuntimeError("mpmath is required for the exact finite-lattice solution")
    with mp.workdps(dps):
        K = mp.mpf(beta)
        N = L * L
        f = lambda k: log_z(k, L)
        d1 = mp.diff(f, K, 1)
        d2 = mp.diff(f, K, 2)
        return float(d1 / N), float(K * K * d2 / N)


def brute_force_moments(L: int, beta: float) -> tuple[float, float, float]:
    """(ln Z, <E>, <E^2>) by enumerating all 2^(L^2) configurations (L <= 4)."""
    n = L * L
    assert n <= 16
    idx = np.arange(1 << n, dtype=np.int64)
    bits = ((idx[:, None] >> np.arange(n)[None, :]) & 1).astype(np.int64)
    s = (2 * bits - 1).reshape(-1, L, L)
    E = -(s * np.roll(s, -1, axis=2)).sum(axis=(1, 2)) - (s * np.roll(s, -1, axis=1)).sum(axis=(1, 2))
    E = E.astype(np.float64)
    w = np.exp(-beta * (E - E.min()))
    Zs = w.sum()
    mE = (w * E).sum() / Zs
    mE2 = (w * E * E).sum() / Zs
    return float(np.log(Zs) - beta * E.min()), float(mE), float(mE2)


def exact_moments(L: int, beta: float, dps: int = 40) -> tuple[float, float, float]:
    """(ln Z, <E>, <E^2>) from the closed form, for comparison with brute force."""
    with mp.workdps(dps):
        K = mp.mpf(beta)
        f = lambda k: log_z(k, L)
        lz = f(K)
        d1 = mp.diff(f, K, 1)
        d2 = mp.diff(f, K, 2)
        mE = -d1
        mE2 = d2 + d1 * d1
        return float(lz), float(mE), float(mE2)


__all__ = ["log_z", "exact_e_cv", "brute_force_moments", "exact_moments"]
