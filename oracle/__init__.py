"""CPU oracle for the per-thread random-number streams and the checkerboard
Ising update of Manssen, Weigel and Hartmann, arXiv:1204.6193.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the product library
never does.  The arithmetic lives in ``oracle.c`` (plain serial C, built here
with gcc into ``oracle/_build``); this module only marshals numpy arrays.

Generator kinds and flags use the same numeric values as the library's C ABI
(they are the public interface both sides implement); see ``oracle.c`` for the
definition of every stream, each citing the passage of the paper it follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")

LCG32, LCG64, MWC, XORWOW, PHILOX4X32_10, XS1024W, MT19937_SHARED, PHILOX4X32_7, LFIB521, LFIB1279 = range(10)
SEED_RANDOM, SEED_LEAPFROG, SEED_SUBSTREAM, MWC_SAME_A, PHILOX_INTRINSIC_KEY = 0, 1, 2, 4, 8
KIND_NAMES = {LCG32: "lcg32", LCG64: "lcg64", MWC: "mwc", XORWOW: "xorwow",
              PHILOX4X32_10: "philox4x32_10", XS1024W: "xs1024w",
              MT19937_SHARED: "mt19937_shared", PHILOX4X32_7: "philox4x32_7", LFIB521: "lfib521",
              LFIB1279: "lfib1279"}
LFIB_LAGS = {LFIB521: (521, 353), LFIB1279: (1279, 861)}

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compiles oracle.c into oracle/_build/liboracle.so (gcc, -O2)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            u64, u32, i32, dbl, p = (ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int,
                                     ctypes.c_double, ctypes.c_void_p)
            sig = {
                "orc_mix64": (u64, [u64]),
                "orc_seed_word": (u64, [u64, u64]),
                "orc_lcg_jump_coeffs": (None, [i32, u64, p, p]),
                "orc_is_prime_u64": (i32, [u64]),
                "orc_mwc_multipliers": (i32, [u64, p]),
                "orc_philox4x32": (None, [p, u32, u32, i32, p]),
                "orc_xs1024_shift_step": (None, [p]),
                "orc_xs_matrix": (i32, [p]),
                "orc_xorwow_matrix": (i32, [p]),
                "orc_matrix_pow2k": (i32, [i32, i32, p]),
                "orc_generate": (i32, [i32, u32, u64, u64, u64, i32, u64, u64, u64, i32, p]),
                "orc_to_f32": (None, [p, u64, p]),
                "orc_box_muller": (None, [p, u64, p]),
                "orc_ising_threshold": (u64, [dbl, i32]),
                "orc_ising_init_spins": (None, [u32, u64, p]),
                "orc_ising_energy": (None, [u32, p, p, p]),
                "orc_ising_run": (i32, [u32, dbl, i32, u32, u64, u32, u64, u32, i32, p, p, p]),
                "orc_mt19937_raw": (None, [u32, u64, p]),
                "orc_lfib_raw": (i32, [u32, u32, i32, p, u64, p]),
                "orc_ising_run_multihit": (i32, [u32, dbl, i32, u32, u64, u32, u32, u32, u64, u32, i32, p, p, p]),
                "orc_ising_half_sweep_given": (i32, [u32, dbl, u32, i32, u32, u32, u64, p, p]),
                "orc_ising_sweep_given": (i32, [u32, dbl, u32, u64, p, p]),
                "orc_ising_multihit_round_given": (i32, [u32, dbl, u32, u32, u32, u64, p, p]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _ptr(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


class OracleError(RuntimeError):
    pass


def _check(st: int, what: str):
    if st != 0:
        raise OracleError(f"{what}: oracle status {st}")


def mix64(z: int) -> int:
    return lib().orc_mix64(z & (2**64 - 1))


def seed_word(seed: int, k: int) -> int:
    return lib().orc_seed_word(seed & (2**64 - 1), k)


def lcg_jump_coeffs(is64: bool, t: int) -> tuple[int, int]:
    at = ctypes.c_uint64()
    ct = ctypes.c_uint64()
    lib().orc_lcg_jump_coeffs(int(is64), t & (2**64 - 1), ctypes.byref(at), ctypes.byref(ct))
    return at.value, ct.value


def is_prime_u64(n: int) -> bool:
    return bool(lib().orc_is_prime_u64(n))


def mwc_multipliers(count: int) -> np.ndarray:
    out = np.zeros(count, dtype=np.uint32)
    _check(lib().orc_mwc_multipliers(count, _ptr(out)), "mwc_multipliers")
    return out


def philox4x32(ctr, key0: int, key1: int, rounds: int = 10) -> np.ndarray:
    c = np.asarray(ctr, dtype=np.uint32).copy()
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32(_ptr(c), key0, key1, rounds, _ptr(out))
    return out


def xs1024_shift_step(words: np.ndarray) -> np.ndarray:
    w = np.ascontiguousarray(words, dtype=np.uint32).copy()
    assert w.shape == (32,)
    lib().orc_xs1024_shift_step(_ptr(w))
    return w


def xs_matrix() -> np.ndarray:
    out = np.zeros((1024, 16), dtype=np.uint64)
    _check(lib().orc_xs_matrix(_ptr(out)), "xs_matrix")
    return out


def xorwow_matrix() -> np.ndarray:
    out = np.zeros((160, 3), dtype=np.uint64)
    _check(lib().orc_xorwow_matrix(_ptr(out)), "xorwow_matrix")
    return out


def matrix_pow2k(which: str, k: int) -> np.ndarray:
    """M^(2^k) for which='xs1024' (1024x1024) or 'xorwow' (160x160)."""
    if which == "xs1024":
        out = np.zeros((1024, 16), dtype=np.uint64)
        _check(lib().orc_matrix_pow2k(0, k, _ptr(out)), "matrix_pow2k")
    else:
        out = np.zeros((160, 3), dtype=np.uint64)
        _check(lib().orc_matrix_pow2k(1, k, _ptr(out)), "matrix_pow2k")
    return out


def generate(kind: int, seed: int, n: int, K: int, *, flags: int = 0, skip: int = 0,
             jump: bool = False, i_lo: int = 0, i_hi: int | None = None,
             philox_rounds: int = 10) -> np.ndarray:
    """Streams s_i[skip + k] for i in [i_lo, i_hi), k < K, shape (i_hi-i_lo, K)."""
    if i_hi is None:
        i_hi = n
    out = np.zeros((i_hi - i_lo, K), dtype=np.uint32)
    _check(lib().orc_generate(kind, flags, seed & (2**64 - 1), n, skip, int(jump), i_lo, i_hi, K,
                              philox_rounds, _ptr(out)), "generate")
    return out


def to_f32(r: np.ndarray) -> np.ndarray:
    r = np.ascontiguousarray(r, dtype=np.uint32)
    out = np.zeros(r.shape, dtype=np.float64)
    lib().orc_to_f32(_ptr(r), r.size, _ptr(out))
    return out


def box_muller(r: np.ndarray) -> np.ndarray:
    """Normals from consecutive pairs along the last axis (even length)."""
    r = np.ascontiguousarray(r, dtype=np.uint32)
    assert r.shape[-1] % 2 == 0
    out = np.zeros(r.shape, dtype=np.float64)
    lib().orc_box_muller(_ptr(r), r.size // 2, _ptr(out))
    return out


def ising_threshold(beta: float, dE: int) -> int:
    return lib().orc_ising_threshold(beta, dE)


def ising_init_spins(L: int, seed: int) -> np.ndarray:
    s = np.zeros((L, L), dtype=np.int8)
    lib().orc_ising_init_spins(L, seed & (2**64 - 1), _ptr(s))
    return s


def ising_energy(spins: np.ndarray) -> tuple[int, int]:
    s = np.ascontiguousarray(spins, dtype=np.int8)
    E = ctypes.c_int64()
    M = ctypes.c_int64()
    lib().orc_ising_energy(s.shape[0], _ptr(s), ctypes.byref(E), ctypes.byref(M))
    return E.value, M.value


def ising_run(L: int, beta: float, kind: int, seed: int, n_sweeps: int, *, G: int = 2,
              flags: int = 0, measure_every: int = 0, spins: np.ndarray | None = None,
              philox_rounds: int = 10):
    """Runs n_sweeps checkerboard sweeps; returns (spins, acc[4], n_meas)."""
    s = ising_init_spins(L, seed) if spins is None else np.ascontiguousarray(spins, dtype=np.int8).copy()
    acc = np.zeros(4, dtype=np.int64)
    nm = ctypes.c_uint64()
    _check(lib().orc_ising_run(L, beta, kind, flags, seed & (2**64 - 1), G, n_sweeps, measure_every,
                               philox_rounds, _ptr(s), _ptr(acc), ctypes.byref(nm)), "ising_run")
    return s, acc, nm.value


def ising_run_multihit(L: int, beta: float, kind: int, seed: int, n_rounds: int, *, k: int, n_strips: int,
                       G: int = 2, flags: int = 0, measure_every: int = 0, spins: np.ndarray | None = None,
                       philox_rounds: int = 10):
    """n_rounds double-checkerboard rounds of k hits; returns (spins, acc[4], n_meas)."""
    s = ising_init_spins(L, seed) if spins is None else np.ascontiguousarray(spins, dtype=np.int8).copy()
    acc = np.zeros(4, dtype=np.int64)
    nm = ctypes.c_uint64()
    _check(lib().orc_ising_run_multihit(L, beta, kind, flags, seed & (2**64 - 1), G, n_strips, k, n_rounds,
                                        measure_every, philox_rounds, _ptr(s), _ptr(acc), ctypes.byref(nm)),
           "ising_run_multihit")
    return s, acc, nm.value


def _lattices(spins: np.ndarray, L: int) -> np.ndarray:
    s = np.ascontiguousarray(spins, dtype=np.int8).copy()
    assert s.shape[-2:] == (L, L)
    return s.reshape(-1, L, L)


def ising_half_sweep_given(spins: np.ndarray, beta: float, colour: int, draws: np.ndarray, *, G: int = 2,
                           rows: tuple[int, int] | None = None) -> np.ndarray:
    """One half-sweep of the oracle's update on each lattice of spins (shape
    (..., L, L)) with the caller's numbers: draws[b, sidx, g] is the g-th
    number of stream sidx of lattice b (L^2 / (2G) streams; only the streams
    of rows [row0, row1) are read).  Returns the new spins."""
    L = spins.shape[-1]
    s = _lattices(spins, L)
    d = np.ascontiguousarray(draws, dtype=np.uint32).reshape(s.shape[0], -1)
    assert d.shape[1] == L * L // 2
    r0, r1 = rows if rows is not None else (0, L)
    _check(lib().orc_ising_half_sweep_given(L, beta, G, colour, r0, r1, s.shape[0], _ptr(d), _ptr(s)),
           "ising_half_sweep_given")
    return s.reshape(spins.shape)


def ising_sweep_given(spins: np.ndarray, beta: float, draws: np.ndarray, *, G: int = 2) -> np.ndarray:
    """One sweep (colour 0 then colour 1) with the caller's numbers:
    draws[b, sidx, d] is the d-th of the 2G numbers of stream sidx."""
    L = spins.shape[-1]
    s = _lattices(spins, L)
    d = np.ascontiguousarray(draws, dtype=np.uint32).reshape(s.shape[0], -1)
    assert d.shape[1] == L * L
    _check(lib().orc_ising_sweep_given(L, beta, G, s.shape[0], _ptr(d), _ptr(s)), "ising_sweep_given")
    return s.reshape(spins.shape)


def ising_multihit_round_given(spins: np.ndarray, beta: float, draws: np.ndarray, *, k: int, n_strips: int,
                               G: int = 2) -> np.ndarray:
    """One multi-hit round with the caller's numbers: draws[b, sidx, d] is
    the d-th of the 2kG numbers of stream sidx."""
    L = spins.shape[-1]
    s = _lattices(spins, L)
    d = np.ascontiguousarray(draws, dtype=np.uint32).reshape(s.shape[0], -1)
    assert d.shape[1] == L * L * k
    _check(lib().orc_ising_multihit_round_given(L, beta, G, n_strips, k, s.shape[0], _ptr(d), _ptr(s)),
           "ising_multihit_round_given")
    return s.reshape(spins.shape)


def lfib_raw(r: int, s: int, bits: int, seeds, K: int) -> np.ndarray:
    """K outputs of x_n = x_(n-r) + x_(n-s) mod 2^bits from seeds x_(-r) .. x_(-1)."""
    sd = np.ascontiguousarray(seeds, dtype=np.uint32)
    assert sd.shape == (r,)
    out = np.zeros(K, dtype=np.uint32)
    _check(lib().orc_lfib_raw(r, s, bits, _ptr(sd), K, _ptr(out)), "lfib_raw")
    return out


def mt19937_raw(seed32: int, K: int) -> np.ndarray:
    out = np.zeros(K, dtype=np.uint32)
    lib().orc_mt19937_raw(seed32, K, _ptr(out))
    return out
