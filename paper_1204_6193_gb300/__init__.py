"""Python binding of librng_gb300.so (C ABI in include/rng_gb300.h).

Argument marshalling only: every function calls the C entry point of the
same name; device buffers are passed as integer addresses (for example
``tensor.data_ptr()``) and CUDA streams as integer handles (for example
``torch.cuda.current_stream().cuda_stream``).  A nonzero status raises
:class:`RngError` carrying the library's own message.  There is no CPU
fallback: without the built library the import fails.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
# RNG_GB300_LIBRARY selects another build of the same library (the
# bounds-check build of build.py, for tests)
LIB_PATH = os.environ.get("RNG_GB300_LIBRARY") or os.path.join(_HERE, "_build", "librng_gb300.so")

RNG_OK, RNG_EINVAL, RNG_ENOMEM, RNG_EUNSUPPORTED, RNG_ECUDA, RNG_ETIMEOUT, RNG_EBUSY = range(7)
(RNG_LCG32, RNG_LCG64, RNG_MWC, RNG_XORWOW, RNG_PHILOX4X32_10, RNG_XS1024W,
 RNG_MT19937_SHARED, RNG_PHILOX4X32_7, RNG_LFIB521, RNG_LFIB1279) = range(10)
RNG_SEED_RANDOM, RNG_SEED_LEAPFROG, RNG_SEED_SUBSTREAM, RNG_MWC_SAME_A, RNG_PHILOX_INTRINSIC_KEY = 0, 1, 2, 4, 8
RNG_STEP_MAJOR, RNG_INSTANCE_MAJOR, RNG_XOR_REDUCE = 0, 1, 2
ISING_INT8, ISING_MULTISPIN32 = 0, 1

KIND_NAMES = {RNG_LCG32: "lcg32", RNG_LCG64: "lcg64", RNG_MWC: "mwc", RNG_XORWOW: "xorwow",
              RNG_PHILOX4X32_10: "philox4x32_10", RNG_XS1024W: "xs1024w",
              RNG_MT19937_SHARED: "mt19937_shared", RNG_PHILOX4X32_7: "philox4x32_7",
              RNG_LFIB521: "lfib521", RNG_LFIB1279: "lfib1279"}
BLOCK_SHARED_KINDS = (RNG_MT19937_SHARED, RNG_LFIB521, RNG_LFIB1279)


class RngError(RuntimeError):
    def __init__(self, status: int, func: str, detail: str):
        super().__init__(f"{func}: status {status}: {detail}")
        self.status = status


if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with paper_1204_6193_gb300.build.build() "
                      "(nvcc, sm_103a); there is no fallback implementation")

_lib = ctypes.CDLL(LIB_PATH)
_u64, _u32, _i32, _f64, _p = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
_pp = ctypes.POINTER(ctypes.c_void_p)

_SIGS = {
    "rng_create": [_pp, _i32, _u64, _u32, _p],
    "rng_create_shard": [_pp, _i32, _u64, _u64, _u64, _u32, _p],
    "rng_destroy": [_p],
    "rng_seed": [_p, _u64],
    "rng_skipahead": [_p, _u64],
    "rng_generate_u32": [_p, _p, _u64, _i32, _p],
    "rng_generate_f32": [_p, _p, _u64, _i32, _p],
    "rng_generate_normal": [_p, _p, _u64, _i32, _p],
    "rng_u32_to_normal": [_p, _p, _u64, _p],
    "rng_get_state": [_p, _p, ctypes.POINTER(ctypes.c_size_t)],
    "rng_set_state": [_p, _p, ctypes.c_size_t],
    "rng_info": [_p, ctypes.POINTER(_i32), ctypes.POINTER(_u64), ctypes.POINTER(_u64), ctypes.POINTER(_u64)],
    "rng_mwc_multipliers": [_u64, _u64, _p],
    "rng_skipahead_noalloc": [_i32, _p, _u64, _u64, _p],
    "ising_create": [_pp, _u32, _f64, _i32, _i32, _u32, _u64, _u32, _p],
    "ising_destroy": [_p],
    "ising_sweep": [_p, _u64, _u32, _p],
    "ising_sweep_plain": [_p, _u64, _u32, _p],
    "ising_sweep_multihit": [_p, _u64, _u32, _u32, _u32, _p],
    "ising_observables": [_p, _p, _p, _p, _p],
    "ising_get_spins": [_p, _p],
    "ising_set_spins": [_p, _p],
    "ising_get_rng": [_p, _pp],
    "ising_set_launch": [_p, _u32, _i32, _u32],
    "ising_set_halo_depth": [_p, _u32],
    "ising_get_halo_depth": [_p, _p],
    "ising_get_launch": [_p, _p, _p, _p],
    "ising_autotune": [_p, _u32, _p, _p],
    "ising_info": [_p, _u32, _p, _p, _p, _p, _p],
    "ising_batch_create": [_pp, _u32, _p, _p, _p, _u64, _u32, _p],
    "ising_batch_sweep": [_p, _u64, _u32, _p],
    "ising_batch_observables": [_p, _u32, _p, _p, _p, _p],
    "ising_batch_get_spins": [_p, _u32, _p],
    "ising_debug_mute_strip": [_p, ctypes.c_int32, _u64],
    "rng_debug_bounds_status": [ctypes.POINTER(_i32), _i32],
    "ising_plan_info": [_p, _p, _p, _p, _p],
    "rng_server_create": [_pp, _u32, _u32, _u32, _u64],
    "rng_server_submit": [_p, _p, ctypes.POINTER(_u64)],
    "rng_server_wait": [_p, _u64, _f64, _p],
    "rng_server_fetch": [_p, _u64, _p, _u64],
    "rng_server_stats": [_p, ctypes.POINTER(_u64), ctypes.POINTER(_u64), ctypes.POINTER(_u64), ctypes.POINTER(_u32)],
    "rng_server_destroy": [_p],
    "rng_issue_peaks": [_p, _p, _p, _p, _p],
}
for _name, _args in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = _i32
_lib.rng_strerror.argtypes = [_i32]
_lib.rng_strerror.restype = ctypes.c_char_p
_lib.rng_last_error.argtypes = []
_lib.rng_last_error.restype = ctypes.c_char_p


# Allocator hooks (rng_set_allocator): int alloc(void **ptr, size_t bytes,
# void *stream, void *ctx) and void free(void *ptr, void *stream, void *ctx).
RNG_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.POINTER(ctypes.c_void_p), ctypes.c_size_t, ctypes.c_void_p,
                                ctypes.c_void_p)
RNG_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)
_lib.rng_set_allocator.argtypes = [RNG_ALLOC_FN, RNG_FREE_FN, _p]
_lib.rng_set_allocator.restype = _i32
_allocator_keepalive = None  # the installed ctypes callbacks must outlive their use


def _call(name: str, *args) -> None:
    st = getattr(_lib, name)(*args)
    if st != RNG_OK:
        raise RngError(st, name, _lib.rng_last_error().decode(errors="replace"))


def _stream(stream) -> int | None:
    if stream is None:
        return None
    return int(getattr(stream, "cuda_stream", stream))


def library() -> ctypes.CDLL:
    return _lib


def rng_set_allocator(alloc=None, free=None) -> None:
    """Installs Python callables as the library's device allocator:
    alloc(nbytes, stream) -> device pointer (int), free(ptr, stream).  With
    no arguments the library returns to cudaMallocAsync."""
    global _allocator_keepalive
    if alloc is None and free is None:
        _call("rng_set_allocator", RNG_ALLOC_FN(), RNG_FREE_FN(), None)
        _allocator_keepalive = None
        return

    def _a(pp, nbytes, stream, _ctx):
        try:
            ptr = int(alloc(int(nbytes), int(stream or 0)))
        except Exception:  # reported to the caller of the library as RNG_ENOMEM
            return 1
        pp[0] = ptr
        return 0 if ptr else 1

    def _f(ptr, stream, _ctx):
        free(int(ptr), int(stream or 0))

    cbs = (RNG_ALLOC_FN(_a), RNG_FREE_FN(_f))
    _call("rng_set_allocator", cbs[0], cbs[1], None)
    _allocator_keepalive = cbs


def use_torch_allocator(enable: bool = True) -> None:
    """Routes the library's device memory through PyTorch's caching
    allocator (or, with enable=False, back to cudaMallocAsync)."""
    if not enable:
        rng_set_allocator()
        return
    import torch

    def alloc(nbytes, stream):
        return torch.cuda.caching_allocator_alloc(nbytes, torch.cuda.current_device(), stream)

    def free(ptr, stream):
        torch.cuda.caching_allocator_delete(ptr)

    rng_set_allocator(alloc, free)


def rng_issue_peaks(stream=None) -> dict:
    """Measured pipe throughputs (thread-instructions per second, whole GPU)."""
    v = [ctypes.c_double() for _ in range(4)]
    _call("rng_issue_peaks", *[ctypes.byref(x) for x in v], _stream(stream))
    return {"lop3": v[0].value, "imad": v[1].value, "shfl": v[2].value, "ffma": v[3].value}


def rng_strerror(status: int) -> str:
    return _lib.rng_strerror(status).decode()


def rng_last_error() -> str:
    return _lib.rng_last_error().decode(errors="replace")


def rng_create(kind: int, n_instances: int, flags: int = 0, stream=None) -> int:
    h = ctypes.c_void_p()
    _call("rng_create", ctypes.byref(h), kind, n_instances, flags, _stream(stream))
    return h.value


def rng_create_shard(kind: int, n_total: int, first: int, count: int, flags: int = 0, stream=None) -> int:
    h = ctypes.c_void_p()
    _call("rng_create_shard", ctypes.byref(h), kind, n_total, first, count, flags, _stream(stream))
    return h.value


def rng_destroy(h: int) -> None:
    _call("rng_destroy", h)


def rng_seed(h: int, seed: int) -> None:
    _call("rng_seed", h, seed & (2**64 - 1))


def rng_skipahead(h: int, n: int) -> None:
    _call("rng_skipahead", h, n)


def rng_generate_u32(h: int, d_out: int, n_per_instance: int, layout: int = RNG_STEP_MAJOR, stream=None) -> None:
    _call("rng_generate_u32", h, d_out, n_per_instance, layout, _stream(stream))


def rng_generate_f32(h: int, d_out: int, n_per_instance: int, layout: int = RNG_STEP_MAJOR, stream=None) -> None:
    _call("rng_generate_f32", h, d_out, n_per_instance, layout, _stream(stream))


def rng_generate_normal(h: int, d_out: int, n_per_instance: int, layout: int = RNG_STEP_MAJOR, stream=None) -> None:
    _call("rng_generate_normal", h, d_out, n_per_instance, layout, _stream(stream))


def rng_u32_to_normal(d_in: int, d_out: int, n_pairs: int, stream=None) -> None:
    _call("rng_u32_to_normal", d_in, d_out, n_pairs, _stream(stream))


def rng_get_state(h: int) -> bytes:
    size = ctypes.c_size_t(0)
    _call("rng_get_state", h, None, ctypes.byref(size))
    buf = ctypes.create_string_buffer(size.value)
    _call("rng_get_state", h, buf, ctypes.byref(size))
    return buf.raw[: size.value]


def rng_set_state(h: int, blob: bytes) -> None:
    buf = ctypes.create_string_buffer(blob, len(blob))
    _call("rng_set_state", h, buf, len(blob))


def rng_info(h: int) -> dict:
    k, n, f, p = _i32(), _u64(), _u64(), _u64()
    _call("rng_info", h, ctypes.byref(k), ctypes.byref(n), ctypes.byref(f), ctypes.byref(p))
    return {"kind": k.value, "n_instances": n.value, "first": f.value, "position": p.value}


def rng_skipahead_noalloc(kind: int, d_state: int, n_instances: int, n: int, stream=None) -> None:
    _call("rng_skipahead_noalloc", kind, d_state, n_instances, n, _stream(stream))


def rng_mwc_multipliers(first: int, count: int):
    import numpy as np
    out = np.zeros(count, dtype=np.uint32)
    _call("rng_mwc_multipliers", first, count, out.ctypes.data)
    return out


# ---------------------------------------------------------------- Ising
def ising_create(L: int, beta: float, layout: int = ISING_INT8, rng_kind: int = RNG_XORWOW, rng_flags: int = 0,
                 seed: int = 0, G: int = 2, stream=None) -> int:
    h = ctypes.c_void_p()
    _call("ising_create", ctypes.byref(h), L, float(beta), layout, rng_kind, rng_flags, seed & (2**64 - 1), G,
          _stream(stream))
    return h.value


def ising_destroy(h: int) -> None:
    _call("ising_destroy", h)


def ising_sweep(h: int, n_sweeps: int, measure_every: int = 0, stream=None) -> None:
    _call("ising_sweep", h, n_sweeps, measure_every, _stream(stream))


def ising_sweep_plain(h: int, n_sweeps: int, measure_every: int = 0, stream=None) -> None:
    _call("ising_sweep_plain", h, n_sweeps, measure_every, _stream(stream))


def ising_sweep_multihit(h: int, n_rounds: int, k: int, n_strips: int, measure_every: int = 0,
                         stream=None) -> None:
    _call("ising_sweep_multihit", h, n_rounds, k, n_strips, measure_every, _stream(stream))


def _obs(name, h, *idx):
    E, M, nm = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_uint64()
    acc = (ctypes.c_int64 * 4)()
    _call(name, h, *idx, ctypes.byref(E), ctypes.byref(M), acc, ctypes.byref(nm))
    return {"E": E.value, "M": M.value, "acc": list(acc), "n_meas": nm.value}


def ising_observables(h: int) -> dict:
    return _obs("ising_observables", h)


def ising_info(h: int, idx: int = 0) -> dict:
    n, L, lay, k, sw = _u32(), _u32(), _i32(), _i32(), _u64()
    _call("ising_info", h, idx, ctypes.byref(n), ctypes.byref(L), ctypes.byref(lay), ctypes.byref(k),
          ctypes.byref(sw))
    return {"n_lattices": n.value, "L": L.value, "layout": lay.value, "kind": k.value, "sweeps": sw.value}


def ising_get_spins(h: int):
    import numpy as np
    L = ising_info(h)["L"]
    out = np.zeros((L, L), dtype=np.int8)
    _call("ising_get_spins", h, out.ctypes.data)
    return out


def ising_set_spins(h: int, spins) -> None:
    import numpy as np
    a = np.ascontiguousarray(spins, dtype=np.int8)
    _call("ising_set_spins", h, a.ctypes.data)


def ising_get_rng(h: int) -> int:
    r = ctypes.c_void_p()
    _call("ising_get_rng", h, ctypes.byref(r))
    return r.value


def ising_set_launch(h: int, threads: int = 0, ctas_per_sm: int = 0, min_sites_per_block: int = 0) -> None:
    _call("ising_set_launch", h, threads, ctas_per_sm, min_sites_per_block)


def ising_set_halo_depth(h: int, depth: int = 0) -> None:
    _call("ising_set_halo_depth", h, depth)


def ising_get_halo_depth(h: int) -> int:
    d = _u32()
    _call("ising_get_halo_depth", h, ctypes.byref(d))
    return d.value


def ising_autotune(h: int, probe_sweeps: int = 64) -> dict:
    t, c = _u32(), _i32()
    _call("ising_autotune", h, probe_sweeps, ctypes.byref(t), ctypes.byref(c))
    return {"threads": t.value, "ctas_per_sm": c.value}


def ising_get_launch(h: int) -> dict:
    t, c, m = _u32(), _i32(), _u32()
    _call("ising_get_launch", h, ctypes.byref(t), ctypes.byref(c), ctypes.byref(m))
    return {"threads": t.value, "ctas_per_sm": c.value, "min_sites": m.value}


AUTOTUNE_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "rng_gb300", "autotune.json")


def _device_name() -> str:
    import torch
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return f"{p.name}/{p.multi_processor_count}"


def _autotune_key(h: int, device: str) -> str:
    import hashlib
    n = ising_info(h, 0)["n_lattices"]
    sig = []
    for i in range(n):
        d = ising_info(h, i)
        sig.append((d["L"], d["layout"], d["kind"]))
    return hashlib.sha1(repr((device, sig)).encode()).hexdigest()


def ising_autotune_cached(h: int, probe_sweeps: int = 64, path: str | None = None, device: str | None = None) -> dict:
    """ising_autotune with a cache of tuned launch shapes (default
    ~/.cache/rng_gb300/autotune.json), keyed by the device and the handle's
    lattices (size, layout, generator kind of each): a hit sets the stored
    shape without timing anything.  Results never depend on the shape."""
    import json
    path = path or AUTOTUNE_CACHE
    key = _autotune_key(h, device or _device_name())
    cache = {}
    if os.path.exists(path):
        try:
            with open(path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
    if key in cache:
        c = cache[key]
        ising_set_launch(h, c["threads"], c["ctas_per_sm"], c["min_sites"])
        ising_set_halo_depth(h, c.get("halo_depth", 0))
        return dict(c, cached=True)
    ising_autotune(h, probe_sweeps)
    c = dict(ising_get_launch(h), halo_depth=ising_get_halo_depth(h))
    cache[key] = c
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1)
    os.replace(tmp, path)
    return dict(c, cached=False)


def ising_batch_create(L, beta, rng_kind, seed: int = 0, G: int = 2, stream=None) -> int:
    import numpy as np
    n = len(L)
    La = np.ascontiguousarray(L, dtype=np.uint32)
    Ba = np.ascontiguousarray(beta, dtype=np.float64)
    Ka = np.ascontiguousarray(rng_kind, dtype=np.int32)
    assert len(Ba) == n and len(Ka) == n
    h = ctypes.c_void_p()
    _call("ising_batch_create", ctypes.byref(h), n, La.ctypes.data, Ba.ctypes.data, Ka.ctypes.data,
          seed & (2**64 - 1), G, _stream(stream))
    return h.value


def ising_batch_sweep(h: int, n_sweeps: int, measure_every: int = 0, stream=None) -> None:
    _call("ising_batch_sweep", h, n_sweeps, measure_every, _stream(stream))


def ising_batch_observables(h: int, idx: int) -> dict:
    return _obs("ising_batch_observables", h, idx)


def ising_batch_get_spins(h: int, idx: int):
    import numpy as np
    L = ising_info(h, idx)["L"]
    out = np.zeros((L, L), dtype=np.int8)
    _call("ising_batch_get_spins", h, idx, out.ctypes.data)
    return out


def ising_debug_mute_strip(h: int, strip: int, wait_budget_ns: int = 0) -> None:
    _call("ising_debug_mute_strip", h, strip, wait_budget_ns)


def rng_debug_bounds_status(reset: bool = False) -> int:
    """The first out-of-range access recorded by the bounds-check build
    (file code * 10000 + line; 0: none).  Raises RngError with
    RNG_EUNSUPPORTED on a library built without the checks."""
    site = _i32()
    _call("rng_debug_bounds_status", ctypes.byref(site), int(reset))
    return site.value


def ising_plan_info(h: int) -> dict:
    g, b, s, t = _u32(), _u32(), _u32(), _u32()
    _call("ising_plan_info", h, ctypes.byref(g), ctypes.byref(b), ctypes.byref(s), ctypes.byref(t))
    return {"groups": g.value, "blocks": b.value, "strips": s.value, "threads": t.value}


# -------------------------------------------------------------- serving
RNG_REQ_DRAW, RNG_REQ_SWEEP = 0, 1
RNG_OUT_U32, RNG_OUT_F32, RNG_OUT_NORMAL = 0, 1, 2


class rng_request_t(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int32), ("kind", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("offset", ctypes.c_uint64), ("count", ctypes.c_uint64), ("out", ctypes.c_int32),
                ("L", ctypes.c_uint32), ("beta", ctypes.c_double), ("sweeps", ctypes.c_uint64)]


class rng_result_t(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("done", ctypes.c_int32), ("bytes", ctypes.c_uint64),
                ("t_submit_ns", ctypes.c_uint64), ("t_start_ns", ctypes.c_uint64), ("t_done_ns", ctypes.c_uint64),
                ("E", ctypes.c_int64), ("M", ctypes.c_int64)]


def rng_server_create(n_sets: int = 512, instances_per_set: int = 4096, n_slots: int = 8,
                      mem_budget_bytes: int = 8 << 30) -> int:
    h = ctypes.c_void_p()
    _call("rng_server_create", ctypes.byref(h), n_sets, instances_per_set, n_slots, mem_budget_bytes)
    return h.value


def rng_server_submit(srv: int, req: rng_request_t) -> int:
    t = _u64()
    _call("rng_server_submit", srv, ctypes.byref(req), ctypes.byref(t))
    return t.value


def rng_server_wait(srv: int, ticket: int, timeout_s: float = -1.0) -> rng_result_t:
    res = rng_result_t()
    _call("rng_server_wait", srv, ticket, timeout_s, ctypes.byref(res))
    return res


def rng_server_fetch(srv: int, ticket: int, host_dst: int | None, nbytes: int) -> None:
    _call("rng_server_fetch", srv, ticket, host_dst, nbytes)


def rng_server_stats(srv: int) -> dict:
    a, b, c, d = _u64(), _u64(), _u64(), _u32()
    _call("rng_server_stats", srv, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d))
    return {"submitted": a.value, "completed": b.value, "mem_in_use": c.value, "max_concurrent": d.value}


def rng_server_destroy(srv: int) -> None:
    _call("rng_server_destroy", srv)
