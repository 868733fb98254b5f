"""Tiny and ragged cases of the generation and Ising kernels, run against
the CPU oracle with whatever build of the library RNG_GB300_LIBRARY names;
prints one JSON line: the cases run, those that disagreed with the oracle,
and the bounds-check build's first recorded out-of-range access (0: none).

Run by tests/test_gpu_bounds.py with the bounds-check build
(paper_1204_6193_gb300/build.py --bounds); needs a GPU."""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import torch  # noqa: E402

import oracle as O  # noqa: E402
import paper_1204_6193_gb300 as R  # noqa: E402

SEED = 0x0123456789ABCDEF
SHARED = (O.MT19937_SHARED, O.LFIB521, O.LFIB1279)


def generate(kind, n, K, out, layout):
    h = R.rng_create(kind, n)
    try:
        R.rng_seed(h, SEED)
        size = n if layout == R.RNG_XOR_REDUCE else n * K
        buf = torch.empty(size, dtype=torch.int32 if out == "u32" else torch.float32, device="cuda")
        {"u32": R.rng_generate_u32, "f32": R.rng_generate_f32, "normal": R.rng_generate_normal}[out](
            h, buf.data_ptr(), K, layout)
        torch.cuda.synchronize()
        return buf.cpu().numpy()
    finally:
        R.rng_destroy(h)


def gen_case(kind, n, K, out, layout):
    got = generate(kind, n, K, out, layout)
    ref = O.generate(kind, SEED, n, K)
    if out == "u32":
        want = ref
    elif out == "f32":
        want = O.to_f32(ref).astype(np.float32)
    else:
        want = O.box_muller(ref.reshape(-1)).reshape(n, K)
    if layout == R.RNG_XOR_REDUCE:
        if out == "normal":
            return bool(np.all(np.abs(got.astype(np.float64) - want.sum(1)) <= K * 2e-6 + 1e-5 * np.abs(want).sum(1)))
        bits = want.view(np.uint32) if out != "u32" else want
        return bool(np.array_equal(got.view(np.uint32), np.bitwise_xor.reduce(bits, axis=1)))
    got = got.reshape(K, n).T if layout == R.RNG_STEP_MAJOR else got.reshape(n, K)
    if out == "normal":
        return bool(np.abs(got.astype(np.float64) - want).max() <= 2e-6)
    return bool(np.array_equal(got.view(np.uint32), want.view(np.uint32)))


def ising_case(L, G, kind, layout, sweeps, hits=0, strips=0, launch=None, depth=0):
    h = R.ising_create(L, 0.4, layout, kind, 0, SEED, G)
    try:
        if launch:
            R.ising_set_launch(h, *launch)
        R.ising_set_halo_depth(h, depth)
        if hits:
            R.ising_sweep_multihit(h, sweeps, hits, strips, 1)
        else:
            R.ising_sweep(h, sweeps, 1)
        spins, obs = R.ising_get_spins(h), R.ising_observables(h)
    finally:
        R.ising_destroy(h)
    if hits:
        ref, acc, nm = O.ising_run_multihit(L, 0.4, kind, SEED, sweeps, k=hits, n_strips=strips, G=G, measure_every=1)
    else:
        ref, acc, nm = O.ising_run(L, 0.4, kind, SEED, sweeps, G=G, measure_every=1)
    return bool(np.array_equal(spins, ref) and obs["acc"] == acc.tolist() and obs["n_meas"] == nm)


def main():
    R.rng_debug_bounds_status(reset=True)
    cases, failed = 0, []
    for kind in range(10):
        shared = kind in SHARED
        sizes = [(4, 100), (3, 66)] if shared else [(33, 10), (64, 7), (100, 2)]
        if kind == O.XS1024W:
            # 2^20 instances select the one-thread-per-state forms of every output
            sizes = [(32, 10), (96, 6), (1 << 20, 2)]
        for n, K in sizes:
            for out in ("u32", "f32", "normal"):
                for layout in (R.RNG_STEP_MAJOR, R.RNG_INSTANCE_MAJOR, R.RNG_XOR_REDUCE):
                    if out == "normal" and K % 2:
                        continue
                    cases += 1
                    if not gen_case(kind, n, K, out, layout):
                        failed.append(f"gen kind={kind} n={n} K={K} {out} layout={layout}")
    for L, G, kind, layout in [(8, 2, O.XORWOW, 0), (16, 1, O.XS1024W, 0), (12, 3, O.LCG32, 0),
                               (64, 2, O.XORWOW, 1), (64, 2, O.PHILOX4X32_10, 0), (128, 2, O.MWC, 1),
                               (48, 4, O.LCG64, 0), (64, 2, O.MT19937_SHARED, 0), (64, 2, O.LFIB521, 1),
                               (32, 2, O.LFIB1279, 0)]:
        cases += 1
        if not ising_case(L, G, kind, layout, 12):
            failed.append(f"ising L={L} G={G} kind={kind} layout={layout}")
    # one strip per block of 1024 threads: roles split by warp with a polling
    # warp (halo depth 1), or a halo of two rows (depth 2)
    for L, G, kind, layout, depth in [(1024, 2, O.XORWOW, 0, 1), (768, 2, O.PHILOX4X32_10, 1, 1), (512, 1, O.LCG32, 0, 1),
                                      (1024, 2, O.XORWOW, 0, 2), (1024, 2, O.XS1024W, 1, 2), (768, 2, O.PHILOX4X32_10, 0, 2),
                                      (1024, 4, O.MWC, 1, 2)]:
        cases += 1
        if not ising_case(L, G, kind, layout, 6, launch=(1024, 1, 0), depth=depth):
            failed.append(f"one-strip ising L={L} G={G} kind={kind} layout={layout} depth={depth}")
    for L, kind, layout, hits, strips in [(64, O.XORWOW, 0, 3, 4), (64, O.XS1024W, 1, 2, 2), (128, O.LCG32, 0, 1, 8)]:
        cases += 1
        if not ising_case(L, 2, kind, layout, 4, hits, strips):
            failed.append(f"multihit L={L} kind={kind} layout={layout} k={hits} strips={strips}")
    site = R.rng_debug_bounds_status()
    print(json.dumps({"cases": cases, "failed": failed, "bounds_site": site}))


if __name__ == "__main__":
    main()
