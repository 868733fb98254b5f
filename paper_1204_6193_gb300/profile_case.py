"""Runs one generation kernel configuration a few times, or one persistent
Ising launch, for profiling a single kernel under a profiler on a small case.

    python -m paper_1204_6193_gb300.profile_case --kind xs1024w --form u32 --n 262144 --K 256 --reps 3
    python -m paper_1204_6193_gb300.profile_case --kind xorwow --ising 1024 --sweeps 200
    python -m paper_1204_6193_gb300.profile_case --kind xorwow --ising 1024 --sweeps 2 --hits 100 --strips 256
    python -m paper_1204_6193_gb300.profile_case --all --outputs 268435456

--all runs one call of every generator kind and form of the bulk workload
with its instance count (per-thread kinds 2^20 instances step-major,
block-shared kinds 2^15 generators instance-major, one per warp) and
--outputs / instances draws, in the order kinds x (u32, f32, normal, u32
XOR-reduced).
"""
import argparse

import torch

import paper_1204_6193_gb300 as R


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--kind", default="lcg32", choices=list(R.KIND_NAMES.values()))
    ap.add_argument("--form", default="u32", choices=["u32", "f32", "normal", "u32_xor"])
    ap.add_argument("--layout", default="step", choices=["step", "instance"])
    ap.add_argument("--n", type=int, default=1 << 18)
    ap.add_argument("--K", type=int, default=256)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--ising", type=int, default=0, help="lattice size L: one persistent Ising launch instead")
    ap.add_argument("--spins", default="int8", choices=["int8", "multispin"])
    ap.add_argument("--sweeps", type=int, default=200, help="sweeps (or multi-hit rounds)")
    ap.add_argument("--hits", type=int, default=0, help="k > 0: multi-hit rounds of k sweeps per strip phase")
    ap.add_argument("--strips", type=int, default=256, help="row strips of the multi-hit update")
    ap.add_argument("--launch", default="", help="threads,ctas_per_sm,min_sites_per_block of the Ising launch")
    ap.add_argument("--all", action="store_true", help="one call of every kind and form")
    ap.add_argument("--outputs", type=int, default=1 << 28, help="outputs per call with --all")
    a = ap.parse_args()
    if a.all:
        run_all(a.outputs)
        return
    kind = {v: k for k, v in R.KIND_NAMES.items()}[a.kind]
    if a.ising:
        layout = R.ISING_INT8 if a.spins == "int8" else R.ISING_MULTISPIN32
        h = R.ising_create(a.ising, 0.4406867935097715, layout, kind, 0, 12345, 2)
        if a.launch:
            R.ising_set_launch(h, *(int(v) for v in a.launch.split(",")))
        if a.hits:
            R.ising_sweep_multihit(h, a.sweeps, a.hits, a.strips)
        else:
            R.ising_sweep(h, a.sweeps)
        R.ising_observables(h)
        R.ising_destroy(h)
        print("ok")
        return
    layout = R.RNG_STEP_MAJOR if a.layout == "step" else R.RNG_INSTANCE_MAJOR
    h = R.rng_create(kind, a.n)
    R.rng_seed(h, 12345)
    out = torch.empty(a.n * (1 if a.form == "u32_xor" else a.K), dtype=torch.int32, device="cuda")
    for _ in range(a.reps):
        if a.form == "u32":
            R.rng_generate_u32(h, out.data_ptr(), a.K, layout)
        elif a.form == "f32":
            R.rng_generate_f32(h, out.data_ptr(), a.K, layout)
        elif a.form == "normal":
            R.rng_generate_normal(h, out.data_ptr(), a.K, layout)
        else:
            R.rng_generate_u32(h, out.data_ptr(), a.K, R.RNG_XOR_REDUCE)
    torch.cuda.synchronize()
    R.rng_destroy(h)
    print("ok")


def run_all(outputs: int) -> None:
    shared = {R.RNG_MT19937_SHARED, R.RNG_LFIB521, R.RNG_LFIB1279}
    out = torch.empty(outputs, dtype=torch.int32, device="cuda")
    for kind in sorted(R.KIND_NAMES):
        n = 1 << 15 if kind in shared else 1 << 20
        K = outputs // n
        layout = R.RNG_INSTANCE_MAJOR if kind in shared else R.RNG_STEP_MAJOR
        h = R.rng_create(kind, n)
        R.rng_seed(h, 12345)
        R.rng_generate_u32(h, out.data_ptr(), K, layout)
        R.rng_generate_f32(h, out.data_ptr(), K, layout)
        R.rng_generate_normal(h, out.data_ptr(), K, layout)
        R.rng_generate_u32(h, out.data_ptr(), K, R.RNG_XOR_REDUCE)
        torch.cuda.synchronize()
        R.rng_destroy(h)
    print("ok")


if __name__ == "__main__":
    main()
