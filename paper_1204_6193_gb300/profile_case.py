"""Runs one generation kernel configuration a few times, for profiling a
single kernel under a profiler on a small case.

    python -m paper_1204_6193_gb300.profile_case --kind xs1024w --form u32 --n 262144 --K 256 --reps 3
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
    a = ap.parse_args()
    kind = {v: k for k, v in R.KIND_NAMES.items()}[a.kind]
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


if __name__ == "__main__":
    main()
