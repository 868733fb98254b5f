#!/usr/bin/env python3
"""Writes normal_poly.h: the polynomial coefficients of the library's
Box-Muller transform (the normal deviates of rng_generate_normal).

    python paper_1204_6193_gb300/csrc/fit_normal_poly.py

Method.  Each function is reduced to a short interval and approximated by a
polynomial whose coefficients are fitted here by Lawson's algorithm (C. L.
Lawson, 1961: iteratively reweighted least squares converging to the
minimax fit) on Chebyshev nodes, in double precision, then rounded to
float:

  -2 ln(1 + t) = t Q(t), t in [sqrt(1/2) - 1, sqrt(2) - 1] (after u =
      2^e (1 + t), the argument reduction of Cody and Waite, "Software
      Manual for the Elementary Functions", 1980), Q(t) = -2 + t R(t) with
      the constant term fixed at -2 and R fitted for relative error of Q
      (the factor -2 of the Box-Muller radius is folded in);
  sin(2 pi x) = x S(x^2), cos(2 pi x) = C(x^2), x in [-1/8, 1/8] (after
      removing the nearest multiple of 1/4 from u2, an exact step on its 24
      fraction bits), fitted for absolute error.

The printed bounds are those of the double-precision polynomials; the float
evaluation on the device adds its rounding, and the GPU tests check the
resulting deviates exhaustively over all 2^24 values of each input word
against the double-precision transform.
"""
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LN_DEG, SIN_DEG, COS_DEG = 7, 3, 3  # degrees of R(t), S(y), C(y)


def chebyshev_nodes(a, b, n=20000):
    k = np.arange(n)
    return (a + b) / 2 + (b - a) / 2 * np.cos(np.pi * (k + 0.5) / n)


def lawson(target, basis, xs, scale, iters=80):
    """Coefficients c minimising max |(sum c_j basis_j - target) / scale| over xs."""
    A = np.stack([bf(xs) for bf in basis], 1)
    y = target(xs)
    s = scale(xs)
    w = np.full(len(xs), 1.0 / len(xs))
    for _ in range(iters):
        W = np.sqrt(w) / s
        c, *_ = np.linalg.lstsq(A * W[:, None], y * W, rcond=None)
        err = np.abs(A @ c - y) / s
        w = w * err
        w /= w.sum()
    return c, float(err.max())


def fit():
    t = chebyshev_nodes(np.sqrt(0.5) - 1, np.sqrt(2) - 1)
    t = t[np.abs(t) > 1e-6]
    r_c, ln_e = lawson(lambda t: (-2 * np.log1p(t) / t + 2) / t,
                       [lambda t, k=k: t**k for k in range(LN_DEG + 1)], t,
                       lambda t: np.abs(2 * np.log1p(t) / t) / np.abs(t))
    ln_c = np.concatenate([[-2.0], r_c])
    x = chebyshev_nodes(0.0, 0.125)
    sin_c, sin_e = lawson(lambda x: np.sin(2 * np.pi * x) / x,
                          [lambda x, k=k: x**(2 * k) for k in range(SIN_DEG + 1)], x, lambda x: 1 / x)
    cos_c, cos_e = lawson(lambda x: np.cos(2 * np.pi * x),
                          [lambda x, k=k: x**(2 * k) for k in range(COS_DEG + 1)], x, lambda x: np.ones_like(x))
    return (ln_c, ln_e), (sin_c, sin_e), (cos_c, cos_e)


def as_float_literal(v):
    f = np.float32(v)
    return f"{float(f).hex()}f /* {float(f):.9g} */"


def main():
    (ln_c, ln_e), (sin_c, sin_e), (cos_c, cos_e) = fit()
    lines = [
        "// normal_poly.h -- written by fit_normal_poly.py (do not edit): polynomial",
        "// coefficients of the Box-Muller transform, fitted by Lawson's algorithm.",
        f"// -2 ln(1+t) = t Q(t), t in [sqrt(1/2)-1, sqrt(2)-1]: max rel. error of Q {ln_e:.2e}",
        f"// sin(2 pi x) = x S(x^2), x in [-1/8, 1/8]: max abs. error {sin_e:.2e}",
        f"// cos(2 pi x) = C(x^2), x in [-1/8, 1/8]: max abs. error {cos_e:.2e}",
        "// (errors of the double-precision polynomials; coefficients of increasing degree)",
        "#pragma once",
        "",
        "namespace rngx {",
        "",
    ]
    for name, c in (("kLnQ", ln_c), ("kSinS", sin_c), ("kCosC", cos_c)):
        lines.append(f"constexpr int {name}Len = {len(c)};")
        lines.append(f"__device__ constexpr float {name}[{len(c)}] = {{")
        lines += [f"    {as_float_literal(v)}," for v in c]
        lines.append("};")
        lines.append("")
    lines.append("}  // namespace rngx")
    with open(os.path.join(HERE, "normal_poly.h"), "w") as f:
        f.write("\n".join(lines) + "\n")
    print(f"-2 ln rel {ln_e:.2e}, sin abs {sin_e:.2e}, cos abs {cos_e:.2e}")


if __name__ == "__main__":
    main()
