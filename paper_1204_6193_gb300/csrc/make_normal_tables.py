#!/usr/bin/env python3
"""Writes normal_tables.h: the two lookup tables of the library's Box-Muller
transform (the normal deviates of rng_generate_normal).

    python paper_1204_6193_gb300/csrc/make_normal_tables.py

The transform maps a pair (r0, r1) of 32-bit draws to
    u1 = m 2^-24, m = (r0 >> 8) + 1 in [1, 2^24];   u2 = (r1 >> 8) 2^-24,
    z0 = sqrt(-2 ln u1) cos(2 pi u2),  z1 = sqrt(-2 ln u1) sin(2 pi u2).

Logarithm.  float(m) is exact.  Its exponent e (0..24) and the 5 mantissa
bits below the leading one select entry (e, i) of LN_TABLE, covering
f = float(m) in [2^e (1 + i/32), 2^e (1 + (i+1)/32)).  An entry holds
c = 2^-24 / u_mid rounded to float (u_mid = the interval's midpoint as a
value of u1) and L = 2 ln(1 / u_mid') where u_mid' = 2^-24 / c is the
point c actually inverts; then
    f c = 1 + d (d exact up to one rounding: one fused multiply-add),
    -2 ln u1 = L - 2 ln(1 + d),  |d| <= 2^-6,
and -2 ln(1 + d) = d (-2 + d (1 - 2d/3)) + O(d^4) (Taylor; the dropped
term, d^4 / 2, is below 3e-8).  The interval just below u1 = 1 and the point u1 = 1
take c = 2^-24 exactly and L = 0, so that d = u1 - 1 is exact there and
-2 ln u1 keeps its relative accuracy as u1 -> 1; L = 2^-100 at u1 = 1, so
that the radius stays positive and its reciprocal square root finite.

Sine and cosine.  u2's top 9 bits, rounded (the index j of the nearest
multiple of 2^-9 turn), select SC_TABLE[j] = (cos 2 pi j/512, sin 2 pi
j/512); the signed residual b = 2 pi (u2 - j/512), |b| <= pi/512, enters by
the angle-addition formulas with cos b = 1 - b^2/2 and sin b = b (the
dropped terms, b^4/24 and b^3/6, are below 6e-11 and 4e-8).

The two tables take 10.5 KB, small enough to sit in every block's shared
memory beside the generators' own arrays.  A float32 emulation of the
device arithmetic over every value of each input word, and the GPU tests
over the same inputs, put the largest deviation from the double-precision
transform near 9e-7 (bound 2e-6).

All values are computed in double precision here and rounded to float.
"""
import math
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LN_BITS = 5          # mantissa bits of the logarithm's table index
SC_BITS = 9          # bits of u2 in the sine/cosine table index
LN_EXPONENTS = 25    # float(m) has exponent 0 .. 24


def f32(x: float) -> float:
    import struct
    return struct.unpack("<f", struct.pack("<f", x))[0]


def ln_table():
    """[(c, L)] for entries (e, i), index e * 2^LN_BITS + i."""
    out = []
    for e in range(LN_EXPONENTS):
        for i in range(1 << LN_BITS):
            if (e == 23 and i == (1 << LN_BITS) - 1) or e == 24:
                # u1 in [1 - 2^-6, 1) and u1 = 1: d = u1 - 1 exactly
                out.append((2.0**-24, 2.0**-100 if e == 24 else 0.0))
                continue
            f_mid = 2.0**e * (1.0 + (i + 0.5) / (1 << LN_BITS))
            c = f32(1.0 / f_mid)
            u_inv = c * 2.0**24           # 1 / u' for the point u' that c inverts exactly
            out.append((c, f32(2.0 * math.log(u_inv))))
    return out


def sc_table():
    n = 1 << SC_BITS
    return [(f32(math.cos(2 * math.pi * j / n)), f32(math.sin(2 * math.pi * j / n))) for j in range(n)]


def hexf(x: float) -> str:
    return f"{float(x).hex()}f"


def main():
    ln = ln_table()
    sc = sc_table()
    lines = [
        "// normal_tables.h -- written by make_normal_tables.py (do not edit): the",
        "// lookup tables of the library's Box-Muller transform.",
        f"// LN_TABLE[e * {1 << LN_BITS} + i] = (c, L) for float(m) in [2^e (1 + i/{1 << LN_BITS}), 2^e (1 + (i+1)/{1 << LN_BITS})):",
        "//   -2 ln(m 2^-24) = L - 2 ln(1 + d), d = float(m) c - 1.",
        f"// SC_TABLE[j] = (cos, sin) of 2 pi j / {1 << SC_BITS}.",
        "#pragma once",
        "",
        "namespace rngx {",
        "",
        f"constexpr int kLnTableBits = {LN_BITS};",
        f"constexpr int kLnTableLen = {len(ln)};",
        f"constexpr int kScTableBits = {SC_BITS};",
        f"constexpr int kScTableLen = {len(sc)};",
        "",
        f"__device__ __align__(16) const float2 kLnTable[{len(ln)}] = {{",
    ]
    for k in range(0, len(ln), 4):
        lines.append("    " + " ".join(f"{{{hexf(c)}, {hexf(L)}}}," for c, L in ln[k:k + 4]))
    lines += ["};", "", f"__device__ __align__(16) const float2 kScTable[{len(sc)}] = {{"]
    for k in range(0, len(sc), 4):
        lines.append("    " + " ".join(f"{{{hexf(c)}, {hexf(s)}}}," for c, s in sc[k:k + 4]))
    lines += ["};", "", "}  // namespace rngx", ""]
    with open(os.path.join(HERE, "normal_tables.h"), "w") as f:
        f.write("\n".join(lines))


if __name__ == "__main__":
    main()
