// normal_poly.h -- written by fit_normal_poly.py (do not edit): polynomial
// coefficients of the Box-Muller transform, fitted by Lawson's algorithm.
// -2 ln(1+t) = t Q(t), t in [sqrt(1/2)-1, sqrt(2)-1]: max rel. error of Q 3.00e-08
// sin(2 pi x) = x S(x^2), x in [-1/8, 1/8]: max abs. error 1.21e-09
// cos(2 pi x) = C(x^2), x in [-1/8, 1/8]: max abs. error 2.76e-08
// (errors of the double-precision polynomials; coefficients of increasing degree)
#pragma once

namespace rngx {

constexpr int kLnQLen = 9;
__device__ constexpr float kLnQ[9] = {
    -0x1.0000000000000p+1f /* -2 */,
    0x1.fffffa0000000p-1f /* 0.999999821 */,
    -0x1.5556f40000000p-1f /* -0.666679025 */,
    0x1.00049a0000000p-1f /* 0.500035107 */,
    -0x1.98d2c00000000p-2f /* -0.399241447 */,
    0x1.535d340000000p-2f /* 0.331410229 */,
    -0x1.3185300000000p-2f /* -0.298359632 */,
    0x1.2504820000000p-2f /* 0.286150008 */,
    -0x1.65c6ee0000000p-3f /* -0.174695835 */,
};

constexpr int kSinSLen = 4;
__device__ constexpr float kSinS[4] = {
    0x1.921fb40000000p+2f /* 6.28318501 */,
    -0x1.4abba80000000p+5f /* -41.341629 */,
    0x1.465a3e0000000p+6f /* 81.5881271 */,
    -0x1.2cf5d40000000p+6f /* -75.2400665 */,
};

constexpr int kCosCLen = 4;
__device__ constexpr float kCosC[4] = {
    0x1.0000000000000p+0f /* 1 */,
    -0x1.3bd3920000000p+4f /* -19.7391529 */,
    0x1.03af5e0000000p+6f /* 64.921257 */,
    -0x1.4e5f080000000p+6f /* -83.592804 */,
};

}  // namespace rngx
