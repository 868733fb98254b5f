// normal_poly.h -- written by fit_normal_poly.py (do not edit): polynomial
// coefficients of the Box-Muller transform, fitted by Lawson's algorithm.
// ln(1+t) = t - t^2/2 + t^3 P(t), t in [sqrt(1/2)-1, sqrt(2)-1]: max rel. error 3.15e-08
// sin(2 pi x) = x S(x^2), x in [-1/8, 1/8]: max abs. error 1.21e-09
// cos(2 pi x) = C(x^2), x in [-1/8, 1/8]: max abs. error 2.76e-08
// (errors of the double-precision polynomials; coefficients of increasing degree)
#pragma once

namespace rngx {

constexpr int kLnPLen = 7;
__device__ constexpr float kLnP[7] = {
    0x1.5556d80000000p-2f /* 0.333339095 */,
    -0x1.0003820000000p-2f /* -0.250013381 */,
    0x1.98d7f20000000p-3f /* 0.199630633 */,
    -0x1.53824a0000000p-3f /* -0.16577585 */,
    0x1.3174640000000p-3f /* 0.149147779 */,
    -0x1.2432b00000000p-3f /* -0.142674804 */,
    0x1.645e3e0000000p-4f /* 0.0870039389 */,
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
