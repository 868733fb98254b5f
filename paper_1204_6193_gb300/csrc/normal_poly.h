// normal_poly.h -- written by fit_normal_poly.py (do not edit): polynomial
// coefficients of the Box-Muller transform, fitted by Lawson's algorithm.
// ln(1+t) = t - t^2/2 + t^3 P(t), t in [sqrt(1/2)-1, sqrt(2)-1]: max rel. error 5.83e-09
// sin(2 pi x) = x S(x^2), x in [-1/8, 1/8]: max abs. error 1.21e-09
// cos(2 pi x) = C(x^2), x in [-1/8, 1/8]: max abs. error 4.74e-11
// (errors of the double-precision polynomials; coefficients of increasing degree)
#pragma once

namespace rngx {

constexpr int kLnPLen = 8;
__device__ constexpr float kLnP[8] = {
    0x1.5555540000000p-2f /* 0.333333313 */,
    -0x1.0002260000000p-2f /* -0.250008196 */,
    0x1.99a0080000000p-3f /* 0.200012267 */,
    -0x1.5472440000000p-3f /* -0.166233569 */,
    0x1.22da200000000p-3f /* 0.142017603 */,
    -0x1.0d854c0000000p-3f /* -0.1316019 */,
    0x1.055b580000000p-3f /* 0.127615631 */,
    -0x1.38b51e0000000p-4f /* -0.0763446018 */,
};

constexpr int kSinSLen = 4;
__device__ constexpr float kSinS[4] = {
    0x1.921fb40000000p+2f /* 6.28318501 */,
    -0x1.4abba80000000p+5f /* -41.341629 */,
    0x1.465a3e0000000p+6f /* 81.5881271 */,
    -0x1.2cf5d40000000p+6f /* -75.2400665 */,
};

constexpr int kCosCLen = 5;
__device__ constexpr float kCosC[5] = {
    0x1.0000000000000p+0f /* 1 */,
    -0x1.3bd3cc0000000p+4f /* -19.7392082 */,
    0x1.03c1dc0000000p+6f /* 64.9393158 */,
    -0x1.55c57c0000000p+6f /* -85.4428558 */,
    0x1.d9c3880000000p+5f /* 59.2204742 */,
};

}  // namespace rngx
