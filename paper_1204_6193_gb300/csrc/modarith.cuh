// modarith.cuh -- 64-bit modular arithmetic on the device (Montgomery form,
// R = 2^64) for the multiply-with-carry generator: the multiplier search
// (Miller-Rabin on a 2^32 - 1 and a 2^31 - 1) and skip-ahead
// (v <- v a^t mod a 2^32 - 1).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace rngx {

struct Mont {
    uint64_t p;      // odd modulus
    uint64_t pinv;   // -p^(-1) mod 2^64
    uint64_t r1;     // R mod p (Montgomery one)
    uint64_t r2;     // R^2 mod p
};

__host__ __device__ inline uint64_t add_mod(uint64_t a, uint64_t b, uint64_t p)
{
    // a, b < p < 2^64
    const uint64_t s = a + b;
    return (s < a || s >= p) ? s - p : s;
}

__device__ __forceinline__ Mont mont_setup(uint64_t p)
{
    Mont m;
    m.p = p;
    uint64_t inv = p;  // p * p = 1 (mod 8): 3 bits correct; Newton doubles
    for (int i = 0; i < 5; i++) inv *= 2 - p * inv;
    m.pinv = 0 - inv;
    // 2^64 mod p: for p > 2^61, 2^64 - p is below 8p, so a few subtractions
    // replace the (slow, emulated) 64-bit remainder
    uint64_t r1 = 0 - p;
    if (p > (1ull << 61)) {
        while (r1 >= p) r1 -= p;
    } else {
        r1 %= p;
    }
    m.r1 = r1;
    uint64_t r = m.r1;
    for (int i = 0; i < 64; i++) r = add_mod(r, r, p);  // r1 * 2^64 mod p
    m.r2 = r;
    return m;
}

// a * b * R^(-1) mod p for a, b < p.
__device__ __forceinline__ uint64_t mont_mul(uint64_t a, uint64_t b, const Mont &m)
{
    const uint64_t lo = a * b, hi = __umul64hi(a, b);
    const uint64_t q = lo * m.pinv;
    const uint64_t qlo_hi = __umul64hi(q, m.p);
    // lo + q p = 0 (mod 2^64): a carry leaves the low word iff lo != 0
    const uint64_t carry = lo != 0;
    uint64_t s = hi + qlo_hi;
    bool ovf = s < hi;
    const uint64_t s2 = s + carry;
    ovf |= s2 < s;
    return (ovf || s2 >= m.p) ? s2 - m.p : s2;
}

__device__ __forceinline__ uint64_t to_mont(uint64_t a, const Mont &m)
{
    return mont_mul(a < m.p ? a : a % m.p, m.r2, m);
}
__device__ __forceinline__ uint64_t from_mont(uint64_t a, const Mont &m) { return mont_mul(a, 1, m); }

// base^e in Montgomery form (base given in Montgomery form)
__device__ __forceinline__ uint64_t mont_pow(uint64_t bm, uint64_t e, const Mont &m)
{
    uint64_t r = m.r1;
    while (e) {
        if (e & 1) r = mont_mul(r, bm, m);
        bm = mont_mul(bm, bm, m);
        e >>= 1;
    }
    return r;
}

// Miller-Rabin for an odd n > 37 with the twelve prime bases 2..37, which
// decide primality of every n < 2^64 exactly.
__device__ inline bool is_prime_odd64(uint64_t n)
{
    const Mont m = mont_setup(n);
    uint64_t d = n - 1;
    int s = 0;
    while (!(d & 1)) {
        d >>= 1;
        s++;
    }
    const uint64_t one = m.r1, minus_one = n - m.r1;
    const uint32_t bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    for (int b = 0; b < 12; b++) {
        uint64_t x = mont_pow(to_mont(bases[b], m), d, m);
        if (x == one || x == minus_one) continue;
        bool comp = true;
        for (int r = 1; r < s; r++) {
            x = mont_mul(x, x, m);
            if (x == minus_one) {
                comp = false;
                break;
            }
        }
        if (comp) return false;
    }
    return true;
}

}  // namespace rngx
