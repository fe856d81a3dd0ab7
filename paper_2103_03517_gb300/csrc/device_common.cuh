// device_common.cuh -- device primitives of libmc: counter-based RNG, the
// FP64 exponential of the Metropolis test, fast division, spin algebra.
#pragma once
#include <stdint.h>

#include "mc_internal.h"

namespace mcgb {

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of the 4x32
// S-box, multipliers 0xD2511F53 / 0xCD9E8D57, Weyl increments 0x9E3779B9 /
// 0xBB67AE85.  Counter = (site or pair, sweep, tag, draw), key = seed.
__device__ __forceinline__ uint4 philox(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = uint64_t(0xD2511F53u) * c.x, p1 = uint64_t(0xCD9E8D57u) * c.z;
        const uint32_t hi0 = uint32_t(p0 >> 32), lo0 = uint32_t(p0), hi1 = uint32_t(p1 >> 32), lo1 = uint32_t(p1);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// The round keys of philox(c, k0, k1) (the key before round r is k + r W),
// computed once for a lattice, and the same ten rounds taking them from
// registers: the same four words as philox(c, k0, k1).
struct PhiloxKeys {
    uint32_t a[10], b[10];
};

__device__ __forceinline__ PhiloxKeys philox_keys(uint32_t k0, uint32_t k1) {
    PhiloxKeys K;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        K.a[r] = k0;
        K.b[r] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return K;
}

__device__ __forceinline__ uint4 philox_rk(uint4 c, const PhiloxKeys& K) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = uint64_t(0xD2511F53u) * c.x, p1 = uint64_t(0xCD9E8D57u) * c.z;
        const uint32_t hi0 = uint32_t(p0 >> 32), lo0 = uint32_t(p0), hi1 = uint32_t(p1 >> 32), lo1 = uint32_t(p1);
        c = make_uint4(hi1 ^ c.y ^ K.a[r], lo1, hi0 ^ c.w ^ K.b[r], lo0);
    }
    return c;
}

// The same ten rounds with the round keys read from shared memory (rk[r] =
// the key pair before round r, written once per lattice by the warp).
__device__ __forceinline__ uint4 philox_smem(uint4 c, const uint2* rk) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint2 k = rk[r];
        const uint64_t p0 = uint64_t(0xD2511F53u) * c.x, p1 = uint64_t(0xCD9E8D57u) * c.z;
        const uint32_t hi0 = uint32_t(p0 >> 32), lo0 = uint32_t(p0), hi1 = uint32_t(p1 >> 32), lo1 = uint32_t(p1);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

// Philox stream tags: bit 0 = colour, bits 1.. = purpose.
enum { kPurposeMove = 0, kPurposePair = 1, kPurposePerm = 2 };
__device__ __forceinline__ uint32_t tag_of(int colour, int purpose) {
    return uint32_t(colour) | (uint32_t(purpose) << 1);
}

__device__ __forceinline__ uint32_t fast_div(uint32_t n, const FastDiv& f) {
    const uint32_t t = __umulhi(n, f.mul);
    return (t + ((n - t) >> f.s1)) >> f.s2;
}

// exp(x) in FP64 with a fixed operation sequence, so that every IEEE
// machine returns the same bits: Cody-Waite reduction x = k ln2 + r with a
// 32-bit head of ln2, the degree-13 Taylor polynomial of e^r by Horner's
// rule (|r| <= ln2/2), and scaling by 2^k as two exact powers of two.
// Constants are the nearest doubles to ln2 (head/tail), 1/ln2 and 1/n!.
// Used for the Metropolis test of Eq. 1 in the FP64 mode.
__device__ __forceinline__ double pow2_bits(int k) {
    return __longlong_as_double((long long)(k + 1023) << 52);
}

__device__ inline double exp_fp64(double x) {
    if (x != x) return x;
    if (x < -746.0) return 0.0;
    if (x > 709.79) return __longlong_as_double(0x7FF0000000000000LL);
    const double kf = floor(x * 0x1.71547652b82fep+0 + 0.5);
    const int k = (int)kf;
    const double r = (x - kf * 0x1.62e42ff000000p-1) - kf * -0x1.718432a1b0e26p-35;
    double p = 0x1.6124613a86d09p-33;      // 1/13!
    p = p * r + 0x1.1eed8eff8d898p-29;     // 1/12!
    p = p * r + 0x1.ae64567f544e4p-26;     // 1/11!
    p = p * r + 0x1.27e4fb7789f5cp-22;     // 1/10!
    p = p * r + 0x1.71de3a556c734p-19;     // 1/9!
    p = p * r + 0x1.a01a01a01a01ap-16;     // 1/8!
    p = p * r + 0x1.a01a01a01a01ap-13;     // 1/7!
    p = p * r + 0x1.6c16c16c16c17p-10;     // 1/6!
    p = p * r + 0x1.1111111111111p-7;      // 1/5!
    p = p * r + 0x1.5555555555555p-5;      // 1/4!
    p = p * r + 0x1.5555555555555p-3;      // 1/3!
    p = p * r + 0x1.0000000000000p-1;      // 1/2!
    p = p * r + 1.0;                       // 1/1!
    p = p * r + 1.0;                       // 1/0!
    const int k1 = k / 2;
    const int k2 = k - k1;
    return (p * pow2_bits(k1)) * pow2_bits(k2);
}

template <typename R>
struct V3 {
    R x, y, z;
};

// Fixed-point conversion of a block partial sum (round to nearest).
__device__ __forceinline__ long long to_fix(double v) { return __double2ll_rn(v * kFixScale); }

}  // namespace mcgb
