// Integer bit logic of the tensor-core split kernels' digit scheme (included by
// hl_tc5.cuh): the fixed-point form of a binary64 value at a block exponent, the
// byte permutations that place its base-256 digits under FP16 exponents, and
// the exact rescaling of an FP32 level sum back to binary64.  Integer operations
// and bit reinterpretations only, so the same code also builds for the host
// (tests/tc_bits_host.cpp checks it against exact arithmetic).
#pragma once

#include <stdint.h>

namespace hl {

constexpr int kT5Digits = 6;

// Fixed-point form of one binary64 value at the block exponent, with every byte
// below the top digit biased by 128 (emax is the largest biased exponent of the
// region, |v| < 2^(emax - 1022) = 2^E):  X = trunc(v 2^(48 - E)), |X| < 2^48,
// returned as y = X + 0x8080808080, so that byte k of y (k < 5) is d_(5-k) + 128
// and y >> 40 (arithmetic) is d_0 in [-256, 256].  Integer operations only.
__device__ __forceinline__ int64_t t5_fixed(double v, int emax)
{
    const uint32_t hi = (uint32_t)__double2hiint(v), lo = (uint32_t)__double2loint(v);
    const int e = (int)((hi >> 20) & 0x7FFu);
    const int sh = emax + 5 - e;  // >= 5 whenever e <= emax
    uint64_t mag = 0;
    if (e != 0 && e != 0x7FF && sh < 64) {
        const uint64_t m53 = ((uint64_t)((hi & 0xFFFFFu) | 0x100000u) << 32) | lo;
        mag = m53 >> sh;
    }
    const int64_t x = (hi >> 31) ? -(int64_t)mag : (int64_t)mag;
    return x + 0x8080808080ll;
}

// Digit words of two biased fixed-point values a and b (adjacent slots): h[i]
// holds digit i of a (low half) and of b (high half) as FP16 bit patterns of
// 1024 + 128 + d (i >= 1: byte 5 - i of y under the exponent of 2^10, placed by
// byte permutations) or 1024 + 512 + d (i = 0, d = y >> 40 in [-256, 256]);
// subtracting kT5SubLow or kT5SubTop (packed FP16, exact) leaves the digits.
constexpr uint32_t kT5SubLow = 0x64806480u;   // FP16 1152 in both halves
constexpr uint32_t kT5SubTop = 0x66006600u;   // FP16 1536 in both halves

__device__ __forceinline__ void t5_digit_words(int64_t a, int64_t b, uint32_t (&h)[kT5Digits])
{
    constexpr uint32_t kHi = 0x64646464u;
    const uint32_t alo = (uint32_t)a, blo = (uint32_t)b;
    const uint32_t ahi = (uint32_t)((uint64_t)a >> 32), bhi = (uint32_t)((uint64_t)b >> 32);
    const uint32_t P = __byte_perm(alo, blo, 0x5140);   // a.b0 b.b0 a.b1 b.b1
    const uint32_t Q = __byte_perm(alo, blo, 0x7362);   // a.b2 b.b2 a.b3 b.b3
    const uint32_t R = __byte_perm(ahi, bhi, 0x4040);   // a.b4 b.b4 (twice)
    h[5] = __byte_perm(P, kHi, 0x4140);
    h[4] = __byte_perm(P, kHi, 0x4342);
    h[3] = __byte_perm(Q, kHi, 0x4140);
    h[2] = __byte_perm(Q, kHi, 0x4342);
    h[1] = __byte_perm(R, kHi, 0x4140);
    const uint32_t ta = (uint32_t)(((int)ahi >> 8) + (512 + 0x6400));
    const uint32_t tb = (uint32_t)(((int)bhi >> 8) + (512 + 0x6400));
    h[0] = __byte_perm(ta, tb, 0x5410);
}

// exact f * 2^k as binary64 (f normal or zero; integer operations only)
__device__ __forceinline__ double t5_scaled_f64(float f, int k)
{
    const uint32_t b = __float_as_uint(f);
    if ((b & 0x7FFFFFFFu) == 0u) return 0.0;
    const int eh = (int)((b >> 23) & 0xFFu) + 896 + k;
    if (eh <= 0) return 0.0;
    const uint32_t m = b & 0x7FFFFFu;
    if (eh >= 2047) return __hiloint2double((int)((b & 0x80000000u) | 0x7FF00000u), 0);
    return __hiloint2double((int)((b & 0x80000000u) | ((uint32_t)eh << 20) | (m >> 3)), (int)(m << 29));
}

}  // namespace hl
