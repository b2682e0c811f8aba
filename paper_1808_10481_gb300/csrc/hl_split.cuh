// binary64 <-> binary32 conversions built from integer operations.
//
// On this part the hardware double<->float conversions issue on the FP64
// pipe (2 per SM per clock), which would make them the bottleneck of the
// FP32-pipe kernels; these bit-level versions run on the integer pipe.
//
//   split_f64(x)  -> (hi, lo): hi = x rounded to nearest-even binary32,
//                    lo = (x - hi) truncated to 24 significant bits, so
//                    |x - hi - lo| <= 2^-47 |x|.  Values below 2^-126 in
//                    magnitude (and remainders below that) flush to zero;
//                    Inf/NaN map to Inf/NaN with lo = 0.
//   f32_to_f64(f) -> the exact binary64 value of a normal or zero binary32
//                    (subnormals flush to zero, Inf/NaN preserved).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace hl {

struct FF {
    float hi, lo;
};

__device__ __forceinline__ FF split_f64(double x)
{
    const unsigned hw = (unsigned)__double2hiint(x);
    const unsigned lw = (unsigned)__double2loint(x);
    const unsigned sgn = hw & 0x80000000u;
    const int ex = (int)((hw >> 20) & 0x7FFu);
    FF out;
    if (ex == 0x7FF) {  // Inf / NaN
        const bool nan = ((hw & 0xFFFFFu) | lw) != 0u;
        out.hi = __uint_as_float(sgn | (nan ? 0x7FC00000u : 0x7F800000u));
        out.lo = 0.f;
        return out;
    }
    const int e = ex - 1023;
    if (ex == 0 || e < -126) {  // zero, subnormal or below binary32's normal range
        out.hi = __uint_as_float(sgn);
        out.lo = 0.f;
        return out;
    }
    unsigned mhi = ((hw & 0xFFFFFu) << 3) | (lw >> 29);  // top 23 mantissa bits
    const unsigned r = lw & 0x1FFFFFFFu;                  // the 29 bits below them
    const bool up = (r > 0x10000000u) || (r == 0x10000000u && (mhi & 1u));
    int eh = e;
    if (up) {
        mhi += 1u;
        if (mhi == 0x800000u) {
            mhi = 0u;
            eh += 1;
        }
    }
    if (eh > 127) {
        out.hi = __uint_as_float(sgn | 0x7F800000u);
        out.lo = 0.f;
        return out;
    }
    out.hi = __uint_as_float(sgn | ((unsigned)(eh + 127) << 23) | mhi);
    // remainder x - hi in units of 2^(e-52), |rem| <= 2^28
    const int rem = up ? (int)r - 0x20000000 : (int)r;
    if (rem == 0) {
        out.lo = 0.f;
        return out;
    }
    const unsigned a = (unsigned)(rem < 0 ? -rem : rem);
    const int p = 31 - __clz((int)a);  // leading bit, p <= 28
    const int E = e - 52 + p;
    if (E < -126) {
        out.lo = 0.f;
        return out;
    }
    const unsigned m = (p >= 23 ? (a >> (p - 23)) : (a << (23 - p))) & 0x7FFFFFu;
    const unsigned lsgn = sgn ^ (rem < 0 ? 0x80000000u : 0u);
    out.lo = __uint_as_float(lsgn | ((unsigned)(E + 127) << 23) | m);
    return out;
}

__device__ __forceinline__ double f32_to_f64(float f)
{
    const unsigned b = __float_as_uint(f);
    const unsigned sgn = b & 0x80000000u;
    const unsigned e8 = (b >> 23) & 0xFFu;
    const unsigned m = b & 0x7FFFFFu;
    if (e8 == 0u) return __hiloint2double((int)sgn, 0);
    const unsigned eh = e8 == 0xFFu ? 0x7FFu : e8 + 896u;  // rebias 127 -> 1023
    return __hiloint2double((int)(sgn | (eh << 20) | (m >> 3)), (int)(m << 29));
}

// ---------------------------------------------------------------------------
// float-float (double-single) arithmetic with the error-free transformations
// TwoSum (Knuth) and TwoProduct through fma (Dekker); the _rn intrinsics keep
// the compiler from contracting or reassociating them.
__device__ __forceinline__ FF ff_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ FF ff_fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ FF ff_add(FF a, FF b)
{
    FF s = ff_two_sum(a.hi, b.hi);
    s.lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return ff_fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ FF ff_sub(FF a, FF b) { return ff_add(a, FF{-b.hi, -b.lo}); }

// acc += c * x, accumulated unnormalised (acc.lo collects every rounding error)
__device__ __forceinline__ void ff_fma(FF &acc, FF c, FF x)
{
    const float p = __fmul_rn(c.hi, x.hi);
    float e = __fmaf_rn(c.hi, x.hi, -p);
    e = __fmaf_rn(c.hi, x.lo, __fmaf_rn(c.lo, x.hi, e));
    const FF s = ff_two_sum(acc.hi, p);
    acc.hi = s.hi;
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(s.lo, e));
}

}  // namespace hl
