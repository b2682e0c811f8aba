// Host double-double arithmetic for building operator tables (host code only).
#pragma once

#include <cmath>
#include <cstdint>

namespace hl {

// Double-double arithmetic (a value is hi + lo with |lo| <= ulp(hi)/2), built
// from the error-free transformations TwoSum (Knuth) and TwoProduct via fma
// (Dekker), so the composed operator carries ~106-bit accuracy before its
// single final rounding to binary64.  Composing W*H directly in binary64
// leaves entry errors up to 1e-13 relative (heavy cancellation), which act as
// a systematic perturbation of the scheme and grow with the step count.
struct DD {
    double hi, lo;
};

static inline DD dd(double x) { return {x, 0.0}; }

static inline DD two_sum(double a, double b)
{
    const double s = a + b;
    const double bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}

static inline DD fast_two_sum(double a, double b)
{
    const double s = a + b;
    return {s, b - (s - a)};
}

static inline DD dd_add(DD a, DD b)
{
    const DD s = two_sum(a.hi, b.hi);
    const DD t = two_sum(a.lo, b.lo);
    DD r = fast_two_sum(s.hi, s.lo + t.hi);
    return fast_two_sum(r.hi, r.lo + t.lo);
}

static inline DD dd_neg(DD a) { return {-a.hi, -a.lo}; }

static inline DD dd_mul(DD a, DD b)
{
    const double p = a.hi * b.hi;
    const double e = std::fma(a.hi, b.hi, -p);
    return fast_two_sum(p, e + (a.hi * b.lo + a.lo * b.hi));
}

static inline DD dd_div(DD a, DD b)
{
    const double q1 = a.hi / b.hi;
    const DD r = dd_add(a, dd_neg(dd_mul(dd(q1), b)));
    const double q2 = r.hi / b.hi;
    const DD r2 = dd_add(r, dd_neg(dd_mul(dd(q2), b)));
    const double q3 = r2.hi / b.hi;
    return dd_add(fast_two_sum(q1, q2), dd(q3));
}

static inline DD dd_int(int64_t v)
{
    const double hi = (double)v;
    return {hi, (double)(v - (int64_t)hi)};
}

static inline int64_t ifact(int n)
{
    int64_t f = 1;
    for (int k = 2; k <= n; ++k) f *= k;
    return f;
}

static inline int64_t ibinom(int a, int l) { return ifact(a) / (ifact(l) * ifact(a - l)); }

}  // namespace hl
