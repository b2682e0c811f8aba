// Double-double numbers for the oracle's double-double build (C++ only).
//
// A value is hi + lo with |lo| <= ulp(hi)/2, about 106 significant bits,
// carried by IEEE binary64 operations and the error-free transformations
// TwoSum (Knuth) and TwoProduct through fma (Dekker), so every platform gives
// the same bits.  Only what the oracle uses is provided.  TEST INFRASTRUCTURE.
#pragma once

#include <cmath>

struct orc_dd {
    double hi, lo;
    orc_dd() = default;
    orc_dd(double x) : hi(x), lo(0.0) {}
    orc_dd(int x) : hi((double)x), lo(0.0) {}
    orc_dd(long x) : hi((double)x), lo((double)(x - (long)(double)x)) {}
    orc_dd(long long x) : hi((double)x), lo((double)(x - (long long)(double)x)) {}
    static orc_dd make(double h, double l)
    {
        orc_dd r;
        r.hi = h;
        r.lo = l;
        return r;
    }
};

static inline orc_dd orc_two_sum(double a, double b)
{
    const double s = a + b;
    const double bb = s - a;
    return orc_dd::make(s, (a - (s - bb)) + (b - bb));
}

static inline orc_dd orc_fast_two_sum(double a, double b)
{
    const double s = a + b;
    return orc_dd::make(s, b - (s - a));
}

static inline orc_dd operator+(orc_dd a, orc_dd b)
{
    const orc_dd s = orc_two_sum(a.hi, b.hi);
    const orc_dd t = orc_two_sum(a.lo, b.lo);
    const orc_dd r = orc_fast_two_sum(s.hi, s.lo + t.hi);
    return orc_fast_two_sum(r.hi, r.lo + t.lo);
}

static inline orc_dd operator-(orc_dd a) { return orc_dd::make(-a.hi, -a.lo); }
static inline orc_dd operator-(orc_dd a, orc_dd b) { return a + (-b); }

static inline orc_dd operator*(orc_dd a, orc_dd b)
{
    const double p = a.hi * b.hi;
    const double e = std::fma(a.hi, b.hi, -p);
    return orc_fast_two_sum(p, e + (a.hi * b.lo + a.lo * b.hi));
}

static inline orc_dd operator/(orc_dd a, orc_dd b)
{
    const double q1 = a.hi / b.hi;
    const orc_dd r = a - orc_dd(q1) * b;
    const double q2 = r.hi / b.hi;
    const orc_dd r2 = r - orc_dd(q2) * b;
    const double q3 = r2.hi / b.hi;
    return orc_fast_two_sum(q1, q2) + orc_dd(q3);
}

static inline orc_dd &operator+=(orc_dd &a, orc_dd b) { return a = a + b; }
static inline orc_dd &operator-=(orc_dd &a, orc_dd b) { return a = a - b; }
static inline orc_dd &operator*=(orc_dd &a, orc_dd b) { return a = a * b; }

// x^e for a non-negative integer exponent e (the only powers the oracle takes)
static inline orc_dd orc_dd_pow(orc_dd x, orc_dd e)
{
    const int n = (int)e.hi;
    orc_dd r(1.0);
    for (int k = 0; k < n; ++k) r = r * x;
    return r;
}

// exp and floor are used only by the point source's Gaussian and wavelet.
// exp to double-double accuracy by argument reduction: x = k ln2 + r with
// |r| <= ln2/2, exp(r) = (exp(r / 2^4))^(2^4), the inner exponential by its
// Taylor series (|r / 2^4| < 0.022, so 18 terms reach 1e-45), then four
// squarings (each doubles the relative error) and an exact scaling by 2^k.
// ln2 is carried as a double-double.
static inline orc_dd orc_dd_exp(orc_dd x)
{
    if (x.hi < -708.0) return orc_dd(0.0);
    const orc_dd ln2 = orc_dd::make(0.6931471805599453094, 2.319046813846299558e-17);
    const double k = std::nearbyint(x.hi / ln2.hi);
    orc_dd r = x - orc_dd(k) * ln2;
    r = orc_dd::make(std::ldexp(r.hi, -4), std::ldexp(r.lo, -4));
    orc_dd term(1.0), sum(1.0);
    for (int n = 1; n <= 18; ++n) {
        term = term * r / orc_dd((double)n);
        sum = sum + term;
    }
    for (int i = 0; i < 4; ++i) sum = sum * sum;
    return orc_dd::make(std::ldexp(sum.hi, (int)k), std::ldexp(sum.lo, (int)k));
}

static inline orc_dd orc_dd_floor(orc_dd x)
{
    double f = std::floor(x.hi);
    if (f == x.hi && x.lo < 0.0) f -= 1.0;
    return orc_dd(f);
}
