// Host build of the device conversion and float-float helpers in
// paper_1808_10481_gb300/csrc/hl_split.cuh, so that their bit-level logic can
// be checked on the CPU against exact arithmetic (tests/test_split_host.py).
//
// The device intrinsics the header uses are bit reinterpretations and IEEE
// binary32 operations with round-to-nearest; each has an exact host
// counterpart below.  Build with -ffp-contract=off so that the compiler keeps
// every rounding the header asks for.
#include <cmath>
#include <cstdint>
#include <cstring>

static inline int __double2hiint(double x)
{
    uint64_t b;
    std::memcpy(&b, &x, 8);
    return (int)(uint32_t)(b >> 32);
}
static inline int __double2loint(double x)
{
    uint64_t b;
    std::memcpy(&b, &x, 8);
    return (int)(uint32_t)b;
}
static inline double __hiloint2double(int hi, int lo)
{
    const uint64_t b = ((uint64_t)(uint32_t)hi << 32) | (uint32_t)lo;
    double x;
    std::memcpy(&x, &b, 8);
    return x;
}
static inline float __uint_as_float(unsigned u)
{
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}
static inline unsigned __float_as_uint(float f)
{
    unsigned u;
    std::memcpy(&u, &f, 4);
    return u;
}
static inline int __clz(int x) { return x == 0 ? 32 : __builtin_clz((unsigned)x); }
static inline float __fadd_rn(float a, float b) { return a + b; }
static inline float __fsub_rn(float a, float b) { return a - b; }
static inline float __fmul_rn(float a, float b) { return a * b; }
static inline float __fmaf_rn(float a, float b, float c) { return std::fmaf(a, b, c); }

#include "../paper_1808_10481_gb300/csrc/hl_split.cuh"

extern "C" {

void split_many(const double *x, float *hi, float *lo, long n)
{
    for (long i = 0; i < n; ++i) {
        const hl::FF f = hl::split_f64(x[i]);
        hi[i] = f.hi;
        lo[i] = f.lo;
    }
}

void widen_many(const float *f, double *out, long n)
{
    for (long i = 0; i < n; ++i) out[i] = hl::f32_to_f64(f[i]);
}

void two_sum_many(const float *a, const float *b, float *s, float *e, long n)
{
    for (long i = 0; i < n; ++i) {
        const hl::FF r = hl::ff_two_sum(a[i], b[i]);
        s[i] = r.hi;
        e[i] = r.lo;
    }
}

// rows dot products of length k in float-float: out = sum_j c[j] * x[r][j]
void ff_dot_many(const float *c_hi, const float *c_lo, const float *x_hi, const float *x_lo, long rows, long k,
                 float *out_hi, float *out_lo)
{
    for (long r = 0; r < rows; ++r) {
        hl::FF acc{0.f, 0.f};
        for (long j = 0; j < k; ++j)
            hl::ff_fma(acc, hl::FF{c_hi[j], c_lo[j]}, hl::FF{x_hi[r * k + j], x_lo[r * k + j]});
        out_hi[r] = acc.hi;
        out_lo[r] = acc.lo;
    }
}

}  // extern "C"
