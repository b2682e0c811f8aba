// Host build of the integer bit logic of the tensor-core digit scheme
// (paper_1808_10481_gb300/csrc/hl_tc_bits.cuh), so that it can be checked on the
// CPU against exact arithmetic (tests/test_tc_bits_host.py).  Every device
// intrinsic the header uses is a bit reinterpretation or a byte permutation;
// each has an exact host counterpart below.
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
static inline unsigned __float_as_uint(float f)
{
    unsigned u;
    std::memcpy(&u, &f, 4);
    return u;
}
// byte n of the result is byte (s >> 4n) & 7 of the 8-byte value {y:x}
static inline unsigned __byte_perm(unsigned x, unsigned y, unsigned s)
{
    const uint64_t v = ((uint64_t)y << 32) | x;
    unsigned r = 0;
    for (int n = 0; n < 4; ++n) r |= (unsigned)((v >> (8 * ((s >> (4 * n)) & 7))) & 0xFF) << (8 * n);
    return r;
}

#include "../paper_1808_10481_gb300/csrc/hl_tc_bits.cuh"

extern "C" {

void fixed_many(const double *v, const int *emax, long long *y, long n)
{
    for (long i = 0; i < n; ++i) y[i] = hl::t5_fixed(v[i], emax[i]);
}

// the six biased FP16 digit words of the pair (y[2i], y[2i+1]) -> w[6i .. 6i+5]
void digit_words_many(const long long *y, unsigned *w, long npairs)
{
    for (long i = 0; i < npairs; ++i) {
        uint32_t h[hl::kT5Digits];
        hl::t5_digit_words(y[2 * i], y[2 * i + 1], h);
        for (int j = 0; j < hl::kT5Digits; ++j) w[6 * i + j] = h[j];
    }
}

void scaled_many(const float *f, const int *k, double *out, long n)
{
    for (long i = 0; i < n; ++i) out[i] = hl::t5_scaled_f64(f[i], k[i]);
}

}  // extern "C"
