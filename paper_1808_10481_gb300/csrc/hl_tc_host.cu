// Host side of the tensor-core split mode: the digit tables of the operator.
//
// The kernels contract the partner data at the 2^d = 4 cell vertices
// directly (no butterfly).  The vertex form of the fused operator follows
// from the butterfly form: the butterfly entry x[pat] weights vertex v by
// prod over axes k with v_k = 1 of (bit k of pat ? -1 : +1), so
//   W[c][v][l][s] = coef(c, l, s) * prod_{k: v_k = 1, pat_k = 1} (-1),
// pat = bfly_pattern(c, s, l), and zero where the structural-zero rule holds.
//
// Exact split (an Ozaki-type scheme): column n is scaled by 2^-e_n with
// max_k |W[k][n]| < 2^e_n, rounded to an integer of 46 bits, and written as
// kTcDigits balanced base-256 digits; digit j carries weight 2^(8 (5 - j)).
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "hl_fp64.cuh"
#include "hl_internal.h"

namespace hl {

static uint16_t bf16_of_small_int(int d)
{
    const float f = (float)d;  // |d| <= 128: 8 significant bits, exact in bfloat16
    uint32_t b;
    std::memcpy(&b, &f, sizeof b);
    return (uint16_t)(b >> 16);
}

// balanced base-256 digits of |X| < 2^46, most significant first
static void digits_of(int64_t X, int *d)
{
    for (int j = kTcDigits - 1; j >= 0; --j) {
        int64_t r = X & 255;
        if (r >= 128) r -= 256;
        d[j] = (int)r;
        X = (X - r) / 256;  // exact
    }
}

bool build_tc_tables(int m, const double *coef, std::vector<uint16_t> &digits, std::vector<int> &expo)
{
    if (m < 0 || m > 3) return false;
    const int D = 2, n = m + 1, NQ = n * n;
    digits.assign((size_t)kTcOps * kTcOpElems, 0);
    expo.assign((size_t)kTcOps * kTcN, 0);
    for (int op = 0; op < kTcOps; ++op) {
        // dense vertex-form operator W[k][s], k padded (16 slots per (component, vertex))
        std::vector<double> W((size_t)128 * kTcN, 0.0);
        const int ncomp = op == 0 ? D : 1;  // partner components: u (D) for the p-half, p for the u-half
        for (int c = 0; c < ncomp; ++c) {
            const int i = op == 0 ? c : op - 1;  // direction of the operator block
            for (int v = 0; v < 4; ++v)
                for (int l = 0; l < NQ; ++l)
                    for (int s = 0; s < NQ; ++s) {
                        if (!coef_nonzero(D, n, i, s, l)) continue;
                        const int pat = bfly_pattern(D, n, i, s, l);
                        const double sign = (__builtin_popcount(v & pat) & 1) ? -1.0 : 1.0;
                        W[(size_t)((c * 4 + v) * 16 + l) * kTcN + s] = sign * coef[coef_index(NQ, i, l, s)];
                    }
        }
        for (int s = 0; s < kTcN; ++s) {
            double mx = 0.0;
            for (int k = 0; k < 128; ++k) mx = std::fmax(mx, std::fabs(W[(size_t)k * kTcN + s]));
            int e = 0;
            if (mx > 0.0) std::frexp(mx, &e);  // mx < 2^e
            expo[(size_t)op * kTcN + s] = e;
            for (int k = 0; k < 128; ++k) {
                const double w = W[(size_t)k * kTcN + s];
                const int64_t X = (int64_t)std::llround(std::ldexp(w, 46 - e));
                int d[kTcDigits];
                digits_of(X, d);
                for (int j = 0; j < kTcDigits; ++j)
                    digits[(size_t)op * kTcOpElems + ((size_t)j * kTcN + s) * kTcKS + k] = bf16_of_small_int(d[j]);
            }
        }
    }
    return true;
}

// FP16 bit pattern of a small integer (|d| <= 256: at most 9 significant bits, exact)
static uint16_t f16_of_small_int(int d)
{
    if (d == 0) return 0;
    const uint16_t sign = d < 0 ? 0x8000u : 0u;
    unsigned a = (unsigned)(d < 0 ? -d : d);
    int e = 0;
    while ((a >> (e + 1)) != 0u) ++e;                       // a in [2^e, 2^(e+1))
    const unsigned mant = (a << (10 - e)) & 0x3FFu;
    return (uint16_t)(sign | (unsigned)((e + 15) << 10) | mant);
}

// the small integer of a BF16 digit of build_tc_tables
static int int_of_bf16(uint16_t b)
{
    const uint32_t bits = (uint32_t)b << 16;
    float f;
    std::memcpy(&f, &bits, sizeof f);
    return (int)f;
}

// Shared-memory operator images of the tcgen05 kernels (hl_tc5.cuh), one per
// half-step, each 14336 FP16: blocks kb of [2 K-chunks][7 NPL rows][8 slots]
// (the no-swizzle K-major layout of the MMA's B operand: 8 rows of 16 bytes
// per core matrix, row n of block kb at ((kb * 2 + chunk) * 7 NPL + n) * 8).
//   p-half: kb = velocity component * 4 + vertex, NPL = 16, row n = j * 16 + s;
//   u-half: kb = vertex, NPL = 32, row n = j * 32 + direction * 16 + s;
// digit rows j = 0..5 come from build_tc_tables, row block j = 6 is zero (it lets
// the first MMA of a tile initialise the accumulators of all seven levels).
bool build_tc5_images(int m, const double *coef, std::vector<uint16_t> &image, std::vector<int> &expo)
{
    std::vector<uint16_t> dig;
    if (!build_tc_tables(m, coef, dig, expo)) return false;
    image.assign((size_t)kTc5ImageElems, 0);
    auto digit = [&](int op, int j, int s, int k) -> uint16_t {
        return f16_of_small_int(int_of_bf16(dig[(size_t)op * kTcOpElems + ((size_t)j * kTcN + s) * kTcKS + k]));
    };
    // p-half
    for (int kb = 0; kb < 8; ++kb)
        for (int ch = 0; ch < 2; ++ch)
            for (int n = 0; n < 7 * 16; ++n)
                for (int kk = 0; kk < 8; ++kk) {
                    const int j = n / 16, s = n % 16, l = ch * 8 + kk;
                    image[(((size_t)kb * 2 + ch) * 112 + n) * 8 + kk] = j < kTcDigits ? digit(0, j, s, kb * 16 + l) : 0;
                }
    // u-half
    uint16_t *u = image.data() + kTc5ImageElems / 2;
    for (int kb = 0; kb < 4; ++kb)
        for (int ch = 0; ch < 2; ++ch)
            for (int n = 0; n < 7 * 32; ++n)
                for (int kk = 0; kk < 8; ++kk) {
                    const int j = n / 32, dir = (n / 16) % 2, s = n % 16, l = ch * 8 + kk;
                    u[(((size_t)kb * 2 + ch) * 224 + n) * 8 + kk] = j < kTcDigits ? digit(1 + dir, j, s, kb * 16 + l) : 0;
                }
    return true;
}

}  // namespace hl

namespace hl {

// 3D (m = 2) operator images of the tcgen05 kernels in hl_tc3.cu.  The vertex
// form of the fused operator: the increment of output slot s from partner slot
// l at vertex v (bit k of v = upper node along axis k) of partner component (or
// direction) i is sign(v, pattern(i, s, l)) coef(i, l, s), the butterfly of the
// FP64 kernels written out per vertex.  Operators: 0 the p-half (K = component
// x vertex x slot = 3 x 8 x 27), 1 + d the u-half's direction d (K = 8 x 27).
// Every column s is scaled by 2^-e_s (expo[op * 32 + s]) and cut into kTcDigits
// balanced base-256 digits (FP16 bit patterns of integers in [-128, 127]).
// Image of one half: 12 units u = (i * 2 + vz) * 2 + kh (i = component for the
// p-half, direction for the u-half; vz the vertex's z bit; kh the half of the
// 32 padded slots), each 4 vertex blocks (vx + 2 vy) of [2 K-chunks of 8 slots]
// [7 x 32 rows n = j * 32 + s][8 FP16]; digit row block j = 6 is zero.
bool build_tc3_images(int m, const double *coef, std::vector<uint16_t> &image, std::vector<int> &expo)
{
    if (m != 2) return false;
    constexpr int D = 3, n = 3, NQ = 27, NS = 32;
    image.assign((size_t)kTc3ImageElems, 0);
    expo.assign((size_t)4 * NS, 0);
    for (int op = 0; op < 4; ++op) {
        const int ncomp = op == 0 ? D : 1;
        const int K = ncomp * 8 * NS;
        // dense vertex-form operator W[k][s], k = (c * 8 + v) * 32 + l
        std::vector<double> W((size_t)K * NS, 0.0);
        for (int c = 0; c < ncomp; ++c) {
            const int i = op == 0 ? c : op - 1;
            for (int v = 0; v < 8; ++v)
                for (int l = 0; l < NQ; ++l)
                    for (int s = 0; s < NQ; ++s) {
                        if (!coef_nonzero(D, n, i, s, l)) continue;
                        const int pat = bfly_pattern(D, n, i, s, l);
                        const double sign = (__builtin_popcount(v & pat) & 1) ? -1.0 : 1.0;
                        W[(size_t)((c * 8 + v) * NS + l) * NS + s] = sign * coef[coef_index(NQ, i, l, s)];
                    }
        }
        std::vector<int> dig((size_t)K * NS * kTcDigits, 0);  // [k][s][j]
        for (int s = 0; s < NQ; ++s) {
            double mx = 0.0;
            for (int k = 0; k < K; ++k) mx = std::fmax(mx, std::fabs(W[(size_t)k * NS + s]));
            int e = 0;
            if (mx > 0.0) std::frexp(mx, &e);  // mx < 2^e
            expo[(size_t)op * NS + s] = e;
            for (int k = 0; k < K; ++k) {
                const int64_t X = (int64_t)std::llround(std::ldexp(W[(size_t)k * NS + s], 46 - e));
                digits_of(X, &dig[((size_t)k * NS + s) * kTcDigits]);
            }
        }
        // rearrange into the units of the half's image
        uint16_t *half = image.data() + (op == 0 ? 0 : kTc3ImageElems / 2);
        for (int c = 0; c < ncomp; ++c) {
            const int i = op == 0 ? c : op - 1;
            for (int vz = 0; vz < 2; ++vz)
                for (int kh = 0; kh < 2; ++kh) {
                    uint16_t *unit = half + (size_t)((i * 2 + vz) * 2 + kh) * kTc3UnitElems;
                    for (int vv = 0; vv < 4; ++vv)
                        for (int ch = 0; ch < 2; ++ch)
                            for (int nn = 0; nn < 7 * NS; ++nn)
                                for (int kk = 0; kk < 8; ++kk) {
                                    const int j = nn / NS, s = nn % NS, l = kh * 16 + ch * 8 + kk;
                                    const int v = vv + 4 * vz;
                                    int d = 0;
                                    if (j < kTcDigits && s < NQ && l < NQ)
                                        d = dig[((size_t)((c * 8 + v) * NS + l) * NS + s) * kTcDigits + j];
                                    unit[(((size_t)vv * 2 + ch) * (7 * NS) + nn) * 8 + kk] = f16_of_small_int(d);
                                }
                }
        }
    }
    return true;
}

}  // namespace hl
