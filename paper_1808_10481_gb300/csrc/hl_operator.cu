// Host construction of the fused per-node operator used by the kernels.
//
// 1D Hermite-Birkhoff system (Section 2, eq. interp): on the cell centred at
// the target node, in xi = (x - x_node)/h, the interpolant sum_a c_a xi^a of
// degree 2m+1 must reproduce the scaled end data (1/l!) d^l/dxi^l at
// xi = -1/2 and xi = +1/2 for l = 0..m:
//     A[l][a]       = binom(a, l) (-1/2)^(a-l)      (lower end)
//     A[m+1+l][a]   = binom(a, l) (+1/2)^(a-l)      (upper end)
// and H = A^{-1} (Gauss-Jordan with partial pivoting, double precision).
//
// Series (Section 2, eqs. update1/LFloop/final1; Section 3.1.2, eqs. pdup,
// vdup; Section 5, eq. lf1update2D): for target slot s and direction i the
// odd time derivatives at the half step, written with Lap^k = sum_{|b|=k}
// k!/b! d^{2b}, give the scaled increment
//     -sum_{k,|b|=k} 2/(2k+1)! k!/b! prod_j (a_j!/s_j!) lam_j^(a_j - s_j) c_a,
//     a = s + 2b + e_i,  lam_j = dt/(2 h_j),
// with terms whose index exceeds 2m+1 on any axis absent (degree 2m+1 per axis).
//
// Fused, butterflied operator: coefficient (i, l, s) multiplies the
// butterflied vertex value of slot l; it equals the all-lower-vertex block
//     M0_i[s][l] = sum_b W_i[s][a] prod_j H[a_j][l_j]
// (H's lower-end columns), negated so that the kernel adds it.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "hl_dd_host.h"
#include "hl_internal.h"
#include "hl_fp64.cuh"

namespace hl {

// H = [C^L; C^R]^{-1} by Gauss-Jordan with partial pivoting in double-double;
// the exact inverse is dyadic (representable in binary64) for m <= 6, so the
// final rounding returns it exactly.
bool hermite_inverse_1d(int m, std::vector<double> &H)
{
    const int A = 2 * m + 2;
    std::vector<DD> a((size_t)A * 2 * A, dd(0.0));  // augmented [A | I]
    for (int l = 0; l <= m; ++l) {
        for (int c = l; c < A; ++c) {
            const double w = (double)ibinom(c, l);
            a[(size_t)l * 2 * A + c] = dd(w * std::ldexp((c - l) % 2 ? -1.0 : 1.0, -(c - l)));
            a[(size_t)(m + 1 + l) * 2 * A + c] = dd(w * std::ldexp(1.0, -(c - l)));
        }
    }
    for (int r = 0; r < A; ++r) a[(size_t)r * 2 * A + A + r] = dd(1.0);
    for (int col = 0; col < A; ++col) {
        int piv = col;
        for (int r = col + 1; r < A; ++r)
            if (std::fabs(a[(size_t)r * 2 * A + col].hi) > std::fabs(a[(size_t)piv * 2 * A + col].hi)) piv = r;
        if (a[(size_t)piv * 2 * A + col].hi == 0.0) return false;
        if (piv != col)
            for (int c = 0; c < 2 * A; ++c) std::swap(a[(size_t)col * 2 * A + c], a[(size_t)piv * 2 * A + c]);
        const DD pv = a[(size_t)col * 2 * A + col];
        for (int c = 0; c < 2 * A; ++c) a[(size_t)col * 2 * A + c] = dd_div(a[(size_t)col * 2 * A + c], pv);
        for (int r = 0; r < A; ++r) {
            if (r == col) continue;
            const DD f = a[(size_t)r * 2 * A + col];
            if (f.hi == 0.0) continue;
            for (int c = 0; c < 2 * A; ++c)
                a[(size_t)r * 2 * A + c] = dd_add(a[(size_t)r * 2 * A + c], dd_neg(dd_mul(f, a[(size_t)col * 2 * A + c])));
        }
    }
    H.assign((size_t)A * A, 0.0);
    for (int r = 0; r < A; ++r)
        for (int c = 0; c < A; ++c) H[(size_t)r * A + c] = a[(size_t)r * 2 * A + A + c].hi;
    return true;
}

// Dense table coef[(i*NQ + l)*NQ + s] (negated series operator), NQ = (m+1)^D,
// composed in double-double and rounded once.  Returns false if the
// structural-zero rule the kernels rely on fails.
bool build_operator(int D, int m, const double lam[3], std::vector<double> &coef)
{
    const int n = m + 1, A = 2 * m + 2;
    int NQ = 1;
    for (int k = 0; k < D; ++k) NQ *= n;
    std::vector<double> H;
    if (!hermite_inverse_1d(m, H)) return false;
    // lam_k^e in double-double, e = 0..2m+1
    std::vector<DD> lp[3];
    for (int k = 0; k < D; ++k) {
        lp[k].assign(A, dd(1.0));
        for (int e = 1; e < A; ++e) lp[k][e] = dd_mul(lp[k][e - 1], dd(lam[k]));
    }
    std::vector<DD> acc((size_t)D * NQ * NQ, dd(0.0));
    for (int i = 0; i < D; ++i) {
        for (int s = 0; s < NQ; ++s) {
            int sv[3] = {0, 0, 0};
            for (int k = 0, t = s; k < D; ++k, t /= n) sv[k] = t % n;
            int bmax[3] = {0, 0, 0};
            bool any = true;
            for (int k = 0; k < D; ++k) {
                const int t0 = sv[k] + (k == i ? 1 : 0);
                if (t0 > 2 * m + 1) any = false;
                bmax[k] = (2 * m + 1 - t0) / 2;
            }
            if (!any) continue;
            for (int b2 = 0; b2 <= (D > 2 ? bmax[2] : 0); ++b2)
                for (int b1 = 0; b1 <= (D > 1 ? bmax[1] : 0); ++b1)
                    for (int b0 = 0; b0 <= bmax[0]; ++b0) {
                        const int b[3] = {b0, b1, b2};
                        const int K = b0 + b1 + b2;
                        int a[3] = {0, 0, 0};
                        // W = 2 K!/(2K+1)! * prod_k [a_k!/(s_k! b_k!)] lam_k^(a_k - s_k);
                        // 2 K!/(2K+1)! = 2 / ((K+1)(K+2)...(2K+1)), divided out one small
                        // integer at a time ((2K+1)! itself overflows int64 for K >= 10)
                        DD w = dd(2.0);
                        for (int j = K + 1; j <= 2 * K + 1; ++j) w = dd_div(w, dd((double)j));
                        for (int k = 0; k < D; ++k) {
                            a[k] = sv[k] + 2 * b[k] + (k == i ? 1 : 0);
                            // a_k!/s_k! is an integer (a_k >= s_k) below 2^53
                            w = dd_mul(w, dd_div(dd_int(ifact(a[k]) / ifact(sv[k])), dd_int(ifact(b[k]))));
                            w = dd_mul(w, lp[k][a[k] - sv[k]]);
                        }
                        for (int l = 0; l < NQ; ++l) {
                            double h = 1.0;  // products of dyadic H entries: exact
                            for (int k = 0, t = l; k < D; ++k, t /= n) h *= H[(size_t)a[k] * A + (t % n)];
                            DD &c = acc[((size_t)i * NQ + l) * NQ + s];
                            c = dd_add(c, dd_neg(dd_mul(w, dd(h))));
                        }
                    }
        }
    }
    coef.resize(acc.size());
    double maxabs = 0.0;
    for (size_t e = 0; e < acc.size(); ++e) {
        coef[e] = acc[e].hi + acc[e].lo;
        maxabs = std::fmax(maxabs, std::fabs(coef[e]));
    }
    // the kernels skip entries the structural rule declares zero: verify it
    for (int i = 0; i < D; ++i)
        for (int l = 0; l < NQ; ++l)
            for (int s = 0; s < NQ; ++s)
                if (!coef_nonzero(D, n, i, s, l)) {
                    double &c = coef[((size_t)i * NQ + l) * NQ + s];
                    if (std::fabs(c) > 1e-13 * maxabs) return false;
                    c = 0.0;  // exact zero: only double-double residue remains here
                }
    return true;
}

// Multiply-adds and adds per node and full step of the fused FP64 kernels.
void fp64_op_counts(int D, int m, double *fma_per_node_step, double *add_per_node_step)
{
    const int n = m + 1;
    int NQ = 1;
    for (int k = 0; k < D; ++k) NQ *= n;
    long nz = 0;
    for (int i = 0; i < D; ++i)
        for (int l = 0; l < NQ; ++l)
            for (int s = 0; s < NQ; ++s) nz += coef_nonzero(D, n, i, s, l) ? 1 : 0;
    const double bfly = (double)D * (1 << D) * NQ;  // one butterfly over NQ slots
    *fma_per_node_step = 2.0 * nz;                  // p-half and u-half share the table
    // butterflies (p-half: D components; u-half: one field) plus the final
    // addition of each increment to the node's own value
    *add_per_node_step = bfly * D + bfly + (double)NQ * (1 + D);
}

}  // namespace hl
