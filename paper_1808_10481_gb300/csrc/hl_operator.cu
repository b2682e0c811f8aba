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

#include "hl_internal.h"
#include "hl_fp64.cuh"

namespace hl {

static double fact(int n)
{
    double f = 1.0;
    for (int k = 2; k <= n; ++k) f *= k;
    return f;
}

static double binom(int a, int l) { return fact(a) / (fact(l) * fact(a - l)); }

bool hermite_inverse_1d(int m, std::vector<double> &H)
{
    const int A = 2 * m + 2;
    std::vector<double> a(A * 2 * A, 0.0);  // augmented [A | I]
    for (int l = 0; l <= m; ++l) {
        for (int c = l; c < A; ++c) {
            const double w = binom(c, l);
            a[l * 2 * A + c] = w * std::pow(-0.5, c - l);
            a[(m + 1 + l) * 2 * A + c] = w * std::pow(0.5, c - l);
        }
    }
    for (int r = 0; r < A; ++r) a[r * 2 * A + A + r] = 1.0;
    for (int col = 0; col < A; ++col) {
        int piv = col;
        for (int r = col + 1; r < A; ++r)
            if (std::fabs(a[r * 2 * A + col]) > std::fabs(a[piv * 2 * A + col])) piv = r;
        if (a[piv * 2 * A + col] == 0.0) return false;
        if (piv != col)
            for (int c = 0; c < 2 * A; ++c) std::swap(a[col * 2 * A + c], a[piv * 2 * A + c]);
        const double inv = 1.0 / a[col * 2 * A + col];
        for (int c = 0; c < 2 * A; ++c) a[col * 2 * A + c] *= inv;
        for (int r = 0; r < A; ++r) {
            if (r == col) continue;
            const double f = a[r * 2 * A + col];
            if (f == 0.0) continue;
            for (int c = 0; c < 2 * A; ++c) a[r * 2 * A + c] -= f * a[col * 2 * A + c];
        }
    }
    H.assign(A * A, 0.0);
    for (int r = 0; r < A; ++r)
        for (int c = 0; c < A; ++c) H[r * A + c] = a[r * 2 * A + A + c];
    return true;
}

// Dense table coef[(i*NQ + l)*NQ + s] (negated series operator), NQ = (m+1)^D.
// Returns false if the structural-zero rule the kernels rely on fails.
bool build_operator(int D, int m, const double lam[3], std::vector<double> &coef)
{
    const int n = m + 1, A = 2 * m + 2;
    int NQ = 1;
    for (int k = 0; k < D; ++k) NQ *= n;
    std::vector<double> H;
    if (!hermite_inverse_1d(m, H)) return false;
    coef.assign((size_t)D * NQ * NQ, 0.0);
    double maxabs = 0.0;
    for (int i = 0; i < D; ++i) {
        for (int s = 0; s < NQ; ++s) {
            int sv[3] = {0, 0, 0};
            for (int k = 0, t = s; k < D; ++k, t /= n) sv[k] = t % n;
            // enumerate b with 2 b_j + s_j + [j==i] <= 2m+1
            int bmax[3] = {0, 0, 0};
            for (int k = 0; k < D; ++k) bmax[k] = (2 * m + 1 - sv[k] - (k == i ? 1 : 0)) / 2;
            bool any = true;
            for (int k = 0; k < D; ++k)
                if (sv[k] + (k == i ? 1 : 0) > 2 * m + 1) any = false;
            if (!any) continue;
            for (int b2 = 0; b2 <= (D > 2 ? bmax[2] : 0); ++b2)
                for (int b1 = 0; b1 <= (D > 1 ? bmax[1] : 0); ++b1)
                    for (int b0 = 0; b0 <= bmax[0]; ++b0) {
                        const int b[3] = {b0, b1, b2};
                        const int K = b0 + b1 + b2;
                        int a[3];
                        double w = 2.0 / fact(2 * K + 1) * fact(K);
                        for (int k = 0; k < D; ++k) {
                            a[k] = sv[k] + 2 * b[k] + (k == i ? 1 : 0);
                            w *= fact(a[k]) / (fact(sv[k]) * fact(b[k])) * std::pow(lam[k], a[k] - sv[k]);
                        }
                        for (int l = 0; l < NQ; ++l) {
                            double h = 1.0;
                            for (int k = 0, t = l; k < D; ++k, t /= n) h *= H[a[k] * A + (t % n)];
                            coef[((size_t)i * NQ + l) * NQ + s] -= w * h;
                        }
                    }
        }
    }
    for (double v : coef) maxabs = std::fmax(maxabs, std::fabs(v));
    // the kernels skip entries the structural rule declares zero: verify it
    for (int i = 0; i < D; ++i)
        for (int l = 0; l < NQ; ++l)
            for (int s = 0; s < NQ; ++s)
                if (!coef_nonzero(D, n, i, s, l) &&
                    std::fabs(coef[((size_t)i * NQ + l) * NQ + s]) > 1e-13 * maxabs)
                    return false;
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
    *add_per_node_step = bfly * D + bfly;           // p-half: D components; u-half: one field
}

}  // namespace hl
