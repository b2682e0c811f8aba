// Hermite-leapfrog step with a spatially varying wave speed (Section 4.2), 1D:
//     p_t + c^2(x) u_x = 0,   u_t + p_x = 0   on the periodic unit interval.
//
// Per node and half-step (one thread per node, binary64 throughout):
//   1. gather the partner field at the two cell vertices and build the degree-2m+1
//      Hermite-Birkhoff interpolant (Section 2, eq. interp) as scaled Taylor
//      coefficients in xi = (x - x_node)/h;
//   2. run the Cauchy-Kowalevsky recurrence with c^2 given at the node by its scaled
//      Taylor coefficients c~_i = h^i/i! d^i c^2, i = 0..2m+1 (Section 4.2's local
//      expansion), on polynomials kept to degree 2m+1: with P_k = h^k d_t^k p and
//      U_k = h^k d_t^k u,  P_(k+1) = -c~ * D U_k  and  U_(k+1) = -D P_k  (D = d/dxi,
//      * the truncated product);
//   3. add 2 sum_{k odd <= 2m+1} lam^k / k! F_k (lam = dt/(2h); F = P for the p-half,
//      whose interpolant is U_0, and F = U for the u-half, whose interpolant is P_0)
//      to the node's own slots 0..m (Section 2, eq. update1).
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "hl_fp64.cuh"
#include "hl_internal.h"

namespace hl {

template <int M>
struct VarParams {
    static constexpr int A = 2 * M + 2;
    double H[A * A];   // Hermite-Birkhoff inverse, row a = coefficient, column = end datum
    double w[A + 1];   // w[k] = 2 lam^k / k!
};

template <int M, bool PHALF>
__global__ void __launch_bounds__(256) k_var_half(const double *__restrict__ S, double *__restrict__ X,
                                                  const double *__restrict__ C2, int n, VarParams<M> vp,
                                                  unsigned *status)
{
    constexpr int NQ = M + 1, A = 2 * M + 2;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    bool bad = false;
    if (j < n) {
        int lo = PHALF ? j - 1 : j;
        if (lo < 0) lo += n;
        int hi = lo + 1;
        if (hi >= n) hi -= n;
        double e[A];
#pragma unroll
        for (int l = 0; l < NQ; ++l) {
            e[l] = __ldg(S + (int64_t)l * n + lo);
            e[NQ + l] = __ldg(S + (int64_t)l * n + hi);
        }
        double c[A], c2[A], inc[A];
#pragma unroll
        for (int a = 0; a < A; ++a) {
            double s = 0.0;
#pragma unroll
            for (int l = 0; l < A; ++l) s = fma(vp.H[a * A + l], e[l], s);
            c[a] = s;
            c2[a] = __ldg(C2 + (int64_t)a * n + j);
            inc[a] = 0.0;
        }
        // c holds U_0 (p-half) or P_0 (u-half); f alternates between the two fields
        double f[A];
#pragma unroll
        for (int a = 0; a < A; ++a) f[a] = c[a];
#pragma unroll
        for (int k = 0; k < 2 * M + 1; ++k) {
            // derivative D f (degree kept), then for the P step the product with c~
            double df[A];
#pragma unroll
            for (int a = 0; a < A - 1; ++a) df[a] = (double)(a + 1) * f[a + 1];
            df[A - 1] = 0.0;
            const bool to_p = PHALF ? (k % 2 == 0) : (k % 2 == 1);  // next order is a P step
            if (to_p) {
#pragma unroll
                for (int a = A - 1; a >= 0; --a) {
                    double s = 0.0;
#pragma unroll
                    for (int i = 0; i <= a; ++i) s = fma(c2[i], df[a - i], s);
                    f[a] = -s;
                }
            } else {
#pragma unroll
                for (int a = 0; a < A; ++a) f[a] = -df[a];
            }
            if ((k + 1) % 2 == 1) {  // odd order k + 1: a term of the update
#pragma unroll
                for (int a = 0; a < NQ; ++a) inc[a] = fma(vp.w[k + 1], f[a], inc[a]);
            }
        }
#pragma unroll
        for (int s = 0; s < NQ; ++s) {
            double *dst = X + (int64_t)s * n + j;
            const double v = *dst + inc[s];
            *dst = v;
            bad |= nonfinite(v);
        }
    }
    report_nonfinite(bad, status);
}

template <int M>
static cudaError_t run_var(const LaunchFp64 &a)
{
    if (!a.c2_primal || !a.c2_dual || a.n_shots != 1) return cudaErrorInvalidValue;
    constexpr int A = 2 * M + 2;
    VarParams<M> vp;
    std::vector<double> H;
    if (!hermite_inverse_1d(M, H)) return cudaErrorInvalidValue;
    for (int i = 0; i < A * A; ++i) vp.H[i] = H[(size_t)i];
    double pw = 1.0, fact = 1.0;
    for (int k = 0; k <= A - 1; ++k) {
        if (k > 0) {
            pw *= a.var_lam;
            fact *= (double)k;
        }
        vp.w[k] = 2.0 * pw / fact;
    }
    vp.w[A] = 0.0;
    const int n = a.n[0];
    const unsigned blocks = (unsigned)((n + 255) / 256);
    cudaError_t e;
    for (int64_t st = 0; st < a.nsteps; ++st) {
        if (a.ev) cudaEventRecord(a.ev[2 * st], a.stream);
        k_var_half<M, true><<<blocks, 256, 0, a.stream>>>(a.U, a.P, a.c2_primal, n, vp, a.status);
        if (a.src && a.src->active) {
            if ((e = launch_source(*a.src, a.shots, a.P, M + 1, a.step0 + st, a.stream)) != cudaSuccess) return e;
        }
        if (a.ev) cudaEventRecord(a.ev[2 * st + 1], a.stream);
        k_var_half<M, false><<<blocks, 256, 0, a.stream>>>(a.P, a.U, a.c2_dual, n, vp, a.status);
    }
    if (a.ev) cudaEventRecord(a.ev[2 * a.nsteps], a.stream);
    return cudaGetLastError();
}

cudaError_t launch_var_d1(const LaunchFp64 &a)
{
    switch (a.m) {
    case 0: return run_var<0>(a);
    case 1: return run_var<1>(a);
    case 2: return run_var<2>(a);
    case 3: return run_var<3>(a);
    case 4: return run_var<4>(a);
    case 5: return run_var<5>(a);
    case 6: return run_var<6>(a);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace hl
