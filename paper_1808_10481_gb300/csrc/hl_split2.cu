// The split two-kernel form of the FP64 half-step (Section 6: the interpolation
// and evolution kernels of the paper's GPU comparison, Figs. 5-6, Table 6), kept
// as an ablation beside the fused kernels of hl_fp64.cuh (HL_OPT_SPLIT).
//
//   interpolation kernel: for every target node and partner component, the
//     tensor-product Hermite-Birkhoff interpolant on the node's cell, its
//     (2m+2)^dim scaled Taylor coefficients computed one axis at a time (apply H
//     along x, then y, then z; Section 2, eq. interp; Section 5) in shared memory,
//     and stored to a global buffer [component][coefficient][node];
//   evolution kernel: for every target node, the Cauchy-Kowalevsky series of the
//     stored coefficients (Section 2, eqs. update1, LFloop, final1; Section 3.1.2,
//     eqs. pdup and vdup) as a sparse term list per output slot, added to the
//     node's own data.
// The stored interpolant makes the pair bound by the round trip of
// (2m+2)^dim coefficients per component through HBM, against the fused kernels'
// (m+1)^dim per vertex read, and the per-axis contraction costs
// dim (2m+2)^(dim+1) multiply-adds per component against the fused butterfly's
// (m+1)^(2 dim) per direction.
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <vector>

#include "hl_dd_host.h"
#include "hl_fp64.cuh"
#include "hl_internal.h"

namespace hl {

template <int D, int M>
struct SplitShape {
    static constexpr int n = M + 1;
    static constexpr int A = 2 * M + 2;
    static constexpr int AD = ipow_c(A, D);            // coefficients per node and component
    static constexpr int NQ = ipow_c(n, D);
    // nodes per block: the largest power of two with NB * AD <= 4096 (32 KB per buffer)
    static constexpr int NB = AD <= 16 ? 256 : AD <= 32 ? 128 : AD <= 64 ? 64 : AD <= 128 ? 32 : AD <= 256 ? 16 : 8;
};

struct SplitH {
    double h[64];  // H[a][e], A x A (A <= 8)
};

template <int D, int M, bool PHALF>
__global__ void __launch_bounds__(256) k_split_interp(const double *__restrict__ S, double *__restrict__ C,
                                                      GridDesc g, int tiles_x, SplitH H)
{
    using SS = SplitShape<D, M>;
    constexpr int A = SS::A, AD = SS::AD, NB = SS::NB, n = SS::n;
    constexpr int NCIN = PHALF ? D : 1;
    extern __shared__ double split_sm[];  // two buffers of NB * AD doubles (dynamic: up to 64 KB)
    double *const bufs[2] = {split_sm, split_sm + NB * AD};
    const int t = blockIdx.x;
    const int tx = t % tiles_x;
    const int64_t row = t / tiles_x;  // y + n1 z
    const int x0 = tx * NB;
    const int lo = PHALF ? -1 : 0;
    const int iy = D >= 2 ? (int)(row % g.n[1]) : 0;
    const int iz = D >= 3 ? (int)(row / g.n[1]) : 0;
    for (int c = 0; c < NCIN; ++c) {
        // gather: entry (e_0, e_1, e_2) of node nb, e_k = v_k n + l_k, at index nb*AD + sum e_k A^k
        for (int idx = threadIdx.x; idx < NB * AD; idx += blockDim.x) {
            const int nb = idx % NB;
            int r = idx / NB;
            int v = 0, l = 0, lstride = 1;
            int e[3] = {0, 0, 0};
#pragma unroll
            for (int k = 0; k < D; ++k) {
                e[k] = r % A;
                r /= A;
                v |= (e[k] / n) << k;
                l += (e[k] % n) * lstride;
                lstride *= n;
            }
            const int x = x0 + nb;
            double val = 0.0;
            if (x < g.n[0]) {
                int cx = x + lo + (v & 1);
                cx = cx < 0 ? cx + g.n[0] : (cx >= g.n[0] ? cx - g.n[0] : cx);
                int cy = 0, cz = 0;
                if (D >= 2) {
                    cy = iy + lo + ((v >> 1) & 1);
                    cy = cy < 0 ? cy + g.n[1] : (cy >= g.n[1] ? cy - g.n[1] : cy);
                }
                if (D >= 3) {
                    cz = iz + lo + ((v >> 2) & 1);
                    cz = cz < 0 ? cz + g.n[2] : (cz >= g.n[2] ? cz - g.n[2] : cz);
                }
                const int64_t node = cx + (int64_t)g.n[0] * (cy + (int64_t)g.n[1] * cz);
                val = __ldg(S + (int64_t)(c * SS::NQ + l) * g.nnode + node);
            }
            int off = 0, st = 1;
#pragma unroll
            for (int k = 0; k < D; ++k) {
                off += e[k] * st;
                st *= A;
            }
            bufs[0][nb * AD + off] = val;
        }
        __syncthreads();
        // one axis at a time: out[.., a_k, ..] = sum_e H[a_k][e] in[.., e, ..]
        int cur = 0;
#pragma unroll
        for (int k = 0; k < D; ++k) {
            const int Sk = k == 0 ? 1 : (k == 1 ? A : A * A);  // stride of axis k
            for (int idx = threadIdx.x; idx < NB * AD; idx += blockDim.x) {
                const int nb = idx / AD, rem = idx % AD;
                const int ak = (rem / Sk) % A;
                const int base = nb * AD + rem - ak * Sk;
                double s = 0.0;
#pragma unroll
                for (int e = 0; e < A; ++e) s = fma(H.h[ak * A + e], bufs[cur][base + e * Sk], s);
                bufs[cur ^ 1][idx] = s;
            }
            __syncthreads();
            cur ^= 1;
        }
        // store coefficient a of node nb to C[c][a][node]
        for (int idx = threadIdx.x; idx < NB * AD; idx += blockDim.x) {
            const int nb = idx % NB, a = idx / NB;
            const int x = x0 + nb;
            if (x < g.n[0]) {
                const int64_t node = x + (int64_t)g.n[0] * row;
                C[(int64_t)(c * AD + a) * g.nnode + node] = bufs[cur][nb * AD + a];
            }
        }
        __syncthreads();
    }
}

// Term list of the evolution: for output (direction i, slot s) the entries
// [beg[i*NQ + s], beg[i*NQ + s + 1]) of (coefficient index, weight).
template <int D, int M, bool PHALF>
__global__ void __launch_bounds__(256) k_split_evolve(const double *__restrict__ C, double *__restrict__ X,
                                                      int64_t nnode, const int *__restrict__ beg,
                                                      const int *__restrict__ idx, const double *__restrict__ w,
                                                      unsigned *status)
{
    using SS = SplitShape<D, M>;
    constexpr int NQ = SS::NQ, AD = SS::AD;
    const int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool bad = false;
    if (node < nnode) {
        if constexpr (PHALF) {
            for (int s = 0; s < NQ; ++s) {
                double acc = 0.0;
                for (int i = 0; i < D; ++i)
                    for (int t = __ldg(beg + i * NQ + s); t < __ldg(beg + i * NQ + s + 1); ++t)
                        acc = fma(__ldg(w + t), __ldg(C + (int64_t)(i * AD + __ldg(idx + t)) * nnode + node), acc);
                double *dst = X + (int64_t)s * nnode + node;
                const double v = *dst + acc;
                *dst = v;
                bad |= nonfinite(v);
            }
        } else {
            for (int i = 0; i < D; ++i)
                for (int s = 0; s < NQ; ++s) {
                    double acc = 0.0;
                    for (int t = __ldg(beg + i * NQ + s); t < __ldg(beg + i * NQ + s + 1); ++t)
                        acc = fma(__ldg(w + t), __ldg(C + (int64_t)__ldg(idx + t) * nnode + node), acc);
                    double *dst = X + (int64_t)(i * NQ + s) * nnode + node;
                    const double v = *dst + acc;
                    *dst = v;
                    bad |= nonfinite(v);
                }
        }
    }
    report_nonfinite(bad, status);
}

// Host term lists: weight of coefficient a = s + 2 beta + e_i in output (i, s),
//   -2 K!/(2K+1)! prod_k a_k!/(s_k! beta_k!) lam_k^(a_k - s_k),  K = |beta|,
// composed in double-double and rounded once (the negation makes the kernel add).
bool build_split_terms(int D, int m, const double lam[3], std::vector<int> &beg, std::vector<int> &idx,
                       std::vector<double> &w)
{
    const int n = m + 1, A = 2 * m + 2;
    int NQ = 1;
    for (int k = 0; k < D; ++k) NQ *= n;
    beg.assign((size_t)D * NQ + 1, 0);
    idx.clear();
    w.clear();
    for (int i = 0; i < D; ++i)
        for (int s = 0; s < NQ; ++s) {
            beg[(size_t)i * NQ + s] = (int)idx.size();
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
                        DD c = dd(-2.0);
                        for (int j = K + 1; j <= 2 * K + 1; ++j) c = dd_div(c, dd((double)j));
                        int a = 0, stride = 1;
                        for (int k = 0; k < D; ++k) {
                            const int ak = sv[k] + 2 * b[k] + (k == i ? 1 : 0);
                            c = dd_mul(c, dd_div(dd_int(ifact(ak) / ifact(sv[k])), dd_int(ifact(b[k]))));
                            for (int e = 0; e < ak - sv[k]; ++e) c = dd_mul(c, dd(lam[k]));
                            a += ak * stride;
                            stride *= A;
                        }
                        idx.push_back(a);
                        w.push_back(c.hi + c.lo);
                    }
        }
    beg[(size_t)D * NQ] = (int)idx.size();
    return true;
}

template <int D, int M>
static cudaError_t run_split_t(const LaunchFp64 &a)
{
    using SS = SplitShape<D, M>;
    static_assert(SS::A <= 8, "SplitH holds A <= 8");
    std::vector<double> Hv;
    if (!hermite_inverse_1d(M, Hv)) return cudaErrorInvalidValue;
    SplitH H;
    for (int e = 0; e < SS::A * SS::A; ++e) H.h[e] = Hv[(size_t)e];
    const GridDesc g{{a.n[0], a.n[1], a.n[2]}, a.nnode};
    const size_t smem = (size_t)2 * SS::NB * SS::AD * sizeof(double);
    static std::atomic<uint64_t> opted_in{0};  // devices on which the attribute is set
    int dev = 0;
    cudaError_t e0 = cudaGetDevice(&dev);
    if (e0 != cudaSuccess) return e0;
    if (!(opted_in.load() & (1ull << (dev & 63)))) {
        if ((e0 = cudaFuncSetAttribute(k_split_interp<D, M, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem)) != cudaSuccess ||
            (e0 = cudaFuncSetAttribute(k_split_interp<D, M, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem)) != cudaSuccess)
            return e0;
        opted_in.fetch_or(1ull << (dev & 63));
    }
    const int tiles_x = (a.n[0] + SS::NB - 1) / SS::NB;
    const int64_t tiles = (int64_t)tiles_x * a.n[1] * a.n[2];
    const unsigned eb = (unsigned)((a.nnode + 255) / 256);
    // both halves share the term lists: output (i, s) of the p-half sums component i of u,
    // output (i, s) of the u-half is direction i of the one component p
    for (int64_t st = 0; st < a.nsteps; ++st) {
        if (a.ev) cudaEventRecord(a.ev[2 * st], a.stream);
        k_split_interp<D, M, true><<<(unsigned)tiles, 256, smem, a.stream>>>(a.U, a.split_coef, g, tiles_x, H);
        k_split_evolve<D, M, true><<<eb, 256, 0, a.stream>>>(a.split_coef, a.P, a.nnode, a.split_beg, a.split_idx,
                                                             a.split_w, a.status);
        if (a.src && a.src->active) {
            const cudaError_t e = launch_source(*a.src, a.shots, a.P, SS::NQ, a.step0 + st, a.stream);
            if (e != cudaSuccess) return e;
        }
        if (a.ev) cudaEventRecord(a.ev[2 * st + 1], a.stream);
        k_split_interp<D, M, false><<<(unsigned)tiles, 256, smem, a.stream>>>(a.P, a.split_coef, g, tiles_x, H);
        k_split_evolve<D, M, false><<<eb, 256, 0, a.stream>>>(a.split_coef, a.U, a.nnode, a.split_beg, a.split_idx,
                                                              a.split_w, a.status);
    }
    if (a.ev) cudaEventRecord(a.ev[2 * a.nsteps], a.stream);
    return cudaGetLastError();
}

cudaError_t launch_split(int dim, const LaunchFp64 &a)
{
    if (!a.split_coef || !a.split_beg || a.n_shots != 1) return cudaErrorInvalidValue;
#define HL_SPLIT_CASE(D_, M_) \
    if (dim == D_ && a.m == M_) return run_split_t<D_, M_>(a);
    HL_SPLIT_CASE(1, 0) HL_SPLIT_CASE(1, 1) HL_SPLIT_CASE(1, 2) HL_SPLIT_CASE(1, 3)
    HL_SPLIT_CASE(2, 0) HL_SPLIT_CASE(2, 1) HL_SPLIT_CASE(2, 2) HL_SPLIT_CASE(2, 3)
    HL_SPLIT_CASE(3, 0) HL_SPLIT_CASE(3, 1) HL_SPLIT_CASE(3, 2) HL_SPLIT_CASE(3, 3)
#undef HL_SPLIT_CASE
    return cudaErrorInvalidValue;
}

}  // namespace hl
