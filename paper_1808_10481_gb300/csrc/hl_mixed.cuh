// Mixed-precision half-step kernels: the fused contraction (butterfly plus
// compile-time-sparse operator, as in hl_fp64.cuh) runs on the FP32 pipe,
// while the node data stay IEEE binary64 and the increment is added to them
// in FP64.
//
//   HL_FP32      : x_h = fl32(x), M_h = fl32(M); out = sum M_h * bfly(x_h)
//                  accumulated in FP32.
//   HL_FP32_COMP : split-precision correction.  x = x_h + x_l and M = M_h + M_l
//                  with x_l = fl32(x - x_h), M_l = fl32(M - M_h); the main sum
//                  M_h x_h and the correction M_h x_l + M_l x_h are accumulated
//                  in separate FP32 registers (the correction is ~2^-24 times
//                  smaller, so its own rounding is negligible) and added in FP64.
//                  The x_l * M_l term is below 2^-48 and dropped.
// Once the contraction leaves the FP64 pipe a step is bound by the HBM traffic
// of the FP64 state, so the FP32 work only has to stay below that time.
#pragma once

#include "hl_fp64.cuh"

namespace hl {

template <int D, int M, bool COMP>
struct CoefF32 {
    float hi[Shape<D, M>::NCOEF];
    float lo[COMP ? Shape<D, M>::NCOEF : 1];
};

template <int D>
__device__ __forceinline__ void butterfly_f(float *x)
{
#pragma unroll
    for (int k = 0; k < D; ++k) {
#pragma unroll
        for (int v = 0; v < (1 << D); ++v) {
            if (!(v & (1 << k))) {
                const float a = x[v], b = x[v | (1 << k)];
                x[v] = a + b;
                x[v | (1 << k)] = a - b;
            }
        }
    }
}

// gather one slot of one component at the 2^D vertices, split into FP32 parts
template <int D, bool COMP>
__device__ __forceinline__ void gather_split(const double *__restrict__ base, const int *vtx, float *xh, float *xl)
{
#pragma unroll
    for (int v = 0; v < (1 << D); ++v) {
        const double x = __ldg(base + vtx[v]);
        xh[v] = __double2float_rn(x);
        if constexpr (COMP) xl[v] = __double2float_rn(x - (double)xh[v]);
    }
}

template <int D, int M, bool COMP>
__global__ void __launch_bounds__(256) k_p_half_f32(const double *__restrict__ U, double *__restrict__ P,
                                                    const ShotDesc *__restrict__ shots, int n_shots,
                                                    CoefF32<D, M, COMP> cf, unsigned *status)
{
    using S = Shape<D, M>;
    int shot;
    ShotDesc sd;
    int64_t node;
    if (!tile_node<D>(shots, n_shots, shot, sd, node)) return;
    const GridDesc g{{sd.n[0], sd.n[1], sd.n[2]}, sd.nnode};
    const double *Us = U + sd.u_off;
    double *Ps = P + sd.p_off;
    int vtx[S::NV];
    vertex_nodes<D>(g, node, -1, vtx);
    float acc[S::NQ], cor[COMP ? S::NQ : 1];
#pragma unroll
    for (int s = 0; s < S::NQ; ++s) {
        acc[s] = 0.f;
        if constexpr (COMP) cor[s] = 0.f;
    }
#pragma unroll
    for (int i = 0; i < D; ++i) {
#pragma unroll
        for (int l = 0; l < S::NQ; ++l) {
            float xh[S::NV], xl[S::NV];
            gather_split<D, COMP>(Us + (int64_t)(i * S::NQ + l) * g.nnode, vtx, xh, xl);
            butterfly_f<D>(xh);
            if constexpr (COMP) butterfly_f<D>(xl);
#pragma unroll
            for (int s = 0; s < S::NQ; ++s) {
                if (coef_nonzero(D, S::n, i, s, l)) {
                    const int c = coef_index(S::NQ, i, l, s);
                    const int pat = bfly_pattern(D, S::n, i, s, l);
                    acc[s] = fmaf(cf.hi[c], xh[pat], acc[s]);
                    if constexpr (COMP) cor[s] = fmaf(cf.hi[c], xl[pat], fmaf(cf.lo[c], xh[pat], cor[s]));
                }
            }
        }
    }
    bool bad = false;
#pragma unroll
    for (int s = 0; s < S::NQ; ++s) {
        double inc = (double)acc[s];
        if constexpr (COMP) inc += (double)cor[s];
        const double v = Ps[(int64_t)s * g.nnode + node] + inc;
        Ps[(int64_t)s * g.nnode + node] = v;
        bad |= !isfinite(v);
    }
    report_nonfinite(bad, status);
}

template <int D, int M, bool COMP, int I0, int NI>
__global__ void __launch_bounds__(256) k_u_half_f32(const double *__restrict__ P, double *__restrict__ U,
                                                    const ShotDesc *__restrict__ shots, int n_shots,
                                                    CoefF32<D, M, COMP> cf, unsigned *status)
{
    using S = Shape<D, M>;
    int shot;
    ShotDesc sd;
    int64_t node;
    if (!tile_node<D>(shots, n_shots, shot, sd, node)) return;
    const GridDesc g{{sd.n[0], sd.n[1], sd.n[2]}, sd.nnode};
    const double *Ps = P + sd.p_off;
    double *Us = U + sd.u_off;
    int vtx[S::NV];
    vertex_nodes<D>(g, node, 0, vtx);
    float acc[NI * S::NQ], cor[COMP ? NI * S::NQ : 1];
#pragma unroll
    for (int e = 0; e < NI * S::NQ; ++e) {
        acc[e] = 0.f;
        if constexpr (COMP) cor[e] = 0.f;
    }
#pragma unroll
    for (int l = 0; l < S::NQ; ++l) {
        float xh[S::NV], xl[S::NV];
        gather_split<D, COMP>(Ps + (int64_t)l * g.nnode, vtx, xh, xl);
        butterfly_f<D>(xh);
        if constexpr (COMP) butterfly_f<D>(xl);
#pragma unroll
        for (int ii = 0; ii < NI; ++ii) {
            const int i = I0 + ii;
#pragma unroll
            for (int s = 0; s < S::NQ; ++s) {
                if (coef_nonzero(D, S::n, i, s, l)) {
                    const int c = coef_index(S::NQ, i, l, s);
                    const int pat = bfly_pattern(D, S::n, i, s, l);
                    acc[ii * S::NQ + s] = fmaf(cf.hi[c], xh[pat], acc[ii * S::NQ + s]);
                    if constexpr (COMP)
                        cor[ii * S::NQ + s] = fmaf(cf.hi[c], xl[pat], fmaf(cf.lo[c], xh[pat], cor[ii * S::NQ + s]));
                }
            }
        }
    }
    bool bad = false;
#pragma unroll
    for (int ii = 0; ii < NI; ++ii)
#pragma unroll
        for (int s = 0; s < S::NQ; ++s) {
            double inc = (double)acc[ii * S::NQ + s];
            if constexpr (COMP) inc += (double)cor[ii * S::NQ + s];
            double *dst = Us + (int64_t)((I0 + ii) * S::NQ + s) * g.nnode + node;
            const double v = *dst + inc;
            *dst = v;
            bad |= !isfinite(v);
        }
    report_nonfinite(bad, status);
}

}  // namespace hl
