// Mixed-precision half-step kernels: the fused contraction of hl_fp64.cuh
// (vertex butterfly plus compile-time-sparse operator) on the FP32 pipe,
// while the node data stay IEEE binary64 and every increment is added to them
// in binary64.
//
// Each field keeps binary32 shadows next to its binary64 state: hi = RN32(x)
// and, for HL_FP32_COMP, lo = x - hi to 24 more bits (hl_split.cuh).  The
// gathers read only the shadows; each kernel's epilogue rewrites the shadows
// of the values it updated, with integer operations (the hardware conversions
// issue on the FP64 pipe).  hl_step refreshes all shadows from the binary64
// state before its first half-step.
//
//   HL_FP32      : operator rounded to binary32, butterfly and contraction in
//                  binary32 (relative rounding 2^-24 amplified by the
//                  operator's cancellation).
//   HL_FP32_COMP : float-float arithmetic (hi + lo pairs, about 48 bits):
//                  error-free TwoSum/TwoProduct in the butterfly and every
//                  multiply-add, operator split into hi + lo; the rounding
//                  error of every step is carried instead of dropped.
#pragma once

#include "hl_fp64.cuh"
#include "hl_split.cuh"

namespace hl {

template <int D, int M, bool COMP>
struct CoefF32 {
    float hi[Shape<D, M>::NCOEF];
    float lo[COMP ? Shape<D, M>::NCOEF : 1];
};

template <bool COMP>
__global__ void k_shadow(const double *__restrict__ X, float *__restrict__ hi, float *__restrict__ lo, int64_t n)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const FF s = split_f64(X[e]);
        hi[e] = s.hi;
        if constexpr (COMP) lo[e] = s.lo;
    }
}

template <int D>
__device__ __forceinline__ void butterfly_f(float *x)
{
#pragma unroll
    for (int k = 0; k < D; ++k)
#pragma unroll
        for (int v = 0; v < (1 << D); ++v)
            if (!(v & (1 << k))) {
                const float a = x[v], b = x[v | (1 << k)];
                x[v] = a + b;
                x[v | (1 << k)] = a - b;
            }
}

template <int D>
__device__ __forceinline__ void butterfly_ff(FF *x)
{
#pragma unroll
    for (int k = 0; k < D; ++k)
#pragma unroll
        for (int v = 0; v < (1 << D); ++v)
            if (!(v & (1 << k))) {
                const FF a = x[v], b = x[v | (1 << k)];
                x[v] = ff_add(a, b);
                x[v | (1 << k)] = ff_sub(a, b);
            }
}

// accumulator of one output: binary32, or float-float
template <bool COMP>
struct Acc;
template <>
struct Acc<false> {
    float v;
    __device__ __forceinline__ void zero() { v = 0.f; }
    __device__ __forceinline__ double to_f64() const { return f32_to_f64(v); }
};
template <>
struct Acc<true> {
    FF v;
    __device__ __forceinline__ void zero() { v = {0.f, 0.f}; }
    __device__ __forceinline__ double to_f64() const
    {
        const FF n = ff_two_sum(v.hi, v.lo);
        return f32_to_f64(n.hi) + f32_to_f64(n.lo);  // exact: the pair spans at most 49 bits
    }
};

// one gathered, butterflied slot: binary32 or float-float values per pattern
template <int D, bool COMP>
struct Slot;
template <int D>
struct Slot<D, false> {
    float x[1 << D];
    __device__ __forceinline__ void load(const float *__restrict__ h, const float *, const int *vtx)
    {
#pragma unroll
        for (int v = 0; v < (1 << D); ++v) x[v] = __ldg(h + vtx[v]);
        butterfly_f<D>(x);
    }
    template <int NC>
    __device__ __forceinline__ void madd(Acc<false> &a, const CoefF32<D, NC, false> &cf, int c, int pat) const
    {
        a.v = fmaf(cf.hi[c], x[pat], a.v);
    }
};
template <int D>
struct Slot<D, true> {
    FF x[1 << D];
    __device__ __forceinline__ void load(const float *__restrict__ h, const float *__restrict__ l, const int *vtx)
    {
#pragma unroll
        for (int v = 0; v < (1 << D); ++v) x[v] = FF{__ldg(h + vtx[v]), __ldg(l + vtx[v])};
        butterfly_ff<D>(x);
    }
    template <int NC>
    __device__ __forceinline__ void madd(Acc<true> &a, const CoefF32<D, NC, true> &cf, int c, int pat) const
    {
        ff_fma(a.v, FF{cf.hi[c], cf.lo[c]}, x[pat]);
    }
};

// new binary64 value and its shadows
template <bool COMP>
__device__ __forceinline__ bool store_value(double *__restrict__ X, float *__restrict__ Xh, float *__restrict__ Xl,
                                            int64_t idx, double inc)
{
    const double v = X[idx] + inc;
    X[idx] = v;
    const FF s = split_f64(v);
    Xh[idx] = s.hi;
    if constexpr (COMP) Xl[idx] = s.lo;
    return !isfinite(v);
}

template <int D, int M, bool COMP>
__global__ void __launch_bounds__(256)
    k_p_half_mx(const float *__restrict__ Uh, const float *__restrict__ Ul, double *__restrict__ P,
                float *__restrict__ Ph, float *__restrict__ Pl, const ShotDesc *__restrict__ shots, int n_shots,
                CoefF32<D, M, COMP> cf, unsigned *status)
{
    using S = Shape<D, M>;
    int shot;
    ShotDesc sd;
    int64_t node;
    if (!tile_node<D>(shots, n_shots, shot, sd, node)) return;
    const GridDesc g{{sd.n[0], sd.n[1], sd.n[2]}, sd.nnode};
    int vtx[S::NV];
    vertex_nodes<D>(g, node, -1, vtx);
    Acc<COMP> acc[S::NQ];
#pragma unroll
    for (int s = 0; s < S::NQ; ++s) acc[s].zero();
#pragma unroll
    for (int i = 0; i < D; ++i) {
#pragma unroll
        for (int l = 0; l < S::NQ; ++l) {
            const int64_t off = sd.u_off + (int64_t)(i * S::NQ + l) * g.nnode;
            Slot<D, COMP> x;
            x.load(Uh + off, COMP ? Ul + off : nullptr, vtx);
#pragma unroll
            for (int s = 0; s < S::NQ; ++s)
                if (coef_nonzero(D, S::n, i, s, l))
                    x.madd(acc[s], cf, coef_index(S::NQ, i, l, s), bfly_pattern(D, S::n, i, s, l));
        }
    }
    bool bad = false;
#pragma unroll
    for (int s = 0; s < S::NQ; ++s)
        bad |= store_value<COMP>(P, Ph, Pl, sd.p_off + (int64_t)s * g.nnode + node, acc[s].to_f64());
    report_nonfinite(bad, status);
}

template <int D, int M, bool COMP, int I0, int NI>
__global__ void __launch_bounds__(256)
    k_u_half_mx(const float *__restrict__ Ph, const float *__restrict__ Pl, double *__restrict__ U,
                float *__restrict__ Uh, float *__restrict__ Ul, const ShotDesc *__restrict__ shots, int n_shots,
                CoefF32<D, M, COMP> cf, unsigned *status)
{
    using S = Shape<D, M>;
    int shot;
    ShotDesc sd;
    int64_t node;
    if (!tile_node<D>(shots, n_shots, shot, sd, node)) return;
    const GridDesc g{{sd.n[0], sd.n[1], sd.n[2]}, sd.nnode};
    int vtx[S::NV];
    vertex_nodes<D>(g, node, 0, vtx);
    Acc<COMP> acc[NI * S::NQ];
#pragma unroll
    for (int e = 0; e < NI * S::NQ; ++e) acc[e].zero();
#pragma unroll
    for (int l = 0; l < S::NQ; ++l) {
        const int64_t off = sd.p_off + (int64_t)l * g.nnode;
        Slot<D, COMP> x;
        x.load(Ph + off, COMP ? Pl + off : nullptr, vtx);
#pragma unroll
        for (int ii = 0; ii < NI; ++ii)
#pragma unroll
            for (int s = 0; s < S::NQ; ++s)
                if (coef_nonzero(D, S::n, I0 + ii, s, l))
                    x.madd(acc[ii * S::NQ + s], cf, coef_index(S::NQ, I0 + ii, l, s),
                           bfly_pattern(D, S::n, I0 + ii, s, l));
    }
    bool bad = false;
#pragma unroll
    for (int ii = 0; ii < NI; ++ii)
#pragma unroll
        for (int s = 0; s < S::NQ; ++s)
            bad |= store_value<COMP>(U, Uh, Ul, sd.u_off + (int64_t)((I0 + ii) * S::NQ + s) * g.nnode + node,
                                     acc[ii * S::NQ + s].to_f64());
    report_nonfinite(bad, status);
}

}  // namespace hl
