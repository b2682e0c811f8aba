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

// ---------------------------------------------------------------------------
// One half-step of a mixed mode.  The partner field's shadows for the block's
// tile plus its one-node halo are staged through shared memory, one partner
// component at a time (a cooperative, coalesced load of every slot, then all
// vertex reads from shared memory).
//   PHALF: partner = U (D components), target = P, cell vertices j-1, j;
//   else : partner = P, target = U components I0 .. I0+NI-1, vertices j, j+1.
// Dynamic shared memory: NQ * R floats per shadow part, R = (TX+1)(TY+1)(2)
// over the axes in use.
template <int D>
__device__ __forceinline__ int region_size()
{
    int r = blockDim.x + 1;
    if (D >= 2) r *= blockDim.y + 1;
    if (D >= 3) r *= 2;
    return r;
}

template <int D, int M, bool COMP, bool PHALF, int I0, int NI>
__global__ void __launch_bounds__(256)
    k_half_mx(const float *__restrict__ Sh, const float *__restrict__ Sl, double *__restrict__ X,
              float *__restrict__ Xh, float *__restrict__ Xl, const ShotDesc *__restrict__ shots, int n_shots,
              CoefF32<D, M, COMP> cf, unsigned *status)
{
    using S = Shape<D, M>;
    extern __shared__ float sm[];
    int shot;
    ShotDesc sd;
    int64_t node;
    const bool active = tile_node<D>(shots, n_shots, shot, sd, node);
    // tile origin (tile_node's arithmetic, for the whole block)
    int t = blockIdx.x - sd.tile_begin;
    const int x0 = (t % sd.tiles[0]) * blockDim.x;
    t /= sd.tiles[0];
    const int y0 = (t % sd.tiles[1]) * blockDim.y;
    const int z0 = t / sd.tiles[1];
    const int lo = PHALF ? -1 : 0;
    const int RX = blockDim.x + 1, RY = D >= 2 ? blockDim.y + 1 : 1, RZ = D >= 3 ? 2 : 1;
    const int R = RX * RY * RZ;
    float *sh = sm;
    float *sl = sm + S::NQ * R;
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    const int nthr = blockDim.x * blockDim.y;
    // this thread's vertex offsets inside the staged region
    int vr[S::NV];
#pragma unroll
    for (int v = 0; v < S::NV; ++v) {
        const int rx = threadIdx.x + (v & 1);
        const int ry = D >= 2 ? threadIdx.y + ((v >> 1) & 1) : 0;
        const int rz = D >= 3 ? ((v >> 2) & 1) : 0;
        vr[v] = rx + RX * (ry + RY * rz);
    }
    constexpr int NACC = PHALF ? S::NQ : NI * S::NQ;
    Acc<COMP> acc[NACC];
#pragma unroll
    for (int e = 0; e < NACC; ++e) acc[e].zero();
    constexpr int NCOMP = PHALF ? D : 1;
#pragma unroll
    for (int c = 0; c < NCOMP; ++c) {
        const int64_t coff = (PHALF ? sd.u_off : sd.p_off) + (int64_t)c * S::NQ * sd.nnode;
        __syncthreads();  // the previous component's reads are done
        for (int e = tid; e < S::NQ * R; e += nthr) {
            const int slot = e / R, r = e % R;
            int rx = r % RX, ry = (r / RX) % RY, rz = r / (RX * RY);
            int gx = x0 + lo + rx, gy = y0 + lo + ry, gz = z0 + lo + rz;
            gx += gx < 0 ? sd.n[0] : (gx >= sd.n[0] ? -sd.n[0] : 0);
            if (D >= 2) gy += gy < 0 ? sd.n[1] : (gy >= sd.n[1] ? -sd.n[1] : 0); else gy = 0;
            if (D >= 3) gz += gz < 0 ? sd.n[2] : (gz >= sd.n[2] ? -sd.n[2] : 0); else gz = 0;
            const int64_t g = coff + (int64_t)slot * sd.nnode + gx + (int64_t)sd.n[0] * (gy + (int64_t)sd.n[1] * gz);
            sh[e] = __ldg(Sh + g);
            if constexpr (COMP) sl[e] = __ldg(Sl + g);
        }
        __syncthreads();
        if (active) {
#pragma unroll
            for (int l = 0; l < S::NQ; ++l) {
                Slot<D, COMP> xs;
#pragma unroll
                for (int v = 0; v < S::NV; ++v) {
                    if constexpr (COMP)
                        xs.x[v] = FF{sh[l * R + vr[v]], sl[l * R + vr[v]]};
                    else
                        xs.x[v] = sh[l * R + vr[v]];
                }
                if constexpr (COMP) butterfly_ff<D>(xs.x); else butterfly_f<D>(xs.x);
                if constexpr (PHALF) {
#pragma unroll
                    for (int s = 0; s < S::NQ; ++s)
                        if (coef_nonzero(D, S::n, c, s, l))
                            xs.madd(acc[s], cf, coef_index(S::NQ, c, l, s), bfly_pattern(D, S::n, c, s, l));
                } else {
#pragma unroll
                    for (int ii = 0; ii < NI; ++ii)
#pragma unroll
                        for (int s = 0; s < S::NQ; ++s)
                            if (coef_nonzero(D, S::n, I0 + ii, s, l))
                                xs.madd(acc[ii * S::NQ + s], cf, coef_index(S::NQ, I0 + ii, l, s),
                                        bfly_pattern(D, S::n, I0 + ii, s, l));
                }
            }
        }
    }
    if (!active) return;
    bool bad = false;
#pragma unroll
    for (int e = 0; e < NACC; ++e) {
        const int64_t idx = (PHALF ? sd.p_off + (int64_t)e * sd.nnode
                                   : sd.u_off + (int64_t)(I0 * S::NQ + e) * sd.nnode) + node;
        bad |= store_value<COMP>(X, Xh, Xl, idx, acc[e].to_f64());
    }
    report_nonfinite(bad, status);
}

}  // namespace hl
