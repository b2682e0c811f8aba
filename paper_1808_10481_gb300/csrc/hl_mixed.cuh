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

#include <type_traits>

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
    return nonfinite(v);
}

// ---------------------------------------------------------------------------
// One half-step of a mixed mode.  The partner field's shadows for the block's
// tile plus its one-node halo are staged through shared memory LC slots at a
// time, in a two-buffer cp.async pipeline with one barrier per stage: while
// the block contracts one stage (component c, slots l0 .. l0+LC-1) the next
// stage is in flight.
//   PHALF: partner = U (D components), target = P, cell vertices j-1, j;
//   else : partner = P, target = U components I0 .. I0+NI-1, vertices j, j+1.
// The staged region is (TX+1)(TY+1)(2) nodes over the axes in use; the
// offset of each region node inside a slot is computed once per block and
// kept in shared memory after the two buffers.
template <int D, int M>
struct MixedStage {
    static constexpr int NQ = Shape<D, M>::NQ;
    static constexpr int LC = M + 1;     // slots per stage (divides NQ)
    static constexpr int NCH = NQ / LC;  // stages per component
};
constexpr int kMixedBufs = 2;  // pipeline depth: shared-memory buffers of LC slots
template <int D>
__host__ __device__ __forceinline__ int region_nodes(int tx, int ty)
{
    int r = tx + 1;
    if (D >= 2) r *= ty + 1;
    if (D >= 3) r *= 2;
    return r;
}

// Compile-time loop: f(std::integral_constant<int, I>) for I = B .. E-1.  The
// stage, slot and output indices of the contraction must be constants so that
// the structural zeros, the butterfly patterns and the coefficient offsets
// resolve at compile time; a plain unrolled loop of this size is not
// guaranteed to be unrolled.
template <int B, int E, class F>
__device__ __forceinline__ void static_for(F &&f)
{
    if constexpr (B < E) {
        f(std::integral_constant<int, B>{});
        static_for<B + 1, E>(f);
    }
}

__device__ __forceinline__ void cp_async4(float *dst, const float *src)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <int D, int M, bool COMP, bool PHALF, int I0, int NI>
__global__ void __launch_bounds__(256)
    k_half_mx(const float *__restrict__ Sh, const float *__restrict__ Sl, double *__restrict__ X,
              float *__restrict__ Xh, float *__restrict__ Xl, const ShotDesc *__restrict__ shots, int n_shots,
              CoefF32<D, M, COMP> cf, unsigned *status)
{
    using S = Shape<D, M>;
    using G = MixedStage<D, M>;
    constexpr int NCOMP = PHALF ? D : 1;
    constexpr int NST = NCOMP * G::NCH;
    constexpr int NPART = COMP ? 2 : 1;
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
    const int RX = blockDim.x + 1, RY = D >= 2 ? blockDim.y + 1 : 1;
    const int R = region_nodes<D>(blockDim.x, blockDim.y);
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    const int nthr = blockDim.x * blockDim.y;
    // offsets inside one slot of every region node, once per block; stored
    // after the two pipeline buffers
    int *soff = reinterpret_cast<int *>(sm + (size_t)kMixedBufs * NPART * G::LC * R);
    for (int r = tid; r < R; r += nthr) {
        int gx = x0 + lo + r % RX, gy = y0 + lo + (r / RX) % RY, gz = z0 + lo + r / (RX * RY);
        gx += gx < 0 ? sd.n[0] : (gx >= sd.n[0] ? -sd.n[0] : 0);
        if (D >= 2) gy += gy < 0 ? sd.n[1] : (gy >= sd.n[1] ? -sd.n[1] : 0); else gy = 0;
        if (D >= 3) gz += gz < 0 ? sd.n[2] : (gz >= sd.n[2] ? -sd.n[2] : 0); else gz = 0;
        soff[r] = gx + sd.n[0] * (gy + sd.n[1] * gz);
    }
    __syncthreads();
    // this thread's cell vertices inside the region
    int vr[S::NV];
#pragma unroll
    for (int v = 0; v < S::NV; ++v) {
        const int rx = threadIdx.x + (v & 1);
        const int ry = D >= 2 ? threadIdx.y + ((v >> 1) & 1) : 0;
        const int rz = D >= 3 ? ((v >> 2) & 1) : 0;
        vr[v] = rx + RX * (ry + RY * rz);
    }
    // stage st (component st / NCH, slots (st % NCH) * LC ...) holds the
    // partner's slots st * LC .. st * LC + LC - 1; it goes to buffer st % kMixedBufs.
    // The source pointers advance one stage at a time and are hidden from the
    // optimiser, so no per-stage address is precomputed and kept live.
    const int64_t base = PHALF ? sd.u_off : sd.p_off;
    const int64_t stage_stride = (int64_t)G::LC * sd.nnode;
    const float *nh = Sh + base;
    const float *nl = COMP ? Sl + base : nullptr;
    auto prefetch = [&](int st) {
        float *bh = sm + (size_t)((st % kMixedBufs) * NPART) * G::LC * R;
        // a rolled loop over the region: few live addresses at a time
#pragma unroll 1
        for (int r = tid; r < R; r += nthr) {
            const int g = soff[r];
#pragma unroll
            for (int j = 0; j < G::LC; ++j) {
                const int64_t so = (int64_t)j * sd.nnode + g;
                cp_async4(bh + j * R + r, nh + so);
                if constexpr (COMP) cp_async4(bh + (G::LC + j) * R + r, nl + so);
            }
        }
        cp_async_commit();
        nh += stage_stride;
        asm volatile("" : "+l"(nh));
        if constexpr (COMP) {
            nl += stage_stride;
            asm volatile("" : "+l"(nl));
        }
    };
    constexpr int NACC = PHALF ? S::NQ : NI * S::NQ;
    Acc<COMP> acc[NACC];
#pragma unroll
    for (int e = 0; e < NACC; ++e) acc[e].zero();
    // one commit group per stage (empty past the last), kMixedBufs - 1 in flight
#pragma unroll
    for (int s0 = 0; s0 < kMixedBufs - 1; ++s0) {
        if (s0 < NST) prefetch(s0); else cp_async_commit();
    }
    // The float-float 3D p-half (27 stages of 27 outputs) fully unrolled is
    // about 30 k instructions and runs slower (instruction fetch) than this
    // rolled loop, which resolves the stage's coefficients at run time.
    constexpr bool kRolled = COMP && D == 3 && PHALF;
    if constexpr (kRolled) {
#pragma unroll 1
        for (int st = 0; st < NST; ++st) {
            cp_async_wait<kMixedBufs - 2>();
            __syncthreads();
            if (st + kMixedBufs - 1 < NST) prefetch(st + kMixedBufs - 1); else cp_async_commit();
            if (active) {
                const int c = st / G::NCH, l0 = (st % G::NCH) * G::LC;
                const float *bh = sm + (size_t)((st % kMixedBufs) * NPART) * G::LC * R;
#pragma unroll
                for (int j = 0; j < G::LC; ++j) {
                    const int l = l0 + j;
                    Slot<D, COMP> xs;
#pragma unroll
                    for (int v = 0; v < S::NV; ++v) xs.x[v] = FF{bh[j * R + vr[v]], bh[(G::LC + j) * R + vr[v]]};
                    butterfly_ff<D>(xs.x);
#pragma unroll
                    for (int s = 0; s < S::NQ; ++s)
                        if (coef_nonzero(D, S::n, c, s, l))
                            xs.madd(acc[s], cf, coef_index(S::NQ, c, l, s), bfly_pattern(D, S::n, c, s, l));
                }
            }
        }
    } else {
        static_for<0, NST>([&](auto stc) {
            constexpr int st = decltype(stc)::value;
            // stage st has landed once at most kMixedBufs - 2 newer groups are
            // pending; after the barrier it is visible to the whole block, and
            // every thread has finished stage st-1, whose buffer the prefetch of
            // stage st + kMixedBufs - 1 then reuses
            cp_async_wait<kMixedBufs - 2>();
            __syncthreads();
            if constexpr (st + kMixedBufs - 1 < NST) prefetch(st + kMixedBufs - 1); else cp_async_commit();
            if (active) {
                constexpr int c = st / G::NCH, l0 = (st % G::NCH) * G::LC;
                const float *bh = sm + (size_t)((st % kMixedBufs) * NPART) * G::LC * R;
                static_for<0, G::LC>([&](auto jc) {
                    constexpr int j = decltype(jc)::value, l = l0 + j;
                    Slot<D, COMP> xs;
#pragma unroll
                    for (int v = 0; v < S::NV; ++v) {
                        if constexpr (COMP)
                            xs.x[v] = FF{bh[j * R + vr[v]], bh[(G::LC + j) * R + vr[v]]};
                        else
                            xs.x[v] = bh[j * R + vr[v]];
                    }
                    if constexpr (COMP) butterfly_ff<D>(xs.x); else butterfly_f<D>(xs.x);
                    if constexpr (PHALF) {
                        static_for<0, S::NQ>([&](auto sc) {
                            constexpr int s = decltype(sc)::value;
                            if constexpr (coef_nonzero(D, S::n, c, s, l))
                                xs.madd(acc[s], cf, coef_index(S::NQ, c, l, s), bfly_pattern(D, S::n, c, s, l));
                        });
                    } else {
                        static_for<0, NI * S::NQ>([&](auto ec) {
                            constexpr int ii = decltype(ec)::value / S::NQ, s = decltype(ec)::value % S::NQ;
                            if constexpr (coef_nonzero(D, S::n, I0 + ii, s, l))
                                xs.madd(acc[ii * S::NQ + s], cf, coef_index(S::NQ, I0 + ii, l, s),
                                        bfly_pattern(D, S::n, I0 + ii, s, l));
                        });
                    }
                });
            }
        });
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
