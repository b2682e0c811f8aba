// Launch logic of the mixed-precision kernels (included once per dimension).
#pragma once

#include <atomic>

#include "hl_internal.h"
#include "hl_mixed.cuh"

namespace hl {

template <int D, int M, bool COMP, bool PHALF, int I0, int NI>
static cudaError_t launch_half(const LaunchFp64 &a, const CoefF32<D, M, COMP> &cf, dim3 grid, dim3 block,
                               size_t smem)
{
    auto kern = k_half_mx<D, M, COMP, PHALF, I0, NI>;
    // allow up to the per-block maximum once per instantiation and device (not
    // per launch, and so never from inside a stream capture after the first call)
    static std::atomic<uint64_t> opted_in{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const uint64_t bit = 1ull << (dev & 63);
    if (!(opted_in.load() & bit)) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        if (e != cudaSuccess) return e;
        opted_in.fetch_or(bit);
    }
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    if (PHALF)
        kern<<<grid, block, smem, a.stream>>>(a.Uh, a.Ul, a.P, a.Ph, a.Pl, a.shots, a.n_shots, cf, a.status);
    else
        kern<<<grid, block, smem, a.stream>>>(a.Ph, a.Pl, a.U, a.Uh, a.Ul, a.shots, a.n_shots, cf, a.status);
    return cudaGetLastError();
}

template <int D, int M, bool COMP, int I>
static cudaError_t launch_u_split_mx(const LaunchFp64 &a, const CoefF32<D, M, COMP> &cf, dim3 grid, dim3 block,
                                     size_t smem)
{
    if constexpr (I < D) {
        cudaError_t e = launch_half<D, M, COMP, false, I, 1>(a, cf, grid, block, smem);
        if (e != cudaSuccess) return e;
        return launch_u_split_mx<D, M, COMP, I + 1>(a, cf, grid, block, smem);
    }
    return cudaSuccess;
}

template <int D, int M, bool COMP>
static cudaError_t run_mixed_t(const LaunchFp64 &a)
{
    using S = Shape<D, M>;
    CoefF32<D, M, COMP> cf;
    for (int c = 0; c < S::NCOEF; ++c) {
        const double v = a.coef_host[c];
        cf.hi[c] = (float)v;
        if constexpr (COMP) cf.lo[c] = (float)(v - (double)cf.hi[c]);
    }
    // shadows of the current binary64 state
    const unsigned sb = 152 * 16;
    k_shadow<COMP><<<sb, 256, 0, a.stream>>>(a.P, a.Ph, a.Pl, a.p_elems);
    k_shadow<COMP><<<sb, 256, 0, a.stream>>>(a.U, a.Uh, a.Ul, a.p_elems * D);
    // keep all D float-float accumulator blocks of the u-half in registers only when small
    // (2D float-float m = 3, 64 accumulators, measured 23% faster split)
    constexpr bool fused = D * S::NQ * (COMP ? 2 : 1) < 64;
    const dim3 grid((unsigned)a.total_tiles), block((unsigned)a.tx, (unsigned)a.ty);
    const int region = region_nodes<D>(a.tx, a.ty);
    // kMixedBufs pipeline buffers of LC slots each (hi, and lo for the
    // compensated mode), then one offset per region node
    const size_t smem = ((size_t)kMixedBufs * MixedStage<D, M>::LC * (COMP ? 2 : 1) + 1) * region * sizeof(float);
    cudaError_t e;
    for (int64_t st = 0; st < a.nsteps; ++st) {
        if (a.ev) cudaEventRecord(a.ev[2 * st], a.stream);
        if ((e = launch_half<D, M, COMP, true, 0, 1>(a, cf, grid, block, smem)) != cudaSuccess) return e;
        if (a.src && a.src->active) {
            if ((e = launch_source(*a.src, a.shots, a.P, S::NQ, a.step0 + st, a.stream, a.Ph, a.Pl)) != cudaSuccess)
                return e;
        }
        if (a.ev) cudaEventRecord(a.ev[2 * st + 1], a.stream);
        if constexpr (fused)
            e = launch_half<D, M, COMP, false, 0, D>(a, cf, grid, block, smem);
        else
            e = launch_u_split_mx<D, M, COMP, 0>(a, cf, grid, block, smem);
        if (e != cudaSuccess) return e;
    }
    if (a.ev) cudaEventRecord(a.ev[2 * a.nsteps], a.stream);
    return cudaGetLastError();
}

template <int D, int M>
static cudaError_t run_mixed(const LaunchFp64 &a)
{
    if (a.nsteps <= 0) return cudaSuccess;
    if (a.used_small) *a.used_small = false;
    if (!a.Ph || !a.Uh || (a.precision == 2 && (!a.Pl || !a.Ul))) return cudaErrorInvalidValue;
    if (a.precision == 2) return run_mixed_t<D, M, true>(a);
    return run_mixed_t<D, M, false>(a);
}

}  // namespace hl
