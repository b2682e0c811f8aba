// Launch logic of the mixed-precision kernels (included once per dimension).
#pragma once

#include "hl_internal.h"
#include "hl_mixed.cuh"

namespace hl {

template <int D, int M, bool COMP, int I>
static void launch_u_split_mx(const LaunchFp64 &a, const CoefF32<D, M, COMP> &cf, dim3 grid, dim3 block)
{
    if constexpr (I < D) {
        k_u_half_mx<D, M, COMP, I, 1><<<grid, block, 0, a.stream>>>(a.Ph, a.Pl, a.U, a.Uh, a.Ul, a.shots, a.n_shots,
                                                                      cf, a.status);
        launch_u_split_mx<D, M, COMP, I + 1>(a, cf, grid, block);
    }
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
    constexpr bool fused = D * S::NQ * (COMP ? 2 : 1) <= 192;
    const dim3 grid((unsigned)a.total_tiles), block((unsigned)a.tx, (unsigned)a.ty);
    for (int64_t st = 0; st < a.nsteps; ++st) {
        if (a.ev) cudaEventRecord(a.ev[2 * st], a.stream);
        k_p_half_mx<D, M, COMP><<<grid, block, 0, a.stream>>>(a.Uh, a.Ul, a.P, a.Ph, a.Pl, a.shots, a.n_shots, cf,
                                                               a.status);
        if (a.src && a.src->active) {
            cudaError_t e = launch_source(*a.src, a.shots, a.P, S::NQ, a.step0 + st, a.stream, a.Ph, a.Pl);
            if (e != cudaSuccess) return e;
        }
        if (a.ev) cudaEventRecord(a.ev[2 * st + 1], a.stream);
        if constexpr (fused)
            k_u_half_mx<D, M, COMP, 0, D><<<grid, block, 0, a.stream>>>(a.Ph, a.Pl, a.U, a.Uh, a.Ul, a.shots,
                                                                         a.n_shots, cf, a.status);
        else
            launch_u_split_mx<D, M, COMP, 0>(a, cf, grid, block);
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
