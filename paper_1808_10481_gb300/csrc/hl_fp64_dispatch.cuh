// Per-dimension launch logic of the FP64 kernels (included once per dimension).
#pragma once

#include <cstring>

#include "hl_fp64.cuh"
#include "hl_internal.h"

namespace hl {

template <int D, int M, int I, class CP>
static void launch_u_split(const LaunchFp64 &a, const CP &cp, dim3 grid, dim3 block)
{
    if constexpr (I < D) {
        k_u_half<D, M, I, 1, CP><<<grid, block, 0, a.stream>>>(a.P, a.U, a.shots, a.n_shots, cp, a.status);
        launch_u_split<D, M, I + 1, CP>(a, cp, grid, block);
    }
}

// tiny single grids: the whole run in one CTA when the state fits in shared
// memory and the per-step work is too small to pay for 2 launches per step
template <int D, int M>
static bool use_small(const LaunchFp64 &a)
{
    using S = Shape<D, M>;
    if (a.n_shots != 1 || (a.src && a.src->active)) return false;
    const size_t smem = (size_t)(D + 1) * S::NQ * a.nnode * sizeof(double);
    if (smem > 200 * 1024) return false;
    if (a.path == PATH_SMALL) return true;
    if (a.path == PATH_GRID) return false;
    return (double)a.nnode * S::NQ * S::NQ * D <= 40000.0;
}

template <int D, int M, class CP>
static cudaError_t run_grid(const LaunchFp64 &a, const CP &cp)
{
    using S = Shape<D, M>;
    const dim3 grid((unsigned)a.total_tiles), block((unsigned)a.tx, (unsigned)a.ty);
    // paired tiles (even height) run two nodes per thread along y: bit 0 of
    // a.pair for the p-half, bit 1 for the u-half
    const bool pair_p = D >= 2 && (a.pair & 1) && a.ty % 2 == 0;
    const bool pair_u = D >= 2 && (a.pair & 2) && a.ty % 2 == 0;
    const dim3 pblock((unsigned)a.tx, (unsigned)(a.ty / 2));
    for (int64_t st = 0; st < a.nsteps; ++st) {
        if (a.ev) cudaEventRecord(a.ev[2 * st], a.stream);
        bool done = false;
        if constexpr (S::kPairP) {
            if (pair_p) {
                k_p_half_pair<D, M, CP><<<grid, pblock, 0, a.stream>>>(a.U, a.P, a.shots, a.n_shots, cp, a.status);
                done = true;
            }
        }
        if (!done) k_p_half<D, M, CP><<<grid, block, 0, a.stream>>>(a.U, a.P, a.shots, a.n_shots, cp, a.status);
        if (a.src && a.src->active) {
            cudaError_t e = launch_source(*a.src, a.shots, a.P, S::NQ, a.step0 + st, a.stream);
            if (e != cudaSuccess) return e;
        }
        if (a.ev) cudaEventRecord(a.ev[2 * st + 1], a.stream);
        done = false;
        if constexpr (S::kPairU) {
            if (pair_u) {
                k_u_half_pair<D, M, CP><<<grid, pblock, 0, a.stream>>>(a.P, a.U, a.shots, a.n_shots, cp, a.status);
                done = true;
            }
        }
        if (!done) {
            if constexpr (S::kUFused)
                k_u_half<D, M, 0, D, CP><<<grid, block, 0, a.stream>>>(a.P, a.U, a.shots, a.n_shots, cp, a.status);
            else
                launch_u_split<D, M, 0, CP>(a, cp, grid, block);
        }
    }
    if (a.ev) cudaEventRecord(a.ev[2 * a.nsteps], a.stream);
    return cudaGetLastError();
}

template <int D, int M>
static cudaError_t run_fp64(const LaunchFp64 &a)
{
    using S = Shape<D, M>;
    if (a.nsteps <= 0) return cudaSuccess;
    if (a.used_small) *a.used_small = false;
    if (a.per_shot_coef) {
        if constexpr (M <= 3) {
            return run_grid<D, M>(a, CoefShots<D, M>{a.coef_dev});
        } else {
            return cudaErrorInvalidValue;  // batched handles support m <= 3
        }
    }
    CoefParam<D, M> cp;
    if constexpr (S::kParam)
        std::memcpy(cp.c.v, a.coef_host, sizeof(cp.c.v));
    else
        cp.c.v = a.coef_dev;
    if (use_small<D, M>(a)) {
        using C = CoefArg<D, M, S::kParam>;
        const GridDesc g{{a.n[0], a.n[1], a.n[2]}, a.nnode};
        const size_t smem = (size_t)(D + 1) * S::NQ * a.nnode * sizeof(double);
        cudaError_t e = cudaFuncSetAttribute(k_small<D, M, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int threads = (int)((a.nnode + 31) / 32 * 32);
        if (threads > 256) threads = 256;
        if (a.used_small) *a.used_small = true;
        if (a.ev) cudaEventRecord(a.ev[0], a.stream);
        k_small<D, M, C><<<1, threads, smem, a.stream>>>(a.P, a.U, g, cp.c, a.nsteps, a.status);
        if (a.ev) cudaEventRecord(a.ev[1], a.stream);
        return cudaGetLastError();
    }
    return run_grid<D, M>(a, cp);
}

}  // namespace hl
