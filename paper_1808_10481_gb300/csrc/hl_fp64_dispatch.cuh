// Per-dimension launch logic of the FP64 kernels (included once per dimension).
#pragma once

#include <cstring>

#include "hl_fp64.cuh"
#include "hl_internal.h"

namespace hl {

template <int D, int M, int I, class C>
static void launch_u_split(const LaunchFp64 &a, const GridDesc &g, const C &coef, int blocks)
{
    if constexpr (I < D) {
        k_u_half<D, M, I, 1, C><<<blocks, 128, 0, a.stream>>>(a.P, a.U, g, coef, a.status);
        launch_u_split<D, M, I + 1, C>(a, g, coef, blocks);
    }
}

// tiny grids: the whole run in one CTA when the state fits in shared memory
// and the per-step work is too small to pay for 2 launches per step
template <int D, int M>
static bool use_small(const LaunchFp64 &a)
{
    using S = Shape<D, M>;
    const size_t smem = (size_t)(D + 1) * S::NQ * a.nnode * sizeof(double);
    if (smem > 200 * 1024) return false;
    if (a.src.active) return false;  // the source is injected between launches
    if (a.path == PATH_SMALL) return true;
    if (a.path == PATH_GRID) return false;
    return (double)a.nnode * S::NQ * S::NQ * D <= 40000.0;
}

template <int D, int M>
static cudaError_t run_fp64(const LaunchFp64 &a)
{
    using S = Shape<D, M>;
    using C = CoefArg<D, M>;
    C coef;
    if constexpr (S::kParam)
        std::memcpy(coef.v, a.coef_host, sizeof(coef.v));
    else
        coef.v = a.coef_dev;
    GridDesc g{{a.n[0], a.n[1], a.n[2]}, a.nnode};
    if (a.nsteps <= 0) return cudaSuccess;
    if (use_small<D, M>(a)) {
        const size_t smem = (size_t)(D + 1) * S::NQ * a.nnode * sizeof(double);
        cudaError_t e = cudaFuncSetAttribute(k_small<D, M, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int threads = (int)((a.nnode + 31) / 32 * 32);
        if (threads > 256) threads = 256;
        if (a.used_small) *a.used_small = true;
        if (a.ev) cudaEventRecord(a.ev[0], a.stream);
        k_small<D, M, C><<<1, threads, smem, a.stream>>>(a.P, a.U, g, coef, a.nsteps, a.status);
        if (a.ev) cudaEventRecord(a.ev[1], a.stream);
        return cudaGetLastError();
    }
    if (a.used_small) *a.used_small = false;
    const int blocks = (int)((a.nnode + 127) / 128);
    for (int64_t st = 0; st < a.nsteps; ++st) {
        if (a.ev) cudaEventRecord(a.ev[2 * st], a.stream);
        k_p_half<D, M, C><<<blocks, 128, 0, a.stream>>>(a.U, a.P, g, coef, a.status);
        if (a.src.active) {
            cudaError_t e = launch_source(a.src, a.P, a.nnode, S::NQ, a.step0 + st, a.stream);
            if (e != cudaSuccess) return e;
        }
        if (a.ev) cudaEventRecord(a.ev[2 * st + 1], a.stream);
        if constexpr (S::kUFused)
            k_u_half<D, M, 0, D, C><<<blocks, 128, 0, a.stream>>>(a.P, a.U, g, coef, a.status);
        else
            launch_u_split<D, M, 0, C>(a, g, coef, blocks);
    }
    if (a.ev) cudaEventRecord(a.ev[2 * a.nsteps], a.stream);
    return cudaGetLastError();
}

}  // namespace hl
