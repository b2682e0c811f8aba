// Digit planes of a field for the tensor-core split kernels (hl_tc3.cu, 3D;
// hl_tc2.cu, 2D): the field's largest binary exponent, then every value cut
// once into its 6 FP16 digit planes at that exponent (the digit scheme of
// hl_tc5.cuh).
//
// Layout: entry (c, i, ch, r, xe) is 16 bytes = 8 FP16 digits i of slots
// 8 ch .. 8 ch + 7 of component c at node row r = y + n1 z and x = xe - 1
// (xe = 0 and n0 + 1 are periodic ghost copies), so that the 129 partner nodes
// of a 128-node tile are one contiguous 2064-byte run for a bulk copy.
#pragma once

#include "hl_fp64.cuh"
#include "hl_tc5.cuh"

namespace hl {

// Largest biased binary exponent of a field (all components and slots) into
// *emax (which the caller zeroes first).  Non-finite values set status bit 1
// and are left out.  (Templated only so that every translation unit has its own.)
template <int Unused>
__global__ void __launch_bounds__(256) k_tc_emax(const double *__restrict__ F, int64_t n, int *emax,
                                                 unsigned *status)
{
    int e = 0;
    bool bad = false;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int ek = (__double2hiint(__ldg(F + k)) >> 20) & 0x7FF;
        bad |= ek == 0x7FF;
        e = max(e, ek == 0x7FF ? 0 : ek);
    }
    report_nonfinite(bad, status);
    e = __reduce_max_sync(0xFFFFFFFFu, e);
    if ((threadIdx.x & 31) == 0) atomicMax(emax, e);
}

// Cut every value of a field with NQ slots per component into its digit planes
// (CH chunks of 8 slots, the padding slots zero), at the field's exponent *emax:
// one thread per (component, row, xe); grid (xe blocks, n1, n2 * ncomp).
template <int NQ, int CH>
__global__ void __launch_bounds__(128) k_tc_cut(const double *__restrict__ F, uint4 *__restrict__ G, int ncomp,
                                                int n0, int n1, int n2, const int *__restrict__ emaxp)
{
    const int xe = blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.z / n2;
    const int r = blockIdx.y + n1 * (blockIdx.z % n2);
    if (xe >= n0 + 2 || c >= ncomp) return;
    int x = xe - 1;
    if (x < 0) x += n0;
    if (x >= n0) x -= n0;
    const int64_t nnode = (int64_t)n0 * n1 * n2;
    const int64_t node = x + (int64_t)n0 * r;
    const int emax = __ldg(emaxp);
    const int64_t R = (int64_t)n1 * n2, XE = n0 + 2;
    const double *src = F + (int64_t)c * NQ * nnode + node;
#pragma unroll
    for (int ch = 0; ch < CH; ++ch) {
        int64_t y[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int s = ch * 8 + k;
            y[k] = t5_fixed(s < NQ ? __ldg(src + (int64_t)s * nnode) : 0.0, emax);
        }
        uint32_t w[4][kT5Digits];
#pragma unroll
        for (int k = 0; k < 4; ++k) t5_digits_f16x2(y[2 * k], y[2 * k + 1], w[k]);
#pragma unroll
        for (int i = 0; i < kT5Digits; ++i)
            G[(((int64_t)(c * kT5Digits + i) * CH + ch) * R + r) * XE + xe] =
                make_uint4(w[0][i], w[1][i], w[2][i], w[3][i]);
    }
}

}  // namespace hl
