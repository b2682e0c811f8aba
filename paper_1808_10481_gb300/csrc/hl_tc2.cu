// Tensor-core split mode (HL_TC_SPLIT) in 2D on one grid, m <= 3: the digit
// scheme of hl_tc5.cuh with the partner field cut once per half-step into
// global digit planes (hl_tc_planes.cuh), as in 3D, instead of inside every
// tile.  The in-tile cut of k_half_tc6 cuts every partner value twice (each
// node is a vertex of the tiles of two grid rows) and keeps that kernel issue-
// bound on the integer pipe; here the tile kernel only copies digit rows.
//
// Per tile (128 nodes of one grid row) and partner component ("unit"): 24 bulk
// copies (6 digits x 2 slot chunks x 2 grid rows) into one of 3 shared-memory
// stages; one lane issues 24 tcgen05.mma (6 data digits x 4 vertices, all levels
// i + j <= 6 at once) into one of two TMEM accumulators; 8 (p-half) or 16
// (u-half) epilogue warps combine the 7 levels in float-float, scale by the
// field exponent and add to the binary64 values.  K = 2 x 4 x 16 = 128 (p-half)
// or 64 (u-half): one exact accumulation per tile.  The operator image of the
// half (28 KB, build_tc5_images) stays in shared memory.
//
// The field exponent is taken by k_tc_emax at the first step of a call and
// after a point source; otherwise it is the largest exponent the kernel that
// wrote the field took over its outputs.  Batches of shots run k_half_tc6.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>

#include "hl_fp64.cuh"
#include "hl_internal.h"
#include "hl_sm100.cuh"
#include "hl_split.cuh"
#include "hl_tc5.cuh"
#include "hl_tc_planes.cuh"

namespace hl {

namespace {

constexpr int kCh = 2;                       // 8-slot chunks (16 padded slots)
constexpr int kRowBytes = kT5RX * 16;        // one copied digit row: 129 entries
constexpr int kStages = 3;
constexpr int kTxBytes = 24 * kRowBytes;
constexpr int kEpiWarp0 = 2;
// Roles: warp 0 producer, warp 1 MMA, then EW epilogue warps, EW / 4 per TMEM lane quarter,
// each owning 8 of the node's output columns (p-half: 16 columns, 8 warps, plus 2 idle warps
// that only reach the final barrier, so that the register split gives 168 a thread; u-half:
// 32 columns, 16 warps)
template <bool PHALF>
struct T2Roles {
    static constexpr int EW = PHALF ? 8 : 16;
    static constexpr int THREADS = PHALF ? 384 : 576;
    static constexpr int NGRP = (PHALF ? 2 : 4) / (EW / 4);   // 8-column groups a thread
    static_assert(THREADS / 32 >= kEpiWarp0 + EW && NGRP * (EW / 4) == (PHALF ? 2 : 4), "role layout");
};
constexpr int kSmemBytes = kT5BBytes + kStages * kT5ABytes + 8 * (2 * kStages + 5) + 16;
static_assert(kSmemBytes <= 227 * 1024, "shared memory");

__device__ __forceinline__ void bulk_copy2(uint32_t dst, const void *src, uint32_t bytes, uint32_t mbar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(mbar)
        : "memory");
}

__device__ __forceinline__ void mbar_arrive_tx2(uint32_t mbar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mbar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive2(uint32_t mbar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(mbar) : "memory");
}

}  // namespace

// One half-step.  PHALF: X = p (NQ slots), partner digit planes of u (2
// components); else X = u (2 directions), partner digit planes of p.
template <int M, bool PHALF>
__global__ void __launch_bounds__(T2Roles<PHALF>::THREADS, 1)
    k_half_tc2(const uint4 *__restrict__ G, double *__restrict__ X, int n0, int n1, int total_tiles,
               const uint4 *__restrict__ Bimg, const int *__restrict__ expo, const int *__restrict__ emaxp,
               int *emax_out, unsigned *status)
{
    constexpr int NQ = (M + 1) * (M + 1);
    constexpr int NCIN = PHALF ? 2 : 1;
    using Op = T5Op<PHALF>;
    using R = T2Roles<PHALF>;
    extern __shared__ __align__(1024) unsigned char t2_sm[];
    unsigned char *Bs = t2_sm;
    unsigned char *As = t2_sm + kT5BBytes;
    uint64_t *bars = reinterpret_cast<uint64_t *>(As + kStages * kT5ABytes);
    uint64_t *a_full = bars, *a_empty = bars + kStages, *acc_full = bars + 2 * kStages,
             *acc_empty = acc_full + 2, *drain = acc_empty + 2;
    volatile int *abort_flag = reinterpret_cast<int *>(drain + 1);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(drain + 1) + 1;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int lo = PHALF ? -1 : 0;
    const int tiles_x = (n0 + kT5TileX - 1) / kT5TileX;
    const int64_t XE = n0 + 2, nnode = (int64_t)n0 * n1;

    if (warp == 0) {
        tmem_alloc(smem_addr(tmem_slot), 2 * Op::TCOLS);
        tc_fence_before();
    }
    if (tid == 32) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(smem_addr(a_full + s), 1);
            mbar_init(smem_addr(a_empty + s), 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(smem_addr(acc_full + a), 1);
            mbar_init(smem_addr(acc_empty + a), R::EW * 32);
        }
        mbar_init(smem_addr(drain), 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    // the half's operator image, once per CTA
    for (int e = tid; e < kT5BBytes / 16; e += R::THREADS) reinterpret_cast<uint4 *>(Bs)[e] = __ldg(Bimg + e);
    fence_async_smem();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ------------------------------------------------------------ producer
        int gu = 0;
        bool dead = false;
        for (int t = blockIdx.x; t < total_tiles && !dead; t += gridDim.x) {
            const int x0 = (t % tiles_x) * kT5TileX;
            const int y = t / tiles_x;
            for (int c = 0; c < NCIN; ++c, ++gu) {
                const int st = gu % kStages;
                if (*abort_flag) {
                    dead = true;
                    break;
                }
                if (gu >= kStages &&
                    !mbar_wait(smem_addr(a_empty + st), (uint32_t)(((gu / kStages) - 1) & 1), kT5WaitLimit)) {
                    *abort_flag = 1;
                    if (lane == 0) atomicOr(status, kStatusTimeout);
                    dead = true;
                    break;
                }
                unsigned char *stage = As + st * kT5ABytes;
                if (lane == 0) mbar_arrive_tx2(smem_addr(a_full + st), (uint32_t)kTxBytes);
                __syncwarp();
                if (lane < 24) {
                    const int i = lane >> 2, ch = (lane >> 1) & 1, vy = lane & 1;
                    int yy = y + lo + vy;
                    if (yy < 0) yy += n1;
                    if (yy >= n1) yy -= n1;
                    const uint4 *src = G + (((int64_t)(c * kT5Digits + i) * kCh + ch) * n1 + yy) * XE + (x0 + lo + 1);
                    const uint32_t dst = smem_addr(stage + i * kT5Plane + ch * kT5Chunk + vy * kRowBytes);
                    bulk_copy2(dst, src, (uint32_t)kRowBytes, smem_addr(a_full + st));
                }
                __syncwarp();
            }
        }
        // copies still in flight land before the CTA leaves
        if (lane == 0) {
            for (int g = max(0, gu - kStages); g < gu; ++g)
                mbar_wait(smem_addr(a_full + g % kStages), (uint32_t)((g / kStages) & 1), kT5WaitLimit);
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issue (one lane)
        if (lane == 0) {
            const uint32_t b0 = smem_addr(Bs);
            int gu = 0, lt = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < total_tiles && ok; t += gridDim.x, ++lt) {
                if (*abort_flag) {
                    ok = false;
                    break;
                }
                const int ac = lt & 1;
                if (lt >= 2 && !mbar_wait(smem_addr(acc_empty + ac), (uint32_t)(((lt >> 1) - 1) & 1), kT5WaitLimit)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                for (int c = 0; c < NCIN; ++c, ++gu) {
                    const int st = gu % kStages;
                    if (!mbar_wait(smem_addr(a_full + st), (uint32_t)((gu / kStages) & 1), kT5WaitLimit)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a0 = smem_addr(As + st * kT5ABytes);
#pragma unroll
                    for (int i = 0; i < kT5Digits; ++i) {
                        const int nlev = i == 0 ? kT5Levels : min(kT5Digits, kT5Levels - i);
                        const uint32_t idesc = umma_idesc_f16(128, Op::NPL * nlev);
#pragma unroll
                        for (int vtx = 0; vtx < 4; ++vtx) {
                            const uint32_t arow = (uint32_t)((vtx >> 1) * kT5RX + (vtx & 1));
                            const uint64_t ad = umma_desc(a0 + (uint32_t)(i * kT5Plane) + arow * 16u, kT5Chunk, 128);
                            const int kb = PHALF ? c * 4 + vtx : vtx;
                            const uint64_t bd = umma_desc(b0 + (uint32_t)(kb * Op::KB_BYTES), Op::NROWS * 16, 128);
                            umma_bf16(tmem + (uint32_t)(ac * Op::TCOLS + Op::NPL * i), ad, bd, idesc,
                                      (c | i | vtx) != 0 ? 1u : 0u);
                        }
                    }
                    umma_commit(smem_addr(a_empty + st));
                }
                if (!ok) break;
                umma_commit(smem_addr(acc_full + ac));
            }
            if (!ok) {
                *abort_flag = 1;
                atomicOr(status, kStatusTimeout);
            }
            // every MMA issued has completed before the tensor memory is released
            umma_commit(smem_addr(drain));
            mbar_wait(smem_addr(drain), 0u, kT5WaitLimit);
        }
    } else if (warp < kEpiWarp0 + R::EW) {
        // ------------------------------------------------------------ epilogue
        const int quarter = warp & 3;                  // the TMEM lanes this warp may read
        const int half = (warp - kEpiWarp0) >> 2;      // which share of the node's outputs
        const int q = 32 * quarter + lane;             // node within the tile = TMEM lane
        const uint32_t tl = tmem + ((uint32_t)(32 * quarter) << 16);
        constexpr int NGRP = R::NGRP;                  // groups of 8 output columns per thread
        const int E = __ldg(emaxp) - 1022;
        int lt = 0, emx = 0;
        bool bad = false;
        for (int t = blockIdx.x; t < total_tiles; t += gridDim.x, ++lt) {
            if (*abort_flag) break;
            const int x0 = (t % tiles_x) * kT5TileX;
            const int y = t / tiles_x;
            const int gx = x0 + q;
            const bool mine = gx < n0;
            const int64_t node = (int64_t)gx + (int64_t)n0 * y;
            const int ac = lt & 1;
            auto load_own = [&](int g, double *o) {
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int col = 8 * (NGRP * half + g) + j;  // within a level: component col / 16
                    const int s = col % 16, oc = col / 16;
                    o[j] = (mine && s < NQ) ? X[(int64_t)(oc * NQ + s) * nnode + node] : 0.0;
                }
            };
            double own[8], nxt[8];
            load_own(0, own);  // in flight while this tile's MMAs run
            if (!mbar_wait(smem_addr(acc_full + ac), (uint32_t)((lt >> 1) & 1), kT5WaitLimit)) {
                *abort_flag = 1;
                atomicOr(status, kStatusTimeout);
                break;
            }
            tc_fence_after();
#pragma unroll
            for (int g = 0; g < NGRP; ++g) {
                const int col0 = 8 * (NGRP * half + g);
                if (g + 1 < NGRP) load_own(g + 1, nxt);  // the next group's values, during this one
                FF tot[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) tot[j] = FF{0.f, 0.f};
#pragma unroll
                for (int batch = 0; batch < 2; ++batch) {
                    const int Lhi = batch == 0 ? kT5Levels - 1 : 2, Llo = batch == 0 ? 3 : 0;
                    float accv[4][8];
#pragma unroll
                    for (int L = Lhi; L >= Llo; --L)
                        tmem_ld8(tl + (uint32_t)(ac * Op::TCOLS + L * Op::NPL + col0), accv[Lhi - L]);
                    tmem_ld_wait();
#pragma unroll
                    for (int L = Lhi; L >= Llo; --L)
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const float val = accv[Lhi - L][j] * __uint_as_float((uint32_t)(127 - 8 * L) << 23);
                            if (L >= 4) {
                                // levels 6..4 in plain FP32: their rounding stays under 2^-54
                                // of the top level's scale
                                tot[j].hi = __fadd_rn(tot[j].hi, val);
                            } else {
                                const FF s2 = ff_two_sum(tot[j].hi, val);
                                tot[j].hi = s2.hi;
                                tot[j].lo = __fadd_rn(tot[j].lo, s2.lo);
                            }
                        }
                }
                if (mine) {
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int s = (col0 + j) % 16, oc = (col0 + j) / 16;
                        if (s >= NQ) continue;
                        const FF nrm = ff_two_sum(tot[j].hi, tot[j].lo);
                        const int k0 = E + __ldg(expo + oc * 16 + s) - 14;
                        const double inc = t5_scaled_f64(nrm.hi, k0) + t5_scaled_f64(nrm.lo, k0);
                        const double nv = own[j] + inc;
                        X[(int64_t)(oc * NQ + s) * nnode + node] = nv;
                        const int ev = (__double2hiint(nv) >> 20) & 0x7FF;
                        bad |= ev == 0x7FF;
                        emx = max(emx, ev == 0x7FF ? 0 : ev);
                    }
                }
                if (g + 1 < NGRP) {
#pragma unroll
                    for (int j = 0; j < 8; ++j) own[j] = nxt[j];
                }
            }
            tc_fence_before();
            mbar_arrive2(smem_addr(acc_empty + ac));
        }
        report_nonfinite(bad, status);
        emx = __reduce_max_sync(0xFFFFFFFFu, emx);
        if (lane == 0) atomicMax(emax_out, emx);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 2 * Op::TCOLS);
}

template <int M>
static cudaError_t run_tc2(const LaunchFp64 &a)
{
    constexpr int NQ = (M + 1) * (M + 1);
    static std::atomic<uint64_t> opted_in{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const uint64_t bit = 1ull << (dev & 63);
    if (!(opted_in.load() & bit)) {
        if ((e = cudaFuncSetAttribute(k_half_tc2<M, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      kSmemBytes)) != cudaSuccess ||
            (e = cudaFuncSetAttribute(k_half_tc2<M, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      kSmemBytes)) != cudaSuccess)
            return e;
        opted_in.fetch_or(bit);
    }
    int sms = 0;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const int n0 = a.n[0], n1 = a.n[1];
    const int64_t nnode = (int64_t)n0 * n1;
    const int tiles = ((n0 + kT5TileX - 1) / kT5TileX) * n1;
    const dim3 grid((unsigned)std::min(tiles, sms));
    const unsigned cut_x = (unsigned)((n0 + 2 + 127) / 128);
    const uint4 *bp = reinterpret_cast<const uint4 *>(a.tc_digits);
    const uint4 *bu = reinterpret_cast<const uint4 *>(a.tc_digits + kT5BBytes / 2);
    const unsigned red_blocks = (unsigned)std::min<int64_t>((nnode * 2 * NQ + 255) / 256, 8 * sms);
    int *emax_u = a.tc3_emax, *emax_p = a.tc3_emax + 1;
    const bool src = a.src && a.src->active;
    for (int64_t st = 0; st < a.nsteps; ++st) {
        if (a.ev) cudaEventRecord(a.ev[2 * st], a.stream);
        if (st == 0) {
            if ((e = cudaMemsetAsync(emax_u, 0, sizeof(int), a.stream)) != cudaSuccess) return e;
            k_tc_emax<0><<<red_blocks, 256, 0, a.stream>>>(a.U, nnode * 2 * NQ, emax_u, a.status);
        }
        k_tc_cut<NQ, kCh><<<dim3(cut_x, (unsigned)n1, 2u), 128, 0, a.stream>>>(a.U, a.tc3_gu, 2, n0, n1, 1, emax_u);
        if ((e = cudaMemsetAsync(emax_p, 0, sizeof(int), a.stream)) != cudaSuccess) return e;
        k_half_tc2<M, true><<<grid, T2Roles<true>::THREADS, kSmemBytes, a.stream>>>(a.tc3_gu, a.P, n0, n1, tiles, bp, a.tc_expo,
                                                                      emax_u, emax_p, a.status);
        if (src) {
            if ((e = launch_source(*a.src, a.shots, a.P, NQ, a.step0 + st, a.stream)) != cudaSuccess) return e;
            if ((e = cudaMemsetAsync(emax_p, 0, sizeof(int), a.stream)) != cudaSuccess) return e;
            k_tc_emax<0><<<red_blocks, 256, 0, a.stream>>>(a.P, nnode * NQ, emax_p, a.status);
        }
        if (a.ev) cudaEventRecord(a.ev[2 * st + 1], a.stream);
        k_tc_cut<NQ, kCh><<<dim3(cut_x, (unsigned)n1, 1u), 128, 0, a.stream>>>(a.P, a.tc3_gp, 1, n0, n1, 1, emax_p);
        if ((e = cudaMemsetAsync(emax_u, 0, sizeof(int), a.stream)) != cudaSuccess) return e;
        k_half_tc2<M, false><<<grid, T2Roles<false>::THREADS, kSmemBytes, a.stream>>>(a.tc3_gp, a.U, n0, n1, tiles, bu,
                                                                       a.tc_expo + 16, emax_p, emax_u, a.status);
    }
    if (a.ev) cudaEventRecord(a.ev[2 * a.nsteps], a.stream);
    return cudaGetLastError();
}

// 2D, one shot, digit planes allocated (tc3_gu/gp/emax): the precut kernels.
cudaError_t launch_tc2_planes(const LaunchFp64 &a)
{
    if (a.n_shots != 1 || !a.tc_digits || !a.tc_expo || !a.tc3_gu || !a.tc3_gp || !a.tc3_emax)
        return cudaErrorInvalidValue;
    switch (a.m) {
    case 0: return run_tc2<0>(a);
    case 1: return run_tc2<1>(a);
    case 2: return run_tc2<2>(a);
    case 3: return run_tc2<3>(a);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace hl
