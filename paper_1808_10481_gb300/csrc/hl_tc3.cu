// Tensor-core split mode (HL_TC_SPLIT) in 3D, m = 2, on the tcgen05 tensor
// cores: the same exact digit scheme as the 2D kernels (hl_tc5.cuh), with three
// changes forced by the size of the 3D contraction.
//
//   * K is 648 (p-half: 3 velocity components x 8 vertices x 27 slots) or 216
//     (u-half), beyond the 128 products whose level sums FP32 holds exactly.
//     The MMAs therefore accumulate groups of K = 4 vertices x 27 slots (one
//     partner component and one z-layer of the cell's vertices) in TMEM, and the
//     epilogue drains every group into float-float running sums: 6 groups a tile.
//   * The operator image (344 KB a half-step) does not fit in shared memory: each
//     unit of work (a group's 16-slot half) streams its 28 KB of operator digits
//     with the data, by bulk copy.
//   * Cutting the partner data into digits inside the tile (as in 2D) would cut
//     every value 4 times (each node is a vertex of 4 tiles' cells along y and z);
//     instead one pass (k_tc_cut) cuts every partner value once per half-step into
//     digit planes in global memory, at one exponent per field (the field's
//     largest binary exponent: k_tc_emax at the first step of a call, afterwards
//     the maximum the kernel that wrote the field took over its outputs), and the
//     tensor-core kernel only copies digit rows into shared memory.
//
// Digit planes of a field with C components: entry (c, i, ch, r, xe) is 16 bytes
// = 8 FP16 digits i of slots 8 ch .. 8 ch + 7 of component c at node row
// r = y + n1 z and x = xe - 1 (xe = 0 and n0 + 1 are periodic ghost copies), so
// that the 129 partner nodes of a 128-node tile are one contiguous 2064-byte run.
//
// Tensor-core kernel (persistent, warp-specialised; one CTA per SM):
//   warp 0 (producer): per unit, 24 bulk copies of digit rows (6 digits x 2 slot
//     chunks x 2 y-rows) and one of the unit's operator digits into one of two
//     shared-memory stages -> a_full[stage] (transaction count);
//   warp 1, one lane (MMA): per unit 24 tcgen05.mma (6 data digits x 4 vertices,
//     all levels i + j <= 6 at once) into one of two TMEM accumulators; after a
//     group's two units, acc_full[acc];
//   warps 2-17 (epilogue, four per TMEM lane quarter, 8 output columns each):
//     levels of a group to float-float, added to the running sums; after the last
//     group of an output set, scale and add to the binary64 node values.
// Every wait is bounded; on expiry the abort flag and the status bit
// HL_ETIMEOUT are set and every role leaves; copies and MMAs in flight are
// waited for before the CTA releases its tensor memory and exits.
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

constexpr int kNQ = 27;                    // slots per node (m = 2)
constexpr int kChunks = 4;                 // 8-slot chunks (32 padded slots)
constexpr int kUnits = 12;                 // units per tile
constexpr int kGroups = 6;                 // drained accumulator groups per tile
constexpr int kRowBytes = kT5RX * 16;      // one copied digit row: 129 entries
constexpr int kBBytes = kTc3UnitElems * 2; // operator digits of one unit (28672)
constexpr int kStageBytes = kT5ABytes + kBBytes;
constexpr int kStages = 2;
constexpr int kTxBytes = 24 * kRowBytes + kBBytes;
constexpr int kEpiWarp0 = 2;
constexpr int kEpiWarps = 16;              // 4 per TMEM lane quarter, 8 of the 32 output columns each
constexpr int kThreads = 32 * (kEpiWarp0 + kEpiWarps);   // producer, MMA, epilogue warps
constexpr int kShares = kEpiWarps / 4;     // epilogue warps per lane quarter
constexpr int kCG = 4 / kShares;           // 8-column groups a thread
static_assert(kCG * kShares == 4, "role layout");
constexpr int kAccCols = 7 * 32;           // one accumulator: 7 levels x 32 columns
constexpr int kSmemBytes = kStages * kStageBytes + 8 * (4 * kStages + 1) + 16;
static_assert(kTxBytes < (1 << 20), "transaction count");

__device__ __forceinline__ void bulk_copy(uint32_t dst, const void *src, uint32_t bytes, uint32_t mbar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(mbar)
        : "memory");
}

__device__ __forceinline__ void mbar_arrive_tx(uint32_t mbar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mbar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive1(uint32_t mbar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(mbar) : "memory");
}

}  // namespace

// One half-step on the tensor cores.  PHALF: X = p, partner digits of u (3
// components), operator 0; else X = u (3 directions), partner digits of p.
template <bool PHALF>
__global__ void __launch_bounds__(kThreads, 1)
    k_half_tc3(const uint4 *__restrict__ G, double *__restrict__ X, int n0, int n1, int n2, int total_tiles,
               const uint4 *__restrict__ Bimg, const int *__restrict__ expo, const int *__restrict__ emaxp,
               int *emax_out, unsigned *status)
{
    extern __shared__ __align__(1024) unsigned char t3_sm[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(t3_sm + kStages * kStageBytes);
    uint64_t *a_full = bars, *a_empty = bars + kStages, *acc_full = bars + 2 * kStages,
             *acc_empty = acc_full + 2, *drain = acc_empty + 2;
    volatile int *abort_flag = reinterpret_cast<int *>(drain + 1);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(drain + 1) + 1;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int lo = PHALF ? -1 : 0;
    const int tiles_x = (n0 + kT5TileX - 1) / kT5TileX;
    const int64_t R = (int64_t)n1 * n2, XE = n0 + 2, nnode = (int64_t)n0 * R;

    if (warp == 0) {
        tmem_alloc(smem_addr(tmem_slot), 512);
        tc_fence_before();
    }
    if (tid == 32) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(smem_addr(a_full + s), 1);
            mbar_init(smem_addr(a_empty + s), 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(smem_addr(acc_full + a), 1);
            mbar_init(smem_addr(acc_empty + a), kEpiWarps * 32);
        }
        mbar_init(smem_addr(drain), 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ------------------------------------------------------------ producer
        int gu = 0;
        bool dead = false;
        for (int t = blockIdx.x; t < total_tiles && !dead; t += gridDim.x) {
            const int x0 = (t % tiles_x) * kT5TileX;
            const int yz = t / tiles_x;
            const int y = yz % n1, z = yz / n1;
            for (int u = 0; u < kUnits; ++u, ++gu) {
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
                const int comp = u / 4, vz = (u / 2) % 2, kh = u % 2;  // comp: component (p-half) or direction
                const int c = PHALF ? comp : 0;                         // digit planes' component
                unsigned char *stage = t3_sm + st * kStageBytes;
                if (lane == 0) mbar_arrive_tx(smem_addr(a_full + st), (uint32_t)kTxBytes);
                __syncwarp();
                if (lane < 24) {
                    const int i = lane >> 2, chl = (lane >> 1) & 1, vy = lane & 1;
                    int yy = y + lo + vy, zz = z + lo + vz;
                    if (yy < 0) yy += n1;
                    if (yy >= n1) yy -= n1;
                    if (zz < 0) zz += n2;
                    if (zz >= n2) zz -= n2;
                    const int64_t r = yy + (int64_t)n1 * zz;
                    const uint4 *src =
                        G + (((int64_t)(c * kT5Digits + i) * kChunks + 2 * kh + chl) * R + r) * XE + (x0 + lo + 1);
                    const uint32_t dst = smem_addr(stage + i * kT5Plane + chl * kT5Chunk + vy * kRowBytes);
                    bulk_copy(dst, src, (uint32_t)kRowBytes, smem_addr(a_full + st));
                } else if (lane == 24) {
                    bulk_copy(smem_addr(stage + kT5ABytes), Bimg + (size_t)u * (kBBytes / 16), (uint32_t)kBBytes,
                              smem_addr(a_full + st));
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
            int gu = 0, gg = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < total_tiles && ok; t += gridDim.x) {
                for (int g = 0; g < kGroups && ok; ++g, ++gg) {
                    if (*abort_flag) {
                        ok = false;
                        break;
                    }
                    const int ac = gg & 1;
                    if (gg >= 2 &&
                        !mbar_wait(smem_addr(acc_empty + ac), (uint32_t)(((gg >> 1) - 1) & 1), kT5WaitLimit)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    for (int kh = 0; kh < 2; ++kh, ++gu) {
                        const int st = gu % kStages;
                        if (!mbar_wait(smem_addr(a_full + st), (uint32_t)((gu / kStages) & 1), kT5WaitLimit)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t a0 = smem_addr(t3_sm + st * kStageBytes);
                        const uint32_t b0 = a0 + (uint32_t)kT5ABytes;
#pragma unroll
                        for (int i = 0; i < kT5Digits; ++i) {
                            const int nlev = i == 0 ? kT5Levels : min(kT5Digits, kT5Levels - i);
                            const uint32_t idesc = umma_idesc_f16(128, 32 * nlev);
#pragma unroll
                            for (int vv = 0; vv < 4; ++vv) {
                                const uint32_t arow = (uint32_t)((vv >> 1) * kT5RX + (vv & 1));
                                const uint64_t ad = umma_desc(a0 + (uint32_t)(i * kT5Plane) + arow * 16u, kT5Chunk, 128);
                                const uint64_t bd = umma_desc(b0 + (uint32_t)(vv * 2 * kAccCols * 16), kAccCols * 16, 128);
                                umma_bf16(tmem + (uint32_t)(ac * kAccCols + 32 * i), ad, bd, idesc,
                                          (kh | i | vv) != 0 ? 1u : 0u);
                            }
                        }
                        umma_commit(smem_addr(a_empty + st));
                    }
                    if (!ok) break;
                    umma_commit(smem_addr(acc_full + ac));
                }
            }
            if (!ok) {
                *abort_flag = 1;
                atomicOr(status, kStatusTimeout);
            }
            // every MMA issued has completed before the tensor memory is released
            umma_commit(smem_addr(drain));
            mbar_wait(smem_addr(drain), 0u, kT5WaitLimit);
        }
    } else {
        // ------------------------------------------------------------ epilogue
        const int quarter = warp & 3;                  // the TMEM lanes this warp may read
        const int share = (warp - kEpiWarp0) >> 2;     // output columns 8 kCG share ...
        const int q = 32 * quarter + lane;             // node within the tile = TMEM lane
        const uint32_t tl = tmem + ((uint32_t)(32 * quarter) << 16);
        constexpr int GPS = PHALF ? 6 : 2;             // groups per output set
        const int E = __ldg(emaxp) - 1022;
        int gg = 0, emx = 0;  // emx: largest biased exponent written (the next cut's field exponent)
        bool bad = false;
        for (int t = blockIdx.x; t < total_tiles; t += gridDim.x) {
            if (*abort_flag) break;
            const int x0 = (t % tiles_x) * kT5TileX;
            const int yz = t / tiles_x;
            const int gx = x0 + q;
            const bool mine = gx < n0;
            const int64_t node = (int64_t)gx + (int64_t)n0 * yz;
            FF run[kCG][8];
            double own[kCG][8];
            bool quit = false;
            for (int g = 0; g < kGroups; ++g, ++gg) {
                const int os = g / GPS;  // output set: 0 (p) or the direction of u
                if (g % GPS == 0) {
#pragma unroll
                    for (int cg = 0; cg < kCG; ++cg)
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const int s = 8 * (kCG * share + cg) + j;
                            run[cg][j] = FF{0.f, 0.f};
                            own[cg][j] = (mine && s < kNQ) ? X[(int64_t)(os * kNQ + s) * nnode + node] : 0.0;
                        }
                }
                const int ac = gg & 1;
                if (!mbar_wait(smem_addr(acc_full + ac), (uint32_t)((gg >> 1) & 1), kT5WaitLimit)) {
                    *abort_flag = 1;
                    atomicOr(status, kStatusTimeout);
                    quit = true;
                    break;
                }
                tc_fence_after();
#pragma unroll
                for (int cg = 0; cg < kCG; ++cg) {
                    const int col0 = 8 * (kCG * share + cg);
                    FF tot[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) tot[j] = FF{0.f, 0.f};
#pragma unroll
                    for (int batch = 0; batch < 2; ++batch) {
                        const int Lhi = batch == 0 ? kT5Levels - 1 : 2, Llo = batch == 0 ? 3 : 0;
                        float accv[4][8];
#pragma unroll
                        for (int L = Lhi; L >= Llo; --L)
                            tmem_ld8(tl + (uint32_t)(ac * kAccCols + 32 * L + col0), accv[Lhi - L]);
                        tmem_ld_wait();
#pragma unroll
                        for (int L = Lhi; L >= Llo; --L)
#pragma unroll
                            for (int j = 0; j < 8; ++j) {
                                const float val = accv[Lhi - L][j] * __uint_as_float((uint32_t)(127 - 8 * L) << 23);
                                if (L >= 4) {
                                    tot[j].hi = __fadd_rn(tot[j].hi, val);
                                } else {
                                    const FF s2 = ff_two_sum(tot[j].hi, val);
                                    tot[j].hi = s2.hi;
                                    tot[j].lo = __fadd_rn(tot[j].lo, s2.lo);
                                }
                            }
                    }
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const FF s2 = ff_two_sum(run[cg][j].hi, tot[j].hi);
                        run[cg][j].hi = s2.hi;
                        run[cg][j].lo = __fadd_rn(__fadd_rn(run[cg][j].lo, tot[j].lo), s2.lo);
                    }
                }
                tc_fence_before();
                mbar_arrive1(smem_addr(acc_empty + ac));
                if (g % GPS == GPS - 1 && mine) {
                    const int op = PHALF ? 0 : 1 + os;
#pragma unroll
                    for (int cg = 0; cg < kCG; ++cg)
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const int s = 8 * (kCG * share + cg) + j;
                            if (s >= kNQ) continue;
                            const FF nrm = ff_two_sum(run[cg][j].hi, run[cg][j].lo);
                            const int k0 = E + __ldg(expo + op * 32 + s) - 14;
                            const double inc = t5_scaled_f64(nrm.hi, k0) + t5_scaled_f64(nrm.lo, k0);
                            const double nv = own[cg][j] + inc;
                            X[(int64_t)(os * kNQ + s) * nnode + node] = nv;
                            const int ev = (__double2hiint(nv) >> 20) & 0x7FF;
                            bad |= ev == 0x7FF;
                            emx = max(emx, ev == 0x7FF ? 0 : ev);
                        }
                }
            }
            if (quit) break;
        }
        report_nonfinite(bad, status);
        emx = __reduce_max_sync(0xFFFFFFFFu, emx);
        if (lane == 0) atomicMax(emax_out, emx);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 512);
}

cudaError_t launch_tc_d3(const LaunchFp64 &a)
{
    if (a.m != 2 || a.n_shots != 1 || !a.tc_digits || !a.tc_expo || !a.tc3_gu || !a.tc3_gp || !a.tc3_emax)
        return cudaErrorInvalidValue;
    static std::atomic<uint64_t> opted_in{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const uint64_t bit = 1ull << (dev & 63);
    if (!(opted_in.load() & bit)) {
        if ((e = cudaFuncSetAttribute(k_half_tc3<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes)) !=
                cudaSuccess ||
            (e = cudaFuncSetAttribute(k_half_tc3<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes)) !=
                cudaSuccess)
            return e;
        opted_in.fetch_or(bit);
    }
    int sms = 0;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const int n0 = a.n[0], n1 = a.n[1], n2 = a.n[2];
    const int64_t nnode = (int64_t)n0 * n1 * n2;
    const int tiles = ((n0 + kT5TileX - 1) / kT5TileX) * n1 * n2;
    const dim3 grid((unsigned)std::min(tiles, sms));
    const unsigned cut_x = (unsigned)((n0 + 2 + 127) / 128);
    const uint4 *bp = reinterpret_cast<const uint4 *>(a.tc_digits);
    const uint4 *bu = reinterpret_cast<const uint4 *>(a.tc_digits + kTc3ImageElems / 2);
    const unsigned red_blocks = (unsigned)std::min<int64_t>((nnode * 3 * kNQ + 255) / 256, 8 * sms);
    int *emax_u = a.tc3_emax, *emax_p = a.tc3_emax + 1;
    // Field exponents: each tensor-core kernel takes the largest exponent of the values it
    // writes (atomic maximum over its warps), which the next half-step's cut of that field
    // uses; only the first step of a call (the state may have been set or changed since) and
    // a point source (it adds to p after the p-half) need the separate pass.
    const bool src = a.src && a.src->active;
    for (int64_t st = 0; st < a.nsteps; ++st) {
        if (a.ev) cudaEventRecord(a.ev[2 * st], a.stream);
        // p-half: the velocity's digit planes, then the products
        if (st == 0) {
            if ((e = cudaMemsetAsync(emax_u, 0, sizeof(int), a.stream)) != cudaSuccess) return e;
            k_tc_emax<0><<<red_blocks, 256, 0, a.stream>>>(a.U, nnode * 3 * kNQ, emax_u, a.status);
        }
        k_tc_cut<kNQ, kChunks><<<dim3(cut_x, (unsigned)n1, (unsigned)(3 * n2)), 128, 0, a.stream>>>(a.U, a.tc3_gu, 3, n0, n1, n2, emax_u);
        if ((e = cudaMemsetAsync(emax_p, 0, sizeof(int), a.stream)) != cudaSuccess) return e;
        k_half_tc3<true><<<grid, kThreads, kSmemBytes, a.stream>>>(a.tc3_gu, a.P, n0, n1, n2, tiles, bp, a.tc_expo,
                                                                   emax_u, emax_p, a.status);
        if (src) {
            if ((e = launch_source(*a.src, a.shots, a.P, kNQ, a.step0 + st, a.stream)) != cudaSuccess) return e;
            if ((e = cudaMemsetAsync(emax_p, 0, sizeof(int), a.stream)) != cudaSuccess) return e;
            k_tc_emax<0><<<red_blocks, 256, 0, a.stream>>>(a.P, nnode * kNQ, emax_p, a.status);
        }
        if (a.ev) cudaEventRecord(a.ev[2 * st + 1], a.stream);
        k_tc_cut<kNQ, kChunks><<<dim3(cut_x, (unsigned)n1, (unsigned)n2), 128, 0, a.stream>>>(a.P, a.tc3_gp, 1, n0, n1, n2, emax_p);
        if ((e = cudaMemsetAsync(emax_u, 0, sizeof(int), a.stream)) != cudaSuccess) return e;
        k_half_tc3<false><<<grid, kThreads, kSmemBytes, a.stream>>>(a.tc3_gp, a.U, n0, n1, n2, tiles, bu, a.tc_expo,
                                                                    emax_p, emax_u, a.status);
    }
    if (a.ev) cudaEventRecord(a.ev[2 * a.nsteps], a.stream);
    return cudaGetLastError();
}

}  // namespace hl
