// Tensor-core split mode (HL_TC_SPLIT), dim = 2, m <= 3, on the fifth-generation
// tensor cores: tcgen05.mma with the accumulators in tensor memory (TMEM),
// operands in shared memory, binary64 node data read and written directly.
//
// The half-step increment of a node is a dot product of the partner data at
// the cell's 4 vertices (K = partner component x vertex x slot) with the vertex
// form of the fused operator (one column per output slot; Section 2, eqs.
// interp and final1; Section 5).  Both sides are cut into 6 balanced base-256
// digits after a power-of-two scaling, so every digit product is an exact
// integer and the sums of one level of digit pairs stay exact in FP32:
//
//   data:     x = v 2^-E, |x| < 1, the block's largest binary exponent E;
//             X = trunc(x 2^48) (an integer of 48 bits), written as
//             X = sum_i d_i 256^(5-i), d_0 in [-256, 256], d_i in [-128, 127];
//   operator: column n scaled by 2^-e_n and cut into 6 digits in [-128, 127]
//             (host tables, build_tc_tables); a 7th zero digit row lets the
//             first MMA initialise every level's accumulator.
//
// Level L = i + j (i data digit, j operator digit) weighs 2^(E + e_n - 14 - 8L).
// Per level and output the sum over the K = 128 (p-half) or 64 (u-half) terms
// of at most 6 digit pairs is below 128 (2^15 + 5 2^14) < 2^24, so the tensor
// core's FP32 accumulation is exact.  Levels L <= 6 are formed (26 digit
// pairs); the epilogue sums them in float-float, scales by 2^(E + e_n - 14)
// and adds the increment to the binary64 value.  Quantisation to 48 bits below
// the block maximum and the dropped levels bound the error by a few 2^-46 of
// max|data| times the operator's column sums per half-step.
//
// A tile is 128 nodes of one grid row (the MMA's M = 128 rows);
// its region is the 129 x 2 partner nodes of the tile's cells.  The digits of
// the region are stored once per partner component; the 4 vertex operands are
// the same digit planes read from 4 different start rows (vertex (vx, vy) of
// node q is region row q + vx + 129 vy), so no data is duplicated per vertex.
// Per component and digit i one MMA per vertex multiplies that A (128 x 16)
// by the operator digits of all levels at once (N = 16 or 32 output columns
// per level, times the levels i+j <= 6) into TMEM columns starting at level i.
//
// The kernel is persistent (one CTA per SM walking the tiles) and warp-
// specialised: producer warps cut the region into digit planes in a ring of
// shared-memory stages, one lane issues the MMAs into one of two TMEM
// accumulators, and epilogue warps combine the levels of the previous tile, so
// that cutting, products and combination of successive tiles overlap.
#pragma once

#include <algorithm>
#include <atomic>

#include "hl_fp64.cuh"
#include "hl_sm100.cuh"
#include "hl_split.cuh"
#include "hl_tc_bits.cuh"

namespace hl {

constexpr int kT5TileX = 128;                 // nodes per tile (MMA rows)
constexpr int kT5RX = kT5TileX + 1;           // region nodes per grid row
constexpr int kT5Rows = 2 * kT5RX;            // region nodes (two grid rows)
constexpr int kT5RowsPad = 264;               // rows of a digit plane (multiple of 8)
constexpr int kT5Levels = 7;
constexpr int kT5Chunk = kT5RowsPad * 16;     // bytes of one 8-slot plane: 264 rows of 16 B
constexpr int kT5Plane = 2 * kT5Chunk;        // one digit of one component (16 slots)
constexpr int kT5ABytes = kT5Digits * kT5Plane;
constexpr int kT5BBytes = 28672;              // operator image of one half-step (either half)
constexpr uint32_t kT5WaitLimit = kMbarWaitLimit;

// Operator image of one half (host-built, build_tc5_images): blocks kb of
// [2 chunks][7 NPL rows][8 BF16], kb = component * 4 + vertex (p-half, NPL = 16)
// or vertex (u-half, NPL = 32, rows n = j * 32 + direction * 16 + slot).
template <bool PHALF>
struct T5Op {
    static constexpr int NPL = PHALF ? 16 : 32;        // output columns per level
    static constexpr int NROWS = kT5Levels * NPL;      // B rows (digit j = 0..6)
    static constexpr int KB_BYTES = 2 * NROWS * 16;
    static constexpr int TCOLS = PHALF ? 128 : 256;    // TMEM allocation
    static_assert((PHALF ? 8 : 4) * KB_BYTES == kT5BBytes, "operator image size");
};

// The six digits of two biased fixed-point values a and b (adjacent slots) as
// FP16 pairs, w[i] = (digit i of a, digit i of b), low half first.  Digits 1..5
// are the biased bytes 4..0: one byte permutation puts each under the exponent
// of 2^10 (FP16 0x64XX = 1024 + byte), one packed subtraction of 1024 + 128
// leaves the digit, exact.  Digit 0 = y >> 40 in [-256, 256] goes in as
// 1024 + 512 + d0 and comes out by subtracting 1536.
__device__ __forceinline__ uint32_t t5_sub_f16x2(uint32_t x, uint32_t c)
{
    uint32_t r;
    asm("sub.rn.f16x2 %0, %1, %2;\n" : "=r"(r) : "r"(x), "r"(c));
    return r;
}

__device__ __forceinline__ void t5_digits_f16x2(int64_t a, int64_t b, uint32_t (&w)[kT5Digits])
{
    t5_digit_words(a, b, w);
#pragma unroll
    for (int i = 1; i < kT5Digits; ++i) w[i] = t5_sub_f16x2(w[i], kT5SubLow);
    w[0] = t5_sub_f16x2(w[0], kT5SubTop);
}

// the 6 digit-plane entries (16 bytes each) of one 8-slot chunk of one region row
__device__ __forceinline__ void t5_store_chunk(unsigned char *As, int row, int ch, const int64_t (&y)[8])
{
    uint32_t w[4][kT5Digits];
#pragma unroll
    for (int k = 0; k < 4; ++k) t5_digits_f16x2(y[2 * k], y[2 * k + 1], w[k]);
#pragma unroll
    for (int i = 0; i < kT5Digits; ++i)
        *reinterpret_cast<uint4 *>(As + i * kT5Plane + ch * kT5Chunk + row * 16) =
            make_uint4(w[0][i], w[1][i], w[2][i], w[3][i]);
}

// Cut the (up to 16) slot values of one region node into its 6 digit planes:
// src + q * nnode is slot q of the node (slots >= NQ are zero).
template <int NQ>
__device__ __forceinline__ void t5_store_row(unsigned char *As, int row, const double *__restrict__ src,
                                             int64_t nnode, int emax)
{
#pragma unroll
    for (int ch = 0; ch < 2; ++ch) {
        if (ch * 8 >= NQ && ch > 0) {  // a chunk of padding slots: zero digits
#pragma unroll
            for (int i = 0; i < kT5Digits; ++i)
                *reinterpret_cast<uint4 *>(As + i * kT5Plane + ch * kT5Chunk + row * 16) = make_uint4(0u, 0u, 0u, 0u);
            continue;
        }
        int64_t y[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) y[k] = t5_fixed(ch * 8 + k < NQ ? __ldg(src + (int64_t)(ch * 8 + k) * nnode) : 0.0, emax);
        t5_store_chunk(As, row, ch, y);
    }
}

// as t5_store_row, from values already in registers
template <int NQ>
__device__ __forceinline__ void t5_store_row_regs(unsigned char *As, int row, const double (&v)[NQ], int emax)
{
#pragma unroll
    for (int ch = 0; ch < 2; ++ch) {
        int64_t y[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) y[k] = t5_fixed(ch * 8 + k < NQ ? v[(ch * 8 + k) % NQ] : 0.0, emax);
        t5_store_chunk(As, row, ch, y);
    }
}

// ---------------------------------------------------------------------------
// Persistent, warp-specialised kernel: one CTA per
// SM walks the tiles t = blockIdx.x, blockIdx.x + gridDim.x, ...; per tile and
// partner component ("unit") the roles hand data along mbarriers:
//   producers (warps 0..PW-1): load their region rows, take the tile's exponent,
//     cut the component into its digit planes in one of kT6Stages shared-memory
//     stages  -> a_full[stage]
//   MMA (warp PW, one lane): per unit 24 tcgen05.mma into one of two TMEM
//     accumulators  -> a_empty[stage] (stage free), acc_full[acc] after the
//     tile's last unit
//   epilogue (the EW warps after it, EW/4 per TMEM lane quarter: one node per
//     thread, the node's outputs split between the quarter's warps): the node's own
//     values are loaded ahead (the first group while the MMAs run, the next while
//     the current one is combined); levels to float-float, scaled, added to the
//     binary64 node data  -> acc_empty[acc]
// so that a tile's cutting overlaps the previous tiles' MMAs and epilogue.
// The two half-steps balance the roles differently: the p-half reads two partner
// components and writes one (9 producer warps, one region row a thread; 4 epilogue
// warps), the u-half reads one and writes two (7 producer warps, rows t and t + 224
// for t < 34; 8 epilogue warps).  Both stay at 128 registers a thread: the register
// file is split between the SM's four sub-partitions, so 14 and 16 warps get the same.
// The tile exponent travels through a ring of kT6ERing slots (e_full).
// Every wait is bounded: on expiry a thread sets the abort flag and the
// status bit, and all roles leave their loops (producers decide together at
// their per-tile barrier); the MMA lane then waits for its MMAs in flight
// before the tensor memory is released.
template <bool PHALF>
struct T6Roles {
    static constexpr int PW = PHALF ? 9 : 7;          // producer warps
    static constexpr int NPROD = PW * 32;
    static constexpr int MMA = PW;                    // MMA warp
    static constexpr int EPI0 = PW + 1;               // first epilogue warp
    static constexpr int EW = PHALF ? 4 : 8;          // epilogue warps
    static constexpr int THREADS = (PW + 1 + EW) * 32;
    static constexpr int NSPLIT = EW / 4;             // warps per TMEM lane quarter
    static constexpr int NGRP = (PHALF ? 2 : 4) / NSPLIT;   // 8-column groups a thread
    static_assert(THREADS <= 512 && 2 * NPROD >= kT5Rows && NGRP * NSPLIT == (PHALF ? 2 : 4), "role layout");
};
constexpr int kT6MaxProdWarps = 9;
constexpr int kT6Stages = 3;
constexpr int kT6ERing = 8;
constexpr int kT6BarBytes = 8 * (2 * kT6Stages + 2 + 2 + kT6ERing + 1);
constexpr int kT6SmemBytes = kT5BBytes + kT6Stages * kT5ABytes + kT6BarBytes + 4 * (kT6ERing + 2 * kT6MaxProdWarps + 4);

// barrier 1 among the NPROD producer threads with an OR of a predicate over them
template <int NPROD>
__device__ __forceinline__ bool producers_sync_or(bool p)
{
    uint32_t out;
    asm volatile(
        "{\n\t.reg .pred pi, po;\n\tsetp.ne.u32 pi, %1, 0;\n\tbar.red.or.pred po, 1, %2, pi;\n\t"
        "selp.u32 %0, 1, 0, po;\n\t}\n"
        : "=r"(out)
        : "r"((uint32_t)p), "n"(NPROD)
        : "memory");
    return out != 0;
}

// the shot of tile t (the last shot whose first tile is <= t)
__device__ __forceinline__ void t6_tile(const ShotDesc *__restrict__ shots, int n_shots, int t, ShotDesc &sd, int &x0,
                                        int &y)
{
    int lo = 0, hi = n_shots - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (shots[mid].tile_begin <= t) lo = mid; else hi = mid - 1;
    }
    sd = shots[lo];
    const int tt = t - sd.tile_begin;
    x0 = (tt % sd.tiles[0]) * kT5TileX;
    y = tt / sd.tiles[0];
}

template <int M, bool PHALF>
__global__ void __launch_bounds__(T6Roles<PHALF>::THREADS, 1)
    k_half_tc6(const double *__restrict__ S, double *__restrict__ X, const ShotDesc *__restrict__ shots, int n_shots,
               int total_tiles, const uint4 *__restrict__ Bimg, const int *__restrict__ expo, unsigned *status)
{
    constexpr int NQ = (M + 1) * (M + 1);
    constexpr int NCIN = PHALF ? 2 : 1;
    using Op = T5Op<PHALF>;
    using R = T6Roles<PHALF>;
    extern __shared__ __align__(1024) unsigned char t6_sm[];
    unsigned char *Bs = t6_sm;
    unsigned char *As = t6_sm + kT5BBytes;
    uint64_t *bars = reinterpret_cast<uint64_t *>(As + kT6Stages * kT5ABytes);
    uint64_t *a_full = bars, *a_empty = bars + kT6Stages, *acc_full = bars + 2 * kT6Stages,
             *acc_empty = acc_full + 2, *e_full = acc_empty + 2, *drain = e_full + kT6ERing;
    int *tileE = reinterpret_cast<int *>(drain + 1);
    int *red = tileE + kT6ERing;                 // [2][R::PW]
    volatile int *abort_flag = red + 2 * kT6MaxProdWarps;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(red + 2 * kT6MaxProdWarps + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (warp == 0) {
        tmem_alloc(smem_addr(tmem_slot), 2 * Op::TCOLS);
        tc_fence_before();
    }
    if (tid == 32) {
        for (int s = 0; s < kT6Stages; ++s) {
            mbar_init(smem_addr(a_full + s), R::NPROD);
            mbar_init(smem_addr(a_empty + s), 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(smem_addr(acc_full + a), 1);
            mbar_init(smem_addr(acc_empty + a), R::EW * 32);
        }
        for (int r = 0; r < kT6ERing; ++r) mbar_init(smem_addr(e_full + r), 1);
        mbar_init(smem_addr(drain), 1);
        *abort_flag = 0;
    }
    for (int e = tid; e < kT5BBytes / 16; e += R::THREADS) reinterpret_cast<uint4 *>(Bs)[e] = __ldg(Bimg + e);
    for (int e = tid; e < kT6Stages * kT5Digits * 2 * (kT5RowsPad - kT5Rows); e += R::THREADS) {
        const int per = 2 * (kT5RowsPad - kT5Rows);
        const int st = e / (kT5Digits * per), dg = (e / per) % kT5Digits, ch = (e / (kT5RowsPad - kT5Rows)) % 2;
        const int r = kT5Rows + e % (kT5RowsPad - kT5Rows);
        *reinterpret_cast<uint4 *>(As + st * kT5ABytes + dg * kT5Plane + ch * kT5Chunk + r * 16) =
            make_uint4(0u, 0u, 0u, 0u);
    }
    fence_async_smem();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int lo = PHALF ? -1 : 0;

    if (warp < R::PW) {
        // ------------------------------------------------------------ producers
        const bool one = tid < kT5Rows;                 // a first region row
        const bool two = tid + R::NPROD < kT5Rows;      // a second region row
        const int r0 = one ? tid : 0, r1 = tid + R::NPROD;
        int u = 0, lt = 0;
        bool dead = false;
        for (int t = blockIdx.x; t < total_tiles; t += gridDim.x, ++lt) {
            ShotDesc sd;
            int x0, y;
            t6_tile(shots, n_shots, t, sd, x0, y);
            const int64_t nnode = sd.nnode;
            const double *Sb = S + (PHALF ? sd.u_off : sd.p_off);
            auto region_node = [&](int r) -> int64_t {
                int gx = (x0 + lo + r % kT5RX) % sd.n[0];
                if (gx < 0) gx += sd.n[0];
                int gy = (y + lo + r / kT5RX) % sd.n[1];
                if (gy < 0) gy += sd.n[1];
                return gx + (int64_t)sd.n[0] * gy;
            };
            const int64_t nd0 = region_node(r0);
            const int64_t nd1 = two ? region_node(r1) : nd0;
            // the first row's first component stays in registers for its cut; everything
            // else is read for its exponent now and again when it is cut (from L1/L2)
            double v0[NQ];
#pragma unroll
            for (int q = 0; q < NQ; ++q) v0[q] = __ldg(Sb + (int64_t)q * nnode + nd0);
            int emax = 0;
            bool bad = false;
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                const int e0 = (__double2hiint(v0[q]) >> 20) & 0x7FF;
                bad |= e0 == 0x7FF;
                emax = max(emax, e0 == 0x7FF ? 0 : e0);
            }
#pragma unroll
            for (int e = NQ; e < NCIN * NQ; ++e) {
                const int e0 = (__double2hiint(__ldg(Sb + (int64_t)e * nnode + nd0)) >> 20) & 0x7FF;
                bad |= e0 == 0x7FF;
                emax = max(emax, e0 == 0x7FF ? 0 : e0);
            }
            if (two) {
                for (int e = 0; e < NCIN * NQ; ++e) {
                    const int e1 = (__double2hiint(__ldg(Sb + (int64_t)e * nnode + nd1)) >> 20) & 0x7FF;
                    bad |= e1 == 0x7FF;
                    emax = max(emax, e1 == 0x7FF ? 0 : e1);
                }
            }
            report_nonfinite(bad, status);
            emax = __reduce_max_sync(0xFFFFFFFFu, emax);
            if (lane == 0) red[(lt & 1) * R::PW + warp] = emax;
            if (producers_sync_or<R::NPROD>(dead || *abort_flag != 0)) break;   // uniform over the producers
#pragma unroll
            for (int w = 0; w < R::PW; ++w) emax = max(emax, red[(lt & 1) * R::PW + w]);
            if (tid == 0) {
                tileE[lt % kT6ERing] = emax;
                mbar_arrive(smem_addr(e_full + lt % kT6ERing));
            }
#pragma unroll
            for (int c = 0; c < NCIN; ++c, ++u) {
                const int st = u % kT6Stages;
                if (dead) continue;
                if (u >= kT6Stages &&
                    !mbar_wait(smem_addr(a_empty + st), (uint32_t)(((u / kT6Stages) - 1) & 1), kT5WaitLimit)) {
                    dead = true;
                    *abort_flag = 1;
                    atomicOr(status, kStatusTimeout);
                    continue;
                }
                if (c > 0) {
#pragma unroll
                    for (int q = 0; q < NQ; ++q) v0[q] = __ldg(Sb + (int64_t)(c * NQ + q) * nnode + nd0);
                }
                if (one) t5_store_row_regs<NQ>(As + st * kT5ABytes, r0, v0, emax);
                if (two) t5_store_row<NQ>(As + st * kT5ABytes, r1, Sb + (int64_t)c * NQ * nnode + nd1, nnode, emax);
                fence_async_smem();
                mbar_arrive(smem_addr(a_full + st));
            }
        }
    } else if (warp == R::MMA) {
        // ------------------------------------------------------------ MMA issue (one lane)
        if (lane == 0) {
            const uint32_t b0 = smem_addr(Bs);
            int u = 0, lt = 0;
            for (int t = blockIdx.x; t < total_tiles; t += gridDim.x, ++lt) {
                if (*abort_flag) break;
                const int ac = lt & 1;
                if (lt >= 2 && !mbar_wait(smem_addr(acc_empty + ac), (uint32_t)(((lt >> 1) - 1) & 1), kT5WaitLimit)) {
                    *abort_flag = 1;
                    atomicOr(status, kStatusTimeout);
                    break;
                }
                tc_fence_after();
                bool ok = true;
                for (int c = 0; c < NCIN; ++c, ++u) {
                    const int st = u % kT6Stages;
                    if (!mbar_wait(smem_addr(a_full + st), (uint32_t)((u / kT6Stages) & 1), kT5WaitLimit)) {
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
                if (!ok) {
                    *abort_flag = 1;
                    atomicOr(status, kStatusTimeout);
                    break;
                }
                umma_commit(smem_addr(acc_full + ac));
            }
            // every MMA issued has completed before the tensor memory is released
            umma_commit(smem_addr(drain));
            mbar_wait(smem_addr(drain), 0u, kT5WaitLimit);
        }
    } else {
        // ------------------------------------------------------------ epilogue
        const int quarter = warp & 3;                 // the TMEM lanes a warp may read
        const int half = (warp - R::EPI0) >> 2;       // which share of the node's outputs
        const int q = 32 * quarter + lane;            // node within the tile = TMEM lane
        const uint32_t tl = tmem + ((uint32_t)(32 * quarter) << 16);
        constexpr int NGRP = R::NGRP;                 // groups of 8 output columns per thread
        int lt = 0;
        bool bad = false;
        for (int t = blockIdx.x; t < total_tiles; t += gridDim.x, ++lt) {
            if (*abort_flag) break;
            ShotDesc sd;
            int x0, y;
            t6_tile(shots, n_shots, t, sd, x0, y);
            const int64_t nnode = sd.nnode;
            double *Xb = X + (PHALF ? sd.p_off : sd.u_off);
            const int gx = x0 + q;
            const bool mine = gx < sd.n[0];
            const int64_t node = (int64_t)gx + (int64_t)sd.n[0] * y;
            const int ac = lt & 1;
            auto load_own = [&](int g, double *own) {
                const int cg = NGRP * half + g;  // column group of the level
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int s = (8 * cg + j) % 16, oc = (8 * cg + j) / 16;
                    own[j] = (mine && s < NQ) ? Xb[(int64_t)(oc * NQ + s) * nnode + node] : 0.0;
                }
            };
            double own[8], nxt[8];
            load_own(0, own);  // in flight while this tile's MMAs run
            if (!mbar_wait(smem_addr(e_full + lt % kT6ERing), (uint32_t)((lt / kT6ERing) & 1), kT5WaitLimit) ||
                !mbar_wait(smem_addr(acc_full + ac), (uint32_t)((lt >> 1) & 1), kT5WaitLimit)) {
                *abort_flag = 1;
                atomicOr(status, kStatusTimeout);
                break;
            }
            tc_fence_after();
            const int E = tileE[lt % kT6ERing] - 1022;
#pragma unroll
            for (int g = 0; g < NGRP; ++g) {
                const int col0 = 8 * (NGRP * half + g);  // within a level: component col0 / 16
                if (g + 1 < NGRP) load_own(g + 1, nxt);
                // levels summed from the smallest weight up, in two batches of TMEM loads
                FF tot[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) tot[j] = FF{0.f, 0.f};
#pragma unroll
                for (int batch = 0; batch < 2; ++batch) {
                    constexpr int kHi = kT5Levels - 1;
                    const int Lhi = batch == 0 ? kHi : 2, Llo = batch == 0 ? 3 : 0;
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
                                // levels 6..4 (each below 2^-8 of level 0's bound) in plain FP32:
                                // their rounding stays under 2^-54 of the top level's scale
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
                        Xb[(int64_t)(oc * NQ + s) * nnode + node] = nv;
                        bad |= nonfinite(nv);
                    }
                }
                if (g + 1 < NGRP) {
#pragma unroll
                    for (int j = 0; j < 8; ++j) own[j] = nxt[j];
                }
            }
            tc_fence_before();
            mbar_arrive(smem_addr(acc_empty + ac));
        }
        report_nonfinite(bad, status);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 2 * Op::TCOLS);
}

template <int M>
static cudaError_t run_tc5(const LaunchFp64 &a)
{
    if (!a.tc_digits || !a.tc_expo || !a.tc_shots || a.tc_tiles <= 0) return cudaErrorInvalidValue;
    static std::atomic<uint64_t> opted_in{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const uint64_t bit = 1ull << (dev & 63);
    if (!(opted_in.load() & bit)) {
        if ((e = cudaFuncSetAttribute(k_half_tc6<M, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      kT6SmemBytes)) != cudaSuccess ||
            (e = cudaFuncSetAttribute(k_half_tc6<M, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      kT6SmemBytes)) != cudaSuccess)
            return e;
        opted_in.fetch_or(bit);
    }
    int sms = 0;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    constexpr int NQ = (M + 1) * (M + 1);
    const uint4 *bp = reinterpret_cast<const uint4 *>(a.tc_digits);
    const uint4 *bu = reinterpret_cast<const uint4 *>(a.tc_digits + kT5BBytes / 2);
    const dim3 grid((unsigned)std::min(a.tc_tiles, sms));  // persistent: one CTA per SM
    for (int64_t st = 0; st < a.nsteps; ++st) {
        if (a.ev) cudaEventRecord(a.ev[2 * st], a.stream);
        k_half_tc6<M, true><<<grid, T6Roles<true>::THREADS, kT6SmemBytes, a.stream>>>(a.U, a.P, a.tc_shots, a.n_shots,
                                                                          a.tc_tiles, bp, a.tc_expo, a.status);
        if (a.src && a.src->active) {
            if ((e = launch_source(*a.src, a.shots, a.P, NQ, a.step0 + st, a.stream)) != cudaSuccess) return e;
        }
        if (a.ev) cudaEventRecord(a.ev[2 * st + 1], a.stream);
        k_half_tc6<M, false><<<grid, T6Roles<false>::THREADS, kT6SmemBytes, a.stream>>>(a.P, a.U, a.tc_shots, a.n_shots,
                                                                           a.tc_tiles, bu, a.tc_expo + 16, a.status);
    }
    if (a.ev) cudaEventRecord(a.ev[2 * a.nsteps], a.stream);
    return cudaGetLastError();
}

}  // namespace hl
