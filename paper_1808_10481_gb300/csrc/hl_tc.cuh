// Tensor-core split mode (HL_TC_SPLIT), dim = 2: the half-step contraction
// as BF16 tensor-core products that are exact, on binary64 node data.
//
// For a tile of nodes the partner data at the cell vertices form the rows of
// A (k = partner component, vertex, slot; 16 slots per block of k, zero
// padded) and the vertex form of the fused operator is B[k][s] (the host's
// digit tables, build_tc_tables).  Both operands are cut into kTcDigits
// base-256 digits after a power-of-two scaling: the block's partner data by
// 2^-E with E from the block maximum (one E per partner component), every
// operator column by its own 2^-e_n.  Partner digits lie in [-256, 256] (the
// first) and [-128, 128] (the others), operator digits in [-128, 127]; the sum
// of one level's products over a component's K = 64 terms, at most 6 digit
// pairs of which one may hold a first partner digit, stays below
// 64 (2^15 + 5 2^14) < 2^23, so the FP32 accumulators of mma.sync hold it
// exactly.  Digit pairs (i, j) with i + j <= kTcLevels - 1 are formed; level
// L = i + j carries weight 2^(E + e_n - 14 - 8 L).  The levels are summed in
// float-float and the increment is added to the binary64 node value.
//
// The partner values enter as their float-float shadows (hi + lo, 48 bits);
// quantisation to 48 bits below the block maximum (46 below each operator
// column maximum) and the dropped levels (L >= kTcLevels) bound the error by a
// few 2^-46 of max|data| times the operator's column sums per half-step.
#pragma once

#include <atomic>

#include "hl_mixed.cuh"

namespace hl {

constexpr int kTcLevels = 7;     // digit pairs with i + j <= 6
constexpr int kTcThreads = 256;  // 8 warps; warp w owns the 16-node row blocks w (and w + 8)

// 2^k as a binary32 (0 below the normal range)
__device__ __forceinline__ float pow2f(int k)
{
    if (k < -126) return 0.f;
    return __uint_as_float((unsigned)(k + 127) << 23);
}

// ldmatrix: four (x4) or two (x2) 8x8 BF16 matrices from shared memory, each
// lane giving the address of one 16-byte row; the registers come out in the
// mma.sync fragment layout
__device__ __forceinline__ void ldsm_x4(uint32_t *r, const void *p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"((unsigned)__cvta_generic_to_shared(p)));
}
__device__ __forceinline__ void ldsm_x2(uint32_t &r0, uint32_t &r1, const void *p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n"
                 : "=r"(r0), "=r"(r1)
                 : "r"((unsigned)__cvta_generic_to_shared(p)));
}

__device__ __forceinline__ void mma_bf16(float *c, const uint32_t *a, uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Partner digit rows: 16 slots (8 words) per (digit, region node); the two
// 16-byte halves of a row are swapped on rows with bit 2 set, so that the
// fragment loads of 8 consecutive rows hit 32 different banks.
__device__ __forceinline__ int tc_word(int row, int w) { return row * 8 + (w ^ (((row >> 2) & 1) << 2)); }

// Shared memory of one block (bytes) for a tile of tx x ty nodes.
__host__ __device__ constexpr size_t tc_smem_bytes(int tx, int ty, int nq, int nops)
{
    return (size_t)nops * kTcOpElems * 2                     // operator digits
           + (size_t)kTcDigits * (tx + 1) * (ty + 1) * 32     // partner digits
           + (size_t)2 * nq * (tx + 1) * (ty + 1) * 4          // staged partner values (hi, lo)
           + (size_t)(tx + 1) * (ty + 1) * 4 + 8 * 4;          // region offsets, reduction
}

// One half-step.  PHALF: partner u (2 components), output p (operator 0); else
// partner p, outputs u components 0 and 1 (operators 1, 2), staged once.  Bd /
// Be: the operators' digits and column exponents, back to back.  MTW: 16-node
// row blocks per warp (tiles of 128 or 256 nodes).
template <int M, bool PHALF, int MTW>
// two blocks per SM for 128-node tiles (measured 1.5x faster than one block
// with more registers); 256-node tiles hold twice the accumulators and run one
__global__ void __launch_bounds__(kTcThreads, MTW == 1 ? 2 : 1)
    k_half_tc(const float *__restrict__ Sh, const float *__restrict__ Sl, double *__restrict__ X,
              float *__restrict__ Xh, float *__restrict__ Xl, const ShotDesc *__restrict__ shots, int n_shots,
              int tx, int ty, const uint16_t *__restrict__ Bd, const int *__restrict__ Be, unsigned *status)
{
    constexpr int NQ = (M + 1) * (M + 1);
    constexpr int NCIN = PHALF ? 2 : 1;  // partner components
    constexpr int NOUT = PHALF ? 1 : 2;  // output components (operators)
    extern __shared__ __align__(16) unsigned char tc_sm[];
    const int RX = tx + 1, R = (tx + 1) * (ty + 1);
    uint16_t *Bs = reinterpret_cast<uint16_t *>(tc_sm);
    uint32_t *As = reinterpret_cast<uint32_t *>(Bs + NOUT * kTcOpElems);  // [digit][region node] rows of 8 words
    float *Fh = reinterpret_cast<float *>(As + (size_t)kTcDigits * R * 8);  // [slot][region node]
    float *Fl = Fh + (size_t)NQ * R;
    int *soff = reinterpret_cast<int *>(Fl + (size_t)NQ * R);
    float *red = reinterpret_cast<float *>(soff + R);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int g = lane >> 2, t = lane & 3;

    int shot;
    ShotDesc sd;
    find_shot(shots, n_shots, shot, sd);
    int tt = blockIdx.x - sd.tile_begin;
    const int x0 = (tt % sd.tiles[0]) * tx;
    tt /= sd.tiles[0];
    const int y0 = (tt % sd.tiles[1]) * ty;
    const int lo = PHALF ? -1 : 0;

    // operator digits (16-byte copies), region offsets (periodic), zero padded slots
    for (int e = tid; e < NOUT * kTcOpElems / 8; e += kTcThreads)
        reinterpret_cast<uint4 *>(Bs)[e] = __ldg(reinterpret_cast<const uint4 *>(Bd) + e);
    for (int r = tid; r < R; r += kTcThreads) {
        int gx = x0 + lo + r % RX, gy = y0 + lo + r / RX;
        gx += gx < 0 ? sd.n[0] : (gx >= sd.n[0] ? -sd.n[0] : 0);
        gy += gy < 0 ? sd.n[1] : (gy >= sd.n[1] ? -sd.n[1] : 0);
        soff[r] = gx + sd.n[0] * gy;
    }
    if constexpr (NQ < 16) {
        for (int e = tid; e < kTcDigits * R * 8; e += kTcThreads) As[e] = 0u;
    }
    int en[NOUT][2][2];  // exponents of this thread's output columns
#pragma unroll
    for (int o = 0; o < NOUT; ++o)
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
            for (int q = 0; q < 2; ++q) en[o][nt][q] = __ldg(Be + o * kTcN + nt * 8 + 2 * t + q);

    const int nmt = tx * ty / 16;
    FF tot[MTW][2][4];
#pragma unroll
    for (int a = 0; a < MTW; ++a)
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) tot[a][nt][e] = FF{0.f, 0.f};

    // epilogue: add the increments of output component oc to the binary64 node
    // data, refresh the shadows, and clear the sums
    bool bad = false;
    auto store_out = [&](int oc) {
#pragma unroll
        for (int a = 0; a < MTW; ++a) {
            const int mt = warp + 8 * a;
            if (mt >= nmt) continue;
#pragma unroll
            for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int q = mt * 16 + g + (e >= 2 ? 8 : 0);
                    const int s = nt * 8 + 2 * t + (e & 1);
                    const int gx = x0 + q % tx, gy = y0 + q / tx;
                    if (s < NQ && gx < sd.n[0] && gy < sd.n[1]) {
                        const int64_t node = gx + (int64_t)sd.n[0] * gy;
                        const int64_t idx = (PHALF ? sd.p_off + (int64_t)s * sd.nnode
                                                   : sd.u_off + (int64_t)(oc * NQ + s) * sd.nnode) + node;
                        Acc<true> inc;
                        inc.v = tot[a][nt][e];
                        bad |= store_value<true>(X, Xh, Xl, idx, inc.to_f64());
                    }
                    tot[a][nt][e] = FF{0.f, 0.f};
                }
        }
    };

    const int64_t base0 = PHALF ? sd.u_off : sd.p_off;
    static_for<0, NCIN>([&](auto cc) {
        constexpr int c = decltype(cc)::value;
        const int64_t base = base0 + (int64_t)c * NQ * sd.nnode;
        __syncthreads();  // offsets ready; the previous component is no longer read
        // stage the component's hi and lo shadows (all copies in flight at once)
#pragma unroll 1
        for (int l = 0; l < NQ; ++l)
#pragma unroll 1
            for (int r = tid; r < R; r += kTcThreads) {
                const int64_t gi = base + (int64_t)l * sd.nnode + soff[r];
                cp_async4(Fh + l * R + r, Sh + gi);
                cp_async4(Fl + l * R + r, Sl + gi);
            }
        cp_async_commit();
        cp_async_wait<0>();
        __syncthreads();
        // block maximum -> scale 2^-E (max |hi| < 2^E, and hi + lo stays below it)
        float mx = 0.f;
#pragma unroll 4
        for (int e = tid; e < NQ * R; e += kTcThreads) mx = fmaxf(mx, fabsf(Fh[e]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) red[warp] = mx;
        __syncthreads();
        mx = red[0];
#pragma unroll
        for (int w = 1; w < kTcThreads / 32; ++w) mx = fmaxf(mx, red[w]);
        const int E = mx > 0.f ? (int)((__float_as_uint(mx) >> 23) & 0xFFu) - 126 : 0;
        // partner digits on the FP32 pipe: with x = (hi + lo) 2^-E, |x| < 1, digit j is
        // the nearest integer to 256 x_j and x_{j+1} = 256 x_j - d_j, the remainder
        // kept exactly as a float-float pair; d_0 lies in [-256, 256], the others in
        // [-128, 128], and x = sum_j d_j 256^-(j+1) to 2^-49.  A thread converts a
        // slot pair of one region node.
        constexpr int NW = (NQ + 1) / 2;  // slot pairs; consecutive threads fill one row's words
        const float sc = pow2f(-E);
#pragma unroll 1
        for (int e = tid; e < NW * R; e += kTcThreads) {
            const int w = e % NW, r = e / NW, l0 = 2 * w;
            float h0 = Fh[l0 * R + r] * sc, q0 = Fl[l0 * R + r] * sc, h1 = 0.f, q1 = 0.f;
            if (l0 + 1 < NQ) {
                h1 = Fh[(l0 + 1) * R + r] * sc;
                q1 = Fl[(l0 + 1) * R + r] * sc;
            }
#pragma unroll
            for (int j = 0; j < kTcDigits; ++j) {
                const float t0 = h0 * 256.f, t1 = h1 * 256.f;
                // round to the nearest integer: 1.5 * 2^23 has a unit last place
                const float d0 = __fsub_rn(__fadd_rn(t0, 12582912.f), 12582912.f);
                const float d1 = __fsub_rn(__fadd_rn(t1, 12582912.f), 12582912.f);
                const FF r0 = ff_two_sum(__fsub_rn(t0, d0), q0 * 256.f);
                const FF r1 = ff_two_sum(__fsub_rn(t1, d1), q1 * 256.f);
                h0 = r0.hi, q0 = r0.lo, h1 = r1.hi, q1 = r1.lo;
                // an integer of at most 8 significant bits: its binary32 bits cut to BF16
                As[tc_word(j * R + r, w)] = (__float_as_uint(d0) >> 16) | (__float_as_uint(d1) & 0xFFFF0000u);
            }
        }
        __syncthreads();
        // exact digit products on the tensor cores, one 16-node row block at a time
        static_for<0, NOUT>([&](auto occ) {
        constexpr int o = decltype(occ)::value;
        const uint16_t *Bo = Bs + o * kTcOpElems;
        static_for<0, MTW>([&](auto ac) {
            constexpr int a = decltype(ac)::value;
            const int mt = warp + 8 * a;
            if (mt < nmt) {
                // ldmatrix row of this lane: A rows (lane % 8) + 8 ((lane / 8) % 2) of
                // the row block, k half lane / 16; B row lane % 8, k half (lane / 8) % 2
                const int qa = mt * 16 + (lane & 7) + 8 * ((lane >> 3) & 1);
                const int rqa = qa % tx + RX * (qa / tx);
                const int kha = lane >> 4, khb = (lane >> 3) & 1;
                // one 8-column half of the outputs at a time (fewer live accumulators)
                static_for<0, 2>([&](auto ntc) {
                    constexpr int nt = decltype(ntc)::value;
                    float acc[kTcLevels][4];
#pragma unroll
                    for (int L = 0; L < kTcLevels; ++L)
#pragma unroll
                        for (int e = 0; e < 4; ++e) acc[L][e] = 0.f;
                    static_for<0, 4>([&](auto vc) {
                        constexpr int v = decltype(vc)::value;
                        const int dv = (v & 1) + RX * (v >> 1);
                        const uint16_t *bcol = Bo + (size_t)(nt * 8 + (lane & 7)) * kTcKS + (c * 4 + v) * 16 + 8 * khb;
                        static_for<0, kTcDigits>([&](auto ic) {
                            constexpr int i = decltype(ic)::value;
                            uint32_t af[4];
                            ldsm_x4(af, As + tc_word(i * R + rqa + dv, 4 * kha));
                            static_for<0, kTcDigits>([&](auto jc) {
                                constexpr int j = decltype(jc)::value;
                                if constexpr (i + j < kTcLevels) {
                                    uint32_t b0, b1;
                                    ldsm_x2(b0, b1, bcol + (size_t)j * kTcN * kTcKS);
                                    mma_bf16(acc[i + j], af, b0, b1);
                                }
                            });
                        });
                    });
                    // levels -> float-float, scaled by 2^(E + e_n - 14 - 8 L) (exact): partner
                    // digit i weighs 2^(E - 8 - 8 i), operator digit j 2^(e_n - 6 - 8 j)
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int k0 = E + en[o][nt][e & 1] - 14;
#pragma unroll
                        for (int L = 0; L < kTcLevels; ++L) {
                            const float val = acc[L][e] * pow2f(k0 - 8 * L);
                            const FF s2 = ff_two_sum(tot[a][nt][e].hi, val);
                            tot[a][nt][e].hi = s2.hi;
                            tot[a][nt][e].lo = __fadd_rn(tot[a][nt][e].lo, s2.lo);
                        }
                    }
                });
            }
        });
        if constexpr (!PHALF) store_out(o);  // the single partner component is complete
        });
    });

    if constexpr (PHALF) store_out(0);
    report_nonfinite(bad, status);
}

template <int M, int MTW>
static cudaError_t run_tc_t(const LaunchFp64 &a)
{
    constexpr int NQ = (M + 1) * (M + 1);
    const size_t smem = tc_smem_bytes(a.tx, a.ty, NQ, 2);  // the u-half holds two operators
    if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
    static std::atomic<uint64_t> opted_in{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const uint64_t bit = 1ull << (dev & 63);
    if (!(opted_in.load() & bit)) {
        if ((e = cudaFuncSetAttribute(k_half_tc<M, true, MTW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      227 * 1024)) != cudaSuccess ||
            (e = cudaFuncSetAttribute(k_half_tc<M, false, MTW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      227 * 1024)) != cudaSuccess)
            return e;
        opted_in.fetch_or(bit);
    }
    const unsigned sb = 152 * 16;
    k_shadow<true><<<sb, 256, 0, a.stream>>>(a.P, a.Ph, a.Pl, a.p_elems);
    k_shadow<true><<<sb, 256, 0, a.stream>>>(a.U, a.Uh, a.Ul, a.p_elems * 2);
    const dim3 grid((unsigned)a.total_tiles);
    for (int64_t st = 0; st < a.nsteps; ++st) {
        if (a.ev) cudaEventRecord(a.ev[2 * st], a.stream);
        k_half_tc<M, true, MTW><<<grid, kTcThreads, tc_smem_bytes(a.tx, a.ty, NQ, 1), a.stream>>>(
            a.Uh, a.Ul, a.P, a.Ph, a.Pl, a.shots, a.n_shots, a.tx, a.ty, a.tc_digits, a.tc_expo, a.status);
        if (a.src && a.src->active) {
            if ((e = launch_source(*a.src, a.shots, a.P, NQ, a.step0 + st, a.stream, a.Ph, a.Pl)) != cudaSuccess)
                return e;
        }
        if (a.ev) cudaEventRecord(a.ev[2 * st + 1], a.stream);
        k_half_tc<M, false, MTW><<<grid, kTcThreads, smem, a.stream>>>(a.Ph, a.Pl, a.U, a.Uh, a.Ul, a.shots, a.n_shots,
                                                                       a.tx, a.ty, a.tc_digits + kTcOpElems,
                                                                       a.tc_expo + kTcN, a.status);
    }
    if (a.ev) cudaEventRecord(a.ev[2 * a.nsteps], a.stream);
    return cudaGetLastError();
}

template <int M>
static cudaError_t run_tc(const LaunchFp64 &a)
{
    if (!a.Ph || !a.Uh || !a.Pl || !a.Ul || !a.tc_digits || !a.tc_expo) return cudaErrorInvalidValue;
    if (a.tx % 16 != 0 || (a.tx * a.ty) % 16 != 0 || a.tx * a.ty > 256) return cudaErrorInvalidConfiguration;
    return a.tx * a.ty <= 128 ? run_tc_t<M, 1>(a) : run_tc_t<M, 2>(a);
}

}  // namespace hl
