// Learned coarse-grid correction (not in the paper): a per-node MLP over the
// coarse solver's Hermite data, trained on fine-grid solutions.
//
//   features of coarse primal node J (2D, m = 3, nq = 16), all times feat_scale
//   except the time feature:
//     p at the 3x3 primal nodes J + {-1,0,1}^2 (dy outer, dx inner)     144
//     u, then v, at the cell vertices: dual nodes J + {-1,0}^2             128
//     t_feature                                                              1
//     zero padding                                                          15  -> 288
//   y = relu(relu(x W1 + b1) W2 + b2) W3 + b3            288 -> 128 -> 128 -> 16
//   p~(J) += out_scale * y   (added in FP64)
//
// Every matrix product runs on the tensor cores with BF16 operands (weights
// and activations rounded to nearest BF16 when staged) and FP32 accumulation.
// The forward runs all three layers of a 128-row tile in one tcgen05 kernel
// (k_mlp_forward_tc, accumulators in tensor memory); the backward's GEMMs,
// whose operands are transposed views and whose weight gradients reduce over
// the batch (split-K), use the warp-level mma.sync m16n8k16 (k_gemm), which
// also serves the forward when a buffer is not 16-byte aligned.  Master
// weights, Adam moments and activations are FP32.  Loss: mean over rows and
// outputs of (y - target)^2.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "../../include/hl.h"
#include "hl_internal.h"
#include "hl_sm100.cuh"
#include "hl_solver.h"

namespace hl {

constexpr int kIn = HL_MLP_IN, kH = HL_MLP_HIDDEN, kOut = HL_MLP_OUT;

// ---------------------------------------------------------------------------
// C[M x N] = A[M x K] B[K x N] (+ bias[n]) (relu) ; element (r, c) of a matrix X
// is X.p[r * X.rs + c * X.cs], so transposes are free.  64x64 block tile,
// 4 warps of 32x32, K in steps of 32.  Both operands are kept in shared memory
// as BF16 with k innermost (A as [m][k], B as [n][k]), so every fragment
// register is one 32-bit shared load.  The next k-step is loaded from global
// memory into registers (float4 along whichever index is contiguous) while the
// current one is multiplied, then converted and stored to the other buffer.
// Split-K: block z covers K range [z*kc, (z+1)*kc) and writes its partial sums
// to part[z]; k_gemm_reduce adds them in a fixed order (deterministic).
struct Mat {
    const float *p;
    int64_t rs, cs;
};

constexpr int BM = 64, BN = 64, BK = 32, PADK = 8;
constexpr int LDS = BK + PADK;  // shared row length (bf16): 80 bytes

__device__ __forceinline__ uint32_t lds_pair(const __nv_bfloat16 *p)
{
    return *reinterpret_cast<const uint32_t *>(p);
}

__device__ __forceinline__ uint32_t pack2(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

// One 64 (outer) x 32 (k) operand tile of the view V(o, k) = p[o*so + k*sk],
// valid for o < olim and k < klim.  Mode 1: k contiguous, mode 2: o
// contiguous (both float4), mode 0: scalar.  16 values per thread.
struct TileLd {
    const float *p;
    int64_t so, sk;
    int olim;
    int mode;
    float v[16];

    __device__ __forceinline__ void load(int o0, int k0, int klim, int tid)
    {
        if (mode == 1) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int idx = tid + i * 128, o = idx >> 3, k = (idx & 7) * 4;
                float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
                if (o0 + o < olim && k0 + k < klim)
                    x = __ldg(reinterpret_cast<const float4 *>(p + (int64_t)(o0 + o) * so + (k0 + k)));
                v[4 * i] = x.x, v[4 * i + 1] = x.y, v[4 * i + 2] = x.z, v[4 * i + 3] = x.w;
            }
        } else if (mode == 2) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int idx = tid + i * 128, k = idx >> 4, o = (idx & 15) * 4;
                float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
                if (o0 + o < olim && k0 + k < klim)
                    x = __ldg(reinterpret_cast<const float4 *>(p + (o0 + o) + (int64_t)(k0 + k) * sk));
                v[4 * i] = x.x, v[4 * i + 1] = x.y, v[4 * i + 2] = x.z, v[4 * i + 3] = x.w;
            }
        } else {
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int idx = tid + i * 128, o = idx >> 5, k = idx & 31;
                v[i] = (o0 + o < olim && k0 + k < klim) ? p[(int64_t)(o0 + o) * so + (int64_t)(k0 + k) * sk] : 0.f;
            }
        }
    }

    __device__ __forceinline__ void store(__nv_bfloat16 (*dst)[LDS], int tid) const
    {
        if (mode == 1) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int idx = tid + i * 128, o = idx >> 3, k = (idx & 7) * 4;
                *reinterpret_cast<uint2 *>(&dst[o][k]) = make_uint2(pack2(v[4 * i], v[4 * i + 1]),
                                                                    pack2(v[4 * i + 2], v[4 * i + 3]));
            }
        } else if (mode == 2) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int idx = tid + i * 128, k = idx >> 4, o = (idx & 15) * 4;
#pragma unroll
                for (int j = 0; j < 4; ++j) dst[o + j][k] = __float2bfloat16_rn(v[4 * i + j]);
            }
        } else {
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int idx = tid + i * 128;
                dst[idx >> 5][idx & 31] = __float2bfloat16_rn(v[i]);
            }
        }
    }
};

// float4 paths need 16-byte aligned rows along the contiguous index and
// extents that are multiples of 4 there
__host__ __forceinline__ int tile_mode(const float *p, int64_t so, int64_t sk, int olim, int K)
{
    const bool al = ((uintptr_t)p & 15) == 0;
    if (al && sk == 1 && so % 4 == 0 && K % 4 == 0) return 1;
    if (al && so == 1 && sk % 4 == 0 && olim % 4 == 0) return 2;
    return 0;
}

__global__ void __launch_bounds__(128, 4) k_gemm(TileLd ta, TileLd tb, float *__restrict__ C, int64_t ldc, int M,
                                              int N, int K, int kc, const float *__restrict__ bias, int relu,
                                              float *__restrict__ part)
{
    __shared__ __align__(16) __nv_bfloat16 As[2][BM][LDS];
    __shared__ __align__(16) __nv_bfloat16 Bt[2][BN][LDS];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int g = lane >> 2, t = lane & 3;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int kbeg = blockIdx.z * kc, kend = min(K, kbeg + kc);
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;
    int cur = 0;
    if (kbeg < kend) {
        ta.load(m0, kbeg, kend, tid);
        tb.load(n0, kbeg, kend, tid);
        ta.store(As[0], tid);
        tb.store(Bt[0], tid);
    }
    __syncthreads();
    for (int k0 = kbeg; k0 < kend; k0 += BK) {
        const bool next = k0 + BK < kend;
        if (next) {  // in flight while this step is multiplied
            ta.load(m0, k0 + BK, kend, tid);
            tb.load(n0, k0 + BK, kend, tid);
        }
#pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
            uint32_t af[2][4], bf[4][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int r = wm + i * 16 + g;
                af[i][0] = lds_pair(&As[cur][r][kk + 2 * t]);
                af[i][1] = lds_pair(&As[cur][r + 8][kk + 2 * t]);
                af[i][2] = lds_pair(&As[cur][r][kk + 2 * t + 8]);
                af[i][3] = lds_pair(&As[cur][r + 8][kk + 2 * t + 8]);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int c = wn + j * 8 + g;
                bf[j][0] = lds_pair(&Bt[cur][c][kk + 2 * t]);
                bf[j][1] = lds_pair(&Bt[cur][c][kk + 2 * t + 8]);
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    asm volatile(
                        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
                        "{%8,%9}, {%0,%1,%2,%3};\n"
                        : "+f"(acc[i][j][0]), "+f"(acc[i][j][1]), "+f"(acc[i][j][2]), "+f"(acc[i][j][3])
                        : "r"(af[i][0]), "r"(af[i][1]), "r"(af[i][2]), "r"(af[i][3]), "r"(bf[j][0]), "r"(bf[j][1]));
        }
        if (next) {  // the other buffer's readers finished at the previous barrier
            ta.store(As[cur ^ 1], tid);
            tb.store(Bt[cur ^ 1], tid);
        }
        __syncthreads();
        cur ^= 1;
    }
    float *out = part ? part + (int64_t)blockIdx.z * M * N : C;
    const int64_t ld = part ? N : ldc;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int r = m0 + wm + i * 16 + g + (e >= 2 ? 8 : 0);
                const int c = n0 + wn + j * 8 + 2 * t + (e & 1);
                if (r < M && c < N) {
                    float v = acc[i][j][e];
                    if (!part) {
                        if (bias) v += bias[c];
                        if (relu) v = fmaxf(v, 0.f);
                    }
                    out[(int64_t)r * ld + c] = v;
                }
            }
}

__global__ void k_gemm_reduce(const float *__restrict__ part, int splits, int M, int N, float *__restrict__ C,
                              int64_t ldc, const float *__restrict__ bias, int relu)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)M * N) return;
    float v = 0.f;
    for (int z = 0; z < splits; ++z) v += part[(int64_t)z * M * N + e];
    const int r = (int)(e / N), c = (int)(e % N);
    if (bias) v += bias[c];
    if (relu) v = fmaxf(v, 0.f);
    C[(int64_t)r * ldc + c] = v;
}

// split-K workspace is owned by the caller (the network handle): splits*M*N floats
static cudaError_t gemm(Mat A, Mat B, float *C, int64_t ldc, int M, int N, int K, const float *bias, int relu,
                        cudaStream_t st, float *work = nullptr, int64_t work_floats = 0)
{
    if (M <= 0 || N <= 0) return cudaSuccess;
    const int tiles = ((N + BN - 1) / BN) * ((M + BM - 1) / BM);
    int splits = 1;
    // few output tiles and a long K (weight gradients over the batch): split K
    while (work && tiles * splits < 2 * 152 && K / (splits * 2) >= 4 * BK &&
           (int64_t)(splits * 2) * M * N <= work_floats)
        splits *= 2;
    const int kc = ((K + splits - 1) / splits + BK - 1) / BK * BK;
    const dim3 grid((unsigned)((N + BN - 1) / BN), (unsigned)((M + BM - 1) / BM), (unsigned)splits);
    // operand views with k as the second index: A(m, k), and B as B(n, k)
    TileLd ta{A.p, A.rs, A.cs, M, tile_mode(A.p, A.rs, A.cs, M, K), {}};
    TileLd tb{B.p, B.cs, B.rs, N, tile_mode(B.p, B.cs, B.rs, N, K), {}};
    // split boundaries stay multiples of BK, so the float4 k-ranges never straddle them
    k_gemm<<<grid, 128, 0, st>>>(ta, tb, C, ldc, M, N, K, kc, bias, relu, splits > 1 ? work : nullptr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || splits == 1) return e;
    const int64_t n = (int64_t)M * N;
    k_gemm_reduce<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(work, splits, M, N, C, ldc, bias, relu);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Forward on the fifth-generation tensor cores (tcgen05): all three layers of
// one 128-row tile in one kernel, activations kept on chip (TMEM accumulators,
// BF16 operands in shared memory); only X is read and Y written.
//
// Persistent and warp-specialised: one CTA of 17 warps per SM walks the row
// tiles; its roles hand each tile along mbarriers.
//   producers (warps 8..15): X rows (FP32 in HBM, coalesced float4) -> the BF16
//     A operand in the X buffer -> x_full.  They start the next tile as soon as
//     the tile's layer-1 MMAs have read the buffer (x_empty), so the HBM reads
//     overlap the rest of the tile.
//   MMA (lane 0 of warp 16): 18 MMAs (K = 16) into TMEM columns 0..127 ->
//     x_empty, acc1;  after h1: 8 MMAs into 128..255 -> acc2;  after h2: 8
//     MMAs (N = 16) into 256..271 -> acc3.
//   epilogue (warps 0..7; warp w reads TMEM lanes 32 (w % 4).. and half w / 4
//     of the columns): acc1 + b1, ReLU, BF16 -> H (the next A operand) -> h1;
//     acc2 -> H again (layer 2 has read H1 by then) -> h2;  acc3 + b3 -> Y.
// For training, the FP32 activations H1 and H2 (after bias and ReLU, before the
// BF16 rounding) can also be written out, for the backward GEMMs.
// Operand layout (no swizzle): the 8-value K chunk c of row r sits at byte
// c * (rows * 16) + r * 16; the descriptor's K stride (LBO) is one chunk and
// its 8-row stride (SBO) 128 bytes.  The rounding points are k_gemm's:
// operands rounded to nearest BF16, FP32 accumulation, bias and ReLU in FP32
// before the next layer's rounding.  Every mbarrier wait is bounded; on expiry
// the thread sets kStatusTimeout in *status (if given) and an abort flag that
// every role checks, all roles leave their loops, and the MMAs in flight are
// drained before TMEM is freed.
constexpr int kFwdRows = 128;                         // MMA M: rows per tile
constexpr int kFwdEpiWarps = 8, kFwdProdWarps = 8;
constexpr int kFwdMmaWarp = kFwdEpiWarps + kFwdProdWarps;
constexpr int kFwdThreads = 32 * (kFwdMmaWarp + 1);
constexpr int kFwdEpiThreads = 32 * kFwdEpiWarps, kFwdProdThreads = 32 * kFwdProdWarps;
constexpr int kFwdChunk = kFwdRows * 16;              // one 8-wide K chunk of a 128-row operand (bytes)
constexpr int kFwdOffH = (kIn / 8) * kFwdChunk;       // after the X buffer: H1, then H2, in one buffer
constexpr int kFwdOffW1 = kFwdOffH + (kH / 8) * kFwdChunk;
constexpr int kFwdOffW2 = kFwdOffW1 + (kIn / 8) * kH * 16;
constexpr int kFwdOffW3 = kFwdOffW2 + (kH / 8) * kH * 16;
constexpr int kFwdOffBias = kFwdOffW3 + (kH / 8) * kOut * 16;
constexpr int kFwdOffBar = kFwdOffBias + (2 * kH + kOut) * 4;
constexpr int kFwdBars = 8;                           // x_full x_empty acc1 h1 acc2 h2 acc3 drain
constexpr int kFwdSmem = kFwdOffBar + 8 * kFwdBars + 16;   // + abort flag, TMEM address
constexpr int kFwdTmemCols = 512;                     // acc1 at 0, acc2 at kH, acc3 at 2 kH
static_assert(kIn % 16 == 0 && kH % 16 == 0 && kOut % 16 == 0 && kOut >= 16, "MMA K and N shapes");
static_assert(kH == kFwdRows, "the hidden width is the A operand's row count of layers 2 and 3");
static_assert(2 * kH + kOut <= kFwdTmemCols, "accumulators fit the allocated TMEM columns");
static_assert(kFwdOffBar % 8 == 0 && kFwdSmem <= 227 * 1024, "shared-memory layout");

// B operand (n, k) = W[k][n] of a row-major K x N weight matrix, rounded to BF16
__device__ __forceinline__ void fwd_stage_weight(unsigned char *dst, const float *__restrict__ W, int K, int N,
                                                 int tid)
{
    const int units = (K / 8) * N;
    for (int u = tid; u < units; u += kFwdThreads) {
        const int c = u / N, n = u % N;
        const float *w = W + (int64_t)(8 * c) * N + n;
        const uint4 v = make_uint4(pack2(__ldg(w), __ldg(w + N)), pack2(__ldg(w + 2 * N), __ldg(w + 3 * N)),
                                   pack2(__ldg(w + 4 * N), __ldg(w + 5 * N)), pack2(__ldg(w + 6 * N), __ldg(w + 7 * N)));
        *reinterpret_cast<uint4 *>(dst + c * (N * 16) + n * 16) = v;
    }
}

// A operand (r, k) = X[row0 + r][k] rounded to BF16, rows at or past `rows` zero, by the
// producer warps (pw = 0..7).  A warp moves 8 rows x 16 floats at a time: 16 fully used
// 32-byte sectors per load; each half-warp stores one 128-byte run of one K chunk.
__device__ __forceinline__ void fwd_stage_x(unsigned char *dst, const float *__restrict__ X, int64_t row0, int rows,
                                            int pw, int lane)
{
    constexpr int CG = kIn / 16;                               // 16-float groups per row
    constexpr int PER = (kFwdRows / 8) * CG / kFwdProdWarps;   // units per warp
    constexpr int BATCH = 12;                                  // loads in flight per thread
    static_assert((kFwdRows / 8) * CG % kFwdProdWarps == 0 && PER % BATCH == 0, "X staging split");
    const int half = lane >> 4, ri = (lane >> 1) & 7, lo = lane & 1;
#pragma unroll 1
    for (int i0 = 0; i0 < PER; i0 += BATCH) {
        float4 x[BATCH];
#pragma unroll
        for (int j = 0; j < BATCH; ++j) {
            const int u = pw + (i0 + j) * kFwdProdWarps;
            const int r = 8 * (u / CG) + ri, c4 = 4 * (u % CG) + 2 * half + lo;
            x[j] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (row0 + r < rows) x[j] = __ldg(reinterpret_cast<const float4 *>(X + (row0 + r) * kIn) + c4);
        }
#pragma unroll
        for (int j = 0; j < BATCH; ++j) {
            const int u = pw + (i0 + j) * kFwdProdWarps;
            const int r = 8 * (u / CG) + ri, c4 = 4 * (u % CG) + 2 * half + lo;
            *reinterpret_cast<uint2 *>(dst + (c4 >> 1) * kFwdChunk + r * 16 + lo * 8) =
                make_uint2(pack2(x[j].x, x[j].y), pack2(x[j].z, x[j].w));
        }
    }
}

// 64 accumulator columns [c0, c0 + 64) of this thread's row r: + bias, ReLU, BF16 into
// the next layer's A operand (K = kH); the FP32 activations also to hout (row of kH
// floats; NULL = not kept)
__device__ __forceinline__ void fwd_epi_hidden(uint32_t tacc, int c0, const float *bias, unsigned char *dst, int r,
                                               float *hout)
{
    float v[4][16];
#pragma unroll
    for (int g = 0; g < 4; ++g) tmem_ld16(tacc + (uint32_t)(c0 + 16 * g), v[g]);
    tmem_ld_wait();
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        const int c = c0 + 16 * g;
        uint32_t w[8];
#pragma unroll
        for (int j = 0; j < 16; ++j) v[g][j] = fmaxf(v[g][j] + bias[c + j], 0.f);
#pragma unroll
        for (int j = 0; j < 8; ++j) w[j] = pack2(v[g][2 * j], v[g][2 * j + 1]);
        if (hout) {
#pragma unroll
            for (int j = 0; j < 4; ++j)
                reinterpret_cast<float4 *>(hout + c)[j] =
                    make_float4(v[g][4 * j], v[g][4 * j + 1], v[g][4 * j + 2], v[g][4 * j + 3]);
        }
        *reinterpret_cast<uint4 *>(dst + (c / 8) * kFwdChunk + r * 16) = make_uint4(w[0], w[1], w[2], w[3]);
        *reinterpret_cast<uint4 *>(dst + (c / 8 + 1) * kFwdChunk + r * 16) = make_uint4(w[4], w[5], w[6], w[7]);
    }
}

__global__ void __launch_bounds__(kFwdThreads, 1)
    k_mlp_forward_tc(const float *__restrict__ X, int rows, const float *__restrict__ W1,
                     const float *__restrict__ b1, const float *__restrict__ W2, const float *__restrict__ b2,
                     const float *__restrict__ W3, const float *__restrict__ b3, float *__restrict__ Y,
                     float *__restrict__ H1out, float *__restrict__ H2out, unsigned *status)
{
    extern __shared__ __align__(1024) unsigned char fw_sm[];
    unsigned char *Xs = fw_sm, *Hs = fw_sm + kFwdOffH;
    unsigned char *W1s = fw_sm + kFwdOffW1, *W2s = fw_sm + kFwdOffW2, *W3s = fw_sm + kFwdOffW3;
    float *bias = reinterpret_cast<float *>(fw_sm + kFwdOffBias);   // b1, b2, b3
    uint64_t *bars = reinterpret_cast<uint64_t *>(fw_sm + kFwdOffBar);
    const uint32_t x_full = smem_addr(bars), x_empty = smem_addr(bars + 1), acc1 = smem_addr(bars + 2),
                   h1 = smem_addr(bars + 3), acc2 = smem_addr(bars + 4), h2 = smem_addr(bars + 5),
                   acc3 = smem_addr(bars + 6), drain = smem_addr(bars + 7);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(bars + kFwdBars);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + kFwdBars) + 1;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tiles = (rows + kFwdRows - 1) / kFwdRows;

    if (warp == kFwdMmaWarp) {
        tmem_alloc(smem_addr(tmem_slot), kFwdTmemCols);
        tc_fence_before();
    }
    if (tid == 0) {
        mbar_init(x_full, kFwdProdThreads);
        mbar_init(x_empty, 1);
        mbar_init(acc1, 1);
        mbar_init(h1, kFwdEpiThreads);
        mbar_init(acc2, 1);
        mbar_init(h2, kFwdEpiThreads);
        mbar_init(acc3, 1);
        mbar_init(drain, 1);
        *abort_flag = 0;
    }
    fwd_stage_weight(W1s, W1, kIn, kH, tid);
    fwd_stage_weight(W2s, W2, kH, kH, tid);
    fwd_stage_weight(W3s, W3, kH, kOut, tid);
    for (int i = tid; i < kH; i += kFwdThreads) {
        bias[i] = __ldg(b1 + i);
        bias[kH + i] = __ldg(b2 + i);
    }
    if (tid < kOut) bias[2 * kH + tid] = __ldg(b3 + tid);
    fence_async_smem();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    // a wait that expires stops every role (the others then time out or see the flag)
    auto wait = [&](uint32_t bar, uint32_t parity) -> bool {
        if (mbar_wait(bar, parity, kMbarWaitLimit)) return true;
        *abort_flag = 1;
        if (status) atomicOr(status, kStatusTimeout);
        return false;
    };

    if (warp >= kFwdEpiWarps && warp < kFwdMmaWarp) {
        // ------------------------------------------------------------ producers
        const int pw = warp - kFwdEpiWarps;
        int j = 0;
        for (int t = blockIdx.x; t < tiles; t += gridDim.x, ++j) {
            if (*abort_flag) break;
            if (j > 0 && !wait(x_empty, (uint32_t)((j - 1) & 1))) break;
            fwd_stage_x(Xs, X, (int64_t)t * kFwdRows, rows, pw, lane);
            fence_async_smem();
            mbar_arrive(x_full);
        }
    } else if (warp == kFwdMmaWarp) {
        // ------------------------------------------------------------ MMA issue
        if (lane == 0) {
            const uint32_t sX = smem_addr(Xs), sH = smem_addr(Hs);
            const uint32_t sW1 = smem_addr(W1s), sW2 = smem_addr(W2s), sW3 = smem_addr(W3s);
            constexpr uint32_t idH = umma_idesc_bf16(kFwdRows, kH), idO = umma_idesc_bf16(kFwdRows, kOut);
            int j = 0;
            for (int t = blockIdx.x; t < tiles; t += gridDim.x, ++j) {
                const uint32_t par = (uint32_t)(j & 1);
                if (*abort_flag || !wait(x_full, par)) break;
                tc_fence_after();
#pragma unroll 1
                for (int s = 0; s < kIn / 16; ++s)
                    umma_bf16(tmem, umma_desc(sX + (uint32_t)(s * 2 * kFwdChunk), kFwdChunk, 128),
                              umma_desc(sW1 + (uint32_t)(s * 2 * kH * 16), kH * 16, 128), idH, s > 0 ? 1u : 0u);
                umma_commit(x_empty);
                umma_commit(acc1);
                if (!wait(h1, par)) break;
                tc_fence_after();
#pragma unroll 1
                for (int s = 0; s < kH / 16; ++s)
                    umma_bf16(tmem + kH, umma_desc(sH + (uint32_t)(s * 2 * kFwdChunk), kFwdChunk, 128),
                              umma_desc(sW2 + (uint32_t)(s * 2 * kH * 16), kH * 16, 128), idH, s > 0 ? 1u : 0u);
                umma_commit(acc2);
                if (!wait(h2, par)) break;
                tc_fence_after();
#pragma unroll 1
                for (int s = 0; s < kH / 16; ++s)
                    umma_bf16(tmem + 2 * kH, umma_desc(sH + (uint32_t)(s * 2 * kFwdChunk), kFwdChunk, 128),
                              umma_desc(sW3 + (uint32_t)(s * 2 * kOut * 16), kOut * 16, 128), idO, s > 0 ? 1u : 0u);
                umma_commit(acc3);
            }
            // every MMA issued has completed before the tensor memory is released
            umma_commit(drain);
            wait(drain, 0u);
        }
    } else {
        // ------------------------------------------------------------ epilogue
        const int quarter = warp & 3, half = warp >> 2;
        const int r = 32 * quarter + lane;                      // row of the tile = TMEM lane
        const uint32_t tl = tmem + ((uint32_t)(32 * quarter) << 16);
        int j = 0;
        for (int t = blockIdx.x; t < tiles; t += gridDim.x, ++j) {
            const uint32_t par = (uint32_t)(j & 1);
            const int64_t row = (int64_t)t * kFwdRows + r;
            const bool keep = row < rows;
            // warp-uniform decisions: the TMEM loads below are warp-collective
            if (!__all_sync(0xFFFFFFFFu, !*abort_flag && wait(acc1, par))) break;
            tc_fence_after();
            fwd_epi_hidden(tl, 64 * half, bias, Hs, r, H1out && keep ? H1out + row * kH : nullptr);
            fence_async_smem();
            tc_fence_before();
            mbar_arrive(h1);
            if (!__all_sync(0xFFFFFFFFu, wait(acc2, par))) break;
            tc_fence_after();
            fwd_epi_hidden(tl + kH, 64 * half, bias + kH, Hs, r, H2out && keep ? H2out + row * kH : nullptr);
            fence_async_smem();
            tc_fence_before();
            mbar_arrive(h2);
            if (!__all_sync(0xFFFFFFFFu, wait(acc3, par))) break;
            tc_fence_after();
            if (half == 0) {
                float v[16];
                tmem_ld16(tl + 2 * kH, v);
                tmem_ld_wait();
                if (keep) {
                    float4 *y = reinterpret_cast<float4 *>(Y + row * kOut);
                    const float *bo = bias + 2 * kH;
#pragma unroll
                    for (int q = 0; q < kOut / 4; ++q)
                        y[q] = make_float4(v[4 * q] + bo[4 * q], v[4 * q + 1] + bo[4 * q + 1],
                                           v[4 * q + 2] + bo[4 * q + 2], v[4 * q + 3] + bo[4 * q + 3]);
                }
            }
            tc_fence_before();
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == kFwdMmaWarp) tmem_dealloc(tmem, kFwdTmemCols);
}

// ---------------------------------------------------------------------------
// elementwise and reduction kernels
__global__ void k_mse(const float *__restrict__ Y, const float *__restrict__ T, float *__restrict__ dY, int64_t n,
                      double *loss)
{
    double local = 0.0;
    const double inv = 1.0 / (double)n;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const float r = Y[e] - T[e];
        dY[e] = (float)(2.0 * r * inv);
        local += (double)r * r;
    }
    for (int o = 16; o > 0; o >>= 1) local += __shfl_down_sync(0xffffffffu, local, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, local * inv);
}

// dH *= (H > 0): the ReLU derivative taken from the post-activation value
__global__ void k_relu_mask(float *__restrict__ dH, const float *__restrict__ H, int64_t n)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        if (!(H[e] > 0.f)) dH[e] = 0.f;
}

// db[c] = sum_r dX[r][c]
__global__ void k_colsum(const float *__restrict__ dX, float *__restrict__ db, int rows, int cols)
{
    const int c = blockIdx.x;
    float s = 0.f;
    for (int r = threadIdx.x; r < rows; r += blockDim.x) s += dX[(int64_t)r * cols + c];
    __shared__ float red[256];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) db[c] = red[0];
}

__global__ void k_adam(float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m1,
                       float *__restrict__ m2, int64_t n, float lr, float b1, float b2, float eps, float c1, float c2)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[e];
        const float a = b1 * m1[e] + (1.f - b1) * gi;
        const float b = b2 * m2[e] + (1.f - b2) * gi * gi;
        m1[e] = a;
        m2[e] = b;
        w[e] -= lr * (a / c1) / (sqrtf(b / c2) + eps);
    }
}

// features of the listed coarse primal nodes (2D, m = 3), slot-major state
__global__ void k_features(const double *__restrict__ P, const double *__restrict__ U, int n0, int n1,
                           int64_t nnode, const int *__restrict__ nodes, int rows, float feat_scale, float t_feature,
                           float *__restrict__ X)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)rows * kIn) return;
    const int r = (int)(e / kIn), col = (int)(e % kIn);
    const int node = nodes ? nodes[r] : r;
    float v = 0.f;
    if (node < 0 || node >= nnode) {  // a bad caller-supplied node reads nothing
        X[e] = 0.f;
        return;
    }
    const int jx = node % n0, jy = node / n0;
    if (col < 144) {
        const int blk = col / 16, q = col % 16;
        const int dy = blk / 3 - 1, dx = blk % 3 - 1;
        const int x = (jx + dx + n0) % n0, y = (jy + dy + n1) % n1;
        v = feat_scale * (float)P[(int64_t)q * nnode + x + (int64_t)n0 * y];
    } else if (col < 272) {
        const int c2 = col - 144;
        const int comp = c2 / 64, blk = (c2 % 64) / 16, q = c2 % 16;
        const int vy = blk / 2 - 1, vx = blk % 2 - 1;
        const int x = (jx + vx + n0) % n0, y = (jy + vy + n1) % n1;
        v = feat_scale * (float)U[(int64_t)(comp * 16 + q) * nnode + x + (int64_t)n0 * y];
    } else if (col == 272) {
        v = t_feature;
    }
    X[e] = v;
}

// targets (restricted fine p - coarse p) / out_scale at the listed coarse nodes
__global__ void k_targets(const double *__restrict__ Pf, int nf0, int64_t nnode_f, int ratio,
                          const double *__restrict__ Pc, int nc0, int64_t nnode_c, const int *__restrict__ nodes,
                          int rows, double inv_scale, float *__restrict__ T)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)rows * kOut) return;
    const int r = (int)(e / kOut), q = (int)(e % kOut);
    const int node = nodes ? nodes[r] : r;
    if (node < 0 || node >= nnode_c) {  // a bad caller-supplied node reads nothing
        T[e] = 0.f;
        return;
    }
    const int jx = node % nc0, jy = node / nc0;
    const int a = (q % 4) + (q / 4);
    double scale = 1.0;
    for (int k = 0; k < a; ++k) scale *= ratio;
    const double fine = Pf[(int64_t)q * nnode_f + (int64_t)jx * ratio + (int64_t)nf0 * ((int64_t)jy * ratio)];
    T[e] = (float)((fine * scale - Pc[(int64_t)q * nnode_c + node]) * inv_scale);
}

__global__ void k_correct(double *__restrict__ P, int64_t nnode, const float *__restrict__ Y, int rows,
                          double out_scale)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)rows * kOut) return;
    const int r = (int)(e / kOut), q = (int)(e % kOut);
    P[(int64_t)q * nnode + r] += out_scale * (double)Y[e];
}

// Sums of squares for the correction's fallback rule: sums[0] += (out_scale Y)^2 over
// every node and slot, sums[1] += (P - snapshot)^2 (the last plain step's change of p).
__global__ void k_corr_norms(const float *__restrict__ Y, const double *__restrict__ P,
                             const double *__restrict__ snap, int64_t nnode, double out_scale, double *sums)
{
    __shared__ double red[2][256];
    double a = 0.0, b = 0.0;
    const int64_t n = nnode * kOut;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / kOut, q = e % kOut;
        const double c = out_scale * (double)Y[e];
        const double d = P[q * nnode + r] - snap[q * nnode + r];
        a = fma(c, c, a);
        b = fma(d, d, b);
    }
    red[0][threadIdx.x] = a;
    red[1][threadIdx.x] = b;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            red[0][threadIdx.x] += red[0][threadIdx.x + o];
            red[1][threadIdx.x] += red[1][threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        atomicAdd(sums, red[0][0]);
        atomicAdd(sums + 1, red[1][0]);
    }
}

// p~ += out_scale Y at every node when the correction passes the fallback rule
// sum (correction)^2 <= ratio^2 sum (last plain increment)^2 (a NaN fails it);
// counts[0] counts applied corrections, counts[1] skipped ones
__global__ void k_correct_checked(double *__restrict__ P, int64_t nnode, const float *__restrict__ Y, double out_scale,
                                  const double *__restrict__ sums, double ratio2, unsigned long long *counts)
{
    const bool ok = sums[0] <= ratio2 * sums[1];
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e == 0) atomicAdd(counts + (ok ? 0 : 1), 1ull);
    if (!ok || e >= nnode * kOut) return;
    const int64_t r = e / kOut, q = e % kOut;
    P[q * nnode + r] += out_scale * (double)Y[e];
}

static unsigned blocks_for(int64_t n, int threads)
{
    int64_t b = (n + threads - 1) / threads;
    if (b > 152 * 32) b = 152 * 32;
    return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace hl

using namespace hl;

// parameter block layout (floats): W1 [kIn][kH], b1 [kH], W2 [kH][kH], b2 [kH], W3 [kH][kOut], b3 [kOut]
static constexpr int64_t OFF_W1 = 0, OFF_B1 = OFF_W1 + (int64_t)kIn * kH, OFF_W2 = OFF_B1 + kH,
                         OFF_B2 = OFF_W2 + (int64_t)kH * kH, OFF_W3 = OFF_B2 + kH, OFF_B3 = OFF_W3 + (int64_t)kH * kOut,
                         N_PARAMS = OFF_B3 + kOut;
static_assert(N_PARAMS == HL_MLP_NPARAMS, "parameter count and header disagree");

// Y (and, if not NULL, the activations H1, H2) = forward(X) by k_mlp_forward_tc when every
// buffer is 16-byte aligned (rows of kIn, kH and kOut floats keep that alignment); *used
// tells the caller whether it ran.
static cudaError_t forward_fused(const float *w, const float *X, int rows, float *Y, float *H1, float *H2,
                                 unsigned *status, cudaStream_t st, bool *used)
{
    *used = false;
    if (rows <= 0) return cudaSuccess;
    if (((uintptr_t)X & 15) || ((uintptr_t)Y & 15) || ((uintptr_t)H1 & 15) || ((uintptr_t)H2 & 15))
        return cudaSuccess;
    static std::atomic<uint64_t> opted_in{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const uint64_t bit = 1ull << (dev & 63);
    if (!(opted_in.load() & bit)) {
        if ((e = cudaFuncSetAttribute(k_mlp_forward_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kFwdSmem)) !=
            cudaSuccess)
            return e;
        opted_in.fetch_or(bit);
    }
    int sms = 0;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const int tiles = (rows + kFwdRows - 1) / kFwdRows;
    k_mlp_forward_tc<<<(unsigned)std::min(tiles, sms), kFwdThreads, kFwdSmem, st>>>(
        X, rows, w + OFF_W1, w + OFF_B1, w + OFF_W2, w + OFF_B2, w + OFF_W3, w + OFF_B3, Y, H1, H2, status);
    *used = true;
    return cudaGetLastError();
}

struct hl_mlp {
    float *w = nullptr, *g = nullptr, *m1 = nullptr, *m2 = nullptr;  // N_PARAMS each
    float *work = nullptr;   // per-row activations: H1, H2, Y, dY, dH2, dH1
    float *splitk = nullptr; // split-K partial sums of the weight gradients
    int64_t rows_cap = 0;
    double *loss = nullptr;  // device
    double *loss_host = nullptr;
    unsigned *status = nullptr;  // device status word of the tensor-core forward (kStatusTimeout)
    int64_t adam_t = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    bool poisoned = false;
};

static thread_local std::string g_mlp_error;
static constexpr int64_t kSplitKFloats = (int64_t)64 * kIn * kH;  // 64 splits of the largest gradient

static int mlp_err(hl_mlp *h, int code, const std::string &msg)
{
    if (h) h->err = msg; else g_mlp_error = msg;
    return code;
}

static int mlp_cuda(hl_mlp *h, cudaError_t e, const char *what)
{
    if (h) h->poisoned = true;
    return mlp_err(h, HL_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define MLP_CK(h, call)                                        \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return mlp_cuda(h, e_, #call);  \
    } while (0)

static int mlp_check(hl_mlp *h)
{
    if (!h) return mlp_err(nullptr, HL_EINVAL, "null mlp handle");
    if (h->poisoned) return mlp_err(h, HL_ESTATE, "mlp handle poisoned: " + h->err);
    return HL_OK;
}

// after a stream synchronisation: a bounded wait of hl_mlp_forward's tensor-core
// kernel that expired poisons the handle
static int mlp_status(hl_mlp *h)
{
    unsigned st = 0;
    MLP_CK(h, cudaMemcpy(&st, h->status, sizeof st, cudaMemcpyDeviceToHost));
    if (st & kStatusTimeout) {
        h->poisoned = true;
        return mlp_err(h, HL_ETIMEOUT, "a bounded wait on the tensor cores expired (handle poisoned)");
    }
    return HL_OK;
}


// rows x (H1, H2, Y, dY, dH2, dH1)
static int ensure_rows(hl_mlp *h, int64_t rows)
{
    if (rows <= h->rows_cap) return HL_OK;
    if (h->work) {
        MLP_CK(h, cudaStreamSynchronize(h->stream));
        cudaFree(h->work);
        h->work = nullptr;
    }
    const int64_t per = 2 * kH + 2 * kOut + 2 * kH;
    cudaError_t e = cudaMalloc(&h->work, (size_t)rows * per * sizeof(float));
    if (e != cudaSuccess) {
        cudaGetLastError();
        h->rows_cap = 0;
        return mlp_err(h, HL_ENOMEM, "mlp workspace allocation failed");
    }
    h->rows_cap = rows;
    return HL_OK;
}

struct Work {
    float *H1, *H2, *Y, *dY, *dH2, *dH1;
};

static Work work_ptrs(hl_mlp *h, int64_t rows)
{
    Work w;
    w.H1 = h->work;
    w.H2 = w.H1 + rows * kH;
    w.Y = w.H2 + rows * kH;
    w.dY = w.Y + rows * kOut;
    w.dH2 = w.dY + rows * kOut;
    w.dH1 = w.dH2 + rows * kH;
    return w;
}

static cudaError_t forward_into(hl_mlp *h, const float *X, int rows, const Work &w, float *Y,
                                cudaStream_t st)
{
    cudaError_t e;
    if ((e = gemm({X, kIn, 1}, {h->w + OFF_W1, kH, 1}, w.H1, kH, rows, kH, kIn, h->w + OFF_B1, 1, st)) != cudaSuccess)
        return e;
    if ((e = gemm({w.H1, kH, 1}, {h->w + OFF_W2, kH, 1}, w.H2, kH, rows, kH, kH, h->w + OFF_B2, 1, st)) != cudaSuccess)
        return e;
    return gemm({w.H2, kH, 1}, {h->w + OFF_W3, kOut, 1}, Y, kOut, rows, kOut, kH, h->w + OFF_B3, 0, st);
}

// the network applied to rows of X: the fused tensor-core kernel, or the three GEMMs
// when X or Y is not 16-byte aligned
static cudaError_t forward_any(hl_mlp *h, const float *X, int rows, float *Y, unsigned *status, cudaStream_t st)
{
    bool used = false;
    cudaError_t e = forward_fused(h->w, X, rows, Y, nullptr, nullptr, status, st, &used);
    if (e != cudaSuccess || used) return e;
    return forward_into(h, X, rows, work_ptrs(h, rows), Y, st);
}

extern "C" int hl_mlp_create(uint64_t seed, hl_mlp **out)
{
    if (!out) return mlp_err(nullptr, HL_EINVAL, "out is NULL");
    *out = nullptr;
    hl_mlp *h = new hl_mlp();
    cudaError_t e;
    if ((e = cudaMalloc(&h->w, N_PARAMS * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&h->g, N_PARAMS * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&h->m1, N_PARAMS * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&h->m2, N_PARAMS * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&h->loss, sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&h->splitk, kSplitKFloats * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&h->status, sizeof(unsigned))) != cudaSuccess ||
        (e = cudaMallocHost(&h->loss_host, sizeof(double))) != cudaSuccess) {
        std::string msg = std::string("mlp set-up failed: ") + cudaGetErrorString(e);
        cudaGetLastError();
        hl_mlp_destroy(h);
        return mlp_err(nullptr, e == cudaErrorMemoryAllocation ? HL_ENOMEM : HL_ECUDA, msg);
    }
    // He initialisation (normal, std sqrt(2/fan_in); last layer sqrt(1/fan_in)), zero biases
    std::vector<float> w(N_PARAMS, 0.f);
    std::mt19937_64 rng(seed);
    std::normal_distribution<float> nd(0.f, 1.f);
    for (int64_t i = 0; i < (int64_t)kIn * kH; ++i) w[OFF_W1 + i] = nd(rng) * std::sqrt(2.f / kIn);
    for (int64_t i = 0; i < (int64_t)kH * kH; ++i) w[OFF_W2 + i] = nd(rng) * std::sqrt(2.f / kH);
    for (int64_t i = 0; i < (int64_t)kH * kOut; ++i) w[OFF_W3 + i] = nd(rng) * std::sqrt(1.f / kH);
    if ((e = cudaMemcpy(h->w, w.data(), N_PARAMS * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemset(h->g, 0, N_PARAMS * sizeof(float))) != cudaSuccess ||
        (e = cudaMemset(h->m1, 0, N_PARAMS * sizeof(float))) != cudaSuccess ||
        (e = cudaMemset(h->m2, 0, N_PARAMS * sizeof(float))) != cudaSuccess ||
        (e = cudaMemset(h->status, 0, sizeof(unsigned))) != cudaSuccess) {
        std::string msg = std::string("mlp set-up failed: ") + cudaGetErrorString(e);
        hl_mlp_destroy(h);
        return mlp_err(nullptr, HL_ECUDA, msg);
    }
    *out = h;
    return HL_OK;
}

extern "C" void hl_mlp_destroy(hl_mlp *h)
{
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream); else cudaDeviceSynchronize();
    cudaFree(h->w);
    cudaFree(h->g);
    cudaFree(h->m1);
    cudaFree(h->m2);
    cudaFree(h->work);
    cudaFree(h->splitk);
    cudaFree(h->status);
    cudaFree(h->loss);
    if (h->loss_host) cudaFreeHost(h->loss_host);
    delete h;
}

extern "C" const char *hl_mlp_last_error(const hl_mlp *h) { return h ? h->err.c_str() : g_mlp_error.c_str(); }

extern "C" int hl_mlp_set_stream(hl_mlp *h, void *cuda_stream)
{
    int rc = mlp_check(h);
    if (rc) return rc;
    MLP_CK(h, cudaStreamSynchronize(h->stream));
    h->stream = (cudaStream_t)cuda_stream;
    return HL_OK;
}

extern "C" int hl_mlp_params(hl_mlp *h, float *get_params, const float *set_params, float *get_grads)
{
    int rc = mlp_check(h);
    if (rc) return rc;
    MLP_CK(h, cudaStreamSynchronize(h->stream));
    if ((rc = mlp_status(h))) return rc;
    if (set_params) {
        MLP_CK(h, cudaMemcpy(h->w, set_params, N_PARAMS * sizeof(float), cudaMemcpyHostToDevice));
        MLP_CK(h, cudaMemset(h->m1, 0, N_PARAMS * sizeof(float)));
        MLP_CK(h, cudaMemset(h->m2, 0, N_PARAMS * sizeof(float)));
        h->adam_t = 0;
    }
    if (get_params) MLP_CK(h, cudaMemcpy(get_params, h->w, N_PARAMS * sizeof(float), cudaMemcpyDeviceToHost));
    if (get_grads) MLP_CK(h, cudaMemcpy(get_grads, h->g, N_PARAMS * sizeof(float), cudaMemcpyDeviceToHost));
    return HL_OK;
}

extern "C" int hl_mlp_forward(hl_mlp *h, const float *X_dev, int rows, float *Y_dev)
{
    int rc = mlp_check(h);
    if (rc) return rc;
    if (rows < 0 || (!X_dev && rows) || (!Y_dev && rows)) return mlp_err(h, HL_EINVAL, "bad forward arguments");
    if (rows == 0) return HL_OK;
    // the tensor-core kernel needs no workspace; the GEMM path keeps H1 and H2 in it
    bool fused = false;
    MLP_CK(h, forward_fused(h->w, X_dev, rows, Y_dev, nullptr, nullptr, h->status, h->stream, &fused));
    if (fused) return HL_OK;
    rc = ensure_rows(h, rows);
    if (rc) return rc;
    MLP_CK(h, forward_into(h, X_dev, rows, work_ptrs(h, rows), Y_dev, h->stream));
    return HL_OK;
}

extern "C" int hl_mlp_loss_grad(hl_mlp *h, const float *X_dev, const float *T_dev, int rows, double *loss)
{
    int rc = mlp_check(h);
    if (rc) return rc;
    if (rows <= 0 || !X_dev || !T_dev) return mlp_err(h, HL_EINVAL, "bad loss_grad arguments");
    rc = ensure_rows(h, rows);
    if (rc) return rc;
    const Work w = work_ptrs(h, rows);
    const cudaStream_t st = h->stream;
    bool fused = false;   // the tensor-core forward keeps H1 and H2 for the backward GEMMs
    MLP_CK(h, forward_fused(h->w, X_dev, rows, w.Y, w.H1, w.H2, h->status, st, &fused));
    if (!fused) MLP_CK(h, forward_into(h, X_dev, rows, w, w.Y, st));
    MLP_CK(h, cudaMemsetAsync(h->loss, 0, sizeof(double), st));
    const int64_t ny = (int64_t)rows * kOut;
    k_mse<<<blocks_for(ny, 256), 256, 0, st>>>(w.Y, T_dev, w.dY, ny, h->loss);
    MLP_CK(h, cudaGetLastError());
    // layer 3
    MLP_CK(h, gemm({w.H2, 1, kH}, {w.dY, kOut, 1}, h->g + OFF_W3, kOut, kH, kOut, rows, nullptr, 0, st, h->splitk,
                   kSplitKFloats));
    k_colsum<<<kOut, 256, 0, st>>>(w.dY, h->g + OFF_B3, rows, kOut);
    MLP_CK(h, gemm({w.dY, kOut, 1}, {h->w + OFF_W3, 1, kOut}, w.dH2, kH, rows, kH, kOut, nullptr, 0, st));
    k_relu_mask<<<blocks_for((int64_t)rows * kH, 256), 256, 0, st>>>(w.dH2, w.H2, (int64_t)rows * kH);
    // layer 2
    MLP_CK(h, gemm({w.H1, 1, kH}, {w.dH2, kH, 1}, h->g + OFF_W2, kH, kH, kH, rows, nullptr, 0, st, h->splitk,
                   kSplitKFloats));
    k_colsum<<<kH, 256, 0, st>>>(w.dH2, h->g + OFF_B2, rows, kH);
    MLP_CK(h, gemm({w.dH2, kH, 1}, {h->w + OFF_W2, 1, kH}, w.dH1, kH, rows, kH, kH, nullptr, 0, st));
    k_relu_mask<<<blocks_for((int64_t)rows * kH, 256), 256, 0, st>>>(w.dH1, w.H1, (int64_t)rows * kH);
    // layer 1
    MLP_CK(h, gemm({X_dev, 1, kIn}, {w.dH1, kH, 1}, h->g + OFF_W1, kH, kIn, kH, rows, nullptr, 0, st, h->splitk,
                   kSplitKFloats));
    k_colsum<<<kH, 256, 0, st>>>(w.dH1, h->g + OFF_B1, rows, kH);
    MLP_CK(h, cudaGetLastError());
    if (loss) {
        MLP_CK(h, cudaMemcpyAsync(h->loss_host, h->loss, sizeof(double), cudaMemcpyDeviceToHost, st));
        MLP_CK(h, cudaStreamSynchronize(st));
        if ((rc = mlp_status(h))) return rc;
        *loss = *h->loss_host;
    }
    return HL_OK;
}

extern "C" int hl_mlp_grad_buffer(hl_mlp *h, float **grads_dev)
{
    if (!grads_dev) return mlp_err(h, HL_EINVAL, "grads_dev is NULL");
    int rc = mlp_check(h);
    if (rc) return rc;
    *grads_dev = h->g;
    return HL_OK;
}

extern "C" int hl_mlp_adam_step(hl_mlp *h, float lr)
{
    int rc = mlp_check(h);
    if (rc) return rc;
    if (!(lr > 0.f) || !std::isfinite(lr)) return mlp_err(h, HL_EINVAL, "lr must be finite and > 0");
    h->adam_t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)h->adam_t), c2 = 1.f - std::pow(b2, (float)h->adam_t);
    k_adam<<<blocks_for(N_PARAMS, 256), 256, 0, h->stream>>>(h->w, h->g, h->m1, h->m2, N_PARAMS, lr, b1, b2, 1e-8f,
                                                            c1, c2);
    MLP_CK(h, cudaGetLastError());
    return HL_OK;
}

// ---------------------------------------------------------------------------
// Minibatch draw on the device: row i of step `step` takes pool row
// splitmix64(seed + (step * rows + i) * golden) mod pool_rows, with SplitMix64
// the counter-based generator of Steele, Lea and Flood (OOPSLA 2014): add the
// golden-ratio increment, then the xor-shift / multiply finaliser.
__device__ __forceinline__ uint64_t splitmix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

__global__ void k_sample(const float *__restrict__ Xp, const float *__restrict__ Tp, int64_t pool_rows, int rows,
                         uint64_t seed, uint64_t step, float *__restrict__ X, float *__restrict__ T)
{
    const int r = blockIdx.x;
    const uint64_t ctr = step * (uint64_t)rows + (uint64_t)r;
    const int64_t src = (int64_t)(splitmix64(seed + (ctr + 1) * 0x9e3779b97f4a7c15ull) % (uint64_t)pool_rows);
    for (int c = threadIdx.x; c < kIn; c += blockDim.x) X[(int64_t)r * kIn + c] = Xp[src * kIn + c];
    if (Tp)
        for (int c = threadIdx.x; c < kOut; c += blockDim.x) T[(int64_t)r * kOut + c] = Tp[src * kOut + c];
}

extern "C" int hl_mlp_sample(hl_mlp *h, const float *X_pool, const float *T_pool, int64_t pool_rows, int rows,
                             uint64_t seed, uint64_t step, float *X_dev, float *T_dev)
{
    int rc = mlp_check(h);
    if (rc) return rc;
    if (!X_pool || !X_dev || pool_rows < 1 || rows < 1 || (T_pool && !T_dev))
        return mlp_err(h, HL_EINVAL, "bad sample arguments");
    k_sample<<<rows, 96, 0, h->stream>>>(X_pool, T_pool, pool_rows, rows, seed, step, X_dev, T_dev);
    MLP_CK(h, cudaGetLastError());
    return HL_OK;
}

// ---------------------------------------------------------------------------
static int solver_ok(const hl_solver *s)
{
    if (!s) return mlp_err(nullptr, HL_EINVAL, "null solver handle");
    if (s->poisoned) return mlp_err(nullptr, HL_ESTATE, "solver handle poisoned");
    if (s->dim != 2 || s->m != 3 || s->shots.size() != 1)
        return mlp_err(nullptr, HL_EINVAL, "the learned correction needs a single 2D m = 3 grid");
    if (!s->unit_box) return mlp_err(nullptr, HL_EINVAL, "the learned correction needs a unit-box grid");
    return HL_OK;
}

extern "C" int hl_features(const hl_solver *coarse, const int *nodes_dev, int rows, float feat_scale,
                           float t_feature, float *X_dev)
{
    int rc = solver_ok(coarse);
    if (rc) return rc;
    if (rows < 0 || (rows && !X_dev)) return mlp_err(nullptr, HL_EINVAL, "bad feature arguments");
    if (!nodes_dev && rows > coarse->shots[0].nnode) return mlp_err(nullptr, HL_EINVAL, "rows exceed the grid");
    if (rows == 0) return HL_OK;
    const Shot &s = coarse->shots[0];
    const int64_t n = (int64_t)rows * kIn;
    k_features<<<(unsigned)((n + 255) / 256), 256, 0, coarse->stream>>>(
        coarse->p, coarse->u, (int)s.n[0], (int)s.n[1], s.nnode, nodes_dev, rows, feat_scale, t_feature, X_dev);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? HL_OK : mlp_err(nullptr, HL_ECUDA, cudaGetErrorString(e));
}

extern "C" int hl_targets(const hl_solver *fine, int ratio, const hl_solver *coarse, const int *nodes_dev, int rows,
                          double out_scale, float *T_dev)
{
    int rc = solver_ok(fine);
    if (rc) return rc;
    rc = solver_ok(coarse);
    if (rc) return rc;
    const Shot &f = fine->shots[0], &c = coarse->shots[0];
    if (ratio < 1 || f.n[0] != c.n[0] * ratio || f.n[1] != c.n[1] * ratio)
        return mlp_err(nullptr, HL_EINVAL, "fine grid must be ratio times the coarse grid");
    if (rows < 0 || (rows && !T_dev) || !(out_scale > 0.0)) return mlp_err(nullptr, HL_EINVAL, "bad target arguments");
    if (!nodes_dev && rows > c.nnode) return mlp_err(nullptr, HL_EINVAL, "rows exceed the grid");
    if (rows == 0) return HL_OK;
    const int64_t n = (int64_t)rows * kOut;
    k_targets<<<(unsigned)((n + 255) / 256), 256, 0, coarse->stream>>>(fine->p, (int)f.n[0], f.nnode, ratio, coarse->p,
                                                                        (int)c.n[0], c.nnode, nodes_dev, rows,
                                                                        1.0 / out_scale, T_dev);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? HL_OK : mlp_err(nullptr, HL_ECUDA, cudaGetErrorString(e));
}

extern "C" int hl_apply_correction(hl_solver *coarse, hl_mlp *mlp, float feat_scale, float t_feature,
                                   double out_scale)
{
    int rc = solver_ok(coarse);
    if (rc) return rc;
    rc = mlp_check(mlp);
    if (rc) return rc;
    const Shot &s = coarse->shots[0];
    const int rows = (int)s.nnode;
    // features (rows x kIn) live after the activations in one workspace
    const int64_t per_row = 2 * kH + 2 * kOut + 2 * kH;
    rc = ensure_rows(mlp, rows + ((int64_t)rows * kIn + per_row - 1) / per_row);
    if (rc) return rc;
    // order the correction after the solver's pending work
    if (mlp->stream != coarse->stream) {
        MLP_CK(mlp, cudaStreamSynchronize(coarse->stream));
    }
    const Work w = work_ptrs(mlp, rows);
    float *X = w.dH1 + (int64_t)rows * kH;
    const int64_t nx = (int64_t)rows * kIn;
    k_features<<<(unsigned)((nx + 255) / 256), 256, 0, mlp->stream>>>(coarse->p, coarse->u, (int)s.n[0], (int)s.n[1],
                                                                       s.nnode, nullptr, rows, feat_scale, t_feature, X);
    MLP_CK(mlp, cudaGetLastError());
    MLP_CK(mlp, forward_any(mlp, X, rows, w.Y, coarse->status, mlp->stream));
    const int64_t ny = (int64_t)rows * kOut;
    k_correct<<<(unsigned)((ny + 255) / 256), 256, 0, mlp->stream>>>(coarse->p, s.nnode, w.Y, rows, out_scale);
    MLP_CK(mlp, cudaGetLastError());
    if (mlp->stream != coarse->stream) MLP_CK(mlp, cudaStreamSynchronize(mlp->stream));
    return HL_OK;
}

// ---------------------------------------------------------------------------
// The learned correction inside the stepping loop (hl_set_correction), with the
// plain solver as fallback: see include/hl.h.
extern "C" int hl_set_correction(hl_solver *h, hl_mlp *mlp, int every_k_steps, float feat_scale, float t_feature,
                                 double out_scale, double max_ratio)
{
    if (!h) return mlp_err(nullptr, HL_EINVAL, "null solver handle");
    if (!mlp) {
        h->corr_mlp = nullptr;
        return HL_OK;
    }
    int rc = solver_ok(h);
    if (rc) return rc;
    rc = mlp_check(mlp);
    if (rc) return rc;
    if (every_k_steps < 1) return mlp_err(nullptr, HL_EINVAL, "every_k_steps must be >= 1");
    if (!(out_scale > 0.0) || !std::isfinite(out_scale) || !std::isfinite(feat_scale) || !std::isfinite(t_feature))
        return mlp_err(nullptr, HL_EINVAL, "scales must be finite (out_scale > 0)");
    if (!(max_ratio > 0.0)) return mlp_err(nullptr, HL_EINVAL, "max_ratio must be > 0");
    if (h->precision != HL_FP64) return mlp_err(nullptr, HL_EINVAL, "the learned correction runs with HL_FP64 stepping");
    const int rows = (int)h->shots[0].nnode;
    const int64_t per_row = 2 * kH + 2 * kOut + 2 * kH;
    rc = ensure_rows(mlp, rows + ((int64_t)rows * kIn + per_row - 1) / per_row);
    if (rc) return rc;
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e == cudaSuccess && !h->corr_snap) e = cudaMalloc(&h->corr_snap, (size_t)h->nq * rows * sizeof(double));
    if (e == cudaSuccess && !h->corr_sums) e = cudaMalloc(&h->corr_sums, 2 * sizeof(double));
    if (e == cudaSuccess && !h->corr_counts) {
        e = cudaMalloc(&h->corr_counts, 2 * sizeof(unsigned long long));
        if (e == cudaSuccess) e = cudaMemset(h->corr_counts, 0, 2 * sizeof(unsigned long long));
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return mlp_err(nullptr, HL_ENOMEM, std::string("correction set-up: ") + cudaGetErrorString(e));
    }
    h->corr_mlp = mlp;
    h->corr_every = every_k_steps;
    h->corr_feat_scale = feat_scale;
    h->corr_t_feature = t_feature;
    h->corr_out_scale = out_scale;
    h->corr_ratio = max_ratio;
    return HL_OK;
}

extern "C" int hl_correction_stats(hl_solver *h, int64_t *applied, int64_t *skipped)
{
    if (!h) return mlp_err(nullptr, HL_EINVAL, "null solver handle");
    unsigned long long c[2] = {0ull, 0ull};
    if (h->corr_counts) {
        cudaError_t e = cudaStreamSynchronize(h->stream);
        if (e == cudaSuccess) e = cudaMemcpy(c, h->corr_counts, sizeof c, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return mlp_err(nullptr, HL_ECUDA, cudaGetErrorString(e));
    }
    if (applied) *applied = (int64_t)c[0];
    if (skipped) *skipped = (int64_t)c[1];
    return HL_OK;
}

namespace hl {

// Stream-ordered: features of every node, the network, the fallback rule's sums, the
// checked FP64 addition.  Runs on st (the solver's stream); no host synchronisation.
cudaError_t apply_correction_checked(hl_solver *h, cudaStream_t st)
{
    hl_mlp *mlp = h->corr_mlp;
    const Shot &s = h->shots[0];
    const int rows = (int)s.nnode;
    const Work w = work_ptrs(mlp, rows);
    float *X = w.dH1 + (int64_t)rows * kH;
    const int64_t nx = (int64_t)rows * kIn;
    k_features<<<(unsigned)((nx + 255) / 256), 256, 0, st>>>(h->p, h->u, (int)s.n[0], (int)s.n[1], s.nnode, nullptr,
                                                              rows, h->corr_feat_scale, h->corr_t_feature, X);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if ((e = forward_any(mlp, X, rows, w.Y, h->status, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(h->corr_sums, 0, 2 * sizeof(double), st)) != cudaSuccess) return e;
    const int64_t ny = (int64_t)rows * kOut;
    k_corr_norms<<<blocks_for(ny, 256), 256, 0, st>>>(w.Y, h->p, h->corr_snap, s.nnode, h->corr_out_scale,
                                                      h->corr_sums);
    k_correct_checked<<<(unsigned)((ny + 255) / 256), 256, 0, st>>>(h->p, s.nnode, w.Y, h->corr_out_scale,
                                                                    h->corr_sums, h->corr_ratio * h->corr_ratio,
                                                                    h->corr_counts);
    return cudaGetLastError();
}

}  // namespace hl
