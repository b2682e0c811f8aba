// FP64 Hermite-leapfrog half-step kernels for sm_103a.
//
// One thread owns one target node.  For the p-half the partner field is u
// (dim components) on the dual grid; for the u-half it is p on the primal
// grid (Section 2, eqs. final1/LFloop; Section 3.1.2, eqs. pdup/vdup).
//
// The fused per-node operator.  Composing the per-axis Hermite-Birkhoff
// inverse H (Section 2, eq. interp; the tensor product of Section 5) with the
// Cauchy-Kowalevsky series gives, for direction i, a linear map from the
// 2^dim vertex blocks to the (m+1)^dim outputs.  Reflecting the cell about its
// centre along axis k swaps the two vertices on that axis and flips the sign
// of odd derivatives; the series term is odd along axis i and even along the
// other axes.  Hence the block of vertex v equals the block of the all-lower
// vertex times prod_{k: v_k = 1} sigma_k with sigma_k = (-1)^(s_k + l_k + [k==i]).
// So the kernel first forms the 2^dim sums/differences of the vertex values
// (a Walsh-Hadamard butterfly over the vertices) and then contracts each
// output slot s with a single (m+1)^dim operator M0_i, picking for every
// (s, l) the butterfly entry whose per-axis sum/difference choice matches the
// parity above.  This needs (m+1)^(2 dim) instead of 2^dim (m+1)^(2 dim)
// multiply-adds per direction.
//
// Structural zeros of M0_i: if l_k = 0 on some axis k with t = s_k + [k==i]
// even and t >= 2, every coefficient index a_k >= t on that axis is even and
// >= 2, and constant end data feed no even coefficient of degree >= 2, so the
// entry vanishes.  The host verifies the rule on the computed operator; the
// kernels skip those entries at compile time.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "hl_internal.h"

namespace hl {

__host__ __device__ constexpr int ipow_c(int b, int e) { return e == 0 ? 1 : b * ipow_c(b, e - 1); }

template <int D, int M>
struct Shape {
    static constexpr int n = M + 1;                 // slots per axis
    static constexpr int NQ = ipow_c(n, D);         // slots per node
    static constexpr int NV = 1 << D;               // cell vertices
    static constexpr int NCOEF = D * NQ * NQ;       // dense (i, l, s) table
    // the table travels in the kernel parameter bank when it fits
    static constexpr bool kParam = NCOEF * 8 <= 28 * 1024;
    // the u-half keeps all dim output blocks live only when they fit in registers
    static constexpr bool kUFused = D * NQ <= 96;
    // paired kernels (two nodes per thread) while both nodes' outputs fit
    static constexpr bool kPairP = D >= 2 && 2 * NQ <= 64;
    static constexpr bool kPairU = D >= 2 && 2 * D * NQ <= 64;
};

__host__ __device__ constexpr bool coef_nonzero(int D, int n, int i, int s, int l)
{
    for (int k = 0; k < D; ++k) {
        const int sk = s % n, lk = l % n;
        s /= n;
        l /= n;
        const int t = sk + (k == i ? 1 : 0);
        if (lk == 0 && (t % 2) == 0 && t >= 2) return false;
    }
    return true;
}

// butterfly entry for (i, s, l): bit k set = difference (lower - upper) on axis k
__host__ __device__ constexpr int bfly_pattern(int D, int n, int i, int s, int l)
{
    int pat = 0;
    for (int k = 0; k < D; ++k) {
        const int sk = s % n, lk = l % n;
        s /= n;
        l /= n;
        if ((sk + lk + (k == i ? 1 : 0)) & 1) pat |= 1 << k;
    }
    return pat;
}

__host__ __device__ constexpr int coef_index(int NQ, int i, int l, int s) { return (i * NQ + l) * NQ + s; }

// Coefficient table holder: by value in the parameter bank, or a global pointer.
template <int D, int M, bool P = Shape<D, M>::kParam>
struct CoefArg;
template <int D, int M>
struct CoefArg<D, M, true> {
    double v[Shape<D, M>::NCOEF];
    __device__ __forceinline__ double get(int idx) const { return v[idx]; }
};
template <int D, int M>
struct CoefArg<D, M, false> {
    const double *__restrict__ v;
    __device__ __forceinline__ double get(int idx) const { return __ldg(v + idx); }
};

struct GridDesc {
    int n[3];        // nodes per axis (1 for unused axes)
    int64_t nnode;   // n0*n1*n2
};

// In-place Walsh-Hadamard butterfly over the 2^D vertex values:
// afterwards x[pat] = sum_v prod_{k: v_k=1} (bit k of pat ? -1 : +1) x_v.
// The levels run in the order x, z, y: with y last, the paired kernels (two
// nodes adjacent along y) share every level but the last and stay bitwise
// identical to the one-node kernels.
template <int D>
__device__ __forceinline__ void butterfly(double *x)
{
    constexpr int order[3] = {0, 2, 1};
#pragma unroll
    for (int o = 0; o < 3; ++o) {
        const int k = order[o];
        if (k >= D) continue;
#pragma unroll
        for (int v = 0; v < (1 << D); ++v) {
            if (!(v & (1 << k))) {
                const double a = x[v], b = x[v | (1 << k)];
                x[v] = a + b;
                x[v | (1 << k)] = a - b;
            }
        }
    }
}

// Node index of the 2^D cell vertices on the partner grid.  lo = -1 for the
// p-half (dual nodes j-1, j), 0 for the u-half (primal nodes j, j+1).
template <int D>
__device__ __forceinline__ void vertex_nodes(const GridDesc &g, int64_t node, int lo, int *vtx)
{
    int j[3] = {0, 0, 0};
    int64_t t = node;
#pragma unroll
    for (int k = 0; k < D; ++k) {
        j[k] = (int)(t % g.n[k]);
        t /= g.n[k];
    }
    int lower[3], upper[3];
#pragma unroll
    for (int k = 0; k < D; ++k) {
        int a = j[k] + lo, b = j[k] + lo + 1;
        if (a < 0) a += g.n[k];
        if (b >= g.n[k]) b -= g.n[k];
        lower[k] = a;
        upper[k] = b;
    }
#pragma unroll
    for (int v = 0; v < (1 << D); ++v) {
        int idx = 0, stride = 1;
#pragma unroll
        for (int k = 0; k < D; ++k) {
            idx += ((v >> k) & 1 ? upper[k] : lower[k]) * stride;
            stride *= g.n[k];
        }
        vtx[v] = idx;
    }
}

// Inf/NaN test on the exponent bits: integer pipe only (a floating-point
// compare would take a slot of the FP64 pipe, the kernels' bottleneck)
__device__ __forceinline__ bool nonfinite(double v)
{
    return ((unsigned)__double2hiint(v) & 0x7FF00000u) == 0x7FF00000u;
}

__device__ __forceinline__ void report_nonfinite(bool bad, unsigned *status)
{
    const unsigned mask = __activemask();
    const unsigned votes = __ballot_sync(mask, bad);
    if (votes && (threadIdx.x & 31) == (unsigned)(__ffs(mask) - 1)) atomicOr(status, 1u);
}

// ---------------------------------------------------------------------------
// p-half at one primal node: out[s] += sum_i sum_l coef(i,l,s) * bfly_i,l[pattern]
// (the host stores the coefficients already negated: p_new = p_old - series).
// Callers start out[] at zero and add the node's own value last, so the
// increment is summed at its own magnitude before the single final rounding.
// Loads go through `ld(comp, slot, vertex_node)`.
template <int D, int M, class C, class Ld>
__device__ __forceinline__ void p_node(const C &coef, const Ld &ld, const int *vtx, double *out)
{
    using S = Shape<D, M>;
#pragma unroll
    for (int i = 0; i < D; ++i) {
#pragma unroll
        for (int l = 0; l < S::NQ; ++l) {
            double x[S::NV];
#pragma unroll
            for (int v = 0; v < S::NV; ++v) x[v] = ld(i, l, vtx[v]);
            butterfly<D>(x);
#pragma unroll
            for (int s = 0; s < S::NQ; ++s) {
                if (coef_nonzero(D, S::n, i, s, l))
                    out[s] = fma(coef.get(coef_index(S::NQ, i, l, s)), x[bfly_pattern(D, S::n, i, s, l)], out[s]);
            }
        }
    }
}

// u-half at one dual node, directions I0..I0+NI-1: out[(i-I0)*NQ + s].
template <int D, int M, int I0, int NI, class C, class Ld>
__device__ __forceinline__ void u_node(const C &coef, const Ld &ld, const int *vtx, double *out)
{
    using S = Shape<D, M>;
#pragma unroll
    for (int l = 0; l < S::NQ; ++l) {
        double x[S::NV];
#pragma unroll
        for (int v = 0; v < S::NV; ++v) x[v] = ld(0, l, vtx[v]);
        butterfly<D>(x);
#pragma unroll
        for (int ii = 0; ii < NI; ++ii) {
            const int i = I0 + ii;
#pragma unroll
            for (int s = 0; s < S::NQ; ++s) {
                if (coef_nonzero(D, S::n, i, s, l))
                    out[ii * S::NQ + s] =
                        fma(coef.get(coef_index(S::NQ, i, l, s)), x[bfly_pattern(D, S::n, i, s, l)], out[ii * S::NQ + s]);
            }
        }
    }
}

struct GlobalLd {
    const double *__restrict__ base;
    int64_t slot_stride;   // nnode
    int nq;
    __device__ __forceinline__ double operator()(int comp, int slot, int node) const
    {
        return __ldg(base + (int64_t)(comp * nq + slot) * slot_stride + node);
    }
};

struct SharedLd {
    const double *base;
    int slot_stride;
    int nq;
    __device__ __forceinline__ double operator()(int comp, int slot, int node) const
    {
        return base[(comp * nq + slot) * slot_stride + node];
    }
};

// ---------------------------------------------------------------------------
// Grid kernels: one launch per half-step over a flattened list of tiles.
// A tile is blockDim.x x blockDim.y nodes of one shot (x-fastest); the shot
// table maps the block index to its shot, so one launch covers any number of
// independent grids (a single solve is a batch of one).

// coefficient providers: one table in the parameter bank for every shot, or a
// per-shot table in global memory
template <int D, int M>
struct CoefParam {
    CoefArg<D, M, Shape<D, M>::kParam> c;
    __device__ __forceinline__ const CoefArg<D, M, Shape<D, M>::kParam> &at(int) const { return c; }
};
template <int D, int M>
struct CoefShots {
    const double *__restrict__ base;   // n_shots tables of NCOEF doubles
    __device__ __forceinline__ CoefArg<D, M, false> at(int shot) const
    {
        return CoefArg<D, M, false>{base + (int64_t)shot * Shape<D, M>::NCOEF};
    }
};

// The shot of this block: the last shot whose first tile is <= blockIdx.x.
__device__ __forceinline__ void find_shot(const ShotDesc *__restrict__ shots, int n_shots, int &shot, ShotDesc &sd)
{
    const int tile = blockIdx.x;
    int lo = 0, hi = n_shots - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (shots[mid].tile_begin <= tile) lo = mid; else hi = mid - 1;
    }
    shot = lo;
    sd = shots[lo];
}

// Locate this block's shot and node; false if the thread is outside the grid.
template <int D>
__device__ __forceinline__ bool tile_node(const ShotDesc *__restrict__ shots, int n_shots, int &shot, ShotDesc &sd,
                                          int64_t &node)
{
    find_shot(shots, n_shots, shot, sd);
    int t = blockIdx.x - sd.tile_begin;
    const int tx = t % sd.tiles[0];
    t /= sd.tiles[0];
    const int ty = t % sd.tiles[1];
    const int tz = t / sd.tiles[1];
    const int ix = tx * blockDim.x + threadIdx.x;
    const int iy = ty * blockDim.y + threadIdx.y;
    if (ix >= sd.n[0] || iy >= sd.n[1] || tz >= sd.n[2]) return false;
    node = ix + (int64_t)sd.n[0] * (iy + (int64_t)sd.n[1] * tz);
    return true;
}

template <int D, int M, class CP>
__global__ void __launch_bounds__(256) k_p_half(const double *__restrict__ U, double *__restrict__ P,
                                                const ShotDesc *__restrict__ shots, int n_shots, CP cp,
                                                unsigned *status)
{
    using S = Shape<D, M>;
    int shot;
    ShotDesc sd;
    int64_t node;
    if (!tile_node<D>(shots, n_shots, shot, sd, node)) return;
    const GridDesc g{{sd.n[0], sd.n[1], sd.n[2]}, sd.nnode};
    const double *Us = U + sd.u_off;
    double *Ps = P + sd.p_off;
    int vtx[S::NV];
    vertex_nodes<D>(g, node, -1, vtx);
    double out[S::NQ];
#pragma unroll
    for (int s = 0; s < S::NQ; ++s) out[s] = 0.0;
    GlobalLd ld{Us, g.nnode, S::NQ};
    p_node<D, M>(cp.at(shot), ld, vtx, out);
    bool bad = false;
#pragma unroll
    for (int s = 0; s < S::NQ; ++s) {
        const double v = Ps[(int64_t)s * g.nnode + node] + out[s];
        Ps[(int64_t)s * g.nnode + node] = v;
        bad |= nonfinite(v);
    }
    report_nonfinite(bad, status);
}

template <int D, int M, int I0, int NI, class CP>
__global__ void __launch_bounds__(256) k_u_half(const double *__restrict__ P, double *__restrict__ U,
                                                const ShotDesc *__restrict__ shots, int n_shots, CP cp,
                                                unsigned *status)
{
    using S = Shape<D, M>;
    int shot;
    ShotDesc sd;
    int64_t node;
    if (!tile_node<D>(shots, n_shots, shot, sd, node)) return;
    const GridDesc g{{sd.n[0], sd.n[1], sd.n[2]}, sd.nnode};
    const double *Ps = P + sd.p_off;
    double *Us = U + sd.u_off;
    int vtx[S::NV];
    vertex_nodes<D>(g, node, 0, vtx);
    double out[NI * S::NQ];
#pragma unroll
    for (int e = 0; e < NI * S::NQ; ++e) out[e] = 0.0;
    GlobalLd ld{Ps, g.nnode, S::NQ};
    u_node<D, M, I0, NI>(cp.at(shot), ld, vtx, out);
    bool bad = false;
#pragma unroll
    for (int ii = 0; ii < NI; ++ii)
#pragma unroll
        for (int s = 0; s < S::NQ; ++s) {
            double *dst = Us + (int64_t)((I0 + ii) * S::NQ + s) * g.nnode + node;
            const double v = *dst + out[ii * S::NQ + s];
            *dst = v;
            bad |= nonfinite(v);
        }
    report_nonfinite(bad, status);
}

// ---------------------------------------------------------------------------
// Paired grid kernels: one thread owns two nodes adjacent along y, rows iy and
// iy+1 of a tile whose height is 2*blockDim.y (the tile table is the same as
// for the one-node kernels).  The two cells share one y-row of vertices, whose
// butterfly levels along x (and z) are computed once for both nodes: per slot
// 3 rows instead of 4 are loaded and reduced.
template <int D>
struct Pair {
    static constexpr int NW = 1 << (D - 1);  // vertices of one y-row: bit 0 = x, bit 1 = z
};

__device__ __forceinline__ int wrap_index(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// Returns how many of the thread's two nodes lie inside the grid (0, 1 or 2).
template <int D>
__device__ __forceinline__ int tile_pair(const ShotDesc *__restrict__ shots, int n_shots, int &shot, ShotDesc &sd,
                                         int &ix, int &iy, int &iz)
{
    find_shot(shots, n_shots, shot, sd);
    int t = blockIdx.x - sd.tile_begin;
    const int tx = t % sd.tiles[0];
    t /= sd.tiles[0];
    const int ty = t % sd.tiles[1];
    iz = t / sd.tiles[1];
    ix = tx * blockDim.x + threadIdx.x;
    iy = ty * (2 * blockDim.y) + 2 * threadIdx.y;
    if (ix >= sd.n[0] || iy >= sd.n[1] || iz >= sd.n[2]) return 0;
    return iy + 1 < sd.n[1] ? 2 : 1;
}

// vertex nodes of the three y-rows iy+lo, iy+lo+1, iy+lo+2 (periodic); node A
// uses rows 0 and 1, node B rows 1 and 2
template <int D>
__device__ __forceinline__ void pair_vertices(const ShotDesc &sd, int ix, int iy, int iz, int lo,
                                              int (&vtx)[3][Pair<D>::NW])
{
    const int xs[2] = {wrap_index(ix + lo, sd.n[0]), wrap_index(ix + lo + 1, sd.n[0])};
    int zs[2] = {0, 0};
    if constexpr (D == 3) {
        zs[0] = wrap_index(iz + lo, sd.n[2]);
        zs[1] = wrap_index(iz + lo + 1, sd.n[2]);
    }
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const int y = wrap_index(iy + lo + r, sd.n[1]);
#pragma unroll
        for (int w = 0; w < Pair<D>::NW; ++w) vtx[r][w] = xs[w & 1] + sd.n[0] * (y + sd.n[1] * zs[(w >> 1) & 1]);
    }
}

// butterflies of both cells for one (component, slot): levels x (and z) per
// row, then the y level over rows (0,1) for A and (1,2) for B
template <int D, class Ld>
__device__ __forceinline__ void pair_butterfly(const Ld &ld, int comp, int slot, const int (&vtx)[3][Pair<D>::NW],
                                               double *xa, double *xb)
{
    constexpr int NW = Pair<D>::NW;
    double r[3][NW];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
#pragma unroll
        for (int w = 0; w < NW; ++w) r[k][w] = ld(comp, slot, vtx[k][w]);
        butterfly<D - 1>(r[k]);
    }
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        const int p0 = (w & 1) | ((w >> 1) << 2);  // row pattern -> cell pattern (y bit = 2)
        xa[p0] = r[0][w] + r[1][w];
        xa[p0 | 2] = r[0][w] - r[1][w];
        xb[p0] = r[1][w] + r[2][w];
        xb[p0 | 2] = r[1][w] - r[2][w];
    }
}

template <int D, int M, class CP>
__global__ void __launch_bounds__(256) k_p_half_pair(const double *__restrict__ U, double *__restrict__ P,
                                                     const ShotDesc *__restrict__ shots, int n_shots, CP cp,
                                                     unsigned *status)
{
    using S = Shape<D, M>;
    int shot, ix, iy, iz;
    ShotDesc sd;
    const int nodes = tile_pair<D>(shots, n_shots, shot, sd, ix, iy, iz);
    if (!nodes) return;
    int vtx[3][Pair<D>::NW];
    pair_vertices<D>(sd, ix, iy, iz, -1, vtx);
    const auto &coef = cp.at(shot);
    const GlobalLd ld{U + sd.u_off, sd.nnode, S::NQ};
    double oa[S::NQ], ob[S::NQ];
#pragma unroll
    for (int s = 0; s < S::NQ; ++s) oa[s] = ob[s] = 0.0;
#pragma unroll
    for (int i = 0; i < D; ++i) {
#pragma unroll
        for (int l = 0; l < S::NQ; ++l) {
            double xa[S::NV], xb[S::NV];
            pair_butterfly<D>(ld, i, l, vtx, xa, xb);
#pragma unroll
            for (int s = 0; s < S::NQ; ++s) {
                if (coef_nonzero(D, S::n, i, s, l)) {
                    const double c = coef.get(coef_index(S::NQ, i, l, s));
                    const int pat = bfly_pattern(D, S::n, i, s, l);
                    oa[s] = fma(c, xa[pat], oa[s]);
                    ob[s] = fma(c, xb[pat], ob[s]);
                }
            }
        }
    }
    double *Ps = P + sd.p_off;
    const int64_t na = ix + (int64_t)sd.n[0] * (iy + (int64_t)sd.n[1] * iz);
    bool bad = false;
#pragma unroll
    for (int s = 0; s < S::NQ; ++s) {
        const double v = Ps[(int64_t)s * sd.nnode + na] + oa[s];
        Ps[(int64_t)s * sd.nnode + na] = v;
        bad |= nonfinite(v);
    }
    if (nodes == 2) {
        const int64_t nb = na + sd.n[0];
#pragma unroll
        for (int s = 0; s < S::NQ; ++s) {
            const double v = Ps[(int64_t)s * sd.nnode + nb] + ob[s];
            Ps[(int64_t)s * sd.nnode + nb] = v;
            bad |= nonfinite(v);
        }
    }
    report_nonfinite(bad, status);
}

template <int D, int M, class CP>
__global__ void __launch_bounds__(256) k_u_half_pair(const double *__restrict__ P, double *__restrict__ U,
                                                     const ShotDesc *__restrict__ shots, int n_shots, CP cp,
                                                     unsigned *status)
{
    using S = Shape<D, M>;
    constexpr int NO = D * S::NQ;
    int shot, ix, iy, iz;
    ShotDesc sd;
    const int nodes = tile_pair<D>(shots, n_shots, shot, sd, ix, iy, iz);
    if (!nodes) return;
    int vtx[3][Pair<D>::NW];
    pair_vertices<D>(sd, ix, iy, iz, 0, vtx);
    const auto &coef = cp.at(shot);
    const GlobalLd ld{P + sd.p_off, sd.nnode, S::NQ};
    double oa[NO], ob[NO];
#pragma unroll
    for (int e = 0; e < NO; ++e) oa[e] = ob[e] = 0.0;
#pragma unroll
    for (int l = 0; l < S::NQ; ++l) {
        double xa[S::NV], xb[S::NV];
        pair_butterfly<D>(ld, 0, l, vtx, xa, xb);
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
            for (int s = 0; s < S::NQ; ++s) {
                if (coef_nonzero(D, S::n, i, s, l)) {
                    const double c = coef.get(coef_index(S::NQ, i, l, s));
                    const int pat = bfly_pattern(D, S::n, i, s, l);
                    oa[i * S::NQ + s] = fma(c, xa[pat], oa[i * S::NQ + s]);
                    ob[i * S::NQ + s] = fma(c, xb[pat], ob[i * S::NQ + s]);
                }
            }
    }
    double *Us = U + sd.u_off;
    const int64_t na = ix + (int64_t)sd.n[0] * (iy + (int64_t)sd.n[1] * iz);
    bool bad = false;
#pragma unroll
    for (int e = 0; e < NO; ++e) {
        const double v = Us[(int64_t)e * sd.nnode + na] + oa[e];
        Us[(int64_t)e * sd.nnode + na] = v;
        bad |= nonfinite(v);
    }
    if (nodes == 2) {
        const int64_t nb = na + sd.n[0];
#pragma unroll
        for (int e = 0; e < NO; ++e) {
            const double v = Us[(int64_t)e * sd.nnode + nb] + ob[e];
            Us[(int64_t)e * sd.nnode + nb] = v;
            bad |= nonfinite(v);
        }
    }
    report_nonfinite(bad, status);
}

// u-half of the small kernel one direction at a time (when dim blocks do not fit in registers)
template <int D, int M, int I, class C, class Ld>
__device__ __forceinline__ void small_u_split(const C &coef, const Ld &ld, const int *vtx, double *sU, int nn,
                                              int node, bool &bad)
{
    if constexpr (I < D) {
        using S = Shape<D, M>;
        double out[S::NQ];
#pragma unroll
        for (int s = 0; s < S::NQ; ++s) out[s] = 0.0;
        u_node<D, M, I, 1>(coef, ld, vtx, out);
#pragma unroll
        for (int s = 0; s < S::NQ; ++s) {
            const double v = sU[(I * S::NQ + s) * nn + node] + out[s];
            sU[(I * S::NQ + s) * nn + node] = v;
            bad |= nonfinite(v);
        }
        small_u_split<D, M, I + 1>(coef, ld, vtx, sU, nn, node, bad);
    }
}

// ---------------------------------------------------------------------------
// Single-CTA persistent kernel for tiny grids: the whole state lives in shared
// memory and all n_steps run in one launch (no launch or grid-barrier cost).
template <int D, int M, class C>
__global__ void __launch_bounds__(256) k_small(double *__restrict__ P, double *__restrict__ U, GridDesc g, C coef,
                                               int64_t nsteps, unsigned *status)
{
    using S = Shape<D, M>;
    extern __shared__ double smem[];
    const int nn = (int)g.nnode;
    double *sP = smem;
    double *sU = smem + (int64_t)S::NQ * nn;
    for (int e = threadIdx.x; e < S::NQ * nn; e += blockDim.x) sP[e] = P[e];
    for (int e = threadIdx.x; e < D * S::NQ * nn; e += blockDim.x) sU[e] = U[e];
    __syncthreads();
    bool bad = false;
    SharedLd ldU{sU, nn, S::NQ};
    SharedLd ldP{sP, nn, S::NQ};
    for (int64_t st = 0; st < nsteps; ++st) {
        for (int node = threadIdx.x; node < nn; node += blockDim.x) {
            int vtx[S::NV];
            vertex_nodes<D>(g, node, -1, vtx);
            double out[S::NQ];
#pragma unroll
            for (int s = 0; s < S::NQ; ++s) out[s] = 0.0;
            p_node<D, M>(coef, ldU, vtx, out);
#pragma unroll
            for (int s = 0; s < S::NQ; ++s) {
                const double v = sP[s * nn + node] + out[s];
                sP[s * nn + node] = v;
                bad |= nonfinite(v);
            }
        }
        __syncthreads();
        for (int node = threadIdx.x; node < nn; node += blockDim.x) {
            int vtx[S::NV];
            vertex_nodes<D>(g, node, 0, vtx);
            if constexpr (S::kUFused) {
                double out[D * S::NQ];
#pragma unroll
                for (int e = 0; e < D * S::NQ; ++e) out[e] = 0.0;
                u_node<D, M, 0, D>(coef, ldP, vtx, out);
#pragma unroll
                for (int e = 0; e < D * S::NQ; ++e) {
                    const double v = sU[e * nn + node] + out[e];
                    sU[e * nn + node] = v;
                    bad |= nonfinite(v);
                }
            } else {
                small_u_split<D, M, 0>(coef, ldP, vtx, sU, nn, node, bad);
            }
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < S::NQ * nn; e += blockDim.x) P[e] = sP[e];
    for (int e = threadIdx.x; e < D * S::NQ * nn; e += blockDim.x) U[e] = sU[e];
    report_nonfinite(bad, status);
}

}  // namespace hl
