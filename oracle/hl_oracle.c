/*
 * Plain FP64 CPU oracle for the Hermite-leapfrog method
 * (Vargas, Hagstrom, Chan, Warburton, "Leapfrog time-stepping for Hermite
 * methods", arXiv 1808.10481).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark load this library.  It shares no code,
 * header, table or constant with the CUDA library: the only operator input it
 * takes is the exact-rational matrix H = [C^L; C^R]^{-1} computed by the
 * oracle's own Python module (hermite.py).
 *
 * Problem (the paper's acoustics system with v = -u, unit wave speed):
 *     p_t + div u = 0,   u_t + grad p = 0   on the periodic unit box.
 * Primal node j (per axis) sits at j*h and holds p; dual node j sits at
 * (j + 1/2)*h and holds every velocity component (Section 2, eqs. pGrid and
 * dGrid; Section 5 for the tensor-product grids).  Node data are scaled
 * derivatives  f~_a = prod_k h_k^{a_k}/a_k! d^a f,  a_k = 0..m  (Section 2;
 * Section 5 for the tensor form).  p is known at t, u at t + dt/2
 * (Section 2, the staggered initial data).
 *
 * Layout (identical to the public host layout of the C-ABI):
 *     f[comp][node][q],  node = ix + nx*(iy + ny*iz),
 *     q = a_0 + (m+1)*(a_1 + (m+1)*a_2).
 *
 * One half-step updates every target node independently:
 *   1. gather the partner field at the 2^d cell vertices;
 *   2. build the tensor-product Hermite-Birkhoff interpolant of degree 2m+1
 *      per axis by applying H along one axis at a time (Section 2, eq. interp;
 *      Section 5, the dimension-by-dimension reconstruction);
 *   3. evaluate, term by term, the odd-order temporal Taylor series whose time
 *      derivatives are exchanged for space derivatives by the
 *      Cauchy-Kowalevsky relations (Section 2, eqs. update1, LFloop, final1;
 *      Section 3.1.2, eqs. pdup and vdup):
 *        p(t+dt) - p(t) = -sum_{k>=0} 2 (dt/2)^{2k+1}/(2k+1)! Lap^k div u(t+dt/2)
 *        u(t+dt/2) - u(t-dt/2) = -sum_{k>=0} 2 (dt/2)^{2k+1}/(2k+1)! grad Lap^k p(t)
 *      with Lap^k = sum_{|beta|=k} k!/beta! d^{2 beta}; the series is summed
 *      until every derivative index exceeds the interpolant degree 2m+1;
 *   4. add the increment to the node's own data (leapfrog).
 * A full step is the p-half over all primal nodes followed by the u-half over
 * all dual nodes (Section 2; Section 6 counts an iteration as both).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* The source is precision-generic.  The default build (C) uses IEEE
 * binary64, the paper's precision (Section 6).  Built as C++ with -DORC_DD it
 * uses double-double arithmetic (dd.hpp, about 106 significant bits): the same
 * steps with a far smaller rounding error, used as the reference for long runs against a
 * 1e-12 bar that lies below the binary64 build's own accumulated rounding. */
#ifdef ORC_DD
#include "dd.hpp"
typedef orc_dd orc_real;
#define ORC_POW orc_dd_pow
#define ORC_EXP orc_dd_exp
#define ORC_FLOOR orc_dd_floor
extern "C" {
#else
typedef double orc_real;
#define ORC_POW pow
#define ORC_EXP exp
#define ORC_FLOOR floor
#endif

#define ORC_MAXD 3
#define ORC_MAXM 6
#define ORC_MAXA (2 * ORC_MAXM + 2)

static orc_real orc_fact(int n)
{
    orc_real f = 1.0;
    for (int k = 2; k <= n; ++k) f *= (orc_real)k;
    return f;
}

static int64_t ipow(int64_t b, int e)
{
    int64_t r = 1;
    for (int i = 0; i < e; ++i) r *= b;
    return r;
}

/* Step 2: reconstruction.  vtx[v*nq + q] holds the partner's scaled data at
 * vertex v (bit k of v: 0 = lower end, 1 = upper end of axis k).  Per axis the
 * stacked data index r = bit*(m+1) + q matches the paper's [v^L; v^R].
 * coef[a], a = a_0 + A*(a_1 + A*a_2), A = 2m+2, receives the scaled Taylor
 * coefficients of the interpolant at the cell centre. */
static void orc_reconstruct(int d, int m, const orc_real *H, const orc_real *vtx, orc_real *coef)
{
    const int n = m + 1, A = 2 * m + 2;
    const int64_t nq = ipow(n, d);
    const int64_t tot = ipow(A, d);
    orc_real *x = (orc_real *)malloc(sizeof(orc_real) * (size_t)tot);
    orc_real *y = (orc_real *)malloc(sizeof(orc_real) * (size_t)tot);
    /* scatter vertex data into the stacked tensor x[r_0 + A*(r_1 + A*r_2)] */
    for (int v = 0; v < (1 << d); ++v) {
        for (int64_t q = 0; q < nq; ++q) {
            int64_t r = 0, stride = 1, qq = q;
            for (int k = 0; k < d; ++k) {
                int qk = (int)(qq % n);
                qq /= n;
                int bit = (v >> k) & 1;
                r += (int64_t)(bit * n + qk) * stride;
                stride *= A;
            }
            x[r] = vtx[(int64_t)v * nq + q];
        }
    }
    /* apply H along axis k, one axis at a time */
    for (int k = 0; k < d; ++k) {
        int64_t sk = ipow(A, k);
        for (int64_t idx = 0; idx < tot; ++idx) {
            int ak = (int)((idx / sk) % A);
            int64_t base = idx - (int64_t)ak * sk;
            orc_real acc = 0.0;
            for (int r = 0; r < A; ++r) acc += H[ak * A + r] * x[base + (int64_t)r * sk];
            y[idx] = acc;
        }
        memcpy(x, y, sizeof(orc_real) * (size_t)tot);
    }
    memcpy(coef, x, sizeof(orc_real) * (size_t)tot);
    free(x);
    free(y);
}

/* Step 3: the Cauchy-Kowalevsky series for target slot s and direction i.
 * In scaled variables the term of order j = 2k+1 with Laplacian split beta
 * (|beta| = k) contributes
 *     2/(2k+1)! * k!/beta! * prod_l [(s_l + 2 beta_l + [l==i])! / s_l!]
 *                          * lam_l^(2 beta_l + [l==i]) * coef[s + 2 beta + e_i]
 * where lam_l = dt/(2 h_l).  Returns the (positive) series value; the caller
 * subtracts it (v = -u sign convention). */
static orc_real orc_series(int d, int m, const orc_real *lam, const orc_real *coef, const int *s, int i)
{
    const int A = 2 * m + 2;
    const int kmax = d * (2 * m + 1); /* generous bound; out-of-range terms are skipped */
    orc_real total = 0.0;
    for (int k = 0; k <= kmax; ++k) {
        /* enumerate beta with |beta| = k, beta_l in 0..k */
        int beta[ORC_MAXD] = {0, 0, 0};
        int lim1 = d > 1 ? k : 0, lim2 = d > 2 ? k : 0;
        for (int b2 = 0; b2 <= lim2; ++b2) {
            for (int b1 = 0; b1 <= lim1; ++b1) {
                int b0 = k - b1 - b2;
                if (b0 < 0) continue;
                beta[0] = b0;
                beta[1] = b1;
                beta[2] = b2;
                int ok = 1;
                int64_t aidx = 0, stride = 1;
                orc_real c = 2.0 / orc_fact(2 * k + 1) * orc_fact(k);
                for (int l = 0; l < d; ++l) {
                    int a = s[l] + 2 * beta[l] + (l == i ? 1 : 0);
                    if (a > 2 * m + 1) { ok = 0; break; }
                    c *= 1.0 / orc_fact(beta[l]);
                    c *= orc_fact(a) / orc_fact(s[l]);
                    c *= ORC_POW(lam[l], (orc_real)(a - s[l]));
                    aidx += (int64_t)a * stride;
                    stride *= A;
                }
                if (!ok) continue;
                total += c * coef[aidx];
            }
        }
    }
    return total;
}

/* Steps 2-3 for one node.  mode 0 (p-half): src holds d velocity components,
 * dst one pressure block; mode 1 (u-half): src holds pressure, dst d velocity
 * blocks.  vtx[(comp*2^d + v)*nq + q]; incr[comp*nq + q] receives the
 * increment to ADD to the target's own data. */
void oracle_node_update(int d, int m, const orc_real *lam, const orc_real *H, int mode,
                        const orc_real *vtx, orc_real *incr)
{
    const int n = m + 1, A = 2 * m + 2;
    const int64_t nq = ipow(n, d);
    const int64_t nv = (int64_t)1 << d;
    const int ncs = mode == 0 ? d : 1;
    orc_real *coef = (orc_real *)malloc(sizeof(orc_real) * (size_t)(ncs * ipow(A, d)));
    for (int c = 0; c < ncs; ++c)
        orc_reconstruct(d, m, H, vtx + (int64_t)c * nv * nq, coef + (int64_t)c * ipow(A, d));
    for (int64_t q = 0; q < nq; ++q) {
        int s[ORC_MAXD] = {0, 0, 0};
        int64_t qq = q;
        for (int k = 0; k < d; ++k) { s[k] = (int)(qq % n); qq /= n; }
        if (mode == 0) {
            orc_real acc = 0.0;
            for (int i = 0; i < d; ++i) acc += orc_series(d, m, lam, coef + (int64_t)i * ipow(A, d), s, i);
            incr[q] = -acc;
        } else {
            for (int i = 0; i < d; ++i) incr[(int64_t)i * nq + q] = -orc_series(d, m, lam, coef, s, i);
        }
    }
    free(coef);
}

/* One half-step over the periodic grid.  mode 0: p-half, the primal node j
 * takes dual nodes j-1 and j as the ends of its cell on each axis; mode 1:
 * u-half, the dual node j takes primal nodes j and j+1.  src is read only,
 * dst is updated in place (each target reads only its own dst data). */
void oracle_half_step(int d, int m, const int64_t *ncell, const orc_real *lam, const orc_real *H,
                      int mode, const orc_real *src, orc_real *dst)
{
    const int n = m + 1;
    const int64_t nq = ipow(n, d);
    const int64_t nv = (int64_t)1 << d;
    int64_t N[ORC_MAXD] = {1, 1, 1};
    int64_t nnode = 1;
    for (int k = 0; k < d; ++k) { N[k] = ncell[k]; nnode *= N[k]; }
    const int ncs = mode == 0 ? d : 1;
    const int ncd = mode == 0 ? 1 : d;
    const int lo_off = mode == 0 ? -1 : 0; /* lower vertex offset on each axis */

#pragma omp parallel for schedule(static)
    for (int64_t node = 0; node < nnode; ++node) {
        int64_t j[ORC_MAXD] = {0, 0, 0};
        int64_t t = node;
        for (int k = 0; k < d; ++k) { j[k] = t % N[k]; t /= N[k]; }
        orc_real *vtx = (orc_real *)malloc(sizeof(orc_real) * (size_t)(ncs * nv * nq));
        orc_real *inc = (orc_real *)malloc(sizeof(orc_real) * (size_t)(ncd * nq));
        /* step 1: gather */
        for (int64_t v = 0; v < nv; ++v) {
            int64_t vn = 0, stride = 1;
            for (int k = 0; k < d; ++k) {
                int64_t jk = j[k] + lo_off + ((v >> k) & 1);
                jk = ((jk % N[k]) + N[k]) % N[k];
                vn += jk * stride;
                stride *= N[k];
            }
            for (int c = 0; c < ncs; ++c)
                for (int64_t q = 0; q < nq; ++q)
                    vtx[((int64_t)c * nv + v) * nq + q] = src[((int64_t)c * nnode + vn) * nq + q];
        }
        /* steps 2-3 */
        oracle_node_update(d, m, lam, H, mode, vtx, inc);
        /* step 4: leapfrog update of the node's own data */
        for (int c = 0; c < ncd; ++c)
            for (int64_t q = 0; q < nq; ++q)
                dst[((int64_t)c * nnode + node) * nq + q] += inc[(int64_t)c * nq + q];
        free(vtx);
        free(inc);
    }
}

/* The half-step of oracle_half_step evaluated only at the listed target nodes:
 * out[(c*n_sample + k)*nq + q] = dst[c][nodes[k]][q] + increment, with the
 * same gather and node update.  dst is read only.  Used to check a large run
 * at sampled nodes from its own state one half-step earlier. */
void oracle_half_step_nodes(int d, int m, const int64_t *ncell, const orc_real *lam, const orc_real *H,
                            int mode, const orc_real *src, const orc_real *dst, const int64_t *nodes,
                            int64_t n_sample, orc_real *out)
{
    const int n = m + 1;
    const int64_t nq = ipow(n, d);
    const int64_t nv = (int64_t)1 << d;
    int64_t N[ORC_MAXD] = {1, 1, 1};
    int64_t nnode = 1;
    for (int k = 0; k < d; ++k) { N[k] = ncell[k]; nnode *= N[k]; }
    const int ncs = mode == 0 ? d : 1;
    const int ncd = mode == 0 ? 1 : d;
    const int lo_off = mode == 0 ? -1 : 0;

#pragma omp parallel for schedule(static)
    for (int64_t smp = 0; smp < n_sample; ++smp) {
        const int64_t node = nodes[smp];
        int64_t j[ORC_MAXD] = {0, 0, 0};
        int64_t t = node;
        for (int k = 0; k < d; ++k) { j[k] = t % N[k]; t /= N[k]; }
        orc_real *vtx = (orc_real *)malloc(sizeof(orc_real) * (size_t)(ncs * nv * nq));
        orc_real *inc = (orc_real *)malloc(sizeof(orc_real) * (size_t)(ncd * nq));
        for (int64_t v = 0; v < nv; ++v) {
            int64_t vn = 0, stride = 1;
            for (int k = 0; k < d; ++k) {
                int64_t jk = j[k] + lo_off + ((v >> k) & 1);
                jk = ((jk % N[k]) + N[k]) % N[k];
                vn += jk * stride;
                stride *= N[k];
            }
            for (int c = 0; c < ncs; ++c)
                for (int64_t q = 0; q < nq; ++q)
                    vtx[((int64_t)c * nv + v) * nq + q] = src[((int64_t)c * nnode + vn) * nq + q];
        }
        oracle_node_update(d, m, lam, H, mode, vtx, inc);
        for (int c = 0; c < ncd; ++c)
            for (int64_t q = 0; q < nq; ++q)
                out[((int64_t)c * n_sample + smp) * nq + q] =
                    dst[((int64_t)c * nnode + node) * nq + q] + inc[(int64_t)c * nq + q];
        free(vtx);
        free(inc);
    }
}

/* n_steps full steps: p-half then u-half (p at t -> t+dt, u at t+dt/2 -> t+3dt/2). */
void oracle_run(int d, int m, const int64_t *ncell, const orc_real *lam, const orc_real *H,
                orc_real *p, orc_real *u, int64_t n_steps)
{
    for (int64_t s = 0; s < n_steps; ++s) {
        oracle_half_step(d, m, ncell, lam, H, 0, u, p);
        oracle_half_step(d, m, ncell, lam, H, 1, p, u);
    }
}

/* ------------------------------------------------------------------------
 * Point source (not in the paper; the workload's Ricker source).  The paper's
 * forced experiments add a source z(x,t) to the pressure equation (Section 4,
 * eq. waveEq1D) without stating its time discretisation; here the source
 *     f(x,t) = amp * R(t) * g(x),
 *     R(t) = (1 - 2 pi^2 f0^2 (t-t0)^2) exp(-pi^2 f0^2 (t-t0)^2),  t0 = 1.2/f0,
 *     g(x) = exp(-|x - x0|^2 / (2 sigma^2))   (nearest periodic image),
 * enters the p-half by the midpoint rule: p~_a += dt * amp * R(t_n + dt/2) * g~_a,
 * with g~_a the exact scaled derivatives prod_k h_k^{a_k}/a_k! d^{a_k} g_k. */
static orc_real orc_ricker(orc_real t, orc_real f0)
{
#ifdef ORC_DD
    const orc_real pi = orc_dd::make(3.141592653589793116, 1.224646799147353207e-16);  /* pi to 106 bits */
#else
    const orc_real pi = 3.14159265358979323846;
#endif
    const orc_real t0 = 1.2 / f0;
    const orc_real arg = pi * pi * f0 * f0 * (t - t0) * (t - t0);
    return (1.0 - 2.0 * arg) * ORC_EXP(-arg);
}

/* scaled derivatives (h^a/a!) d^a/dx^a exp(-z^2/2), z = (x - c)/sigma, a = 0..m:
 * d^a exp(-z^2/2)/dx^a = (-1/sigma)^a He_a(z) exp(-z^2/2) (probabilists' Hermite). */
static void orc_gauss_1d(orc_real dx, orc_real sigma, orc_real h, int m, orc_real *out)
{
    const orc_real z = dx / sigma;
    const orc_real g = ORC_EXP(-0.5 * z * z);
    orc_real he_prev = 1.0, he = z;
    for (int a = 0; a <= m; ++a) {
        orc_real hea = a == 0 ? 1.0 : (a == 1 ? z : 0.0);
        if (a >= 2) {
            orc_real next = z * he - (orc_real)(a - 1) * he_prev;
            he_prev = he;
            he = next;
            hea = he;
        }
        out[a] = ORC_POW(-h / sigma, (orc_real)a) / orc_fact(a) * hea * g;
    }
}

void oracle_add_source(int d, int m, const int64_t *ncell, const orc_real *x0, orc_real sigma, orc_real f0,
                       orc_real amp, orc_real t_mid, orc_real dt, orc_real *p)
{
    const int n = m + 1;
    const int64_t nq = ipow(n, d);
    int64_t N[ORC_MAXD] = {1, 1, 1};
    int64_t nnode = 1;
    for (int k = 0; k < d; ++k) { N[k] = ncell[k]; nnode *= N[k]; }
    const orc_real w = dt * amp * orc_ricker(t_mid, f0);
#pragma omp parallel for schedule(static)
    for (int64_t node = 0; node < nnode; ++node) {
        orc_real fac[ORC_MAXD][ORC_MAXM + 1];
        int64_t t = node;
        for (int k = 0; k < d; ++k) {
            const int64_t j = t % N[k];
            t /= N[k];
            const orc_real h = 1.0 / (orc_real)N[k];
            orc_real dx = (orc_real)j * h - x0[k];
            dx -= ORC_FLOOR(dx + 0.5);          /* nearest periodic image */
            orc_gauss_1d(dx, sigma, h, m, fac[k]);
        }
        for (int64_t q = 0; q < nq; ++q) {
            orc_real g = 1.0;
            int64_t qq = q;
            for (int k = 0; k < d; ++k) { g *= fac[k][qq % n]; qq /= n; }
            p[node * nq + q] += w * g;
        }
    }
}

/* n_steps steps with the point source added after each p-half. */
void oracle_run_source(int d, int m, const int64_t *ncell, const orc_real *lam, const orc_real *H, orc_real dt,
                       const orc_real *x0, orc_real sigma, orc_real f0, orc_real amp, int64_t step0,
                       orc_real *p, orc_real *u, int64_t n_steps)
{
    for (int64_t s = 0; s < n_steps; ++s) {
        oracle_half_step(d, m, ncell, lam, H, 0, u, p);
        oracle_add_source(d, m, ncell, x0, sigma, f0, amp, ((orc_real)(step0 + s) + 0.5) * dt, dt, p);
        oracle_half_step(d, m, ncell, lam, H, 1, p, u);
    }
}

void oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int oracle_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

#ifdef ORC_DD
}  /* extern "C" */
#endif
