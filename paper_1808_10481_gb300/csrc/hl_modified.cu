// The modified Hermite-leapfrog scheme (Section 4.3) for the 1D pressure-velocity
// system p_t + u_x = 0, u_t + p_x = 0 on the periodic unit interval: both fields
// on both grids, even derivative slots updated by the difference of the forward
// and backward temporal Taylor expansions about the midpoint (eq. hy1), odd slots
// by their sum (eq. lfw2), with the full series (every term the degree-2m+1
// interpolant supports).
//
// Fused per-node operator.  With the interpolant coefficients c_a = sum_l H[a][l]
// (lower_l) + H[a][m+1+l] (upper_l) and the reflection symmetry of the
// Hermite-Birkhoff inverse, H[a][m+1+l] = (-1)^(a+l) H[a][l], only odd a enter
// (hy1 pairs an even slot s with odd time orders k, lfw2 an odd slot with even k;
// a = s + k is odd in both), so c_a = sum_l H[a][l] x_l with the vertex
// butterfly x_l = lower_l - (-1)^l upper_l.  The new value of slot s is
//     f~_s(t + dt) = sigma_s f~_s(t) + sum_l W[s][l] x_l(g),
//     W[s][l] = 2 sum_k C(s+k, k) lam^k tau_k H[s+k][l],  lam = dt / (2h),
// sigma_s = +1 (s even) or -1 (s odd), tau_k = -1 (k odd: d_t^k p = -d_x^k u and
// d_t^k u = -d_x^k p) or +1 (k even), and g the partner field the time derivative
// exchanges into: p's even slots read u, its odd slots p; u's even slots read p,
// its odd slots u.  W is composed in double-double on the host and rounded once.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/hl.h"
#include "hl_dd_host.h"
#include "hl_fp64.cuh"
#include "hl_internal.h"

namespace hl {

constexpr int kModMaxM = 6;

struct ModCoef {
    double w[(kModMaxM + 1) * (kModMaxM + 1)];  // W[s][l]; the same for both target fields
};

static bool build_modified_operator(int m, double lam, std::vector<double> &W)
{
    std::vector<double> H;
    if (!hermite_inverse_1d(m, H)) return false;
    const int n = m + 1, A = 2 * m + 2;
    std::vector<DD> lp(A, dd(1.0));
    for (int e = 1; e < A; ++e) lp[e] = dd_mul(lp[e - 1], dd(lam));
    W.assign((size_t)n * n, 0.0);
    for (int s = 0; s <= m; ++s)
        for (int l = 0; l <= m; ++l) {
            DD acc = dd(0.0);
            for (int k = (s % 2 == 0) ? 1 : 0; s + k <= 2 * m + 1; k += 2) {
                const double tau = (k % 2) ? -1.0 : 1.0;
                DD t = dd_mul(dd_int(2 * ibinom(s + k, k)), lp[k]);
                t = dd_mul(t, dd(tau * H[(size_t)(s + k) * A + l]));  // H entries are dyadic: exact
                acc = dd_add(acc, t);
            }
            W[(size_t)s * n + l] = acc.hi + acc.lo;
        }
    return true;
}

// One half-step of one grid: (Pt, Ut) <- update from the other grid (Po, Uo).
// Node j's cell has the other grid's nodes j + off and j + off + 1 as vertices.
template <int M>
__global__ void __launch_bounds__(256) k_mod_half(const double *__restrict__ Po, const double *__restrict__ Uo,
                                                  double *__restrict__ Pt, double *__restrict__ Ut, int n, int off,
                                                  ModCoef c, unsigned *status)
{
    constexpr int NQ = M + 1;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    bool bad = false;
    if (j < n) {
        int lo = j + off;
        if (lo < 0) lo += n;
        int hi = lo + 1;
        if (hi >= n) hi -= n;
        double xp[NQ], xu[NQ];
#pragma unroll
        for (int l = 0; l < NQ; ++l) {
            const double pl = __ldg(Po + (int64_t)l * n + lo), ph = __ldg(Po + (int64_t)l * n + hi);
            const double ul = __ldg(Uo + (int64_t)l * n + lo), uh = __ldg(Uo + (int64_t)l * n + hi);
            xp[l] = (l % 2 == 0) ? pl - ph : pl + ph;
            xu[l] = (l % 2 == 0) ? ul - uh : ul + uh;
        }
#pragma unroll
        for (int s = 0; s < NQ; ++s) {
            // p: even slots read u, odd slots p; u: even slots read p, odd slots u
            const double *gp = (s % 2 == 0) ? xu : xp;
            const double *gu = (s % 2 == 0) ? xp : xu;
            double ap = 0.0, au = 0.0;
#pragma unroll
            for (int l = 0; l < NQ; ++l) {
                ap = fma(c.w[s * NQ + l], gp[l], ap);
                au = fma(c.w[s * NQ + l], gu[l], au);
            }
            double *dp = Pt + (int64_t)s * n + j;
            double *du = Ut + (int64_t)s * n + j;
            const double np = (s % 2 == 0) ? *dp + ap : ap - *dp;
            const double nu = (s % 2 == 0) ? *du + au : au - *du;
            *dp = np;
            *du = nu;
            bad |= nonfinite(np) | nonfinite(nu);
        }
    }
    report_nonfinite(bad, status);
}

template <int M>
static cudaError_t run_mod(const double *PP, const double *UP, const double *PD, const double *UD, int n,
                           const ModCoef &c, int64_t nsteps, cudaStream_t st, unsigned *status)
{
    const unsigned blocks = (unsigned)((n + 255) / 256);
    for (int64_t k = 0; k < nsteps; ++k) {
        k_mod_half<M><<<blocks, 256, 0, st>>>(PD, UD, const_cast<double *>(PP), const_cast<double *>(UP), n, -1, c,
                                             status);
        k_mod_half<M><<<blocks, 256, 0, st>>>(PP, UP, const_cast<double *>(PD), const_cast<double *>(UD), n, 0, c,
                                             status);
    }
    return cudaGetLastError();
}

}  // namespace hl

using namespace hl;

struct hl_mod {
    int m = 0;
    int64_t n = 0;
    double dt = 0.0;
    int64_t steps = 0;
    double *state = nullptr;    // 4 arrays [q][node]: p primal, u primal, p dual, u dual
    double *staging = nullptr;  // host layout copies, 4 x [node][q]
    unsigned *status = nullptr;
    unsigned *status_host = nullptr;
    cudaStream_t stream = nullptr;
    ModCoef coef;
    bool poisoned = false;
    std::string err;
};

static thread_local std::string g_mod_error;

static int mod_err(hl_mod *h, int code, const std::string &msg)
{
    if (h)
        h->err = msg;
    else
        g_mod_error = msg;
    return code;
}

static int mod_cuda(hl_mod *h, cudaError_t e, const char *what)
{
    if (h) h->poisoned = true;
    return mod_err(h, HL_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define MOD_CK(h, call)                                         \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return mod_cuda(h, e_, #call);   \
    } while (0)

static int mod_usable(hl_mod *h)
{
    if (!h) return mod_err(nullptr, HL_EINVAL, "null handle");
    if (h->poisoned) return mod_err(h, HL_ESTATE, "handle poisoned by an earlier CUDA failure: " + h->err);
    return HL_OK;
}

extern "C" void hl_mod_destroy(hl_mod *h)
{
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream); else cudaDeviceSynchronize();
    cudaFree(h->state);
    cudaFree(h->staging);
    cudaFree(h->status);
    if (h->status_host) cudaFreeHost(h->status_host);
    delete h;
}

extern "C" int hl_mod_create(int m, int64_t n_cells, double dt, hl_mod **out)
{
    if (out) *out = nullptr;
    if (!out) return mod_err(nullptr, HL_EINVAL, "out is NULL");
    if (m < 0 || m > kModMaxM) return mod_err(nullptr, HL_EINVAL, "m must be in 0..6");
    if (n_cells < 2 || n_cells >= (int64_t(1) << 31) / (m + 1)) return mod_err(nullptr, HL_EINVAL, "n_cells out of range");
    if (!(dt > 0.0) || !(dt < 1.0 / (double)n_cells)) return mod_err(nullptr, HL_EINVAL, "dt must satisfy 0 < dt < h");
    hl_mod *h = new hl_mod();
    h->m = m;
    h->n = n_cells;
    h->dt = dt;
    std::vector<double> W;
    if (!build_modified_operator(m, dt * (double)n_cells / 2.0, W)) {
        delete h;
        return mod_err(nullptr, HL_EINVAL, "operator construction failed");
    }
    std::memset(&h->coef, 0, sizeof(h->coef));
    std::memcpy(h->coef.w, W.data(), W.size() * sizeof(double));
    const size_t bytes = (size_t)4 * (m + 1) * n_cells * sizeof(double);
    cudaError_t e;
    if ((e = cudaMalloc(&h->state, bytes)) != cudaSuccess || (e = cudaMalloc(&h->staging, bytes)) != cudaSuccess ||
        (e = cudaMalloc(&h->status, sizeof(unsigned))) != cudaSuccess ||
        (e = cudaMallocHost(&h->status_host, sizeof(unsigned))) != cudaSuccess ||
        (e = cudaMemset(h->state, 0, bytes)) != cudaSuccess ||
        (e = cudaMemset(h->status, 0, sizeof(unsigned))) != cudaSuccess) {
        const int code = e == cudaErrorMemoryAllocation ? HL_ENOMEM : HL_ECUDA;
        std::string msg = std::string("device set-up failed: ") + cudaGetErrorString(e);
        cudaGetLastError();
        hl_mod_destroy(h);
        return mod_err(nullptr, code, msg);
    }
    *out = h;
    return HL_OK;
}

extern "C" const char *hl_mod_last_error(const hl_mod *h) { return h ? h->err.c_str() : g_mod_error.c_str(); }

extern "C" int hl_mod_set_stream(hl_mod *h, void *cuda_stream)
{
    int rc = mod_usable(h);
    if (rc) return rc;
    MOD_CK(h, cudaStreamSynchronize(h->stream));
    h->stream = (cudaStream_t)cuda_stream;
    return HL_OK;
}

extern "C" int hl_mod_set_initial(hl_mod *h, const double *pp, const double *up, const double *pd, const double *ud)
{
    int rc = mod_usable(h);
    if (rc) return rc;
    if (!pp || !up || !pd || !ud) return mod_err(h, HL_EINVAL, "NULL initial data");
    const int nq = h->m + 1;
    const size_t one = (size_t)nq * h->n;
    const double *src[4] = {pp, up, pd, ud};
    for (int a = 0; a < 4; ++a) {
        MOD_CK(h, cudaMemcpyAsync(h->staging + a * one, src[a], one * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        MOD_CK(h, launch_aos_to_soa(h->staging + a * one, h->state + a * one, 1, h->n, nq, h->stream));
    }
    MOD_CK(h, cudaMemsetAsync(h->status, 0, sizeof(unsigned), h->stream));
    MOD_CK(h, cudaStreamSynchronize(h->stream));
    h->steps = 0;
    return HL_OK;
}

extern "C" int hl_mod_step(hl_mod *h, int64_t n_steps)
{
    int rc = mod_usable(h);
    if (rc) return rc;
    if (n_steps < 0) return mod_err(h, HL_EINVAL, "n_steps must be >= 0");
    if (n_steps == 0) return HL_OK;
    const size_t one = (size_t)(h->m + 1) * h->n;
    const double *PP = h->state, *UP = PP + one, *PD = UP + one, *UD = PD + one;
    const int n = (int)h->n;
    cudaError_t e;
    switch (h->m) {
    case 0: e = run_mod<0>(PP, UP, PD, UD, n, h->coef, n_steps, h->stream, h->status); break;
    case 1: e = run_mod<1>(PP, UP, PD, UD, n, h->coef, n_steps, h->stream, h->status); break;
    case 2: e = run_mod<2>(PP, UP, PD, UD, n, h->coef, n_steps, h->stream, h->status); break;
    case 3: e = run_mod<3>(PP, UP, PD, UD, n, h->coef, n_steps, h->stream, h->status); break;
    case 4: e = run_mod<4>(PP, UP, PD, UD, n, h->coef, n_steps, h->stream, h->status); break;
    case 5: e = run_mod<5>(PP, UP, PD, UD, n, h->coef, n_steps, h->stream, h->status); break;
    default: e = run_mod<6>(PP, UP, PD, UD, n, h->coef, n_steps, h->stream, h->status); break;
    }
    if (e != cudaSuccess) return mod_cuda(h, e, "hl_mod_step kernel launch");
    h->steps += n_steps;
    return HL_OK;
}

extern "C" int hl_mod_get_fields(hl_mod *h, double *pp, double *up, double *pd, double *ud)
{
    int rc = mod_usable(h);
    if (rc) return rc;
    const int nq = h->m + 1;
    const size_t one = (size_t)nq * h->n;
    double *dst[4] = {pp, up, pd, ud};
    for (int a = 0; a < 4; ++a) {
        if (!dst[a]) continue;
        MOD_CK(h, launch_soa_to_aos(h->state + a * one, h->staging + a * one, 1, h->n, nq, h->stream));
        MOD_CK(h, cudaMemcpyAsync(dst[a], h->staging + a * one, one * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    }
    MOD_CK(h, cudaMemcpyAsync(h->status_host, h->status, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream));
    MOD_CK(h, cudaMemsetAsync(h->status, 0, sizeof(unsigned), h->stream));
    MOD_CK(h, cudaStreamSynchronize(h->stream));
    if (*h->status_host & 1u) return mod_err(h, HL_ENONFINITE, "non-finite value produced by the update");
    return HL_OK;
}

extern "C" int hl_mod_info(const hl_mod *h, int64_t *steps, double *t_primal, double *t_dual)
{
    if (!h) return mod_err(nullptr, HL_EINVAL, "null handle");
    if (steps) *steps = h->steps;
    if (t_primal) *t_primal = (double)h->steps * h->dt;
    if (t_dual) *t_dual = ((double)h->steps + 0.5) * h->dt;
    return HL_OK;
}
