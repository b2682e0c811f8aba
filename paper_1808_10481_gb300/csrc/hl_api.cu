// C ABI of the Hermite-leapfrog solver (declared in include/hl.h).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/hl.h"
#include "hl_internal.h"

using namespace hl;

struct hl_solver {
    int dim = 0, m = 0;
    int64_t n[3] = {1, 1, 1};
    double dt = 0.0;
    double lam[3] = {0.0, 0.0, 0.0};
    int64_t nnode = 0, nq = 0;
    double *p = nullptr, *u = nullptr;          // active device state, slot-major
    double *p_own = nullptr, *u_own = nullptr;  // library-owned state
    double *staging = nullptr;                  // host-layout staging, (dim+1)*nnode*nq
    unsigned *status = nullptr;                 // device status word
    unsigned *status_host = nullptr;            // pinned mirror
    double *coef_dev = nullptr;
    std::vector<double> coef;
    cudaStream_t stream = nullptr;
    int64_t steps = 0;
    bool poisoned = false;
    int precision = HL_FP64;
    int path = PATH_AUTO;
    std::string err;
    // opt-in kernel timing (HL_OPT_TIMING)
    bool timing = false;
    std::vector<cudaEvent_t> ev_pool;
    struct Pending { size_t first; int64_t nsteps; bool small; };
    std::vector<Pending> pending;
    size_t ev_used = 0;
    double t_p_ms = 0.0, t_u_ms = 0.0, t_small_ms = 0.0;
    int64_t n_p = 0, n_u = 0, n_small = 0;
    // point source
    SourceDesc src;
    int *src_nodes = nullptr;
    double *src_table = nullptr;
};

static thread_local std::string g_create_error;

static int set_err(hl_solver *h, int code, const std::string &msg)
{
    if (h)
        h->err = msg;
    else
        g_create_error = msg;
    return code;
}

static int fail_cuda(hl_solver *h, cudaError_t e, const char *what)
{
    if (h) h->poisoned = true;
    return set_err(h, HL_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define HL_CK(h, call)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return fail_cuda(h, e_, #call); \
    } while (0)

static int resolve_timing(hl_solver *h);

static int check_usable(hl_solver *h)
{
    if (!h) return set_err(nullptr, HL_EINVAL, "null handle");
    if (h->poisoned) return set_err(h, HL_ESTATE, "handle poisoned by an earlier CUDA failure: " + h->err);
    return HL_OK;
}

static void release(hl_solver *h)
{
    if (!h) return;
    for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
    if (h->src_nodes) cudaFree(h->src_nodes);
    if (h->src_table) cudaFree(h->src_table);
    if (h->p_own) cudaFree(h->p_own);
    if (h->u_own) cudaFree(h->u_own);
    if (h->staging) cudaFree(h->staging);
    if (h->status) cudaFree(h->status);
    if (h->status_host) cudaFreeHost(h->status_host);
    if (h->coef_dev) cudaFree(h->coef_dev);
    delete h;
}

extern "C" int hl_create(int dim, int m, const int64_t *n_cells, double dt, hl_solver **out)
{
    if (out) *out = nullptr;
    if (!out) return set_err(nullptr, HL_EINVAL, "out is NULL");
    if (dim < 1 || dim > 3) return set_err(nullptr, HL_EINVAL, "dim must be 1, 2 or 3");
    if (m < 0 || m > 6) return set_err(nullptr, HL_EINVAL, "m must be in 0..6");
    if (dim == 3 && m > 3) return set_err(nullptr, HL_EINVAL, "dim = 3 supports m <= 3");
    if (!n_cells) return set_err(nullptr, HL_EINVAL, "n_cells is NULL");
    int64_t nnode = 1;
    double hmin = 1.0;
    for (int k = 0; k < dim; ++k) {
        if (n_cells[k] < 2) return set_err(nullptr, HL_EINVAL, "every n_cells entry must be >= 2");
        if (n_cells[k] > (int64_t(1) << 30)) return set_err(nullptr, HL_EINVAL, "n_cells entry too large");
        nnode *= n_cells[k];
        if (nnode >= (int64_t(1) << 31)) return set_err(nullptr, HL_EINVAL, "more than 2^31-1 nodes per grid");
        hmin = std::fmin(hmin, 1.0 / (double)n_cells[k]);
    }
    if (!(dt > 0.0) || !std::isfinite(dt)) return set_err(nullptr, HL_EINVAL, "dt must be finite and > 0");
    if (!(dt < hmin)) return set_err(nullptr, HL_EINVAL, "dt must be below min h (c dt/dx < 1)");

    hl_solver *h = new hl_solver();
    h->dim = dim;
    h->m = m;
    h->dt = dt;
    h->nnode = nnode;
    h->nq = 1;
    for (int k = 0; k < dim; ++k) {
        h->n[k] = n_cells[k];
        h->lam[k] = dt * (double)n_cells[k] / 2.0;
        h->nq *= (m + 1);
    }
    if (!build_operator(dim, m, h->lam, h->coef)) {
        delete h;
        return set_err(nullptr, HL_EINVAL, "operator construction failed its structural check");
    }
    const size_t pbytes = (size_t)nnode * h->nq * sizeof(double);
    cudaError_t e;
    if ((e = cudaMalloc(&h->p_own, pbytes)) != cudaSuccess ||
        (e = cudaMalloc(&h->u_own, pbytes * dim)) != cudaSuccess ||
        (e = cudaMalloc(&h->staging, pbytes * (dim + 1))) != cudaSuccess ||
        (e = cudaMalloc(&h->status, sizeof(unsigned))) != cudaSuccess ||
        (e = cudaMallocHost(&h->status_host, sizeof(unsigned))) != cudaSuccess ||
        (e = cudaMalloc(&h->coef_dev, h->coef.size() * sizeof(double))) != cudaSuccess) {
        const int code = (e == cudaErrorMemoryAllocation) ? HL_ENOMEM : HL_ECUDA;
        std::string msg = std::string("device set-up failed: ") + cudaGetErrorString(e);
        cudaGetLastError();
        release(h);
        return set_err(nullptr, code, msg);
    }
    if ((e = cudaMemset(h->p_own, 0, pbytes)) != cudaSuccess || (e = cudaMemset(h->u_own, 0, pbytes * dim)) != cudaSuccess ||
        (e = cudaMemset(h->status, 0, sizeof(unsigned))) != cudaSuccess ||
        (e = cudaMemcpy(h->coef_dev, h->coef.data(), h->coef.size() * sizeof(double), cudaMemcpyHostToDevice)) !=
            cudaSuccess) {
        std::string msg = std::string("device set-up failed: ") + cudaGetErrorString(e);
        release(h);
        return set_err(nullptr, HL_ECUDA, msg);
    }
    h->p = h->p_own;
    h->u = h->u_own;
    *out = h;
    return HL_OK;
}

extern "C" void hl_destroy(hl_solver *h)
{
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    else cudaDeviceSynchronize();
    release(h);
}

extern "C" const char *hl_last_error(const hl_solver *h)
{
    if (!h) return g_create_error.c_str();
    return h->err.c_str();
}

extern "C" int hl_set_stream(hl_solver *h, void *cuda_stream)
{
    int rc = check_usable(h);
    if (rc) return rc;
    HL_CK(h, cudaStreamSynchronize(h->stream));
    h->stream = (cudaStream_t)cuda_stream;
    return HL_OK;
}

extern "C" int hl_set_precision(hl_solver *h, int mode)
{
    int rc = check_usable(h);
    if (rc) return rc;
    if (mode != HL_FP64) return set_err(h, HL_EINVAL, "unknown precision mode");
    h->precision = mode;
    return HL_OK;
}

extern "C" int hl_set_option(hl_solver *h, int option, int64_t value)
{
    int rc = check_usable(h);
    if (rc) return rc;
    if (option == HL_OPT_KERNEL_PATH) {
        if (value < 0 || value > 2) return set_err(h, HL_EINVAL, "kernel path must be 0, 1 or 2");
        h->path = (int)value;
        return HL_OK;
    }
    if (option == HL_OPT_TIMING) {
        if (value < 0 || value > 1) return set_err(h, HL_EINVAL, "timing must be 0 or 1");
        HL_CK(h, cudaStreamSynchronize(h->stream));
        if (h->timing) {
            int rc2 = resolve_timing(h);
            if (rc2) return rc2;
        }
        h->timing = value != 0;
        return HL_OK;
    }
    return set_err(h, HL_EINVAL, "unknown option");
}

extern "C" int hl_kernel_times(hl_solver *h, double *ms, int64_t *launches)
{
    int rc = check_usable(h);
    if (rc) return rc;
    HL_CK(h, cudaStreamSynchronize(h->stream));
    if (h->timing) {
        rc = resolve_timing(h);
        if (rc) return rc;
    }
    if (ms) {
        ms[0] = h->t_p_ms;
        ms[1] = h->t_u_ms;
        ms[2] = h->t_small_ms;
    }
    if (launches) {
        launches[0] = h->n_p;
        launches[1] = h->n_u;
        launches[2] = h->n_small;
    }
    h->t_p_ms = h->t_u_ms = h->t_small_ms = 0.0;
    h->n_p = h->n_u = h->n_small = 0;
    return HL_OK;
}

static int copy_in(hl_solver *h, const double *p, const double *u, cudaMemcpyKind kind)
{
    const size_t pb = (size_t)h->nnode * h->nq * sizeof(double);
    double *sp = h->staging, *su = h->staging + (size_t)h->nnode * h->nq;
    HL_CK(h, cudaMemcpyAsync(sp, p, pb, kind, h->stream));
    HL_CK(h, cudaMemcpyAsync(su, u, pb * h->dim, kind, h->stream));
    HL_CK(h, launch_aos_to_soa(sp, h->p, 1, h->nnode, (int)h->nq, h->stream));
    HL_CK(h, launch_aos_to_soa(su, h->u, h->dim, h->nnode, (int)h->nq, h->stream));
    HL_CK(h, cudaMemsetAsync(h->status, 0, sizeof(unsigned), h->stream));
    h->steps = 0;
    return HL_OK;
}

extern "C" int hl_set_initial(hl_solver *h, const double *p, const double *u)
{
    int rc = check_usable(h);
    if (rc) return rc;
    if (!p || !u) return set_err(h, HL_EINVAL, "p and u must be non-NULL");
    rc = copy_in(h, p, u, cudaMemcpyHostToDevice);
    if (rc) return rc;
    HL_CK(h, cudaStreamSynchronize(h->stream));
    return HL_OK;
}

extern "C" int hl_set_initial_device(hl_solver *h, const double *p_dev, const double *u_dev)
{
    int rc = check_usable(h);
    if (rc) return rc;
    if (!p_dev || !u_dev) return set_err(h, HL_EINVAL, "p_dev and u_dev must be non-NULL");
    return copy_in(h, p_dev, u_dev, cudaMemcpyDeviceToDevice);
}

// fold the durations of recorded launches into the handle's totals (stream synchronised)
static int resolve_timing(hl_solver *h)
{
    for (const auto &pd : h->pending) {
        float ms = 0.f;
        if (pd.small) {
            HL_CK(h, cudaEventElapsedTime(&ms, h->ev_pool[pd.first], h->ev_pool[pd.first + 1]));
            h->t_small_ms += ms;
            h->n_small += 1;
            continue;
        }
        for (int64_t s = 0; s < pd.nsteps; ++s) {
            HL_CK(h, cudaEventElapsedTime(&ms, h->ev_pool[pd.first + 2 * s], h->ev_pool[pd.first + 2 * s + 1]));
            h->t_p_ms += ms;
            HL_CK(h, cudaEventElapsedTime(&ms, h->ev_pool[pd.first + 2 * s + 1], h->ev_pool[pd.first + 2 * s + 2]));
            h->t_u_ms += ms;
        }
        h->n_p += pd.nsteps;
        h->n_u += pd.nsteps;
    }
    h->pending.clear();
    h->ev_used = 0;
    return HL_OK;
}

static int read_status(hl_solver *h, bool clear)
{
    HL_CK(h, cudaMemcpyAsync(h->status_host, h->status, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream));
    if (clear) HL_CK(h, cudaMemsetAsync(h->status, 0, sizeof(unsigned), h->stream));
    HL_CK(h, cudaStreamSynchronize(h->stream));
    if (h->timing) {
        int rc = resolve_timing(h);
        if (rc) return rc;
    }
    if (*h->status_host & 1u) return set_err(h, HL_ENONFINITE, "non-finite value produced by the update");
    return HL_OK;
}

extern "C" int hl_get_fields_device(hl_solver *h, double *p_dev, double *u_dev)
{
    int rc = check_usable(h);
    if (rc) return rc;
    if (p_dev) HL_CK(h, launch_soa_to_aos(h->p, p_dev, 1, h->nnode, (int)h->nq, h->stream));
    if (u_dev) HL_CK(h, launch_soa_to_aos(h->u, u_dev, h->dim, h->nnode, (int)h->nq, h->stream));
    return HL_OK;
}

extern "C" int hl_get_fields(hl_solver *h, double *p, double *u, double *t_p, double *t_u)
{
    int rc = check_usable(h);
    if (rc) return rc;
    const size_t pb = (size_t)h->nnode * h->nq * sizeof(double);
    double *sp = h->staging, *su = h->staging + (size_t)h->nnode * h->nq;
    if (p) {
        HL_CK(h, launch_soa_to_aos(h->p, sp, 1, h->nnode, (int)h->nq, h->stream));
        HL_CK(h, cudaMemcpyAsync(p, sp, pb, cudaMemcpyDeviceToHost, h->stream));
    }
    if (u) {
        HL_CK(h, launch_soa_to_aos(h->u, su, h->dim, h->nnode, (int)h->nq, h->stream));
        HL_CK(h, cudaMemcpyAsync(u, su, pb * h->dim, cudaMemcpyDeviceToHost, h->stream));
    }
    if (t_p) *t_p = (double)h->steps * h->dt;
    if (t_u) *t_u = ((double)h->steps + 0.5) * h->dt;
    return read_status(h, true);
}

extern "C" int hl_sync(hl_solver *h)
{
    int rc = check_usable(h);
    if (rc) return rc;
    return read_status(h, true);
}

extern "C" int hl_step(hl_solver *h, int64_t n_steps)
{
    int rc = check_usable(h);
    if (rc) return rc;
    if (n_steps < 0) return set_err(h, HL_EINVAL, "n_steps must be >= 0");
    if (n_steps == 0) return HL_OK;
    LaunchFp64 a;
    a.m = h->m;
    for (int k = 0; k < 3; ++k) a.n[k] = (int)h->n[k];
    a.nnode = h->nnode;
    a.coef_host = h->coef.data();
    a.coef_dev = h->coef_dev;
    a.P = h->p;
    a.U = h->u;
    a.nsteps = n_steps;
    a.stream = h->stream;
    a.status = h->status;
    a.path = h->path;
    a.src = h->src;
    a.step0 = h->steps;
    a.ev = nullptr;
    bool used_small = false;
    a.used_small = &used_small;
    size_t first = 0;
    if (h->timing) {
        const size_t need = h->ev_used + 2 * (size_t)n_steps + 1;
        while (h->ev_pool.size() < need) {
            cudaEvent_t e;
            HL_CK(h, cudaEventCreate(&e));
            h->ev_pool.push_back(e);
        }
        first = h->ev_used;
        a.ev = h->ev_pool.data() + first;
    }
    cudaError_t e = cudaSuccess;
    switch (h->dim) {
    case 1: e = launch_fp64_d1(a); break;
    case 2: e = launch_fp64_d2(a); break;
    case 3: e = launch_fp64_d3(a); break;
    }
    if (e != cudaSuccess) return fail_cuda(h, e, "hl_step kernel launch");
    if (h->timing) {
        h->pending.push_back({first, n_steps, used_small});
        h->ev_used = first + (used_small ? 2 : 2 * (size_t)n_steps + 1);
    }
    h->steps += n_steps;
    return HL_OK;
}

extern "C" int hl_set_source(hl_solver *h, const double *x0, double sigma, double f0, double amp)
{
    int rc = check_usable(h);
    if (rc) return rc;
    if (amp == 0.0) {
        HL_CK(h, cudaStreamSynchronize(h->stream));
        if (h->src_nodes) cudaFree(h->src_nodes);
        if (h->src_table) cudaFree(h->src_table);
        h->src_nodes = nullptr;
        h->src_table = nullptr;
        h->src = SourceDesc();
        return HL_OK;
    }
    if (!x0) return set_err(h, HL_EINVAL, "x0 is NULL");
    for (int k = 0; k < h->dim; ++k)
        if (!std::isfinite(x0[k])) return set_err(h, HL_EINVAL, "x0 must be finite");
    if (!(sigma > 0.0) || !std::isfinite(sigma)) return set_err(h, HL_EINVAL, "sigma must be finite and > 0");
    if (!(f0 > 0.0) || !std::isfinite(f0)) return set_err(h, HL_EINVAL, "f0 must be finite and > 0");
    if (!std::isfinite(amp)) return set_err(h, HL_EINVAL, "amp must be finite");
    std::vector<int> nodes;
    std::vector<double> table;
    if (!build_source_table(h->dim, h->m, h->n, x0, sigma, nodes, table))
        return set_err(h, HL_EINVAL, "source box too large");
    HL_CK(h, cudaStreamSynchronize(h->stream));
    if (h->src_nodes) cudaFree(h->src_nodes);
    if (h->src_table) cudaFree(h->src_table);
    h->src_nodes = nullptr;
    h->src_table = nullptr;
    h->src = SourceDesc();
    HL_CK(h, cudaMalloc(&h->src_nodes, nodes.size() * sizeof(int)));
    HL_CK(h, cudaMalloc(&h->src_table, table.size() * sizeof(double)));
    HL_CK(h, cudaMemcpy(h->src_nodes, nodes.data(), nodes.size() * sizeof(int), cudaMemcpyHostToDevice));
    HL_CK(h, cudaMemcpy(h->src_table, table.data(), table.size() * sizeof(double), cudaMemcpyHostToDevice));
    h->src.active = true;
    h->src.nb = (int)nodes.size();
    h->src.nodes = h->src_nodes;
    h->src.table = h->src_table;
    h->src.dt = h->dt;
    h->src.amp = amp;
    h->src.f0 = f0;
    return HL_OK;
}

extern "C" int hl_bind_device(hl_solver *h, double *p_dev, double *u_dev)
{
    int rc = check_usable(h);
    if (rc) return rc;
    if (!p_dev && !u_dev) {
        HL_CK(h, cudaStreamSynchronize(h->stream));
        const size_t pb = (size_t)h->nnode * h->nq * sizeof(double);
        HL_CK(h, cudaMemset(h->p_own, 0, pb));
        HL_CK(h, cudaMemset(h->u_own, 0, pb * h->dim));
        h->p = h->p_own;
        h->u = h->u_own;
        return HL_OK;
    }
    if (!p_dev || !u_dev) return set_err(h, HL_EINVAL, "bind both buffers or neither");
    if (((uintptr_t)p_dev | (uintptr_t)u_dev) & 15u) return set_err(h, HL_EINVAL, "device buffers must be 16-byte aligned");
    h->p = p_dev;
    h->u = u_dev;
    return HL_OK;
}

extern "C" int hl_info(const hl_solver *h, int64_t *nnode, int64_t *nq, int64_t *steps)
{
    if (!h) return set_err(nullptr, HL_EINVAL, "null handle");
    if (nnode) *nnode = h->nnode;
    if (nq) *nq = h->nq;
    if (steps) *steps = h->steps;
    return HL_OK;
}

extern "C" int hl_op_counts(int dim, int m, double *fma_per_node_step, double *add_per_node_step)
{
    if (dim < 1 || dim > 3 || m < 0 || m > 6) return set_err(nullptr, HL_EINVAL, "dim/m out of range");
    double f = 0, a = 0;
    fp64_op_counts(dim, m, &f, &a);
    if (fma_per_node_step) *fma_per_node_step = f;
    if (add_per_node_step) *add_per_node_step = a;
    return HL_OK;
}

// ---------------------------------------------------------------------------
// layout copies: [comp][node][q] <-> [comp][q][node] through a 32x33 tile
namespace hl {

__global__ void k_aos_to_soa(const double *__restrict__ src, double *__restrict__ dst, int64_t nnode, int nq)
{
    __shared__ double tile[32][33];
    const int comp = blockIdx.z;
    const int64_t n0 = (int64_t)blockIdx.x * 32;
    const int q0 = blockIdx.y * 32;
    const double *s = src + (int64_t)comp * nnode * nq;
    double *d = dst + (int64_t)comp * nnode * nq;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int64_t node = n0 + r;
        const int q = q0 + threadIdx.x;
        if (node < nnode && q < nq) tile[r][threadIdx.x] = s[node * nq + q];
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int q = q0 + r;
        const int64_t node = n0 + threadIdx.x;
        if (node < nnode && q < nq) d[(int64_t)q * nnode + node] = tile[threadIdx.x][r];
    }
}

__global__ void k_soa_to_aos(const double *__restrict__ src, double *__restrict__ dst, int64_t nnode, int nq)
{
    __shared__ double tile[32][33];
    const int comp = blockIdx.z;
    const int64_t n0 = (int64_t)blockIdx.x * 32;
    const int q0 = blockIdx.y * 32;
    const double *s = src + (int64_t)comp * nnode * nq;
    double *d = dst + (int64_t)comp * nnode * nq;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int q = q0 + r;
        const int64_t node = n0 + threadIdx.x;
        if (node < nnode && q < nq) tile[threadIdx.x][r] = s[(int64_t)q * nnode + node];
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int64_t node = n0 + r;
        const int q = q0 + threadIdx.x;
        if (node < nnode && q < nq) d[node * nq + q] = tile[r][threadIdx.x];
    }
}

cudaError_t launch_aos_to_soa(const double *src, double *dst, int ncomp, int64_t nnode, int nq, cudaStream_t st)
{
    dim3 grid((unsigned)((nnode + 31) / 32), (unsigned)((nq + 31) / 32), (unsigned)ncomp);
    k_aos_to_soa<<<grid, dim3(32, 8), 0, st>>>(src, dst, nnode, nq);
    return cudaGetLastError();
}

cudaError_t launch_soa_to_aos(const double *src, double *dst, int ncomp, int64_t nnode, int nq, cudaStream_t st)
{
    dim3 grid((unsigned)((nnode + 31) / 32), (unsigned)((nq + 31) / 32), (unsigned)ncomp);
    k_soa_to_aos<<<grid, dim3(32, 8), 0, st>>>(src, dst, nnode, nq);
    return cudaGetLastError();
}

}  // namespace hl
