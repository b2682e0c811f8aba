// C ABI of the Hermite-leapfrog solver (declared in include/hl.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/hl.h"
#include "hl_internal.h"
#include "hl_solver.h"

using namespace hl;

static thread_local std::string g_create_error;

void hl::set_handleless_error(const char *msg) { g_create_error = msg; }

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

#define HL_CK(h, call)                                          \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return fail_cuda(h, e_, #call);  \
    } while (0)

static int resolve_timing(hl_solver *h);

static int check_usable(hl_solver *h)
{
    if (!h) return set_err(nullptr, HL_EINVAL, "null handle");
    if (h->poisoned) return set_err(h, HL_ESTATE, "handle poisoned by an earlier CUDA failure: " + h->err);
    return HL_OK;
}

static void free_source(hl_solver *h)
{
    if (h->src_node) cudaFree(h->src_node);
    if (h->src_shot) cudaFree(h->src_shot);
    if (h->src_table) cudaFree(h->src_table);
    h->src_node = h->src_shot = nullptr;
    h->src_table = nullptr;
    h->src = SourceDesc();
}

static void release(hl_solver *h)
{
    if (!h) return;
    for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
    free_source(h);
    if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    if (h->p_own) cudaFree(h->p_own);
    if (h->u_own) cudaFree(h->u_own);
    if (h->staging) cudaFree(h->staging);
    if (h->status) cudaFree(h->status);
    if (h->status_host) cudaFreeHost(h->status_host);
    if (h->coef_dev) cudaFree(h->coef_dev);
    if (h->shot_desc_dev) cudaFree(h->shot_desc_dev);
    if (h->Ph) cudaFree(h->Ph);
    if (h->Pl) cudaFree(h->Pl);
    if (h->Uh) cudaFree(h->Uh);
    if (h->Ul) cudaFree(h->Ul);
    if (h->tc_digits) cudaFree(h->tc_digits);
    if (h->tc_expo) cudaFree(h->tc_expo);
    if (h->tc_shots) cudaFree(h->tc_shots);
    if (h->tc3_gu) cudaFree(h->tc3_gu);
    if (h->tc3_gp) cudaFree(h->tc3_gp);
    if (h->tc3_emax) cudaFree(h->tc3_emax);
    if (h->c2_primal) cudaFree(h->c2_primal);
    if (h->c2_dual) cudaFree(h->c2_dual);
    if (h->split_coef) cudaFree(h->split_coef);
    if (h->split_beg) cudaFree(h->split_beg);
    if (h->split_idx) cudaFree(h->split_idx);
    if (h->split_w) cudaFree(h->split_w);
    if (h->corr_snap) cudaFree(h->corr_snap);
    if (h->corr_sums) cudaFree(h->corr_sums);
    if (h->corr_counts) cudaFree(h->corr_counts);
    delete h;
}

// (re)build the device shot table for tile shape `tile`
static int build_tiles(hl_solver *h, int tile)
{
    int tx = kTiles[tile][0], ty = kTiles[tile][1];
    if (h->dim == 1) {  // one row of nodes: fold the tile into x
        tx *= ty;
        ty = 1;
    }
    std::vector<ShotDesc> sd(h->shots.size());
    int64_t tiles = 0;
    for (size_t s = 0; s < h->shots.size(); ++s) {
        const Shot &sh = h->shots[s];
        ShotDesc &d = sd[s];
        for (int k = 0; k < 3; ++k) d.n[k] = (int)sh.n[k];
        d.tiles[0] = (int)((sh.n[0] + tx - 1) / tx);
        d.tiles[1] = (int)((sh.n[1] + ty - 1) / ty);
        d.tiles[2] = (int)sh.n[2];
        d.nnode = sh.nnode;
        d.p_off = sh.p_off;
        d.u_off = sh.u_off;
        d.tile_begin = (int)tiles;
        d.pad = 0;
        tiles += (int64_t)d.tiles[0] * d.tiles[1] * d.tiles[2];
        if (tiles >= (int64_t(1) << 31)) return set_err(h, HL_EINVAL, "too many tiles for one launch");
    }
    if (!h->shot_desc_dev) HL_CK(h, cudaMalloc(&h->shot_desc_dev, sd.size() * sizeof(ShotDesc)));
    HL_CK(h, cudaStreamSynchronize(h->stream));
    HL_CK(h, cudaMemcpy(h->shot_desc_dev, sd.data(), sd.size() * sizeof(ShotDesc), cudaMemcpyHostToDevice));
    h->shot_desc = sd;
    h->total_tiles = (int)tiles;
    h->tile = tile;
    return HL_OK;
}

// inv_h: per-shot node spacings as 1/h_k (NULL: the unit box, h_k = 1/n_cells[k])
static int create_common(int dim, int m, int n_shots, const int64_t *n_cells, const double *inv_h, const double *dt,
                         hl_solver **out)
{
    if (out) *out = nullptr;
    if (!out) return set_err(nullptr, HL_EINVAL, "out is NULL");
    if (dim < 1 || dim > 3) return set_err(nullptr, HL_EINVAL, "dim must be 1, 2 or 3");
    if (m < 0 || m > 6) return set_err(nullptr, HL_EINVAL, "m must be in 0..6");
    if (dim == 3 && m > 3) return set_err(nullptr, HL_EINVAL, "dim = 3 supports m <= 3");
    if (n_shots < 1 || n_shots > kMaxShots) return set_err(nullptr, HL_EINVAL, "n_shots must be in 1..256");
    if (n_shots > 1 && m > 3) return set_err(nullptr, HL_EINVAL, "batched handles support m <= 3");
    if (!n_cells || !dt) return set_err(nullptr, HL_EINVAL, "n_cells or dt is NULL");
    std::vector<Shot> shots(n_shots);
    int64_t nq = 1;
    for (int k = 0; k < dim; ++k) nq *= (m + 1);
    int64_t p_elems = 0;
    bool unit_box = true;
    for (int s = 0; s < n_shots; ++s) {
        Shot &sh = shots[s];
        double hmin = HUGE_VAL;
        double inv[3] = {1.0, 1.0, 1.0};
        sh.nnode = 1;
        for (int k = 0; k < dim; ++k) {
            const int64_t nk = n_cells[(size_t)s * dim + k];
            if (nk < 2) return set_err(nullptr, HL_EINVAL, "every n_cells entry must be >= 2");
            if (nk > (int64_t(1) << 30)) return set_err(nullptr, HL_EINVAL, "n_cells entry too large");
            sh.n[k] = nk;
            sh.nnode *= nk;
            if (sh.nnode >= (int64_t(1) << 31)) return set_err(nullptr, HL_EINVAL, "more than 2^31-1 nodes per grid");
            inv[k] = inv_h ? inv_h[(size_t)s * dim + k] : (double)nk;
            if (!(inv[k] > 0.0) || !std::isfinite(inv[k])) return set_err(nullptr, HL_EINVAL, "inv_h must be finite and > 0");
            if (inv[k] != (double)nk) unit_box = false;
            hmin = std::fmin(hmin, 1.0 / inv[k]);
        }
        if (!(dt[s] > 0.0) || !std::isfinite(dt[s])) return set_err(nullptr, HL_EINVAL, "dt must be finite and > 0");
        if (!(dt[s] < hmin)) return set_err(nullptr, HL_EINVAL, "dt must be below min h (c dt/dx < 1)");
        sh.dt = dt[s];
        for (int k = 0; k < dim; ++k) sh.lam[k] = dt[s] * inv[k] / 2.0;
        sh.p_off = p_elems;
        sh.u_off = p_elems * dim;
        p_elems += sh.nnode * nq;
        if (p_elems * (dim + 1) > (int64_t(1) << 38)) return set_err(nullptr, HL_EINVAL, "state too large");
    }

    hl_solver *h = new hl_solver();
    h->dim = dim;
    h->m = m;
    h->nq = nq;
    h->shots = shots;
    h->p_elems = p_elems;
    h->u_elems = p_elems * dim;
    h->per_shot_coef = n_shots > 1;
    h->unit_box = unit_box;
    h->use_graph = n_shots > 1;
    for (int s = 0; s < n_shots; ++s) {
        std::vector<double> c;
        if (!build_operator(dim, m, shots[s].lam, c)) {
            delete h;
            return set_err(nullptr, HL_EINVAL, "operator construction failed its structural check");
        }
        h->coef.insert(h->coef.end(), c.begin(), c.end());
    }
    const size_t pb = (size_t)p_elems * sizeof(double);
    cudaError_t e;
    if ((e = cudaMalloc(&h->p_own, pb)) != cudaSuccess || (e = cudaMalloc(&h->u_own, pb * dim)) != cudaSuccess ||
        (e = cudaMalloc(&h->staging, pb * (dim + 1))) != cudaSuccess ||
        (e = cudaMalloc(&h->status, sizeof(unsigned))) != cudaSuccess ||
        (e = cudaMallocHost(&h->status_host, sizeof(unsigned))) != cudaSuccess ||
        (e = cudaMalloc(&h->coef_dev, h->coef.size() * sizeof(double))) != cudaSuccess) {
        const int code = (e == cudaErrorMemoryAllocation) ? HL_ENOMEM : HL_ECUDA;
        std::string msg = std::string("device set-up failed: ") + cudaGetErrorString(e);
        cudaGetLastError();
        release(h);
        return set_err(nullptr, code, msg);
    }
    if ((e = cudaMemset(h->p_own, 0, pb)) != cudaSuccess || (e = cudaMemset(h->u_own, 0, pb * dim)) != cudaSuccess ||
        (e = cudaMemset(h->status, 0, sizeof(unsigned))) != cudaSuccess ||
        (e = cudaMemcpy(h->coef_dev, h->coef.data(), h->coef.size() * sizeof(double), cudaMemcpyHostToDevice)) !=
            cudaSuccess ||
        (e = cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking)) != cudaSuccess) {
        std::string msg = std::string("device set-up failed: ") + cudaGetErrorString(e);
        release(h);
        return set_err(nullptr, HL_ECUDA, msg);
    }
    h->p = h->p_own;
    h->u = h->u_own;
    if (build_tiles(h, 0) != HL_OK) {
        std::string msg = h->err;
        release(h);
        return set_err(nullptr, HL_ECUDA, msg);
    }
    *out = h;
    return HL_OK;
}

extern "C" int hl_create(int dim, int m, const int64_t *n_cells, double dt, hl_solver **out)
{
    return create_common(dim, m, 1, n_cells, nullptr, &dt, out);
}

extern "C" int hl_create_spacing(int dim, int m, const int64_t *n_cells, const double *inv_h, double dt,
                                 hl_solver **out)
{
    if (!inv_h) {
        if (out) *out = nullptr;
        return set_err(nullptr, HL_EINVAL, "inv_h is NULL");
    }
    return create_common(dim, m, 1, n_cells, inv_h, &dt, out);
}

extern "C" int hl_create_batch(int dim, int m, int n_shots, const int64_t *n_cells, const double *dt, hl_solver **out)
{
    return create_common(dim, m, n_shots, n_cells, nullptr, dt, out);
}

extern "C" void hl_destroy(hl_solver *h)
{
    if (!h) return;
    if (h->stream)
        cudaStreamSynchronize(h->stream);
    else
        cudaDeviceSynchronize();
    if (h->cap_stream) cudaStreamSynchronize(h->cap_stream);
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
    if (mode != HL_FP64 && mode != HL_FP32 && mode != HL_FP32_COMP && mode != HL_TC_SPLIT)
        return set_err(h, HL_EINVAL, "unknown precision mode");
    if (mode == HL_TC_SPLIT && h->dim == 1)
        return set_err(h, HL_EINVAL, "the tensor-core split mode supports dim = 2 and 3");
    if (mode == HL_TC_SPLIT && h->dim == 3 && (h->m != 2 || h->shots.size() != 1))
        return set_err(h, HL_EINVAL, "the 3D tensor-core split mode supports m = 2 and one shot");
    if (mode != HL_FP64 && h->c2_primal)
        return set_err(h, HL_EINVAL, "a variable wave speed runs in HL_FP64 only");
    if (mode != HL_FP64 && h->split_coef)
        return set_err(h, HL_EINVAL, "the split two-kernel form runs in HL_FP64 only");
    if ((mode == HL_FP32 || mode == HL_FP32_COMP) && h->walls_active)
        return set_err(h, HL_EINVAL, "walls run in HL_FP64 or HL_TC_SPLIT");
    if (mode != HL_FP64) {
        if (h->m > 3 || (h->dim == 3 && h->m > 2))
            return set_err(h, HL_EINVAL, "mixed precision supports m <= 3 (m <= 2 in 3D)");
        // one FP32 table serves every shot: the shots' lam must agree (they do
        // when every dt is C_CFL times that shot's h)
        for (const Shot &s : h->shots)
            for (int k = 0; k < h->dim; ++k)
                if (std::fabs(s.lam[k] - h->shots[0].lam[k]) > 1e-12 * std::fabs(h->shots[0].lam[k]))
                    return set_err(h, HL_EINVAL, "mixed precision needs the same dt/h on every shot");
    }
    if (mode == HL_FP32 || mode == HL_FP32_COMP) {
        // binary32 shadows of both fields (lo parts only for the compensated mode)
        HL_CK(h, cudaStreamSynchronize(h->stream));
        const size_t n = (size_t)h->p_elems;
        if (!h->Ph) HL_CK(h, cudaMalloc(&h->Ph, n * sizeof(float)));
        if (!h->Uh) HL_CK(h, cudaMalloc(&h->Uh, n * h->dim * sizeof(float)));
        if (mode == HL_FP32_COMP) {
            if (!h->Pl) HL_CK(h, cudaMalloc(&h->Pl, n * sizeof(float)));
            if (!h->Ul) HL_CK(h, cudaMalloc(&h->Ul, n * h->dim * sizeof(float)));
        }
    }
    if (mode == HL_TC_SPLIT && h->dim == 3 && (!h->tc_digits || !h->tc3_gu)) {
        // 3D: operator images streamed per unit, digit planes of both fields
        // (with periodic ghost columns and a tail the last tile's row copies may
        // reach into), the fields' exponent words
        std::vector<uint16_t> img;
        std::vector<int> ex;
        if (!build_tc3_images(h->m, h->coef.data(), img, ex))
            return set_err(h, HL_EINVAL, "3D tensor-core tables need m = 2");
        const Shot &sh = h->shots[0];
        const size_t ngu = tc_plane_elems(3, 4, (int)sh.n[0], (int)sh.n[1], (int)sh.n[2]);
        const size_t ngp = tc_plane_elems(1, 4, (int)sh.n[0], (int)sh.n[1], (int)sh.n[2]);
        HL_CK(h, cudaStreamSynchronize(h->stream));
        if (!h->tc_digits) HL_CK(h, cudaMalloc(&h->tc_digits, img.size() * sizeof(uint16_t)));
        if (!h->tc_expo) HL_CK(h, cudaMalloc(&h->tc_expo, ex.size() * sizeof(int)));
        if (!h->tc3_emax) HL_CK(h, cudaMalloc(&h->tc3_emax, 2 * sizeof(int)));
        if (!h->tc3_gu) HL_CK(h, cudaMalloc(&h->tc3_gu, ngu * sizeof(uint4)));
        if (!h->tc3_gp) HL_CK(h, cudaMalloc(&h->tc3_gp, ngp * sizeof(uint4)));
        HL_CK(h, cudaMemset(h->tc3_gu, 0, ngu * sizeof(uint4)));
        HL_CK(h, cudaMemset(h->tc3_gp, 0, ngp * sizeof(uint4)));
        HL_CK(h, cudaMemcpy(h->tc_digits, img.data(), img.size() * sizeof(uint16_t), cudaMemcpyHostToDevice));
        HL_CK(h, cudaMemcpy(h->tc_expo, ex.data(), ex.size() * sizeof(int), cudaMemcpyHostToDevice));
        h->tc_tiles = (int)(((sh.n[0] + kTc5TileX - 1) / kTc5TileX) * sh.n[1] * sh.n[2]);
    }
    if (mode == HL_TC_SPLIT && h->dim == 2 && (!h->tc_digits || !h->tc_expo || !h->tc_shots)) {
        // the tcgen05 kernels read the binary64 state directly: operator images,
        // their column exponents and a tile table of 128-node row tiles
        std::vector<uint16_t> img;
        std::vector<int> ex;
        if (!build_tc5_images(h->m, h->coef.data(), img, ex))
            return set_err(h, HL_EINVAL, "tensor-core tables need m <= 3");
        std::vector<ShotDesc> sd(h->shots.size());
        int64_t tiles = 0;
        for (size_t s = 0; s < h->shots.size(); ++s) {
            const Shot &sh = h->shots[s];
            ShotDesc &d = sd[s];
            for (int k = 0; k < 3; ++k) d.n[k] = (int)sh.n[k];
            d.tiles[0] = (int)((sh.n[0] + kTc5TileX - 1) / kTc5TileX);
            d.tiles[1] = (int)sh.n[1];
            d.tiles[2] = 1;
            d.nnode = sh.nnode;
            d.p_off = sh.p_off;
            d.u_off = sh.u_off;
            d.tile_begin = (int)tiles;
            d.pad = 0;
            tiles += (int64_t)d.tiles[0] * d.tiles[1];
            if (tiles >= (int64_t(1) << 31)) return set_err(h, HL_EINVAL, "too many tiles for one launch");
        }
        HL_CK(h, cudaStreamSynchronize(h->stream));
        if (!h->tc_digits) HL_CK(h, cudaMalloc(&h->tc_digits, img.size() * sizeof(uint16_t)));
        if (!h->tc_expo) HL_CK(h, cudaMalloc(&h->tc_expo, ex.size() * sizeof(int)));
        if (!h->tc_shots) HL_CK(h, cudaMalloc(&h->tc_shots, sd.size() * sizeof(ShotDesc)));
        HL_CK(h, cudaMemcpy(h->tc_digits, img.data(), img.size() * sizeof(uint16_t), cudaMemcpyHostToDevice));
        HL_CK(h, cudaMemcpy(h->tc_expo, ex.data(), ex.size() * sizeof(int), cudaMemcpyHostToDevice));
        HL_CK(h, cudaMemcpy(h->tc_shots, sd.data(), sd.size() * sizeof(ShotDesc), cudaMemcpyHostToDevice));
        h->tc_tiles = (int)tiles;
        if (h->shots.size() == 1) {
            // one grid: digit planes of both fields, cut once per half-step (hl_tc2.cu)
            const Shot &s0 = h->shots[0];
            const size_t ngu = tc_plane_elems(2, 2, (int)s0.n[0], (int)s0.n[1], 1);
            const size_t ngp = tc_plane_elems(1, 2, (int)s0.n[0], (int)s0.n[1], 1);
            if (!h->tc3_emax) HL_CK(h, cudaMalloc(&h->tc3_emax, 2 * sizeof(int)));
            if (!h->tc3_gu) HL_CK(h, cudaMalloc(&h->tc3_gu, ngu * sizeof(uint4)));
            if (!h->tc3_gp) HL_CK(h, cudaMalloc(&h->tc3_gp, ngp * sizeof(uint4)));
            HL_CK(h, cudaMemset(h->tc3_gu, 0, ngu * sizeof(uint4)));
            HL_CK(h, cudaMemset(h->tc3_gp, 0, ngp * sizeof(uint4)));
        }
    }
    h->precision = mode;
    return HL_OK;
}

extern "C" int hl_set_option(hl_solver *h, int option, int64_t value)
{
    int rc = check_usable(h);
    if (rc) return rc;
    switch (option) {
    case HL_OPT_KERNEL_PATH:
        if (value < 0 || value > 2) return set_err(h, HL_EINVAL, "kernel path must be 0, 1 or 2");
        h->path = (int)value;
        return HL_OK;
    case HL_OPT_TIMING:
        if (value < 0 || value > 1) return set_err(h, HL_EINVAL, "timing must be 0 or 1");
        HL_CK(h, cudaStreamSynchronize(h->stream));
        if (h->timing) {
            rc = resolve_timing(h);
            if (rc) return rc;
        }
        h->timing = value != 0;
        return HL_OK;
    case HL_OPT_GRAPH:
        if (value < 0 || value > 1) return set_err(h, HL_EINVAL, "graph must be 0 or 1");
        h->use_graph = value != 0;
        return HL_OK;
    case HL_OPT_TILE:
        if (value < 0 || value >= kNumTiles) return set_err(h, HL_EINVAL, "tile index out of range");
        return build_tiles(h, (int)value);
    case HL_OPT_STEP:
        if (value < 0) return set_err(h, HL_EINVAL, "step counter must be >= 0");
        h->steps = value;  // read when the next hl_step is issued (source clock, field times)
        return HL_OK;
    case HL_OPT_SPLIT: {
        if (value < 0 || value > 1) return set_err(h, HL_EINVAL, "split must be 0 or 1");
        HL_CK(h, cudaStreamSynchronize(h->stream));
        if (value == 0) {
            if (h->split_coef) cudaFree(h->split_coef);
            h->split_coef = nullptr;
            return HL_OK;
        }
        if (h->shots.size() != 1 || h->m > 3 || h->precision != HL_FP64 || h->c2_primal)
            return set_err(h, HL_EINVAL, "the split form needs one grid, m <= 3, HL_FP64 and unit speed");
        std::vector<int> beg, idx;
        std::vector<double> w;
        if (!build_split_terms(h->dim, h->m, h->shots[0].lam, beg, idx, w))
            return set_err(h, HL_EINVAL, "split term lists failed");
        int64_t ad = 1;
        for (int k = 0; k < h->dim; ++k) ad *= 2 * h->m + 2;
        const size_t cbytes = (size_t)h->dim * ad * h->shots[0].nnode * sizeof(double);
        cudaError_t e = cudaSuccess;
        if (!h->split_coef) e = cudaMalloc(&h->split_coef, cbytes);
        if (e == cudaSuccess && !h->split_beg) e = cudaMalloc(&h->split_beg, beg.size() * sizeof(int));
        if (e == cudaSuccess && !h->split_idx) e = cudaMalloc(&h->split_idx, idx.size() * sizeof(int));
        if (e == cudaSuccess && !h->split_w) e = cudaMalloc(&h->split_w, w.size() * sizeof(double));
        if (e != cudaSuccess) {
            cudaGetLastError();
            if (h->split_coef) cudaFree(h->split_coef);
            h->split_coef = nullptr;
            return set_err(h, HL_ENOMEM, std::string("split buffers: ") + cudaGetErrorString(e));
        }
        HL_CK(h, cudaMemcpy(h->split_beg, beg.data(), beg.size() * sizeof(int), cudaMemcpyHostToDevice));
        HL_CK(h, cudaMemcpy(h->split_idx, idx.data(), idx.size() * sizeof(int), cudaMemcpyHostToDevice));
        HL_CK(h, cudaMemcpy(h->split_w, w.data(), w.size() * sizeof(double), cudaMemcpyHostToDevice));
        return HL_OK;
    }
    default:
        return set_err(h, HL_EINVAL, "unknown option");
    }
}

// ---------------------------------------------------------------------------
// state copies between the host layout and the slot-major device layout
static int copy_in(hl_solver *h, const double *p, const double *u, cudaMemcpyKind kind)
{
    double *sp = h->staging, *su = h->staging + h->p_elems;
    HL_CK(h, cudaMemcpyAsync(sp, p, (size_t)h->p_elems * sizeof(double), kind, h->stream));
    HL_CK(h, cudaMemcpyAsync(su, u, (size_t)h->u_elems * sizeof(double), kind, h->stream));
    for (const Shot &s : h->shots) {
        HL_CK(h, launch_aos_to_soa(sp + s.p_off, h->p + s.p_off, 1, s.nnode, (int)h->nq, h->stream));
        HL_CK(h, launch_aos_to_soa(su + s.u_off, h->u + s.u_off, h->dim, s.nnode, (int)h->nq, h->stream));
    }
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
    if (*h->status_host & 2u) {
        h->poisoned = true;
        return set_err(h, HL_ETIMEOUT, "a bounded wait on the tensor cores expired (handle poisoned)");
    }
    if (*h->status_host & 1u) return set_err(h, HL_ENONFINITE, "non-finite value produced by the update");
    return HL_OK;
}

extern "C" int hl_get_fields_device(hl_solver *h, double *p_dev, double *u_dev)
{
    int rc = check_usable(h);
    if (rc) return rc;
    for (const Shot &s : h->shots) {
        if (p_dev) HL_CK(h, launch_soa_to_aos(h->p + s.p_off, p_dev + s.p_off, 1, s.nnode, (int)h->nq, h->stream));
        if (u_dev)
            HL_CK(h, launch_soa_to_aos(h->u + s.u_off, u_dev + s.u_off, h->dim, s.nnode, (int)h->nq, h->stream));
    }
    return HL_OK;
}

extern "C" int hl_get_fields(hl_solver *h, double *p, double *u, double *t_p, double *t_u)
{
    int rc = check_usable(h);
    if (rc) return rc;
    double *sp = h->staging, *su = h->staging + h->p_elems;
    rc = hl_get_fields_device(h, p ? sp : nullptr, u ? su : nullptr);
    if (rc) return rc;
    if (p) HL_CK(h, cudaMemcpyAsync(p, sp, (size_t)h->p_elems * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    if (u) HL_CK(h, cudaMemcpyAsync(u, su, (size_t)h->u_elems * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    if (t_p) *t_p = (double)h->steps * h->shots[0].dt;
    if (t_u) *t_u = ((double)h->steps + 0.5) * h->shots[0].dt;
    return read_status(h, true);
}

extern "C" int hl_sync(hl_solver *h)
{
    int rc = check_usable(h);
    if (rc) return rc;
    return read_status(h, true);
}

// ---------------------------------------------------------------------------
static LaunchFp64 launch_args(hl_solver *h, double *P, double *U, int64_t n_steps)
{
    LaunchFp64 a;
    a.m = h->m;
    for (int k = 0; k < 3; ++k) a.n[k] = (int)h->shots[0].n[k];
    a.nnode = h->shots[0].nnode;
    a.coef_host = h->coef.data();
    a.coef_dev = h->coef_dev;
    a.per_shot_coef = h->per_shot_coef;
    a.shots = h->shot_desc_dev;
    a.n_shots = (int)h->shots.size();
    a.total_tiles = h->total_tiles;
    a.tx = h->dim == 1 ? kTiles[h->tile][0] * kTiles[h->tile][1] : kTiles[h->tile][0];
    a.ty = h->dim == 1 ? 1 : kTiles[h->tile][1];
    a.pair = h->dim == 1 ? 0 : kTiles[h->tile][2];
    a.P = P;
    a.U = U;
    a.nsteps = n_steps;
    a.stream = h->stream;
    a.status = h->status;
    a.path = h->path;
    a.ev = nullptr;
    a.used_small = nullptr;
    a.src = &h->src;
    a.step0 = h->steps;
    a.precision = h->precision;
    a.Ph = h->Ph;
    a.Pl = h->Pl;
    a.Uh = h->Uh;
    a.Ul = h->Ul;
    a.p_elems = h->p_elems;
    a.tc_digits = h->tc_digits;
    a.tc_expo = h->tc_expo;
    a.tc_shots = h->tc_shots;
    a.tc_tiles = h->tc_tiles;
    a.tc3_gu = h->tc3_gu;
    a.tc3_gp = h->tc3_gp;
    a.tc3_emax = h->tc3_emax;
    a.c2_primal = h->c2_primal;
    a.c2_dual = h->c2_dual;
    a.var_lam = h->shots[0].lam[0];
    a.split_coef = h->split_coef;
    a.split_beg = h->split_beg;
    a.split_idx = h->split_idx;
    a.split_w = h->split_w;
    return a;
}

static cudaError_t dispatch(int dim, const LaunchFp64 &a)
{
    if (a.c2_primal) return dim == 1 ? launch_var_d1(a) : cudaErrorInvalidValue;
    if (a.split_coef && a.precision == HL_FP64) return launch_split(dim, a);
    if (a.precision == HL_TC_SPLIT) {
        if (dim == 2) return a.tc3_gu ? launch_tc2_planes(a) : launch_tc_d2(a);  // one grid : a batch
        return dim == 3 ? launch_tc_d3(a) : cudaErrorInvalidValue;
    }
    if (a.precision != HL_FP64) {
        switch (dim) {
        case 1: return launch_mixed_d1(a);
        case 2: return launch_mixed_d2(a);
        case 3: return launch_mixed_d3(a);
        }
        return cudaErrorInvalidValue;
    }
    switch (dim) {
    case 1: return launch_fp64_d1(a);
    case 2: return launch_fp64_d2(a);
    case 3: return launch_fp64_d3(a);
    }
    return cudaErrorInvalidValue;
}

// The steps of one hl_step call with the learned correction applied after every
// corr_every-th step of the handle's step count (hl_set_correction): each block of
// steps runs as plain launches, p is copied before the block's last step (the
// fallback rule compares the correction with that step's change), then the
// correction runs on the same stream.  Without a correction: one dispatch.
static cudaError_t run_steps(hl_solver *h, const LaunchFp64 &a)
{
    if (h->walls_active) {
        // the ghost planes are filled before every p-half: one step per dispatch
        cudaError_t e = cudaSuccess;
        const int n[3] = {(int)h->shots[0].n[0], (int)h->shots[0].n[1], (int)h->shots[0].n[2]};
        for (int64_t st = 0; st < a.nsteps; ++st) {
            if ((e = launch_fill_ghosts(a.U, a.P, n, h->dim, h->m, h->walls, a.stream)) != cudaSuccess) return e;
            LaunchFp64 b = a;
            b.nsteps = 1;
            b.step0 = a.step0 + st;
            b.ev = a.ev ? a.ev + 2 * st : nullptr;
            if ((e = dispatch(h->dim, b)) != cudaSuccess) return e;
        }
        return e;
    }
    if (!h->corr_mlp) return dispatch(h->dim, a);
    const int64_t k = h->corr_every;
    const size_t pb = (size_t)h->p_elems * sizeof(double);
    int64_t done = 0;
    cudaError_t e = cudaSuccess;
    while (done < a.nsteps) {
        const int64_t S = a.step0 + done;                 // steps completed before this block
        const int64_t to_next = k - (S % k);              // 1..k steps to the next correction
        const int64_t chunk = std::min<int64_t>(to_next, a.nsteps - done);
        const bool corr = chunk == to_next;
        LaunchFp64 b = a;
        b.step0 = S;
        b.ev = a.ev ? a.ev + 2 * done : nullptr;
        b.nsteps = corr ? chunk - 1 : chunk;
        if (b.nsteps > 0 && (e = dispatch(h->dim, b)) != cudaSuccess) return e;
        if (corr) {
            if ((e = cudaMemcpyAsync(h->corr_snap, a.P, pb, cudaMemcpyDeviceToDevice, a.stream)) != cudaSuccess) return e;
            b.step0 = S + chunk - 1;
            b.ev = a.ev ? a.ev + 2 * (done + chunk - 1) : nullptr;
            b.nsteps = 1;
            if ((e = dispatch(h->dim, b)) != cudaSuccess) return e;
            if ((e = apply_correction_checked(h, a.stream)) != cudaSuccess) return e;
        }
        done += chunk;
    }
    return e;
}

extern "C" int hl_step(hl_solver *h, int64_t n_steps)
{
    int rc = check_usable(h);
    if (rc) return rc;
    if (n_steps < 0) return set_err(h, HL_EINVAL, "n_steps must be >= 0");
    if (n_steps == 0) return HL_OK;
    LaunchFp64 a = launch_args(h, h->p, h->u, n_steps);
    if (h->use_graph) {
        // the whole call as one CUDA graph, launched on a private stream that is
        // ordered after, and joined back into, the handle's stream
        if (h->graph_exec) {
            HL_CK(h, cudaStreamSynchronize(h->cap_stream));
            cudaGraphExecDestroy(h->graph_exec);
            h->graph_exec = nullptr;
        }
        a.stream = h->cap_stream;
        a.path = PATH_GRID;
        HL_CK(h, cudaEventRecord(h->ev_fork, h->stream));
        HL_CK(h, cudaStreamWaitEvent(h->cap_stream, h->ev_fork, 0));
        HL_CK(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
        const cudaError_t e = run_steps(h, a);
        cudaGraph_t graph = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(h->cap_stream, &graph);
        if (e != cudaSuccess || e2 != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return fail_cuda(h, e != cudaSuccess ? e : e2, "hl_step graph capture");
        }
        const cudaError_t e3 = cudaGraphInstantiate(&h->graph_exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e3 != cudaSuccess) return fail_cuda(h, e3, "cudaGraphInstantiate");
        HL_CK(h, cudaGraphLaunch(h->graph_exec, h->cap_stream));
        HL_CK(h, cudaEventRecord(h->ev_join, h->cap_stream));
        HL_CK(h, cudaStreamWaitEvent(h->stream, h->ev_join, 0));
        h->steps += n_steps;
        return HL_OK;
    }
    bool used_small = false;
    a.used_small = &used_small;
    size_t first = 0;
    if (h->timing) {
        const size_t need = h->ev_used + 2 * (size_t)n_steps + 1;
        while (h->ev_pool.size() < need) {
            cudaEvent_t ev;
            HL_CK(h, cudaEventCreate(&ev));
            h->ev_pool.push_back(ev);
        }
        first = h->ev_used;
        a.ev = h->ev_pool.data() + first;
    }
    const cudaError_t e = run_steps(h, a);
    if (e != cudaSuccess) return fail_cuda(h, e, "hl_step kernel launch");
    if (h->timing) {
        h->pending.push_back({first, n_steps, used_small});
        h->ev_used = first + (used_small ? 2 : 2 * (size_t)n_steps + 1);
    }
    h->steps += n_steps;
    return HL_OK;
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

extern "C" int hl_autotune(hl_solver *h, int64_t steps_per_trial, int *best_tile, double *ms_per_tile)
{
    int rc = check_usable(h);
    if (rc) return rc;
    if (steps_per_trial < 1) return set_err(h, HL_EINVAL, "steps_per_trial must be >= 1");
    // trials run on scratch copies of the state, so the solution is not advanced;
    // the scratch is released on every return (cudaFree waits for the trials)
    struct Scratch {
        double *sp = nullptr, *su = nullptr;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        ~Scratch()
        {
            if (e0) cudaEventDestroy(e0);
            if (e1) cudaEventDestroy(e1);
            if (sp) cudaFree(sp);
            if (su) cudaFree(su);
        }
    } scr;
    double *&sp = scr.sp, *&su = scr.su;
    cudaEvent_t &e0 = scr.e0, &e1 = scr.e1;
    const size_t pb = (size_t)h->p_elems * sizeof(double);
    HL_CK(h, cudaStreamSynchronize(h->stream));
    cudaError_t e;
    if ((e = cudaMalloc(&sp, pb)) != cudaSuccess || (e = cudaMalloc(&su, pb * h->dim)) != cudaSuccess) {
        cudaGetLastError();
        return set_err(h, HL_ENOMEM, std::string("autotune scratch: ") + cudaGetErrorString(e));
    }
    HL_CK(h, cudaEventCreate(&e0));
    HL_CK(h, cudaEventCreate(&e1));
    const int keep_tile = h->tile;
    int best = keep_tile;
    double best_ms = 1e300;
    for (int t = 0; t < kNumTiles; ++t) {
        if (ms_per_tile) ms_per_tile[t] = -1.0;
        if (h->dim == 1 && kTiles[t][1] != 1) continue;  // 1D folds tiles into x
        if (h->precision == HL_TC_SPLIT && t != 0) continue;  // its kernels use their own 128-node tiles
        rc = build_tiles(h, t);
        if (rc) break;
        HL_CK(h, cudaMemcpyAsync(sp, h->p, pb, cudaMemcpyDeviceToDevice, h->stream));
        HL_CK(h, cudaMemcpyAsync(su, h->u, pb * h->dim, cudaMemcpyDeviceToDevice, h->stream));
        LaunchFp64 a = launch_args(h, sp, su, 1);
        a.path = PATH_GRID;
        a.src = nullptr;
        HL_CK(h, dispatch(h->dim, a));  // warm-up
        a.nsteps = steps_per_trial;
        HL_CK(h, cudaEventRecord(e0, h->stream));
        HL_CK(h, dispatch(h->dim, a));
        HL_CK(h, cudaEventRecord(e1, h->stream));
        HL_CK(h, cudaEventSynchronize(e1));
        float ms = 0.f;
        HL_CK(h, cudaEventElapsedTime(&ms, e0, e1));
        if (ms_per_tile) ms_per_tile[t] = ms / steps_per_trial;
        if (ms < best_ms) {
            best_ms = ms;
            best = t;
        }
    }
    HL_CK(h, cudaMemsetAsync(h->status, 0, sizeof(unsigned), h->stream));  // trial data may be anything
    HL_CK(h, cudaStreamSynchronize(h->stream));
    if (rc) {
        build_tiles(h, keep_tile);
        return rc;
    }
    rc = build_tiles(h, best);
    if (rc) return rc;
    if (best_tile) *best_tile = best;
    return HL_OK;
}

// ---------------------------------------------------------------------------
extern "C" int hl_set_sources(hl_solver *h, const double *x0, const double *sigma, const double *f0,
                              const double *amp)
{
    int rc = check_usable(h);
    if (rc) return rc;
    if (!x0 || !sigma || !f0 || !amp) return set_err(h, HL_EINVAL, "NULL source argument");
    if (!h->unit_box) return set_err(h, HL_EINVAL, "point sources need a unit-box handle (inv_h = n_cells)");
    const int ns = (int)h->shots.size();
    for (int s = 0; s < ns; ++s) {
        if (amp[s] == 0.0) continue;
        for (int k = 0; k < h->dim; ++k)
            if (!std::isfinite(x0[(size_t)s * h->dim + k])) return set_err(h, HL_EINVAL, "x0 must be finite");
        if (!(sigma[s] > 0.0) || !std::isfinite(sigma[s])) return set_err(h, HL_EINVAL, "sigma must be finite and > 0");
        if (!(f0[s] > 0.0) || !std::isfinite(f0[s])) return set_err(h, HL_EINVAL, "f0 must be finite and > 0");
        if (!std::isfinite(amp[s])) return set_err(h, HL_EINVAL, "amp must be finite");
    }
    std::vector<int> node, shot;
    std::vector<double> table;
    for (int s = 0; s < ns; ++s) {
        if (amp[s] == 0.0) continue;
        std::vector<int> nd;
        std::vector<double> tb;
        if (!build_source_table(h->dim, h->m, h->shots[s].n, x0 + (size_t)s * h->dim, sigma[s], nd, tb))
            return set_err(h, HL_EINVAL, "source box too large");
        node.insert(node.end(), nd.begin(), nd.end());
        shot.insert(shot.end(), nd.size(), s);
        table.insert(table.end(), tb.begin(), tb.end());
        if (node.size() >= ((size_t)1 << 30)) return set_err(h, HL_EINVAL, "source boxes too large");
    }
    HL_CK(h, cudaStreamSynchronize(h->stream));
    if (h->cap_stream) HL_CK(h, cudaStreamSynchronize(h->cap_stream));
    free_source(h);
    if (node.empty()) return HL_OK;
    HL_CK(h, cudaMalloc(&h->src_node, node.size() * sizeof(int)));
    HL_CK(h, cudaMalloc(&h->src_shot, shot.size() * sizeof(int)));
    HL_CK(h, cudaMalloc(&h->src_table, table.size() * sizeof(double)));
    HL_CK(h, cudaMemcpy(h->src_node, node.data(), node.size() * sizeof(int), cudaMemcpyHostToDevice));
    HL_CK(h, cudaMemcpy(h->src_shot, shot.data(), shot.size() * sizeof(int), cudaMemcpyHostToDevice));
    HL_CK(h, cudaMemcpy(h->src_table, table.data(), table.size() * sizeof(double), cudaMemcpyHostToDevice));
    h->src.active = true;
    h->src.n_entries = (int)node.size();
    h->src.node = h->src_node;
    h->src.shot = h->src_shot;
    h->src.table = h->src_table;
    h->src.dt.resize(ns);
    h->src.amp.assign(amp, amp + ns);
    h->src.f0.assign(f0, f0 + ns);
    for (int s = 0; s < ns; ++s) h->src.dt[s] = h->shots[s].dt;
    return HL_OK;
}

extern "C" int hl_set_source(hl_solver *h, const double *x0, double sigma, double f0, double amp)
{
    int rc = check_usable(h);
    if (rc) return rc;
    if (!x0 && amp != 0.0) return set_err(h, HL_EINVAL, "x0 is NULL");
    const size_t ns = h->shots.size();
    std::vector<double> xs(ns * h->dim, 0.0), sg(ns, sigma), ff(ns, f0), aa(ns, amp);
    for (size_t s = 0; s < ns; ++s)
        for (int k = 0; k < h->dim; ++k) xs[s * h->dim + k] = x0 ? x0[k] : 0.0;
    return hl_set_sources(h, xs.data(), sg.data(), ff.data(), aa.data());
}

extern "C" int hl_set_wave_speed(hl_solver *h, const double *c2_primal, const double *c2_dual)
{
    int rc = check_usable(h);
    if (rc) return rc;
    if (!c2_primal && !c2_dual) {
        HL_CK(h, cudaStreamSynchronize(h->stream));
        if (h->c2_primal) cudaFree(h->c2_primal);
        if (h->c2_dual) cudaFree(h->c2_dual);
        h->c2_primal = h->c2_dual = nullptr;
        return HL_OK;
    }
    if (!c2_primal || !c2_dual) return set_err(h, HL_EINVAL, "give both tables or neither");
    if (h->dim != 1 || h->shots.size() != 1) return set_err(h, HL_EINVAL, "a variable wave speed needs dim = 1 and one grid");
    if (h->precision != HL_FP64) return set_err(h, HL_EINVAL, "a variable wave speed runs in HL_FP64 only");
    if (h->split_coef) return set_err(h, HL_EINVAL, "the split two-kernel form has unit speed");
    const int64_t n = h->shots[0].nnode;
    const int A = 2 * h->m + 2;
    double cmax2 = 0.0;
    std::vector<double> tp((size_t)A * n), td((size_t)A * n);  // device layout [i][node]
    for (int64_t j = 0; j < n; ++j)
        for (int i = 0; i < A; ++i) {
            const double a = c2_primal[(size_t)j * A + i], b = c2_dual[(size_t)j * A + i];
            if (!std::isfinite(a) || !std::isfinite(b)) return set_err(h, HL_EINVAL, "wave speed tables must be finite");
            if (i == 0) {
                if (!(a > 0.0) || !(b > 0.0)) return set_err(h, HL_EINVAL, "c^2 must be positive at every node");
                cmax2 = std::fmax(cmax2, std::fmax(a, b));
            }
            tp[(size_t)i * n + j] = a;
            td[(size_t)i * n + j] = b;
        }
    const double hx = 1.0 / (2.0 * h->shots[0].lam[0] / h->shots[0].dt);  // h = dt / (2 lam)
    if (!(std::sqrt(cmax2) * h->shots[0].dt < hx))
        return set_err(h, HL_EINVAL, "dt must satisfy max c * dt < h at the node values of c^2");
    HL_CK(h, cudaStreamSynchronize(h->stream));
    if (!h->c2_primal) HL_CK(h, cudaMalloc(&h->c2_primal, tp.size() * sizeof(double)));
    if (!h->c2_dual) HL_CK(h, cudaMalloc(&h->c2_dual, td.size() * sizeof(double)));
    HL_CK(h, cudaMemcpy(h->c2_primal, tp.data(), tp.size() * sizeof(double), cudaMemcpyHostToDevice));
    HL_CK(h, cudaMemcpy(h->c2_dual, td.data(), td.size() * sizeof(double), cudaMemcpyHostToDevice));
    return HL_OK;
}

extern "C" int hl_set_walls(hl_solver *h, const int *kinds)
{
    int rc = check_usable(h);
    if (rc) return rc;
    if (!kinds) {
        h->walls_active = false;
        for (int k = 0; k < 3; ++k) h->walls[k] = 0;
        return HL_OK;
    }
    if (h->shots.size() != 1) return set_err(h, HL_EINVAL, "walls need one grid");
    if (h->precision == HL_FP32 || h->precision == HL_FP32_COMP)
        return set_err(h, HL_EINVAL, "walls run in HL_FP64 or HL_TC_SPLIT (the FP32 modes keep shadows)");
    bool any = false;
    for (int k = 0; k < h->dim; ++k) {
        if (kinds[k] < HL_WALL_PERIODIC || kinds[k] > HL_WALL_NEUMANN) return set_err(h, HL_EINVAL, "unknown wall kind");
        if (kinds[k] != HL_WALL_PERIODIC && h->shots[0].n[k] < 4)
            return set_err(h, HL_EINVAL, "a walled axis needs at least 4 planes (2 cells and 2 ghosts)");
        any |= kinds[k] != HL_WALL_PERIODIC;
    }
    for (int k = 0; k < 3; ++k) h->walls[k] = k < h->dim ? kinds[k] : 0;
    h->walls_active = any;
    return HL_OK;
}

extern "C" int hl_bind_device(hl_solver *h, double *p_dev, double *u_dev)
{
    int rc = check_usable(h);
    if (rc) return rc;
    if (!p_dev && !u_dev) {
        HL_CK(h, cudaStreamSynchronize(h->stream));
        const size_t pb = (size_t)h->p_elems * sizeof(double);
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
    int64_t tot = 0;
    for (const Shot &s : h->shots) tot += s.nnode;
    if (nnode) *nnode = tot;
    if (nq) *nq = h->nq;
    if (steps) *steps = h->steps;
    return HL_OK;
}

extern "C" int hl_operator_table(int dim, int m, const double *lam, double *out)
{
    if (dim < 1 || dim > 3 || m < 0 || m > 6 || !lam || !out) return set_err(nullptr, HL_EINVAL, "bad arguments");
    double l3[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < dim; ++k) l3[k] = lam[k];
    std::vector<double> c;
    if (!build_operator(dim, m, l3, c)) return set_err(nullptr, HL_EINVAL, "operator construction failed");
    std::memcpy(out, c.data(), c.size() * sizeof(double));
    return HL_OK;
}

extern "C" int hl_tc_tables(int m, const double *lam, uint16_t *digits, int *expo)
{
    if (m < 0 || m > 3 || !lam || !digits || !expo) return set_err(nullptr, HL_EINVAL, "bad arguments");
    static_assert(HL_TC_TABLE_ELEMS == kTcOps * kTcOpElems && HL_TC_EXPO_ELEMS == kTcOps * kTcN,
                  "tensor-core table sizes and header disagree");
    const double l3[3] = {lam[0], lam[1], 0.0};
    std::vector<double> c;
    if (!build_operator(2, m, l3, c)) return set_err(nullptr, HL_EINVAL, "operator construction failed");
    std::vector<uint16_t> dig;
    std::vector<int> ex;
    if (!build_tc_tables(m, c.data(), dig, ex)) return set_err(nullptr, HL_EINVAL, "tensor-core tables need m <= 3");
    std::memcpy(digits, dig.data(), dig.size() * sizeof(uint16_t));
    std::memcpy(expo, ex.data(), ex.size() * sizeof(int));
    return HL_OK;
}

extern "C" int hl_tc_image(int dim, int m, const double *lam, uint16_t *image, int64_t image_elems, int *expo,
                           int64_t expo_elems)
{
    static_assert(HL_TC_IMAGE2_ELEMS == kTc5ImageElems && HL_TC_IMAGE3_ELEMS == kTc3ImageElems,
                  "tensor-core image sizes and header disagree");
    if (!lam || !image || !expo || !((dim == 2 && m >= 0 && m <= 3) || (dim == 3 && m == 2)))
        return set_err(nullptr, HL_EINVAL, "bad arguments (dim 2 with m <= 3, or dim 3 with m = 2)");
    const int64_t need_img = dim == 2 ? HL_TC_IMAGE2_ELEMS : HL_TC_IMAGE3_ELEMS;
    const int64_t need_ex = dim == 2 ? HL_TC_EXPO_ELEMS : HL_TC_EXPO3_ELEMS;
    if (image_elems < need_img || expo_elems < need_ex) return set_err(nullptr, HL_EINVAL, "buffers too short");
    const double l3[3] = {lam[0], lam[1], dim == 3 ? lam[2] : 0.0};
    std::vector<double> c;
    if (!build_operator(dim, m, l3, c)) return set_err(nullptr, HL_EINVAL, "operator construction failed");
    std::vector<uint16_t> img;
    std::vector<int> ex;
    const bool ok = dim == 2 ? build_tc5_images(m, c.data(), img, ex) : build_tc3_images(m, c.data(), img, ex);
    if (!ok || (int64_t)img.size() != need_img || (int64_t)ex.size() != need_ex)
        return set_err(nullptr, HL_EINVAL, "tensor-core image construction failed");
    std::memcpy(image, img.data(), img.size() * sizeof(uint16_t));
    std::memcpy(expo, ex.data(), ex.size() * sizeof(int));
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
