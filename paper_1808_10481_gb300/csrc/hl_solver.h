// The solver handle (shared by the library's translation units).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/hl.h"
#include "hl_internal.h"

namespace hl {

// tile (thread block) shapes the autotuner chooses from: (TX, TY)
// {nodes per tile along x, along y, pairing}: pairing bit 0 runs the FP64
// p-half, bit 1 the u-half, with two nodes per thread along y (blocks of
// x * y/2 threads)
constexpr int kTiles[][3] = {{128, 1, 0}, {256, 1, 0}, {64, 2, 0}, {32, 4, 0}, {32, 8, 0},
                             {64, 4, 0},  {16, 8, 0},  {16, 16, 0}, {32, 4, 3}, {32, 8, 3},
                             {64, 4, 3},  {16, 16, 3}, {32, 8, 1},  {64, 4, 1}};
constexpr int kNumTiles = (int)(sizeof(kTiles) / sizeof(kTiles[0]));
static_assert(kNumTiles == HL_NUM_TILES, "tile table and header disagree");

struct Shot {
    int64_t n[3] = {1, 1, 1};
    double dt = 0.0;
    double lam[3] = {0.0, 0.0, 0.0};
    int64_t nnode = 0;
    int64_t p_off = 0;   // element offset in the slot-major p array (and host p array)
    int64_t u_off = 0;   // element offset in the slot-major u array (and host u array)
};

}  // namespace hl

struct hl_mlp;

struct hl_solver {
    int dim = 0, m = 0;
    int64_t nq = 0;
    std::vector<hl::Shot> shots;
    int64_t p_elems = 0, u_elems = 0;           // totals over shots
    double *p = nullptr, *u = nullptr;          // active device state, slot-major
    double *p_own = nullptr, *u_own = nullptr;  // library-owned state
    double *staging = nullptr;                  // host-layout staging, p_elems + u_elems
    unsigned *status = nullptr;                 // device status word
    unsigned *status_host = nullptr;            // pinned mirror
    std::vector<double> coef;                   // n_shots dense tables (shot 0 first)
    double *coef_dev = nullptr;
    bool per_shot_coef = false;
    bool unit_box = true;                       // h_k = 1/n_k on every axis (hl_create_spacing may differ)
    // tiles
    int tile = 0;
    std::vector<hl::ShotDesc> shot_desc;
    hl::ShotDesc *shot_desc_dev = nullptr;
    int total_tiles = 0;
    // streams and graph capture
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    bool use_graph = false;
    int64_t steps = 0;
    bool poisoned = false;
    int precision = HL_FP64;
    int path = hl::PATH_AUTO;
    std::string err;
    // opt-in kernel timing (HL_OPT_TIMING)
    bool timing = false;
    std::vector<cudaEvent_t> ev_pool;
    struct Pending {
        size_t first;
        int64_t nsteps;
        bool small;
    };
    std::vector<Pending> pending;
    size_t ev_used = 0;
    double t_p_ms = 0.0, t_u_ms = 0.0, t_small_ms = 0.0;
    int64_t n_p = 0, n_u = 0, n_small = 0;
    // point sources
    hl::SourceDesc src;
    float *Ph = nullptr, *Pl = nullptr, *Uh = nullptr, *Ul = nullptr;  // mixed-precision shadows
    uint16_t *tc_digits = nullptr;  // HL_TC_SPLIT operator images of both halves (build_tc5_images)
    int *tc_expo = nullptr;         // and their column exponents
    hl::ShotDesc *tc_shots = nullptr;  // HL_TC_SPLIT tile table: 128-node tiles of one grid row
    int tc_tiles = 0;
    uint4 *tc3_gu = nullptr, *tc3_gp = nullptr;  // 3D HL_TC_SPLIT: digit planes of u and p (hl_tc3.cu)
    int *tc3_emax = nullptr;                     // and the fields' exponent words
    double *c2_primal = nullptr, *c2_dual = nullptr;  // variable wave speed tables (dim = 1), [i][node]
    // split two-kernel ablation (HL_OPT_SPLIT)
    double *split_coef = nullptr;
    int *split_beg = nullptr, *split_idx = nullptr;
    double *split_w = nullptr;
    // reflecting walls (hl_set_walls): kind per axis, 0 = periodic
    int walls[3] = {0, 0, 0};
    bool walls_active = false;
    // learned correction inside hl_step (hl_set_correction)
    hl_mlp *corr_mlp = nullptr;
    int corr_every = 0;
    float corr_feat_scale = 1.f, corr_t_feature = 0.f;
    double corr_out_scale = 1.0, corr_ratio = 1.0;
    double *corr_snap = nullptr;               // p before the last plain step of a block
    double *corr_sums = nullptr;               // fallback rule: sum correction^2, sum increment^2
    unsigned long long *corr_counts = nullptr; // applied, skipped
    int *src_node = nullptr, *src_shot = nullptr;
    double *src_table = nullptr;
};


namespace hl {
// the learned correction of hl_set_correction, stream-ordered (hl_mlp.cu)
cudaError_t apply_correction_checked(hl_solver *h, cudaStream_t st);
}  // namespace hl
