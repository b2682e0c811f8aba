// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace hl {

constexpr int kMaxShots = 256;  // shots per batched handle

bool hermite_inverse_1d(int m, std::vector<double> &H);
bool build_operator(int D, int m, const double lam[3], std::vector<double> &coef);
void fp64_op_counts(int D, int m, double *fma_per_node_step, double *add_per_node_step);

// One grid of a launch (a single solve is a batch of one).
struct ShotDesc {
    int n[3];          // nodes per axis (1 for unused axes)
    int tiles[3];      // tiles per axis: ceil(n0/TX), ceil(n1/TY), n2
    int64_t nnode;     // n0*n1*n2
    int64_t p_off;     // element offset of the shot's p block [q][node]
    int64_t u_off;     // element offset of the shot's u block [comp][q][node]
    int tile_begin;    // first tile of the shot in the launch
    int pad;
};

// Per-step source weights dt_s * amp_s * R((n + 1/2) dt_s) of every shot.
struct SourceWeights {
    double w[kMaxShots];
};

// Point sources of the p-half (see hl_source.cu): one Gaussian box per shot.
struct SourceDesc {
    bool active = false;
    int n_entries = 0;              // box nodes over all shots
    const int *node = nullptr;      // device: shot-local node index of each entry
    const int *shot = nullptr;      // device: shot of each entry
    const double *table = nullptr;  // device: [entry][q] scaled Gaussian data
    std::vector<double> dt, amp, f0;  // host, per shot (amp = 0: no source)
};
double ricker(double t, double f0);
bool build_source_table(int dim, int m, const int64_t *n, const double *x0, double sigma,
                        std::vector<int> &nodes, std::vector<double> &table);
// Ph/Pl (may be NULL): binary32 shadows of P refreshed at the updated nodes
cudaError_t launch_source(const SourceDesc &s, const ShotDesc *shots_dev, double *P, int nq, int64_t step,
                          cudaStream_t st, float *Ph = nullptr, float *Pl = nullptr);

enum KernelPath { PATH_AUTO = 0, PATH_SMALL = 1, PATH_GRID = 2 };

// Arguments of one FP64 stepping call (n_steps full steps).
struct LaunchFp64 {
    int m;
    int n[3];                 // shape of shot 0 (the single-CTA path needs one shot)
    int64_t nnode;
    const double *coef_host;  // single dense (i, l, s) table, D*NQ*NQ doubles
    const double *coef_dev;   // device table(s): one, or n_shots back to back
    bool per_shot_coef;       // use coef_dev + shot*NCOEF
    const ShotDesc *shots;    // device shot table
    int n_shots;
    int total_tiles;
    int tx, ty;               // tile shape (nodes per tile along x, y)
    int pair = 0;             // FP64 kernels with two nodes per thread along y: bit 0 p-half, bit 1 u-half
    double *P;                // p blocks [q][node] of every shot
    double *U;                // u blocks [comp][q][node] of every shot
    int64_t nsteps;
    cudaStream_t stream;
    unsigned *status;         // device status word (bit 0: non-finite)
    int path;                 // KernelPath
    // optional timing: 2*nsteps+1 events recorded before each p-half, before
    // each u-half and after the last u-half (NULL = no timing); for the
    // single-CTA path only ev[0] and ev[1] bracket the whole launch
    cudaEvent_t *ev;
    bool *used_small;         // set to whether the single-CTA path ran
    const SourceDesc *src;    // point sources injected after every p-half (may be NULL)
    int64_t step0;            // index of the first step (source time)
    int precision;            // HL_FP64 (0), HL_FP32 (1), HL_FP32_COMP (2), HL_TC_SPLIT (3)
    // binary32 shadows of P and U for the mixed modes (lo for HL_FP32_COMP and HL_TC_SPLIT)
    float *Ph, *Pl, *Uh, *Ul;
    int64_t p_elems;          // elements of P over all shots (U has dim times more)
    // HL_TC_SPLIT: operator images of both halves (build_tc5_images), their column
    // exponents (kTcOps x kTcN), and the mode's own tile table (128-node tiles)
    const uint16_t *tc_digits = nullptr;
    const int *tc_expo = nullptr;
    const ShotDesc *tc_shots = nullptr;
    int tc_tiles = 0;
    // 3D: digit planes of the partner fields (hl_tc3.cu) and their exponent words
    uint4 *tc3_gu = nullptr, *tc3_gp = nullptr;
    int *tc3_emax = nullptr;
    // variable wave speed (dim = 1, one grid): device tables [i][node] of the scaled
    // Taylor coefficients of c^2 at the primal and dual nodes, i = 0..2m+1; dt/(2h)
    const double *c2_primal = nullptr;
    const double *c2_dual = nullptr;
    double var_lam = 0.0;
    // split two-kernel ablation (HL_OPT_SPLIT): interpolant buffer [comp][coef][node] and
    // the evolution's term lists (build_split_terms), device
    double *split_coef = nullptr;
    const int *split_beg = nullptr, *split_idx = nullptr;
    const double *split_w = nullptr;
};

// Tensor-core split mode (HL_TC_SPLIT, dim = 2, m <= 3).  Each operator is the
// vertex form of the fused half-step operator, B[k][n] with k = (partner
// component, vertex, slot) padded to 16 slots and n = output slot (16); every
// column n is scaled by 2^-e_n and cut into kTcDigits balanced base-256
// digits (signed integers in [-128, 127], exact in BF16).  Operators: 0 the
// p-half (K = 128), 1 + i the u-half's component i (K = 64).
constexpr int kTcDigits = 6;                  // digits per operand (46 bits)
constexpr int kTcOps = 3;
constexpr int kTcN = 16;                      // output columns per operator
constexpr int kTcKS = 136;                    // row stride (bf16) of a digit row: 128 + 8 padding
constexpr int kTcOpElems = kTcDigits * kTcN * kTcKS;
bool build_tc_tables(int m, const double *coef, std::vector<uint16_t> &digits, std::vector<int> &expo);
// The tcgen05 kernels' shared-memory operator images of both halves (2 x 14336
// BF16), rearranged from build_tc_tables' digits (see hl_tc5.cuh).
constexpr int kTc5ImageElems = 2 * 14336;
bool build_tc5_images(int m, const double *coef, std::vector<uint16_t> &image, std::vector<int> &expo);
constexpr int kTc5TileX = 128;  // nodes per tile of the tcgen05 kernels
// 3D (m = 2) operator images (hl_tc3.cu): per half 12 units of 4 x 2 x 224 x 8 FP16
constexpr int kTc3UnitElems = 4 * 2 * 224 * 8;
constexpr int kTc3ImageElems = 2 * 12 * kTc3UnitElems;
bool build_tc3_images(int m, const double *coef, std::vector<uint16_t> &image, std::vector<int> &expo);

cudaError_t launch_fp64_d1(const LaunchFp64 &a);
cudaError_t launch_fp64_d2(const LaunchFp64 &a);
cudaError_t launch_fp64_d3(const LaunchFp64 &a);
cudaError_t launch_mixed_d1(const LaunchFp64 &a);  // precision 1 or 2, m <= 3
cudaError_t launch_mixed_d2(const LaunchFp64 &a);
cudaError_t launch_mixed_d3(const LaunchFp64 &a);
cudaError_t launch_tc_d2(const LaunchFp64 &a);     // precision HL_TC_SPLIT, m <= 3
cudaError_t launch_tc_d3(const LaunchFp64 &a);     // precision HL_TC_SPLIT, m = 2, one shot
cudaError_t launch_tc2_planes(const LaunchFp64 &a);  // HL_TC_SPLIT, dim = 2, one shot, digit planes
// elements (uint4) of a field's digit planes (hl_tc_planes.cuh)
inline size_t tc_plane_elems(int ncomp, int CH, int n0, int n1, int n2)
{
    return (size_t)ncomp * 6 * CH * (size_t)n1 * n2 * (size_t)(n0 + 2) + 256;
}
cudaError_t launch_var_d1(const LaunchFp64 &a);    // variable wave speed, dim = 1, FP64
cudaError_t launch_split(int dim, const LaunchFp64 &a);  // split two-kernel FP64 ablation, m <= 3
// ghost planes of the walled axes (kinds: 0 periodic, 1 dirichlet, 2 neumann), in axis order
cudaError_t launch_fill_ghosts(double *U, double *P, const int *n, int dim, int m, const int *kinds, cudaStream_t st);
bool build_split_terms(int D, int m, const double lam[3], std::vector<int> &beg, std::vector<int> &idx,
                       std::vector<double> &w);

// message returned by hl_last_error(NULL) for calls that have no handle
void set_handleless_error(const char *msg);

// host-layout <-> device-layout copies, ncomp blocks of [nnode][nq] <-> [nq][nnode]
cudaError_t launch_aos_to_soa(const double *src, double *dst, int ncomp, int64_t nnode, int nq, cudaStream_t st);
cudaError_t launch_soa_to_aos(const double *src, double *dst, int ncomp, int64_t nnode, int nq, cudaStream_t st);

}  // namespace hl
