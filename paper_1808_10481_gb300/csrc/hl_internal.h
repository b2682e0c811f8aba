// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace hl {

bool hermite_inverse_1d(int m, std::vector<double> &H);
bool build_operator(int D, int m, const double lam[3], std::vector<double> &coef);
void fp64_op_counts(int D, int m, double *fma_per_node_step, double *add_per_node_step);

// Point source of the p-half (see hl_source.cu).
struct SourceDesc {
    bool active = false;
    int nb = 0;                      // box nodes
    const int *nodes = nullptr;      // device, node index of each box node
    const double *table = nullptr;   // device, [q][box node] scaled Gaussian data
    double dt = 0.0, amp = 0.0, f0 = 1.0;
};
double ricker(double t, double f0);
bool build_source_table(int dim, int m, const int64_t *n, const double *x0, double sigma,
                        std::vector<int> &nodes, std::vector<double> &table);
cudaError_t launch_source(const SourceDesc &s, double *P, int64_t nnode, int nq, int64_t step, cudaStream_t st);

enum KernelPath { PATH_AUTO = 0, PATH_SMALL = 1, PATH_GRID = 2 };

// Arguments of one FP64 stepping call (n_steps full steps).
struct LaunchFp64 {
    int m;
    int n[3];
    int64_t nnode;
    const double *coef_host;  // dense (i, l, s) table, D*NQ*NQ doubles
    const double *coef_dev;   // the same table in device memory
    double *P;                // p[q][node]
    double *U;                // u[comp][q][node]
    int64_t nsteps;
    cudaStream_t stream;
    unsigned *status;         // device status word (bit 0: non-finite)
    int path;                 // KernelPath
    // optional timing: 2*nsteps+1 events recorded before each p-half, before
    // each u-half and after the last u-half (NULL = no timing); for the
    // single-CTA path only ev[0] and ev[1] bracket the whole launch
    cudaEvent_t *ev;
    bool *used_small;         // set to whether the single-CTA path ran
    SourceDesc src;           // point source injected after every p-half
    int64_t step0;            // index of the first step (source time)
};

cudaError_t launch_fp64_d1(const LaunchFp64 &a);
cudaError_t launch_fp64_d2(const LaunchFp64 &a);
cudaError_t launch_fp64_d3(const LaunchFp64 &a);

// host-layout <-> device-layout copies, ncomp blocks of [nnode][nq] <-> [nq][nnode]
cudaError_t launch_aos_to_soa(const double *src, double *dst, int ncomp, int64_t nnode, int nq, cudaStream_t st);
cudaError_t launch_soa_to_aos(const double *src, double *dst, int ncomp, int64_t nnode, int nq, cudaStream_t st);

}  // namespace hl
