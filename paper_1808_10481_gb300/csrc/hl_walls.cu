// Reflecting walls by ghost mirroring (Section 5.2; Section 5.3 for Maxwell's
// equations in transverse-magnetic form, this system with p = E_z and
// u = (-H_y, H_x)), filled on the device before every p-half inside hl_step.
//
// The handle steps a periodic grid whose walled axes carry N + 2 planes
// (hl_create_spacing with the true spacing): local plane 0 is an unused primal
// plane and a dual ghost, planes 1 .. N+1 hold the primal nodes 0 .. N (both
// walls), planes 1 .. N the dual nodes 0 .. N-1, plane N+1 the second dual
// ghost.  Before every step, for each walled axis k in order:
//     u ghost plane 0     = sign * u plane 1,
//     u ghost plane N + 1 = sign * u plane N,
//     p plane 0           = 0,
// with sign = s (-1)^(a_k) for the tangential components and -s (-1)^(a_k) for
// component k, a_k the derivative order along k of the slot and s = -1 for a
// "dirichlet" wall (p = 0, p odd across it) and +1 for a "neumann" wall
// (d_k p = 0, p even).  The p-half then reads the ghosts at the wall nodes; the
// u-half reads primal planes only.  Axes filled in order give edge and corner
// ghosts the product of the mirrors.
#include <cuda_runtime.h>

#include <cstdint>

#include "hl_internal.h"

namespace hl {

__global__ void k_fill_ghosts(double *__restrict__ U, double *__restrict__ P, int n0, int n1, int n2, int dim, int m,
                              int axis, int parity)
{
    const int n[3] = {n0, n1, n2};
    const int na = n[axis];
    const int64_t nnode = (int64_t)n0 * n1 * n2;
    const int64_t plane = nnode / na;
    int nq = 1;
    for (int k = 0; k < dim; ++k) nq *= (m + 1);
    int stride_q = 1;  // slot stride of axis `axis` in q
    for (int k = 0; k < axis; ++k) stride_q *= (m + 1);
    int64_t stride_n = 1;  // node stride of axis `axis`
    for (int k = 0; k < axis; ++k) stride_n *= n[k];
    const int64_t total_u = (int64_t)dim * nq * plane;
    const int64_t total = total_u + (int64_t)nq * plane;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const bool is_u = e < total_u;
        const int64_t r = is_u ? e : e - total_u;
        const int64_t pi = r % plane;          // node within the plane
        const int64_t cq = r / plane;          // component * nq + slot (u), or slot (p)
        // node index with coordinate 0 along the axis: split pi into the parts below and above it
        const int64_t low = pi % stride_n, high = pi / stride_n;
        const int64_t base = low + high * stride_n * na;
        if (is_u) {
            const int c = (int)(cq / nq), q = (int)(cq % nq);
            const int ak = (q / stride_q) % (m + 1);
            const double sign = (double)((c == axis ? -parity : parity) * ((ak & 1) ? -1 : 1));
            double *f = U + cq * nnode;
            f[base] = sign * f[base + stride_n];
            f[base + (int64_t)(na - 1) * stride_n] = sign * f[base + (int64_t)(na - 2) * stride_n];
        } else {
            P[cq * nnode + base] = 0.0;
        }
    }
}

cudaError_t launch_fill_ghosts(double *U, double *P, const int *n, int dim, int m, const int *kinds, cudaStream_t st)
{
    for (int k = 0; k < dim; ++k) {
        if (kinds[k] == 0) continue;
        const int parity = kinds[k] == 1 ? -1 : 1;  // 1 = dirichlet (p odd), 2 = neumann (p even)
        k_fill_ghosts<<<152 * 4, 256, 0, st>>>(U, P, n[0], n[1], n[2], dim, m, k, parity);
    }
    return cudaGetLastError();
}

}  // namespace hl
