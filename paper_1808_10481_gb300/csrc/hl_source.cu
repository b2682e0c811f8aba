// Point source for the p-half (the workload's Ricker source; the paper only
// forces its manufactured-solution runs, Section 4, eq. waveEq1D, without
// stating the time discretisation).
//
//   f(x,t) = amp * R(t) * g(x),  R(t) = (1 - 2 pi^2 f0^2 (t-t0)^2) exp(-pi^2 f0^2 (t-t0)^2),
//   t0 = 1.2/f0,  g(x) = exp(-|x - x0|^2 / (2 sigma^2))  (nearest periodic image),
// injected by the midpoint rule after the p-half of step n:
//   p~_a += dt * amp * R((n + 1/2) dt) * g~_a,
// g~_a = prod_k (h_k^{a_k}/a_k!) d^{a_k}/dx_k^{a_k} exp(-(x_k - x0_k)^2/(2 sigma^2)).
// The table g~ is built once on the host over the box of nodes within
// 10 sigma of x0 on every axis (g < exp(-50) outside), stored [box node][q].
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <vector>

#include "hl_internal.h"
#include "hl_split.cuh"

namespace hl {

double ricker(double t, double f0)
{
    const double pi = 3.14159265358979323846;
    const double t0 = 1.2 / f0;
    const double a = pi * pi * f0 * f0 * (t - t0) * (t - t0);
    return (1.0 - 2.0 * a) * std::exp(-a);
}

// (h/sigma)^a/a! (-1)^a He_a(z) exp(-z^2/2), He = probabilists' Hermite polynomials
static void gauss_scaled_1d(double dx, double sigma, double h, int m, double *out)
{
    const double z = dx / sigma;
    const double g = std::exp(-0.5 * z * z);
    double hm1 = 0.0, hcur = 1.0;  // He_{a-1}, He_a
    double fact = 1.0;
    for (int a = 0; a <= m; ++a) {
        if (a > 0) fact *= a;
        out[a] = std::pow(-h / sigma, a) / fact * hcur * g;
        const double next = z * hcur - a * hm1;
        hm1 = hcur;
        hcur = next;
    }
}

bool build_source_table(int dim, int m, const int64_t *n, const double *x0, double sigma,
                        std::vector<int> &nodes, std::vector<double> &table)
{
    const int nqa = m + 1;
    int64_t nq = 1;
    for (int k = 0; k < dim; ++k) nq *= nqa;
    // per axis: the node indices within 10 sigma (all nodes if the box wraps)
    std::vector<int> idx[3];
    std::vector<double> fac[3];
    for (int k = 0; k < 3; ++k) {
        if (k >= dim) {
            idx[k] = {0};
            fac[k].assign(nqa, 0.0);
            fac[k][0] = 1.0;
            continue;
        }
        const double h = 1.0 / (double)n[k];
        const int64_t r = (int64_t)std::ceil(10.0 * sigma / h);
        const int64_t c = (int64_t)std::llround(x0[k] / h);
        std::vector<int64_t> js;
        if (2 * r + 1 >= n[k]) {
            for (int64_t j = 0; j < n[k]; ++j) js.push_back(j);
        } else {
            for (int64_t j = c - r; j <= c + r; ++j) js.push_back(((j % n[k]) + n[k]) % n[k]);
        }
        for (int64_t j : js) {
            double dx = (double)j * h - x0[k];
            dx -= std::floor(dx + 0.5);
            idx[k].push_back((int)j);
            const size_t off = fac[k].size();
            fac[k].resize(off + nqa);
            gauss_scaled_1d(dx, sigma, h, m, fac[k].data() + off);
        }
    }
    const size_t nb = idx[0].size() * idx[1].size() * idx[2].size();
    if (nb > (size_t)1 << 28) return false;
    nodes.resize(nb);
    table.assign(nb * (size_t)nq, 0.0);
    size_t b = 0;
    for (size_t i2 = 0; i2 < idx[2].size(); ++i2)
        for (size_t i1 = 0; i1 < idx[1].size(); ++i1)
            for (size_t i0 = 0; i0 < idx[0].size(); ++i0, ++b) {
                nodes[b] = (int)(idx[0][i0] + n[0] * ((int64_t)idx[1][i1] + n[1] * (int64_t)idx[2][i2]));
                for (int64_t q = 0; q < nq; ++q) {
                    const int a0 = (int)(q % nqa), a1 = (int)((q / nqa) % nqa), a2 = (int)(q / (nqa * nqa));
                    table[b * (size_t)nq + q] =
                        fac[0][i0 * nqa + a0] * fac[1][i1 * nqa + a1] * fac[2][i2 * nqa + a2];
                }
            }
    return true;
}

__global__ void k_source(double *__restrict__ P, const ShotDesc *__restrict__ shots, const int *__restrict__ node,
                         const int *__restrict__ shot, const double *__restrict__ table, int ne, int nq,
                         SourceWeights w, float *__restrict__ Ph, float *__restrict__ Pl)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ne) return;
    const int s = shot[e];
    const ShotDesc sd = shots[s];
    const int64_t base = sd.p_off + node[e];
    for (int q = 0; q < nq; ++q) {
        const int64_t idx = base + (int64_t)q * sd.nnode;
        const double v = P[idx] + w.w[s] * table[(int64_t)e * nq + q];
        P[idx] = v;
        if (Ph) {  // keep the mixed-precision shadows in step with the binary64 value
            const FF sp = split_f64(v);
            Ph[idx] = sp.hi;
            if (Pl) Pl[idx] = sp.lo;
        }
    }
}

cudaError_t launch_source(const SourceDesc &s, const ShotDesc *shots_dev, double *P, int nq, int64_t step,
                          cudaStream_t st, float *Ph, float *Pl)
{
    if (!s.active || s.n_entries == 0) return cudaSuccess;
    SourceWeights w;
    const size_t ns = s.dt.size();
    for (size_t i = 0; i < (size_t)kMaxShots; ++i)
        w.w[i] = (i < ns && s.amp[i] != 0.0) ? s.dt[i] * s.amp[i] * ricker(((double)step + 0.5) * s.dt[i], s.f0[i])
                                            : 0.0;
    k_source<<<(s.n_entries + 127) / 128, 128, 0, st>>>(P, shots_dev, s.node, s.shot, s.table, s.n_entries, nq, w,
                                                        Ph, Pl);
    return cudaGetLastError();
}

}  // namespace hl
