// FP64 stepping without any device allocation.
//
// Some callers cannot call cudaMalloc at all: code that runs inside a
// pre-sized memory budget (a simulation coupled into another application
// that owns the whole device pool), real-time or safety-checked loops that
// forbid allocation after start-up, or hosts whose allocator is locked while
// they work.  For them hl_step_noalloc advances a grid held in caller-owned
// device buffers and allocates nothing on the device.  Everything the FP64
// kernels need beyond their inputs and outputs -- the status word, the
// one-entry shot table and, when it does not fit the kernel parameter bank,
// the operator table -- lives in the file-scope array below, which every GPU
// that loads the library holds until the process exits.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/hl.h"
#include "hl_internal.h"

namespace {

// Layout: [0, 256) status word; [256, 512) shot table; [512, end) operator table.
constexpr size_t kScratchBytes = HL_NOALLOC_SCRATCH_BYTES;
constexpr size_t kStatusOff = 0, kShotOff = 256, kCoefOff = 512;
static_assert(sizeof(hl::ShotDesc) <= kCoefOff - kShotOff, "shot table does not fit its slot");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned char *g_scratch_ptr[kMaxDevices] = {};  // device address of the array, per device

// once per device, with that device current: the array's device address
cudaError_t scratch_for_current_device(unsigned char **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = (unsigned char *)p;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

// stream-ordered initialisation of the scratch: shot table written, status cleared
__global__ void k_noalloc_init(unsigned char *scratch, hl::ShotDesc sd)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        *(unsigned *)(scratch + kStatusOff) = 0u;
        *(hl::ShotDesc *)(scratch + kShotOff) = sd;
    }
}

// errors are reported through hl_last_error(NULL), like hl_create's
int fail(int code, const char *msg)
{
    hl::set_handleless_error(msg);
    return code;
}

}  // namespace

extern "C" int hl_step_noalloc(int dim, int m, const int64_t *n_cells, double dt, double *p_dev, double *u_dev,
                               int64_t n_steps, void *cuda_stream)
{
    if (dim < 1 || dim > 3) return fail(HL_EINVAL, "dim must be 1, 2 or 3");
    if (m < 0 || m > 6 || (dim == 3 && m > 3)) return fail(HL_EINVAL, "m out of range (0..6, 3D 0..3)");
    if (!n_cells || !p_dev || !u_dev) return fail(HL_EINVAL, "NULL argument");
    if (n_steps < 0) return fail(HL_EINVAL, "n_steps must be >= 0");
    if (((uintptr_t)p_dev | (uintptr_t)u_dev) & 15u) return fail(HL_EINVAL, "device buffers must be 16-byte aligned");
    int64_t nnode = 1;
    double hmin = 1.0;
    double lam[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < dim; ++k) {
        if (n_cells[k] < 2 || n_cells[k] > (int64_t(1) << 30)) return fail(HL_EINVAL, "n_cells entry out of range");
        nnode *= n_cells[k];
        if (nnode >= (int64_t(1) << 31)) return fail(HL_EINVAL, "more than 2^31-1 nodes");
        hmin = hmin < 1.0 / (double)n_cells[k] ? hmin : 1.0 / (double)n_cells[k];
        lam[k] = dt * (double)n_cells[k] / 2.0;
    }
    if (!(dt > 0.0) || !(dt < hmin)) return fail(HL_EINVAL, "dt must satisfy 0 < dt < min h");
    int nq = 1;
    for (int k = 0; k < dim; ++k) nq *= (m + 1);
    const size_t ncoef = (size_t)dim * nq * nq;
    const bool in_params = ncoef * sizeof(double) <= 28 * 1024;  // same rule as the kernels
    if (!in_params && kCoefOff + ncoef * sizeof(double) > kScratchBytes)
        return fail(HL_EINVAL, "operator table exceeds the static scratch maximum (HL_NOALLOC_SCRATCH_BYTES)");
    if (n_steps == 0) return HL_OK;

    std::vector<double> coef;  // host memory only
    if (!hl::build_operator(dim, m, lam, coef)) return fail(HL_EINVAL, "operator construction failed");
    // both buffers must be device memory of the current device: the kernels
    // run there and use that device's copy of the scratch array (a pointer into
    // another GPU would be dereferenced as a peer address)
    int cur = 0;
    cudaError_t e = cudaGetDevice(&cur);
    if (e != cudaSuccess) return fail(HL_ECUDA, cudaGetErrorString(e));
    for (const void *ptr : {(const void *)p_dev, (const void *)u_dev}) {
        cudaPointerAttributes at;
        e = cudaPointerGetAttributes(&at, ptr);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(HL_EINVAL, "p_dev/u_dev are not CUDA device pointers");
        }
        if ((at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) || at.device != cur)
            return fail(HL_EINVAL, "p_dev and u_dev must be device memory of the current device");
    }
    unsigned char *scratch = nullptr;
    e = scratch_for_current_device(&scratch);
    if (e != cudaSuccess) return fail(HL_ECUDA, cudaGetErrorString(e));
    cudaStream_t st = (cudaStream_t)cuda_stream;

    hl::ShotDesc sd;
    std::memset(&sd, 0, sizeof(sd));
    const int tx = 128, ty = 1;
    for (int k = 0; k < 3; ++k) sd.n[k] = k < dim ? (int)n_cells[k] : 1;
    sd.tiles[0] = (sd.n[0] + tx - 1) / tx;
    sd.tiles[1] = (sd.n[1] + ty - 1) / ty;
    sd.tiles[2] = sd.n[2];
    sd.nnode = nnode;
    sd.p_off = 0;
    sd.u_off = 0;
    sd.tile_begin = 0;
    k_noalloc_init<<<1, 32, 0, st>>>(scratch, sd);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(HL_ECUDA, cudaGetErrorString(e));
    if (!in_params) {
        e = cudaMemcpyAsync(scratch + kCoefOff, coef.data(), ncoef * sizeof(double), cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return fail(HL_ECUDA, cudaGetErrorString(e));
    }

    hl::LaunchFp64 a;
    std::memset(&a, 0, sizeof(a));
    a.m = m;
    for (int k = 0; k < 3; ++k) a.n[k] = sd.n[k];
    a.nnode = nnode;
    a.coef_host = coef.data();
    a.coef_dev = (const double *)(scratch + kCoefOff);
    a.per_shot_coef = false;
    a.shots = (const hl::ShotDesc *)(scratch + kShotOff);
    a.n_shots = 1;
    a.total_tiles = sd.tiles[0] * sd.tiles[1] * sd.tiles[2];
    a.tx = tx;
    a.ty = ty;
    a.P = p_dev;
    a.U = u_dev;
    a.nsteps = n_steps;
    a.stream = st;
    a.status = (unsigned *)(scratch + kStatusOff);
    a.path = hl::PATH_GRID;
    a.ev = nullptr;
    a.used_small = nullptr;
    a.src = nullptr;
    a.step0 = 0;
    a.precision = HL_FP64;
    a.Ph = a.Pl = a.Uh = a.Ul = nullptr;
    a.p_elems = nnode * nq;
    e = dim == 1 ? hl::launch_fp64_d1(a) : dim == 2 ? hl::launch_fp64_d2(a) : hl::launch_fp64_d3(a);
    if (e != cudaSuccess) return fail(HL_ECUDA, cudaGetErrorString(e));
    unsigned status = 0;
    e = cudaMemcpyAsync(&status, scratch + kStatusOff, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(HL_ECUDA, cudaGetErrorString(e));
    if (status & 1u) return fail(HL_ENONFINITE, "non-finite value produced by the update");
    return HL_OK;
}
