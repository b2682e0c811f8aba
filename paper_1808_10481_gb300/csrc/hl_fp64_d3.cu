// FP64 kernels instantiated for dim = 3.
#include "hl_fp64_dispatch.cuh"

namespace hl {

cudaError_t launch_fp64_d3(const LaunchFp64 &a)
{
    switch (a.m) {
    case 0: return run_fp64<3, 0>(a);
    case 1: return run_fp64<3, 1>(a);
    case 2: return run_fp64<3, 2>(a);
    case 3: return run_fp64<3, 3>(a);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace hl
