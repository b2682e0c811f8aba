// FP64 kernels instantiated for dim = 1.
#include "hl_fp64_dispatch.cuh"

namespace hl {

cudaError_t launch_fp64_d1(const LaunchFp64 &a)
{
    switch (a.m) {
    case 0: return run_fp64<1, 0>(a);
    case 1: return run_fp64<1, 1>(a);
    case 2: return run_fp64<1, 2>(a);
    case 3: return run_fp64<1, 3>(a);
    case 4: return run_fp64<1, 4>(a);
    case 5: return run_fp64<1, 5>(a);
    case 6: return run_fp64<1, 6>(a);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace hl
