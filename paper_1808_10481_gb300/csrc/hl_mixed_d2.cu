// Mixed-precision kernels instantiated for dim = 2 (m <= 3).
#include "hl_mixed_dispatch.cuh"

namespace hl {

cudaError_t launch_mixed_d2(const LaunchFp64 &a)
{
    switch (a.m) {
    case 0: return run_mixed<2, 0>(a);
    case 1: return run_mixed<2, 1>(a);
    case 2: return run_mixed<2, 2>(a);
    case 3: return run_mixed<2, 3>(a);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace hl
