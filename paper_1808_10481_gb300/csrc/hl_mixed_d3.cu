// Mixed-precision kernels instantiated for dim = 3 (m <= 2: larger tables exceed the parameter bank).
#include "hl_mixed_dispatch.cuh"

namespace hl {

cudaError_t launch_mixed_d3(const LaunchFp64 &a)
{
    switch (a.m) {
    case 0: return run_mixed<3, 0>(a);
    case 1: return run_mixed<3, 1>(a);
    case 2: return run_mixed<3, 2>(a);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace hl
