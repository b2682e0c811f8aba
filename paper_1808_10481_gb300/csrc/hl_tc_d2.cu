// Tensor-core split mode instantiated for dim = 2 (m <= 3): tcgen05 kernels.
#include "hl_tc5.cuh"

namespace hl {

cudaError_t launch_tc_d2(const LaunchFp64 &a)
{
    switch (a.m) {
    case 0: return run_tc5<0>(a);
    case 1: return run_tc5<1>(a);
    case 2: return run_tc5<2>(a);
    case 3: return run_tc5<3>(a);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace hl
