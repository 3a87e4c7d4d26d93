// Direct-path kernels (stencils gathered from global memory) for kernel
// width I = 6, all storages and modes.
#include "block_kernel.cuh"

namespace trk {

cudaError_t launch_direct_i6(int mode, const BlockArgs& a, int deg_hi, cudaStream_t st)
{
    if (deg_hi) return dispatch_direct<6, 6 + 1>(mode, a, st);
    return dispatch_direct<6, 6 - 1>(mode, a, st);
}

}  // namespace trk
