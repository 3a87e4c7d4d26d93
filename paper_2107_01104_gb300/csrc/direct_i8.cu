// Direct-path kernels (stencils gathered from global memory) for kernel
// width I = 8, all storages and modes.
#include "block_kernel.cuh"

namespace trk {

cudaError_t launch_direct_i8(int mode, const BlockArgs& a, int deg_hi, cudaStream_t st)
{
    if (deg_hi) return dispatch_direct<8, 8 + 1>(mode, a, st);
    return dispatch_direct<8, 8 - 1>(mode, a, st);
}

}  // namespace trk
