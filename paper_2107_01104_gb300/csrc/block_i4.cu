// Block kernels for kernel width I = 4 (all storages and modes).
#include "block_kernel.cuh"

namespace trk {

cudaError_t launch_block_i4(int mode, const BlockArgs& a, int64_t nblocks, int deg_hi, cudaStream_t st)
{
    if (deg_hi) return dispatch_store_mode<4, 4 + 1>(mode, a, nblocks, st);
    return dispatch_store_mode<4, 4 - 1>(mode, a, nblocks, st);
}

}  // namespace trk
