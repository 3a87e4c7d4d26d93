// Block kernels for kernel width I = 8 (all storages and modes).
#include "block_kernel.cuh"

namespace trk {

cudaError_t launch_block_i8(int mode, const BlockArgs& a, int64_t nblocks, int deg_hi, cudaStream_t st)
{
    if (deg_hi) return dispatch_store_mode<8, 8 + 1>(mode, a, nblocks, st);
    return dispatch_store_mode<8, 8 - 1>(mode, a, nblocks, st);
}

}  // namespace trk
