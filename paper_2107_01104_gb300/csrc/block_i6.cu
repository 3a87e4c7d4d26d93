// Block kernels for kernel width I = 6 (all storages and modes).
#include "block_kernel.cuh"

namespace trk {

cudaError_t launch_block_i6(int mode, const BlockArgs& a, const void* tmap, int64_t nblocks, int deg_hi,
                            cudaStream_t st)
{
    const CUtensorMap* m = static_cast<const CUtensorMap*>(tmap);
    if (deg_hi) return dispatch_store_mode<6, 6 + 1>(mode, a, m, nblocks, st);
    return dispatch_store_mode<6, 6 - 1>(mode, a, m, nblocks, st);
}

}  // namespace trk
