// Adjoint block kernels for kernel width I = 4 (all storages).
#include "adjoint_kernel.cuh"

namespace trk {

cudaError_t launch_adjoint_i4(const AdjArgs& a, int64_t nblocks, int deg_hi, cudaStream_t st)
{
    if (deg_hi) return dispatch_adjoint<4, 4 + 1>(a, nblocks, st);
    return dispatch_adjoint<4, 4 - 1>(a, nblocks, st);
}

}  // namespace trk
