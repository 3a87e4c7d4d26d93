// Adjoint block kernels for kernel width I = 6 (all storages).
#include "adjoint_kernel.cuh"

namespace trk {

cudaError_t launch_adjoint_i6(const AdjArgs& a, int64_t nblocks, int deg_hi, cudaStream_t st)
{
    if (deg_hi) return dispatch_adjoint<6, 6 + 1>(a, nblocks, st);
    return dispatch_adjoint<6, 6 - 1>(a, nblocks, st);
}

}  // namespace trk
