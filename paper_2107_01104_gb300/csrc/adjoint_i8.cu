// Adjoint block kernels for kernel width I = 8 (all storages).
#include "adjoint_kernel.cuh"

namespace trk {

cudaError_t launch_adjoint_i8(const AdjArgs& a, int64_t nblocks, int deg_hi, cudaStream_t st)
{
    if (deg_hi) return dispatch_adjoint<8, 8 + 1>(a, nblocks, st);
    return dispatch_adjoint<8, 8 - 1>(a, nblocks, st);
}

}  // namespace trk
