// Column step kernels for kernel width I = 6 (float32 fields, RK2 and Adams-Bashforth).
#include "column_kernel.cuh"

namespace trk {

cudaError_t launch_column_i6(int mode, const ColumnArgs& ca, int deg_hi, int nsm, cudaStream_t st)
{
    if (deg_hi) return dispatch_column<6, 6 + 1>(mode, ca, nsm, st);
    return dispatch_column<6, 6 - 1>(mode, ca, nsm, st);
}

}  // namespace trk
