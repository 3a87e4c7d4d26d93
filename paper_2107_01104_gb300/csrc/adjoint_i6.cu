// Adjoint block kernels for kernel width I = 6 (all storages).
#include "adjoint_kernel.cuh"

namespace trk {

cudaError_t launch_adjoint_i6(const AdjArgs& a, int64_t nblocks, int deg_hi, cudaStream_t st)
{
    if (deg_hi) return dispatch_adjoint<6, 6 + 1>(a, nblocks, st);
    return dispatch_adjoint<6, 6 - 1>(a, nblocks, st);
}

cudaError_t launch_adjoint_gather(int I, const AdjArgs& a, cudaStream_t st)
{
    const int64_t n3 = (int64_t)a.g.N * a.g.N * a.g.N;
    const unsigned grid = (unsigned)((n3 + 255) / 256);
    const bool f64 = a.f.storage == ST_F64;
    switch (I) {
        case 4:
            if (f64) k_adj_gather<double, adj_halo(4)><<<grid, 256, 0, st>>>(a);
            else k_adj_gather<float, adj_halo(4)><<<grid, 256, 0, st>>>(a);
            break;
        case 6:
            if (f64) k_adj_gather<double, adj_halo(6)><<<grid, 256, 0, st>>>(a);
            else k_adj_gather<float, adj_halo(6)><<<grid, 256, 0, st>>>(a);
            break;
        default:
            if (f64) k_adj_gather<double, adj_halo(8)><<<grid, 256, 0, st>>>(a);
            else k_adj_gather<float, adj_halo(8)><<<grid, 256, 0, st>>>(a);
            break;
    }
    return cudaGetLastError();
}

}  // namespace trk
