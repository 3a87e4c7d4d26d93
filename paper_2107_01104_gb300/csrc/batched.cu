// Batched AB2 advection: many particle sets of uneven size and different
// kernels (I = 4, 6, 8; value or value + gradient outputs) advanced by ONE
// persistent launch per step.  CTAs take work items from a per-set atomic
// counter, set after set: an item is a non-empty cell block (halo-staged
// path) or, for sparse sets, a chunk of 256 sorted particles gathered straight
// from global memory (direct path, through the node-major copy of the field:
// one 16-byte load per stencil node).  The choice per set is made on the
// host (tracker_host.cu) by timing both paths once.
#include <algorithm>

#include "block_kernel.cuh"

namespace trk {

namespace {

// tmap: the tensor map of the field with the AB2 halo box of width I (float32
// storage), or null for cp.async halo copies
template <int I, int DEG, int STORE>
__device__ __noinline__ void run_item(const BatchSet& S, int b, int j0, int j1, unsigned char* smem,
                                      const CUtensorMap* tmap)
{
    // batched fields have three components: 16-byte node loads, plain ones (a
    // texture-fetch variant beside them in this function made the compiler
    // spill several KB per item on the float32 paths)
    constexpr int NM = NM_VEC4;
    if (S.direct) {
        if (S.deriv) process_block<float, I, DEG, MODE_AB2_D, STORE, false, NM>(S.a, b, j0, j1, smem);
        else process_block<float, I, DEG, MODE_AB2, STORE, false, NM>(S.a, b, j0, j1, smem);
        return;
    }
    if constexpr (STORE == ST_F32) {
        if (tmap) {
            if (S.deriv) process_block<float, I, DEG, MODE_AB2_D, STORE, true, NM_NONE, HC_TMA>(S.a, b, j0, j1, smem, tmap);
            else process_block<float, I, DEG, MODE_AB2, STORE, true, NM_NONE, HC_TMA>(S.a, b, j0, j1, smem, tmap);
            return;
        }
    }
    if (S.deriv) process_block<float, I, DEG, MODE_AB2_D, STORE, true>(S.a, b, j0, j1, smem);
    else process_block<float, I, DEG, MODE_AB2, STORE, true>(S.a, b, j0, j1, smem);
}

// m4, m6, m8: tensor maps of the field with the AB2 halo boxes of widths 4, 6, 8
// (read only when use_tma, float32 storage)
template <int STORE>
__global__ void __launch_bounds__(NT, 2) k_batched(const BatchSet* __restrict__ sets, int nsets, int* ctr,
                                                   const __grid_constant__ CUtensorMap m4,
                                                   const __grid_constant__ CUtensorMap m6,
                                                   const __grid_constant__ CUtensorMap m8, int use_tma)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ int s_item;
    for (int s = 0; s < nsets; ++s) {
        const BatchSet& S = sets[s];
        const int n_items = S.direct ? S.n_items : *S.count;
        for (;;) {
            if (threadIdx.x == 0) s_item = atomicAdd(ctr + s, 1);
            __syncthreads();
            const int it = s_item;
            __syncthreads();
            if (it >= n_items) break;
            int b = 0, j0, j1;
            if (S.direct) {
                j0 = it * PB;
                j1 = (int)((int64_t)j0 + PB < S.a.np ? (int64_t)j0 + PB : S.a.np);
            } else {
                b = S.list[it];
                j0 = S.a.offsets[b];
                j1 = S.a.offsets[b + 1];
            }
            const CUtensorMap* tm = !use_tma ? nullptr : (S.I == 4 ? &m4 : (S.I == 6 ? &m6 : &m8));
            switch (S.I * 2 + S.deg_hi) {
                case 8: run_item<4, 3, STORE>(S, b, j0, j1, smem_raw, tm); break;
                case 9: run_item<4, 5, STORE>(S, b, j0, j1, smem_raw, tm); break;
                case 12: run_item<6, 5, STORE>(S, b, j0, j1, smem_raw, tm); break;
                case 13: run_item<6, 7, STORE>(S, b, j0, j1, smem_raw, tm); break;
                case 16: run_item<8, 7, STORE>(S, b, j0, j1, smem_raw, tm); break;
                default: run_item<8, 9, STORE>(S, b, j0, j1, smem_raw, tm); break;
            }
            __syncthreads();   // the item's shared memory may be re-used by the next item
        }
    }
}

// flags[b] = 1 if block b holds particles
__global__ void k_nonempty_flags(const int32_t* __restrict__ offsets, int64_t nblocks, uint32_t* __restrict__ flags)
{
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nblocks) flags[b] = offsets[b + 1] > offsets[b] ? 1u : 0u;
}

// after the exclusive scan of the flags: list[pos[b]] = b for non-empty b
__global__ void k_nonempty_compact(const int32_t* __restrict__ offsets, int64_t nblocks, const uint32_t* __restrict__ pos,
                                   int32_t* __restrict__ list, int32_t* __restrict__ count)
{
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nblocks) return;
    const bool ne = offsets[b + 1] > offsets[b];
    if (ne) list[pos[b]] = (int32_t)b;
    if (b == nblocks - 1) *count = (int32_t)(pos[b] + (ne ? 1u : 0u));
}

constexpr size_t max_batched_smem()
{
    constexpr size_t a = std::max(block_smem_bytes<float, 4, MODE_AB2>(),
                                  std::max(block_smem_bytes<float, 6, MODE_AB2>(), block_smem_bytes<float, 8, MODE_AB2>()));
    constexpr size_t b = std::max(block_smem_bytes<float, 4, MODE_AB2, HC_TMA>(),
                                  std::max(block_smem_bytes<float, 6, MODE_AB2, HC_TMA>(),
                                           block_smem_bytes<float, 8, MODE_AB2, HC_TMA>()));
    return std::max(a, b);
}

}  // namespace

size_t nonempty_scratch_bytes(int64_t nblocks)
{
    return ((size_t)nblocks * 4 + 255) / 256 * 256 + scan_scratch_bytes_u32(nblocks);
}

cudaError_t launch_nonempty_list(const int32_t* offsets, int64_t nblocks, int32_t* list, int32_t* count, void* scratch,
                                 cudaStream_t st, int64_t* launches)
{
    uint32_t* flags = reinterpret_cast<uint32_t*>(scratch);
    uint32_t* scan_tmp = flags + ((size_t)nblocks * 4 + 255) / 256 * 64;
    const unsigned grid = (unsigned)((nblocks + 255) / 256);
    k_nonempty_flags<<<grid, 256, 0, st>>>(offsets, nblocks, flags);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = scan_exclusive_u32(flags, nblocks, scan_tmp, st, launches);
    if (e != cudaSuccess) return e;
    k_nonempty_compact<<<grid, 256, 0, st>>>(offsets, nblocks, flags, list, count);
    if (launches) *launches += 2;
    return cudaGetLastError();
}

cudaError_t launch_batched(int storage, const BatchSet* sets, int nsets, int* ctr, int nsm, const void* const* maps,
                           cudaStream_t st)
{
    constexpr size_t smem = max_batched_smem();
    static_assert(2 * (smem + 1024) <= 233472, "two batched CTAs must fit on an SM");
    const CUtensorMap none{};
    const bool tma = maps && maps[0] && maps[1] && maps[2];
    const CUtensorMap& m4 = tma ? *static_cast<const CUtensorMap*>(maps[0]) : none;
    const CUtensorMap& m6 = tma ? *static_cast<const CUtensorMap*>(maps[1]) : none;
    const CUtensorMap& m8 = tma ? *static_cast<const CUtensorMap*>(maps[2]) : none;
    static bool attr_set[3] = {false, false, false};
    const int grid = nsm * 2;
    if (storage == ST_F32) {
        if (!attr_set[ST_F32]) {
            cudaError_t e = cudaFuncSetAttribute(k_batched<ST_F32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            attr_set[ST_F32] = true;
        }
        k_batched<ST_F32><<<grid, NT, smem, st>>>(sets, nsets, ctr, m4, m6, m8, tma ? 1 : 0);
    } else if (storage == ST_BF16X2) {
        if (!attr_set[ST_BF16X2]) {
            cudaError_t e =
                cudaFuncSetAttribute(k_batched<ST_BF16X2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            attr_set[ST_BF16X2] = true;
        }
        k_batched<ST_BF16X2><<<grid, NT, smem, st>>>(sets, nsets, ctr, none, none, none, 0);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace trk
