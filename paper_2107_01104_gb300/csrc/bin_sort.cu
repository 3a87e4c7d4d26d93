// Cell binning (Sec. 3.3.1 "Ordering the particles locally"): block keys,
// a stable LSD radix sort of (key, index) pairs, the offset array, and the
// scatter back to the caller's particle order (the single-GPU counterpart of
// the in-order output of Sec. 3.4).
//
// The paper orders particles by x3 slice with an incomplete quicksort and
// keeps an offset[] array of group starts.  Here the groups are blocks of
// cells.  tracker_bin (and tracker_bin_static) use a stable radix sort, so the
// permutation is unique and reproducible (ties keep the incoming order).
// Everything else re-bins with a counting sort: block counts (from the update
// phase of a step, or from the keys), one scan, then one scatter of either the
// particle state (time steps) or a permutation (interpolation, the adjoint,
// batched sets).  The blocks and their offsets are those of the stable sort;
// the order inside a block is not reproducible, and no result depends on it.
#include <algorithm>

#include "internal.cuh"

namespace trk {

namespace {

constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;   // 4096 keys per tile
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_SUB = RS_TILE / RS_WARPS;       // 512 keys per warp, in order
constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_CHUNK = SCAN_THREADS * SCAN_ITEMS;

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

__global__ void k_keys(GridGeom g, int64_t np, const double* __restrict__ pos, uint32_t* __restrict__ keys,
                       int* flags, uint32_t* __restrict__ counts)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    int c[3];
    bool ok = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        ok &= split_cell(pos[a * np + p], g.inv_delta, g.mask, c[a]);
    }
    if (!ok) atomicOr(flags + FLAG_NONFINITE, 1);
    const uint32_t key = block_key(g, c[0], c[1], c[2]);
    keys[p] = key;
    if (counts) atomicAdd(counts + key, 1u);
}

// Block counts -> offsets (exclusive scan, offsets[nblocks] = total) and the
// scatter cursors (a copy of the offsets); the counts are zeroed for the next
// step.  One CTA of CS_THREADS threads; warp w owns a contiguous chunk of the
// counts and walks it with consecutive lanes (coalesced): a first pass sums
// the chunk, one scan of the warp totals, and a second pass scans 32 counts
// at a time with shuffles, carrying the running prefix.
constexpr int CS_THREADS = 1024;

__global__ void __launch_bounds__(CS_THREADS) k_count_scan(uint32_t* __restrict__ counts, int64_t nblocks,
                                                           int32_t* __restrict__ offsets, int32_t* __restrict__ cursor)
{
    constexpr int NWS = CS_THREADS / 32;
    __shared__ uint32_t warp_pre[NWS];
    __shared__ uint32_t s_total;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int64_t chunk = ((nblocks + NWS - 1) / NWS + 31) / 32 * 32;
    const int64_t c0 = min((int64_t)w * chunk, nblocks), c1 = min(c0 + chunk, nblocks);
    uint32_t sum = 0;
#pragma unroll 8
    for (int64_t i = c0 + lane; i < c1; i += 32) sum += counts[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (lane == 0) warp_pre[w] = sum;
    __syncthreads();
    if (w == 0) {
        const uint32_t x = warp_pre[lane];
        uint32_t inc = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        warp_pre[lane] = inc - x;                    // exclusive prefix of warp lane's chunk
        if (lane == 31) s_total = inc;
    }
    __syncthreads();
    uint32_t carry = warp_pre[w];
    constexpr int U = 8;                             // 32-count steps whose loads are issued together
    for (int64_t base = c0; base < c1; base += 32 * U) {
        uint32_t cv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t i = base + 32 * u + lane;
            cv[u] = i < c1 ? counts[i] : 0u;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t i = base + 32 * u + lane;
            uint32_t inc = cv[u];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += y;
            }
            if (i < c1) {
                const int32_t e = (int32_t)(carry + inc - cv[u]);
                offsets[i] = e;
                cursor[i] = e;
                counts[i] = 0u;
            }
            carry += __shfl_sync(0xffffffffu, inc, 31);
        }
    }
    if (tid == 0) offsets[nblocks] = (int32_t)s_total;
}

// The same for large grids, over all SMs: tiles of CT_TILE counts (nblocks a
// multiple of CT_TILE).  k_tile_sums sums each tile; k_tile_scan adds the sums
// of the preceding tiles and scans its own tile, CT_PER counts per thread
// read and written as 16-byte vectors.
constexpr int CT_THREADS = 256, CT_PER = 16, CT_TILE = CT_THREADS * CT_PER;
// Largest grid one CTA scans.  At 2^15 blocks (256^3 in 8^3 blocks) the two
// launches over all SMs already win: 9.5 us less per step of the 256^3
// headline workload on GB300 (0.5454 -> 0.5359 ms).
#ifndef TRK_SCAN_ONE_CTA
#define TRK_SCAN_ONE_CTA 16384
#endif
constexpr int64_t COUNT_SCAN_ONE_CTA = TRK_SCAN_ONE_CTA;

__device__ __forceinline__ uint32_t block_sum_u32(uint32_t v, uint32_t* red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();   // red may still be read by a previous call
    if (lane == 0) red[w] = v;
    __syncthreads();
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < CT_THREADS / 32; ++i) s += red[i];
    return s;
}

__global__ void __launch_bounds__(CT_THREADS) k_tile_sums(const uint32_t* __restrict__ counts,
                                                          uint32_t* __restrict__ tile_sums)
{
    __shared__ uint32_t red[CT_THREADS / 32];
    const uint4* c = reinterpret_cast<const uint4*>(counts + (int64_t)blockIdx.x * CT_TILE) + threadIdx.x;
    uint32_t s = 0;
#pragma unroll
    for (int u = 0; u < CT_PER / 4; ++u) {
        const uint4 v = c[u * CT_THREADS];
        s += v.x + v.y + v.z + v.w;
    }
    s = block_sum_u32(s, red);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = s;
}

__global__ void __launch_bounds__(CT_THREADS) k_tile_scan(uint32_t* __restrict__ counts,
                                                          const uint32_t* __restrict__ tile_sums, int64_t nblocks,
                                                          int32_t* __restrict__ offsets, int32_t* __restrict__ cursor)
{
    __shared__ uint32_t red[CT_THREADS / 32];
    __shared__ uint32_t wpre[CT_THREADS / 32];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int tile = blockIdx.x;
    // sum of the preceding tiles
    uint32_t pre = 0;
    for (int i = tid; i < tile; i += CT_THREADS) pre += tile_sums[i];
    pre = block_sum_u32(pre, red);
    // thread t owns counts [t CT_PER, (t + 1) CT_PER) of the tile
    const int64_t base = (int64_t)tile * CT_TILE + (int64_t)tid * CT_PER;
    uint4* c = reinterpret_cast<uint4*>(counts + base);
    uint32_t v[CT_PER];
#pragma unroll
    for (int u = 0; u < CT_PER / 4; ++u) {
        const uint4 q = c[u];
        v[4 * u] = q.x, v[4 * u + 1] = q.y, v[4 * u + 2] = q.z, v[4 * u + 3] = q.w;
    }
    uint32_t own = 0;
#pragma unroll
    for (int u = 0; u < CT_PER; ++u) own += v[u];
    uint32_t inc = own;   // inclusive scan of the per-thread sums over the warp, then the warps
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) wpre[w] = inc;
    __syncthreads();
    uint32_t wp = 0;
    for (int i = 0; i < w; ++i) wp += wpre[i];
    uint32_t run = pre + wp + inc - own;   // exclusive prefix of this thread's first count
    int4* o4 = reinterpret_cast<int4*>(offsets + base);
    int4* k4 = reinterpret_cast<int4*>(cursor + base);
#pragma unroll
    for (int u = 0; u < CT_PER / 4; ++u) {
        int4 e;
        e.x = (int32_t)run;
        run += v[4 * u];
        e.y = (int32_t)run;
        run += v[4 * u + 1];
        e.z = (int32_t)run;
        run += v[4 * u + 2];
        e.w = (int32_t)run;
        run += v[4 * u + 3];
        o4[u] = e;
        k4[u] = e;
        c[u] = make_uint4(0u, 0u, 0u, 0u);
    }
    if (base + CT_PER == nblocks) offsets[nblocks] = (int32_t)run;
}

// Counting-sort scatter of the particle state: particle j goes to the next
// free slot of its block.  Lanes of a warp with the same key take one
// cursor increment together (the state arrives grouped by the previous
// step's blocks, so most of a warp shares a key) and are ranked by lane, so
// their writes are contiguous.  The order of the groups inside a block
// follows the atomics (not reproducible); every particle's arithmetic is
// independent of the order, so the step results do not depend on it.
__global__ void k_scatter_state(int64_t np, const uint32_t* __restrict__ keys, int32_t* __restrict__ cursor,
                                const double* __restrict__ pos_in, const int32_t* __restrict__ id_in,
                                const float* __restrict__ rhs_in, int rhs_rows, double* __restrict__ pos_out,
                                int32_t* __restrict__ id_out, float* __restrict__ rhs_out, int* flags)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned valid = __ballot_sync(0xffffffffu, j < np);
    if (j >= np) return;
    const uint32_t key = keys[j];
    const int lane = threadIdx.x & 31;
    const unsigned peers = __match_any_sync(valid, key);
    const int leader = __ffs(peers) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(cursor + key, __popc(peers));
    base = __shfl_sync(peers, base, leader);
    const int64_t d = (int64_t)base + __popc(peers & ((1u << lane) - 1u));
    if (d < 0 || d >= np) {
        atomicOr(flags + FLAG_BINNING, 1);
        return;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) pos_out[a * np + d] = pos_in[a * np + j];
    id_out[d] = id_in ? id_in[j] : (int32_t)j;
    for (int r = 0; r < rhs_rows; ++r) rhs_out[r * np + d] = rhs_in[r * np + j];
}

// Counting-sort permutation: perm[d] = j, d the next free slot of particle
// j's block (cursor from the count scan).  Warp-aggregated like
// k_scatter_state; the order inside a block follows the atomics.  Used where
// every particle's result is independent of that order (interpolation, the
// adjoint, batched sets): the blocks and their offsets are those of the
// stable sort.
__global__ void k_scatter_perm(int64_t np, const uint32_t* __restrict__ keys, int32_t* __restrict__ cursor,
                               int32_t* __restrict__ perm, int* flags)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned valid = __ballot_sync(0xffffffffu, j < np);
    if (j >= np) return;
    const uint32_t key = keys[j];
    const int lane = threadIdx.x & 31;
    const unsigned peers = __match_any_sync(valid, key);
    const int leader = __ffs(peers) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(cursor + key, __popc(peers));
    base = __shfl_sync(peers, base, leader);
    const int64_t d = (int64_t)base + __popc(peers & ((1u << lane) - 1u));
    if (d < 0 || d >= np) {
        atomicOr(flags + FLAG_BINNING, 1);
        return;
    }
    perm[d] = (int32_t)j;
}

// Block counts of np keys, one atomic add per group of equal keys in a warp
// (keys written by a step kernel arrive grouped by the previous binning).
__global__ void k_count_keys(int64_t np, const uint32_t* __restrict__ keys, uint32_t* __restrict__ counts)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned valid = __ballot_sync(0xffffffffu, j < np);
    if (j >= np) return;
    const uint32_t key = keys[j];
    const unsigned peers = __match_any_sync(valid, key);
    if ((int)(threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(counts + key, (uint32_t)__popc(peers));
}

__global__ void k_radix_hist(const uint32_t* __restrict__ keys, int64_t n, int shift, int64_t ntiles,
                             uint32_t* __restrict__ tile_hist)
{
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
#pragma unroll
    for (int i = 0; i < RS_ITEMS; ++i) {
        const int64_t idx = base + (int64_t)i * RS_THREADS + threadIdx.x;
        if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & 255u], 1u);
    }
    __syncthreads();
    tile_hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter of one tile.  Warp w owns keys [base + 512 w, base + 512 (w+1))
// in order; ranks among equal digits come from __match_any_sync.
__global__ void k_radix_scatter(const uint32_t* __restrict__ keys_in, const int32_t* __restrict__ vals_in, int64_t n,
                                int shift, int64_t ntiles, const uint32_t* __restrict__ tile_off,
                                uint32_t* __restrict__ keys_out, int32_t* __restrict__ vals_out)
{
    __shared__ uint32_t cnt[RS_WARPS][256];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t base = (int64_t)blockIdx.x * RS_TILE + (int64_t)w * RS_SUB;
    uint32_t k[RS_ITEMS];
    int32_t v[RS_ITEMS];
    uint32_t d[RS_ITEMS];
#pragma unroll
    for (int i = 0; i < RS_ITEMS; ++i) {
        const int64_t idx = base + i * 32 + lane;
        const bool valid = idx < n;
        k[i] = valid ? keys_in[idx] : 0u;
        v[i] = valid ? (vals_in ? vals_in[idx] : (int32_t)idx) : 0;
        d[i] = valid ? ((k[i] >> shift) & 255u) : 256u;
    }
    for (int e = threadIdx.x; e < RS_WARPS * 256; e += RS_THREADS) (&cnt[0][0])[e] = 0;
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int i = 0; i < RS_ITEMS; ++i) {
        const unsigned peers = __match_any_sync(0xffffffffu, d[i]);
        if (d[i] < 256u && lane == __ffs(peers) - 1) cnt[w][d[i]] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    {
        const int dg = threadIdx.x;   // one digit per thread
        uint32_t run = tile_off[(int64_t)dg * ntiles + blockIdx.x];
#pragma unroll
        for (int ww = 0; ww < RS_WARPS; ++ww) {
            const uint32_t x = cnt[ww][dg];
            cnt[ww][dg] = run;
            run += x;
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < RS_ITEMS; ++i) {
        const unsigned peers = __match_any_sync(0xffffffffu, d[i]);
        if (d[i] < 256u) {
            const uint32_t pos = cnt[w][d[i]] + __popc(peers & lt);
            keys_out[pos] = k[i];
            vals_out[pos] = v[i];
        }
        __syncwarp();
        if (d[i] < 256u && lane == __ffs(peers) - 1) cnt[w][d[i]] += __popc(peers);
        __syncwarp();
    }
}

// Exclusive scan of one chunk of SCAN_CHUNK values; writes the chunk total.
__global__ void k_scan_chunk(uint32_t* __restrict__ data, int64_t len, uint32_t* __restrict__ chunk_sums)
{
    __shared__ uint32_t wsum[SCAN_THREADS / 32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_CHUNK + (int64_t)threadIdx.x * SCAN_ITEMS;
    uint32_t x[SCAN_ITEMS];
    uint32_t tot = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        x[i] = (base + i < len) ? data[base + i] : 0u;
        const uint32_t y = x[i];
        x[i] = tot;
        tot += y;
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t incl = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    if (w == 0) {
        uint32_t s = wsum[lane];
        uint32_t si = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, si, o);
            if (lane >= o) si += y;
        }
        wsum[lane] = si - s;   // exclusive warp offsets
        if (lane == 31 && chunk_sums) chunk_sums[blockIdx.x] = si;
    }
    __syncthreads();
    const uint32_t off = wsum[w] + (incl - tot);
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i)
        if (base + i < len) data[base + i] = x[i] + off;
}

__global__ void k_scan_add(uint32_t* __restrict__ data, int64_t len, const uint32_t* __restrict__ chunk_off)
{
    const int64_t base = (int64_t)blockIdx.x * SCAN_CHUNK;
    const uint32_t off = chunk_off[blockIdx.x];
    for (int64_t i = base + threadIdx.x; i < base + SCAN_CHUNK && i < len; i += SCAN_THREADS) data[i] += off;
}

size_t scan_scratch_bytes(int64_t len)
{
    size_t total = 0;
    while (len > SCAN_CHUNK) {
        len = ceil_div(len, SCAN_CHUNK);
        total += align256((size_t)len * sizeof(uint32_t));
    }
    return total;
}

cudaError_t scan_exclusive(uint32_t* data, int64_t len, uint32_t* scratch, cudaStream_t st, int64_t* launches)
{
    if (len <= 0) return cudaSuccess;
    const int64_t nchunks = ceil_div(len, SCAN_CHUNK);
    if (nchunks == 1) {
        k_scan_chunk<<<1, SCAN_THREADS, 0, st>>>(data, len, nullptr);
        if (launches) *launches += 1;
        return cudaGetLastError();
    }
    uint32_t* sums = scratch;
    uint32_t* rest = scratch + align256((size_t)nchunks * sizeof(uint32_t)) / sizeof(uint32_t);
    k_scan_chunk<<<(unsigned)nchunks, SCAN_THREADS, 0, st>>>(data, len, sums);
    cudaError_t e = scan_exclusive(sums, nchunks, rest, st, launches);
    if (e != cudaSuccess) return e;
    k_scan_add<<<(unsigned)nchunks, SCAN_THREADS, 0, st>>>(data, len, sums);
    if (launches) *launches += 2;
    return cudaGetLastError();
}

// offsets[b] = first sorted position whose key is >= b (b = 0 .. nblocks): a
// binary search per block over the sorted keys, grid-stride, so the work is
// spread over all threads whatever the gaps between occupied blocks.
__global__ void k_offsets(const uint32_t* __restrict__ keys, int64_t n, int64_t nblocks, int32_t* __restrict__ offsets)
{
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b <= nblocks;
         b += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = n;   // lower bound of b in keys[0, n)
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if ((int64_t)keys[mid] < b) lo = mid + 1;
            else hi = mid;
        }
        offsets[b] = (int32_t)lo;
    }
}

__global__ void k_unpermute_pos(int64_t np, const double* __restrict__ src, const int32_t* __restrict__ id,
                                double* __restrict__ dst)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= np) return;
    const int64_t p = id[j];
#pragma unroll
    for (int a = 0; a < 3; ++a) dst[a * np + p] = src[a * np + j];
}

__global__ void k_unpermute_rhs(int64_t np, const float* __restrict__ src, const int32_t* __restrict__ id,
                                float* __restrict__ dst, int rows)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= np) return;
    const int64_t p = id[j];
    for (int r = 0; r < rows; ++r) dst[r * np + p] = src[r * np + j];
}

// Fills the ghost-padded storage: padded node (x1, x2, x3) in [-PAD, N+PAD)^3
// takes the value of node (x mod N) of the dense source (periodic ghosts).
template <typename S>
__global__ void k_convert_padded(int storage, const S* __restrict__ src, int C, int N, void* __restrict__ dst)
{
    const int NP = N + 2 * PAD;
    const int64_t plane = (int64_t)NP * NP * NP;
    const int64_t total = plane * C;
    const int mask = N - 1;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = i / plane, r = i - k * plane;
        const int x3 = (int)(r / ((int64_t)NP * NP)), r2 = (int)(r - (int64_t)x3 * NP * NP);
        const int x2 = r2 / NP, x1 = r2 - x2 * NP;
        const int64_t si = (((int64_t)k * N + ((x3 - PAD) & mask)) * N + ((x2 - PAD) & mask)) * N + ((x1 - PAD) & mask);
        const S x = src[si];
        if (storage == ST_F64) {
            reinterpret_cast<double*>(dst)[i] = (double)x;
        } else if (storage == ST_F32) {
            reinterpret_cast<float*>(dst)[i] = (float)x;
        } else {
            // split of the float32-rounded value: hi = RN_bf16(x), lo = RN_bf16(x - hi)
            const float xf = (float)x;
            const __nv_bfloat16 hi = __float2bfloat16_rn(xf);
            const __nv_bfloat16 lo = __float2bfloat16_rn(xf - __bfloat162float(hi));
            reinterpret_cast<__nv_bfloat16*>(dst)[i] = hi;
            reinterpret_cast<__nv_bfloat16*>(dst)[total + i] = lo;
        }
    }
}

// nm[i][k] = f[k][i] (k < C), 0 for C <= k < nmc: each thread one node, reads
// coalesced per component, writes its nmc values contiguously
__global__ void k_node_major(const float* __restrict__ f, int C, int nmc, int64_t plane, float* __restrict__ nm)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < plane; i += (int64_t)gridDim.x * blockDim.x)
        for (int k = 0; k < nmc; ++k) nm[i * nmc + k] = k < C ? f[k * plane + i] : 0.0f;
}

// node i: the hi and lo halves of its three components, interleaved, then two zeros
__global__ void k_node_major_bf16(const __nv_bfloat16* __restrict__ hi, const __nv_bfloat16* __restrict__ lo,
                                  int64_t plane, uint4* __restrict__ nm)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < plane; i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t w[3];
#pragma unroll
        for (int k = 0; k < 3; ++k)
            w[k] = (uint32_t)__bfloat16_as_ushort(hi[k * plane + i]) |
                   ((uint32_t)__bfloat16_as_ushort(lo[k * plane + i]) << 16);
        nm[i] = make_uint4(w[0], w[1], w[2], 0u);
    }
}

unsigned grid_for(int64_t n, int threads) { return (unsigned)ceil_div(n > 0 ? n : 1, threads); }

}  // namespace

size_t scan_scratch_bytes_u32(int64_t len) { return scan_scratch_bytes(len); }

cudaError_t scan_exclusive_u32(uint32_t* data, int64_t len, uint32_t* scratch, cudaStream_t st, int64_t* launches)
{
    return scan_exclusive(data, len, scratch, st, launches);
}

cudaError_t launch_keys(const GridGeom& g, int64_t np, const double* pos, uint32_t* keys, int* flags, cudaStream_t st)
{
    if (np <= 0) return cudaSuccess;
    k_keys<<<grid_for(np, 256), 256, 0, st>>>(g, np, pos, keys, flags, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_keys_count(const GridGeom& g, int64_t np, const double* pos, uint32_t* keys, uint32_t* counts,
                              int* flags, cudaStream_t st)
{
    if (np <= 0) return cudaSuccess;
    k_keys<<<grid_for(np, 256), 256, 0, st>>>(g, np, pos, keys, flags, counts);
    return cudaGetLastError();
}

size_t count_scan_scratch_bytes(int64_t nblocks)
{
    return (size_t)((nblocks + CT_TILE - 1) / CT_TILE) * sizeof(uint32_t);
}

cudaError_t launch_count_scan(uint32_t* counts, int64_t nblocks, int32_t* offsets, int32_t* cursor,
                              uint32_t* scratch, cudaStream_t st, int64_t* launches)
{
    if (nblocks <= COUNT_SCAN_ONE_CTA || nblocks % CT_TILE != 0) {
        k_count_scan<<<1, CS_THREADS, 0, st>>>(counts, nblocks, offsets, cursor);
        if (launches) *launches += 1;
        return cudaGetLastError();
    }
    const unsigned tiles = (unsigned)(nblocks / CT_TILE);
    k_tile_sums<<<tiles, CT_THREADS, 0, st>>>(counts, scratch);
    k_tile_scan<<<tiles, CT_THREADS, 0, st>>>(counts, scratch, nblocks, offsets, cursor);
    if (launches) *launches += 2;
    return cudaGetLastError();
}

cudaError_t launch_scatter_state(int64_t np, const uint32_t* keys, int32_t* cursor, const double* pos_in,
                                 const int32_t* id_in, const float* rhs_in, int rhs_rows, double* pos_out,
                                 int32_t* id_out, float* rhs_out, int* flags, cudaStream_t st)
{
    if (np <= 0) return cudaSuccess;
    k_scatter_state<<<grid_for(np, 256), 256, 0, st>>>(np, keys, cursor, pos_in, id_in, rhs_in, rhs_in ? rhs_rows : 0,
                                                      pos_out, id_out, rhs_out, flags);
    return cudaGetLastError();
}

size_t radix_scratch_bytes(int64_t n)
{
    const int64_t ntiles = ceil_div(n > 0 ? n : 1, RS_TILE);
    const int64_t hist_len = 256 * ntiles;
    return align256((size_t)hist_len * 4) + scan_scratch_bytes(hist_len) + 4 * align256((size_t)(n > 0 ? n : 1) * 4);
}

cudaError_t radix_sort(const uint32_t* keys, int64_t n, int bits, uint32_t* keys_sorted, int32_t* perm, void* scratch,
                       cudaStream_t st, int64_t* launches)
{
    if (n <= 0) return cudaSuccess;
    const int64_t ntiles = ceil_div(n, RS_TILE);
    const int64_t hist_len = 256 * ntiles;
    char* p = reinterpret_cast<char*>(scratch);
    uint32_t* hist = reinterpret_cast<uint32_t*>(p);
    p += align256((size_t)hist_len * 4);
    uint32_t* scan_tmp = reinterpret_cast<uint32_t*>(p);
    p += scan_scratch_bytes(hist_len);
    uint32_t* ka = reinterpret_cast<uint32_t*>(p);
    p += align256((size_t)n * 4);
    int32_t* va = reinterpret_cast<int32_t*>(p);
    p += align256((size_t)n * 4);
    uint32_t* kb = reinterpret_cast<uint32_t*>(p);
    p += align256((size_t)n * 4);
    int32_t* vb = reinterpret_cast<int32_t*>(p);

    const int passes = bits <= 0 ? 1 : (bits + 7) / 8;
    const uint32_t* kin = keys;
    const int32_t* vin = nullptr;   // identity for the first pass
    for (int ps = 0; ps < passes; ++ps) {
        const bool last = ps == passes - 1;
        uint32_t* kout = last ? keys_sorted : ((ps & 1) ? kb : ka);
        int32_t* vout = last ? perm : ((ps & 1) ? vb : va);
        const int shift = 8 * ps;
        k_radix_hist<<<(unsigned)ntiles, RS_THREADS, 0, st>>>(kin, n, shift, ntiles, hist);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        e = scan_exclusive(hist, hist_len, scan_tmp, st, launches);
        if (e != cudaSuccess) return e;
        k_radix_scatter<<<(unsigned)ntiles, RS_THREADS, 0, st>>>(kin, vin, n, shift, ntiles, hist, kout, vout);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        if (launches) *launches += 2;
        kin = kout;
        vin = vout;
    }
    return cudaSuccess;
}

cudaError_t launch_offsets(const uint32_t* keys_sorted, int64_t n, int64_t nblocks, int32_t* offsets, cudaStream_t st)
{
    const unsigned grid = (unsigned)std::min<int64_t>(ceil_div(nblocks + 1, 256), 152 * 64);
    k_offsets<<<grid, 256, 0, st>>>(keys_sorted, n, nblocks, offsets);
    return cudaGetLastError();
}

cudaError_t launch_scatter_perm(int64_t np, const uint32_t* keys, int32_t* cursor, int32_t* perm, int* flags,
                                cudaStream_t st)
{
    if (np <= 0) return cudaSuccess;
    k_scatter_perm<<<grid_for(np, 256), 256, 0, st>>>(np, keys, cursor, perm, flags);
    return cudaGetLastError();
}

cudaError_t launch_count_keys(int64_t np, const uint32_t* keys, uint32_t* counts, cudaStream_t st)
{
    if (np <= 0) return cudaSuccess;
    k_count_keys<<<grid_for(np, 256), 256, 0, st>>>(np, keys, counts);
    return cudaGetLastError();
}

cudaError_t launch_unpermute_pos(int64_t np, const double* src, const int32_t* id, double* dst, cudaStream_t st)
{
    if (np <= 0) return cudaSuccess;
    k_unpermute_pos<<<grid_for(np, 256), 256, 0, st>>>(np, src, id, dst);
    return cudaGetLastError();
}

cudaError_t launch_unpermute_rhs(int64_t np, const float* src, const int32_t* id, float* dst, int rows, cudaStream_t st)
{
    if (np <= 0) return cudaSuccess;
    k_unpermute_rhs<<<grid_for(np, 256), 256, 0, st>>>(np, src, id, dst, rows);
    return cudaGetLastError();
}

cudaError_t launch_node_major(const float* f, int C, int nmc, int64_t plane, float* nm, cudaStream_t st)
{
    k_node_major<<<(unsigned)std::min<int64_t>(ceil_div(plane, 256), 1 << 20), 256, 0, st>>>(f, C, nmc, plane, nm);
    return cudaGetLastError();
}

cudaError_t launch_node_major_bf16(const __nv_bfloat16* hi, const __nv_bfloat16* lo, int64_t plane, void* nm,
                                   cudaStream_t st)
{
    k_node_major_bf16<<<(unsigned)std::min<int64_t>(ceil_div(plane, 256), 1 << 20), 256, 0, st>>>(
        hi, lo, plane, reinterpret_cast<uint4*>(nm));
    return cudaGetLastError();
}

cudaError_t launch_convert_field(int storage, int src_f64, const void* src, int C, int N, void* dst, cudaStream_t st)
{
    const int64_t NP = N + 2 * PAD;
    const int64_t n = NP * NP * NP * C;
    const unsigned grid = (unsigned)std::min<int64_t>(ceil_div(n, 256), 152 * 64);
    if (src_f64) k_convert_padded<double><<<grid, 256, 0, st>>>(storage, reinterpret_cast<const double*>(src), C, N, dst);
    else k_convert_padded<float><<<grid, 256, 0, st>>>(storage, reinterpret_cast<const float*>(src), C, N, dst);
    return cudaGetLastError();
}

}  // namespace trk
