// Internal declarations shared by the CUDA translation units of libtracker.
// Not part of the public ABI (see include/tracker.h).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "coeffs.inc"

namespace trk {

// ---------------------------------------------------------------------------
// Device error flags (one int each in a small device array owned by the
// tracker).  Set with atomicOr, read and cleared by tracker_sync().
// ---------------------------------------------------------------------------
// FLAG_BINNING: a counting-sort scatter found a block fuller than its count
// (cannot happen when every step counts what it writes; guarded anyway).
// FLAG_HALO_TIMEOUT: a tensor copy of a block's halo did not complete within
// the wait limit (the block was skipped; reported as an internal error).
enum { FLAG_NONFINITE = 0, FLAG_CFL = 1, FLAG_BINNING = 2, FLAG_HALO_TIMEOUT = 3, NUM_FLAGS = 4 };

// Storage codes (same values as trk_storage in tracker.h).
enum { ST_F64 = 0, ST_F32 = 1, ST_BF16X2 = 2 };

// Block-kernel modes.
// MODE_AB2_D: AB2 step that also writes du_k/dX_j at the step's start.
enum { MODE_INTERP = 0, MODE_INTERP_DERIV = 1, MODE_RK2 = 2, MODE_AB2 = 3, MODE_AB2_D = 4 };

constexpr int BLK = 8;        // cell-block edge used by the block kernels
constexpr int LBLK = 3;       // log2(BLK)

// The stored field is ghost-padded: PAD periodic copies on each side of every
// axis, so a block's halo is a plain box (no wrap) and its rows can be read
// with aligned 16-byte vector loads.  Component k, node (x1, x2, x3) with
// x in [-PAD, N + PAD) lives at k * plane + ((x3 + PAD) * NP + (x2 + PAD)) * NP + (x1 + PAD).
constexpr int PAD = 8;

struct FieldView {
    int storage;              // ST_*
    int C;                    // components
    int NP;                   // padded extent N + 2 PAD
    int64_t plane;            // NP^3 values per component
    const double* f64;        // [C][NP^3]                (ST_F64)
    const float* f32;         // [C][NP^3]                (ST_F32)
    const __nv_bfloat16* hi;  // [C][NP^3] high parts     (ST_BF16X2)
    const __nv_bfloat16* lo;  // [C][NP^3] low parts      (ST_BF16X2)
    const float* nm;          // node-major copy for the direct path, or null: float32 fields [NP^3][nmc];
                              // split-bf16 fields with C = 3: 16 bytes per node (hi0 lo0 hi1 lo1 hi2 lo2 0 0)
    int nmc;                  // float32: floats per node in nm, 4 for C = 3 (one 16-byte load per node), else C
    unsigned long long nm_tex; // texture object over nm (16-byte texels, C = 3), or 0 for plain loads
};

__host__ __device__ __forceinline__ int64_t padded_index(int NP, int x1, int x2, int x3)
{
    return ((int64_t)(x3 + PAD) * NP + (x2 + PAD)) * NP + (x1 + PAD);
}

// ---------------------------------------------------------------------------
// Halo box of the block kernel's TMA staging (cp.async.bulk.tensor): one
// tensor copy per component chunk writes a dense box [3][H][BY][BX] of the
// padded field into shared memory.  The box starts XOFF elements before the
// halo (its x origin rounded down to 16 bytes, as a tensor copy must be);
// BX (a multiple of 16 bytes) and BY >= H are padded so that the warp-wide
// stencil loads of the lane map of kernel width I meet as few shared-memory
// bank conflicts as the dense pitch allows (BX = row pitch, BX*BY = plane
// pitch).  Used on the host to encode the tensor map and on the device for
// the lane offsets.
// ---------------------------------------------------------------------------
// largest number of distinct words sharing a bank among `n` lane offsets
// (in elements of esz bytes; a warp's 8-byte loads are served as two halves
// of 16 lanes over 16 double-width banks)
__host__ __device__ constexpr int bank_degree(const int* offs, int n, int esz)
{
    int worst = 0;
    const int halves = esz == 8 ? 2 : 1, lanes = 32 / halves, banks = esz == 8 ? 16 : 32;
    for (int h = 0; h < halves; ++h) {
        for (int b = 0; b < banks; ++b) {
            int seen[32] = {};
            int ns = 0;
            for (int l = h * lanes; l < (h + 1) * lanes && l < n; ++l) {
                const int o = offs[l];
                if (((o % banks) + banks) % banks != b) continue;
                bool dup = false;
                for (int q = 0; q < ns; ++q) dup = dup || seen[q] == o;
                if (!dup && ns < 32) seen[ns++] = o;
            }
            worst = ns > worst ? ns : worst;
        }
    }
    return worst;
}

// worst bank degree of the stencil loads of kernel width I for row pitch S2
// and plane pitch S3 (the lane maps of Lane<T, I, D>::load)
__host__ __device__ constexpr int lane_map_degree(int I, int S2, int S3, int esz)
{
    int worst = 0;
    int offs[32] = {};
    if (I == 8) {
        for (int l = 0; l < 32; ++l) offs[l] = (l & 7) + S2 * (l >> 3);
        worst = bank_degree(offs, 32, esz);
    } else if (I == 6) {
        for (int l = 0; l < 32; ++l) offs[l] = (l < 30 ? (l % 6) + S2 * (l / 6) : (l % 6));      // pass A
        const int a = bank_degree(offs, 32, esz);
        for (int l = 0; l < 32; ++l) offs[l] = (l < 30 ? (l % 6) + S3 * (l / 6) : (l % 6));      // pass B
        const int b = bank_degree(offs, 32, esz);
        worst = a > b ? a : b;
    } else {
        for (int l = 0; l < 32; ++l) offs[l] = (l & 3) + S2 * ((l >> 2) & 3) + S3 * (l >> 4);
        worst = bank_degree(offs, 32, esz);
    }
    return worst;
}

struct TmaBox {
    int H, XOFF, BX, BY;
    __host__ __device__ constexpr int S2() const { return BX; }
    __host__ __device__ constexpr int S3() const { return BX * BY; }
    __host__ __device__ constexpr int SC() const { return BX * BY * H; }
};

// The box for kernel width I, RK2 margin `margin` (0 or 1) and element size esz:
// among row pitches up to 6 vectors beyond the minimum and plane heights up
// to 8 rows beyond H, the lowest bank degree, then the smallest box.
__host__ __device__ constexpr TmaBox tma_box(int I, int margin, int esz)
{
    const int H = 8 + I - 1 + 2 * margin;          // BLK + I - 1 + 2 margin
    const int G = I / 2 - 1 + margin;
    const int VEC = 16 / esz;
    const int XOFF = ((8 - G) % VEC + VEC) % VEC;   // PAD = 8
    const int bx0 = (H + XOFF + VEC - 1) / VEC * VEC;
    TmaBox best{H, XOFF, bx0, H};
    int best_deg = 1 << 20, best_size = 1 << 30;
    for (int bx = bx0; bx <= bx0 + 6 * VEC; bx += VEC)
        for (int by = H; by <= H + 8; ++by) {
            const int d = lane_map_degree(I, bx, bx * by, esz);
            const int size = bx * by;
            if (d < best_deg || (d == best_deg && size < best_size)) {
                best_deg = d;
                best_size = size;
                best = TmaBox{H, XOFF, bx, by};
            }
        }
    return best;
}

// Kernel weights beta_i(s), s = t - 1/2, as polynomial coefficients, passed by
// value so that the kernels read them as constant-bank operands.
template <typename T>
struct CoefTable {
    T c[TRK_TAB_MAX_I][TRK_TAB_MAX_DEG];   // beta_i
    T d[TRK_TAB_MAX_I][TRK_TAB_MAX_DEG];   // beta_i' (d/dt)
};

struct GridGeom {
    int N, mask;
    int lb1, lb2, lb3;        // log2 of the binning block edges
    int nb1, nb2, nb3;        // blocks per axis
    double inv_delta;         // fl(N / L)
};

// Arguments of the block and direct kernels (interpolation, RK2 step, AB step).
struct BlockArgs {
    GridGeom g;
    FieldView f;
    CoefTable<float> cf;      // weights for float32 arithmetic
    CoefTable<double> cd;     // weights for float64 arithmetic
    int64_t np;               // particle count (stride of the [3][np] arrays)
    const int32_t* offsets;   // [nblocks + 1]
    const int32_t* perm;      // sorted position j -> index into the *_in arrays, or null (identity)
    const double* pos_in;     // [3][np]
    const int32_t* id_in;     // [np] or null (then id = perm[j])
    const float* rhs_in;      // [ab_order-1][3][np] AB history (u_{n-1} first) or null
    double* pos_out;          // [3][np], written at j
    int32_t* id_out;          // [np], written at j
    float* rhs_out;           // [ab_order-1][3][np], written at j
    uint32_t* key_out;        // [np], written at j
    uint32_t* counts;         // [nblocks] block counts of the new keys (added into) or null
    void* out;                // interpolation outputs [nout][np], written at id
    int out_f64;
    int history_valid;        // AB: valid history entries on entry, 0 .. ab_order-1
    int ab_order;             // AB order k (2, 3, 4); the history holds k-1 entries
    int ppc;                  // direct kernel: particles per CTA (1 .. 256; 0 means 256)
    double dt;
    int* flags;
};

constexpr int AB_MAX_HIST = 3;   // history entries of the highest supported order (AB4)

// where the direct path gathers a float32 stencil from: the component-major
// field, the node-major copy per component, or the node-major copy as one
// 16-byte load per node (three components padded to four floats), by plain
// loads or by texture fetches (the same bits, on the texture data path)
enum { NM_NONE = 0, NM_SCALAR = 1, NM_VEC4 = 2, NM_TEX4 = 3 };

// dt-free Adams-Bashforth increment of order q (1..4): sum_j beta^q_j u_{n-j}
// with u_n = f0 and u_{n-j} = hist(j - 1), summed newest first; beta^q are the
// textbook weights (integrals over one step of the Lagrange basis on the past
// steps).
template <class HIST>
__device__ __forceinline__ double ab_increment(int q, double f0, const HIST& hist)
{
    switch (q) {
        case 1: return f0;
        case 2: return 1.5 * f0 + (-0.5) * hist(0);
        case 3: return (23.0 / 12.0) * f0 + (-16.0 / 12.0) * hist(0) + (5.0 / 12.0) * hist(1);
        default:
            return (55.0 / 24.0) * f0 + (-59.0 / 24.0) * hist(0) + (37.0 / 24.0) * hist(1) +
                   (-9.0 / 24.0) * hist(2);
    }
}

// Arguments of the adjoint block kernel (one RK2 step, backwards).
struct AdjArgs {
    GridGeom g;
    FieldView f;
    CoefTable<float> cf;
    CoefTable<double> cd;
    int64_t np;
    const int32_t* offsets;   // [nblocks + 1] of the binned positions
    const int32_t* perm;      // sorted position j -> particle index
    const double* pos;        // [3][np] X at the start of the step, particle order
    const double* lam_in;     // [3][np] dLoss/dX' (particle order)
    double* lam_out;          // [3][np] dLoss/dX   (particle order)
    double* gfield;           // [3][N^3] dLoss/dfield (dense, added into) or null
    void* gscratch;           // [nblocks][3][H^3] per-block W^T partial sums (float, or double for
                              // float64 storage), or null: float64 atomics instead
    double dt;
    int* flags;
};

// One particle set of a batched step, resident in device memory.
struct BatchSet {
    BlockArgs a;              // set's step arguments (field, weights, state buffers)
    const int32_t* list;      // non-empty blocks in key order (halo path)
    const int32_t* count;     // number of non-empty blocks (device, halo path)
    int n_items;              // number of 256-particle chunks (direct path)
    int I, deg_hi, deriv, direct;
};

// Arguments of the column step kernel (RK2 / AB over column segments of cell
// blocks, float32 fields, I = 4 or 6).  The state arrays a.pos_out / a.rhs_out
// hold the particles grouped by block and are updated in place; a.perm and
// a.id_* are unused (the scatter kernel has grouped the state).
constexpr int MAXSEG = 64;    // largest column segment (slabs per work item)

struct ColumnArgs {
    BlockArgs a;
    int nseg;                 // slabs per work item (divides nb3, <= MAXSEG)
    int64_t nitems;           // work items: nb1 * nb2 * (nb3 / nseg)
    int* ctr;                 // work counter, zero at launch
    uint32_t* counts;         // [nblocks] block counts of the new keys (added into) or null
};

// ---------------------------------------------------------------------------
// Cell split (Sec. 2.2 steps 1-3), bit-exact with the float64 reference:
//   g = X * fl(N/L), c0 = floor(g), t = g - c0, c = c0 mod N.
// __dmul_rn/__dsub_rn forbid fused multiply-adds.  Positions beyond 2^51
// cells are rejected (returned false) together with NaN/Inf.
// ---------------------------------------------------------------------------
// |g| < 2^51, false for NaN and Inf: the biased exponent of g is below
// 1023 + 51 (an integer test, which keeps it off the float64 pipe)
__device__ __forceinline__ bool cell_in_range(double g)
{
    return ((__double2hiint(g) >> 20) & 0x7ff) < 1074;
}

__device__ __forceinline__ bool split_axis(double X, double inv_delta, int mask, int& c, double& t)
{
    const double g = __dmul_rn(X, inv_delta);
    if (!cell_in_range(g)) {
        c = 0;
        t = 0.0;
        return false;
    }
    const double c0 = floor(g);
    t = __dsub_rn(g, c0);
    c = (int)(__double2ll_rz(c0) & (long long)mask);
    return true;
}

// The cell only (for block keys): floor(g) by one conversion rounding down,
// which equals floor then truncation for |g| < 2^51.
__device__ __forceinline__ bool split_cell(double X, double inv_delta, int mask, int& c)
{
    const double g = __dmul_rn(X, inv_delta);
    if (!cell_in_range(g)) {
        c = 0;
        return false;
    }
    c = (int)(__double2ll_rd(g) & (long long)mask);
    return true;
}

__device__ __forceinline__ uint32_t block_key(const GridGeom& g, int c1, int c2, int c3)
{
    return (uint32_t)((((c3 >> g.lb3) * g.nb2) + (c2 >> g.lb2)) * g.nb1 + (c1 >> g.lb1));
}

// ---------------------------------------------------------------------------
// Host-side launchers (defined in the .cu files).  All take a stream and
// return a cudaError_t.
// ---------------------------------------------------------------------------
cudaError_t launch_keys(const GridGeom& g, int64_t np, const double* pos, uint32_t* keys, int* flags,
                        cudaStream_t st);

// Scratch layout for the radix sort of n keys.
size_t radix_scratch_bytes(int64_t n);
// Stable LSD radix sort of (keys, index) by the low `bits` bits of keys.
// keys_sorted and perm receive the result; scratch is radix_scratch_bytes(n).
cudaError_t radix_sort(const uint32_t* keys, int64_t n, int bits, uint32_t* keys_sorted, int32_t* perm,
                       void* scratch, cudaStream_t st, int64_t* launches);

cudaError_t launch_offsets(const uint32_t* keys_sorted, int64_t n, int64_t nblocks, int32_t* offsets,
                           cudaStream_t st);

// Scatter sorted state back to the caller's order: dst[a][id[j]] = src[a][j].
cudaError_t launch_unpermute_pos(int64_t np, const double* src, const int32_t* id, double* dst, cudaStream_t st);
cudaError_t launch_unpermute_rhs(int64_t np, const float* src, const int32_t* id, float* dst, int rows, cudaStream_t st);

// Fill the ghost-padded storage from a dense field src[C][N][N][N] (periodic ghosts).
cudaError_t launch_convert_field(int storage, int src_f64, const void* src, int C, int N, void* dst, cudaStream_t st);
// node-major copy nm[node][nmc] of the padded float32 field f[C][node] (plane nodes);
// floats C .. nmc-1 of a node are zero
cudaError_t launch_node_major(const float* f, int C, int nmc, int64_t plane, float* nm, cudaStream_t st);
// node-major copy of a three-component split-bf16 field (hi planes, then lo planes): 16 bytes per node
cudaError_t launch_node_major_bf16(const __nv_bfloat16* hi, const __nv_bfloat16* lo, int64_t plane, void* nm,
                                   cudaStream_t st);

// dLoss/dfield from the per-block partial sums: every node adds, in a fixed
// order, the partials of the non-empty blocks whose halo holds it
cudaError_t launch_adjoint_gather(int I, const AdjArgs& a, cudaStream_t st);
// halo edge of the adjoint kernel for kernel width I (stage-2 margin included)
constexpr int adj_halo(int I) { return BLK + I - 1 + 2; }
cudaError_t launch_adjoint_i4(const AdjArgs& a, int64_t nblocks, int deg_hi, cudaStream_t st);
cudaError_t launch_adjoint_i6(const AdjArgs& a, int64_t nblocks, int deg_hi, cudaStream_t st);
cudaError_t launch_adjoint_i8(const AdjArgs& a, int64_t nblocks, int deg_hi, cudaStream_t st);

// Exclusive scan of a uint32 array in place; scratch is scan_scratch_bytes_u32(len).
size_t scan_scratch_bytes_u32(int64_t len);
cudaError_t scan_exclusive_u32(uint32_t* data, int64_t len, uint32_t* scratch, cudaStream_t st, int64_t* launches);

// Compacted list of the non-empty blocks (in key order) and its length.
size_t nonempty_scratch_bytes(int64_t nblocks);
cudaError_t launch_nonempty_list(const int32_t* offsets, int64_t nblocks, int32_t* list, int32_t* count, void* scratch,
                                 cudaStream_t st, int64_t* launches);

// One persistent launch over all sets (float32 or split-bf16 storage); grid = 2 CTAs per SM.
// maps: null, or three CUtensorMap pointers (AB2 halo boxes of widths 4, 6, 8) for
// tensor-copy halos of the float32 field
cudaError_t launch_batched(int storage, const BatchSet* sets, int nsets, int* ctr, int nsm, const void* const* maps,
                           cudaStream_t st);

// Sets the thread-local message returned by tracker_last_error().
void set_error_message(const char* msg);

// True if p points into memory of device dev (or managed memory): the check
// the binning entry points make on caller arrays that their kernels write.
bool device_pointer_ok(const void* p, int dev);

// Block kernels, one entry per kernel width I (block_i4.cu, block_i6.cu, block_i8.cu).
// deg_hi selects the degree-(I+1) instantiation (spline with m = I/2).
cudaError_t launch_column_i4(int mode, const ColumnArgs& ca, int deg_hi, int nsm, cudaStream_t st);
cudaError_t launch_column_i6(int mode, const ColumnArgs& ca, int deg_hi, int nsm, cudaStream_t st);
// counting-sort binning of the step path: keys with block counts; counts ->
// offsets + cursors (counts zeroed); scatter of the state into its blocks
cudaError_t launch_keys_count(const GridGeom& g, int64_t np, const double* pos, uint32_t* keys, uint32_t* counts,
                              int* flags, cudaStream_t st);
// Small grids are scanned by one CTA (one launch); larger grids take two
// launches over all SMs with count_scan_scratch_bytes of scratch.
size_t count_scan_scratch_bytes(int64_t nblocks);
cudaError_t launch_count_scan(uint32_t* counts, int64_t nblocks, int32_t* offsets, int32_t* cursor,
                              uint32_t* scratch, cudaStream_t st, int64_t* launches);
// counting-sort permutation of keys (cursor from launch_count_scan): perm[d] = j
cudaError_t launch_scatter_perm(int64_t np, const uint32_t* keys, int32_t* cursor, int32_t* perm, int* flags,
                                cudaStream_t st);
// counts[key] += number of particles with that key
cudaError_t launch_count_keys(int64_t np, const uint32_t* keys, uint32_t* counts, cudaStream_t st);
cudaError_t launch_scatter_state(int64_t np, const uint32_t* keys, int32_t* cursor, const double* pos_in,
                                 const int32_t* id_in, const float* rhs_in, int rhs_rows, double* pos_out,
                                 int32_t* id_out, float* rhs_out, int* flags, cudaStream_t st);
// tmap: a CUtensorMap of the padded field with the box tma_box(I, margin of
// the mode, element size) for tensor-copy halo staging (float32 and float64
// storage), or null for cp.async element copies
cudaError_t launch_block_i4(int mode, const BlockArgs& a, const void* tmap, int64_t nblocks, int deg_hi,
                            cudaStream_t st);
cudaError_t launch_block_i6(int mode, const BlockArgs& a, const void* tmap, int64_t nblocks, int deg_hi,
                            cudaStream_t st);
cudaError_t launch_block_i8(int mode, const BlockArgs& a, const void* tmap, int64_t nblocks, int deg_hi,
                            cudaStream_t st);
// direct path (sparse particle sets): a.np sorted particles, PB per CTA, stencils from global memory
cudaError_t launch_direct_i4(int mode, const BlockArgs& a, int deg_hi, cudaStream_t st);
cudaError_t launch_direct_i6(int mode, const BlockArgs& a, int deg_hi, cudaStream_t st);
cudaError_t launch_direct_i8(int mode, const BlockArgs& a, int deg_hi, cudaStream_t st);

}  // namespace trk
