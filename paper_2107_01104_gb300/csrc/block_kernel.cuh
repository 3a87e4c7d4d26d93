// Block kernels: one CTA per cell block of BLK^3 cells (the block grouping of
// Sec. 3.3.1, with the paper's x3 slices generalised to cubes).  They serve
// interpolation, the batched steps, and the time steps of the storages and
// kernel widths the column kernel (column_kernel.cuh) does not cover; this
// file also holds the pieces both share (lane maps, weights, reductions).
//
// A CTA stages the block's field halo in shared memory once (cp.async element
// copies for float32/float64 storage, issued before P1 and completed before
// the first barrier; 16-byte vector loads through registers for split bf16)
// and runs the per-particle work in phases separated by __syncthreads():
//
//   P1  one thread per particle: read X through the sort permutation, split it
//       into cell c and offset t (float64, Sec. 2.2 steps 1-3), keep X, the
//       caller id and the AB history in shared memory for P3;
//   Q   one warp per particle: evaluate the 1-D weights beta_i per axis, gather
//       the I x I x I stencil from shared memory into registers and contract it
//       (Eq. triple_sum, separably as in Sec. 3.3), reduce across the warp.
//       For RK2 the warp then forms the stage-2 point in cell-relative
//       coordinates, t* = t + dt u(X) / delta, and contracts again, re-using
//       the stencil registers when X* lies in the same cell;
//   P3  one thread per particle: float64 position update (RK2 or AB) from the
//       staged X, new cell split and block key for the next re-binning,
//       coalesced write-out.
//
// Warp-per-particle lane maps (every warp-wide shared load hits 32 distinct
// banks, see Layout):
//   I = 8: lane = (i1 in 0..7, j in 0..3); i2 = j and j+4; i3 = 0..7
//   I = 6: lane = (i1 in 0..5, j in 0..4); pass A i2 = j, i3 = 0..5;
//          pass B i2 = 5, i3 = j; pass C (lanes 0..5) i2 = i3 = 5
//   I = 4: lane = (i1, i2 in 0..3, p in 0..1); i3 = p and p+2
#pragma once

#include <cuda.h>   // CUtensorMap (type only; the library does not link the driver API)

#include "internal.cuh"

namespace trk {

constexpr int NT = 256;           // threads per CTA
constexpr int NW = NT / 32;       // warps per CTA
constexpr int PB = NT;            // particles per batch (one per thread in the P phases)

// ---------------------------------------------------------------------------
// Shared-memory layout of the halo: [3 components][H][H][S2], row stride S2,
// plane stride S3, component stride SC.  S2, S3: the smallest strides for
// which the lane map of kernel width I reads 32 distinct banks.
// ---------------------------------------------------------------------------
constexpr bool distinct_banks(const int* offs, int n)
{
    bool seen[32] = {};
    for (int l = 0; l < n; ++l) {
        int b = ((offs[l] % 32) + 32) % 32;
        if (seen[b]) return false;
        seen[b] = true;
    }
    return true;
}

template <int I>
constexpr bool row_ok(int S2)
{
    int offs[32] = {};
    if (I == 8) {
        for (int l = 0; l < 32; ++l) offs[l] = (l & 7) + S2 * (l >> 3);
        return distinct_banks(offs, 32);
    } else if (I == 6) {
        for (int l = 0; l < 30; ++l) offs[l] = (l % 6) + S2 * (l / 6);
        return distinct_banks(offs, 30);
    } else {
        for (int l = 0; l < 16; ++l) offs[l] = (l & 3) + S2 * ((l >> 2) & 3);
        return distinct_banks(offs, 16);
    }
}

template <int I>
constexpr bool plane_ok(int S2, int S3)
{
    int offs[32] = {};
    if (I == 8) {
        return true;
    } else if (I == 6) {
        for (int l = 0; l < 30; ++l) offs[l] = (l % 6) + S3 * (l / 6);
        return distinct_banks(offs, 30);
    } else {
        for (int l = 0; l < 32; ++l) offs[l] = (l & 3) + S2 * ((l >> 2) & 3) + S3 * (l >> 4);
        return distinct_banks(offs, 32);
    }
}

template <int I>
constexpr int find_s3(int H, int S2)
{
    for (int s = S2 * H; s < S2 * H + 64; ++s)
        if (plane_ok<I>(S2, s)) return s;
    return -1;
}

template <int I>
constexpr int find_s2(int H)
{
    for (int s = H; s < H + 64; ++s)
        if (row_ok<I>(s) && find_s3<I>(H, s) > 0) return s;
    return -1;
}

template <int I, int H>
struct Layout {
    static constexpr int S2 = find_s2<I>(H);
    static constexpr int S3 = find_s3<I>(H, S2);
    static constexpr int SC = S3 * H;
    static_assert(S2 > 0 && S3 > 0, "no conflict-free halo layout");
};

// ---------------------------------------------------------------------------
// Weight polynomials
// ---------------------------------------------------------------------------
template <typename T, class A>
__device__ __forceinline__ const CoefTable<T>& table(const A& a)
{
    if constexpr (sizeof(T) == 4) return a.cf;
    else return a.cd;
}

template <typename T, int DEG>
struct Row {
    T c[DEG + 1];
};

template <typename T, int DEG>
__device__ __forceinline__ Row<T, DEG> load_row(const T (&tab)[TRK_TAB_MAX_I][TRK_TAB_MAX_DEG], int i)
{
    Row<T, DEG> r;
#pragma unroll
    for (int d = 0; d <= DEG; ++d) r.c[d] = tab[i][d];
    return r;
}

template <typename T, int DEG>
__device__ __forceinline__ T horner(const Row<T, DEG>& r, T s)
{
    T acc = r.c[DEG];
#pragma unroll
    for (int d = DEG - 1; d >= 0; --d) acc = fma(acc, s, r.c[d]);
    return acc;
}

// compile-time row of a table held in the (grid-constant) kernel parameters
template <typename T, int DEG>
__device__ __forceinline__ T horner_c(const T (&row)[TRK_TAB_MAX_DEG], T s)
{
    T acc = row[DEG];
#pragma unroll
    for (int d = DEG - 1; d >= 0; --d) acc = fma(acc, s, row[d]);
    return acc;
}

// ---------------------------------------------------------------------------
// Loaders: ld(k, a1, a2, a3) = component k of node c + a - (I/2 - 1)
// ---------------------------------------------------------------------------
template <typename T, int S2_, int S3_, int SC_>
struct SmemLd {
    static constexpr int S2 = S2_, S3 = S3_, SC = SC_;
    static constexpr bool kShared = true, kNode4 = false;
    const T* base;
    __device__ __forceinline__ T operator()(int k, int a1, int a2, int a3) const
    {
        return base[k * SC + a3 * S3 + a2 * S2 + a1];
    }
};

template <typename T, int STORE>
__device__ __forceinline__ T fetch(const FieldView& f, int k, int64_t idx)
{
    const int64_t o = (int64_t)k * f.plane + idx;
    if constexpr (STORE == ST_F64) return (T)__ldg(f.f64 + o);
    else if constexpr (STORE == ST_F32) return (T)__ldg(f.f32 + o);
    else return (T)(__bfloat162float(f.hi[o]) + __bfloat162float(f.lo[o]));
}

// Global-memory loader (stencils outside a staged halo, and the direct path).
// The cell c lies in [0, N) and a stencil node is at most I/2 <= PAD cells
// from it, so every node is inside the ghost-padded array: no periodic wrap,
// and each node is a fixed offset from the stencil's first node.
template <typename T, int STORE, int I>
struct GlobalLd {
    static constexpr bool kShared = false, kNode4 = false;
    FieldView f;
    int base;            // padded index of node (c1, c2, c3) - (I/2 - 1) within a component
    int k0, kmax;        // component k reads min(k0 + k, kmax)
    __device__ __forceinline__ T operator()(int k, int a1, int a2, int a3) const
    {
        // a padded component holds (N + 2 PAD)^3 < 2^31 nodes for N <= 1024: 32-bit offsets
        const int NP = f.NP;
        return fetch<T, STORE>(f, min(k0 + k, kmax), (int64_t)(base + (a3 * NP + a2) * NP + a1));
    }
};

// Global-memory loader from the node-major float32 copy (the direct path): the
// C components of a node are adjacent, so a stencil row of I nodes is I*C*4
// contiguous bytes instead of C separate runs of I*4 bytes, which roughly
// halves the DRAM sectors a sparse particle's stencil costs.
template <typename T, int I>
struct NodeLd {
    static constexpr bool kShared = false, kNode4 = false;
    const float* nm;
    int base;            // padded index of node (c1, c2, c3) - (I/2 - 1)
    int NP, nmc, k0, kmax;
    __device__ __forceinline__ T operator()(int k, int a1, int a2, int a3) const
    {
        const int node = base + (a3 * NP + a2) * NP + a1;
        return (T)__ldg(nm + (int64_t)node * nmc + min(k0 + k, kmax));
    }
};

// The three velocity components of a node as one aligned 16-byte load from the
// padded node-major copy (float32: nmc = 4; split-bf16: the three hi/lo pairs,
// each value formed as float(hi) + float(lo) as in fetch()).  Where the copy
// has a texture object the load is a texture fetch (element type, no
// filtering: the same bits), on the texture data path; the loads a caller
// marks plain (a few of the stencil rows) stay on the load/store
// data path, so that the two paths, which the gathers otherwise saturate one
// at a time, share the stencil.
template <int I, int STORE, bool TEX = false>
struct NodeLd4 {
    static constexpr bool kShared = false, kNode4 = true;
    const void* nm;             // the node-major copy
    int base, NP;
    unsigned long long tex;     // texture fetches: the texture object over nm
    // plain: a compile-time constant once the caller's loops are unrolled
    __device__ __forceinline__ float4 node(int a1, int a2, int a3, bool plain = false) const
    {
        const int i = base + (a3 * NP + a2) * NP + a1;
        if constexpr (STORE == ST_F32) {
            if (TEX && !plain) return tex1Dfetch<float4>((cudaTextureObject_t)tex, i);
            return __ldg(reinterpret_cast<const float4*>(nm) + i);
        } else {
            const uint4 w = TEX && !plain ? tex1Dfetch<uint4>((cudaTextureObject_t)tex, i)
                                          : __ldg(reinterpret_cast<const uint4*>(nm) + i);
            auto val = [](uint32_t x) {
                return __bfloat162float(__ushort_as_bfloat16((unsigned short)(x & 0xffffu))) +
                       __bfloat162float(__ushort_as_bfloat16((unsigned short)(x >> 16)));
            };
            return make_float4(val(w.x), val(w.y), val(w.z), 0.0f);
        }
    }
};

// c1, c2, c3 in [0, N)
template <typename T, int STORE, int I>
__device__ __forceinline__ GlobalLd<T, STORE, I> global_ld(const FieldView& f, int c1, int c2, int c3, int k0,
                                                           int kmax)
{
    constexpr int LO = I / 2 - 1;
    return GlobalLd<T, STORE, I>{f, (int)padded_index(f.NP, c1 - LO, c2 - LO, c3 - LO), k0, kmax};
}

// ---------------------------------------------------------------------------
// 1-D weights, once per particle and axis: lane l < 3I evaluates
// beta_i(s_a) (a = l / I, i = l % I) by Horner's rule and stores it in the
// warp's weight buffer wv[3][8] (and beta' in wd[3][8] when D); the lanes then
// read the weights they need.
// ---------------------------------------------------------------------------
template <typename T, int I, int DEG, bool D>
struct WeightEval {
    Row<T, DEG> r, dr;
    int ax, i;
    bool act;
    __device__ void init(const CoefTable<T>& tb, int lane)
    {
        act = lane < 3 * I;
        ax = act ? lane / I : 0;
        i = act ? lane % I : 0;
        r = load_row<T, DEG>(tb.c, i);
        if (D) dr = load_row<T, DEG>(tb.d, i);
    }
    __device__ __forceinline__ void eval(T s1, T s2, T s3, T* wv, T* wd) const
    {
        // every lane evaluates (idle lanes on a valid row) and only active lanes store
        const T s = ax == 0 ? s1 : (ax == 1 ? s2 : s3);
        const T w = horner(r, s);
        T dw = 0;
        if (D) dw = horner(dr, s);
        __syncwarp();                        // previous readers of the buffer are done
        if (act) wv[ax * 8 + i] = w;
        if (D && act) wd[ax * 8 + i] = dw;
        __syncwarp();
    }
    // value weights (no derivatives) of two points a and b into wva and wvb
    __device__ __forceinline__ void eval_values2(const T (&sa)[3], const T (&sb)[3], T* wva, T* wvb) const
    {
        const T xa = ax == 0 ? sa[0] : (ax == 1 ? sa[1] : sa[2]);
        const T xb = ax == 0 ? sb[0] : (ax == 1 ? sb[1] : sb[2]);
        const T wa = horner(r, xa), wb = horner(r, xb);
        __syncwarp();
        if (act) {
            wva[ax * 8 + i] = wa;
            wvb[ax * 8 + i] = wb;
        }
        __syncwarp();
    }
};

// ---------------------------------------------------------------------------
// Per-lane stencil registers and contraction, one specialisation per I.
//   acc[k] = u_k partial; with D also acc[3 + 3k + j] = d u_k / d t_j partial.
// Idle lanes read a duplicate of an active lane's address (a broadcast, not a
// bank conflict) and carry zero weights.
// ---------------------------------------------------------------------------
// n consecutive weights of a warp's buffer (the same for every lane) by
// 16-byte broadcast loads: p is 16-byte aligned (the weight buffers are
// 32-byte aligned and every run starts at a multiple of 16 bytes)
template <int n, typename T>
__device__ __forceinline__ void bcast_load(const T* p, T (&w)[n])
{
    static_assert(n % 2 == 0, "runs of even length");
    if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int i = 0; i + 4 <= n; i += 4) {
            const float4 v = *reinterpret_cast<const float4*>(p + i);
            w[i] = v.x;
            w[i + 1] = v.y;
            w[i + 2] = v.z;
            w[i + 3] = v.w;
        }
        if constexpr (n % 4 == 2) {
            const float2 v = *reinterpret_cast<const float2*>(p + n - 2);
            w[n - 2] = v.x;
            w[n - 1] = v.y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < n; i += 2) {
            const double2 v = *reinterpret_cast<const double2*>(p + i);
            w[i] = v.x;
            w[i + 1] = v.y;
        }
    }
}

template <typename T, int I, bool D>
struct Lane;

template <typename T, bool D>
struct Lane<T, 8, D> {
    int i1, j;
    T f[3][2][8];
    __device__ void init(int lane)
    {
        i1 = lane & 7;
        j = lane >> 3;
    }
    template <class LD>
    __device__ __forceinline__ void load(const LD& ld)
    {
        if constexpr (LD::kShared) {
            // one lane pointer, then compile-time offsets
            const T* pa = ld.base + (i1 + j * LD::S2);
#pragma unroll
            for (int k = 0; k < 3; ++k)
#pragma unroll
                for (int h = 0; h < 2; ++h)
#pragma unroll
                    for (int i3 = 0; i3 < 8; ++i3) f[k][h][i3] = pa[k * LD::SC + 4 * h * LD::S2 + i3 * LD::S3];
        } else if constexpr (LD::kNode4) {
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int i3 = 0; i3 < 8; ++i3) {
                    const float4 v = ld.node(i1, j + 4 * h, i3, (i3 & 3) == 1);   // rows i3 = 1, 5 plain
                    f[0][h][i3] = v.x;
                    f[1][h][i3] = v.y;
                    f[2][h][i3] = v.z;
                }
        } else {
#pragma unroll
            for (int k = 0; k < 3; ++k)
#pragma unroll
                for (int h = 0; h < 2; ++h)
#pragma unroll
                    for (int i3 = 0; i3 < 8; ++i3) f[k][h][i3] = ld(k, i1, j + 4 * h, i3);
        }
    }
    // transpose of the gather: add w(node) mu_k into every node this lane
    // gathers; TWO adds wa(node) ma_k + wb(node) mb_k (two weight sets on the
    // same stencil) with one add per node
    template <bool TWO, class ADD>
    __device__ __forceinline__ void scatter_n(const T* wa, const T (&ma)[3], const T* wb, const T (&mb)[3],
                                              const ADD& add) const
    {
        const T w1a = wa[i1], w1b = TWO ? wb[i1] : (T)0;
        T w3a[8], w3b[8];
        bcast_load(wa + 16, w3a);
        if (TWO) bcast_load(wb + 16, w3b);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const T a12a = w1a * wa[8 + j + 4 * h];
            const T a12b = TWO ? w1b * wb[8 + j + 4 * h] : (T)0;
#pragma unroll
            for (int i3 = 0; i3 < 8; ++i3) {
                const T wA = a12a * w3a[i3];
                const T wB = TWO ? a12b * w3b[i3] : (T)0;
#pragma unroll
                for (int k = 0; k < 3; ++k) add(k, i1, j + 4 * h, i3, TWO ? fma(wA, ma[k], wB * mb[k]) : wA * ma[k]);
            }
        }
    }
    __device__ __forceinline__ void contract(const T* wv, const T* wd, T (&acc)[12]) const
    {
        T w3[8], dw3[8];
        bcast_load(wv + 16, w3);
        if (D) bcast_load(wd + 16, dw3);
        const T w1 = wv[i1];
        const T w2[2] = {wv[8 + j], wv[12 + j]};
        T dw1 = 0, dw2[2] = {0, 0};
        if (D) {
            dw1 = wd[i1];
            dw2[0] = wd[8 + j];
            dw2[1] = wd[12 + j];
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            T v = 0, d1 = 0, d2 = 0, d3 = 0;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                T pv = 0, pd = 0;
#pragma unroll
                for (int i3 = 0; i3 < 8; ++i3) {
                    pv = fma(w3[i3], f[k][h][i3], pv);
                    if (D) pd = fma(dw3[i3], f[k][h][i3], pd);
                }
                v = fma(w1 * w2[h], pv, v);
                if (D) {
                    d1 = fma(dw1 * w2[h], pv, d1);
                    d2 = fma(w1 * dw2[h], pv, d2);
                    d3 = fma(w1 * w2[h], pd, d3);
                }
            }
            acc[k] = v;
            if (D) {
                acc[3 + 3 * k + 0] = d1;
                acc[3 + 3 * k + 1] = d2;
                acc[3 + 3 * k + 2] = d3;
            }
        }
    }
};

template <typename T, bool D>
struct Lane<T, 6, D> {
    int i1, j;
    bool act, actc;
    T f[3][8];                               // pass A (6), pass B, pass C
    __device__ void init(int lane)
    {
        act = lane < 30;
        actc = lane < 6;
        i1 = lane % 6;                       // lanes 30, 31 duplicate lanes 0, 1
        j = act ? lane / 6 : 0;
    }
    template <class LD>
    __device__ __forceinline__ void load(const LD& ld)
    {
        if constexpr (LD::kShared) {
            const T* pa = ld.base + (i1 + j * LD::S2);                  // pass A: row (i1, j)
            const T* pb = ld.base + (i1 + 5 * LD::S2 + j * LD::S3);     // pass B: node (i1, 5, j)
            const T* pc = ld.base + (i1 + 5 * LD::S2 + 5 * LD::S3);     // pass C: node (i1, 5, 5)
#pragma unroll
            for (int k = 0; k < 3; ++k) {
#pragma unroll
                for (int i3 = 0; i3 < 6; ++i3) f[k][i3] = pa[k * LD::SC + i3 * LD::S3];
                f[k][6] = pb[k * LD::SC];
                f[k][7] = pc[k * LD::SC];
            }
        } else if constexpr (LD::kNode4) {
#pragma unroll
            for (int i3 = 0; i3 < 8; ++i3) {
                // pass A: row (i1, j) at i3 < 6; pass B: node (i1, 5, j); pass C: node (i1, 5, 5);
                // pass B plain (5 of the 36 stencil rows; measured on GB300 at 256^3 and 1/16
                // per cell: 0.415 ms per RK2 step, 0.421 with pass A at i3 = 2 plain too,
                // 0.435 with no plain rows, 0.445 with three plain rows of pass A)
                const float4 v = i3 < 6 ? ld.node(i1, j, i3)
                                        : (i3 == 6 ? ld.node(i1, 5, j, true) : ld.node(i1, 5, 5));
                f[0][i3] = v.x;
                f[1][i3] = v.y;
                f[2][i3] = v.z;
            }
        } else {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
#pragma unroll
                for (int i3 = 0; i3 < 6; ++i3) f[k][i3] = ld(k, i1, j, i3);
                f[k][6] = ld(k, i1, 5, j);
                f[k][7] = ld(k, i1, 5, 5);
            }
        }
    }
    template <bool TWO, class ADD>
    __device__ __forceinline__ void scatter_n(const T* wa, const T (&ma)[3], const T* wb, const T (&mb)[3],
                                              const ADD& add) const
    {
        auto val = [&](T wA, T wB, int k) { return TWO ? fma(wA, ma[k], wB * mb[k]) : wA * ma[k]; };
        const T w1a = wa[i1], w25a = wa[13];
        const T w1b = TWO ? wb[i1] : (T)0, w25b = TWO ? wb[13] : (T)0;
        T w3a[6], w3b[6];
        bcast_load(wa + 16, w3a);
        if (TWO) bcast_load(wb + 16, w3b);
        if (act) {
            const T a12a = w1a * wa[8 + j], a12b = TWO ? w1b * wb[8 + j] : (T)0;
#pragma unroll
            for (int i3 = 0; i3 < 6; ++i3) {
                const T wA = a12a * w3a[i3], wB = TWO ? a12b * w3b[i3] : (T)0;
#pragma unroll
                for (int k = 0; k < 3; ++k) add(k, i1, j, i3, val(wA, wB, k));
            }
            const T wA = w1a * w25a * wa[16 + j], wB = TWO ? w1b * w25b * wb[16 + j] : (T)0;
#pragma unroll
            for (int k = 0; k < 3; ++k) add(k, i1, 5, j, val(wA, wB, k));
        }
        if (actc) {
            const T wA = w1a * w25a * w3a[5], wB = TWO ? w1b * w25b * w3b[5] : (T)0;
#pragma unroll
            for (int k = 0; k < 3; ++k) add(k, i1, 5, 5, val(wA, wB, k));
        }
    }
    __device__ __forceinline__ void contract(const T* wv, const T* wd, T (&acc)[12]) const
    {
        T w3[6], dw3[6];
        bcast_load(wv + 16, w3);
        if (D) bcast_load(wd + 16, dw3);
        const T w1 = wv[i1], w2j = wv[8 + j], w3j = wv[16 + j], w25 = wv[13];
        const T z = 0;
        // coefficients of the three passes (zero on idle lanes)
        const T aA = act ? w1 * w2j : z;
        const T aB = act ? w1 * w25 * w3j : z;
        const T aC = actc ? w1 * w25 * w3[5] : z;
        T dw1 = 0, dw2j = 0, dw3j = 0, dw25 = 0;
        if (D) {
            dw1 = wd[i1];
            dw2j = wd[8 + j];
            dw3j = wd[16 + j];
            dw25 = wd[13];
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            T pv = 0, pd = 0;
#pragma unroll
            for (int i3 = 0; i3 < 6; ++i3) {
                pv = fma(w3[i3], f[k][i3], pv);
                if (D) pd = fma(dw3[i3], f[k][i3], pd);
            }
            acc[k] = fma(aA, pv, fma(aB, f[k][6], aC * f[k][7]));
            if (D) {
                const T b1 = act ? dw1 * w2j : z, b2 = act ? w1 * dw2j : z;
                const T c1 = act ? dw1 * w25 * w3j : z, c2 = act ? w1 * dw25 * w3j : z, c3 = act ? w1 * w25 * dw3j : z;
                const T e1 = actc ? dw1 * w25 * w3[5] : z, e2 = actc ? w1 * dw25 * w3[5] : z;
                const T e3 = actc ? w1 * w25 * dw3[5] : z;
                acc[3 + 3 * k + 0] = fma(b1, pv, fma(c1, f[k][6], e1 * f[k][7]));
                acc[3 + 3 * k + 1] = fma(b2, pv, fma(c2, f[k][6], e2 * f[k][7]));
                acc[3 + 3 * k + 2] = fma(aA, pd, fma(c3, f[k][6], e3 * f[k][7]));
            }
        }
    }
};

template <typename T, bool D>
struct Lane<T, 4, D> {
    int i1, i2, p;
    T f[3][2];
    __device__ void init(int lane)
    {
        i1 = lane & 3;
        i2 = (lane >> 2) & 3;
        p = lane >> 4;
    }
    template <class LD>
    __device__ __forceinline__ void load(const LD& ld)
    {
        if constexpr (LD::kShared) {
            const T* pa = ld.base + (i1 + i2 * LD::S2 + p * LD::S3);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                f[k][0] = pa[k * LD::SC];
                f[k][1] = pa[k * LD::SC + 2 * LD::S3];
            }
        } else if constexpr (LD::kNode4) {
            const float4 a = ld.node(i1, i2, p), b = ld.node(i1, i2, p + 2);
            f[0][0] = a.x;
            f[1][0] = a.y;
            f[2][0] = a.z;
            f[0][1] = b.x;
            f[1][1] = b.y;
            f[2][1] = b.z;
        } else {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                f[k][0] = ld(k, i1, i2, p);
                f[k][1] = ld(k, i1, i2, p + 2);
            }
        }
    }
    template <bool TWO, class ADD>
    __device__ __forceinline__ void scatter_n(const T* wa, const T (&ma)[3], const T* wb, const T (&mb)[3],
                                              const ADD& add) const
    {
        auto val = [&](T wA, T wB, int k) { return TWO ? fma(wA, ma[k], wB * mb[k]) : wA * ma[k]; };
        const T a12a = wa[i1] * wa[8 + i2], a12b = TWO ? wb[i1] * wb[8 + i2] : (T)0;
        const T w0a = a12a * wa[16 + p], w1a = a12a * wa[18 + p];
        const T w0b = TWO ? a12b * wb[16 + p] : (T)0, w1b = TWO ? a12b * wb[18 + p] : (T)0;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            add(k, i1, i2, p, val(w0a, w0b, k));
            add(k, i1, i2, p + 2, val(w1a, w1b, k));
        }
    }
    __device__ __forceinline__ void contract(const T* wv, const T* wd, T (&acc)[12]) const
    {
        const T w1 = wv[i1], w2 = wv[8 + i2];
        const T w3a = wv[16 + p], w3b = wv[18 + p];
        T dw1 = 0, dw2 = 0, dw3a = 0, dw3b = 0;
        if (D) {
            dw1 = wd[i1];
            dw2 = wd[8 + i2];
            dw3a = wd[16 + p];
            dw3b = wd[18 + p];
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const T pv = fma(w3a, f[k][0], w3b * f[k][1]);
            acc[k] = w1 * w2 * pv;
            if (D) {
                const T pd = fma(dw3a, f[k][0], dw3b * f[k][1]);
                acc[3 + 3 * k + 0] = dw1 * w2 * pv;
                acc[3 + 3 * k + 1] = w1 * dw2 * pv;
                acc[3 + 3 * k + 2] = w1 * w2 * pd;
            }
        }
    }
};

// ---------------------------------------------------------------------------
// Warp reductions.  reduce4: three values (padded to four) summed over the 32
// lanes in 6 shuffles; lane l ends with value 2*bit4(l) + bit3(l).
// reduce16: twelve values (padded to 16) in 16 shuffles; lane l ends with
// value 8*bit4 + 4*bit3 + 2*bit2 + bit1.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T xor_shfl(T v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }

template <typename T>
__device__ __forceinline__ T reduce4(const T (&acc)[12], int lane)
{
    const bool b4 = lane & 16, b3 = lane & 8;
    const T z = 0;
    // level 16: keep values (0,1) or (2,3)
    T k0 = b4 ? acc[2] : acc[0];
    T k1 = b4 ? z : acc[1];
    k0 += xor_shfl(b4 ? acc[0] : acc[2], 16);
    k1 += xor_shfl(b4 ? acc[1] : z, 16);
    // level 8: keep one value, then a full reduction of it
    T m = b3 ? k1 : k0;
    m += xor_shfl(b3 ? k0 : k1, 8);
    m += xor_shfl(m, 4);
    m += xor_shfl(m, 2);
    m += xor_shfl(m, 1);
    return m;
}

template <typename T>
__device__ __forceinline__ T reduce16(const T (&acc)[12], int lane)
{
    T v[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = i < 12 ? acc[i] : (T)0;
#pragma unroll
    for (int lev = 0; lev < 4; ++lev) {
        const int off = 16 >> lev;
        const int half = 8 >> lev;
        const bool hi = lane & off;
#pragma unroll
        for (int i = 0; i < half; ++i) {
            const T send = hi ? v[i] : v[i + half];
            const T keep = hi ? v[i + half] : v[i];
            v[i] = keep + xor_shfl(send, off);
        }
    }
    v[0] += xor_shfl(v[0], 1);
    return v[0];
}

// ---------------------------------------------------------------------------
// Halo staging: 16-byte vector loads of the ghost-padded field rows.
// ---------------------------------------------------------------------------
template <int STORE>
struct VecOf {
    static constexpr int n = STORE == ST_F64 ? 2 : (STORE == ST_F32 ? 4 : 8);
};

template <typename T, int STORE, int VEC>
__device__ __forceinline__ void load_vec(const FieldView& f, int64_t g, T (&vals)[VEC])
{
    if constexpr (STORE == ST_F32) {
        const float4 w = __ldg(reinterpret_cast<const float4*>(f.f32 + g));
        vals[0] = w.x;
        vals[1] = w.y;
        vals[2] = w.z;
        vals[3] = w.w;
    } else if constexpr (STORE == ST_F64) {
        const double2 w = __ldg(reinterpret_cast<const double2*>(f.f64 + g));
        vals[0] = (T)w.x;
        vals[1] = (T)w.y;
    } else {
        const uint4 hv = __ldg(reinterpret_cast<const uint4*>(f.hi + g));
        const uint4 lv = __ldg(reinterpret_cast<const uint4*>(f.lo + g));
        const uint32_t hw[4] = {hv.x, hv.y, hv.z, hv.w}, lw[4] = {lv.x, lv.y, lv.z, lv.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            vals[2 * e] = (T)(__uint_as_float(hw[e] << 16) + __uint_as_float(lw[e] << 16));
            vals[2 * e + 1] = (T)(__uint_as_float(hw[e] & 0xffff0000u) + __uint_as_float(lw[e] & 0xffff0000u));
        }
    }
}

// The halo is kc * H planes (component k, z) of H rows of NV 16-byte vectors.
// Thread t owns one (row y, vector v) slot of one of PPI planes per iteration;
// that slot, its global/shared offsets inside a plane and its edge predicates
// are fixed for the whole loop, and only the plane index advances (one
// division by the constant H per iteration).  Iterations are batched UNR deep
// so their loads are in flight together.  KC > 0: compile-time component
// count; KC = 0: runtime count kc.
template <typename T, int STORE, int H, int G, int S2, int S3, int SC, int KC>
__device__ __forceinline__ void load_halo(T* halo, const FieldView& f, int k0, int kc, int o1, int o2, int o3)
{
    constexpr int VEC = VecOf<STORE>::n;
    constexpr int OFF = ((PAD - G) % VEC + VEC) % VEC;   // block origins are multiples of 8
    constexpr int NV = (OFF + H + VEC - 1) / VEC;        // vectors per halo row
    constexpr int SLOTS = H * NV;                        // vector slots per plane
    constexpr int PPI = NT / SLOTS;                      // planes per iteration
    static_assert(PPI >= 1, "a halo plane needs more vector slots than threads");
    constexpr int UNR = 4;
    const int nplanes = (KC > 0 ? KC : kc) * H;
    const int NP = f.NP;
    const int64_t NP2 = (int64_t)NP * NP;
    const int pslot = threadIdx.x / SLOTS;
    const int q = threadIdx.x - pslot * SLOTS;
    const int y = q / NV, v = q - (q / NV) * NV;
    if (pslot >= PPI) return;                            // idle threads of the last partial plane group
    const int64_t gslot = (int64_t)k0 * f.plane + (int64_t)(o3 + PAD) * NP2 + (int64_t)(o2 + PAD + y) * NP +
                          (o1 + PAD - OFF) + v * VEC;
    const int sslot = y * S2 + v * VEC - OFF;
    bool ok[VEC];
#pragma unroll
    for (int e = 0; e < VEC; ++e) ok[e] = v * VEC + e - OFF >= 0 && v * VEC + e - OFF < H;
    for (int p0 = pslot; p0 < nplanes; p0 += UNR * PPI) {
        T vals[UNR][VEC];
        int soff[UNR];
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
            const int p = p0 + u * PPI;
            const int k = p / H, z = p - (p / H) * H;
            soff[u] = k * SC + z * S3 + sslot;
            if (p < nplanes) load_vec<T, STORE, VEC>(f, gslot + (int64_t)k * f.plane + (int64_t)z * NP2, vals[u]);
        }
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
            if (p0 + u * PPI < nplanes) {
#pragma unroll
                for (int e = 0; e < VEC; ++e)
                    if (ok[e]) halo[soff[u] + e] = vals[u][e];
            }
        }
    }
}

// cp.async copies of one 4- or 8-byte element, global -> shared (cached in L1,
// which the overlapping halos of neighbouring blocks re-use).
template <typename T>
__device__ __forceinline__ void cp_async_elem(uint32_t dst, const T* src)
{
    if constexpr (sizeof(T) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(dst), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(dst), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Asynchronous halo staging for float32 / float64 storage (the shared-memory
// element type equals the stored type).  Every element is copied global ->
// shared by cp.async, so nothing passes through registers and the thread is
// free for other work while the copies land.  Lanes run along x1: thread t
// copies column x = t mod H of rows t / H + r * RP (RP = NT / H rows per pass),
// so a warp's copies cover about two contiguous rows.  Components k0 .. k0+kc-1
// (KC > 0: compile-time count).  The caller completes the copies with
// cp_async_wait_all() before the barrier that publishes the halo.
template <typename T, int STORE, int H, int S2, int S3, int SC, int KC>
__device__ __forceinline__ void load_halo_async(T* halo, const FieldView& f, int k0, int kc, int x0, int y0, int z0)
{
    static_assert(STORE == ST_F32 || STORE == ST_F64, "split-bf16 halos are converted through registers");
    static_assert(sizeof(T) == (STORE == ST_F64 ? 8 : 4), "element type must equal the stored type");
    constexpr int RP = NT / H;                           // rows per pass
    constexpr int NPASS = (H + RP - 1) / RP;
    static_assert(RP >= 1, "halo row longer than the thread count");
    const int x = threadIdx.x % H, yr = threadIdx.x / H;
    if (yr >= (RP < H ? RP : H)) return;
    const T* gbase;
    if constexpr (STORE == ST_F64) gbase = f.f64;
    else gbase = f.f32;
    const int64_t NP2 = (int64_t)f.NP * f.NP;
    const T* g = gbase + (int64_t)k0 * f.plane + (int64_t)z0 * NP2 + (int64_t)(y0 + yr) * f.NP + (x0 + x);
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(halo) + (uint32_t)((yr * S2 + x) * (int)sizeof(T));
    // one pass row at a time; the plane loop walks a pointer (unrolling it
    // whole would hoist every plane's address into registers)
#pragma unroll
    for (int k = 0; k < (KC > 0 ? KC : 3); ++k) {
        if (KC == 0 && k >= kc) break;
#pragma unroll
        for (int r = 0; r < NPASS; ++r) {
            if (NPASS > 1 && yr + r * RP >= H) break;
            const T* gz = g + (int64_t)k * f.plane + (int64_t)(r * RP) * f.NP;
            uint32_t sz = s + (uint32_t)((k * SC + r * RP * S2) * (int)sizeof(T));
#pragma unroll 5
            for (int z = 0; z < H; ++z) {
                cp_async_elem<T>(sz, gz);
                gz += NP2;
                sz += S3 * (int)sizeof(T);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Tensor-memory-accelerator halo staging (HC_TMA): one cp.async.bulk.tensor
// copy per component chunk, issued by one thread, completion counted in bytes
// on an mbarrier that every thread waits on.  The tensor map covers the
// padded field [C][NP][NP][NP] (4-D, x1 innermost) with the box of tma_box.
// ---------------------------------------------------------------------------
enum { HC_ASYNC = 0, HC_TMA = 1 };

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

// one thread: announce `bytes` for the barrier's current phase and start the copy of
// the box at tensor coordinates (x, y, z, k) into dst
__device__ __forceinline__ void tma_issue(void* dst, const CUtensorMap* map, int x, int y, int z, int k, uint64_t* bar,
                                          uint32_t bytes)
{
    // shared-memory reads of the previous halo (generic proxy) are ordered
    // before the copy's writes (async proxy)
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];\n" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(k), "r"(smem_addr(bar))
        : "memory");
}

// Waits for the barrier's phase `parity` to complete; false after the
// iteration limit (each try_wait itself suspends for a bounded time), so a
// copy that never lands cannot hang the kernel.
constexpr int kTmaWaitLimit = 1 << 22;
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity)
{
    const uint32_t a = smem_addr(bar);
    for (int it = 0; it < kTmaWaitLimit; ++it) {
        uint32_t done = 0;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Stage components k0 .. k0+kc-1 (KC > 0: compile-time count) of the halo
// whose origin is the cell (o1, o2, o3): cp.async for float32 / float64
// storage, registers (with the bf16 hi + lo sum) for split bf16.  With
// WAIT = false the float32 / float64 copies may still be in flight on return.
template <typename T, int STORE, int H, int G, int S2, int S3, int SC, int KC, bool WAIT>
__device__ __forceinline__ void stage_halo(T* halo, const FieldView& f, int k0, int kc, int o1, int o2, int o3)
{
    if constexpr (STORE == ST_BF16X2) {
        load_halo<T, STORE, H, G, S2, S3, SC, KC>(halo, f, k0, kc, o1, o2, o3);
    } else {
        load_halo_async<T, STORE, H, S2, S3, SC, KC>(halo, f, k0, kc, o1 + PAD, o2 + PAD, o3 + PAD);
        if (WAIT) cp_async_wait_all();
    }
}

__device__ __forceinline__ int pack_rel(int r1, int r2, int r3) { return r1 | (r2 << 8) | (r3 << 16); }
__device__ __forceinline__ int pack_cell(int c1, int c2, int c3) { return c1 | (c2 << 10) | (c3 << 20); }

// Per-particle record written in P1 and read (broadcast) by the Q warps.
template <typename T>
struct alignas(4 * sizeof(T)) PRec {
    T t[3];         // offsets in the cell (Sec. 2.2 step 3, normalised by delta)
    T relf;         // packed relative cell (pack_rel), bit-cast into T's storage
};

// Byte offsets of the shared-memory regions, each 32-byte aligned (the
// particle records are read and written as 16- or 32-byte vectors).
constexpr size_t align32(size_t x) { return (x + 31) & ~size_t(31); }

// STAGE: what P1 keeps for later phases besides the records: 0 = caller ids
// (outputs in caller order), 1 = ids + float64 positions (RK2 update),
// 2 = ids + positions + the AB history (up to AB_MAX_HIST entries of 3).
template <typename T, int SC, int STAGE>
struct SmemPlan {
    static constexpr size_t rec = align32((size_t)3 * SC * sizeof(T));
    static constexpr size_t k = align32(rec + PB * sizeof(PRec<T>));
    static constexpr size_t w = align32(k + (STAGE >= 1 ? (size_t)6 * PB * sizeof(T) : 0));   // k values: steps only
    static constexpr size_t cell = align32(w + (size_t)NW * 48 * sizeof(T));
    static constexpr size_t id = align32(cell + PB * sizeof(int));
    static constexpr size_t x = align32(id + PB * sizeof(int));
    static constexpr size_t rhs = align32(x + (STAGE >= 1 ? (size_t)3 * PB * sizeof(double) : 0));
    static constexpr size_t mbar = align32(rhs + (STAGE >= 2 ? (size_t)3 * AB_MAX_HIST * PB * sizeof(float) : 0));
    static constexpr size_t total = mbar + 16;   // the halo copy's mbarrier (tensor-copy staging)
};

template <int MODE>
__host__ __device__ constexpr int stage_of()
{
    return MODE == MODE_RK2 ? 1 : ((MODE == MODE_AB2 || MODE == MODE_AB2_D) ? 2 : 0);
}

// ---------------------------------------------------------------------------
// The block kernel.
// ---------------------------------------------------------------------------
// Processes the sorted particles [j0, j1) of cell block b.  HALO = false skips
// the halo staging and gathers every stencil from global memory (the direct
// path for sparse particle sets, where a halo would serve one or two
// particles); its shared-memory plan has no halo region and b is unused.
// NM (with HALO = false, float32 storage): the gathers read the node-major
// copy a.f.nm, as one 16-byte load per node when NM == NM_VEC4 (three
// components padded to four floats), else per component (NM_SCALAR).  Must be
// called by all threads of the CTA.
// HC (with HALO): HC_ASYNC stages the halo with cp.async element copies (or
// through registers for split bf16); HC_TMA with one tensor copy per chunk
// through tmap (float32 and float64 storage), in the padded box of tma_box.
template <typename T, int I, int DEG, int MODE, int STORE, bool HALO, int NM = NM_NONE, int HC = HC_ASYNC>
__device__ __forceinline__ void process_block(const BlockArgs& a, int b, int j0, int j1, unsigned char* smem_raw,
                                              const CUtensorMap* tmap = nullptr)
{
    constexpr bool IS_AB2 = (MODE == MODE_AB2 || MODE == MODE_AB2_D);
    constexpr bool IS_STEP = (MODE == MODE_RK2 || IS_AB2);
    constexpr bool D = (MODE == MODE_INTERP_DERIV || MODE == MODE_AB2_D);
    constexpr int MARGIN = (MODE == MODE_RK2) ? 1 : 0;     // halo margin for the stage-2 point
    constexpr int H = BLK + I - 1 + 2 * MARGIN;
    constexpr int G = I / 2 - 1 + MARGIN;                   // halo origin = block origin - G
    constexpr int LO = I / 2 - 1;                           // stencil node offset
    constexpr int RMAX = H - 1 - I / 2;                     // largest cell whose stencil fits the halo
    constexpr bool TMA = HALO && HC == HC_TMA;
    static_assert(!TMA || STORE == ST_F32 || STORE == ST_F64, "tensor-copy halos: float32 or float64 storage");
    constexpr TmaBox TB = tma_box(I, MARGIN, (int)sizeof(T));
    using Lay = Layout<I, H>;
    constexpr int S2 = TMA ? TB.S2() : Lay::S2, S3 = TMA ? TB.S3() : Lay::S3, SC = TMA ? TB.SC() : Lay::SC;
    constexpr int XOFF = TMA ? TB.XOFF : 0;   // the box starts XOFF elements before the halo in x1
    using SL = SmemLd<T, S2, S3, SC>;

    using SM = SmemPlan<T, HALO ? SC : 0, stage_of<MODE>()>;
    T* halo = reinterpret_cast<T*>(smem_raw);                               // [3][SC] (HALO only)
    PRec<T>* p_rec = reinterpret_cast<PRec<T>*>(smem_raw + SM::rec);        // [PB]
    T* p_k = reinterpret_cast<T*>(smem_raw + SM::k);                        // [6][PB]: k1 (3), k2 (3)
    T* wbuf = reinterpret_cast<T*>(smem_raw + SM::w);                       // [NW][2][24] weights
    int* p_cell = reinterpret_cast<int*>(smem_raw + SM::cell);              // [PB]
    int* p_id = reinterpret_cast<int*>(smem_raw + SM::id);                  // [PB] caller ids
    double* p_x = reinterpret_cast<double*>(smem_raw + SM::x);              // [3][PB] positions (steps)
    float* p_rhs = reinterpret_cast<float*>(smem_raw + SM::rhs);            // [3 * (k-1)][PB] AB history
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem_raw + SM::mbar);      // halo copy barrier (TMA)

    if (j0 >= j1) return;

    const int mask = a.g.mask;
    const int nb1 = a.g.nb1, nb2 = a.g.nb2;
    const int bx = b % nb1, by = (b / nb1) % nb2, bz = b / (nb1 * nb2);
    const int o1 = bx * BLK - G, o2 = by * BLK - G, o3 = bz * BLK - G;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t np = a.np;
    const double inv_delta = a.g.inv_delta;
    T* wv = wbuf + warp * 48;
    T* wd = wv + 24;

    WeightEval<T, I, DEG, D> W;
    W.init(table<T>(a), lane);
    Lane<T, I, D> L;
    L.init(lane);

    const int nchunks = IS_STEP ? 1 : (a.f.C + 2) / 3;
    const T dtid = (T)(a.dt * inv_delta);
    const int rcomp = ((lane & 16) ? 2 : 0) + ((lane & 8) ? 1 : 0);   // component held after reduce4
    const bool writer = (lane & 7) == 0 && rcomp < 3;                 // lanes 0, 8, 16

    // a stencil from global memory at cell (c1, c2, c3) in [0, N)^3, components k0 + k (clamped to kmax)
    static_assert(NM == NM_NONE || (!HALO && (STORE == ST_F32 || (STORE == ST_BF16X2 && NM >= NM_VEC4))),
                  "node-major gathers: direct path, float32 or (three components) split-bf16 storage");
    auto gload = [&](int c1, int c2, int c3, int k0, int kmax) {
        const int base = (int)padded_index(a.f.NP, c1 - LO, c2 - LO, c3 - LO);
        if constexpr (NM == NM_TEX4)   // three components, one 16-byte texel per node
            L.load(NodeLd4<I, STORE, true>{a.f.nm, base, a.f.NP, a.f.nm_tex});
        else if constexpr (NM == NM_VEC4)   // three components, 16 bytes per node (split bf16: chunk k0 / 3)
            L.load(NodeLd4<I, STORE>{a.f.nm + (int64_t)(k0 / 3) * a.f.plane * 4, base, a.f.NP, 0});
        else if constexpr (NM == NM_SCALAR)
            L.load(NodeLd<T, I>{a.f.nm, base, a.f.NP, a.f.nmc, k0, kmax});
        else
            L.load(global_ld<T, STORE, I>(a.f, c1, c2, c3, k0, kmax));
    };

    // the halo of component chunk ch (all three velocity components for the steps)
    constexpr bool ASYNC = STORE != ST_BF16X2;
    uint32_t tma_phase = 0;
    if constexpr (TMA) {
        if (tid == 0) mbar_init(mbar);
        __syncthreads();
    }
    auto issue_halo = [&](int ch) {
        if constexpr (TMA) {
            constexpr uint32_t bytes = (uint32_t)(3 * SC * sizeof(T));
            if (tid == 0) tma_issue(halo, tmap, o1 + PAD - XOFF, o2 + PAD, o3 + PAD, 3 * ch, mbar, bytes);
        } else if constexpr (IS_STEP) {
            stage_halo<T, STORE, H, G, S2, S3, SC, 3, false>(halo, a.f, 0, 3, o1, o2, o3);
        } else {
            stage_halo<T, STORE, H, G, S2, S3, SC, 0, false>(halo, a.f, 3 * ch, min(3, a.f.C - 3 * ch), o1, o2, o3);
        }
    };

    for (int batch = j0; batch < j1; batch += PB) {
        const int nbat = min(PB, j1 - batch);
        if (ASYNC && HALO && batch == j0) issue_halo(0);   // copies in flight while P1 runs
        // ---------------- P1: split, stage what P3 and the writers need ----------------
        if (tid < nbat) {
            const int j = batch + tid;
            const int src = a.perm ? a.perm[j] : j;
            bool ok = true;
            int c[3];
            PRec<T> rec;
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) {
                const double x = a.pos_in[ax * np + src];
                double t;
                ok &= split_axis(x, inv_delta, mask, c[ax], t);
                rec.t[ax] = (T)t;
                if constexpr (IS_STEP) p_x[ax * PB + tid] = x;
            }
            if constexpr (IS_AB2) {   // the AB history rows; entries beyond the valid ones are zero
                for (int r = 0; r < 3 * (a.ab_order - 1); ++r)
                    p_rhs[r * PB + tid] = r < 3 * a.history_valid ? a.rhs_in[r * np + src] : 0.0f;
            }
            p_id[tid] = a.id_in ? a.id_in[src] : src;
            if (!ok) atomicOr(a.flags + FLAG_NONFINITE, 1);
            // a particle always lies in its own block (its key came from the same
            // split); the clamp only keeps a corrupted permutation inside the halo
            const int r1 = min(max((c[0] - o1) & mask, LO), RMAX);
            const int r2 = min(max((c[1] - o2) & mask, LO), RMAX);
            const int r3 = min(max((c[2] - o3) & mask, LO), RMAX);
            const int rp = HALO ? pack_rel(r1, r2, r3) : -1;
            if constexpr (sizeof(T) == 4) rec.relf = __int_as_float(rp);
            else rec.relf = __longlong_as_double((long long)rp);
            p_rec[tid] = rec;
            p_cell[tid] = pack_cell(c[0], c[1], c[2]);
        }
        // ---------------- Q: interpolation ----------------
        for (int ch = 0; ch < nchunks; ++ch) {
            if (HALO && !ASYNC && batch == j0 && ch == 0) issue_halo(0);
            if (HALO && nchunks > 1 && (ch > 0 || batch != j0)) {
                __syncthreads();   // previous readers of the halo are done
                issue_halo(ch);
            }
            if constexpr (TMA) {
                // a copy was issued for this (batch, chunk) unless the one halo chunk of an
                // earlier batch is still in place; every thread waits for it, and if it did
                // not land within the limit the block is skipped (all threads agree) and the
                // host is told
                const bool issued = (batch == j0 && ch == 0) || nchunks > 1;
                bool ok = true;
                if (issued) {
                    ok = mbar_wait(mbar, tma_phase);
                    tma_phase ^= 1u;
                }
                if (__syncthreads_or(!ok)) {
                    if (tid == 0) atomicOr(a.flags + FLAG_HALO_TIMEOUT, 1);
                    return;
                }
            } else {
                if constexpr (HALO && ASYNC) cp_async_wait_all();
                __syncthreads();
            }
            for (int q = warp; q < nbat; q += NW) {
                const PRec<T> rec = p_rec[q];
                int rp;
                if constexpr (sizeof(T) == 4) rp = __float_as_int(rec.relf);
                else rp = (int)__double_as_longlong(rec.relf);
                const T t1 = rec.t[0], t2 = rec.t[1], t3 = rec.t[2];
                const int r1 = rp & 255, r2 = (rp >> 8) & 255, r3 = (rp >> 16) & 255;
                if constexpr (HALO) {
                    L.load(SL{halo + (r3 - LO) * S3 + (r2 - LO) * S2 + (r1 - LO) + XOFF});
                } else {
                    const int pc = p_cell[q];
                    gload(pc & 1023, (pc >> 10) & 1023, (pc >> 20) & 1023, 3 * ch, a.f.C - 1);
                }
                W.eval(t1 - (T)0.5, t2 - (T)0.5, t3 - (T)0.5, wv, wd);
                T acc[12];
                L.contract(wv, wd, acc);
                if constexpr (MODE == MODE_RK2) {
                    // ---- stage 1 result in every lane
                    const T m = reduce4(acc, lane);
                    const T k1[3] = {__shfl_sync(0xffffffffu, m, 0), __shfl_sync(0xffffffffu, m, 8),
                                     __shfl_sync(0xffffffffu, m, 16)};
                    // ---- stage-2 point, cell-relative: t* = t + dt k1 / delta
                    T ts[3] = {fma(dtid, k1[0], t1), fma(dtid, k1[1], t2), fma(dtid, k1[2], t3)};
                    int dc[3];
#pragma unroll
                    for (int ax = 0; ax < 3; ++ax) {
                        const T fl = floor(ts[ax]);
                        dc[ax] = (int)fl;
                        ts[ax] -= fl;
                    }
                    // in the same cell the stage-1 stencil in L is re-used
                    if ((dc[0] | dc[1] | dc[2]) != 0) {
                        const int s1 = r1 + dc[0], s2 = r2 + dc[1], s3 = r3 + dc[2];
                        const bool in =
                            HALO && s1 >= LO && s1 <= RMAX && s2 >= LO && s2 <= RMAX && s3 >= LO && s3 <= RMAX;
                        if (in) {
                            L.load(SL{halo + (s3 - LO) * S3 + (s2 - LO) * S2 + (s1 - LO) + XOFF});
                        } else {
                            // left the staged halo, or (direct path) moved more than one cell
                            const bool far = HALO || abs(dc[0]) > 1 || abs(dc[1]) > 1 || abs(dc[2]) > 1;
                            if (far && lane == 0) atomicOr(a.flags + FLAG_CFL, 1);
                            const int pc = p_cell[q];
                            gload(((pc & 1023) + dc[0]) & mask, (((pc >> 10) & 1023) + dc[1]) & mask,
                                  (((pc >> 20) & 1023) + dc[2]) & mask, 0, 2);
                        }
                    }
                    W.eval(ts[0] - (T)0.5, ts[1] - (T)0.5, ts[2] - (T)0.5, wv, wd);
                    L.contract(wv, wd, acc);
                    const T m2 = reduce4(acc, lane);
                    if (writer) {
                        p_k[rcomp * PB + q] = rcomp == 0 ? k1[0] : (rcomp == 1 ? k1[1] : k1[2]);
                        p_k[(3 + rcomp) * PB + q] = m2;
                    }
                } else if constexpr (MODE == MODE_AB2) {
                    const T m = reduce4(acc, lane);
                    if (writer) {
                        p_k[rcomp * PB + q] = m;
                        if (a.out) {   // per-step output u(X) in caller order
                            const int qid = p_id[q];
                            reinterpret_cast<float*>(a.out)[(int64_t)rcomp * np + qid] = (float)m;
                        }
                    }
                } else if constexpr (MODE == MODE_AB2_D) {
                    // value v sits in lanes 2v, 2v + 1: u_k at v = k, d u_k / d t_j at v = 3 + 3k + j
                    const T m = reduce16(acc, lane);
                    const int v = lane >> 1;
                    if ((lane & 1) == 0 && v < 3) p_k[v * PB + q] = m;
                    if ((lane & 1) == 0 && v >= 3 && v < 12 && a.out) {
                        const int qid = p_id[q];
                        reinterpret_cast<float*>(a.out)[(int64_t)(v - 3) * np + qid] = (float)((double)m * inv_delta);
                    }
                } else if constexpr (MODE == MODE_INTERP) {
                    const T m = reduce4(acc, lane);
                    const int kc = min(3, a.f.C - 3 * ch);
                    if (writer && rcomp < kc) {
                        const int qid = p_id[q];
                        const int64_t o = (int64_t)(3 * ch + rcomp) * np + qid;
                        if (a.out_f64) reinterpret_cast<double*>(a.out)[o] = (double)m;
                        else reinterpret_cast<float*>(a.out)[o] = (float)m;
                    }
                } else {
                    // gradient: value index v = 8 bit4 + 4 bit3 + 2 bit2 + bit1; d u_k/d t_j at v = 3 + 3k + j
                    const T m = reduce16(acc, lane);
                    const int v = ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 +
                                  ((lane >> 1) & 1);
                    const int kc = min(3, a.f.C - 3 * ch);
                    if ((lane & 1) == 0 && v >= 3 && v < 3 + 3 * kc) {
                        const int qid = p_id[q];
                        const int row = 9 * ch + (v - 3);
                        const int64_t o = (int64_t)row * np + qid;
                        const double g = (double)m * inv_delta;
                        if (a.out_f64) reinterpret_cast<double*>(a.out)[o] = g;
                        else reinterpret_cast<float*>(a.out)[o] = (float)g;
                    }
                }
            }
        }
        __syncthreads();
        if constexpr (IS_STEP) {
            // ---------------- P3: update, re-split, write ----------------
            const unsigned valid = __ballot_sync(0xffffffffu, tid < nbat);
            if (tid < nbat) {
                const int j = batch + tid;
                const int id = p_id[tid];
                int cn[3];
                bool ok = true;
#pragma unroll
                for (int ax = 0; ax < 3; ++ax) {
                    const double k1 = (double)p_k[ax * PB + tid];
                    const double x0 = p_x[ax * PB + tid];
                    double xn;
                    if constexpr (MODE == MODE_RK2) {
                        const double k2 = (double)p_k[(3 + ax) * PB + tid];
                        xn = x0 + (0.5 * a.dt) * (k1 + k2);
                    } else {   // ABk, order min(k, 1 + history)
                        const int q = min(a.ab_order, a.history_valid + 1);
                        const double inc = ab_increment(q, k1, [&](int e) {
                            return (double)p_rhs[(3 * e + ax) * PB + tid];
                        });
                        xn = x0 + a.dt * inc;
                        // new history: u_n, then the older entries shifted by one
                        a.rhs_out[ax * np + j] = (float)k1;
                        for (int e = 1; e < a.ab_order - 1; ++e)
                            a.rhs_out[(3 * e + ax) * np + j] = p_rhs[(3 * (e - 1) + ax) * PB + tid];
                    }
                    ok &= split_cell(xn, inv_delta, mask, cn[ax]);
                    a.pos_out[ax * np + j] = xn;
                }
                if (!ok) atomicOr(a.flags + FLAG_NONFINITE, 1);
                a.id_out[j] = id;
                const uint32_t key = block_key(a.g, cn[0], cn[1], cn[2]);
                a.key_out[j] = key;
                if (a.counts) {   // block counts of the next binning, one add per group of equal keys
                    const unsigned peers = __match_any_sync(valid, key);
                    if (lane == __ffs(peers) - 1) atomicAdd(a.counts + key, (uint32_t)__popc(peers));
                }
            }
            __syncthreads();
        }
    }
}

#ifndef TRK_F32_MIN_BLOCKS
#define TRK_F32_MIN_BLOCKS 3   // resident CTAs per SM the float32 kernels are register-capped for (I = 4, 6)
#endif

// tmap: the tensor map of the padded field (read only with HC == HC_TMA)
// resident CTAs per SM the block kernel is register-capped for: float32 I = 4, 6
// TRK_F32_MIN_BLOCKS; I = 8 two, three for value interpolation of a float32
// field (its shared-memory plan has no k values and fits three CTAs; 79-80
// registers without spills)
template <typename T, int I, int MODE, int STORE>
constexpr int block_min_ctas()
{
    if constexpr (sizeof(T) != 4) return 1;
    else if constexpr (I != 8) return TRK_F32_MIN_BLOCKS;
    else return MODE == MODE_INTERP && STORE == ST_F32 ? 3 : 2;
}

template <typename T, int I, int DEG, int MODE, int STORE, int HC>
__global__ void __launch_bounds__(NT, block_min_ctas<T, I, MODE, STORE>())
    k_block(const __grid_constant__ BlockArgs a, const __grid_constant__ CUtensorMap tmap)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int b = blockIdx.x;
    process_block<T, I, DEG, MODE, STORE, true, NM_NONE, HC>(a, b, a.offsets[b], a.offsets[b + 1], smem_raw, &tmap);
}

// particles per CTA of the direct kernel: a.ppc in [1, PB], 0 for PB (a launch
// shape the tuner chooses; every value gives the same results)
__host__ __device__ __forceinline__ int direct_ppc(const BlockArgs& a) { return a.ppc > 0 && a.ppc < PB ? a.ppc : PB; }

// Direct path: CTA c takes the sorted particles [c ppc, (c + 1) ppc) and
// gathers their stencils from global memory (no halo, no cell-block grid);
// float32 fields are read from the node-major copy a.f.nm.
template <typename T, int I>
constexpr int direct_min_ctas()
{
    return sizeof(T) == 4 ? (I == 8 ? 2 : TRK_F32_MIN_BLOCKS) : 1;
}

// shared-memory carveout (percent of the SM's 228 KB) that holds `ctas` CTAs of
// `smem` dynamic bytes each, with the 1 KB the system reserves per CTA
inline int carveout_percent(size_t smem, int ctas)
{
    const size_t per_cta = (smem + 1024 + 127) / 128 * 128;
    const size_t pct = (ctas * per_cta * 100 + 233471) / 233472;
    return (int)(pct < 100 ? pct : 100);
}

template <typename T, int I, int DEG, int MODE, int STORE, int NM>
__global__ void __launch_bounds__(NT, direct_min_ctas<T, I>())
    k_direct(const __grid_constant__ BlockArgs a)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int ppc = direct_ppc(a);
    const int64_t j0 = (int64_t)blockIdx.x * ppc;
    const int64_t j1 = j0 + ppc < a.np ? j0 + ppc : a.np;
    process_block<T, I, DEG, MODE, STORE, false, NM>(a, 0, (int)j0, (int)j1, smem_raw);
}

template <typename T, int I, int MODE>
constexpr size_t direct_smem_bytes()
{
    return SmemPlan<T, 0, stage_of<MODE>()>::total;
}

template <typename T, int I, int DEG, int MODE, int STORE, int NM>
cudaError_t launch_direct_nm(const BlockArgs& a, cudaStream_t st)
{
    constexpr size_t smem = direct_smem_bytes<T, I, MODE>();
    static_assert(smem <= 232448, "direct shared-memory plan exceeds the per-block limit");
    auto kern = k_direct<T, I, DEG, MODE, STORE, NM>;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        // the gathers run through L1: ask for no more shared memory than the resident
        // CTAs use (0.8% faster at 256^3, 1/16 per cell: 192 instead of 124 KB of L1)
        e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 carveout_percent(smem, direct_min_ctas<T, I>()));
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const int ppc = direct_ppc(a);
    kern<<<(unsigned)((a.np + ppc - 1) / ppc), NT, smem, st>>>(a);
    return cudaGetLastError();
}

// 16-byte node loads: texture fetches where the copy has a texture, else plain loads
template <typename T, int I, int DEG, int MODE, int STORE>
cudaError_t launch_direct_vec(const BlockArgs& a, cudaStream_t st)
{
    if (a.f.nm_tex) return launch_direct_nm<T, I, DEG, MODE, STORE, NM_TEX4>(a, st);
    return launch_direct_nm<T, I, DEG, MODE, STORE, NM_VEC4>(a, st);
}

// float32 fields read the node-major copy (16-byte node loads for three
// components, which the time steps always have, as texture fetches where the
// copy has textures), other storages the field
template <typename T, int I, int DEG, int MODE, int STORE>
cudaError_t launch_direct_t(const BlockArgs& a, cudaStream_t st)
{
    if (a.np <= 0) return cudaSuccess;
    constexpr bool STEP = MODE == MODE_RK2 || MODE == MODE_AB2;
    if constexpr (STORE == ST_F32) {
        if (!a.f.nm) return cudaErrorInvalidValue;   // the node-major copy is required
        if (STEP || (a.f.C == 3 && a.f.nmc == 4)) return launch_direct_vec<T, I, DEG, MODE, STORE>(a, st);
        if constexpr (!STEP) return launch_direct_nm<T, I, DEG, MODE, STORE, NM_SCALAR>(a, st);
        return cudaErrorInvalidValue;
    } else if constexpr (STORE == ST_BF16X2) {
        // the node-major copy (16 bytes per node and chunk of three components;
        // always there for three components, i.e. for every time step), else
        // the component-major field
        if (a.f.nm) return launch_direct_vec<T, I, DEG, MODE, STORE>(a, st);
        if (a.f.C == 3) return cudaErrorInvalidValue;
        return launch_direct_nm<T, I, DEG, MODE, STORE, NM_NONE>(a, st);
    } else {
        return launch_direct_nm<T, I, DEG, MODE, STORE, NM_NONE>(a, st);
    }
}

template <int I, int DEG>
cudaError_t dispatch_direct(int mode, const BlockArgs& a, cudaStream_t st)
{
    const int s = a.f.storage;
#define TRK_CASE(M)                                                                    \
    case M:                                                                            \
        if (s == ST_F64) return launch_direct_t<double, I, DEG, M, ST_F64>(a, st);     \
        if (s == ST_F32) return launch_direct_t<float, I, DEG, M, ST_F32>(a, st);      \
        return launch_direct_t<float, I, DEG, M, ST_BF16X2>(a, st);
    switch (mode) {
        TRK_CASE(MODE_INTERP)
        TRK_CASE(MODE_INTERP_DERIV)
        TRK_CASE(MODE_RK2)
        TRK_CASE(MODE_AB2)
    }
#undef TRK_CASE
    return cudaErrorInvalidValue;
}

template <typename T, int I, int MODE, int HC = HC_ASYNC>
constexpr size_t block_smem_bytes()
{
    constexpr int MARGIN = (MODE == MODE_RK2) ? 1 : 0;
    constexpr int H = BLK + I - 1 + 2 * MARGIN;
    using Lay = Layout<I, H>;
    constexpr int SC = HC == HC_TMA ? tma_box(I, MARGIN, (int)sizeof(T)).SC() : Lay::SC;
    return SmemPlan<T, SC, stage_of<MODE>()>::total;
}

template <typename T, int I, int DEG, int MODE, int STORE, int HC>
cudaError_t launch_block_hc(const BlockArgs& a, const CUtensorMap& tmap, int64_t nblocks, cudaStream_t st)
{
    constexpr size_t smem = block_smem_bytes<T, I, MODE, HC>();
    static_assert(smem <= 232448, "block shared-memory plan exceeds the per-block limit");
    auto kern = k_block<T, I, DEG, MODE, STORE, HC>;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    if (nblocks <= 0) return cudaSuccess;
    kern<<<(unsigned)nblocks, NT, smem, st>>>(a, tmap);
    return cudaGetLastError();
}

// tmap: the tensor map of the padded field for this mode's box (tma_box), or
// null for the cp.async / register staging
template <typename T, int I, int DEG, int MODE, int STORE>
cudaError_t launch_block_t(const BlockArgs& a, const CUtensorMap* tmap, int64_t nblocks, cudaStream_t st)
{
    if constexpr (STORE == ST_F32 || STORE == ST_F64) {
        if (tmap) return launch_block_hc<T, I, DEG, MODE, STORE, HC_TMA>(a, *tmap, nblocks, st);
    }
    const CUtensorMap none{};
    return launch_block_hc<T, I, DEG, MODE, STORE, HC_ASYNC>(a, none, nblocks, st);
}

template <int I, int DEG>
cudaError_t dispatch_store_mode(int mode, const BlockArgs& a, const CUtensorMap* tmap, int64_t nblocks, cudaStream_t st)
{
    const int s = a.f.storage;
#define TRK_CASE(M)                                                                               \
    case M:                                                                                       \
        if (s == ST_F64) return launch_block_t<double, I, DEG, M, ST_F64>(a, tmap, nblocks, st); \
        if (s == ST_F32) return launch_block_t<float, I, DEG, M, ST_F32>(a, tmap, nblocks, st);  \
        return launch_block_t<float, I, DEG, M, ST_BF16X2>(a, nullptr, nblocks, st);
    switch (mode) {
        TRK_CASE(MODE_INTERP)
        TRK_CASE(MODE_INTERP_DERIV)
        TRK_CASE(MODE_RK2)
        TRK_CASE(MODE_AB2)
    }
#undef TRK_CASE
    return cudaErrorInvalidValue;
}

}  // namespace trk
