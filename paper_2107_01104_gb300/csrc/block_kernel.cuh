// Block kernels: one CTA per cell block of BLK^3 cells (the block grouping of
// Sec. 3.3.1, with the paper's x3 slices generalised to cubes).
//
// A CTA stages the block's field halo in shared memory once and then runs
// the per-particle work in phases separated by __syncthreads():
//
//   P1  one thread per particle: read X through the sort permutation, split it
//       into cell c and offset t (float64, Sec. 2.2 steps 1-3);
//   Q1  one warp per particle: evaluate the 1-D weights beta_i once per axis,
//       gather the I x I x I stencil from shared memory and contract it
//       (Eq. triple_sum, separably as in Sec. 3.3), reduce across the warp;
//   P2  (RK2) one thread per particle: stage-2 point X* = X + dt k1;
//   Q2  (RK2) warp per particle at X*;
//   P3  one thread per particle: float64 update of X (RK2 or AB2), new cell
//       split and block key for the next re-binning, coalesced write-out.
//
// Warp-per-particle lane maps (chosen so that every warp-wide shared load
// hits 32 distinct banks, see Layout):
//   I = 8: lane = (i1 in 0..7, j in 0..3); i2 = j and j+4; loop i3 in 0..7
//   I = 6: lane = (i1 in 0..5, j in 0..4); pass A i2 = j, i3 = 0..5;
//          pass B i2 = 5, i3 = j; pass C (lanes 0..5) i2 = i3 = 5
//   I = 4: lane = (i1, i2 in 0..3, p in 0..1); i3 = p and p+2
#pragma once

#include "internal.cuh"

namespace trk {

constexpr int NT = 256;           // threads per CTA
constexpr int NW = NT / 32;       // warps per CTA
constexpr int PB = NT;            // particles per batch (one per thread in the P phases)

static __constant__ double c_coef_d[TRK_NUM_TABLES][TRK_TAB_MAX_I][TRK_TAB_MAX_DEG] = TRK_COEF_INIT;
static __constant__ float c_coef_f[TRK_NUM_TABLES][TRK_TAB_MAX_I][TRK_TAB_MAX_DEG] = TRK_COEF_INIT;
static __constant__ double c_dcoef_d[TRK_NUM_TABLES][TRK_TAB_MAX_I][TRK_TAB_MAX_DEG] = TRK_DCOEF_INIT;
static __constant__ float c_dcoef_f[TRK_NUM_TABLES][TRK_TAB_MAX_I][TRK_TAB_MAX_DEG] = TRK_DCOEF_INIT;

template <typename T> __device__ __forceinline__ T coef(int tab, int i, int d);
template <> __device__ __forceinline__ float coef<float>(int tab, int i, int d) { return c_coef_f[tab][i][d]; }
template <> __device__ __forceinline__ double coef<double>(int tab, int i, int d) { return c_coef_d[tab][i][d]; }
template <typename T> __device__ __forceinline__ T dcoef(int tab, int i, int d);
template <> __device__ __forceinline__ float dcoef<float>(int tab, int i, int d) { return c_dcoef_f[tab][i][d]; }
template <> __device__ __forceinline__ double dcoef<double>(int tab, int i, int d) { return c_dcoef_d[tab][i][d]; }

// ---------------------------------------------------------------------------
// Shared-memory layout of the halo: [3 components][H][H][S2], row stride S2,
// plane stride S3, component stride SC.  S2 and S3 are the smallest strides
// for which the lane map of kernel width I reads 32 distinct banks.
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

// Joint search: smallest row stride S2 >= H that admits a plane stride S3.
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
// Horner evaluation of beta_i(s) (s = t - 1/2) from a register row or from
// the constant table.
// ---------------------------------------------------------------------------
template <typename T, int DEG>
struct Row {
    T c[DEG + 1];
};

template <typename T, int DEG>
__device__ __forceinline__ Row<T, DEG> load_row(int tab, int i, bool deriv)
{
    Row<T, DEG> r;
#pragma unroll
    for (int d = 0; d <= DEG; ++d) r.c[d] = deriv ? dcoef<T>(tab, i, d) : coef<T>(tab, i, d);
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

template <typename T, int DEG>
__device__ __forceinline__ T horner_tab(int tab, int i, T s)
{
    T acc = coef<T>(tab, i, DEG);
#pragma unroll
    for (int d = DEG - 1; d >= 0; --d) acc = fma(acc, s, coef<T>(tab, i, d));
    return acc;
}

template <typename T, int DEG>
__device__ __forceinline__ T dhorner_tab(int tab, int i, T s)
{
    // derivative polynomial has degree DEG - 1
    T acc = dcoef<T>(tab, i, DEG - 1);
#pragma unroll
    for (int d = DEG - 2; d >= 0; --d) acc = fma(acc, s, dcoef<T>(tab, i, d));
    return acc;
}

// Per-lane coefficient rows (lane-dependent node indices), loaded once per CTA.
template <typename T, int I, int DEG, bool D>
struct LaneRows;

template <typename T, int DEG, bool D>
struct LaneRows<T, 8, DEG, D> {
    Row<T, DEG> a, b, c;        // rows i1, j, j+4
    Row<T, DEG> da, db, dc;     // derivative rows (used when D)
    __device__ void load(int tab, int lane)
    {
        const int i1 = lane & 7, j = lane >> 3;
        a = load_row<T, DEG>(tab, i1, false);
        b = load_row<T, DEG>(tab, j, false);
        c = load_row<T, DEG>(tab, j + 4, false);
        if (D) {
            da = load_row<T, DEG>(tab, i1, true);
            db = load_row<T, DEG>(tab, j, true);
            dc = load_row<T, DEG>(tab, j + 4, true);
        }
    }
};

template <typename T, int DEG, bool D>
struct LaneRows<T, 6, DEG, D> {
    Row<T, DEG> a, b;           // rows i1, j
    Row<T, DEG> da, db;
    __device__ void load(int tab, int lane)
    {
        const int i1 = lane % 6, j = min(lane / 6, 5);
        a = load_row<T, DEG>(tab, i1, false);
        b = load_row<T, DEG>(tab, j, false);
        if (D) {
            da = load_row<T, DEG>(tab, i1, true);
            db = load_row<T, DEG>(tab, j, true);
        }
    }
};

template <typename T, int DEG, bool D>
struct LaneRows<T, 4, DEG, D> {
    Row<T, DEG> a, b, c, e;     // rows i1, i2, p, p+2
    Row<T, DEG> da, db, dc, de;
    __device__ void load(int tab, int lane)
    {
        const int i1 = lane & 3, i2 = (lane >> 2) & 3, p = lane >> 4;
        a = load_row<T, DEG>(tab, i1, false);
        b = load_row<T, DEG>(tab, i2, false);
        c = load_row<T, DEG>(tab, p, false);
        e = load_row<T, DEG>(tab, p + 2, false);
        if (D) {
            da = load_row<T, DEG>(tab, i1, true);
            db = load_row<T, DEG>(tab, i2, true);
            dc = load_row<T, DEG>(tab, p, true);
            de = load_row<T, DEG>(tab, p + 2, true);
        }
    }
};

// ---------------------------------------------------------------------------
// Warp-level stencil gather + contraction for one particle.
// ld(k, a1, a2, a3) returns component k of node (c + a - (I/2 - 1)).
// On return (before the warp reduction) every lane holds a partial sum:
//   acc[k]            value      u_k
//   acc[3 + 3k + j]   derivative d u_k / d t_j  (when D)
// ---------------------------------------------------------------------------
template <typename T, int DEG, bool D, class LD>
__device__ __forceinline__ void gather_i8(const LD& ld, int lane, int tab, const LaneRows<T, 8, DEG, D>& R,
                                          T s1, T s2, T s3, T (&acc)[12])
{
    const int i1 = lane & 7, j = lane >> 3;
    const T w1 = horner(R.a, s1);
    const T w2[2] = {horner(R.b, s2), horner(R.c, s2)};
    T w3[8], dw3[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        w3[i] = horner_tab<T, DEG>(tab, i, s3);
        if (D) dw3[i] = dhorner_tab<T, DEG>(tab, i, s3);
    }
    T dw1 = 0, dw2[2] = {0, 0};
    if (D) {
        dw1 = horner(R.da, s1);
        dw2[0] = horner(R.db, s2);
        dw2[1] = horner(R.dc, s2);
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        T pv[3] = {0, 0, 0}, pd[3] = {0, 0, 0};
#pragma unroll
        for (int i3 = 0; i3 < 8; ++i3) {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const T f = ld(k, i1, j + 4 * h, i3);
                pv[k] = fma(w3[i3], f, pv[k]);
                if (D) pd[k] = fma(dw3[i3], f, pd[k]);
            }
        }
        const T a12 = w1 * w2[h];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            acc[k] = fma(a12, pv[k], acc[k]);
            if (D) {
                acc[3 + 3 * k + 0] = fma(dw1 * w2[h], pv[k], acc[3 + 3 * k + 0]);
                acc[3 + 3 * k + 1] = fma(w1 * dw2[h], pv[k], acc[3 + 3 * k + 1]);
                acc[3 + 3 * k + 2] = fma(a12, pd[k], acc[3 + 3 * k + 2]);
            }
        }
    }
}

template <typename T, int DEG, bool D, class LD>
__device__ __forceinline__ void gather_i6(const LD& ld, int lane, int tab, const LaneRows<T, 6, DEG, D>& R,
                                          T s1, T s2, T s3, T (&acc)[12])
{
    const int i1 = lane % 6, j = min(lane / 6, 5);
    const bool act = lane < 30;
    const T w1 = horner(R.a, s1), w2j = horner(R.b, s2), w3j = horner(R.b, s3);
    const T w25 = horner_tab<T, DEG>(tab, 5, s2);
    T w3[6], dw3[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        w3[i] = horner_tab<T, DEG>(tab, i, s3);
        if (D) dw3[i] = dhorner_tab<T, DEG>(tab, i, s3);
    }
    T dw1 = 0, dw2j = 0, dw3j = 0, dw25 = 0;
    if (D) {
        dw1 = horner(R.da, s1);
        dw2j = horner(R.db, s2);
        dw3j = horner(R.db, s3);
        dw25 = dhorner_tab<T, DEG>(tab, 5, s2);
    }
    if (act) {
        // pass A: i2 = j, i3 = 0..5
        T pv[3] = {0, 0, 0}, pd[3] = {0, 0, 0};
#pragma unroll
        for (int i3 = 0; i3 < 6; ++i3) {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const T f = ld(k, i1, j, i3);
                pv[k] = fma(w3[i3], f, pv[k]);
                if (D) pd[k] = fma(dw3[i3], f, pd[k]);
            }
        }
        const T a12 = w1 * w2j;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            acc[k] = fma(a12, pv[k], acc[k]);
            if (D) {
                acc[3 + 3 * k + 0] = fma(dw1 * w2j, pv[k], acc[3 + 3 * k + 0]);
                acc[3 + 3 * k + 1] = fma(w1 * dw2j, pv[k], acc[3 + 3 * k + 1]);
                acc[3 + 3 * k + 2] = fma(a12, pd[k], acc[3 + 3 * k + 2]);
            }
        }
        // pass B: i2 = 5, i3 = j
        const T wb = w1 * w25 * w3j;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const T f = ld(k, i1, 5, j);
            acc[k] = fma(wb, f, acc[k]);
            if (D) {
                acc[3 + 3 * k + 0] = fma(dw1 * w25 * w3j, f, acc[3 + 3 * k + 0]);
                acc[3 + 3 * k + 1] = fma(w1 * dw25 * w3j, f, acc[3 + 3 * k + 1]);
                acc[3 + 3 * k + 2] = fma(w1 * w25 * dw3j, f, acc[3 + 3 * k + 2]);
            }
        }
    }
    if (lane < 6) {
        // pass C: i2 = i3 = 5
        const T wc = w1 * w25 * w3[5];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const T f = ld(k, i1, 5, 5);
            acc[k] = fma(wc, f, acc[k]);
            if (D) {
                acc[3 + 3 * k + 0] = fma(dw1 * w25 * w3[5], f, acc[3 + 3 * k + 0]);
                acc[3 + 3 * k + 1] = fma(w1 * dw25 * w3[5], f, acc[3 + 3 * k + 1]);
                acc[3 + 3 * k + 2] = fma(w1 * w25 * dw3[5], f, acc[3 + 3 * k + 2]);
            }
        }
    }
}

template <typename T, int DEG, bool D, class LD>
__device__ __forceinline__ void gather_i4(const LD& ld, int lane, int tab, const LaneRows<T, 4, DEG, D>& R,
                                          T s1, T s2, T s3, T (&acc)[12])
{
    const int i1 = lane & 3, i2 = (lane >> 2) & 3, p = lane >> 4;
    const T w1 = horner(R.a, s1), w2 = horner(R.b, s2);
    const T w3a = horner(R.c, s3), w3b = horner(R.e, s3);
    T dw1 = 0, dw2 = 0, dw3a = 0, dw3b = 0;
    if (D) {
        dw1 = horner(R.da, s1);
        dw2 = horner(R.db, s2);
        dw3a = horner(R.dc, s3);
        dw3b = horner(R.de, s3);
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const T f0 = ld(k, i1, i2, p), f1 = ld(k, i1, i2, p + 2);
        const T pv = fma(w3a, f0, w3b * f1);
        acc[k] = fma(w1 * w2, pv, acc[k]);
        if (D) {
            const T pd = fma(dw3a, f0, dw3b * f1);
            acc[3 + 3 * k + 0] = fma(dw1 * w2, pv, acc[3 + 3 * k + 0]);
            acc[3 + 3 * k + 1] = fma(w1 * dw2, pv, acc[3 + 3 * k + 1]);
            acc[3 + 3 * k + 2] = fma(w1 * w2, pd, acc[3 + 3 * k + 2]);
        }
    }
}

template <typename T, int I, int DEG, bool D, class LD>
__device__ __forceinline__ void gather(const LD& ld, int lane, int tab, const LaneRows<T, I, DEG, D>& R, T s1, T s2,
                                       T s3, T (&acc)[12])
{
#pragma unroll
    for (int r = 0; r < 12; ++r) acc[r] = 0;
    if constexpr (I == 8) gather_i8<T, DEG, D>(ld, lane, tab, R, s1, s2, s3, acc);
    else if constexpr (I == 6) gather_i6<T, DEG, D>(ld, lane, tab, R, s1, s2, s3, acc);
    else gather_i4<T, DEG, D>(ld, lane, tab, R, s1, s2, s3, acc);
    constexpr int NV = D ? 12 : 3;
#pragma unroll
    for (int r = 0; r < NV; ++r) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], o);
    }
}

// ---------------------------------------------------------------------------
// Loaders
// ---------------------------------------------------------------------------
template <typename T, int S2, int S3, int SC>
struct SmemLd {
    const T* base;   // node (c - (I/2 - 1)) of component 0
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

// Global-memory loader with periodic wrap (for stencils outside the staged halo).
template <typename T, int STORE, int I>
struct GlobalLd {
    FieldView f;
    int c1, c2, c3, k0, kmax, N, mask;
    __device__ __forceinline__ T operator()(int k, int a1, int a2, int a3) const
    {
        const int x1 = (c1 + a1 - (I / 2 - 1)) & mask;
        const int x2 = (c2 + a2 - (I / 2 - 1)) & mask;
        const int x3 = (c3 + a3 - (I / 2 - 1)) & mask;
        const int kk = min(k0 + k, kmax);
        return fetch<T, STORE>(f, kk, ((int64_t)x3 * N + x2) * N + x1);
    }
};

template <typename T, int STORE, int H, int S2, int S3, int SC>
__device__ __forceinline__ void load_halo(T* halo, const FieldView& f, int k0, int ox, int oy, int oz, int N,
                                          int mask)
{
    constexpr int NPC = H * H * H;
    for (int k = 0; k < 3; ++k) {
        const int kk = k0 + k;
        if (kk >= f.C) break;
        for (int e = threadIdx.x; e < NPC; e += NT) {
            const int x = e % H, yz = e / H, y = yz % H, z = yz / H;
            const int64_t gi = ((int64_t)((oz + z) & mask) * N + ((oy + y) & mask)) * N + ((ox + x) & mask);
            halo[k * SC + z * S3 + y * S2 + x] = fetch<T, STORE>(f, kk, gi);
        }
    }
}

__device__ __forceinline__ int pack_rel(int r1, int r2, int r3) { return r1 | (r2 << 8) | (r3 << 16); }
__device__ __forceinline__ int pack_cell(int c1, int c2, int c3) { return c1 | (c2 << 10) | (c3 << 20); }

// ---------------------------------------------------------------------------
// The block kernel.
// ---------------------------------------------------------------------------
template <typename T, int I, int DEG, int MODE, int STORE>
__global__ void __launch_bounds__(NT) k_block(const BlockArgs a)
{
    constexpr bool IS_STEP = (MODE == MODE_RK2 || MODE == MODE_AB2);
    constexpr bool D = (MODE == MODE_INTERP_DERIV);
    constexpr int MARGIN = (MODE == MODE_RK2) ? 1 : 0;     // halo margin for the stage-2 point
    constexpr int H = BLK + I - 1 + 2 * MARGIN;
    constexpr int G = I / 2 - 1 + MARGIN;                   // halo origin = block origin - G
    using Lay = Layout<I, H>;
    constexpr int S2 = Lay::S2, S3 = Lay::S3, SC = Lay::SC;
    constexpr int LO = I / 2 - 1;                           // stencil node offset

    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* halo = reinterpret_cast<T*>(smem_raw);
    T* p_t = halo + 3 * SC;                                 // [3][PB]
    T* p_k1 = p_t + 3 * PB;                                 // [3][PB]
    T* p_k2 = p_k1 + 3 * PB;                                // [3][PB]
    int* p_rel = reinterpret_cast<int*>(p_k2 + 3 * PB);     // [PB]
    int* p_cell = p_rel + PB;                               // [PB]

    const int b = blockIdx.x;
    const int j0 = a.offsets[b], j1 = a.offsets[b + 1];
    if (j0 >= j1) return;

    const int N = a.g.N, mask = a.g.mask;
    const int nb1 = a.g.nb1, nb2 = a.g.nb2;
    const int bx = b % nb1, by = (b / nb1) % nb2, bz = b / (nb1 * nb2);
    const int o1 = bx * BLK - G, o2 = by * BLK - G, o3 = bz * BLK - G;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t np = a.np;
    const double inv_delta = a.g.inv_delta;

    LaneRows<T, I, DEG, D> R;
    R.load(a.tab, lane);

    const int nchunks = IS_STEP ? 1 : (a.f.C + 2) / 3;

    for (int batch = j0; batch < j1; batch += PB) {
        const int nbat = min(PB, j1 - batch);
        // ---------------- P1: split ----------------
        double X[3] = {0, 0, 0};
        float hr[3] = {0, 0, 0};
        int id = 0;
        int c[3] = {0, 0, 0};
        if (tid < nbat) {
            const int j = batch + tid;
            const int src = a.perm[j];
            id = a.id_in ? a.id_in[src] : src;
            bool ok = true;
            double t[3];
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) {
                X[ax] = a.pos_in[ax * np + src];
                ok &= split_axis(X[ax], inv_delta, mask, c[ax], t[ax]);
                p_t[ax * PB + tid] = (T)t[ax];
            }
            if (!ok) atomicOr(a.flags + FLAG_NONFINITE, 1);
            const int r1 = (c[0] - o1) & mask, r2 = (c[1] - o2) & mask, r3 = (c[2] - o3) & mask;
            // a particle always lies in its own block; the guard only keeps a
            // corrupted permutation from indexing outside the staged halo
            const bool in = r1 >= LO && r1 <= H - 1 - I / 2 && r2 >= LO && r2 <= H - 1 - I / 2 &&
                            r3 >= LO && r3 <= H - 1 - I / 2;
            p_rel[tid] = in ? pack_rel(r1, r2, r3) : -1;
            p_cell[tid] = pack_cell(c[0], c[1], c[2]);
            if (MODE == MODE_AB2 && a.history_valid) {
#pragma unroll
                for (int ax = 0; ax < 3; ++ax) hr[ax] = a.rhs_in[ax * np + src];
            }
        }
        // ---------------- Q1: interpolation at X ----------------
        for (int ch = 0; ch < nchunks; ++ch) {
            if (batch == j0 || nchunks > 1) {
                if (ch > 0 || batch != j0) __syncthreads();   // previous readers of the halo are done
                load_halo<T, STORE, H, S2, S3, SC>(halo, a.f, 3 * ch, o1, o2, o3, N, mask);
            }
            __syncthreads();
            for (int q = warp; q < nbat; q += NW) {
                const int rp = p_rel[q];
                const T s1 = p_t[q] - (T)0.5, s2 = p_t[PB + q] - (T)0.5, s3 = p_t[2 * PB + q] - (T)0.5;
                T acc[12];
                if (rp >= 0) {
                    const int r1 = rp & 255, r2 = (rp >> 8) & 255, r3 = (rp >> 16) & 255;
                    SmemLd<T, S2, S3, SC> ld{halo + (r3 - LO) * S3 + (r2 - LO) * S2 + (r1 - LO)};
                    gather<T, I, DEG, D>(ld, lane, a.tab, R, s1, s2, s3, acc);
                } else {
                    const int pc = p_cell[q];
                    GlobalLd<T, STORE, I> ld{a.f, pc & 1023, (pc >> 10) & 1023, (pc >> 20) & 1023, 3 * ch,
                                             a.f.C - 1, N, mask};
                    gather<T, I, DEG, D>(ld, lane, a.tab, R, s1, s2, s3, acc);
                }
                if constexpr (IS_STEP) {
                    if (lane < 3) p_k1[lane * PB + q] = acc[lane];
                } else {
                    const int qid = a.id_in ? a.id_in[a.perm[batch + q]] : a.perm[batch + q];
                    const int kc = min(3, a.f.C - 3 * ch);
                    const int nout = D ? 3 * kc : kc;
                    if (lane < nout) {
                        // lane r -> output row: value k = r, or derivative (k, j) = (r/3, r%3)
                        T v;
                        int row;
                        if (D) {
                            v = 0;
#pragma unroll
                            for (int r = 0; r < 9; ++r)
                                if (r == lane) v = acc[3 + r];
                            v *= (T)inv_delta;
                            row = 9 * ch + lane;
                        } else {
                            v = lane == 0 ? acc[0] : (lane == 1 ? acc[1] : acc[2]);
                            row = 3 * ch + lane;
                        }
                        if (a.out_f64) reinterpret_cast<double*>(a.out)[(int64_t)row * np + qid] = (double)v;
                        else reinterpret_cast<float*>(a.out)[(int64_t)row * np + qid] = (float)v;
                    }
                }
            }
        }
        if constexpr (!IS_STEP) {
            __syncthreads();
            continue;
        } else {
            __syncthreads();
            if constexpr (MODE == MODE_RK2) {
                // ---------------- P2: stage-2 point ----------------
                if (tid < nbat) {
                    int cs[3];
                    T ts[3];
                    if constexpr (sizeof(T) == 4) {
                        // cell-relative float32: t* = t + dt k1 / delta
                        const float sc = (float)(a.dt * inv_delta);
#pragma unroll
                        for (int ax = 0; ax < 3; ++ax) {
                            const float tt = fmaf(sc, (float)p_k1[ax * PB + tid], (float)p_t[ax * PB + tid]);
                            const float fl = floorf(tt);
                            cs[ax] = (c[ax] + (int)fl) & mask;
                            ts[ax] = tt - fl;
                        }
                    } else {
                        bool ok = true;
#pragma unroll
                        for (int ax = 0; ax < 3; ++ax) {
                            const double xs = X[ax] + a.dt * (double)p_k1[ax * PB + tid];
                            double tt;
                            ok &= split_axis(xs, inv_delta, mask, cs[ax], tt);
                            ts[ax] = (T)tt;
                        }
                        if (!ok) atomicOr(a.flags + FLAG_NONFINITE, 1);
                    }
                    const int r1 = (cs[0] - o1) & mask, r2 = (cs[1] - o2) & mask, r3 = (cs[2] - o3) & mask;
                    const bool in = r1 >= LO && r1 <= H - 1 - I / 2 && r2 >= LO && r2 <= H - 1 - I / 2 &&
                                    r3 >= LO && r3 <= H - 1 - I / 2;
                    if (!in) atomicOr(a.flags + FLAG_CFL, 1);
                    p_rel[tid] = in ? pack_rel(r1, r2, r3) : -1;
                    p_cell[tid] = pack_cell(cs[0], cs[1], cs[2]);
#pragma unroll
                    for (int ax = 0; ax < 3; ++ax) p_t[ax * PB + tid] = ts[ax];
                }
                __syncthreads();
                // ---------------- Q2: interpolation at X* ----------------
                for (int q = warp; q < nbat; q += NW) {
                    const int rp = p_rel[q];
                    const T s1 = p_t[q] - (T)0.5, s2 = p_t[PB + q] - (T)0.5, s3 = p_t[2 * PB + q] - (T)0.5;
                    T acc[12];
                    if (rp >= 0) {
                        const int r1 = rp & 255, r2 = (rp >> 8) & 255, r3 = (rp >> 16) & 255;
                        SmemLd<T, S2, S3, SC> ld{halo + (r3 - LO) * S3 + (r2 - LO) * S2 + (r1 - LO)};
                        gather<T, I, DEG, D>(ld, lane, a.tab, R, s1, s2, s3, acc);
                    } else {
                        const int pc = p_cell[q];
                        GlobalLd<T, STORE, I> ld{a.f, pc & 1023, (pc >> 10) & 1023, (pc >> 20) & 1023, 0, 2, N, mask};
                        gather<T, I, DEG, D>(ld, lane, a.tab, R, s1, s2, s3, acc);
                    }
                    if (lane < 3) p_k2[lane * PB + q] = acc[lane];
                }
                __syncthreads();
            }
            // ---------------- P3: update, re-split, write ----------------
            if (tid < nbat) {
                const int j = batch + tid;
                double Xn[3];
                int cn[3];
                bool ok = true;
#pragma unroll
                for (int ax = 0; ax < 3; ++ax) {
                    const double k1 = (double)p_k1[ax * PB + tid];
                    if constexpr (MODE == MODE_RK2) {
                        const double k2 = (double)p_k2[ax * PB + tid];
                        Xn[ax] = X[ax] + (0.5 * a.dt) * (k1 + k2);
                    } else {
                        const double inc = a.history_valid ? (1.5 * k1 - 0.5 * (double)hr[ax]) : k1;
                        Xn[ax] = X[ax] + a.dt * inc;
                        a.rhs_out[ax * np + j] = (float)k1;
                    }
                    double tt;
                    ok &= split_axis(Xn[ax], inv_delta, mask, cn[ax], tt);
                    a.pos_out[ax * np + j] = Xn[ax];
                }
                if (!ok) atomicOr(a.flags + FLAG_NONFINITE, 1);
                a.id_out[j] = id;
                a.key_out[j] = block_key(a.g, cn[0], cn[1], cn[2]);
            }
            __syncthreads();
        }
    }
}

template <typename T, int I, int MODE>
constexpr size_t block_smem_bytes()
{
    constexpr int MARGIN = (MODE == MODE_RK2) ? 1 : 0;
    constexpr int H = BLK + I - 1 + 2 * MARGIN;
    using Lay = Layout<I, H>;
    return (size_t)(3 * Lay::SC + 9 * PB) * sizeof(T) + 2 * PB * sizeof(int);
}

template <typename T, int I, int DEG, int MODE, int STORE>
cudaError_t launch_block_t(const BlockArgs& a, int64_t nblocks, cudaStream_t st)
{
    constexpr size_t smem = block_smem_bytes<T, I, MODE>();
    auto kern = k_block<T, I, DEG, MODE, STORE>;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    if (nblocks <= 0) return cudaSuccess;
    kern<<<(unsigned)nblocks, NT, smem, st>>>(a);
    return cudaGetLastError();
}

template <int I, int DEG>
cudaError_t dispatch_store_mode(int mode, const BlockArgs& a, int64_t nblocks, cudaStream_t st)
{
    const int s = a.f.storage;
#define TRK_CASE(M)                                                                   \
    case M:                                                                           \
        if (s == ST_F64) return launch_block_t<double, I, DEG, M, ST_F64>(a, nblocks, st); \
        if (s == ST_F32) return launch_block_t<float, I, DEG, M, ST_F32>(a, nblocks, st);  \
        return launch_block_t<float, I, DEG, M, ST_BF16X2>(a, nblocks, st);
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
