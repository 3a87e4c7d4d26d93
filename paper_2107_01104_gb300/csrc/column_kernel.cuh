// Column step kernel: persistent, warp-specialised, software-pipelined RK2 /
// Adams-Bashforth steps for float32 fields and kernel widths I = 4, 6.
//
// The paper distributes the particles in slabs along x3 and interpolates each
// slab against its own field slab plus ghost layers (Sec. 3.3.1).  Here a CTA
// takes work items from a counter; an item is a column segment: the cell
// blocks (bx, by, z0 .. z0 + nseg - 1) stacked along x3.  The CTA walks the
// segment slab by slab with the field halo kept in a ring of x3 planes:
// moving to the next slab brings in only BLK new planes (the other H - BLK
// planes are shared with the previous slab).
//
// Ring: R = H + BLK plane positions, plane z at position z mod R.  The BLK
// planes that slab s + 1 adds to the window of slab s land on positions that
// only slab s - 1 used (window(s) and the new planes of s + 1 together span
// H + BLK = R consecutive planes), so they can be copied as soon as slab s - 1
// is finished, while slab s is being interpolated.  Positions 0 .. I - 2 are
// mirrored at R .. R + I - 2, so every stencil reads I consecutive positions
// with the constant plane stride S3 of the block kernel's bank-conflict-free
// layout.
//
// Work inside a segment is a sequence of tasks: up to PBC particles of one
// slab (a slab with more particles has several tasks, an empty slab one empty
// task).  Two kinds of warps run the tasks as a pipeline:
//
//   particle warps (NPW: 1 for RK2, 2 for Adams-Bashforth, whose single
//     stencil per step leaves one warp's float64 work on the critical path):
//     warp w owns the tasks tau = w mod NPW.  For its task tau it prefetches
//     the positions (and AB history) of its task tau + 2 NPW by cp.async,
//     splits the positions of its task tau + NPW in float64 into the records
//     the interpolation warps read (P1), then, once task tau is interpolated,
//     does the float64 update, re-split and write-back of task tau (P3).  All
//     float64 work is lane-dense here.
//   interpolation warps (NQW warps): for task tau, wait for its records, on
//     the first task of a slab copy that slab's successor's new planes into
//     the ring (cp.async), then gather and contract the stencils, one warp
//     per particle (stage 1 and, for RK2, stage 2), and hand k1 (k2) to the
//     particle warp that owns the task.
//
// Hand-offs use NB = 2 NPW named barriers per direction (records and k values
// in NB buffers): REC[tau % NB] (the owning particle warp arrives,
// interpolation warps wait) and KV[tau % NB] (interpolation warps arrive, the
// owner waits).  Input slots rotate over NS = 3 NPW.
//
// Particle state is read from and written back to the same arrays, grouped
// by block beforehand (counting-sort scatter), so each task's inputs are
// contiguous.  Input buffers rotate over three slots.  The update phase also
// counts the new block keys for the next binning.
#pragma once

#include <algorithm>

#include "block_kernel.cuh"

namespace trk {

constexpr int PBC = 64;              // particles per task
constexpr int NQW_MAX = 10;          // interpolation warps at most (weight buffers)

// warp roles and buffer counts of a step mode
template <int MODE>
struct ColCfg {
    static constexpr int NPW = MODE == MODE_RK2 ? 1 : 2;   // particle warps
    static constexpr int NQW = 10;                           // interpolation warps
    static constexpr int NTC = (NQW + NPW) * 32;             // threads per CTA
    static constexpr int NQT = NQW * 32;
    static constexpr int NB = 2 * NPW;                       // record / k buffers, barriers per direction (power of 2)
    static constexpr int NS = 3 * NPW;                       // input slots
    static constexpr int BCNT = NQT + 32;                    // threads at a hand-off barrier
    static_assert(NQW <= NQW_MAX, "weight buffers");
    static_assert(NPW == 1 || NPW == 2, "one or two particle warps");
};

template <int I, int H>
struct RingGeom {
    static constexpr int R = H + BLK;    // plane positions
    static constexpr int M = I - 1;      // mirrored positions
    static constexpr int P = R + M;      // allocated planes per component
};

template <size_t RING_BYTES, bool AB2, int NB, int NS>
struct ColPlan {
    static constexpr size_t rec = align32(RING_BYTES);                                    // [NB][PBC] records
    static constexpr size_t cell = align32(rec + (size_t)NB * PBC * sizeof(PRec<float>));  // [NB][PBC]
    static constexpr size_t k = align32(cell + (size_t)NB * PBC * sizeof(int));           // [NB][6][PBC]
    static constexpr size_t w = align32(k + (size_t)NB * 6 * PBC * sizeof(float));         // [NQW_MAX][48]
    static constexpr size_t x = align32(w + (size_t)NQW_MAX * 48 * sizeof(float));         // [NS][3][PBC]
    static constexpr size_t rhs = align32(x + (size_t)NS * 3 * PBC * sizeof(double));      // [NS][3 AB_MAX_HIST][PBC]
    static constexpr size_t seg = align32(rhs + (AB2 ? (size_t)NS * 3 * AB_MAX_HIST * PBC * sizeof(float) : 0));
    static constexpr size_t total = seg + (size_t)2 * MAXSEG * sizeof(int);
};

template <int I, int MODE>
constexpr size_t column_smem_bytes()
{
    constexpr int MARGIN = (MODE == MODE_RK2) ? 1 : 0;
    constexpr int H = BLK + I - 1 + 2 * MARGIN;
    using RG = RingGeom<I, H>;
    using CC = ColCfg<MODE>;
    return ColPlan<(size_t)3 * RG::P * Layout<I, H>::S3 * sizeof(float), MODE == MODE_AB2, CC::NB, CC::NS>::total;
}

// named barriers (0 is __syncthreads): REC + 0 .. NB-1, then KV + 0 .. NB-1
constexpr int BAR_REC = 1;

// compile-time barrier ids (a runtime id makes ptxas reserve all sixteen)
template <int ID>
__device__ __forceinline__ void bar_sync(int count)
{
    asm volatile("bar.sync %0, %1;\n" ::"n"(ID), "r"(count) : "memory");
}
template <int ID>
__device__ __forceinline__ void bar_arrive(int count)
{
    asm volatile("bar.arrive %0, %1;\n" ::"n"(ID), "r"(count) : "memory");
}
// barrier BASE + i, 0 <= i < NB (NB = 2 or 4)
template <int BASE, int NB>
__device__ __forceinline__ void bar_sync_idx(int i, int count)
{
    static_assert(NB == 2 || NB == 4, "two or four buffers");
    if constexpr (NB == 2) {
        if (i == 0) bar_sync<BASE>(count);
        else bar_sync<BASE + 1>(count);
    } else {
        if (i == 0) bar_sync<BASE>(count);
        else if (i == 1) bar_sync<BASE + 1>(count);
        else if (i == 2) bar_sync<BASE + 2>(count);
        else bar_sync<BASE + 3>(count);
    }
}
template <int BASE, int NB>
__device__ __forceinline__ void bar_arrive_idx(int i, int count)
{
    static_assert(NB == 2 || NB == 4, "two or four buffers");
    if constexpr (NB == 2) {
        if (i == 0) bar_arrive<BASE>(count);
        else bar_arrive<BASE + 1>(count);
    } else {
        if (i == 0) bar_arrive<BASE>(count);
        else if (i == 1) bar_arrive<BASE + 1>(count);
        else if (i == 2) bar_arrive<BASE + 2>(count);
        else bar_arrive<BASE + 3>(count);
    }
}

// A task: particles [j0, j0 + n) of slab s; first = first task of the slab.
struct Task {
    int s, j0, n;
    bool first;
};

__device__ __forceinline__ Task first_task(const int* s_beg, const int* s_end)
{
    return Task{0, s_beg[0], min(s_end[0] - s_beg[0], PBC), true};
}

// s == nseg marks the end of the segment
__device__ __forceinline__ Task next_task(const Task& t, const int* s_beg, const int* s_end, int nseg)
{
    if (t.s >= nseg) return t;
    if (t.j0 + PBC < s_end[t.s]) return Task{t.s, t.j0 + PBC, min(s_end[t.s] - (t.j0 + PBC), PBC), false};
    const int s = t.s + 1;
    if (s >= nseg) return Task{nseg, 0, 0, false};
    return Task{s, s_beg[s], min(s_end[s] - s_beg[s], PBC), true};
}

template <int I, int DEG, int MODE>
__global__ void __launch_bounds__(ColCfg<MODE>::NTC, 2) k_column(const __grid_constant__ ColumnArgs ca)
{
    using T = float;
    static_assert(MODE == MODE_RK2 || MODE == MODE_AB2, "column kernel: time steps only");
    constexpr bool IS_AB2 = MODE == MODE_AB2;
    constexpr int MARGIN = (MODE == MODE_RK2) ? 1 : 0;
    constexpr int H = BLK + I - 1 + 2 * MARGIN;
    constexpr int G = I / 2 - 1 + MARGIN;
    constexpr int LO = I / 2 - 1;
    constexpr int RMAX = H - 1 - I / 2;
    using Lay = Layout<I, H>;
    constexpr int S2 = Lay::S2, S3 = Lay::S3;
    using RG = RingGeom<I, H>;
    constexpr int R = RG::R, M = RG::M;
    constexpr int SC = RG::P * S3;                 // ring component stride
    using CC = ColCfg<MODE>;
    constexpr int NPW = CC::NPW, NQW = CC::NQW, NB = CC::NB, NS = CC::NS, BCNT = CC::BCNT;
    constexpr int BAR_KV = BAR_REC + NB;
    using CP = ColPlan<(size_t)3 * SC * sizeof(T), IS_AB2, NB, NS>;
    using SL = SmemLd<T, S2, S3, SC>;
    static_assert(H - I < R && H * H <= CC::NQT, "ring geometry");
    static_assert(BAR_KV + NB <= 16, "named barriers");

    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ int s_item;
    T* ring = reinterpret_cast<T*>(smem_raw);
    PRec<T>* p_rec = reinterpret_cast<PRec<T>*>(smem_raw + CP::rec);   // [NB][PBC]
    int* p_cell = reinterpret_cast<int*>(smem_raw + CP::cell);          // [NB][PBC]
    T* p_k = reinterpret_cast<T*>(smem_raw + CP::k);                    // [NB][6][PBC]
    T* wbuf = reinterpret_cast<T*>(smem_raw + CP::w);                   // [NQW][48]
    double* p_x = reinterpret_cast<double*>(smem_raw + CP::x);          // [NS][3][PBC]
    float* p_rhs = reinterpret_cast<float*>(smem_raw + CP::rhs);        // [NS][3 AB_MAX_HIST][PBC] (AB)
    int* s_beg = reinterpret_cast<int*>(smem_raw + CP::seg);            // [MAXSEG]
    int* s_end = s_beg + MAXSEG;                                        // [MAXSEG]

    const BlockArgs& a = ca.a;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool pwarp = warp >= NQW;                                     // a particle warp
    const int mask = a.g.mask, nb1 = a.g.nb1, nb2 = a.g.nb2;
    const int64_t np = a.np;
    const double inv_delta = a.g.inv_delta;
    const int64_t NP2 = (int64_t)a.f.NP * a.f.NP;
    const int nseg = ca.nseg;

    for (;;) {
        if (tid == 0) s_item = atomicAdd(ca.ctr, 1);
        __syncthreads();
        const int64_t item = s_item;
        __syncthreads();
        if (item >= ca.nitems) break;
        const int64_t ncol = (int64_t)nb1 * nb2;
        const int col = (int)(item % ncol);
        const int z0 = (int)(item / ncol) * nseg;                    // first slab (block index along x3)
        const int bx = col % nb1, by = col / nb1;
        const int o1 = bx * BLK - G, o2 = by * BLK - G;
        bool any = false;
        if (tid < nseg) {
            const int64_t b = ((int64_t)(z0 + tid) * nb2 + by) * nb1 + bx;
            s_beg[tid] = a.offsets[b];
            s_end[tid] = a.offsets[b + 1];
            any = s_end[tid] > s_beg[tid];
        }
        if (!__syncthreads_or(any)) continue;                        // empty segment
        const int za0 = z0 * BLK - G;                                // first window plane of slab 0

        if (pwarp) {
            // =========================== particle warp ===========================
            auto issue_inputs = [&](const Task& t, int slot) {
#pragma unroll
                for (int h = 0; h < PBC / 32; ++h) {
                    const int i = lane + 32 * h;
                    if (i < t.n) {
#pragma unroll
                        for (int ax = 0; ax < 3; ++ax) {
                            const uint32_t d =
                                (uint32_t)__cvta_generic_to_shared(p_x + (slot * 3 + ax) * PBC + i);
                            cp_async_elem<double>(d, a.pos_out + ax * np + t.j0 + i);
                        }
                        if constexpr (IS_AB2) {   // the valid AB history rows
                            for (int r = 0; r < 3 * a.history_valid; ++r) {
                                const uint32_t dr = (uint32_t)__cvta_generic_to_shared(
                                    p_rhs + (slot * 3 * AB_MAX_HIST + r) * PBC + i);
                                cp_async_elem<float>(dr, a.rhs_out + r * np + t.j0 + i);
                            }
                        }
                    }
                }
                asm volatile("cp.async.commit_group;\n" ::: "memory");
            };
            // P1: split the positions of task t (input slot) into record buffer rb
            auto p1 = [&](const Task& t, int slot, int rb) {
                const int o3 = (z0 + t.s) * BLK - G;
#pragma unroll
                for (int h = 0; h < PBC / 32; ++h) {
                    const int i = lane + 32 * h;
                    if (i >= t.n) continue;
                    bool ok = true;
                    int c[3];
                    PRec<T> rec;
#pragma unroll
                    for (int ax = 0; ax < 3; ++ax) {
                        double tt;
                        ok &= split_axis(p_x[(slot * 3 + ax) * PBC + i], inv_delta, mask, c[ax], tt);
                        rec.t[ax] = (T)tt;
                    }
                    if (!ok) atomicOr(a.flags + FLAG_NONFINITE, 1);
                    // a particle lies in its own block; the clamp only keeps corrupted input inside the window
                    const int r1 = min(max((c[0] - o1) & mask, LO), RMAX);
                    const int r2 = min(max((c[1] - o2) & mask, LO), RMAX);
                    const int r3 = min(max((c[2] - o3) & mask, LO), RMAX);
                    rec.relf = __int_as_float(pack_rel(r1, r2, r3));
                    p_rec[rb * PBC + i] = rec;
                    p_cell[rb * PBC + i] = pack_cell(c[0], c[1], c[2]);
                }
            };
            // P3: update, re-split and write back task t from k buffer kb and input slot
            auto p3 = [&](const Task& t, int slot, int kb) {
                const T* kk = p_k + kb * 6 * PBC;
#pragma unroll
                for (int h = 0; h < PBC / 32; ++h) {
                    const int i = lane + 32 * h;
                    const unsigned valid = __ballot_sync(0xffffffffu, i < t.n);
                    if (i >= t.n) continue;
                    const int64_t j = (int64_t)t.j0 + i;
                    int cn[3];
                    bool ok = true;
#pragma unroll
                    for (int ax = 0; ax < 3; ++ax) {
                        const double k1 = (double)kk[ax * PBC + i];
                        const double x0 = p_x[(slot * 3 + ax) * PBC + i];
                        double xn;
                        if constexpr (MODE == MODE_RK2) {
                            const double k2 = (double)kk[(3 + ax) * PBC + i];
                            xn = x0 + (0.5 * a.dt) * (k1 + k2);
                        } else {   // ABk, order min(k, 1 + history)
                            const float* hs = p_rhs + slot * 3 * AB_MAX_HIST * PBC + i;
                            const int q = min(a.ab_order, a.history_valid + 1);
                            const double inc =
                                ab_increment(q, k1, [&](int e) { return (double)hs[(3 * e + ax) * PBC]; });
                            xn = x0 + a.dt * inc;
                            // new history in place: u_n, then the valid older entries shifted by one
                            a.rhs_out[ax * np + j] = (float)k1;
                            for (int e = 1; e < a.ab_order - 1; ++e)
                                a.rhs_out[(3 * e + ax) * np + j] = e - 1 < a.history_valid ? hs[(3 * (e - 1) + ax) * PBC] : 0.0f;
                        }
                        ok &= split_cell(xn, inv_delta, mask, cn[ax]);
                        a.pos_out[ax * np + j] = xn;
                    }
                    if (!ok) atomicOr(a.flags + FLAG_NONFINITE, 1);
                    const uint32_t key = block_key(a.g, cn[0], cn[1], cn[2]);
                    a.key_out[j] = key;
                    if (ca.counts) {   // block counts of the next binning, one add per group of equal keys
                        const unsigned peers = __match_any_sync(valid, key);
                        if (lane == __ffs(peers) - 1) atomicAdd(ca.counts + key, (uint32_t)__popc(peers));
                    }
                }
            };

            // this warp's tasks: tau = pw, pw + NPW, pw + 2 NPW, ...
            const unsigned pw = NPW == 1 ? 0u : (unsigned)(warp - NQW);
            auto adv = [&](Task t) {
#pragma unroll
                for (int i = 0; i < NPW; ++i) t = next_task(t, s_beg, s_end, nseg);
                return t;
            };
            Task t0 = first_task(s_beg, s_end);
            if (NPW > 1 && pw > 0) t0 = next_task(t0, s_beg, s_end, nseg);
            Task t1 = adv(t0);
            Task t2 = adv(t1);
            unsigned tau = pw;
            issue_inputs(t0, tau % NS);                // empty groups for end markers
            issue_inputs(t1, (tau + NPW) % NS);
            asm volatile("cp.async.wait_group 1;\n" ::: "memory");
            __syncwarp();
            if (t0.s < nseg) {
                p1(t0, tau % NS, tau & (NB - 1));
                __syncwarp();
                bar_arrive_idx<BAR_REC, NB>(tau & (NB - 1), BCNT);
            }
            for (; t0.s < nseg; tau += NPW) {
                // inputs of tau + 2 NPW (their slot was last read by P3 of tau - NPW)
                if (t2.s < nseg) issue_inputs(t2, (tau + 2 * NPW) % NS);
                else asm volatile("cp.async.commit_group;\n" ::: "memory");
                if (t1.s < nseg) {
                    asm volatile("cp.async.wait_group 1;\n" ::: "memory");   // inputs of tau + NPW
                    __syncwarp();
                    // record buffer (tau + NPW) % NB was last read for task tau - NPW (its KV is passed)
                    p1(t1, (tau + NPW) % NS, (tau + NPW) & (NB - 1));
                    __syncwarp();
                    bar_arrive_idx<BAR_REC, NB>((tau + NPW) & (NB - 1), BCNT);
                }
                bar_sync_idx<BAR_KV, NB>(tau & (NB - 1), BCNT);                // task tau interpolated
                p3(t0, tau % NS, tau & (NB - 1));
                t0 = t1;
                t1 = t2;
                t2 = adv(t2);
            }
            asm volatile("cp.async.wait_all;\n" ::: "memory");
        } else {
            // ======================== interpolation warps ========================
            T* wv = wbuf + warp * 48;
            T* wd = wv + 24;
            WeightEval<T, I, DEG, false> W;
            W.init(a.cf, lane);
            Lane<T, I, false> L;
            L.init(lane);
            const T dtid = (T)(a.dt * inv_delta);
            const int rcomp = ((lane & 16) ? 2 : 0) + ((lane & 8) ? 1 : 0);   // component held after reduce4
            const bool writer = (lane & 7) == 0 && rcomp < 3;                 // lanes 0, 8, 16
            // copy slot of this thread in a halo plane: column cx, row cy (lanes along x1)
            const int cx = tid % H, cy = tid / H;
            const bool copier = cy < H;
            const uint32_t ring_s =
                (uint32_t)__cvta_generic_to_shared(ring) + (uint32_t)((cy * S2 + cx) * (int)sizeof(T));
            const float* gxy = a.f.f32 + (int64_t)(o2 + PAD + cy) * a.f.NP + (o1 + PAD + cx);

            // cnt field planes from absolute plane za on, into ring positions za mod R (and mirrors)
            auto issue_planes = [&](int za, int cnt) {
                if (copier) {
                    int p = (za % R + R) % R;
                    const float* gz = gxy + (int64_t)(za + PAD) * NP2;
                    for (int qz = 0; qz < cnt; ++qz) {
#pragma unroll
                        for (int k = 0; k < 3; ++k) {
                            cp_async_elem<T>(ring_s + (uint32_t)((k * SC + p * S3) * (int)sizeof(T)),
                                             gz + k * a.f.plane);
                            if (p < M)
                                cp_async_elem<T>(ring_s + (uint32_t)((k * SC + (p + R) * S3) * (int)sizeof(T)),
                                                 gz + k * a.f.plane);
                        }
                        gz += NP2;
                        p = p + 1 == R ? 0 : p + 1;
                    }
                }
                asm volatile("cp.async.commit_group;\n" ::: "memory");
            };

            issue_planes(za0, H);                                   // window of slab 0
            asm volatile("cp.async.wait_all;\n" ::: "memory");
            Task t = first_task(s_beg, s_end);
            for (unsigned tau = 0; t.s < nseg; ++tau) {
                bar_sync_idx<BAR_REC, NB>(tau & (NB - 1), BCNT);   // records of tau ready; every warp is done with tau - 1
                if (t.first && t.s + 1 < nseg) issue_planes(za0 + (t.s + 1) * BLK + H - BLK, BLK);
                const int rb = tau & (NB - 1);
                const PRec<T>* recs = p_rec + rb * PBC;
                const int* cells = p_cell + rb * PBC;
                T* kk = p_k + rb * 6 * PBC;
                const int o3 = (z0 + t.s) * BLK - G;
                const int wpos = (o3 % R + R) % R;                  // ring position of window plane 0
                for (int q = warp; q < t.n; q += NQW) {
                    const PRec<T> rec = recs[q];
                    const int rp = __float_as_int(rec.relf);
                    const T t1 = rec.t[0], t2 = rec.t[1], t3 = rec.t[2];
                    const int r1 = rp & 255, r2 = (rp >> 8) & 255, r3 = (rp >> 16) & 255;
                    int pa = wpos + r3 - LO;
                    pa = pa >= R ? pa - R : pa;
                    L.load(SL{ring + pa * S3 + (r2 - LO) * S2 + (r1 - LO)});
                    W.eval(t1 - (T)0.5, t2 - (T)0.5, t3 - (T)0.5, wv, wd);
                    T acc[12];
                    L.contract(wv, wd, acc);
                    const T m = reduce4(acc, lane);
                    if constexpr (MODE == MODE_RK2) {
                        const T k1[3] = {__shfl_sync(0xffffffffu, m, 0), __shfl_sync(0xffffffffu, m, 8),
                                         __shfl_sync(0xffffffffu, m, 16)};
                        // stage-2 point, cell-relative: t* = t + dt k1 / delta
                        T ts[3] = {fma(dtid, k1[0], t1), fma(dtid, k1[1], t2), fma(dtid, k1[2], t3)};
                        int dc[3];
#pragma unroll
                        for (int ax = 0; ax < 3; ++ax) {
                            const T fl = floor(ts[ax]);
                            dc[ax] = (int)fl;
                            ts[ax] -= fl;
                        }
                        if ((dc[0] | dc[1] | dc[2]) != 0) {
                            const int s1 = r1 + dc[0], s2 = r2 + dc[1], s3 = r3 + dc[2];
                            const bool in =
                                s1 >= LO && s1 <= RMAX && s2 >= LO && s2 <= RMAX && s3 >= LO && s3 <= RMAX;
                            if (in) {
                                int pb = wpos + s3 - LO;
                                pb = pb >= R ? pb - R : pb;
                                L.load(SL{ring + pb * S3 + (s2 - LO) * S2 + (s1 - LO)});
                            } else {
                                if (lane == 0) atomicOr(a.flags + FLAG_CFL, 1);
                                const int pc = cells[q];
                                L.load(global_ld<T, ST_F32, I>(a.f, ((pc & 1023) + dc[0]) & mask,
                                                               (((pc >> 10) & 1023) + dc[1]) & mask,
                                                               (((pc >> 20) & 1023) + dc[2]) & mask, 0, 2));
                            }
                        }
                        W.eval(ts[0] - (T)0.5, ts[1] - (T)0.5, ts[2] - (T)0.5, wv, wd);
                        L.contract(wv, wd, acc);
                        const T m2 = reduce4(acc, lane);
                        if (writer) {
                            kk[rcomp * PBC + q] = rcomp == 0 ? k1[0] : (rcomp == 1 ? k1[1] : k1[2]);
                            kk[(3 + rcomp) * PBC + q] = m2;
                        }
                    } else {
                        if (writer) kk[rcomp * PBC + q] = m;
                    }
                }
                bar_arrive_idx<BAR_KV, NB>(tau & (NB - 1), BCNT);    // k of tau ready
                const Task tn = next_task(t, s_beg, s_end, nseg);
                // the next slab's planes (copied at the start of this slab) must have landed
                // before its first task; the barrier that opens that task publishes them
                if (tn.first) asm volatile("cp.async.wait_all;\n" ::: "memory");
                t = tn;
            }
        }
    }
}

template <int I, int DEG, int MODE>
cudaError_t launch_column_t(const ColumnArgs& ca, int nsm, cudaStream_t st)
{
    constexpr size_t smem = column_smem_bytes<I, MODE>();
    static_assert(smem <= 232448, "column shared-memory plan exceeds the per-block limit");
    auto kern = k_column<I, DEG, MODE>;
    static int grid_per_sm = 0;
    if (!grid_per_sm) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int occ = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, ColCfg<MODE>::NTC, smem);
        if (e != cudaSuccess) return e;
        grid_per_sm = occ > 0 ? occ : 1;
    }
    if (ca.nitems <= 0) return cudaSuccess;
    const int64_t grid = std::min<int64_t>(ca.nitems, (int64_t)grid_per_sm * nsm);
    kern<<<(unsigned)grid, ColCfg<MODE>::NTC, smem, st>>>(ca);
    return cudaGetLastError();
}

template <int I, int DEG>
cudaError_t dispatch_column(int mode, const ColumnArgs& ca, int nsm, cudaStream_t st)
{
    if (mode == MODE_RK2) return launch_column_t<I, DEG, MODE_RK2>(ca, nsm, st);
    if (mode == MODE_AB2) return launch_column_t<I, DEG, MODE_AB2>(ca, nsm, st);
    return cudaErrorInvalidValue;
}

}  // namespace trk
