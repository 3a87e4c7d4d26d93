// Discrete adjoint of one RK2 (Heun) step, per cell block.
//
// Forward map (Eq. tracers, RK2): X* = X + dt u(X), X' = X + dt/2 (u(X) + u(X*)).
// Given lambda = dLoss/dX' per particle, with J = du/dX and W(X) the linear
// map from the field to u(X) (weights beta x beta x beta of Eq. triple_sum):
//   lambda* = dt/2 J(X*)^T lambda
//   mu      = dt/2 lambda + dt lambda*
//   lambda <- lambda + lambda* + J(X)^T mu                      (dLoss/dX)
//   gfield += W(X)^T mu + W(X*)^T (dt/2 lambda)                (dLoss/dfield)
// The paper has no adjoint; this is the transpose of its interpolation and
// time step, written for gradient-based use of the tracker.
//
// Phases (one CTA per block, as the forward block kernel):
//   P1  thread per particle: split X, load lambda (float64)
//   Q1  warp per particle: gathers at X and X* with value and derivative
//       weights -> u(X), J(X), J(X*)
//   P2  thread per particle: the float64 lambda recurrence above
// Modes (AM): ADJ_SLAB and ADJ_SMEM run one CTA per cell block with the
// field halo staged in shared memory; ADJ_DIRECT (sparse particle sets, a null
// a.offsets) runs PBA sorted particles per CTA and gathers every stencil from
// global memory, like the forward direct kernel.
//
//   Q2  warp per particle: W^T scatter.  With scratch (ADJ_SLAB): atomic adds
//       straight into the block's slab of gscratch, [3][H][H][H] (float32 /
//       float64 adds are native reductions in L2; shared-memory float adds on
//       this GPU are compare-and-swap loops), summed per node afterwards by
//       k_adj_gather in a fixed cross-block order; the slabs are zero on
//       entry and the gather leaves them zero.  Without scratch: a shared-
//       memory accumulator laid out like the halo (the halo buffer is
//       re-used), flushed with one float64 atomic add per touched halo node
//       into gfield (ADJ_SMEM).  ADJ_DIRECT adds straight into gfield, one
//       float64 atomic per stencil node (one for both stages when X and X*
//       share a cell).  Inside a block the adds arrive in any order.
#pragma once

#include "block_kernel.cuh"

namespace trk {

constexpr int PBA = 128;   // particles per adjoint batch (keeps the float64 I = 8 plan under 227 KB)

enum { ADJ_SMEM = 0, ADJ_SLAB = 1, ADJ_DIRECT = 2 };   // where the W^T scatter goes (see above)

// two-element vector of T for zeroing shared memory
template <typename T>
struct Vec2;
template <>
struct Vec2<float> {
    using type = float2;
    __device__ static float2 zero() { return make_float2(0.0f, 0.0f); }
};
template <>
struct Vec2<double> {
    using type = double2;
    __device__ static double2 zero() { return make_double2(0.0, 0.0); }
};

template <typename T, int SC>
struct AdjPlan {
    static constexpr size_t rec = align32((size_t)3 * SC * sizeof(T));
    static constexpr size_t rec2 = align32(rec + PBA * sizeof(PRec<T>));
    static constexpr size_t jac = align32(rec2 + PBA * sizeof(PRec<T>));         // [PBA][18] J(X), J(X*)
    static constexpr size_t mu = align32(jac + (size_t)PBA * 18 * sizeof(T));    // [PBA][6]  mu, dt/2 lambda
    static constexpr size_t w = align32(mu + (size_t)PBA * 6 * sizeof(T));
    static constexpr size_t cell = align32(w + (size_t)NW * 48 * sizeof(T));     // [PBA] cells at X
    static constexpr size_t cell2 = cell + PBA * sizeof(int);                    // [PBA] cells at X*
    static constexpr size_t total = cell2 + PBA * sizeof(int);
    static_assert(total <= 232448, "adjoint shared-memory plan exceeds the per-block limit");
};

template <typename T, int I, int DEG, int STORE, int AM>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? 2 : 1) k_adjoint(const __grid_constant__ AdjArgs a)
{
    constexpr bool HALO = AM != ADJ_DIRECT;
    constexpr int H = BLK + I - 1 + 2;
    constexpr int G = I / 2;
    constexpr int LO = I / 2 - 1;
    constexpr int RMAX = H - 1 - I / 2;
    using Lay = Layout<I, H>;
    constexpr int S2 = Lay::S2, S3 = Lay::S3, SC = Lay::SC;
    using SL = SmemLd<T, S2, S3, SC>;
    using SM = AdjPlan<T, SC>;

    extern __shared__ __align__(128) unsigned char smem_raw[];
    T* halo = reinterpret_cast<T*>(smem_raw);                     // field, then the W^T accumulator
    PRec<T>* p_rec = reinterpret_cast<PRec<T>*>(smem_raw + SM::rec);
    PRec<T>* p_rec2 = reinterpret_cast<PRec<T>*>(smem_raw + SM::rec2);
    T* p_jac = reinterpret_cast<T*>(smem_raw + SM::jac);
    T* p_mu = reinterpret_cast<T*>(smem_raw + SM::mu);
    T* wbuf = reinterpret_cast<T*>(smem_raw + SM::w);
    int* p_cell = reinterpret_cast<int*>(smem_raw + SM::cell);
    int* p_cell2 = reinterpret_cast<int*>(smem_raw + SM::cell2);

    const int b = HALO ? (int)blockIdx.x : 0;
    const int j0 = HALO ? a.offsets[b] : (int)blockIdx.x * PBA;
    const int j1 = HALO ? a.offsets[b + 1] : (int)min((int64_t)j0 + PBA, a.np);
    if (j0 >= j1) return;

    const int N = a.g.N, mask = a.g.mask;
    const int nb1 = a.g.nb1, nb2 = a.g.nb2;
    const int bx = b % nb1, by = (b / nb1) % nb2, bz = b / (nb1 * nb2);
    const int o1 = bx * BLK - G, o2 = by * BLK - G, o3 = bz * BLK - G;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t np = a.np;
    const double inv_delta = a.g.inv_delta;
    const double dt = a.dt;
    T* wv = wbuf + warp * 48;
    T* wd = wv + 24;
    const T dtid = (T)(dt * inv_delta);

    WeightEval<T, I, DEG, true> W;
    W.init(table<T>(a), lane);
    Lane<T, I, true> L;
    L.init(lane);

    constexpr bool ASYNC = STORE != ST_BF16X2;
    for (int batch = j0; batch < j1; batch += PBA) {
        const int nbat = min(PBA, j1 - batch);
        // the first batch's halo copies run while P1 splits (later batches re-use the
        // halo buffer as the previous batch's accumulator until it is flushed)
        if (HALO && ASYNC && batch == j0) stage_halo<T, STORE, H, G, S2, S3, SC, 3, false>(halo, a.f, 0, 3, o1, o2, o3);
        // ---------------- P1 ----------------
        double lam[3] = {0, 0, 0};
        int id = 0;
        if (tid < nbat) {
            id = a.perm[batch + tid];
            bool ok = true;
            int c[3];
            PRec<T> rec;
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) {
                double t;
                ok &= split_axis(a.pos[ax * np + id], inv_delta, mask, c[ax], t);
                rec.t[ax] = (T)t;
                lam[ax] = a.lam_in[ax * np + id];
            }
            if (!ok) atomicOr(a.flags + FLAG_NONFINITE, 1);
            const int r1 = (c[0] - o1) & mask, r2 = (c[1] - o2) & mask, r3 = (c[2] - o3) & mask;
            const bool in = HALO && r1 >= LO && r1 <= RMAX && r2 >= LO && r2 <= RMAX && r3 >= LO && r3 <= RMAX;
            const int rp = in ? pack_rel(r1, r2, r3) : -1;
            if constexpr (sizeof(T) == 4) rec.relf = __int_as_float(rp);
            else rec.relf = __longlong_as_double((long long)rp);
            p_rec[tid] = rec;
            p_cell[tid] = pack_cell(c[0], c[1], c[2]);
        }
        if (batch != j0) __syncthreads();   // the accumulator of the previous batch is flushed
        if constexpr (HALO) {
            if (!ASYNC || batch != j0) stage_halo<T, STORE, H, G, S2, S3, SC, 3, true>(halo, a.f, 0, 3, o1, o2, o3);
            else cp_async_wait_all();
        }
        __syncthreads();
        // ---------------- Q1: u(X), J(X), J(X*) ----------------
        for (int q = warp; q < nbat; q += NW) {
            const PRec<T> rec = p_rec[q];
            int rp;
            if constexpr (sizeof(T) == 4) rp = __float_as_int(rec.relf);
            else rp = (int)__double_as_longlong(rec.relf);
            const int r1 = rp & 255, r2 = (rp >> 8) & 255, r3 = (rp >> 16) & 255;
            const int pc = p_cell[q];
            const int c1 = pc & 1023, c2 = (pc >> 10) & 1023, c3 = (pc >> 20) & 1023;
            if (rp >= 0) L.load(SL{halo + (r3 - LO) * S3 + (r2 - LO) * S2 + (r1 - LO)});
            else L.load(global_ld<T, STORE, I>(a.f, c1, c2, c3, 0, 2));
            W.eval(rec.t[0] - (T)0.5, rec.t[1] - (T)0.5, rec.t[2] - (T)0.5, wv, wd);
            T acc[12];
            L.contract(wv, wd, acc);
            T m = reduce16(acc, lane);        // value v sits in lanes 2v and 2v + 1
            const T k1[3] = {__shfl_sync(0xffffffffu, m, 0), __shfl_sync(0xffffffffu, m, 2),
                             __shfl_sync(0xffffffffu, m, 4)};
            const int v = lane >> 1;
            if ((lane & 1) == 0 && v >= 3 && v < 12) p_jac[q * 18 + (v - 3)] = m * (T)inv_delta;
            // stage-2 point, cell-relative: t* = t + dt k1 / delta
            T ts[3] = {fma(dtid, k1[0], rec.t[0]), fma(dtid, k1[1], rec.t[1]), fma(dtid, k1[2], rec.t[2])};
            int dc[3];
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) {
                const T fl = floor(ts[ax]);
                dc[ax] = (int)fl;
                ts[ax] -= fl;
            }
            const int s1 = r1 + dc[0], s2 = r2 + dc[1], s3 = r3 + dc[2];
            const bool in2 = rp >= 0 && s1 >= LO && s1 <= RMAX && s2 >= LO && s2 <= RMAX && s3 >= LO && s3 <= RMAX;
            const int cs1 = (c1 + dc[0]) & mask, cs2 = (c2 + dc[1]) & mask, cs3 = (c3 + dc[2]) & mask;
            // (direct: in the same cell the stage-1 stencil in L is re-used)
            if ((dc[0] | dc[1] | dc[2]) != 0 || (HALO && rp < 0)) {
                if (in2) {
                    L.load(SL{halo + (s3 - LO) * S3 + (s2 - LO) * S2 + (s1 - LO)});
                } else {
                    // left the staged halo, or (direct) moved more than one cell
                    const bool far = HALO || abs(dc[0]) > 1 || abs(dc[1]) > 1 || abs(dc[2]) > 1;
                    if (far && lane == 0) atomicOr(a.flags + FLAG_CFL, 1);
                    L.load(global_ld<T, STORE, I>(a.f, cs1, cs2, cs3, 0, 2));
                }
            }
            W.eval(ts[0] - (T)0.5, ts[1] - (T)0.5, ts[2] - (T)0.5, wv, wd);
            L.contract(wv, wd, acc);
            m = reduce16(acc, lane);
            if ((lane & 1) == 0 && v >= 3 && v < 12) p_jac[q * 18 + 9 + (v - 3)] = m * (T)inv_delta;
            if (lane == 0) {
                PRec<T> r2c;
                r2c.t[0] = ts[0];
                r2c.t[1] = ts[1];
                r2c.t[2] = ts[2];
                const int rp2 = in2 ? pack_rel(s1, s2, s3) : -1;
                if constexpr (sizeof(T) == 4) r2c.relf = __int_as_float(rp2);
                else r2c.relf = __longlong_as_double((long long)rp2);
                p_rec2[q] = r2c;
                p_cell2[q] = pack_cell(cs1, cs2, cs3);
            }
        }
        __syncthreads();
        // ---------------- P2: lambda recurrence (float64) ----------------
        if (tid < nbat) {
            const T* Jx = p_jac + tid * 18;        // J(X)[k][j] at 3k + j
            const T* Js = Jx + 9;                  // J(X*)
            double ls[3], mu[3];
#pragma unroll
            for (int jj = 0; jj < 3; ++jj) {
                double s2 = 0;
#pragma unroll
                for (int k = 0; k < 3; ++k) s2 += (double)Js[3 * k + jj] * lam[k];
                ls[jj] = 0.5 * dt * s2;
            }
#pragma unroll
            for (int k = 0; k < 3; ++k) mu[k] = 0.5 * dt * lam[k] + dt * ls[k];
#pragma unroll
            for (int jj = 0; jj < 3; ++jj) {
                double s1 = 0;
#pragma unroll
                for (int k = 0; k < 3; ++k) s1 += (double)Jx[3 * k + jj] * mu[k];
                a.lam_out[jj * np + id] = lam[jj] + ls[jj] + s1;
            }
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                p_mu[tid * 6 + k] = (T)mu[k];
                p_mu[tid * 6 + 3 + k] = (T)(0.5 * dt * lam[k]);
            }
        }
        if (!a.gfield) {
            __syncthreads();
            continue;
        }
        // ---------------- Q2: W^T scatter ----------------
        if constexpr (AM != ADJ_SMEM) {
            __syncthreads();   // p_mu of every particle
            constexpr int H3 = H * H * H;
            T* slab = reinterpret_cast<T*>(a.gscratch) + (int64_t)b * 3 * H3;
            // the adds of a stencil at packed halo-relative cell rp
            auto add_slab = [&](int rp) {
                T* base = slab + (((rp >> 16) & 255) - LO) * H * H + (((rp >> 8) & 255) - LO) * H + ((rp & 255) - LO);
                return [=](int k, int a1, int a2, int a3, T val) { atomicAdd(base + k * H3 + (a3 * H + a2) * H + a1, val); };
            };
            const int64_t NN3g = (int64_t)N * N * N;
            for (int q = warp; q < nbat; q += NW) {
                const PRec<T> recs[2] = {p_rec[q], p_rec2[q]};
                int rps[2];
#pragma unroll
                for (int stage = 0; stage < 2; ++stage) {
                    if constexpr (sizeof(T) == 4) rps[stage] = __float_as_int(recs[stage].relf);
                    else rps[stage] = (int)__double_as_longlong(recs[stage].relf);
                }
                const T mus[2][3] = {{p_mu[q * 6 + 0], p_mu[q * 6 + 1], p_mu[q * 6 + 2]},
                                     {p_mu[q * 6 + 3], p_mu[q * 6 + 4], p_mu[q * 6 + 5]}};
                const bool same = HALO ? (rps[0] >= 0 && rps[0] == rps[1]) : p_cell[q] == p_cell2[q];
                if (same) {
                    // X and X* in the same cell: one stencil, both weight sets, one add per node
                    const T sa[3] = {recs[0].t[0] - (T)0.5, recs[0].t[1] - (T)0.5, recs[0].t[2] - (T)0.5};
                    const T sb[3] = {recs[1].t[0] - (T)0.5, recs[1].t[1] - (T)0.5, recs[1].t[2] - (T)0.5};
                    W.eval_values2(sa, sb, wv, wd);
                    if constexpr (HALO) {
                        L.template scatter_n<true>(wv, mus[0], wd, mus[1], add_slab(rps[0]));
                    } else {
                        const int pc = p_cell[q];
                        const int c1 = pc & 1023, c2 = (pc >> 10) & 1023, c3 = (pc >> 20) & 1023;
                        double* gf = a.gfield;
                        L.template scatter_n<true>(wv, mus[0], wd, mus[1], [&](int k, int a1, int a2, int a3, T val) {
                            const int x1 = (c1 + a1 - LO) & mask, x2 = (c2 + a2 - LO) & mask, x3 = (c3 + a3 - LO) & mask;
                            atomicAdd(gf + k * NN3g + ((int64_t)x3 * N + x2) * N + x1, (double)val);
                        });
                    }
                    continue;
                }
#pragma unroll
                for (int stage = 0; stage < 2; ++stage) {
                    const PRec<T>& rec = recs[stage];
                    const int rp = rps[stage];
                    W.eval(rec.t[0] - (T)0.5, rec.t[1] - (T)0.5, rec.t[2] - (T)0.5, wv, wd);
                    if (HALO && rp >= 0) {
                        L.template scatter_n<false>(wv, mus[stage], wv, mus[stage], add_slab(rp));
                    } else {
                        const int pc = stage == 0 ? p_cell[q] : p_cell2[q];
                        const int c1 = pc & 1023, c2 = (pc >> 10) & 1023, c3 = (pc >> 20) & 1023;
                        double* gf = a.gfield;
                        L.template scatter_n<false>(wv, mus[stage], wv, mus[stage],
                                                    [&](int k, int a1, int a2, int a3, T val) {
                            const int x1 = (c1 + a1 - LO) & mask, x2 = (c2 + a2 - LO) & mask, x3 = (c3 + a3 - LO) & mask;
                            atomicAdd(gf + k * NN3g + ((int64_t)x3 * N + x2) * N + x1, (double)val);
                        });
                    }
                }
            }
            __syncthreads();   // the batch's records are read before the next batch's P1
            continue;
        }
        static_assert(SC % 2 == 0, "the accumulator is zeroed two values at a time");
        for (int e = tid; e < 3 * SC / 2; e += NT) reinterpret_cast<typename Vec2<T>::type*>(halo)[e] = Vec2<T>::zero();
        __syncthreads();
        const int64_t NN3 = (int64_t)N * N * N;
        auto add_smem = [&](T* base) {
            return [=](int k, int a1, int a2, int a3, T val) { atomicAdd(base + k * SC + a3 * S3 + a2 * S2 + a1, val); };
        };
        auto base_of = [&](int rp) {
            return halo + ((rp >> 16) & 255) * S3 - LO * S3 + ((rp >> 8) & 255) * S2 - LO * S2 + (rp & 255) - LO;
        };
        for (int q = warp; q < nbat; q += NW) {
            const PRec<T> recs[2] = {p_rec[q], p_rec2[q]};
            int rps[2];
#pragma unroll
            for (int stage = 0; stage < 2; ++stage) {
                if constexpr (sizeof(T) == 4) rps[stage] = __float_as_int(recs[stage].relf);
                else rps[stage] = (int)__double_as_longlong(recs[stage].relf);
            }
            const T mus[2][3] = {{p_mu[q * 6 + 0], p_mu[q * 6 + 1], p_mu[q * 6 + 2]},
                                 {p_mu[q * 6 + 3], p_mu[q * 6 + 4], p_mu[q * 6 + 5]}};
            if (rps[0] >= 0 && rps[0] == rps[1]) {
                // X and X* in the same cell: one stencil, both weight sets, one add per node
                const T sa[3] = {recs[0].t[0] - (T)0.5, recs[0].t[1] - (T)0.5, recs[0].t[2] - (T)0.5};
                const T sb[3] = {recs[1].t[0] - (T)0.5, recs[1].t[1] - (T)0.5, recs[1].t[2] - (T)0.5};
                W.eval_values2(sa, sb, wv, wd);
                L.template scatter_n<true>(wv, mus[0], wd, mus[1], add_smem(base_of(rps[0])));
                continue;
            }
#pragma unroll
            for (int stage = 0; stage < 2; ++stage) {
                const PRec<T>& rec = recs[stage];
                const int rp = rps[stage];
                W.eval(rec.t[0] - (T)0.5, rec.t[1] - (T)0.5, rec.t[2] - (T)0.5, wv, wd);
                if (rp >= 0) {
                    L.template scatter_n<false>(wv, mus[stage], wv, mus[stage], add_smem(base_of(rp)));
                } else {
                    const int pc = stage == 0 ? p_cell[q] : p_cell2[q];
                    const int c1 = pc & 1023, c2 = (pc >> 10) & 1023, c3 = (pc >> 20) & 1023;
                    double* gf = a.gfield;
                    L.template scatter_n<false>(wv, mus[stage], wv, mus[stage],
                                                [&](int k, int a1, int a2, int a3, T val) {
                        const int x1 = (c1 + a1 - LO) & mask, x2 = (c2 + a2 - LO) & mask, x3 = (c3 + a3 - LO) & mask;
                        atomicAdd(gf + k * NN3 + ((int64_t)x3 * N + x2) * N + x1, (double)val);
                    });
                }
            }
        }
        __syncthreads();
        // flush the accumulator: one float64 atomic per touched halo node
        for (int e = tid; e < 3 * H * H * H; e += NT) {
            const int x = e % H, yz = e / H, y = yz % H, zk = yz / H, z = zk % H, k = zk / H;
            const T val = halo[k * SC + z * S3 + y * S2 + x];
            if (val != (T)0) {
                const int64_t gi = ((int64_t)((o3 + z) & mask) * N + ((o2 + y) & mask)) * N + ((o1 + x) & mask);
                atomicAdd(a.gfield + k * NN3 + gi, (double)val);
            }
        }
    }
}

// h + l += x, keeping the rounding error of the float32 add in l: Knuth's
// TwoSum gives the rounded sum s = fl(h + x) and its error e with
// h + x = s + e exactly; the errors are summed in l
__device__ __forceinline__ void two_sum_acc(float& h, float& l, float x)
{
    const float s = __fadd_rn(h, x);
    const float bv = __fsub_rn(s, h);
    const float e = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bv)), __fsub_rn(x, bv));
    h = s;
    l = __fadd_rn(l, e);
}

// dLoss/dfield[k][node] += sum over the non-empty blocks whose halo holds the
// node of their partial sums, in a fixed order of the blocks.  Along each
// axis the blocks are those with integer index bi in
// [ceil((x + G - H + 1) / BLK), floor((x + G) / BLK)], at halo offset
// x + G - BLK bi in [0, H), taken mod nb (periodic images of the same block
// included).
template <typename T, int H>
__global__ void k_adj_gather(const __grid_constant__ AdjArgs a)
{
    constexpr int G = (H - BLK - 1) / 2;                     // I / 2 for H = BLK + I + 1
    constexpr int H3 = H * H * H;
    const int N = a.g.N;
    const int64_t NN3 = (int64_t)N * N * N;
    const int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (node >= NN3) return;
    const int lg = __ffs(N) - 1;                              // log2 N (N a power of two)
    const int x1 = (int)(node & (N - 1)), x2 = (int)((node >> lg) & (N - 1)), x3 = (int)(node >> (2 * lg));
    // per axis: the blocks bi whose halo [BLK bi - G, BLK bi - G + H) holds x, i.e.
    // bi in [ceil((x + G - H + 1) / BLK), floor((x + G) / BLK)]; arithmetic shifts floor for negatives
    auto range = [&](int x, int& lo, int& hi) {
        hi = (x + G) >> LBLK;
        lo = -((-(x + G - H + 1)) >> LBLK);                   // ceiling of (x + G - H + 1) / BLK
    };
    int z0, z1, y0, y1, w0, w1;
    range(x3, z0, z1);
    range(x2, y0, y1);
    range(x1, w0, w1);
    const int m3 = a.g.nb3 - 1, m2 = a.g.nb2 - 1, m1 = a.g.nb1 - 1;   // block counts are powers of two
    // fixed trip counts (at most H / BLK + 1 blocks per axis) with predicates, so
    // that every emptiness check, then every partial read, is issued at once
    constexpr int NA = H / BLK + 1;
    int64_t bidx[NA * NA * NA];
    int hoff[NA * NA * NA];
    bool use[NA * NA * NA];
#pragma unroll
    for (int iz = 0; iz < NA; ++iz)
#pragma unroll
        for (int iy = 0; iy < NA; ++iy)
#pragma unroll
            for (int ix = 0; ix < NA; ++ix) {
                const int c = (iz * NA + iy) * NA + ix;
                const int bzi = z0 + iz, byi = y0 + iy, bxi = w0 + ix;
                const int hz = x3 + G - BLK * bzi, hy = x2 + G - BLK * byi, hx = x1 + G - BLK * bxi;
                bidx[c] = ((int64_t)(bzi & m3) * a.g.nb2 + (byi & m2)) * a.g.nb1 + (bxi & m1);
                hoff[c] = (hz * H + hy) * H + hx;
                use[c] = bzi <= z1 && byi <= y1 && bxi <= w1;
            }
#pragma unroll
    for (int c = 0; c < NA * NA * NA; ++c)
        if (use[c]) use[c] = a.offsets[bidx[c] + 1] != a.offsets[bidx[c]];   // empty block: no partials
    double s0 = 0, s1 = 0, s2 = 0;
    const T* gs = reinterpret_cast<const T*>(a.gscratch);
    if constexpr (sizeof(T) == 4) {
        // float32 partials: a compensated float32 sum (Ogita, Rump and Oishi's
        // Sum2: the sum as hi + lo within ~1e-13 of the sum of the magnitudes)
        // instead of float64 adds, whose pipe this GPU has little of (with
        // float64 adds the gather ran at 86% of that pipe)
        float h[3] = {0.f, 0.f, 0.f}, l[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int c = 0; c < NA * NA * NA; ++c)
            if (use[c]) {
                const T* sb = gs + bidx[c] * 3 * H3 + hoff[c];
#pragma unroll
                for (int k = 0; k < 3; ++k) two_sum_acc(h[k], l[k], (float)sb[k * H3]);
            }
        s0 = (double)h[0] + (double)l[0];
        s1 = (double)h[1] + (double)l[1];
        s2 = (double)h[2] + (double)l[2];
    } else {
#pragma unroll
        for (int c = 0; c < NA * NA * NA; ++c)
            if (use[c]) {
                const T* sb = gs + bidx[c] * 3 * H3 + hoff[c];
                s0 += (double)sb[0];
                s1 += (double)sb[H3];
                s2 += (double)sb[2 * H3];
            }
    }
    // every slab value is read by exactly one node: leave the slabs zero for the
    // next step's atomic adds
    T* gz = reinterpret_cast<T*>(a.gscratch);
#pragma unroll
    for (int c = 0; c < NA * NA * NA; ++c)
        if (use[c]) {
            T* sb = gz + bidx[c] * 3 * H3 + hoff[c];
            sb[0] = (T)0;
            sb[H3] = (T)0;
            sb[2 * H3] = (T)0;
        }
    a.gfield[node] += s0;
    a.gfield[NN3 + node] += s1;
    a.gfield[2 * NN3 + node] += s2;
}

template <typename T, int I, int DEG, int STORE, int AM>
cudaError_t launch_adjoint_g(const AdjArgs& a, int64_t nblocks, cudaStream_t st)
{
    constexpr int H = BLK + I - 1 + 2;
    constexpr size_t smem = AdjPlan<T, Layout<I, H>::SC>::total;
    auto kern = k_adjoint<T, I, DEG, STORE, AM>;
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

// no offsets: the direct mode over a.np sorted particles; with per-block
// scratch the W^T adds go to the block's slab in global memory
template <typename T, int I, int DEG, int STORE>
cudaError_t launch_adjoint_t(const AdjArgs& a, int64_t nblocks, cudaStream_t st)
{
    if (!a.offsets) return launch_adjoint_g<T, I, DEG, STORE, ADJ_DIRECT>(a, (a.np + PBA - 1) / PBA, st);
    if (a.gscratch) return launch_adjoint_g<T, I, DEG, STORE, ADJ_SLAB>(a, nblocks, st);
    return launch_adjoint_g<T, I, DEG, STORE, ADJ_SMEM>(a, nblocks, st);
}

template <int I, int DEG>
cudaError_t dispatch_adjoint(const AdjArgs& a, int64_t nblocks, cudaStream_t st)
{
    if (a.f.storage == ST_F64) return launch_adjoint_t<double, I, DEG, ST_F64>(a, nblocks, st);
    if (a.f.storage == ST_F32) return launch_adjoint_t<float, I, DEG, ST_F32>(a, nblocks, st);
    return launch_adjoint_t<float, I, DEG, ST_BF16X2>(a, nblocks, st);
}

}  // namespace trk
