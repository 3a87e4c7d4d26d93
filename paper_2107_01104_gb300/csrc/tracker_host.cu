// C ABI of libtracker (declared and documented in include/tracker.h).
//
// The tracker owns its field copy and all scratch (sort buffers, the offset
// array, the sorted particle state of the time steppers, device flags).
// Every entry point validates its arguments on the host, issues kernels on
// the tracker's stream and returns a status; nothing here computes on the CPU.
#include <algorithm>
#include <array>
#include <cmath>
#include <string>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include <cuda.h>   // CUtensorMap and its enums (the encoder is looked up at run time)

#include "internal.cuh"
#include "tracker.h"

using namespace trk;

namespace {

thread_local char g_err[512] = "";

int fail(int code, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

#define CUDA_TRY(x)                                                                     \
    do {                                                                                \
        cudaError_t e_ = (x);                                                           \
        if (e_ != cudaSuccess) return fail(TRK_ECUDA, "%s: %s", #x, cudaGetErrorString(e_)); \
    } while (0)

struct TableInfo {
    int family, I, m, deg;
};
const TableInfo kTables[TRK_NUM_TABLES] = TRK_TABLE_INFO;
const double kCoef[TRK_NUM_TABLES][TRK_TAB_MAX_I][TRK_TAB_MAX_DEG] = TRK_COEF_INIT;
const double kDCoef[TRK_NUM_TABLES][TRK_TAB_MAX_I][TRK_TAB_MAX_DEG] = TRK_DCOEF_INIT;

int find_table(int family, int I, int m)
{
    for (int k = 0; k < TRK_NUM_TABLES; ++k) {
        const TableInfo& t = kTables[k];
        if (t.family != family || t.I != I) continue;
        if (family == TRK_LAGRANGE || t.m == m) return k;
    }
    return -1;
}

int ilog2(int64_t x)
{
    int r = 0;
    while ((int64_t(1) << r) < x) ++r;
    return r;
}

bool is_pow2(int64_t x) { return x > 0 && (x & (x - 1)) == 0; }

template <typename P>
cudaError_t dev_alloc(P** p, size_t bytes)
{
    *p = nullptr;
    if (bytes == 0) return cudaSuccess;
    return cudaMalloc(reinterpret_cast<void**>(p), bytes);
}

void dev_free(void* p)
{
    if (p) cudaFree(p);
}

constexpr int PB_HOST = 256;   // particles per direct-path work item (the block kernels' batch)

struct GraphCache {
    cudaGraphExec_t exec = nullptr;
    uint64_t key = 0;
    int64_t kernels = 0;
};

// Per-set buffers of tracker_advance_batched.
struct SetState {
    int64_t cap = 0;
    int64_t nb = 0;                   // block count the per-block arrays were sized for
    uint32_t* keys = nullptr;
    uint32_t* counts = nullptr;       // [nblocks] block counts of the next binning (zero between binnings)
    int32_t* perm = nullptr;
    int32_t* offsets = nullptr;
    int32_t* list = nullptr;
    int32_t* count = nullptr;
    double* pos_s[2] = {nullptr, nullptr};
    int32_t* id_s[2] = {nullptr, nullptr};
    float* rhs_s[2] = {nullptr, nullptr};
};

uint64_t mix(uint64_t h, uint64_t v)
{
    h ^= v + 0x9e3779b97f4a7c15ULL + (h << 6) + (h >> 2);
    return h;
}

}  // namespace

void trk::set_error_message(const char* msg) { snprintf(g_err, sizeof(g_err), "%s", msg ? msg : ""); }

struct tracker {
    int device = -1;                  // CUDA device the tracker's buffers live on (current at create)
    int N = 0;
    double L = 0;
    int family = 0, I = 0, m = 0, storage = 0;
    int tab = -1, deg = 0, deg_hi = 0;
    cudaStream_t stream = nullptr;
    GridGeom g{};
    int64_t nblocks = 0;
    int key_bits = 0;
    // field
    int C = 0;
    void* field = nullptr;
    float* field_nm = nullptr;        // node-major copy of the field for the direct path (float32; split-bf16 with C a multiple of 3), built on first use
    bool nm_skip = false;             // split-bf16, C > 3: the copy could not be allocated for this field
    cudaTextureObject_t nm_tex = 0;   // 16-byte-texel texture over field_nm (C = 3), or 0 for plain loads
    size_t nm_bytes = 0;
    bool nm_valid = false;
    // sort scratch
    int64_t sort_cap = 0;             // keys, perm
    int64_t radix_cap = 0;            // sort_scratch, keys_sorted (stable binning)
    void* sort_scratch = nullptr;
    uint32_t* keys = nullptr;
    uint32_t* keys_sorted = nullptr;
    int32_t* perm = nullptr;
    int32_t* offsets = nullptr;
    // sorted state of the steppers
    int64_t state_cap = 0;
    double* pos_s[2] = {nullptr, nullptr};
    int32_t* id_s[2] = {nullptr, nullptr};
    float* rhs_s[2] = {nullptr, nullptr};
    int* d_flags = nullptr;
    int64_t launches = 0;
    // adjoint scratch: checkpoints, one segment of trajectory, lambda ping-pong
    size_t adj_bytes = 0;
    double* adj_buf = nullptr;
    size_t adj_scratch_bytes = 0;    // per-block W^T partial sums of the field gradient
    void* adj_scratch = nullptr;
    // CUDA-graph replay of step pairs, on a tracker-owned stream joined to the caller's
    cudaStream_t gstream = nullptr;
    cudaEvent_t gev[2] = {nullptr, nullptr};
    uint64_t gen = 1;                 // bumped whenever a buffer baked into a graph is reallocated
    GraphCache adv_graph, batch_graph;
    // batched sets
    std::vector<SetState> sets;
    void* ne_scratch = nullptr;       // non-empty-list scratch
    int64_t ne_cap = 0;
    BatchSet* d_desc = nullptr;       // [3][nsets] descriptors: first step, parity 0, parity 1
    int* d_ctr = nullptr;             // [nsets] work counters
    int desc_cap = 0;
    std::vector<std::pair<uint64_t, int>> tune_cache;   // set signature -> direct path?
    int nsm = 0;
    int step_kernel = TRK_STEP_AUTO;  // trk_step_kernel
    std::vector<std::pair<uint64_t, int>> interp_cache; // (np, C, deriv, out dtype) -> interpolation kernel
    int last_kernel = TRK_STEP_AUTO;  // kernel of the latest tracker_advance or tracker_interpolate
    int* d_colctr = nullptr;          // work counter of the column kernel
    int col_seg = 8;                  // column kernel: x3 slabs per work item (power of two)
    int dir_blk = BLK;                // direct path: edge of its cubic binning blocks (default shape only)
    int dir_ppc = 256;                // direct path: particles per CTA
    int64_t bin_cap = 0;              // entries of offsets / counts / cursor (largest geometry in use)
    int tune_source = TRK_TUNE_DEFAULT;   // how the latest call's parameters were chosen
    std::array<int, 5> last_tuning = {TRK_STEP_AUTO, BLK, 8, 0, 256};   // path, dir_blk, col_seg, tma, ppc of the latest call
    std::vector<std::pair<std::string, std::array<int, 5>>> step_tune;   // tuner decisions by workload
    // tensor maps of the padded field for the block kernel's tensor-copy halos,
    // one per stage-2 margin (interpolation and AB: 0, RK2: 1)
    CUtensorMap tmap[2];
    bool tmap_ok[2] = {false, false};
    CUtensorMap batch_map[3];         // batched sets: AB2 halo boxes of widths 4, 6, 8
    int halo_copy = TRK_HALO_AUTO;    // trk_halo_copy: how the block kernel stages its halo
    bool auto_tma = true;             // TRK_HALO_AUTO's current choice (tensor copies, where there is a map)
    uint32_t* d_counts = nullptr;     // [nblocks] block counts (counting-sort binning of the column path)
    int32_t* d_cursor = nullptr;      // [nblocks] scatter cursors
    uint32_t* d_scan_tmp = nullptr;   // tile sums of the multi-CTA count scan
    // instrumentation: event pairs per kernel class
    bool prof = false;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_pairs[3];
    int64_t prof_launches[3] = {0, 0, 0};
};

namespace {

enum { PROF_STEP = 0, PROF_BIN = 1, PROF_OTHER = 2 };

cudaEvent_t next_event(tracker* t)
{
    if (t->ev_used == t->ev_pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        t->ev_pool.push_back(e);
    }
    return t->ev_pool[t->ev_used++];
}

// Records an event pair around a region of kernel launches when profiling.
struct ProfScope {
    tracker* t;
    int cls;
    int64_t n;
    cudaEvent_t a = nullptr;
    ProfScope(tracker* t_, int cls_, int64_t n_ = 1) : t(t_), cls(cls_), n(n_)
    {
        if (t->prof && (a = next_event(t))) cudaEventRecord(a, t->stream);
    }
    ~ProfScope()
    {
        if (!a) return;
        cudaEvent_t b = next_event(t);
        if (!b) return;
        cudaEventRecord(b, t->stream);
        t->prof_pairs[cls].emplace_back(a, b);
        t->prof_launches[cls] += n;
    }
};

// The binning arrays (offsets, block counts, scatter cursors, scan scratch)
// for at least nb blocks; grown, never shrunk (the direct path's tuned block
// edge may need more blocks than the tracker's block shape).
int ensure_bin(tracker* t, int64_t nb)
{
    if (nb <= t->bin_cap) return TRK_OK;
    dev_free(t->offsets);
    dev_free(t->d_counts);
    dev_free(t->d_cursor);
    dev_free(t->d_scan_tmp);
    t->offsets = nullptr;
    t->d_counts = nullptr;
    t->d_cursor = nullptr;
    t->d_scan_tmp = nullptr;
    t->bin_cap = 0;
    t->gen += 1;
    if (dev_alloc(&t->offsets, (size_t)(nb + 1) * sizeof(int32_t)) != cudaSuccess ||
        dev_alloc(&t->d_counts, (size_t)nb * sizeof(uint32_t)) != cudaSuccess ||
        dev_alloc(&t->d_cursor, (size_t)nb * sizeof(int32_t)) != cudaSuccess ||
        dev_alloc(&t->d_scan_tmp, std::max<size_t>(count_scan_scratch_bytes(nb), 16)) != cudaSuccess) {
        cudaGetLastError();
        return fail(TRK_ENOMEM, "cannot allocate binning arrays for %lld blocks", (long long)nb);
    }
    CUDA_TRY(cudaMemset(t->d_counts, 0, (size_t)nb * sizeof(uint32_t)));
    t->bin_cap = nb;
    return TRK_OK;
}

int set_geometry(tracker* t, int bx, int by, int bz)
{
    const int N = t->N;
    for (int b : {bx, by, bz})
        if (!is_pow2(b) || b > N) return fail(TRK_EINVAL, "block edge %d must be a power of two <= N=%d", b, N);
    t->g.lb1 = ilog2(bx);
    t->g.lb2 = ilog2(by);
    t->g.lb3 = ilog2(bz);
    t->g.nb1 = N / bx;
    t->g.nb2 = N / by;
    t->g.nb3 = N / bz;
    t->nblocks = (int64_t)t->g.nb1 * t->g.nb2 * t->g.nb3;
    t->key_bits = ilog2(t->nblocks);
    return ensure_bin(t, t->nblocks);
}

// keys and permutation of np particles (every binning)
int ensure_sort(tracker* t, int64_t np)
{
    if (np <= t->sort_cap) return TRK_OK;
    t->gen += 1;
    dev_free(t->keys);
    dev_free(t->perm);
    t->keys = nullptr;
    t->perm = nullptr;
    t->sort_cap = 0;
    if (dev_alloc(&t->keys, (size_t)np * 4) != cudaSuccess || dev_alloc(&t->perm, (size_t)np * 4) != cudaSuccess) {
        cudaGetLastError();
        return fail(TRK_ENOMEM, "cannot allocate binning buffers for %lld particles", (long long)np);
    }
    t->sort_cap = np;
    return TRK_OK;
}

// radix-sort scratch and sorted keys of the stable binning (tracker_bin only)
int ensure_radix(tracker* t, int64_t np)
{
    if (np <= t->radix_cap) return TRK_OK;
    dev_free(t->sort_scratch);
    dev_free(t->keys_sorted);
    t->sort_scratch = nullptr;
    t->keys_sorted = nullptr;
    t->radix_cap = 0;
    if (dev_alloc(&t->sort_scratch, radix_scratch_bytes(np)) != cudaSuccess ||
        dev_alloc(&t->keys_sorted, (size_t)np * 4) != cudaSuccess) {
        cudaGetLastError();
        return fail(TRK_ENOMEM, "cannot allocate radix-sort scratch for %lld particles", (long long)np);
    }
    t->radix_cap = np;
    return TRK_OK;
}

int ensure_state(tracker* t, int64_t np)
{
    if (np <= t->state_cap) return TRK_OK;
    t->gen += 1;
    for (int i = 0; i < 2; ++i) {
        dev_free(t->pos_s[i]);
        dev_free(t->id_s[i]);
        dev_free(t->rhs_s[i]);
        t->pos_s[i] = nullptr;
        t->id_s[i] = nullptr;
        t->rhs_s[i] = nullptr;
    }
    t->state_cap = 0;
    for (int i = 0; i < 2; ++i) {
        if (dev_alloc(&t->pos_s[i], (size_t)np * 24) != cudaSuccess || dev_alloc(&t->id_s[i], (size_t)np * 4) != cudaSuccess ||
            dev_alloc(&t->rhs_s[i], (size_t)np * 12 * AB_MAX_HIST) != cudaSuccess) {
            cudaGetLastError();
            return fail(TRK_ENOMEM, "cannot allocate particle state for %lld particles", (long long)np);
        }
    }
    t->state_cap = np;
    return TRK_OK;
}

FieldView field_view(const tracker* t)
{
    FieldView f{};
    f.storage = t->storage;
    f.C = t->C;
    f.NP = t->N + 2 * PAD;
    f.plane = (int64_t)f.NP * f.NP * f.NP;
    if (t->storage == ST_F64) f.f64 = reinterpret_cast<const double*>(t->field);
    else if (t->storage == ST_F32) f.f32 = reinterpret_cast<const float*>(t->field);
    else {
        f.hi = reinterpret_cast<const __nv_bfloat16*>(t->field);
        f.lo = f.hi + f.plane * t->C;
    }
    f.nm = t->nm_valid ? t->field_nm : nullptr;
    f.nm_tex = t->nm_valid ? (unsigned long long)t->nm_tex : 0ull;
    f.nmc = t->C == 3 ? 4 : t->C;
    return f;
}

// The tensor map the block kernel stages its halos with for `mode`, or null
// for cp.async element copies (TRK_HALO_ASYNC, no map for this field, or a
// storage the tensor copies do not cover).
const void* halo_tmap(const tracker* t, int mode)
{
    const int margin = mode == MODE_RK2 ? 1 : 0;
    const bool tma = t->halo_copy == TRK_HALO_TMA || (t->halo_copy == TRK_HALO_AUTO && t->auto_tma);
    if (!tma || !t->tmap_ok[margin]) return nullptr;
    return &t->tmap[margin];
}

bool halo_tmap_exists(const tracker* t, int mode) { return t->tmap_ok[mode == MODE_RK2 ? 1 : 0]; }

cudaError_t launch_block(tracker* t, int mode, const BlockArgs& a)
{
    ProfScope ps(t, PROF_STEP);
    t->launches += 1;
    const void* m = halo_tmap(t, mode);
    switch (t->I) {
        case 4: return launch_block_i4(mode, a, m, t->nblocks, t->deg_hi, t->stream);
        case 6: return launch_block_i6(mode, a, m, t->nblocks, t->deg_hi, t->stream);
        default: return launch_block_i8(mode, a, m, t->nblocks, t->deg_hi, t->stream);
    }
}

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime
// (the library does not link the driver API); null if unavailable.
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled()
{
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess && p)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

// Tensor maps of the padded field f[C][NP][NP][NP] (4-D, x1 innermost) with the
// block kernel's halo box for both stage-2 margins: float32 and float64
// storage with at least three components (a chunk of three per copy; the
// last chunk of a C that is not a multiple of three reads zeros beyond C,
// which no output uses).  Left unset (cp.async staging) otherwise.
// the tensor map of the tracker's field with the halo box of kernel width I
// and stage-2 margin `margin` (tma_box); false if it cannot be made
bool encode_field_map(const tracker* t, int I, int margin, CUtensorMap* out)
{
    const EncodeTiledFn enc = encode_tiled();
    if (!enc || (t->storage != TRK_F32 && t->storage != TRK_F64) || t->C < 3 || !t->field) return false;
    const int esz = t->storage == TRK_F64 ? 8 : 4;
    const cuuint64_t NP = (cuuint64_t)(t->N + 2 * PAD);
    const cuuint64_t dims[4] = {NP, NP, NP, (cuuint64_t)t->C};
    const cuuint64_t strides[3] = {NP * esz, NP * NP * esz, NP * NP * NP * esz};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const TmaBox b = tma_box(I, margin, esz);
    const cuuint32_t box[4] = {(cuuint32_t)b.BX, (cuuint32_t)b.BY, (cuuint32_t)b.H, 3};
    return enc(out, esz == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, t->field, dims,
               strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

void build_tmaps(tracker* t)
{
    for (int margin = 0; margin < 2; ++margin) t->tmap_ok[margin] = encode_field_map(t, t->I, margin, &t->tmap[margin]);
}

cudaError_t launch_direct(tracker* t, int mode, const BlockArgs& a)
{
    ProfScope ps(t, PROF_STEP);
    t->launches += 1;
    switch (t->I) {
        case 4: return launch_direct_i4(mode, a, t->deg_hi, t->stream);
        case 6: return launch_direct_i6(mode, a, t->deg_hi, t->stream);
        default: return launch_direct_i8(mode, a, t->deg_hi, t->stream);
    }
}

// Stable binning (tracker_bin): keys (caller order) -> sorted keys, perm, offsets.
int bin_into(tracker* t, int64_t np, const double* pos, uint32_t* keys, int32_t* perm, int32_t* offsets)
{
    ProfScope ps(t, PROF_BIN);
    CUDA_TRY(launch_keys(t->g, np, pos, keys, t->d_flags, t->stream));
    t->launches += 1;
    CUDA_TRY(radix_sort(keys, np, t->key_bits, t->keys_sorted, perm, t->sort_scratch, t->stream, &t->launches));
    CUDA_TRY(launch_offsets(t->keys_sorted, np, t->nblocks, offsets, t->stream));
    t->launches += 1;
    return TRK_OK;
}

// Counting-sort binning of interpolation and the adjoint: keys and block
// counts from the positions, offsets and cursors from one scan, then the
// permutation t->perm (grouped by block; the order inside a block is not
// reproducible, and every particle's result is independent of it).
int bin_counting(tracker* t, int64_t np, const double* pos)
{
    ProfScope ps(t, PROF_BIN);
    CUDA_TRY(cudaMemsetAsync(t->d_counts, 0, (size_t)t->nblocks * sizeof(uint32_t), t->stream));
    CUDA_TRY(launch_keys_count(t->g, np, pos, t->keys, t->d_counts, t->d_flags, t->stream));
    CUDA_TRY(launch_count_scan(t->d_counts, t->nblocks, t->offsets, t->d_cursor, t->d_scan_tmp, t->stream,
                               &t->launches));
    CUDA_TRY(launch_scatter_perm(np, t->keys, t->d_cursor, t->perm, t->d_flags, t->stream));
    t->launches += 2;
    return TRK_OK;
}

// Every call that launches work or allocates must run with the tracker's
// device current: its buffers live there, and a launch on another device
// would hand that device foreign pointers.
int check_device(const tracker* t)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return fail(TRK_ECUDA, "no current CUDA device");
    }
    if (dev != t->device)
        return fail(TRK_EINVAL, "the tracker lives on CUDA device %d but device %d is current", t->device, dev);
    return TRK_OK;
}

int check_np(int64_t np)
{
    if (np < 0 || np > 2147483647LL) return fail(TRK_EINVAL, "np=%lld out of range [0, 2^31-1]", (long long)np);
    return TRK_OK;
}

int check_block_kernel_shape(const tracker* t)
{
    if (t->g.lb1 != LBLK || t->g.lb2 != LBLK || t->g.lb3 != LBLK)
        return fail(TRK_EINVAL, "interpolation and advection need the %dx%dx%d block shape", BLK, BLK, BLK);
    return TRK_OK;
}

BlockArgs base_args(tracker* t)
{
    BlockArgs a{};
    a.g = t->g;
    a.f = field_view(t);
    for (int i = 0; i < TRK_TAB_MAX_I; ++i)
        for (int d = 0; d < TRK_TAB_MAX_DEG; ++d) {
            a.cd.c[i][d] = kCoef[t->tab][i][d];
            a.cd.d[i][d] = kDCoef[t->tab][i][d];
            a.cf.c[i][d] = (float)kCoef[t->tab][i][d];
            a.cf.d[i][d] = (float)kDCoef[t->tab][i][d];
        }
    a.offsets = t->offsets;
    a.flags = t->d_flags;
    a.ab_order = 2;
    a.ppc = t->dir_ppc;
    return a;
}

// Runs body() (which issues the work of a step pair on t->stream) as a CUDA
// graph on the tracker's own stream, capturing it the first time and whenever
// key changes, then replaying it reps times.  The caller's stream and the
// graph stream are joined with events both ways.
template <class F>
int replay_graph(tracker* t, GraphCache& gc, uint64_t key, int reps, F&& body)
{
    if (reps <= 0) return TRK_OK;
    cudaStream_t user = t->stream;
    CUDA_TRY(cudaEventRecord(t->gev[0], user));
    CUDA_TRY(cudaStreamWaitEvent(t->gstream, t->gev[0], 0));
    if (!gc.exec || gc.key != key) {
        if (gc.exec) cudaGraphExecDestroy(gc.exec);
        gc.exec = nullptr;
        const int64_t l0 = t->launches;
        t->stream = t->gstream;
        cudaError_t e = cudaStreamBeginCapture(t->gstream, cudaStreamCaptureModeThreadLocal);
        int rc = e == cudaSuccess ? body() : fail(TRK_ECUDA, "cudaStreamBeginCapture: %s", cudaGetErrorString(e));
        cudaGraph_t g = nullptr;
        const cudaError_t e2 = e == cudaSuccess ? cudaStreamEndCapture(t->gstream, &g) : cudaSuccess;
        t->stream = user;
        if (rc != TRK_OK || e2 != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            return rc != TRK_OK ? rc : fail(TRK_ECUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(e2));
        }
        e = cudaGraphInstantiate(&gc.exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            gc.exec = nullptr;
            return fail(TRK_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
        }
        gc.kernels = t->launches - l0;
        t->launches = l0;
        gc.key = key;
    }
    for (int r = 0; r < reps; ++r) {
        CUDA_TRY(cudaGraphLaunch(gc.exec, t->gstream));
        t->launches += gc.kernels;
    }
    CUDA_TRY(cudaEventRecord(t->gev[1], t->gstream));
    CUDA_TRY(cudaStreamWaitEvent(user, t->gev[1], 0));
    return TRK_OK;
}

// slabs per column-kernel work item: the tracker's setting, at most the column height
int column_segment(const tracker* t) { return std::max(1, std::min(t->g.nb3, t->col_seg)); }

bool column_available(const tracker* t)
{
    return t->storage == ST_F32 && (t->I == 4 || t->I == 6) && t->g.lb1 == LBLK && t->g.lb2 == LBLK &&
           t->g.lb3 == LBLK;
}

bool default_shape(const tracker* t) { return t->g.lb1 == LBLK && t->g.lb2 == LBLK && t->g.lb3 == LBLK; }

// Binning geometry of a step path: the tracker's block shape, except that the
// direct path bins by cubes of edge dir_blk when the shape is the default
// (the direct kernel takes 256 grouped particles per CTA whatever the blocks
// are; the block edge only sets how compact each CTA's particles are).
struct BinGeom {
    GridGeom g;
    int64_t nb;
};
BinGeom geom_of(const tracker* t, int path)
{
    if (path != TRK_STEP_DIRECT || t->dir_blk == BLK || !default_shape(t)) return {t->g, t->nblocks};
    BinGeom b{t->g, 0};
    const int lb = ilog2(t->dir_blk);
    b.g.lb1 = b.g.lb2 = b.g.lb3 = lb;
    b.g.nb1 = b.g.nb2 = b.g.nb3 = t->N >> lb;
    b.nb = (int64_t)b.g.nb1 * b.g.nb2 * b.g.nb3;
    return b;
}
bool same_geom(const GridGeom& a, const GridGeom& b) { return a.lb1 == b.lb1 && a.lb2 == b.lb2 && a.lb3 == b.lb3; }

void destroy_nm_texture(tracker* t)
{
    if (t->nm_tex) cudaDestroyTextureObject(t->nm_tex);
    t->nm_tex = 0;
}

// The direct kernel fetches the 16-byte nodes of the node-major copy through
// a texture object (the same bits, on the texture data path instead of the
// load/store one) where the copy is at most kNmTextureL2 times the L2 size, or
// the environment variable TRK_NM_TEXTURE_BYTES (0: never), and its node count
// fits the device's linear-texture width.  Measured on the direct kernel:
// with the copy at 2.5 times L2 (256^3) its stencil gathers are bound by the
// L1 data path and the texture fetches take 16% less time; at 19 times L2 and
// above (512^3, 1024^3) the gathers are bound by DRAM, where the texture
// fetches took 10 to 11% more time than plain loads.
constexpr double kNmTextureL2 = 4.0;

void create_nm_texture(tracker* t, int64_t plane, size_t bytes, bool f32)
{
    int maxlin = 0, l2 = 0, dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&maxlin, cudaDevAttrMaxTexture1DLinearWidth, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    double cap = kNmTextureL2 * l2;
    if (const char* env = getenv("TRK_NM_TEXTURE_BYTES")) cap = strtod(env, nullptr);
    if ((double)bytes > cap || plane > (int64_t)maxlin) return;
    cudaResourceDesc rd{};
    rd.resType = cudaResourceTypeLinear;
    rd.res.linear.devPtr = t->field_nm;
    rd.res.linear.desc = f32 ? cudaCreateChannelDesc<float4>() : cudaCreateChannelDesc<uint4>();
    rd.res.linear.sizeInBytes = bytes;
    cudaTextureDesc td{};
    td.readMode = cudaReadModeElementType;
    if (cudaCreateTextureObject(&t->nm_tex, &rd, &td, nullptr) != cudaSuccess) {
        cudaGetLastError();
        t->nm_tex = 0;
    }
}

// The node-major copy of a float32 field that the direct kernel reads, made
// (or refreshed after tracker_set_field) before the first direct launch that
// needs it; never inside a graph capture (the first step of a call is eager).
int ensure_node_major(tracker* t)
{
    // split bf16: one 16-byte record per node and chunk of three components,
    // the chunks one after the other (C = 3: one chunk)
    const bool f32 = t->storage == ST_F32, bf16 = t->storage == ST_BF16X2 && t->C % 3 == 0;
    if (!(f32 || bf16) || t->nm_valid || t->nm_skip) return TRK_OK;
    const int64_t NP = t->N + 2 * PAD;
    const int64_t plane = NP * NP * NP;
    const int nmc = f32 ? (t->C == 3 ? 4 : t->C) : 4 * (t->C / 3);
    const size_t bytes = (size_t)plane * nmc * sizeof(float);   // 16 bytes per node for C = 3
    if (t->nm_bytes != bytes) {
        destroy_nm_texture(t);
        dev_free(t->field_nm);
        t->field_nm = nullptr;
        t->nm_bytes = 0;
        t->gen += 1;                  // captured graphs hold the old pointer
        if (dev_alloc(&t->field_nm, bytes) != cudaSuccess) {
            cudaGetLastError();
            // split bf16 with more than three components: the direct kernel reads
            // the component-major field instead
            if (bf16 && t->C > 3) {
                t->nm_skip = true;
                return TRK_OK;
            }
            return fail(TRK_ENOMEM, "cannot allocate the node-major field copy (%zu bytes)", bytes);
        }
        t->nm_bytes = bytes;
    }
    // the 16-byte node loads of the direct kernel (a copy first made for C = 4
    // has the same size but no texture)
    if (t->C == 3 && !t->nm_tex) create_nm_texture(t, plane, bytes, f32);
    {
        ProfScope ps(t, PROF_OTHER);
        if (f32) {
            CUDA_TRY(launch_node_major(reinterpret_cast<const float*>(t->field), t->C, nmc, plane, t->field_nm, t->stream));
        } else {
            const __nv_bfloat16* hi = reinterpret_cast<const __nv_bfloat16*>(t->field);
            const __nv_bfloat16* lo = hi + plane * t->C;
            for (int ch = 0; ch < t->C / 3; ++ch)
                CUDA_TRY(launch_node_major_bf16(hi + plane * 3 * ch, lo + plane * 3 * ch, plane,
                                                t->field_nm + plane * 4 * ch, t->stream));
        }
    }
    t->launches += f32 ? 1 : t->C / 3;
    t->nm_valid = true;
    return TRK_OK;
}

// Below this many particles per grid cell the automatic choice gathers every
// stencil straight from global memory (direct path) instead of sweeping the
// field, without timing: on GB300 (float32, spline I = 6) the direct step wins
// there for RK2 and AB on every grid measured (256^3: RK2 0.381 vs 0.534 ms at
// 1/24 per cell, AB2 0.287 vs 0.328 ms).  Above it the kernels are timed.
constexpr double kDirectDensity = 0.05;

// Without a column kernel (float64 or split-bf16 storage, I = 8, other block
// shapes) the choice is between the block and the direct kernel, whose
// binnings differ, so it is a density threshold, measured on GB300 (256^3,
// RK2, block vs direct ms per step): float32 I = 8 1.24 vs 0.73 at 1/16 per
// cell, 2.61 vs 2.65 at 1/4; float64 7.12 vs 6.02 and 24.7 vs 23.9;
// split-bf16 (node-major copy) 1.19 vs 0.59 and 2.45 vs 2.20.
double direct_threshold(const tracker* t) { return column_available(t) ? kDirectDensity : 0.25; }

// Below this many particles per grid cell the adjoint runs without halos
// (direct mode); above it one CTA per cell block stages the block's halo.
// Measured on GB300 (256^3 float32, spline I = 6, 20 RK2 steps, direct vs
// halo ms per call): 23 vs 72 at 1/64 per cell, 74 vs 100 at 1/16, 282 vs
// 221 at 1/4.
constexpr double kAdjDirectDensity = 0.125;

// Remembers a timing decision; the oldest is dropped beyond kCacheMax entries
// (a caller whose particle counts keep changing re-times now and then).
constexpr size_t kCacheMax = 256;
void remember(std::vector<std::pair<uint64_t, int>>& cache, uint64_t sig, int choice)
{
    if (cache.size() >= kCacheMax) cache.erase(cache.begin());
    cache.emplace_back(sig, choice);
}

// Densities (particles per cell) between which AUTO times the column and the
// direct kernel on the first tracker_advance call of a (np, scheme) and keeps
// the faster: the crossover moves with the grid (L2 holds a 256^3 float32
// field but not a 512^3 one) and with the scheme.
constexpr double kProbeMin = 0.01, kProbeMax = 0.25;

// The kernel tracker_advance (and, between BLOCK and DIRECT, tracker_interpolate)
// uses for np particles before any timing.
int step_path(const tracker* t, int64_t np)
{
    if (t->step_kernel != TRK_STEP_AUTO) return t->step_kernel;
    if ((double)np < direct_threshold(t) * (double)t->N * t->N * t->N) return TRK_STEP_DIRECT;
    return column_available(t) ? TRK_STEP_COLUMN : TRK_STEP_BLOCK;
}

// One RK2/ABk step of tracker_advance: re-bin, then the fused step kernel.
// Every path re-bins with the counting sort: block counts (from the previous
// step's update phase, or from the initial keys), one scan giving the offsets
// and cursors, one scatter of the particle state into its blocks.  Then the
// column kernel, the block kernel (one CTA per cell block), or the direct
// kernel (PB grouped particles per CTA, stencils gathered from global
// memory) updates the grouped state in place and counts the new keys.
// first: read the caller's arrays (identity ids).  AB steps: order
// k = ab_order, `hist` valid history entries for this step.
int advance_step(tracker* t, int64_t np, int path, int mode, int ab_order, int hist, double dt, int cur, bool first,
                 const double* pos, const float* rhs)
{
    const int nxt = cur ^ 1;
    const bool ab = mode == MODE_AB2;
    const BinGeom bg = geom_of(t, path);
    {
        ProfScope ps(t, PROF_BIN);
        const float* rin = ab && hist > 0 ? (first ? rhs : t->rhs_s[cur]) : nullptr;
        CUDA_TRY(launch_count_scan(t->d_counts, bg.nb, t->offsets, t->d_cursor, t->d_scan_tmp, t->stream,
                                   &t->launches));
        CUDA_TRY(launch_scatter_state(np, t->keys, t->d_cursor, first ? pos : t->pos_s[cur],
                                      first ? nullptr : t->id_s[cur], rin, 3 * (ab_order - 1), t->pos_s[nxt],
                                      t->id_s[nxt], t->rhs_s[nxt], t->d_flags, t->stream));
        t->launches += 1;
    }
    if (path == TRK_STEP_COLUMN) {
        ColumnArgs ca{};
        ca.a = base_args(t);
        ca.a.np = np;
        ca.a.dt = dt;
        ca.a.pos_out = t->pos_s[nxt];
        ca.a.rhs_out = t->rhs_s[nxt];
        ca.a.key_out = t->keys;
        ca.a.history_valid = ab ? hist : 0;
        ca.a.ab_order = ab_order;
        ca.nseg = column_segment(t);
        ca.nitems = (int64_t)t->g.nb1 * t->g.nb2 * (t->g.nb3 / ca.nseg);
        ca.ctr = t->d_colctr;
        ca.counts = t->d_counts;
        CUDA_TRY(cudaMemsetAsync(t->d_colctr, 0, sizeof(int), t->stream));
        ProfScope ps(t, PROF_STEP);
        t->launches += 1;
        if (t->I == 4) CUDA_TRY(launch_column_i4(mode, ca, t->deg_hi, t->nsm, t->stream));
        else CUDA_TRY(launch_column_i6(mode, ca, t->deg_hi, t->nsm, t->stream));
        return TRK_OK;
    }
    BlockArgs a = base_args(t);
    a.g = bg.g;
    a.np = np;
    a.dt = dt;
    a.perm = nullptr;   // the state is grouped: read and written at j
    a.pos_in = a.pos_out = t->pos_s[nxt];
    a.id_in = a.id_out = t->id_s[nxt];
    a.rhs_in = a.rhs_out = t->rhs_s[nxt];
    a.history_valid = ab ? hist : 0;
    a.ab_order = ab_order;
    a.key_out = t->keys;
    a.counts = t->d_counts;
    if (path == TRK_STEP_DIRECT) CUDA_TRY(launch_direct(t, mode, a));
    else CUDA_TRY(launch_block(t, mode, a));
    return TRK_OK;
}

// ---------------------------------------------------------------------------
// Tuner of the time-step path.  A candidate fixes the step kernel and its
// launch shape: the column kernel's segment length (x3 slabs per work item),
// the direct kernel's binning block edge, the block kernel's halo copy
// (cp.async or tensor copies).  On the first tracker_advance call of a
// workload (grid, kernel, storage, SM count, density bucket, scheme) with
// enough steps, every candidate runs kTuneStepsPerCand real steps of the call,
// timed with CUDA events, and the fastest is kept for the rest of the call and
// for later calls; all candidates give bit-identical steps.  Decisions are
// also appended to the file named by the environment variable TRK_TUNE_CACHE
// (if set), which a new tracker reads at creation.
// ---------------------------------------------------------------------------
constexpr int64_t kTuneMinNp = 32768;   // below this a step is launch-bound: no timing
constexpr int kTuneStepsPerCand = 2;    // the first run of a kernel may load its module: keep the faster

struct Cand {
    int path, dir_blk, col_seg, tma;
    int ppc = PB_HOST;               // direct kernel: particles per CTA
};

std::string tune_key(const tracker* t, int64_t np, int mode, int ab_order)
{
    const double dens = (double)np / ((double)t->N * t->N * t->N);
    const int bucket = (int)std::floor(2.0 * std::log2(dens));   // half-octave density buckets
    char buf[200];
    snprintf(buf, sizeof(buf), "advance2 N=%d family=%d I=%d m=%d storage=%d sm=%d dens2=%d mode=%d order=%d", t->N,
             t->family, t->I, t->m, t->storage, t->nsm, bucket, mode, ab_order);
    return buf;
}

bool valid_cand(const tracker* t, const Cand& c)
{
    const bool path_ok = c.path == TRK_STEP_DIRECT || c.path == TRK_STEP_BLOCK ||
                         (c.path == TRK_STEP_COLUMN && column_available(t));
    return path_ok && is_pow2(c.dir_blk) && c.dir_blk <= t->N && is_pow2(c.col_seg) && c.col_seg <= MAXSEG &&
           (c.tma == 0 || c.tma == 1) && (c.ppc == 64 || c.ppc == 128 || c.ppc == 256);
}

void apply_cand(tracker* t, const Cand& c)
{
    if (t->dir_blk == c.dir_blk && t->col_seg == c.col_seg && t->auto_tma == (c.tma != 0) && t->dir_ppc == c.ppc) return;
    t->dir_blk = c.dir_blk;
    t->col_seg = c.col_seg;
    t->auto_tma = c.tma != 0;
    t->dir_ppc = c.ppc;
    t->gen += 1;                      // captured step graphs hold the old launch shapes
}

void remember_tuning(tracker* t, const std::string& key, const Cand& c, bool persist)
{
    if (t->step_tune.size() >= kCacheMax) t->step_tune.erase(t->step_tune.begin());
    t->step_tune.push_back({key, {c.path, c.dir_blk, c.col_seg, c.tma, c.ppc}});
    const char* path = getenv("TRK_TUNE_CACHE");
    if (!persist || !path || !*path) return;
    if (FILE* f = fopen(path, "a")) {
        fprintf(f, "%s|%d %d %d %d %d\n", key.c_str(), c.path, c.dir_blk, c.col_seg, c.tma, c.ppc);
        fclose(f);
    }
}

bool lookup_tuning(const tracker* t, const std::string& key, Cand* out)
{
    for (auto it = t->step_tune.rbegin(); it != t->step_tune.rend(); ++it)
        if (it->first == key) {
            *out = Cand{it->second[0], it->second[1], it->second[2], it->second[3], it->second[4]};
            return true;
        }
    return false;
}

// Decisions of earlier processes (TRK_TUNE_CACHE): lines "key|path dir_blk
// col_seg tma ppc"; malformed lines and values this tracker cannot run are skipped.
void load_tune_file(tracker* t)
{
    const char* path = getenv("TRK_TUNE_CACHE");
    if (!path || !*path) return;
    FILE* f = fopen(path, "r");
    if (!f) return;
    char line[512];
    while (fgets(line, sizeof(line), f)) {
        char* bar = strchr(line, '|');
        if (!bar) continue;
        *bar = 0;
        Cand c{};
        if (sscanf(bar + 1, "%d %d %d %d %d", &c.path, &c.dir_blk, &c.col_seg, &c.tma, &c.ppc) != 5 || !valid_cand(t, c))
            continue;
        remember_tuning(t, line, c, false);
    }
    fclose(f);
}

// Particles per CTA of the direct kernel when nothing was timed: the largest
// of 256, 128, 64 that still gives three CTAs per SM (smaller sets leave SMs
// idle with 256: at 256^3 and 1.5e-3 particles per cell, 25,000 particles,
// 128 per CTA took 0.044 ms per RK2 step against 0.065 ms).
int default_ppc(const tracker* t, int64_t np)
{
    for (int p : {256, 128})
        if ((np + p - 1) / p >= 3 * (int64_t)std::max(t->nsm, 1)) return p;
    return 64;
}

// The candidates for np particles (measured on GB300, 256^3 float32, spline
// I = 6, RK2 and AB2 from 1.5e-3 to 1/2 particle per cell: the winners were
// always among these): the column kernel with segments of 8 and 16 slabs
// from kProbeMin particles per cell on; the block kernel with both halo
// copies (the tensor-copy box wins where few particles share a halo, the
// bank-conflict-free cp.async layout where many do) from kBlockMin on, or from
// kProbeMin on without a column kernel; the direct kernel with binning edges
// 8 and 16 up to one particle per cell.  Other block shapes than the default
// run only the direct kernel.
constexpr double kBlockMin = 0.1;
std::vector<Cand> tune_candidates(const tracker* t, int64_t np)
{
    std::vector<Cand> c;
    const double dens = (double)np / ((double)t->N * t->N * t->N);
    if (!default_shape(t)) return {Cand{TRK_STEP_DIRECT, BLK, 8, 1}};
    const bool col = column_available(t);
    if (col && dens >= kProbeMin)
        for (int seg : {8, 16})
            if (seg <= t->g.nb3) c.push_back({TRK_STEP_COLUMN, BLK, seg, 1});
    if (dens >= (col ? kBlockMin : kProbeMin)) {
        if (t->tmap_ok[0] && t->tmap_ok[1]) c.push_back({TRK_STEP_BLOCK, BLK, 8, 1});
        c.push_back({TRK_STEP_BLOCK, BLK, 8, 0});
    }
    if (dens <= 1.0)
        for (int b : {8, 16})
            for (int ppc : {256, 128})
                if (b <= t->N) c.push_back({TRK_STEP_DIRECT, b, 8, 1, ppc});
    return c;
}

// keys and block counts of the grouped state pos_s[cur] in geometry bg (after
// a change of binning geometry between two steps)
int rekey(tracker* t, int64_t np, int cur, const BinGeom& bg)
{
    ProfScope ps(t, PROF_BIN);
    CUDA_TRY(cudaMemsetAsync(t->d_counts, 0, (size_t)bg.nb * sizeof(uint32_t), t->stream));
    CUDA_TRY(launch_keys_count(bg.g, np, t->pos_s[cur], t->keys, t->d_counts, t->d_flags, t->stream));
    t->launches += 1;
    return TRK_OK;
}

uint64_t dbits(double x)
{
    uint64_t u;
    memcpy(&u, &x, 8);
    return u;
}

}  // namespace

extern "C" {

const char* tracker_last_error(void) { return g_err; }

int tracker_create(tracker** out, int N, double L, int family, int I, int m, int storage, void* stream)
{
    g_err[0] = 0;
    if (!out) return fail(TRK_EINVAL, "out is NULL");
    *out = nullptr;
    if (!is_pow2(N) || N < 16 || N > 1024) return fail(TRK_EINVAL, "N=%d must be a power of two in [16, 1024]", N);
    if (!(L > 0) || !std::isfinite(L)) return fail(TRK_EINVAL, "L must be finite and > 0");
    if (family != TRK_LAGRANGE && family != TRK_SPLINE) return fail(TRK_EINVAL, "unknown kernel family %d", family);
    if (I != 4 && I != 6 && I != 8) return fail(TRK_EINVAL, "I=%d unsupported (4, 6, 8)", I);
    if (family == TRK_SPLINE && (m < 0 || m > I / 2)) return fail(TRK_EINVAL, "spline smoothness m=%d outside [0, %d]", m, I / 2);
    if (storage != TRK_F64 && storage != TRK_F32 && storage != TRK_BF16X2) return fail(TRK_EINVAL, "unknown storage %d", storage);
    const int tab = find_table(family, I, family == TRK_LAGRANGE ? 0 : m);
    if (tab < 0) return fail(TRK_EINVAL, "no coefficient table for (family=%d, I=%d, m=%d)", family, I, m);
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return fail(TRK_ECUDA, "no CUDA device");
    }
    tracker* t = new tracker();
    if (cudaGetDevice(&t->device) != cudaSuccess) {
        cudaGetLastError();
        delete t;
        return fail(TRK_ECUDA, "no current CUDA device");
    }
    t->N = N;
    t->L = L;
    t->family = family;
    t->I = I;
    t->m = m;
    t->storage = storage;
    t->tab = tab;
    t->deg = kTables[tab].deg;
    t->deg_hi = t->deg > I - 1;
    t->stream = reinterpret_cast<cudaStream_t>(stream);
    t->g.N = N;
    t->g.mask = N - 1;
    t->g.inv_delta = (double)N / L;
    int rc = set_geometry(t, BLK, BLK, BLK);
    if (rc == TRK_OK && dev_alloc(&t->d_colctr, sizeof(int)) != cudaSuccess)
        rc = fail(TRK_ENOMEM, "cannot allocate the column work counter");
    if (rc == TRK_OK && dev_alloc(&t->d_flags, NUM_FLAGS * sizeof(int)) != cudaSuccess)
        rc = fail(TRK_ENOMEM, "cannot allocate device flags");
    if (rc == TRK_OK && cudaMemset(t->d_flags, 0, NUM_FLAGS * sizeof(int)) != cudaSuccess)
        rc = fail(TRK_ECUDA, "cudaMemset flags failed");
    if (rc == TRK_OK && (cudaStreamCreateWithFlags(&t->gstream, cudaStreamNonBlocking) != cudaSuccess ||
                         cudaEventCreateWithFlags(&t->gev[0], cudaEventDisableTiming) != cudaSuccess ||
                         cudaEventCreateWithFlags(&t->gev[1], cudaEventDisableTiming) != cudaSuccess))
        rc = fail(TRK_ECUDA, "cannot create the graph stream");
    if (rc == TRK_OK) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&t->nsm, cudaDevAttrMultiProcessorCount, dev);
    }
    if (rc != TRK_OK) {
        tracker_destroy(t);
        return rc;
    }
    load_tune_file(t);
    *out = t;
    return TRK_OK;
}

int tracker_destroy(tracker* t)
{
    if (!t) return TRK_OK;
    // release the buffers on the device that holds them, then restore the caller's device
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) cudaGetLastError();
    if (t->device >= 0 && cur != t->device) cudaSetDevice(t->device);
    if (t->stream) cudaStreamSynchronize(t->stream);
    else cudaDeviceSynchronize();
    dev_free(t->field);
    dev_free(t->sort_scratch);
    dev_free(t->keys);
    dev_free(t->keys_sorted);
    dev_free(t->perm);
    dev_free(t->offsets);
    for (int i = 0; i < 2; ++i) {
        dev_free(t->pos_s[i]);
        dev_free(t->id_s[i]);
        dev_free(t->rhs_s[i]);
    }
    if (t->gstream) cudaStreamSynchronize(t->gstream);
    dev_free(t->d_flags);
    dev_free(t->adj_buf);
    dev_free(t->adj_scratch);
    if (t->adv_graph.exec) cudaGraphExecDestroy(t->adv_graph.exec);
    if (t->batch_graph.exec) cudaGraphExecDestroy(t->batch_graph.exec);
    for (SetState& ss : t->sets) {
        for (void* p : {(void*)ss.keys, (void*)ss.counts, (void*)ss.perm, (void*)ss.offsets, (void*)ss.list,
                        (void*)ss.count, (void*)ss.pos_s[0], (void*)ss.pos_s[1], (void*)ss.id_s[0], (void*)ss.id_s[1],
                        (void*)ss.rhs_s[0], (void*)ss.rhs_s[1]})
            dev_free(p);
    }
    dev_free(t->ne_scratch);
    dev_free(t->d_desc);
    dev_free(t->d_ctr);
    dev_free(t->d_colctr);
    dev_free(t->d_counts);
    dev_free(t->d_cursor);
    dev_free(t->d_scan_tmp);
    destroy_nm_texture(t);
    dev_free(t->field_nm);
    if (t->gev[0]) cudaEventDestroy(t->gev[0]);
    if (t->gev[1]) cudaEventDestroy(t->gev[1]);
    if (t->gstream) cudaStreamDestroy(t->gstream);
    for (cudaEvent_t e : t->ev_pool) cudaEventDestroy(e);
    if (cur >= 0 && cur != t->device) cudaSetDevice(cur);
    delete t;
    return TRK_OK;
}

int tracker_profile(tracker* t, int enable)
{
    if (!t) return fail(TRK_EINVAL, "tracker is NULL");
    if (int rc_dev = check_device(t)) return rc_dev;
    if (enable) {
        CUDA_TRY(cudaStreamSynchronize(t->stream));
        t->ev_used = 0;
        for (int c = 0; c < 3; ++c) {
            t->prof_pairs[c].clear();
            t->prof_launches[c] = 0;
        }
    }
    t->prof = enable != 0;
    return TRK_OK;
}

int tracker_profile_read(tracker* t, double* ms, int64_t* launches)
{
    if (!t || !ms || !launches) return fail(TRK_EINVAL, "NULL argument");
    if (int rc_dev = check_device(t)) return rc_dev;
    CUDA_TRY(cudaStreamSynchronize(t->stream));
    for (int c = 0; c < 3; ++c) {
        double tot = 0;
        for (auto& pr : t->prof_pairs[c]) {
            float x = 0;
            CUDA_TRY(cudaEventElapsedTime(&x, pr.first, pr.second));
            tot += x;
        }
        ms[c] = tot;
        launches[c] = t->prof_launches[c];
    }
    return TRK_OK;
}

int tracker_set_stream(tracker* t, void* stream)
{
    if (!t) return fail(TRK_EINVAL, "tracker is NULL");
    t->stream = reinterpret_cast<cudaStream_t>(stream);
    return TRK_OK;
}

int tracker_sync(tracker* t)
{
    if (!t) return fail(TRK_EINVAL, "tracker is NULL");
    if (int rc_dev = check_device(t)) return rc_dev;
    CUDA_TRY(cudaStreamSynchronize(t->stream));
    int h[NUM_FLAGS];
    CUDA_TRY(cudaMemcpy(h, t->d_flags, sizeof(h), cudaMemcpyDeviceToHost));
    CUDA_TRY(cudaMemset(t->d_flags, 0, sizeof(h)));
    if (h[FLAG_NONFINITE]) return fail(TRK_ENONFINITE, "a position was non-finite or beyond 2^51 cells");
    if (h[FLAG_BINNING]) return fail(TRK_ECUDA, "internal error: block counts did not match the binned particles");
    if (h[FLAG_HALO_TIMEOUT]) return fail(TRK_ECUDA, "internal error: a halo tensor copy did not complete (block skipped)");
    if (h[FLAG_CFL]) return fail(TRK_ECFL, "a particle moved more than one cell in one stage (result computed exactly)");
    return TRK_OK;
}

int tracker_set_field(tracker* t, const void* src, int C, int src_dtype, int src_on_host)
{
    if (!t) return fail(TRK_EINVAL, "tracker is NULL");
    if (int rc_dev = check_device(t)) return rc_dev;
    if (!src) return fail(TRK_EINVAL, "src is NULL");
    if (C < 1 || C > 16) return fail(TRK_EINVAL, "C=%d outside [1, 16]", C);
    if (src_dtype != TRK_DTYPE_F64 && src_dtype != TRK_DTYPE_F32) return fail(TRK_EINVAL, "unknown src_dtype %d", src_dtype);
    const int64_t n = (int64_t)C * t->N * t->N * t->N;
    const int64_t NP = t->N + 2 * PAD;
    const int64_t n_stored = (int64_t)C * NP * NP * NP;
    const size_t esz = t->storage == TRK_F64 ? 8 : 4;
    if (t->C != C || !t->field) {
        dev_free(t->field);
        t->field = nullptr;
        t->C = 0;
        if (dev_alloc(&t->field, (size_t)n_stored * esz) != cudaSuccess) {
            cudaGetLastError();
            return fail(TRK_ENOMEM, "cannot allocate field storage (%zu bytes)", (size_t)n_stored * esz);
        }
        t->C = C;
    }
    const size_t src_bytes = (size_t)n * (src_dtype == TRK_DTYPE_F64 ? 8 : 4);
    const void* dsrc = src;
    void* staging = nullptr;
    if (src_on_host) {
        if (dev_alloc(&staging, src_bytes) != cudaSuccess) {
            cudaGetLastError();
            return fail(TRK_ENOMEM, "cannot allocate staging buffer (%zu bytes)", src_bytes);
        }
        CUDA_TRY(cudaMemcpyAsync(staging, src, src_bytes, cudaMemcpyHostToDevice, t->stream));
        dsrc = staging;
    }
    {
        ProfScope ps(t, PROF_OTHER);
        CUDA_TRY(launch_convert_field(t->storage, src_dtype == TRK_DTYPE_F64, dsrc, C, t->N, t->field, t->stream));
    }
    t->nm_skip = false;
    t->nm_valid = false;              // the node-major copy is refreshed before its next use
    t->launches += 1;
    build_tmaps(t);
    if (staging) {
        CUDA_TRY(cudaStreamSynchronize(t->stream));
        dev_free(staging);
    }
    return TRK_OK;
}

int tracker_set_block(tracker* t, int bx, int by, int bz)
{
    if (!t) return fail(TRK_EINVAL, "tracker is NULL");
    if (int rc_dev = check_device(t)) return rc_dev;
    return set_geometry(t, bx, by, bz);
}

int64_t tracker_num_blocks(const tracker* t) { return t ? t->nblocks : -1; }

int tracker_set_step_kernel(tracker* t, int kind)
{
    if (!t) return fail(TRK_EINVAL, "tracker is NULL");
    if (kind != TRK_STEP_AUTO && kind != TRK_STEP_BLOCK && kind != TRK_STEP_COLUMN && kind != TRK_STEP_DIRECT)
        return fail(TRK_EINVAL, "unknown step kernel %d", kind);
    if (kind == TRK_STEP_COLUMN && !column_available(t))
        return fail(TRK_EINVAL, "no column kernel for this tracker (needs F32 storage, I = 4 or 6, 8x8x8 blocks)");
    t->step_kernel = kind;
    t->gen += 1;                      // captured step graphs hold the other kernels
    return TRK_OK;
}

int tracker_step_kernel_for(const tracker* t, int64_t np)
{
    if (!t) return fail(TRK_EINVAL, "tracker is NULL");
    if (np < 0) return fail(TRK_EINVAL, "np=%lld < 0", (long long)np);
    return step_path(t, np);
}

int tracker_last_step_kernel(const tracker* t)
{
    if (!t) return fail(TRK_EINVAL, "tracker is NULL");
    return t->last_kernel;
}

int tracker_set_tuning(tracker* t, const trk_tuning* p)
{
    if (!t) return fail(TRK_EINVAL, "tracker is NULL");
    if (!p) {   // back to the automatic choice
        t->step_kernel = TRK_STEP_AUTO;
        t->halo_copy = TRK_HALO_AUTO;
        apply_cand(t, Cand{TRK_STEP_AUTO, BLK, 8, 1});
        t->gen += 1;
        return TRK_OK;
    }
    if (p->step_kernel != TRK_STEP_BLOCK && p->step_kernel != TRK_STEP_COLUMN && p->step_kernel != TRK_STEP_DIRECT)
        return fail(TRK_EINVAL, "step_kernel must be TRK_STEP_BLOCK, _COLUMN or _DIRECT");
    if (p->halo_copy != TRK_HALO_ASYNC && p->halo_copy != TRK_HALO_TMA)
        return fail(TRK_EINVAL, "halo_copy must be TRK_HALO_ASYNC or TRK_HALO_TMA");
    const Cand c{p->step_kernel, p->direct_block, p->column_segment, p->halo_copy == TRK_HALO_TMA ? 1 : 0,
                 p->direct_particles == 0 ? 256 : p->direct_particles};
    if (!valid_cand(t, c))
        return fail(TRK_EINVAL, "invalid tuning (direct_block a power of two <= N, column_segment a power of two "
                                "<= %d, direct_particles 128 or 256, a column kernel only for F32 storage with "
                                "I = 4, 6 and 8^3 blocks)", MAXSEG);
    t->step_kernel = c.path;
    t->halo_copy = p->halo_copy;
    apply_cand(t, c);
    t->gen += 1;
    return TRK_OK;
}

int tracker_get_tuning(const tracker* t, trk_tuning* out)
{
    if (!t || !out) return fail(TRK_EINVAL, "NULL argument");
    out->step_kernel = t->last_tuning[0];
    out->direct_block = t->last_tuning[1];
    out->column_segment = t->last_tuning[2];
    out->halo_copy = t->last_tuning[3] ? TRK_HALO_TMA : TRK_HALO_ASYNC;
    out->direct_particles = t->last_tuning[4];
    out->source = t->tune_source;
    return TRK_OK;
}

int tracker_set_halo_copy(tracker* t, int kind)
{
    if (!t) return fail(TRK_EINVAL, "tracker is NULL");
    if (kind != TRK_HALO_AUTO && kind != TRK_HALO_ASYNC && kind != TRK_HALO_TMA)
        return fail(TRK_EINVAL, "unknown halo copy %d", kind);
    t->halo_copy = kind;
    t->gen += 1;                      // captured step graphs hold the other kernels
    return TRK_OK;
}

int tracker_halo_copy(const tracker* t, int mode)
{
    if (!t) return fail(TRK_EINVAL, "tracker is NULL");
    if (mode != 0 && mode != 1) return fail(TRK_EINVAL, "mode must be 0 (interpolation, AB) or 1 (RK2)");
    return halo_tmap(t, mode ? MODE_RK2 : MODE_INTERP) ? TRK_HALO_TMA : TRK_HALO_ASYNC;
}

int tracker_field_texture(const tracker* t)
{
    if (!t) return fail(TRK_EINVAL, "tracker is NULL");
    return t->nm_valid && t->nm_tex && t->C == 3 ? 1 : 0;
}

int64_t tracker_launch_count(const tracker* t) { return t ? t->launches : -1; }

int tracker_bin(tracker* t, int64_t np, const double* pos, int32_t* keys, int32_t* perm, int32_t* offsets)
{
    if (!t) return fail(TRK_EINVAL, "tracker is NULL");
    if (int rc_dev = check_device(t)) return rc_dev;
    int rc = check_np(np);
    if (rc) return rc;
    if (np > 0 && (!pos || !perm)) return fail(TRK_EINVAL, "pos and perm must not be NULL");
    if (!offsets) return fail(TRK_EINVAL, "offsets must not be NULL");
    for (const void* p : {(const void*)(np > 0 ? pos : nullptr), (const void*)keys, (const void*)(np > 0 ? perm : nullptr),
                          (const void*)offsets})
        if (p && !device_pointer_ok(p, t->device))
            return fail(TRK_EINVAL, "tracker_bin: every array must be device memory of the tracker's device %d", t->device);
    if ((rc = ensure_sort(t, np)) || (rc = ensure_radix(t, np))) return rc;
    uint32_t* k = keys ? reinterpret_cast<uint32_t*>(keys) : t->keys;
    return bin_into(t, np, pos, k, perm, offsets);
}

int tracker_interpolate(tracker* t, int64_t np, const double* pos, void* out, int out_dtype, int deriv)
{
    if (!t) return fail(TRK_EINVAL, "tracker is NULL");
    if (int rc_dev = check_device(t)) return rc_dev;
    int rc = check_np(np);
    if (rc) return rc;
    if (!t->field) return fail(TRK_ENOFIELD, "no field set");
    if (np > 0 && (!pos || !out)) return fail(TRK_EINVAL, "pos and out must not be NULL");
    if (out_dtype != TRK_DTYPE_F64 && out_dtype != TRK_DTYPE_F32) return fail(TRK_EINVAL, "unknown out_dtype %d", out_dtype);
    bool direct = step_path(t, np) == TRK_STEP_DIRECT;
    // AUTO: a cached timing decision, or time the block and the direct kernel
    // now (they write the same values; the better one depends on density, C
    // and the grid)
    bool probe = false;
    int interp_choice = -1;   // remembered: 0 block (cp.async halo), 1 block (tensor copy), 2 direct
    const uint64_t sig = mix(mix(mix(mix(0x1f, (uint64_t)np), (uint64_t)t->C), (uint64_t)deriv), (uint64_t)out_dtype);
    const bool block_shape = t->g.lb1 == LBLK && t->g.lb2 == LBLK && t->g.lb3 == LBLK;
    if (t->step_kernel == TRK_STEP_AUTO && np > 0 && block_shape) {
        int cached = -1;
        for (const auto& e : t->interp_cache)
            if (e.first == sig) cached = e.second;
        if (cached >= 0) {
            direct = cached == 2;
            interp_choice = cached;
        } else {
            const double dens = (double)np / ((double)t->N * t->N * t->N);
            cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
            CUDA_TRY(cudaStreamIsCapturing(t->stream, &cs));
            probe = dens >= kProbeMin && dens <= kProbeMax && cs == cudaStreamCaptureStatusNone;
        }
    }
    if (!direct && (rc = check_block_kernel_shape(t))) return rc;
    if (np == 0) return TRK_OK;
    if ((rc = ensure_sort(t, np))) return rc;
    if ((direct || probe) && (rc = ensure_node_major(t))) return rc;
    // the kernels read the positions through the permutation (gathering them
    // into block order first measured slower overall: 1024^3, I = 8, 2^27
    // tracers, the block kernel gains 5.2 ms, the gather costs 7.8 ms)
    if ((rc = bin_counting(t, np, pos))) return rc;
    BlockArgs a = base_args(t);
    a.np = np;
    a.perm = t->perm;
    a.pos_in = pos;
    a.ppc = default_ppc(t, np);
    a.out = out;
    a.out_f64 = out_dtype == TRK_DTYPE_F64;
    const int mode = deriv ? MODE_INTERP_DERIV : MODE_INTERP;
    if (probe) {
        // the block kernel with each halo copy it has, then the direct kernel;
        // all write the same values, the fastest is remembered
        const bool saved = t->auto_tma;
        std::vector<int> kinds;   // 0: block, cp.async halo; 1: block, tensor copy; 2: direct
        if (t->halo_copy == TRK_HALO_AUTO && halo_tmap_exists(t, mode)) kinds.push_back(1);
        kinds.push_back(t->halo_copy == TRK_HALO_TMA && halo_tmap_exists(t, mode) ? 1 : 0);
        kinds.push_back(2);
        std::vector<cudaEvent_t> ev(kinds.size() + 1, nullptr);
        for (auto& e : ev)
            if (cudaEventCreate(&e) != cudaSuccess) rc = fail(TRK_ECUDA, "cudaEventCreate failed");
        std::vector<float> ms(kinds.size(), 0.f);
        if (rc == TRK_OK) {
            cudaError_t e = cudaEventRecord(ev[0], t->stream);
            for (size_t i = 0; e == cudaSuccess && i < kinds.size(); ++i) {
                t->auto_tma = kinds[i] == 1;
                e = kinds[i] == 2 ? launch_direct(t, mode, a) : launch_block(t, mode, a);
                if (e == cudaSuccess) e = cudaEventRecord(ev[i + 1], t->stream);
            }
            if (e == cudaSuccess) e = cudaEventSynchronize(ev.back());
            for (size_t i = 0; e == cudaSuccess && i < kinds.size(); ++i) e = cudaEventElapsedTime(&ms[i], ev[i], ev[i + 1]);
            if (e != cudaSuccess) rc = fail(TRK_ECUDA, "timing the interpolation kernels: %s", cudaGetErrorString(e));
        }
        t->auto_tma = saved;
        for (auto& e : ev)
            if (e) cudaEventDestroy(e);
        if (rc) return rc;
        size_t best = 0;
        for (size_t i = 1; i < kinds.size(); ++i)
            if (ms[i] < ms[best]) best = i;
        remember(t->interp_cache, sig, kinds[best]);
        t->last_kernel = kinds[best] == 2 ? TRK_STEP_DIRECT : TRK_STEP_BLOCK;
        return TRK_OK;
    }
    if (direct) {
        CUDA_TRY(launch_direct(t, mode, a));
    } else {
        const bool saved = t->auto_tma;
        if (interp_choice >= 0) t->auto_tma = interp_choice == 1;
        const cudaError_t e = launch_block(t, mode, a);
        t->auto_tma = saved;
        CUDA_TRY(e);
    }
    t->last_kernel = direct ? TRK_STEP_DIRECT : TRK_STEP_BLOCK;
    return TRK_OK;
}

int tracker_advance(tracker* t, int64_t np, double* pos, float* rhs, double dt, int steps, int scheme,
                    int history_valid)
{
    if (!t) return fail(TRK_EINVAL, "tracker is NULL");
    if (int rc_dev = check_device(t)) return rc_dev;
    int rc = check_np(np);
    if (rc) return rc;
    if (!t->field) return fail(TRK_ENOFIELD, "no field set");
    if (t->C != 3) return fail(TRK_EINVAL, "advection needs a 3-component field (C=%d)", t->C);
    if (scheme != TRK_RK2 && scheme != TRK_AB2 && scheme != TRK_AB3 && scheme != TRK_AB4)
        return fail(TRK_EINVAL, "unknown scheme %d", scheme);
    const int k = scheme == TRK_RK2 ? 0 : scheme + 1;   // Adams-Bashforth order
    if (k && !rhs && np > 0) return fail(TRK_EINVAL, "AB%d needs the rhs history array", k);
    if (k && (history_valid < 0 || history_valid > k - 1))
        return fail(TRK_EINVAL, "history_valid=%d outside [0, %d] for AB%d", history_valid, k - 1, k);
    if (!std::isfinite(dt)) return fail(TRK_EINVAL, "dt must be finite");
    if (steps < 0) return fail(TRK_EINVAL, "steps=%d < 0", steps);
    if (np > 0 && !pos) return fail(TRK_EINVAL, "pos must not be NULL");
    const int mode = k ? MODE_AB2 : MODE_RK2;
    const int ab_order = k ? k : 2;
    int path = step_path(t, np);
    // AUTO: a remembered tuning decision for this workload, or time the
    // candidates now (steps of this call), or the density rule with the
    // default launch shapes
    std::vector<Cand> cands;
    std::string key;
    t->tune_source = t->step_kernel == TRK_STEP_AUTO ? TRK_TUNE_DEFAULT : TRK_TUNE_FIXED;
    if (t->step_kernel == TRK_STEP_AUTO && np > 0) {
        key = tune_key(t, np, mode, ab_order);
        Cand hit{};
        if (lookup_tuning(t, key, &hit)) {
            apply_cand(t, hit);
            path = hit.path;
            t->tune_source = TRK_TUNE_CACHED;
        } else {
            cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
            CUDA_TRY(cudaStreamIsCapturing(t->stream, &cs));
            cands = tune_candidates(t, np);
            const bool timed = np >= kTuneMinNp && cands.size() >= 2 &&
                               steps >= kTuneStepsPerCand * (int)cands.size() + 2 && cs == cudaStreamCaptureStatusNone;
            if (!timed) cands.clear();
            apply_cand(t, Cand{path, BLK, 8, 1, default_ppc(t, np)});
        }
    }
    if (path != TRK_STEP_DIRECT && (rc = check_block_kernel_shape(t))) return rc;
    if (np == 0 || steps == 0) return TRK_OK;
    if ((rc = ensure_sort(t, np))) return rc;
    if ((rc = ensure_state(t, np))) return rc;
    bool any_direct = path == TRK_STEP_DIRECT;
    for (const Cand& c : cands) {
        any_direct = any_direct || c.path == TRK_STEP_DIRECT;
        Cand save{path, t->dir_blk, t->col_seg, t->auto_tma, t->dir_ppc};
        apply_cand(t, c);
        rc = ensure_bin(t, geom_of(t, c.path).nb);
        apply_cand(t, save);
        if (rc) return rc;
    }
    if ((rc = ensure_bin(t, geom_of(t, path).nb))) return rc;
    if (any_direct && (rc = ensure_node_major(t))) return rc;
    // initial keys and block counts from the caller's positions
    GridGeom last_g = geom_of(t, path).g;
    {
        const BinGeom bg = geom_of(t, path);
        ProfScope ps(t, PROF_BIN);
        CUDA_TRY(cudaMemsetAsync(t->d_counts, 0, (size_t)bg.nb * sizeof(uint32_t), t->stream));
        CUDA_TRY(launch_keys_count(bg.g, np, pos, t->keys, t->d_counts, t->d_flags, t->stream));
        t->launches += 1;
    }
    // the first step reads the caller's arrays; the others ping-pong between
    // the tracker's state buffers.  AB steps run one by one until the history
    // is full (k - 1 entries); from then on every step is the same and pairs
    // of steps are replayed from a CUDA graph.
    int hist = k ? history_valid : 0;
    int cur = 0, rest = steps;
    bool first = true;
    auto eager = [&](int p) {
        const BinGeom bg = geom_of(t, p);
        if (!first && !same_geom(bg.g, last_g)) {   // counts of the last step are in another geometry
            const int r = rekey(t, np, cur, bg);
            if (r) return r;
        }
        last_g = bg.g;
        const int r = advance_step(t, np, p, mode, ab_order, hist, dt, cur, first, first ? pos : nullptr,
                                   first ? rhs : nullptr);
        if (r == TRK_OK) {
            first = false;
            cur ^= 1;
            --rest;
            if (k) hist = std::min(hist + 1, k - 1);
        }
        return r;
    };
    if ((rc = eager(path))) return rc;
    if (!cands.empty()) {
        // kTuneStepsPerCand timed steps per candidate, then the fastest
        const int nst = kTuneStepsPerCand * (int)cands.size();
        std::vector<cudaEvent_t> ev(nst + 1, nullptr);
        for (auto& e : ev)
            if (cudaEventCreate(&e) != cudaSuccess) rc = fail(TRK_ECUDA, "cudaEventCreate failed");
        for (int i = 0; rc == TRK_OK && i < nst; ++i) {
            const Cand& c = cands[i / kTuneStepsPerCand];
            apply_cand(t, c);
            if (cudaEventRecord(ev[i], t->stream) != cudaSuccess) rc = fail(TRK_ECUDA, "cudaEventRecord failed");
            if (rc == TRK_OK) rc = eager(c.path);
        }
        std::vector<float> ms(nst, 0.f);
        if (rc == TRK_OK && (cudaEventRecord(ev[nst], t->stream) != cudaSuccess || cudaEventSynchronize(ev[nst]) != cudaSuccess))
            rc = fail(TRK_ECUDA, "timing the step candidates failed");
        for (int i = 0; rc == TRK_OK && i < nst; ++i)
            if (cudaEventElapsedTime(&ms[i], ev[i], ev[i + 1]) != cudaSuccess) rc = fail(TRK_ECUDA, "cudaEventElapsedTime failed");
        for (auto& e : ev)
            if (e) cudaEventDestroy(e);
        if (rc) return rc;
        int best = 0;
        float best_ms = 0.f;
        for (int c = 0; c < (int)cands.size(); ++c) {
            float m = ms[c * kTuneStepsPerCand];
            for (int r = 1; r < kTuneStepsPerCand; ++r) m = std::min(m, ms[c * kTuneStepsPerCand + r]);
            if (c == 0 || m < best_ms) {
                best = c;
                best_ms = m;
            }
        }
        apply_cand(t, cands[best]);
        path = cands[best].path;
        remember_tuning(t, key, cands[best], true);
        t->tune_source = TRK_TUNE_TIMED;
        const BinGeom bg = geom_of(t, path);
        if (!same_geom(bg.g, last_g)) {
            if ((rc = rekey(t, np, cur, bg))) return rc;
            last_g = bg.g;
        }
    }
    for (; rest > 0 && k && hist < k - 1;)
        if ((rc = eager(path))) return rc;
    if (!t->prof && rest >= 2) {
        uint64_t key = mix(mix(mix(mix(0, (uint64_t)np), (uint64_t)mode), t->gen), dbits(dt));
        key = mix(mix(mix(key, (uint64_t)(uintptr_t)t->field), (uint64_t)ab_order), (uint64_t)path);
        key = mix(mix(mix(mix(key, (uint64_t)t->dir_blk), (uint64_t)t->col_seg), (uint64_t)t->auto_tma),
                  (uint64_t)t->dir_ppc);
        const int c0 = cur;
        rc = replay_graph(t, t->adv_graph, mix(key, (uint64_t)c0), rest / 2, [&]() {
            int r = advance_step(t, np, path, mode, ab_order, hist, dt, c0, false, nullptr, nullptr);
            return r ? r : advance_step(t, np, path, mode, ab_order, hist, dt, c0 ^ 1, false, nullptr, nullptr);
        });
        if (rc) return rc;
        rest -= 2 * (rest / 2);
    }
    for (; rest > 0; --rest) {
        if ((rc = advance_step(t, np, path, mode, ab_order, hist, dt, cur, false, nullptr, nullptr))) return rc;
        cur ^= 1;
    }
    t->last_kernel = path;
    t->last_tuning = {path, t->dir_blk, t->col_seg, halo_tmap(t, mode) ? 1 : 0, t->dir_ppc};
    ProfScope ps(t, PROF_OTHER);
    CUDA_TRY(launch_unpermute_pos(np, t->pos_s[cur], t->id_s[cur], pos, t->stream));
    t->launches += 1;
    if (k) {
        CUDA_TRY(launch_unpermute_rhs(np, t->rhs_s[cur], t->id_s[cur], rhs, 3 * (k - 1), t->stream));
        t->launches += 1;
    }
    return TRK_OK;
}

static cudaError_t launch_adjoint(tracker* t, const AdjArgs& a)
{
    ProfScope ps(t, PROF_STEP);
    t->launches += 1;
    switch (t->I) {
        case 4: return launch_adjoint_i4(a, t->nblocks, t->deg_hi, t->stream);
        case 6: return launch_adjoint_i6(a, t->nblocks, t->deg_hi, t->stream);
        default: return launch_adjoint_i8(a, t->nblocks, t->deg_hi, t->stream);
    }
}

static int ensure_set(tracker* t, SetState& ss, int64_t np)
{
    if (np <= ss.cap && ss.nb == t->nblocks) return TRK_OK;
    t->gen += 1;
    for (void* p : {(void*)ss.keys, (void*)ss.counts, (void*)ss.perm, (void*)ss.offsets, (void*)ss.list,
                    (void*)ss.count, (void*)ss.pos_s[0], (void*)ss.pos_s[1], (void*)ss.id_s[0], (void*)ss.id_s[1],
                    (void*)ss.rhs_s[0], (void*)ss.rhs_s[1]})
        dev_free(p);
    ss = SetState{};
    bool ok = dev_alloc(&ss.keys, (size_t)np * 4) == cudaSuccess &&
              dev_alloc(&ss.counts, (size_t)t->nblocks * 4) == cudaSuccess &&
              dev_alloc(&ss.perm, (size_t)np * 4) == cudaSuccess &&
              dev_alloc(&ss.offsets, (size_t)(t->nblocks + 1) * 4) == cudaSuccess &&
              dev_alloc(&ss.list, (size_t)t->nblocks * 4) == cudaSuccess && dev_alloc(&ss.count, 4) == cudaSuccess;
    for (int i = 0; i < 2 && ok; ++i)
        ok = dev_alloc(&ss.pos_s[i], (size_t)np * 24) == cudaSuccess && dev_alloc(&ss.id_s[i], (size_t)np * 4) == cudaSuccess &&
             dev_alloc(&ss.rhs_s[i], (size_t)np * 12) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        return fail(TRK_ENOMEM, "cannot allocate the buffers of a particle set (%lld particles)", (long long)np);
    }
    ss.cap = np;
    ss.nb = t->nblocks;
    return TRK_OK;
}

// Initial keys and block counts of one set from positions in the caller's order.
static int keys_set(tracker* t, SetState& ss, int64_t np, const double* pos)
{
    ProfScope ps(t, PROF_BIN);
    CUDA_TRY(cudaMemsetAsync(ss.counts, 0, (size_t)t->nblocks * sizeof(uint32_t), t->stream));
    CUDA_TRY(launch_keys_count(t->g, np, pos, ss.keys, ss.counts, t->d_flags, t->stream));
    t->launches += 1;
    return TRK_OK;
}

// Re-binning of one set by counting sort: the block counts (from keys_set, or
// added by the previous step's kernel) scanned into offsets and cursors (the
// counts are left zero), the permutation, and (halo path) the non-empty block
// list.  The cursors and scan scratch are the tracker's, shared by the sets,
// which are binned one after another on the stream.
static int bin_set(tracker* t, SetState& ss, int64_t np, bool direct)
{
    ProfScope ps(t, PROF_BIN);
    CUDA_TRY(launch_count_scan(ss.counts, t->nblocks, ss.offsets, t->d_cursor, t->d_scan_tmp, t->stream,
                               &t->launches));
    CUDA_TRY(launch_scatter_perm(np, ss.keys, t->d_cursor, ss.perm, t->d_flags, t->stream));
    t->launches += 1;
    if (!direct) CUDA_TRY(launch_nonempty_list(ss.offsets, t->nblocks, ss.list, ss.count, t->ne_scratch, t->stream,
                                               &t->launches));
    return TRK_OK;
}

static int batched_launch(tracker* t, const BatchSet* d_desc, int nsets)
{
    ProfScope ps(t, PROF_STEP);
    CUDA_TRY(cudaMemsetAsync(t->d_ctr, 0, (size_t)nsets * sizeof(int), t->stream));
    // tensor-copy halos for the halo-staged sets of a float32 field, one box per kernel width
    const void* maps[3] = {nullptr, nullptr, nullptr};
    const bool tma = t->halo_copy == TRK_HALO_TMA || (t->halo_copy == TRK_HALO_AUTO && t->auto_tma);
    if (tma && t->storage == TRK_F32) {
        bool ok = true;
        for (int i = 0; i < 3; ++i) {
            ok = ok && encode_field_map(t, 4 + 2 * i, 0, &t->batch_map[i]);
            maps[i] = &t->batch_map[i];
        }
        if (!ok) maps[0] = maps[1] = maps[2] = nullptr;
    }
    CUDA_TRY(launch_batched(t->storage, d_desc, nsets, t->d_ctr, t->nsm, maps[0] ? maps : nullptr, t->stream));
    t->launches += 1;
    return TRK_OK;
}

int tracker_advance_batched(tracker* t, int nsets, const trk_set* sets, double dt, int steps, int history_valid)
{
    history_valid = history_valid ? 1 : 0;   // AB2: one history entry, valid or not
    if (!t) return fail(TRK_EINVAL, "tracker is NULL");
    if (int rc_dev = check_device(t)) return rc_dev;
    if (nsets < 0 || (nsets > 0 && !sets)) return fail(TRK_EINVAL, "bad set list");
    if (!t->field) return fail(TRK_ENOFIELD, "no field set");
    if (t->C != 3) return fail(TRK_EINVAL, "batched advection needs a 3-component field (C=%d)", t->C);
    if (t->storage != TRK_F32 && t->storage != TRK_BF16X2)
        return fail(TRK_EINVAL, "batched advection runs on float32 or split-bf16 field storage");
    if (!std::isfinite(dt)) return fail(TRK_EINVAL, "dt must be finite");
    if (steps < 0) return fail(TRK_EINVAL, "steps=%d < 0", steps);
    int rc = check_block_kernel_shape(t);
    if (rc) return rc;
    // the direct items of the sets read the node-major copy of the field
    if (nsets > 0 && steps > 0 && (rc = ensure_node_major(t))) return rc;
    std::vector<int> tabs(nsets);
    int64_t npmax = 0;
    for (int s = 0; s < nsets; ++s) {
        const trk_set& S = sets[s];
        if ((rc = check_np(S.np))) return rc;
        if (S.np > 0 && (!S.pos || !S.rhs)) return fail(TRK_EINVAL, "set %d: pos and rhs must not be NULL", s);
        if (S.I != 4 && S.I != 6 && S.I != 8) return fail(TRK_EINVAL, "set %d: I=%d unsupported", s, S.I);
        if (S.family != TRK_LAGRANGE && S.family != TRK_SPLINE) return fail(TRK_EINVAL, "set %d: bad family", s);
        if (S.family == TRK_SPLINE && (S.m < 0 || S.m > S.I / 2)) return fail(TRK_EINVAL, "set %d: bad m=%d", s, S.m);
        if (S.deriv != 0 && S.deriv != 1) return fail(TRK_EINVAL, "set %d: deriv must be 0 or 1", s);
        tabs[s] = find_table(S.family, S.I, S.family == TRK_LAGRANGE ? 0 : S.m);
        if (tabs[s] < 0) return fail(TRK_EINVAL, "set %d: no coefficient table", s);
        npmax = std::max(npmax, S.np);
    }
    if (nsets == 0 || steps == 0 || npmax == 0) return TRK_OK;
    if ((int)t->sets.size() < nsets) t->sets.resize(nsets);
    for (int s = 0; s < nsets; ++s)
        if ((rc = ensure_set(t, t->sets[s], std::max<int64_t>(sets[s].np, 1)))) return rc;
    if (t->ne_cap < t->nblocks) {
        dev_free(t->ne_scratch);
        t->ne_scratch = nullptr;
        t->gen += 1;
        if (dev_alloc(&t->ne_scratch, nonempty_scratch_bytes(t->nblocks)) != cudaSuccess) {
            cudaGetLastError();
            return fail(TRK_ENOMEM, "cannot allocate the block-list scratch");
        }
        t->ne_cap = t->nblocks;
    }
    if (t->desc_cap < nsets) {
        dev_free(t->d_desc);
        dev_free(t->d_ctr);
        t->d_desc = nullptr;
        t->d_ctr = nullptr;
        t->gen += 1;
        if (dev_alloc(&t->d_desc, (size_t)3 * nsets * sizeof(BatchSet)) != cudaSuccess ||
            dev_alloc(&t->d_ctr, (size_t)nsets * sizeof(int)) != cudaSuccess) {
            cudaGetLastError();
            return fail(TRK_ENOMEM, "cannot allocate the set descriptors");
        }
        t->desc_cap = nsets;
    }
    // host-side descriptors: [0] first step, [1] parity 0 -> 1, [2] parity 1 -> 0
    std::vector<BatchSet> h(3 * (size_t)nsets);
    const BlockArgs base = base_args(t);
    std::vector<int> direct(nsets, 0);
    for (int s = 0; s < nsets; ++s) {
        const trk_set& S = sets[s];
        SetState& ss = t->sets[s];
        BlockArgs a = base;
        for (int i = 0; i < TRK_TAB_MAX_I; ++i)
            for (int d = 0; d < TRK_TAB_MAX_DEG; ++d) {
                a.cd.c[i][d] = kCoef[tabs[s]][i][d];
                a.cd.d[i][d] = kDCoef[tabs[s]][i][d];
                a.cf.c[i][d] = (float)kCoef[tabs[s]][i][d];
                a.cf.d[i][d] = (float)kDCoef[tabs[s]][i][d];
            }
        a.np = S.np;
        a.perm = ss.perm;
        a.offsets = ss.offsets;
        a.dt = dt;
        a.key_out = ss.keys;
        a.counts = ss.counts;
        a.out = S.out;
        for (int v = 0; v < 3; ++v) {
            BatchSet& B = h[(size_t)v * nsets + s];
            B.a = a;
            const int cur = v == 2 ? 1 : 0;
            if (v == 0) {
                B.a.pos_in = S.pos;
                B.a.id_in = nullptr;
                B.a.rhs_in = S.rhs;
                B.a.history_valid = history_valid;
            } else {
                B.a.pos_in = ss.pos_s[cur];
                B.a.id_in = ss.id_s[cur];
                B.a.rhs_in = ss.rhs_s[cur];
                B.a.history_valid = 1;
            }
            B.a.pos_out = ss.pos_s[cur ^ 1];
            B.a.id_out = ss.id_s[cur ^ 1];
            B.a.rhs_out = ss.rhs_s[cur ^ 1];
            B.list = ss.list;
            B.count = ss.count;
            B.n_items = (int)((S.np + PB_HOST - 1) / PB_HOST);
            B.I = S.I;
            B.deg_hi = kTables[tabs[s]].deg > S.I - 1;
            B.deriv = S.deriv;
            B.direct = 0;
        }
    }
    // per-set path: halo-staged blocks or direct gathers, chosen by timing both once
    for (int s = 0; s < nsets; ++s) {
        const trk_set& S = sets[s];
        if (S.np == 0) {   // empty set: no items (the direct path reads n_items = 0)
            direct[s] = 1;
            for (int v = 0; v < 3; ++v) h[(size_t)v * nsets + s].direct = 1;
            continue;
        }
        const uint64_t sig = mix(mix(mix(mix(mix(0, (uint64_t)S.np), (uint64_t)S.I), (uint64_t)S.deriv),
                                     (uint64_t)tabs[s]), (uint64_t)t->N);
        int choice = -1;
        for (auto& kv : t->tune_cache)
            if (kv.first == sig) choice = kv.second;
        if (choice < 0) {
            SetState& ss = t->sets[s];
            const size_t vb = (size_t)S.np * 24;
            CUDA_TRY(cudaMemcpyAsync(ss.pos_s[1], S.pos, vb, cudaMemcpyDeviceToDevice, t->stream));
            if ((rc = keys_set(t, ss, S.np, ss.pos_s[1]))) return rc;
            if ((rc = bin_set(t, ss, S.np, false))) return rc;
            BatchSet probe = h[(size_t)nsets + s];           // parity-0 layout: reads pos_s[0] ...
            probe.a.pos_in = ss.pos_s[1];                     // ... so point it at the copy
            probe.a.id_in = nullptr;
            probe.a.rhs_in = nullptr;
            probe.a.history_valid = 0;
            probe.a.pos_out = ss.pos_s[0];
            probe.a.id_out = ss.id_s[0];
            probe.a.rhs_out = ss.rhs_s[0];
            probe.a.out = nullptr;
            float best[2] = {0, 0};
            cudaEvent_t e0, e1;
            CUDA_TRY(cudaEventCreate(&e0));
            CUDA_TRY(cudaEventCreate(&e1));
            for (int variant = 0; variant < 2; ++variant) {
                probe.direct = variant;
                CUDA_TRY(cudaMemcpyAsync(t->d_desc, &probe, sizeof(BatchSet), cudaMemcpyHostToDevice, t->stream));
                for (int rep = 0; rep < 2; ++rep) {
                    CUDA_TRY(cudaEventRecord(e0, t->stream));
                    if ((rc = batched_launch(t, t->d_desc, 1))) return rc;
                    CUDA_TRY(cudaEventRecord(e1, t->stream));
                    CUDA_TRY(cudaEventSynchronize(e1));
                    CUDA_TRY(cudaEventElapsedTime(&best[variant], e0, e1));
                }
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            choice = best[1] < best[0] ? 1 : 0;
            remember(t->tune_cache, sig, choice);
        }
        direct[s] = choice;
        for (int v = 0; v < 3; ++v) h[(size_t)v * nsets + s].direct = choice;
    }
    CUDA_TRY(cudaMemcpyAsync(t->d_desc, h.data(), h.size() * sizeof(BatchSet), cudaMemcpyHostToDevice, t->stream));
    CUDA_TRY(cudaStreamSynchronize(t->stream));   // h may be released after this
    auto step = [&](int v) -> int {
        for (int s = 0; s < nsets; ++s) {
            if (sets[s].np == 0) continue;
            if (v == 0) {
                int r = keys_set(t, t->sets[s], sets[s].np, sets[s].pos);
                if (r) return r;
            }
            int r = bin_set(t, t->sets[s], sets[s].np, direct[s]);
            if (r) return r;
        }
        return batched_launch(t, t->d_desc + (size_t)v * nsets, nsets);
    };
    if ((rc = step(0))) return rc;
    int cur = 1;
    int rest = steps - 1;
    if (!t->prof && rest >= 2) {
        uint64_t key = mix(mix(mix(0, t->gen), (uint64_t)nsets), dbits(dt));
        for (int s = 0; s < nsets; ++s)
            key = mix(mix(mix(mix(mix(key, (uint64_t)sets[s].np), (uint64_t)sets[s].I), (uint64_t)tabs[s]),
                          (uint64_t)direct[s] * 2 + sets[s].deriv),
                      (uint64_t)(uintptr_t)sets[s].out);
        // the state is in buffer 1 after the first step: parity 1 -> 0, then 0 -> 1
        rc = replay_graph(t, t->batch_graph, key, rest / 2, [&]() {
            int r = step(2);
            return r ? r : step(1);
        });
        if (rc) return rc;
        rest -= 2 * (rest / 2);
    }
    for (; rest > 0; --rest) {
        if ((rc = step(cur == 1 ? 2 : 1))) return rc;
        cur ^= 1;
    }
    ProfScope ps(t, PROF_OTHER);
    for (int s = 0; s < nsets; ++s) {
        if (sets[s].np == 0) continue;
        SetState& ss = t->sets[s];
        CUDA_TRY(launch_unpermute_pos(sets[s].np, ss.pos_s[cur], ss.id_s[cur], sets[s].pos, t->stream));
        CUDA_TRY(launch_unpermute_rhs(sets[s].np, ss.rhs_s[cur], ss.id_s[cur], sets[s].rhs, 3, t->stream));
        t->launches += 2;
    }
    return TRK_OK;
}

int tracker_adjoint(tracker* t, int64_t np, const double* pos0, const double* lambdaT, double dt, int steps,
                    int ckpt_every, double* grad_pos0, double* grad_field)
{
    if (!t) return fail(TRK_EINVAL, "tracker is NULL");
    if (int rc_dev = check_device(t)) return rc_dev;
    int rc = check_np(np);
    if (rc) return rc;
    if (!t->field) return fail(TRK_ENOFIELD, "no field set");
    if (t->C != 3) return fail(TRK_EINVAL, "the adjoint needs a 3-component field (C=%d)", t->C);
    if (!std::isfinite(dt)) return fail(TRK_EINVAL, "dt must be finite");
    if (steps < 0) return fail(TRK_EINVAL, "steps=%d < 0", steps);
    if (ckpt_every < 1) return fail(TRK_EINVAL, "ckpt_every=%d < 1", ckpt_every);
    if (np > 0 && (!pos0 || !lambdaT || !grad_pos0)) return fail(TRK_EINVAL, "pos0, lambdaT and grad_pos0 must not be NULL");
    // sparse sets: the direct adjoint (no halos, stencils from global memory,
    // float64 atomic adds straight into grad_field)
    const bool adj_direct = t->step_kernel == TRK_STEP_DIRECT ||
                            (t->step_kernel == TRK_STEP_AUTO &&
                             (double)np < kAdjDirectDensity * (double)t->N * t->N * t->N);
    if (!adj_direct && (rc = check_block_kernel_shape(t))) return rc;
    if (np == 0) return TRK_OK;
    const size_t vec = (size_t)3 * np;                 // doubles per position / lambda array
    if (steps == 0) {
        CUDA_TRY(cudaMemcpyAsync(grad_pos0, lambdaT, vec * 8, cudaMemcpyDeviceToDevice, t->stream));
        return TRK_OK;
    }
    if ((rc = ensure_sort(t, np))) return rc;
    if ((rc = ensure_state(t, np))) return rc;
    const int K = std::min(ckpt_every, steps);
    const int nseg = (steps + K - 1) / K;
    // layout: nseg checkpoints | K segment states | 2 lambdas
    const size_t need = (size_t)(nseg + K + 2) * vec * 8;
    if (need > t->adj_bytes) {
        dev_free(t->adj_buf);
        t->adj_buf = nullptr;
        t->adj_bytes = 0;
        if (dev_alloc(&t->adj_buf, need) != cudaSuccess) {
            cudaGetLastError();
            return fail(TRK_ENOMEM, "cannot allocate adjoint checkpoints (%zu bytes)", need);
        }
        t->adj_bytes = need;
    }
    // field gradient: per-block partial sums (atomic adds into zeroed slabs) and a
    // gather per node in a fixed block order, while the scratch stays below 8 GB
    // (else float64 atomics per halo node)
    void* gscratch = nullptr;
    if (grad_field && !adj_direct) {
        const int H = adj_halo(t->I);
        const size_t sb = (size_t)t->nblocks * 3 * H * H * H * (t->storage == TRK_F64 ? 8 : 4);
        size_t cap = (size_t)8 << 30;
        if (const char* env = getenv("TRK_ADJ_SCRATCH_BYTES")) cap = (size_t)strtoull(env, nullptr, 10);
        if (sb <= cap) {
            if (sb > t->adj_scratch_bytes) {
                dev_free(t->adj_scratch);
                t->adj_scratch = nullptr;
                t->adj_scratch_bytes = 0;
                if (dev_alloc(&t->adj_scratch, sb) == cudaSuccess) t->adj_scratch_bytes = sb;
                else cudaGetLastError();
            }
            gscratch = t->adj_scratch;
            // every gather leaves the slabs it read zero; clearing them here as well
            // keeps a call that failed half-way from leaking into the next one
            if (gscratch) CUDA_TRY(cudaMemsetAsync(gscratch, 0, sb, t->stream));
        }
    }
    double* ckpt = t->adj_buf;
    double* seg = ckpt + (size_t)nseg * vec;
    double* lam[2] = {seg + (size_t)K * vec, seg + (size_t)(K + 1) * vec};
    // forward sweep keeping a checkpoint every K steps
    CUDA_TRY(cudaMemcpyAsync(ckpt, pos0, vec * 8, cudaMemcpyDeviceToDevice, t->stream));
    for (int sg = 1; sg < nseg; ++sg) {
        double* dst = ckpt + (size_t)sg * vec;
        CUDA_TRY(cudaMemcpyAsync(dst, ckpt + (size_t)(sg - 1) * vec, vec * 8, cudaMemcpyDeviceToDevice, t->stream));
        if ((rc = tracker_advance(t, np, dst, nullptr, dt, K, TRK_RK2, 0))) return rc;
    }
    // backward sweep: recompute each segment from its checkpoint, then step back through it
    CUDA_TRY(cudaMemcpyAsync(lam[0], lambdaT, vec * 8, cudaMemcpyDeviceToDevice, t->stream));
    int cur = 0;
    for (int sg = nseg - 1; sg >= 0; --sg) {
        const int s0 = sg * K, s1 = std::min(steps, s0 + K);
        CUDA_TRY(cudaMemcpyAsync(seg, ckpt + (size_t)sg * vec, vec * 8, cudaMemcpyDeviceToDevice, t->stream));
        for (int i = 1; i < s1 - s0; ++i) {
            double* dst = seg + (size_t)i * vec;
            CUDA_TRY(cudaMemcpyAsync(dst, seg + (size_t)(i - 1) * vec, vec * 8, cudaMemcpyDeviceToDevice, t->stream));
            if ((rc = tracker_advance(t, np, dst, nullptr, dt, 1, TRK_RK2, 0))) return rc;
        }
        for (int i = s1 - s0 - 1; i >= 0; --i) {
            const double* X = seg + (size_t)i * vec;
            if ((rc = bin_counting(t, np, X))) return rc;
            AdjArgs a{};
            const BlockArgs b = base_args(t);
            a.g = b.g;
            a.f = b.f;
            a.cf = b.cf;
            a.cd = b.cd;
            a.np = np;
            a.offsets = adj_direct ? nullptr : t->offsets;   // null: the direct mode
            a.perm = t->perm;
            a.pos = X;
            a.lam_in = lam[cur];
            a.lam_out = lam[cur ^ 1];
            a.gfield = grad_field;
            a.gscratch = grad_field ? gscratch : nullptr;
            a.dt = dt;
            a.flags = t->d_flags;
            CUDA_TRY(launch_adjoint(t, a));
            if (a.gscratch) {
                ProfScope ps(t, PROF_OTHER);   // the node gather of the field gradient
                t->launches += 1;
                CUDA_TRY(launch_adjoint_gather(t->I, a, t->stream));
            }
            cur ^= 1;
        }
    }
    CUDA_TRY(cudaMemcpyAsync(grad_pos0, lam[cur], vec * 8, cudaMemcpyDeviceToDevice, t->stream));
    return TRK_OK;
}

}  // extern "C"
