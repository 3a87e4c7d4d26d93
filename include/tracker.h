/*
 * tracker.h -- C ABI of the GB300 tracer-advection library.
 *
 * Implements the particle-tracking hot path of Lalescu, Bramas, Rampp and
 * Wilczek, "An Efficient Particle Tracking Algorithm for Large-Scale Parallel
 * Pseudo-Spectral Simulations of Turbulence" (arXiv:2107.01104): tracers
 * dX/dt = u(X) (Eq. tracers) in a frozen periodic field on [0, L)^3 sampled on
 * an N^3 grid (Sec. 2.1), interpolated with separable kernels of I nodes per
 * axis (Sec. 2.2, Eq. triple_sum), particles kept grouped by cell block with
 * an offset array (Sec. 3.3.1), advanced by RK2 (Heun) or Adams-Bashforth
 * (orders 2-4).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - All array pointers are DEVICE pointers unless a parameter says
 *   otherwise.  The caller owns them; the library never frees them.
 * - positions  pos[3][np]     float64, SoA (all x1, then all x2, then x3),
 *                             unwrapped (any finite value; reduced mod L
 *                             inside the cell split, Sec. 2.2 step 1).
 * - fields     f[C][N][N][N]  component-major, x3 slowest, x1 fastest.
 * - outputs    out[C][np]     in the caller's particle order.
 * - Calls are asynchronous on the tracker's CUDA stream (given at create or
 *   by tracker_set_stream).  Argument errors are reported synchronously by
 *   the return value.  Device-side conditions (non-finite positions, a
 *   particle moving more than one cell in one RK2 stage) set a device flag
 *   that tracker_sync() reads back and reports.
 * - Every function returns TRK_OK (0) or a negative trk_status.  After a
 *   failure tracker_last_error() returns a message (thread-local).
 * - np is limited to 2^31 - 1 particles per call; N must be a power of two
 *   with 16 <= N <= 1024; I in {4, 6, 8}.
 * - There is no CPU fallback: every computation runs in this library's
 *   CUDA kernels (sm_103a).  A missing GPU is TRK_ECUDA.
 * - A tracker belongs to the CUDA device that was current when it was
 *   created, where all its buffers live.  Every later call that launches
 *   work or allocates must be made with that device current; otherwise it
 *   returns TRK_EINVAL without touching the GPU.  tracker_destroy makes the
 *   tracker's device current by itself and restores the caller's device.
 */
#ifndef TRACKER_H
#define TRACKER_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tracker tracker;

typedef enum {
    TRK_OK = 0,
    TRK_EINVAL = -1,      /* bad argument (message says which) */
    TRK_ENOMEM = -2,      /* device allocation failed */
    TRK_ECUDA = -3,       /* CUDA runtime error (message has the CUDA string) */
    TRK_ENONFINITE = -4,  /* a position was NaN/Inf or beyond 2^51 cells (device flag) */
    TRK_ENOFIELD = -6,    /* no field set yet */
    TRK_ECFL = -7,        /* a particle moved more than one cell in one stage (device flag; result still exact) */
    TRK_EIO = -8          /* a state file could not be written or read, or failed its checks */
} trk_status;

typedef enum { TRK_LAGRANGE = 0, TRK_SPLINE = 1 } trk_family;

/* Field storage inside the tracker.  Weights and accumulation are float32
 * for F32 and BF16X2, float64 for F64.  BF16X2 keeps hi = RN_bf16(x) and
 * lo = RN_bf16(x - hi) as two planes (4 bytes per value, about 16
 * significant bits). */
typedef enum { TRK_F64 = 0, TRK_F32 = 1, TRK_BF16X2 = 2 } trk_storage;

typedef enum { TRK_RK2 = 0, TRK_AB2 = 1, TRK_AB3 = 2, TRK_AB4 = 3 } trk_scheme;

typedef enum { TRK_DTYPE_F64 = 0, TRK_DTYPE_F32 = 1 } trk_dtype;

typedef enum { TRK_STEP_AUTO = 0, TRK_STEP_BLOCK = 1, TRK_STEP_COLUMN = 2, TRK_STEP_DIRECT = 3 } trk_step_kernel;

typedef enum { TRK_HALO_AUTO = 0, TRK_HALO_ASYNC = 1, TRK_HALO_TMA = 2 } trk_halo_copy;

/* ---------------------------------------------------------------------- */
/* Lifetime                                                                */
/* ---------------------------------------------------------------------- */

/* Create a tracker for an N^3 periodic grid on [0, L)^3 (the paper uses
 * L = 2 pi, Sec. 2.1) with interpolation kernel (family, I, m):
 *   TRK_LAGRANGE: I-node Lagrange polynomials (Sec. 2.2), m ignored;
 *   TRK_SPLINE:   the spline family cited in Sec. 2.2: degree 2m+1 on each
 *                 cell, C^m across cells, node derivatives from centred
 *                 (I-1)-point differences; 0 <= m <= I/2.
 * storage selects the field storage (trk_storage).  stream is a
 * cudaStream_t (NULL = legacy default stream).  *out receives the handle.
 * Errors: TRK_EINVAL (unsupported N, I, m, storage, L <= 0), TRK_ECUDA,
 * TRK_ENOMEM. */
int tracker_create(tracker** out, int N, double L, int family, int I, int m, int storage, void* stream);

/* Release every device buffer the tracker owns.  NULL is accepted. */
int tracker_destroy(tracker* t);

/* Message for the last failing call on this thread ("" if none). */
const char* tracker_last_error(void);

/* Replace the stream later calls are issued on. */
int tracker_set_stream(tracker* t, void* stream);

/* Wait for the tracker's stream, then read and clear the device flags:
 * returns TRK_ENONFINITE or TRK_ECFL if a kernel raised one since the
 * last sync, else TRK_OK (or TRK_ECUDA). */
int tracker_sync(tracker* t);

/* ---------------------------------------------------------------------- */
/* Field                                                                   */
/* ---------------------------------------------------------------------- */

/* Copy a field f[C][N][N][N] (1 <= C <= 16), float64 (src_dtype
 * TRK_DTYPE_F64) or float32 (TRK_DTYPE_F32), into the tracker's storage,
 * converting to its trk_storage.  src_on_host = 1 reads a host pointer
 * (copied through the stream), 0 a device pointer.  The source may be freed
 * once the call has completed on the stream.  The field is frozen between
 * calls (Sec. 2.2 interpolates a given field).  Errors: TRK_EINVAL,
 * TRK_ENOMEM, TRK_ECUDA. */
int tracker_set_field(tracker* t, const void* src, int C, int src_dtype, int src_on_host);

/* ---------------------------------------------------------------------- */
/* Binning (Sec. 3.3.1, "Ordering the particles locally")                  */
/* ---------------------------------------------------------------------- */

/* Block shape used for grouping: bx x by x bz cells, each a power of two
 * dividing N (default 8 x 8 x 8).  bx = by = N, bz = 1 reproduces the
 * paper's x3 slices. */
int tracker_set_block(tracker* t, int bx, int by, int bz);

/* Number of blocks (N/bx)(N/by)(N/bz) for the current block shape. */
int64_t tracker_num_blocks(const tracker* t);

/* Stable counting sort of np particles by block key
 *   key = ((c3/bz) * (N/by) + c2/by) * (N/bx) + c1/bx,
 * where c is the cell of Sec. 2.2 step 2, split from X as
 *   g = X * fl(N/L), c0 = floor(g), t = g - c0, c = c0 mod N
 * (IEEE float64, no fused multiply-add; bit-exact and reproducible).
 * Outputs (device, int32): keys[np] in the incoming order (may be NULL),
 * perm[np] (perm[j] = incoming index of the j-th particle in sorted
 * order, ties kept in incoming order), offsets[nblocks+1] (offsets[b] =
 * first sorted position of block b, offsets[nblocks] = np: the paper's
 * offset array).  pos and the outputs must be device memory of the
 * tracker's device (checked, TRK_EINVAL otherwise); the caller sizes them
 * (np, np, nblocks + 1 entries).  Errors: TRK_EINVAL, TRK_ENOMEM;
 * non-finite positions raise the TRK_ENONFINITE device flag. */
int tracker_bin(tracker* t, int64_t np, const double* pos, int32_t* keys, int32_t* perm, int32_t* offsets);

/* ---------------------------------------------------------------------- */
/* Interpolation (Sec. 2.2 step 4, Eq. triple_sum; separable, Sec. 3.3)   */
/* ---------------------------------------------------------------------- */

/* out[k][p] = u_k(X_p) for every field component k < C (deriv = 0), or
 * out[(3k + j)][p] = d u_k / d X_j at X_p (deriv = 1; derivative kernels
 * beta' on axis j, times N/L).  out_dtype is TRK_DTYPE_F32 or
 * TRK_DTYPE_F64 (any storage).  Particles are binned internally (a counting
 * sort by block: block counts, one scan, a scatter of the permutation; the
 * order inside a block does not change any result); results are written in
 * the caller's order.  Errors: TRK_EINVAL, TRK_ENOFIELD, TRK_ENOMEM. */
int tracker_interpolate(tracker* t, int64_t np, const double* pos, void* out, int out_dtype, int deriv);

/* ---------------------------------------------------------------------- */
/* Advection (Eq. tracers)                                                 */
/* ---------------------------------------------------------------------- */

/* Advance np tracers by `steps` steps of size dt in the tracker's
 * 3-component field (C must be 3).
 *   TRK_RK2 (Heun): k1 = u(X), X* = X + dt k1, k2 = u(X*),
 *                   X' = X + dt/2 (k1 + k2).
 *   TRK_AB2, TRK_AB3, TRK_AB4 (Adams-Bashforth of order k = 2, 3, 4, the
 *            paper's multi-step scheme, Sec. 2.2 and the rhs array of
 *            Sec. 3.3.1):
 *                   X' = X + dt sum_{j<q} beta^q_j u_{n-j},
 *                   q = min(k, 1 + number of valid history entries), with
 *                   the textbook weights (q = 1 forward Euler; 2: 3/2,
 *                   -1/2; 3: 23/12, -16/12, 5/12; 4: 55/24, -59/24, 37/24,
 *                   -9/24), so a run without history starts at lower
 *                   orders.  rhs[k-1][3][np] (float32, caller order) holds
 *                   u_{n-1}, u_{n-2}, ... (newest first); history_valid
 *                   (0 .. k-1) says how many of them are valid on entry; on
 *                   return rhs holds the k-1 newest u (entries not yet
 *                   filled are zero) and min(history_valid + steps, k-1)
 *                   of them are valid.  rhs may be NULL for RK2.
 * pos[3][np] is read and overwritten in the caller's order.  Particles are
 * re-binned after every step (the update/re-sort of Sec. 3.3.1); the steps
 * are replayed from a captured CUDA graph (Adams-Bashforth runs step by step
 * until its history is full).  A particle that moves more
 * than one cell in one stage is still computed exactly (through a slower
 * path) and raises TRK_ECFL at the next tracker_sync.
 * Errors: TRK_EINVAL, TRK_ENOFIELD, TRK_ENOMEM. */
int tracker_advance(tracker* t, int64_t np, double* pos, float* rhs, double dt, int steps, int scheme,
                    int history_valid);

/* Step kernel used by tracker_advance and tracker_interpolate (trk_step_kernel):
 *   TRK_STEP_COLUMN: a persistent kernel that walks column segments of cell
 *     blocks along x3 (the x3 slabs of Sec. 3.3.1): the field halo stays in a
 *     ring of x3 planes, so a slab brings in only the planes it does not
 *     share with the previous one, and the next slab's planes and particles
 *     are copied in while the current slab is interpolated.  Its re-binning
 *     is a counting sort: the update phase counts the new block keys, a scan
 *     gives the offsets, and a scatter moves the particle state into its
 *     blocks (the order inside a block is not reproducible; no result
 *     depends on it).  Available for TRK_F32 storage with I = 4 or 6 in the
 *     8 x 8 x 8 block shape.
 *   TRK_STEP_BLOCK: one thread block per cell block, reading the state
 *     through the sort permutation (all storages and kernels).
 *   TRK_STEP_DIRECT: for sparse particle sets (the paper's production runs
 *     carry ~1e-3 tracers per grid cell, Sec. 4): particles sorted by block
 *     as for BLOCK, 64 to 256 of them per thread block, each stencil gathered
 *     from the field in global memory, so no field sweep and no halo per
 *     cell block (all storages and kernels, any block shape; float32 fields
 *     and split-bf16 fields whose component count is a multiple of three are
 *     read from a node-major copy the tracker keeps, made on first use: 16
 *     bytes per node for three float32 components, one 16-byte record per
 *     node and chunk of three split-bf16 components (a split-bf16 field
 *     whose copy cannot be allocated is read from the field itself); where
 *     a three-component copy is at most four times the L2 size (or the byte
 *     count in the environment variable TRK_NM_TEXTURE_BYTES, 0 for never)
 *     it is read through a texture object: the same bits, on the texture
 *     data path instead of the load/store one, which the gathers of a copy
 *     that mostly hits in L2 otherwise saturate).  The stage-2
 *     point of RK2 is gathered wherever it lies; TRK_ECFL is raised when it
 *     is more than one cell away.
 *   TRK_STEP_AUTO (default): the tuner's choice (see tracker_set_tuning):
 *     on the first call of a workload with enough steps, every candidate
 *     kernel and launch shape is timed on real steps of the call and the
 *     fastest kept; otherwise DIRECT below 0.05 particles per grid cell
 *     (np < 0.05 N^3), else COLUMN where available; without a column kernel
 *     DIRECT below 0.25 per cell, else BLOCK (measured crossovers).
 *     tracker_interpolate uses DIRECT or BLOCK; between 0.01 and 0.25 per
 *     cell its first call per (np, C, deriv, out_dtype) runs the block kernel
 *     with each halo copy and the direct kernel (they write the same values)
 *     and keeps the fastest: which one wins depends on C (the direct kernel
 *     gathers every component of a node at once for C = 3).
 * All kernels perform the same floating-point operations in the same
 * order, so their results are bit-identical.  TRK_STEP_COLUMN on a tracker
 * without a column kernel is TRK_EINVAL.  Errors: TRK_EINVAL. */
int tracker_set_step_kernel(tracker* t, int kind);

/* The trk_step_kernel (COLUMN, BLOCK or DIRECT) that tracker_advance starts
 * with for np particles under the current setting, before any timing;
 * negative status on error. */
int tracker_step_kernel_for(const tracker* t, int64_t np);

/* The trk_step_kernel the latest tracker_advance ran its remaining steps
 * with, or the latest tracker_interpolate used (after any timing);
 * TRK_STEP_AUTO before the first call; negative status on error. */
int tracker_last_step_kernel(const tracker* t);

/* How the block kernel (TRK_STEP_BLOCK, and the block side of interpolation)
 * stages each cell block's field halo in shared memory (the slab ghost
 * layers of Sec. 3.3.1, per cell block):
 *   TRK_HALO_ASYNC: cp.async copies of single elements (float32, float64) or
 *     16-byte vector loads through registers (split bf16);
 *   TRK_HALO_TMA: one tensor copy (cp.async.bulk.tensor) per chunk of three
 *     components, issued by one thread and awaited on an mbarrier, into a
 *     box padded so that the stencil loads meet few shared-memory bank
 *     conflicts (float32 and float64 storage with at least three
 *     components; elsewhere the cp.async staging is used);
 *   TRK_HALO_AUTO (default): TRK_HALO_TMA where the field has a tensor map
 *     (faster where few particles share a halo: 0.338 vs 0.526 ms per RK2
 *     step at 256^3, I = 6, 1/64 particle per cell), unless the tuner (the
 *     first timed tracker_advance or tracker_interpolate call of a workload)
 *     measured the cp.async halo faster (e.g. 2.93 vs 3.20 ms at 1/2 per
 *     cell, where the smem reads dominate); else TRK_HALO_ASYNC.
 * Both give bit-identical results.  A tensor copy that does not complete
 * within its wait limit skips its block and makes tracker_sync return
 * TRK_ECUDA.  Errors: TRK_EINVAL. */
int tracker_set_halo_copy(tracker* t, int kind);

/* Launch shape of the time-step path.  step_kernel: TRK_STEP_COLUMN, _BLOCK
 * or _DIRECT; direct_block: edge of the cubic cell blocks the direct kernel's
 * particles are binned by (a power of two <= N; with the default 8^3 block
 * shape; it sets how compact each thread block's particles are);
 * column_segment: x3 slabs per work item of the column kernel (a power of
 * two <= 64, at most N/8); halo_copy: the block kernel's TRK_HALO_ASYNC or
 * TRK_HALO_TMA; direct_particles: particles per thread block of the direct
 * kernel (64, 128 or 256; 0 in tracker_set_tuning means 256; untimed calls
 * use the largest that gives three thread blocks per SM).  source
 * (tracker_get_tuning only): how they were chosen. */
typedef enum { TRK_TUNE_DEFAULT = 0, TRK_TUNE_TIMED = 1, TRK_TUNE_CACHED = 2, TRK_TUNE_FIXED = 3 } trk_tune_source;
typedef struct {
    int step_kernel;
    int direct_block;
    int column_segment;
    int halo_copy;
    int direct_particles;
    int source;
} trk_tuning;

/* Autotuning (no counterpart in the paper).  With TRK_STEP_AUTO (the
 * default), the first tracker_advance call of a workload -- grid, kernel,
 * storage, SM count, density bucket (half octaves of particles per cell) and
 * scheme -- that has at least 2 x (candidates) + 2 steps and at least 32768
 * particles times every candidate launch shape on 2 of its own steps (CUDA
 * events; the host waits once; skipped while the stream is being captured)
 * and keeps the fastest for the rest of the call and for later calls
 * (TRK_TUNE_TIMED, then TRK_TUNE_CACHED).  Candidates: from 0.01 particles
 * per cell on, the column kernel with segments 8 and 16; the block kernel
 * with tensor-copy and with cp.async halos from 0.1 per cell on (from 0.01
 * without a column kernel); the direct kernel with block edges 8 and 16 and
 * 256 or 128 particles per thread block, up to one particle per cell.
 * Other calls use the density rule of tracker_set_step_kernel with the
 * default shape, the direct kernel with the largest of 256, 128, 64
 * particles per thread block that gives three per SM (TRK_TUNE_DEFAULT).  Every
 * candidate gives bit-identical steps.  When the environment variable
 * TRK_TUNE_CACHE names a file, decisions are appended to it (one line per
 * workload) and trackers created later read it.
 * tracker_set_tuning fixes a launch shape (TRK_TUNE_FIXED; no timing); NULL
 * returns to automatic tuning.  Errors: TRK_EINVAL. */
int tracker_set_tuning(tracker* t, const trk_tuning* tuning);

/* The launch shape the latest tracker_advance ran its remaining steps with,
 * and how it was chosen. */
int tracker_get_tuning(const tracker* t, trk_tuning* out);

/* The halo copy (TRK_HALO_ASYNC or TRK_HALO_TMA) the block kernel uses now
 * for interpolation and AB steps (mode 0) or RK2 steps (mode 1). */
int tracker_halo_copy(const tracker* t, int mode);

/* 1 if the direct kernel reads the node-major copy of the current field
 * through a texture object, 0 if by plain loads or if no copy has been made
 * yet (the copy is made by the first direct launch after tracker_set_field);
 * negative status on error. */
int tracker_field_texture(const tracker* t);

/* ---------------------------------------------------------------------- */
/* Batched advection: many particle sets, one persistent launch per step  */
/* ---------------------------------------------------------------------- */

typedef struct {
    int64_t np;          /* particles in this set */
    double* pos;         /* [3][np] float64, device, in/out */
    float* rhs;          /* [3][np] float32 AB2 history, device, in/out */
    float* out;          /* [nout][np] float32 per-step outputs, device, or NULL:
                            nout = 3 (u at the step's start, deriv = 0) or
                            9 (du_k/dX_j as 3k+j, deriv = 1) */
    int family, I, m;    /* kernel of this set */
    int deriv;           /* 0: outputs u; 1: outputs the gradient as well */
} trk_set;

/* Advance every set by `steps` AB2 steps (history_valid: 0 = no history,
 * any other value = the one AB2 entry is valid; applied to all sets) in the
 * tracker's 3-component
 * field.  Each step is one persistent kernel over a shared work list of
 * (set, block) items, so sets of very different sizes and kernels share
 * one launch; the step sequence is captured in a CUDA graph and replayed.
 * Errors: TRK_EINVAL, TRK_ENOFIELD, TRK_ENOMEM. */
int tracker_advance_batched(tracker* t, int nsets, const trk_set* sets, double dt, int steps,
                            int history_valid);

/* ---------------------------------------------------------------------- */
/* Tracer-set checkpoints (in-order particle output and restart, Sec. 3.4) */
/* ---------------------------------------------------------------------- */

/* What a state file holds besides the arrays.  N, L, family, I, m record the
 * writer's grid and kernel (a reader compares them with its own tracker);
 * scheme and history_valid describe the AB history (as in tracker_advance);
 * step, time and dt are the run's counters (an AB history is only valid for
 * the dt it was made with). */
typedef struct {
    int32_t N;
    double L;
    int32_t family, I, m;
    int64_t np;
    int32_t scheme;
    int32_t history_valid;
    int64_t step;
    double time;
    double dt;
} trk_state_info;

/* Write a tracer set to a binary file: a 96-byte header (magic, version, the
 * info fields, checksums of header and payload), then pos[3][np] float64 and,
 * for ABk, rhs[3(k-1)][np] float32, all in the caller's particle order (the
 * order tracker_advance returns).  Little-endian, no padding.  pos and rhs
 * are HOST pointers (copy device arrays first); rhs is ignored for RK2.  The
 * file is written under a temporary name and renamed into place, so a failed
 * write leaves an existing file intact.  Errors: TRK_EINVAL (bad fields or
 * NULL arrays), TRK_EIO (open/write/rename failed). */
int tracker_state_write(const char* path, const trk_state_info* info, const double* pos, const float* rhs);

/* Read only the header of a state file into *info (to size the buffers).
 * Errors: TRK_EINVAL, TRK_EIO (missing file, wrong magic or version,
 * header checksum mismatch, invalid fields). */
int tracker_state_read_info(const char* path, trk_state_info* info);

/* Read a state file into HOST buffers pos[3][np] and, for ABk,
 * rhs[3(k-1)][np]; np must equal the file's particle count.  *info receives
 * the header.  The payload checksum is verified after reading (the buffers
 * then hold the file's bytes even when TRK_EIO reports a mismatch).
 * Errors: TRK_EINVAL (np differs, NULL arrays), TRK_EIO (as above, a
 * truncated payload, trailing bytes, payload checksum mismatch). */
int tracker_state_read(const char* path, int64_t np, double* pos, float* rhs, trk_state_info* info);

/* ---------------------------------------------------------------------- */
/* Adjoint (no counterpart in the paper: gradient of a loss through RK2)   */
/* ---------------------------------------------------------------------- */

/* Discrete adjoint of `steps` RK2 steps from pos0 (not modified).  Given
 * lambdaT[3][np] = dLoss/dX_T (float64, caller order), writes
 * grad_pos0[3][np] = dLoss/dX_0 (float64) and, if grad_field is not NULL,
 * ADDS dLoss/dfield into grad_field[3][N][N][N] (float64).  The forward
 * trajectory is recomputed from checkpoints taken every ckpt_every steps.
 * Per step, backwards, with J = du/dX and W(X) the field-to-u(X) map:
 *   lambda* = dt/2 J(X*)^T lambda,  mu = dt/2 lambda + dt lambda*,
 *   grad_field += W(X)^T mu + W(X*)^T (dt/2 lambda),
 *   lambda <- lambda + lambda* + J(X)^T mu.
 * Two modes (same values up to rounding order of the field gradient):
 *   halo mode (TRK_STEP_AUTO at 1/8 tracer per grid cell or more, or
 *     TRK_STEP_BLOCK / TRK_STEP_COLUMN): one thread block per cell block
 *     with the field halo in shared memory; the field gradient is
 *     accumulated per cell block (atomic adds into the block's slab of
 *     scratch) and then summed per grid node over the blocks whose halo
 *     holds it, in a fixed block order.  The scratch holds
 *     nblocks * 3 * (I + 9)^3 values (float32, float64 for TRK_F64 storage;
 *     1.3 GB at N = 256, I = 6); when this exceeds the byte count in the
 *     environment variable TRK_ADJ_SCRATCH_BYTES (default 8 GiB) or cannot
 *     be allocated, each block accumulates in shared memory and adds its
 *     partial sums with float64 atomics instead.
 *   direct mode (TRK_STEP_AUTO below 1/8 tracer per cell, or
 *     TRK_STEP_DIRECT): no halos; 128 sorted particles per thread block,
 *     stencils gathered from the field in global memory, and each stencil
 *     node's contribution added to grad_field with a float64 atomic add.
 *     The position gradient is bit-identical to the halo mode's.
 * Errors: TRK_EINVAL, TRK_ENOFIELD, TRK_ENOMEM. */
int tracker_adjoint(tracker* t, int64_t np, const double* pos0, const double* lambdaT, double dt, int steps,
                    int ckpt_every, double* grad_pos0, double* grad_field);

/* Number of kernel launches this tracker has issued since creation
 * (graph replays count each kernel node).  For instrumentation. */
int64_t tracker_launch_count(const tracker* t);

/* Instrumentation.  tracker_profile(t, 1) clears and starts recording CUDA
 * events on the tracker's stream around each kernel class; 0 stops.  While
 * recording, tracker_advance launches its kernels directly instead of
 * replaying a CUDA graph.  tracker_profile_read waits for the stream and
 * returns the accumulated device time in milliseconds and the number of
 * timed launches per class:
 *   [0] interpolation / step kernels (the per-block gather-contract-update),
 *   [1] binning (block keys, radix-sort passes, offsets),
 *   [2] everything else (field conversion, scatter back to caller order).
 * ms and launches each point to 3 host values. */
int tracker_profile(tracker* t, int enable);
int tracker_profile_read(tracker* t, double* ms, int64_t* launches);

/* Instrumentation (no counterpart in the paper): the fused multiply-add rate
 * of the current device, float32 (dtype TRK_DTYPE_F32) or float64
 * (TRK_DTYPE_F64), measured by a short kernel of independent FMA chains on
 * every SM (about 10 ms, on the legacy default stream, synchronous).
 * *fma_per_s receives FMAs per second (one FMA = 2 flops): the denominator
 * of the FMA-bound fraction of the float32 and float64 interpolation forms.
 * Errors: TRK_EINVAL, TRK_ENOMEM, TRK_ECUDA. */
int tracker_probe_fma(int dtype, double* fma_per_s);

/* ---------------------------------------------------------------------- */
/* Binning without allocation                                              */
/* ---------------------------------------------------------------------- */

/* The same stable block binning as tracker_bin, for callers that cannot
 * allocate device memory (an allocator owned by another framework, code
 * that must not allocate after start-up, drivers that only receive
 * pre-allocated buffers).  It needs no tracker and allocates nothing: its
 * scratch is one fixed device array of about 6.3 MB inside the library,
 * reserved on every GPU that loads the library until the process exits.
 * The paper has no counterpart; this is a deployment convenience.
 *
 * Arguments as in tracker_bin, plus the grid (N, L) and block shape
 * (bx, by, bz) that a tracker would hold; nonfinite (device int32, may be
 * NULL) receives 1 if a position was non-finite, else 0.  stream is a
 * cudaStream_t of the current device.  pos and every output must be device
 * memory of the current device (checked: TRK_EINVAL otherwise), sized by the
 * caller: keys and perm np entries, offsets nblocks + 1 =
 * (N/bx)(N/by)(N/bz) + 1 entries, nonfinite one.  np may not exceed 262144
 * (2^18): larger calls return TRK_EINVAL with a message.  The first call on a device looks up the
 * array's device address, so make that first call before any stream
 * capture.  Every call reuses the same array, which keeps the last call's
 * contents; calls that overlap on the GPU (other streams, other threads)
 * race on it and must be serialised by the caller. */
int tracker_bin_static(int64_t np, const double* pos, int N, double L, int bx, int by, int bz, int32_t* keys,
                       int32_t* perm, int32_t* offsets, int32_t* nonfinite, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* TRACKER_H */
