// Block binning that allocates no memory: tracker_bin_static.
//
// Some callers cannot call cudaMalloc: code that runs inside another
// framework's memory pool or allocator hooks, code that must not allocate
// after start-up (real-time or capture-replay loops), and drivers that are
// only handed pre-allocated device buffers.  For them this entry point needs
// no tracker (whose creation allocates) and no allocation of its own: the
// radix-sort scratch lives in one file-scope device array of fixed size,
// reserved when the library is loaded and held until the process exits.
//
// The array is shared by every call on a device and keeps the contents of the
// last call; each call rewrites everything it reads before reading it, and
// clears its non-finite flag.  Calls whose work overlaps on the GPU (two
// streams, or two host threads) race on the array and must be serialised by
// the caller.
#include <cstdio>
#include <mutex>

#include "internal.cuh"
#include "tracker.h"

using namespace trk;

namespace {

// Capacity: at most 2^18 particles per call.  Layout of the scratch array:
//   [0, 256)                         non-finite flag (int)
//   [256, 256 + 4 NMAX)              block keys in the incoming order
//   [.., + 4 NMAX)                   sorted keys
//   [.., + radix scratch)            radix-sort histograms, scan partials, ping-pong buffers
constexpr int64_t NMAX = int64_t(1) << 18;
constexpr size_t KEYS_OFF = 256;
constexpr size_t SORTED_OFF = KEYS_OFF + 4 * NMAX;
constexpr size_t RADIX_OFF = SORTED_OFF + 4 * NMAX;
constexpr size_t RADIX_RESERVE = 4 * 4 * NMAX + 256 * 1024;   // 4 ping-pong arrays + histograms/scan
constexpr size_t SCRATCH_BYTES = RADIX_OFF + RADIX_RESERVE;    // about 6.3 MB

static __device__ __align__(256) unsigned char g_bin_scratch[SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
unsigned char* g_ptr[MAX_DEVICES] = {};

int fail(int code, const char* msg)
{
    set_error_message(msg);
    return code;
}

// Device address of the scratch array for the current device, looked up once
// per device (cudaGetSymbolAddress must run with that device current).
int scratch_for_current_device(unsigned char** out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
        cudaGetLastError();
        return fail(TRK_ECUDA, "tracker_bin_static: no current CUDA device");
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_ptr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_bin_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return fail(TRK_ECUDA, "tracker_bin_static: cudaGetSymbolAddress of the scratch array failed");
        }
        g_ptr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_ptr[dev];
    return TRK_OK;
}

int ilog2_ceil(int64_t x)
{
    int r = 0;
    while ((int64_t(1) << r) < x) ++r;
    return r;
}

bool pow2(int64_t x) { return x > 0 && (x & (x - 1)) == 0; }

int check_dev_ptr(const void* p, int dev, const char* name)
{
    if (!p || device_pointer_ok(p, dev)) return TRK_OK;
    char msg[160];
    snprintf(msg, sizeof(msg), "tracker_bin_static: %s must be device memory of the current device %d", name, dev);
    return fail(TRK_EINVAL, msg);
}

}  // namespace

bool trk::device_pointer_ok(const void* p, int dev)
{
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    return at.type == cudaMemoryTypeDevice && at.device == dev;
}

extern "C" {

int tracker_bin_static(int64_t np, const double* pos, int N, double L, int bx, int by, int bz, int32_t* keys,
                       int32_t* perm, int32_t* offsets, int32_t* nonfinite, void* stream)
{
    set_error_message("");
    if (np < 0 || np > NMAX)
        return fail(TRK_EINVAL, "tracker_bin_static: np outside [0, 262144] (the fixed scratch holds 2^18 particles)");
    if (!pow2(N) || N < 16 || N > 1024) return fail(TRK_EINVAL, "tracker_bin_static: N must be a power of two in [16, 1024]");
    if (!(L > 0)) return fail(TRK_EINVAL, "tracker_bin_static: L must be > 0");
    for (int b : {bx, by, bz})
        if (!pow2(b) || b > N) return fail(TRK_EINVAL, "tracker_bin_static: block edges must be powers of two <= N");
    if (!offsets || (np > 0 && (!pos || !perm))) return fail(TRK_EINVAL, "tracker_bin_static: NULL array argument");
    if (radix_scratch_bytes(NMAX) > RADIX_RESERVE) return fail(TRK_ECUDA, "tracker_bin_static: scratch reserve too small");

    unsigned char* s = nullptr;
    int rc = scratch_for_current_device(&s);
    if (rc) return rc;
    int dev = -1;
    cudaGetDevice(&dev);
    if ((rc = check_dev_ptr(np > 0 ? pos : nullptr, dev, "pos")) || (rc = check_dev_ptr(keys, dev, "keys")) ||
        (rc = check_dev_ptr(np > 0 ? perm : nullptr, dev, "perm")) || (rc = check_dev_ptr(offsets, dev, "offsets")) ||
        (rc = check_dev_ptr(nonfinite, dev, "nonfinite")))
        return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);

    GridGeom g{};
    g.N = N;
    g.mask = N - 1;
    g.inv_delta = (double)N / L;
    g.lb1 = ilog2_ceil(bx);
    g.lb2 = ilog2_ceil(by);
    g.lb3 = ilog2_ceil(bz);
    g.nb1 = N / bx;
    g.nb2 = N / by;
    g.nb3 = N / bz;
    const int64_t nblocks = (int64_t)g.nb1 * g.nb2 * g.nb3;

    int* flag = reinterpret_cast<int*>(s);
    uint32_t* k = keys ? reinterpret_cast<uint32_t*>(keys) : reinterpret_cast<uint32_t*>(s + KEYS_OFF);
    uint32_t* ks = reinterpret_cast<uint32_t*>(s + SORTED_OFF);
    if (cudaMemsetAsync(flag, 0, sizeof(int), st) != cudaSuccess) {
        cudaGetLastError();
        return fail(TRK_ECUDA, "tracker_bin_static: clearing the flag failed");
    }
    cudaError_t e = launch_keys(g, np, pos, k, flag, st);
    if (e == cudaSuccess) e = radix_sort(k, np, ilog2_ceil(nblocks), ks, perm, s + RADIX_OFF, st, nullptr);
    if (e == cudaSuccess) e = launch_offsets(ks, np, nblocks, offsets, st);
    if (e == cudaSuccess && nonfinite) e = cudaMemcpyAsync(nonfinite, flag, sizeof(int), cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(TRK_ECUDA, "tracker_bin_static: kernel launch failed");
    }
    return TRK_OK;
}

}  // extern "C"
