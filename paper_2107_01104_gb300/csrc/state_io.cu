// Tracer-set checkpoints: the single-GPU form of the paper's ordered particle
// output and restart (Sec. 3.4), as one plain binary file per set.
//
// The state is written in the caller's particle order (tracker_advance
// returns positions and AB histories in that order, its last kernel being the
// inverse-permutation gather), so a restart reads back exactly the arrays the
// run was holding and continues bit for bit.
//
// File layout (little-endian, no padding):
//   0   char[8]  magic "TRKSTAT1"
//   8   u32      format version (1)
//   12  u32      header bytes (HEADER_BYTES)
//   16  i32 N, i32 family, i32 I, i32 m, f64 L
//   40  i64 np, i32 scheme, i32 history_valid, i64 step, f64 time, f64 dt
//   80  u64      checksum of the payload
//   88  u64      checksum of bytes 0 .. 87
//   96  payload: positions [3][np] f64, then for ABk (k = scheme + 1) the
//       history [3 (k-1)][np] f32
// The checksum is FNV-1a style over 64-bit little-endian words (then the tail
// bytes one by one): h = (h xor w) * 1099511628211 from 14695981039346656037.
// Host code only; all pointers are host memory.
#include <cerrno>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <unistd.h>

#include "tracker.h"
#include "internal.cuh"

namespace {

int fail(int code, const char* fmt, ...)
{
    char msg[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(msg, sizeof(msg), fmt, ap);
    va_end(ap);
    trk::set_error_message(msg);
    return code;
}

constexpr char kMagic[8] = {'T', 'R', 'K', 'S', 'T', 'A', 'T', '1'};
constexpr uint32_t kVersion = 1;
constexpr uint32_t HEADER_BYTES = 96;
constexpr uint64_t kFnvOffset = 14695981039346656037ull, kFnvPrime = 1099511628211ull;

uint64_t checksum(uint64_t h, const void* data, size_t n)
{
    const unsigned char* p = static_cast<const unsigned char*>(data);
    size_t i = 0;
    for (; i + 8 <= n; i += 8) {
        uint64_t w;
        memcpy(&w, p + i, 8);
        h = (h ^ w) * kFnvPrime;
    }
    for (; i < n; ++i) h = (h ^ p[i]) * kFnvPrime;
    return h;
}

bool little_endian()
{
    const uint32_t x = 1;
    unsigned char b;
    memcpy(&b, &x, 1);
    return b == 1;
}

// history rows of a scheme: 3 (k - 1) for ABk, none for RK2
int history_rows(int scheme) { return scheme == TRK_RK2 ? 0 : 3 * scheme; }

struct Writer {
    std::vector<unsigned char> b;
    template <class V>
    void put(V v)
    {
        const size_t o = b.size();
        b.resize(o + sizeof(V));
        memcpy(b.data() + o, &v, sizeof(V));
    }
};

struct Reader {
    const unsigned char* p;
    size_t o = 0;
    template <class V>
    V get()
    {
        V v;
        memcpy(&v, p + o, sizeof(V));
        o += sizeof(V);
        return v;
    }
};

std::vector<unsigned char> encode_header(const trk_state_info& s, uint64_t payload_sum)
{
    Writer w;
    for (char c : kMagic) w.put(c);
    w.put(kVersion);
    w.put(HEADER_BYTES);
    w.put((int32_t)s.N);
    w.put((int32_t)s.family);
    w.put((int32_t)s.I);
    w.put((int32_t)s.m);
    w.put((double)s.L);
    w.put((int64_t)s.np);
    w.put((int32_t)s.scheme);
    w.put((int32_t)s.history_valid);
    w.put((int64_t)s.step);
    w.put((double)s.time);
    w.put((double)s.dt);
    w.put(payload_sum);
    w.put(checksum(kFnvOffset, w.b.data(), w.b.size()));
    return w.b;
}

int check_info(const trk_state_info& s)
{
    if (s.np < 0 || s.np > 2147483647LL) return fail(TRK_EINVAL, "np=%lld out of range", (long long)s.np);
    if (s.scheme < TRK_RK2 || s.scheme > TRK_AB4) return fail(TRK_EINVAL, "unknown scheme %d", s.scheme);
    const int k = s.scheme == TRK_RK2 ? 0 : s.scheme + 1;
    if (s.history_valid < 0 || s.history_valid > (k ? k - 1 : 0))
        return fail(TRK_EINVAL, "history_valid=%d invalid for scheme %d", s.history_valid, s.scheme);
    return TRK_OK;
}

// reads and validates the header; f is positioned at the payload
int read_header(FILE* f, const char* path, trk_state_info* s, uint64_t* payload_sum)
{
    unsigned char h[HEADER_BYTES];
    if (fread(h, 1, HEADER_BYTES, f) != HEADER_BYTES)
        return fail(TRK_EIO, "%s: truncated header", path);
    if (memcmp(h, kMagic, 8) != 0) return fail(TRK_EIO, "%s: not a tracer-state file", path);
    Reader r{h};
    r.o = 8;
    const uint32_t version = r.get<uint32_t>(), hb = r.get<uint32_t>();
    if (version != kVersion || hb != HEADER_BYTES)
        return fail(TRK_EIO, "%s: unsupported format version %u", path, version);
    s->N = r.get<int32_t>();
    s->family = r.get<int32_t>();
    s->I = r.get<int32_t>();
    s->m = r.get<int32_t>();
    s->L = r.get<double>();
    s->np = r.get<int64_t>();
    s->scheme = r.get<int32_t>();
    s->history_valid = r.get<int32_t>();
    s->step = r.get<int64_t>();
    s->time = r.get<double>();
    s->dt = r.get<double>();
    *payload_sum = r.get<uint64_t>();
    const uint64_t hsum = r.get<uint64_t>();
    if (hsum != checksum(kFnvOffset, h, HEADER_BYTES - 8)) return fail(TRK_EIO, "%s: header checksum mismatch", path);
    if (check_info(*s) != TRK_OK) return fail(TRK_EIO, "%s: invalid header fields", path);
    return TRK_OK;
}

}  // namespace

extern "C" {

int tracker_state_write(const char* path, const trk_state_info* info, const double* pos, const float* rhs)
{
    if (!path || !info) return fail(TRK_EINVAL, "path and info must not be NULL");
    if (!little_endian()) return fail(TRK_EIO, "tracer-state files are little-endian; this host is not");
    int rc = check_info(*info);
    if (rc) return rc;
    const int64_t np = info->np;
    const int rows = history_rows(info->scheme);
    if (np > 0 && (!pos || (rows && !rhs))) return fail(TRK_EINVAL, "pos (and rhs for AB) must not be NULL");
    const size_t pos_bytes = (size_t)np * 3 * sizeof(double), rhs_bytes = (size_t)np * rows * sizeof(float);
    uint64_t sum = checksum(kFnvOffset, pos, pos_bytes);
    sum = checksum(sum, rhs, rhs_bytes);
    const std::vector<unsigned char> hdr = encode_header(*info, sum);
    // write a temporary file next to the target, then rename it into place
    const std::string tmp = std::string(path) + ".tmp" + std::to_string((long long)getpid());
    FILE* f = fopen(tmp.c_str(), "wb");
    if (!f) return fail(TRK_EIO, "%s: %s", tmp.c_str(), strerror(errno));
    bool ok = fwrite(hdr.data(), 1, hdr.size(), f) == hdr.size();
    ok = ok && (pos_bytes == 0 || fwrite(pos, 1, pos_bytes, f) == pos_bytes);
    ok = ok && (rhs_bytes == 0 || fwrite(rhs, 1, rhs_bytes, f) == rhs_bytes);
    ok = (fflush(f) == 0) && ok;
    ok = (fclose(f) == 0) && ok;
    if (!ok || rename(tmp.c_str(), path) != 0) {
        const int e = errno;
        remove(tmp.c_str());
        return fail(TRK_EIO, "%s: write failed: %s", path, strerror(e));
    }
    return TRK_OK;
}

int tracker_state_read_info(const char* path, trk_state_info* info)
{
    if (!path || !info) return fail(TRK_EINVAL, "path and info must not be NULL");
    FILE* f = fopen(path, "rb");
    if (!f) return fail(TRK_EIO, "%s: %s", path, strerror(errno));
    uint64_t sum;
    const int rc = read_header(f, path, info, &sum);
    fclose(f);
    return rc;
}

int tracker_state_read(const char* path, int64_t np, double* pos, float* rhs, trk_state_info* info)
{
    if (!path || !info) return fail(TRK_EINVAL, "path and info must not be NULL");
    FILE* f = fopen(path, "rb");
    if (!f) return fail(TRK_EIO, "%s: %s", path, strerror(errno));
    uint64_t sum;
    int rc = read_header(f, path, info, &sum);
    if (rc) {
        fclose(f);
        return rc;
    }
    const int rows = history_rows(info->scheme);
    if (info->np != np) {
        fclose(f);
        return fail(TRK_EINVAL, "%s holds %lld particles, the buffers %lld", path, (long long)info->np,
                         (long long)np);
    }
    if (np > 0 && (!pos || (rows && !rhs))) {
        fclose(f);
        return fail(TRK_EINVAL, "pos (and rhs for AB) must not be NULL");
    }
    const size_t pos_bytes = (size_t)np * 3 * sizeof(double), rhs_bytes = (size_t)np * rows * sizeof(float);
    bool ok = pos_bytes == 0 || fread(pos, 1, pos_bytes, f) == pos_bytes;
    ok = ok && (rhs_bytes == 0 || fread(rhs, 1, rhs_bytes, f) == rhs_bytes);
    const bool at_end = ok && fgetc(f) == EOF;
    fclose(f);
    if (!ok) return fail(TRK_EIO, "%s: truncated payload", path);
    if (!at_end) return fail(TRK_EIO, "%s: trailing bytes after the payload", path);
    uint64_t got = checksum(kFnvOffset, pos, pos_bytes);
    got = checksum(got, rhs, rhs_bytes);
    if (got != sum) return fail(TRK_EIO, "%s: payload checksum mismatch", path);
    return TRK_OK;
}

}  // extern "C"
