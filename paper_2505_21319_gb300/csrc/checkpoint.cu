// Checkpoint / resume of a fit (host code only): the parameter grid, Adam's
// two moments, the step count and the configuration of the fit in one flat
// little-endian file.
//
//   offset   0  "EFUNCCKP"                       8 bytes
//            8  format version (1)               uint32
//           12  header bytes (128)               uint32
//           16  R, W                             int32 x 2
//           24  log_beta0                        float32
//           28  channels                         int32
//           32  n (floats per array)             int64
//           40  step                             int64
//           48  seed                             uint64
//           56  loss, adam.decoupled             int32 x 2
//           64  lr, beta1, beta2, eps, wd        float64 x 5
//          104  zero                             16 bytes
//          120  FNV-1a 64 of bytes 0..119        uint64
//          128  params, m, v                     float32 x 3n
//   128 + 12n  FNV-1a 64 of the 12n payload bytes  uint64
//
// The file is written to a temporary name beside the target (unique per
// process and call), flushed to the storage device, renamed over the target
// and the directory entry flushed as well, so a crash or power loss at any
// point leaves either the previous checkpoint or the complete new one.
#include <fcntl.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>
#include <unistd.h>

#include <atomic>
#include <string>

#include "common.cuh"

namespace {

constexpr char kMagic[8] = {'E', 'F', 'U', 'N', 'C', 'C', 'K', 'P'};
constexpr uint32_t kVersion = 1;
constexpr uint32_t kHeaderBytes = 128;
constexpr int64_t kMaxFloats = (int64_t)1 << 40;

// FNV-1a, 64-bit (Fowler, Noll, Vo): offset basis and prime of the
// published definition.
struct Fnv {
    uint64_t h = 14695981039346656037ull;
    void add(const void *p, size_t n)
    {
        const unsigned char *b = static_cast<const unsigned char *>(p);
        for (size_t i = 0; i < n; ++i) {
            h ^= b[i];
            h *= 1099511628211ull;
        }
    }
};

// little-endian field writers / readers on a byte buffer
template <class T>
void put(unsigned char *buf, size_t off, T v)
{
    unsigned char b[sizeof(T)];
    memcpy(b, &v, sizeof(T));
    for (size_t i = 0; i < sizeof(T); ++i) buf[off + i] = b[i];   // hosts of this library are little-endian
}

template <class T>
T get(const unsigned char *buf, size_t off)
{
    T v;
    memcpy(&v, buf + off, sizeof(T));
    return v;
}

bool info_ok(const efunc_checkpoint_info *in)
{
    if (!in || in->R < 1 || in->R > efunc::kMaxR || in->W < 1 || in->channels < 1 || in->step < 0) return false;
    const int64_t cells = (int64_t)in->R * in->R * in->R;
    return in->n == cells * in->channels && in->n <= kMaxFloats;
}

void encode_header(const efunc_checkpoint_info *in, unsigned char *h)
{
    memset(h, 0, kHeaderBytes);
    memcpy(h, kMagic, 8);
    put<uint32_t>(h, 8, kVersion);
    put<uint32_t>(h, 12, kHeaderBytes);
    put<int32_t>(h, 16, in->R);
    put<int32_t>(h, 20, in->W);
    put<float>(h, 24, in->log_beta0);
    put<int32_t>(h, 28, in->channels);
    put<int64_t>(h, 32, in->n);
    put<int64_t>(h, 40, in->step);
    put<uint64_t>(h, 48, in->seed);
    put<int32_t>(h, 56, in->loss);
    put<int32_t>(h, 60, in->adam.decoupled);
    put<double>(h, 64, in->adam.lr);
    put<double>(h, 72, in->adam.beta1);
    put<double>(h, 80, in->adam.beta2);
    put<double>(h, 88, in->adam.eps);
    put<double>(h, 96, in->adam.weight_decay);
    Fnv f;
    f.add(h, 120);
    put<uint64_t>(h, 120, f.h);
}

// Parses and checks a header; false if it is not a valid version-1 header.
bool decode_header(const unsigned char *h, efunc_checkpoint_info *out)
{
    if (memcmp(h, kMagic, 8) != 0 || get<uint32_t>(h, 8) != kVersion || get<uint32_t>(h, 12) != kHeaderBytes)
        return false;
    Fnv f;
    f.add(h, 120);
    if (f.h != get<uint64_t>(h, 120)) return false;
    efunc_checkpoint_info in{};
    in.R = get<int32_t>(h, 16);
    in.W = get<int32_t>(h, 20);
    in.log_beta0 = get<float>(h, 24);
    in.channels = get<int32_t>(h, 28);
    in.n = get<int64_t>(h, 32);
    in.step = get<int64_t>(h, 40);
    in.seed = get<uint64_t>(h, 48);
    in.loss = get<int32_t>(h, 56);
    in.adam.decoupled = get<int32_t>(h, 60);
    in.adam.lr = get<double>(h, 64);
    in.adam.beta1 = get<double>(h, 72);
    in.adam.beta2 = get<double>(h, 80);
    in.adam.eps = get<double>(h, 88);
    in.adam.weight_decay = get<double>(h, 96);
    if (!info_ok(&in)) return false;
    *out = in;
    return true;
}

struct File {
    FILE *f = nullptr;
    explicit File(FILE *p) : f(p) {}
    ~File()
    {
        if (f) fclose(f);
    }
};

// Reads and checks the header of an open checkpoint.
efunc_status read_header(FILE *f, efunc_checkpoint_info *info)
{
    unsigned char h[kHeaderBytes];
    if (fread(h, 1, kHeaderBytes, f) != kHeaderBytes) return EFUNC_ERR_IO;
    return decode_header(h, info) ? EFUNC_OK : EFUNC_ERR_IO;
}

}  // namespace

extern "C" {

efunc_status efunc_checkpoint_save(const char *path, const efunc_checkpoint_info *info, const float *params,
                                   const float *m, const float *v)
{
    if (!path || !*path || !info_ok(info) || !params || !m || !v) return EFUNC_ERR_ARG;
    unsigned char h[kHeaderBytes];
    encode_header(info, h);
    static std::atomic<unsigned long long> calls{0};   // two saves in one process never share a temporary
    const std::string tmp = std::string(path) + ".tmp" + std::to_string((long)getpid()) + "." +
                            std::to_string(calls.fetch_add(1));
    Fnv sum;
    {
        File out(fopen(tmp.c_str(), "wb"));
        if (!out.f) return EFUNC_ERR_IO;
        bool ok = fwrite(h, 1, kHeaderBytes, out.f) == kHeaderBytes;
        for (const float *a : {params, m, v}) {
            const size_t bytes = (size_t)info->n * sizeof(float);
            ok = ok && fwrite(a, 1, bytes, out.f) == bytes;
            if (ok) sum.add(a, bytes);
        }
        unsigned char t[8];
        put<uint64_t>(t, 0, sum.h);
        ok = ok && fwrite(t, 1, 8, out.f) == 8;
        ok = ok && fflush(out.f) == 0;
        ok = ok && fsync(fileno(out.f)) == 0;   // the data is on the device before the rename
        const int rc = fclose(out.f);
        out.f = nullptr;
        if (!ok || rc != 0) {
            remove(tmp.c_str());
            return EFUNC_ERR_IO;
        }
    }
    if (rename(tmp.c_str(), path) != 0) {
        remove(tmp.c_str());
        return EFUNC_ERR_IO;
    }
    // the rename itself lives in the directory: flush it too
    const std::string p(path);
    const size_t slash = p.find_last_of('/');
    const std::string dir = slash == std::string::npos ? std::string(".") : (slash == 0 ? std::string("/")
                                                                                           : p.substr(0, slash));
    const int dfd = open(dir.c_str(), O_RDONLY | O_DIRECTORY);
    if (dfd < 0) return EFUNC_ERR_IO;
    const int drc = fsync(dfd);
    close(dfd);
    return drc == 0 ? EFUNC_OK : EFUNC_ERR_IO;
}

efunc_status efunc_checkpoint_info_read(const char *path, efunc_checkpoint_info *info)
{
    if (!path || !info) return EFUNC_ERR_ARG;
    File in(fopen(path, "rb"));
    if (!in.f) return EFUNC_ERR_IO;
    return read_header(in.f, info);
}

efunc_status efunc_checkpoint_load(const char *path, efunc_checkpoint_info *info, float *params, float *m, float *v,
                                   int64_t capacity)
{
    if (!path || !info || !params || !m || !v || capacity < 0) return EFUNC_ERR_ARG;
    File in(fopen(path, "rb"));
    if (!in.f) return EFUNC_ERR_IO;
    efunc_checkpoint_info got{};
    efunc_status st = read_header(in.f, &got);
    if (st) return st;
    if (got.n > capacity) return EFUNC_ERR_ARG;
    Fnv sum;
    for (float *a : {params, m, v}) {
        const size_t bytes = (size_t)got.n * sizeof(float);
        if (fread(a, 1, bytes, in.f) != bytes) return EFUNC_ERR_IO;
        sum.add(a, bytes);
    }
    unsigned char t[9];
    if (fread(t, 1, 9, in.f) != 8 || get<uint64_t>(t, 0) != sum.h) return EFUNC_ERR_IO;   // nothing may follow
    *info = got;
    return EFUNC_OK;
}

}  // extern "C"
