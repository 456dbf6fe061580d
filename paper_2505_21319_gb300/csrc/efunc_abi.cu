// The C ABI (include/efunc.h): argument validation, workspace layout, launch
// order of the hot path, and the launch counter / event profiler.
#include <math.h>
#include <stddef.h>
#include <map>
#include <mutex>
#include <string.h>
#include <tuple>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "adam_clock.cuh"
#include "common.cuh"
#include "sort_copies.cuh"

namespace efunc {

efunc_status cuda_fail(cudaError_t e = cudaSuccess);

namespace {

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// ----------------------------------------------------------- profiling

struct Pending {
    int kid;
    cudaEvent_t start, stop;
};

std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<Pending> g_pending;
std::vector<cudaEvent_t> g_free_events;
double g_ms[K_COUNT];
int64_t g_count[K_COUNT];
int64_t g_launches = 0;
// set while this thread captures a CUDA graph: its launches are counted in
// g_captured (they run once per replay), not timed
thread_local bool g_in_capture = false;
thread_local int64_t g_captured = 0;

const char *const kKernelNames[K_COUNT] = {"bin",       "scan_reduce", "scan_top",       "scan_emit", "scatter",
                                           "pack_keys", "forward",     "fused_backward", "fused_fit", "adam",
                                           "mean_shift", "variant_pack", "variant_forward", "variant_backward",
                                           "variant_fit", "cosine_pack", "cosine_forward", "cosine_backward",
                                           "cosine_fit", "eval", "f64", "batched", "batched_stats", "enc_conv", "enc_wgrad", "enc_aux", "grouped",
                                           "eval_finish"};

cudaEvent_t take_event()
{
    if (!g_free_events.empty()) {
        cudaEvent_t e = g_free_events.back();
        g_free_events.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// Resolves pending event pairs into totals.  Caller holds g_prof_mu.
int drain_pending()
{
    int rc = 0;
    for (Pending &p : g_pending) {
        if (p.start && p.stop) {
            float ms = 0.f;
            if (cudaEventSynchronize(p.stop) == cudaSuccess && cudaEventElapsedTime(&ms, p.start, p.stop) == cudaSuccess) {
                g_ms[p.kid] += ms;
                g_count[p.kid] += 1;
            } else {
                rc = -1;
            }
        }
        if (p.start) g_free_events.push_back(p.start);
        if (p.stop) g_free_events.push_back(p.stop);
    }
    g_pending.clear();
    return rc;
}

}  // namespace

// Every launch is also an NVTX range named after its kernel (a no-op unless
// a tool such as ncu --nvtx is attached), so that profiles can select the
// sort, the key pack, the fused kernels and Adam by name.
static_assert(sizeof(kKernelNames) / sizeof(kKernelNames[0]) == K_COUNT, "one name per kernel id");

void launch_begin(int kid, cudaStream_t s)
{
    nvtxRangePushA(kKernelNames[kid]);
    if (g_in_capture) {
        ++g_captured;
        return;
    }
    std::lock_guard<std::mutex> lk(g_prof_mu);
    ++g_launches;
    if (!g_prof_on) return;
    Pending p{kid, take_event(), nullptr};
    if (p.start) cudaEventRecord(p.start, s);
    g_pending.push_back(p);
}

void launch_end(int kid, cudaStream_t s)
{
    nvtxRangePop();
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (!g_prof_on || g_in_capture || g_pending.empty() || g_pending.back().kid != kid || g_pending.back().stop)
        return;
    cudaEvent_t e = take_event();
    if (e) cudaEventRecord(e, s);
    g_pending.back().stop = e;
}

// ------------------------------------------------ per-device property cache

int current_device()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return dev;
}

std::recursive_mutex &device_cache_mutex()
{
    static std::recursive_mutex mu;
    return mu;
}

int &device_cache_slot(int dev, const void *key, int tag)
{
    static std::map<std::tuple<int, const void *, int>, int> slots;   // references stay valid on insertion
    return slots[std::make_tuple(dev, key, tag)];
}

int device_sm_count()
{
    static const char key = 0;
    return per_device_cached(&key, 0, [] {
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, current_device()) != cudaSuccess) {
            cudaGetLastError();
            sms = 0;
        }
        return sms > 0 ? sms : 1;
    });
}

// ------------------------------------------------------------- layout

Layout make_layout(int R, int64_t J, int key_records, int channels, bool two_sort_buffers, bool fit_regions)
{
    Layout L{};
    L.P = (R + 1 + kBrick - 1) / kBrick;
    L.nbins = (int64_t)L.P * L.P * L.P * 64;
    L.nscan_blocks = (L.nbins + kScanSegment - 1) / kScanSegment;
    L.max_items = (J + kChunk - 1) / kChunk + (J < L.nbins ? J : L.nbins);
    const size_t A = 256;
    size_t off = 0;
    L.ctrl = off;      off = align_up(off + sizeof(Ctrl), A);
    L.hist = off;      off = align_up(off + (size_t)hist_entries(L.nbins) * 4, A);
    L.blocksum = off;  off = align_up(off + (size_t)L.nscan_blocks * 8, A);
    L.rank = off;      off = align_up(off + (size_t)J * 4, A);
    L.sorted = off;    off = align_up(off + (size_t)J * 16, A);
    L.perm = off;      off = align_up(off + (size_t)J * 4, A);
    L.items = off;     off = align_up(off + (size_t)L.max_items * 16, A);
    L.keys = off;      off = align_up(off + (size_t)R * R * R * key_records * 16, A);
    if (fit_regions) {
        L.grad = off;  off = align_up(off + (size_t)R * R * R * channels * 4, A);
        L.stage = off; off = align_up(off + (size_t)J * 32, A);   // two host-batch staging buffers
    }
    L.two_sort_buffers = two_sort_buffers;
    if (two_sort_buffers) {
        L.ctrl2 = off;     off = align_up(off + sizeof(Ctrl), A);
        L.hist2 = off;     off = align_up(off + (size_t)hist_entries(L.nbins) * 4, A);
        L.blocksum2 = off; off = align_up(off + (size_t)L.nscan_blocks * 8, A);
        L.rank2 = off;     off = align_up(off + (size_t)J * 4, A);
        L.sorted2 = off;   off = align_up(off + (size_t)J * 16, A);
        L.items2 = off;    off = align_up(off + (size_t)L.max_items * 16, A);
    }
    L.total = off;
    return L;
}

}  // namespace efunc

using namespace efunc;

namespace {

constexpr int64_t kMaxJ = (int64_t)1 << 30;
constexpr int32_t kMaxGraphBatches = 64;   // a captured period holds lcm(2, n_batches) steps

bool grid_ok(const efunc_grid *g) { return g && g->R >= 1 && g->R <= kMaxR; }

efunc_status check_grid(const efunc_grid *g)
{
    if (!grid_ok(g)) return EFUNC_ERR_ARG;
    if (g->W != kW) return EFUNC_ERR_UNSUPPORTED;
    if (!isfinite(g->log_beta0)) return EFUNC_ERR_NONFINITE;
    return EFUNC_OK;
}

// fit: the in-line fit needs the gradient and staging regions too
efunc_status check_workspace(const efunc_grid *g, int64_t J, const void *ws, size_t ws_bytes, bool fit = false)
{
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u)) return EFUNC_ERR_WORKSPACE;
    if (ws_bytes < (fit ? make_layout(g->R, J) : eval_layout(g->R, J)).total) return EFUNC_ERR_WORKSPACE;
    return EFUNC_OK;
}

// FP64 calls: the forward's layout followed by the FP32 rows that choose
// the windows (J x 16 B), the FP64 rows in sorted order (J x 32 B) and the
// FP64 key records (R^3 x 4 x 32 B).
struct Layout64 {
    Layout L;
    size_t rows32, rows64, keys64, total;
};

Layout64 layout64(int R, int64_t J)
{
    Layout64 X{};
    X.L = eval_layout(R, J);
    size_t off = X.L.total;
    X.rows32 = off; off = align_up(off + (size_t)J * 16, 256);
    X.rows64 = off; off = align_up(off + (size_t)J * 32, 256);
    X.keys64 = off; off = align_up(off + (size_t)R * R * R * kKeyRecords * 32, 256);
    X.total = off;
    return X;
}

struct Views {
    Layout L;
    char *base;
    Ctrl *ctrl() const { return reinterpret_cast<Ctrl *>(base + L.ctrl); }
    uint32_t *hist() const { return reinterpret_cast<uint32_t *>(base + L.hist); }
    unsigned long long *blocksum() const { return reinterpret_cast<unsigned long long *>(base + L.blocksum); }
    uint32_t *rank() const { return reinterpret_cast<uint32_t *>(base + L.rank); }
    float4 *sorted() const { return reinterpret_cast<float4 *>(base + L.sorted); }
    int *perm() const { return reinterpret_cast<int *>(base + L.perm); }
    Item *items() const { return reinterpret_cast<Item *>(base + L.items); }
    float4 *keys() const { return reinterpret_cast<float4 *>(base + L.keys); }
    float *grad() const { return reinterpret_cast<float *>(base + L.grad); }
    // staging buffer b (0 or 1) of a host batch: J rows of 4 floats each
    float4 *stage(int b, int64_t J) const { return reinterpret_cast<float4 *>(base + L.stage) + (size_t)b * (size_t)J; }
};

// One of the two sort buffers of a pipelined fit (buffer 0 is the one every
// other call uses).
struct SortBuf {
    Ctrl *ctrl;
    uint32_t *hist;
    unsigned long long *blocksum;
    uint32_t *rank;
    float4 *sorted;
    Item *items;
    Item *gtop;   // grouped items are stored from here down
};

SortBuf sort_buf(const Views &v, int b)
{
    const Layout &L = v.L;
    char *p = v.base;
    if (b == 0)
        return {v.ctrl(), v.hist(), v.blocksum(), v.rank(), v.sorted(), v.items(), v.items() + L.max_items - 1};
    Item *it2 = reinterpret_cast<Item *>(p + L.items2);
    return {reinterpret_cast<Ctrl *>(p + L.ctrl2), reinterpret_cast<uint32_t *>(p + L.hist2),
            reinterpret_cast<unsigned long long *>(p + L.blocksum2), reinterpret_cast<uint32_t *>(p + L.rank2),
            reinterpret_cast<float4 *>(p + L.sorted2), it2, it2 + L.max_items - 1};
}

// Queries per octet at most of the grouped items of a single-shape fit:
// large sparse batches (at least 2^18 queries, at most 16 per bin on average)
// group their sparse octets; denser batches keep one item per cell, and so do
// small ones, whose few items the second (grouped) launch would only
// lengthen (measured on one GB300: 64^3 x 2^22 1.59 instead of 3.03 ms per
// step, 32^3 x 2^18 0.26 instead of 0.41, 16^3 x 65,536 0.13 instead of 0.067).
int fit_group_max(const Layout &L, int64_t J) { return (J >= (1 << 18) && J <= 16 * L.nbins) ? kGroupMax : 0; }

cudaError_t sort_into_buf(const SortBuf &b, const Layout &L, int R, const float *q, int64_t J, int q_stride,
                          cudaStream_t s, int narrow_blocks, int group_max = 0)
{
    cudaError_t e = cudaMemsetAsync(b.ctrl, 0, sizeof(Ctrl), s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(b.hist, 0, (size_t)hist_entries(L.nbins) * 4, s);
    if (e != cudaSuccess) return e;
    SortArgs a{};
    a.q = q;
    a.J = J;
    a.q_stride = q_stride;
    a.R = R;
    a.P = L.P;
    a.nbins = L.nbins;
    a.hist = b.hist;
    a.blocksum = b.blocksum;
    a.rank = b.rank;
    a.sorted = b.sorted;
    a.perm = nullptr;
    a.items = b.items;
    a.ctrl = b.ctrl;
    a.group_max = group_max;
    a.gtop = b.gtop;
    return launch_sort(a, s, narrow_blocks);
}

// Clears the control block and histogram, then sorts q into the workspace
// (or into the caller's sorted / perm buffers when given).
cudaError_t sort_into(const Views &v, int R, const float *q, int64_t J, int q_stride, float4 *sorted, int *perm,
                      cudaStream_t s, int group_max = 0)
{
    cudaError_t e = cudaMemsetAsync(v.ctrl(), 0, sizeof(Ctrl), s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(v.hist(), 0, (size_t)hist_entries(v.L.nbins) * 4, s);
    if (e != cudaSuccess) return e;
    SortArgs a{};
    a.q = q;
    a.J = J;
    a.q_stride = q_stride;
    a.R = R;
    a.P = v.L.P;
    a.nbins = v.L.nbins;
    a.hist = v.hist();
    a.blocksum = v.blocksum();
    a.rank = v.rank();
    a.sorted = sorted;
    a.perm = perm;
    a.items = v.items();
    a.ctrl = v.ctrl();
    a.group_max = group_max;
    a.gtop = v.items() + v.L.max_items - 1;
    return launch_sort(a, s);
}

// Packs the parameters into key records, then fills the fused-kernel arguments.
cudaError_t pack_keys(const Views &v, const efunc_grid *g, const float *params, cudaStream_t s)
{
    PackArgs p{};
    p.params = params;
    p.keys = v.keys();
    p.R = g->R;
    p.log_beta0 = (double)g->log_beta0;
    return launch_pack_keys(p, s);
}

FusedArgs fused_args(const Views &v, const efunc_grid *g)
{
    FusedArgs f{};
    f.keys = v.keys();
    f.R = g->R;
    f.sorted = v.sorted();
    f.perm = v.perm();
    f.items = v.items();
    f.ctrl = v.ctrl();
    return f;
}

// Per-device streams and events of efunc_fit: the copy stream overlaps the
// host->device copy of batch s+1 with the computation of batch s; the sort
// stream sorts batch s+1 into the other sort buffer meanwhile (pipelined
// fit).  Created on the first fit on a device and kept for the process.
struct CopyPipe {
    bool ready = false;
    cudaStream_t stream = nullptr;
    cudaStream_t sort_stream = nullptr;
    cudaEvent_t copied[2] = {nullptr, nullptr};
    cudaEvent_t freed[2] = {nullptr, nullptr};
    cudaEvent_t sorted[2] = {nullptr, nullptr};
    cudaEvent_t consumed[2] = {nullptr, nullptr};
    cudaEvent_t packed = nullptr;
    cudaEvent_t joined = nullptr;   // the sort stream's end of a captured period
    std::mutex mu;                  // held by a fit while it enqueues its steps
    cudaStream_t capture_stream = nullptr;   // origin of graph captures (the caller's may be the legacy stream)
};
constexpr int kMaxPipes = 64;
std::mutex g_pipe_mu;
CopyPipe g_pipes[kMaxPipes];

cudaError_t copy_pipe(CopyPipe **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxPipes) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_pipe_mu);
    CopyPipe &p = g_pipes[dev];
    if (!p.ready) {
        if ((e = cudaStreamCreateWithFlags(&p.stream, cudaStreamNonBlocking)) != cudaSuccess) return e;
        if ((e = cudaStreamCreateWithFlags(&p.sort_stream, cudaStreamNonBlocking)) != cudaSuccess) return e;
        for (int b = 0; b < 2; ++b) {
            if ((e = cudaEventCreateWithFlags(&p.copied[b], cudaEventDisableTiming)) != cudaSuccess) return e;
            if ((e = cudaEventCreateWithFlags(&p.freed[b], cudaEventDisableTiming)) != cudaSuccess) return e;
            if ((e = cudaEventCreateWithFlags(&p.sorted[b], cudaEventDisableTiming)) != cudaSuccess) return e;
            if ((e = cudaEventCreateWithFlags(&p.consumed[b], cudaEventDisableTiming)) != cudaSuccess) return e;
        }
        if ((e = cudaEventCreateWithFlags(&p.packed, cudaEventDisableTiming)) != cudaSuccess) return e;
        if ((e = cudaEventCreateWithFlags(&p.joined, cudaEventDisableTiming)) != cudaSuccess) return e;
        if ((e = cudaStreamCreateWithFlags(&p.capture_stream, cudaStreamNonBlocking)) != cudaSuccess) return e;
        p.ready = true;
    }
    *out = &p;
    return cudaSuccess;
}

bool is_host_pointer(const void *p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();   // clear the sticky-free error of an unknown pointer
        return true;
    }
    return at.type == cudaMemoryTypeHost || at.type == cudaMemoryTypeUnregistered;
}

}  // namespace

namespace efunc {

// the CUDA error behind this thread's last EFUNC_ERR_CUDA (efunc_last_cuda_error)
thread_local int g_last_cuda = 0;

// Records and clears the runtime's pending error of a failed CUDA call (so it
// cannot surface in a later call's launch check) and returns EFUNC_ERR_CUDA.
efunc_status cuda_fail(cudaError_t e)
{
    const cudaError_t pending = cudaGetLastError();
    if (e == cudaSuccess) e = pending;
    g_last_cuda = e == cudaSuccess ? (int)cudaErrorUnknown : (int)e;
    return EFUNC_ERR_CUDA;
}

}  // namespace efunc

namespace {

efunc_status cuda_status(cudaError_t e) { return e == cudaSuccess ? EFUNC_OK : cuda_fail(e); }

efunc_status check_adam(const efunc_adam *a)
{
    if (!a) return EFUNC_ERR_ARG;
    if (!isfinite(a->lr) || !isfinite(a->beta1) || !isfinite(a->beta2) || !isfinite(a->eps) ||
        !isfinite(a->weight_decay))
        return EFUNC_ERR_NONFINITE;
    if (a->beta1 < 0.0 || a->beta1 >= 1.0 || a->beta2 < 0.0 || a->beta2 >= 1.0 || a->eps < 0.0 ||
        (a->decoupled != 0 && a->decoupled != 1))
        return EFUNC_ERR_ARG;
    return EFUNC_OK;
}

// ------------------------------------------------------- ablation variants

constexpr int kVariantNV[4] = {1, 4, 10, 20};

bool variant_ok(const efunc_variant *v)
{
    return v && v->sets >= 1 && v->sets <= 3 && v->degree >= 0 && v->degree <= 3 &&
           (v->learn_scale == 0 || v->learn_scale == 1);
}

int variant_channels_of(const efunc_variant *v)
{
    const int ns = (v->sets & 1) + ((v->sets >> 1) & 1);
    return ((v->sets & 2) ? 3 : 0) + v->learn_scale * ns + kVariantNV[v->degree] * ns;
}

Layout variant_layout(const efunc_grid *g, const efunc_variant *v, int64_t J, bool two_sort_buffers = false)
{
    return make_layout(g->R, J, variant_key_records(v->sets, v->degree), variant_channels_of(v), two_sort_buffers);
}

efunc_status check_variant_workspace(const efunc_grid *g, const efunc_variant *v, int64_t J, const void *ws,
                                     size_t ws_bytes)
{
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u)) return EFUNC_ERR_WORKSPACE;
    if (ws_bytes < variant_layout(g, v, J).total) return EFUNC_ERR_WORKSPACE;
    return EFUNC_OK;
}

VariantArgs variant_args(const Views &vw, const efunc_grid *g, const efunc_variant *v, const float *params)
{
    VariantArgs a{};
    a.sets = v->sets;
    a.deg = v->degree;
    a.learn = v->learn_scale;
    a.channels = variant_channels_of(v);
    a.params = params;
    a.log_beta0 = (double)g->log_beta0;
    a.keys = vw.keys();
    a.R = g->R;
    a.sorted = vw.sorted();
    a.perm = vw.perm();
    a.items = vw.items();
    a.ctrl = vw.ctrl();
    return a;
}

// ---------------------------------------------- cosine-series decomposition

bool bands_ok(int32_t B) { return B >= 1 && B <= kMaxBands; }

Layout cosine_layout(const efunc_grid *g, int32_t B, int64_t J, bool two_sort_buffers = false)
{
    return make_layout(g->R, J, 2 * B, 5 * B, two_sort_buffers);
}

efunc_status check_cosine_workspace(const efunc_grid *g, int32_t B, int64_t J, const void *ws, size_t ws_bytes)
{
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u)) return EFUNC_ERR_WORKSPACE;
    if (ws_bytes < cosine_layout(g, B, J).total) return EFUNC_ERR_WORKSPACE;
    return EFUNC_OK;
}

CosineArgs cosine_args(const Views &vw, const efunc_grid *g, int32_t B, const float *params)
{
    CosineArgs a{};
    a.B = B;
    a.params = params;
    a.log_beta0 = (double)g->log_beta0;
    a.keys = vw.keys();
    a.R = g->R;
    a.sorted = vw.sorted();
    a.perm = vw.perm();
    a.items = vw.items();
    a.ctrl = vw.ctrl();
    return a;
}

AdamArgs adam_args(const efunc_adam *ad, int64_t n, float *p, float *g, float *m, float *v, int64_t step)
{
    AdamArgs a{};
    a.p = p; a.g = g; a.m = m; a.v = v;
    a.n = n;
    a.beta1 = (float)ad->beta1;
    a.one_minus_beta1 = (float)(1.0 - ad->beta1);
    a.beta2 = (float)ad->beta2;
    a.one_minus_beta2 = (float)(1.0 - ad->beta2);
    a.eps = (float)ad->eps;
    a.wd = (float)ad->weight_decay;
    a.decay = (float)(1.0 - ad->lr * ad->weight_decay);
    a.decoupled = ad->decoupled;
    const double bc1 = 1.0 - pow(ad->beta1, (double)step);
    const double bc2 = 1.0 - pow(ad->beta2, (double)step);
    a.step_size = (float)(ad->lr / bc1);
    a.inv_sqrt_bc2 = (float)(1.0 / sqrt(bc2));
    return a;
}

// efunc_fit with the sort of batch s+1 (on the library's sort stream, into
// the second sort buffer) overlapped with the fused kernel and Adam of batch
// s on the caller's stream.  The fused kernel's persistent grid leaves one
// sort block's registers free on every SM so the two run side by side.
// Events order the buffers: sorted[b] (sort done) before the fused kernel
// that reads buffer b; consumed[b] (Adam of that step done, it reads the loss
// sums in buffer b's control block) before the next sort into b; packed (the
// key pack of step s done) before the sort of s+1, so that the sort starts
// together with the fused kernel instead of ahead of it (started earlier it
// runs at full speed and takes memory bandwidth from the fused kernel's
// first items; started with it, it trickles along on its one block per SM).
efunc_status fit_pipelined(const efunc_grid *grid, const efunc_adam *adam, int32_t loss, float eikonal_weight,
                           float *params, float *m, float *v, const float *qo, int64_t J, int32_t n_batches,
                           int32_t steps, int64_t step0, float *stats, void *workspace, cudaStream_t s)
{
    const int R = grid->R;
    Views vw{make_layout(R, J, kKeyRecords, kSlots, true), static_cast<char *>(workspace)};
    const bool q_host = is_host_pointer(qo);
    const bool stats_host = stats && is_host_pointer(stats);
    const int64_t n = (int64_t)R * R * R * kSlots;
    float *grad = vw.grad();
    CopyPipe *pipe = nullptr;
    if (copy_pipe(&pipe) != cudaSuccess) return cuda_fail();
    std::lock_guard<std::mutex> pipe_lock(pipe->mu);   // fits on one device enqueue one at a time
    cudaStream_t ss = pipe->sort_stream;
    const size_t batch_bytes = (size_t)J * 16;
    auto batch = [&](int32_t it) { return qo + (size_t)(it % n_batches) * (size_t)J * 4; };
    const bool eik = eikonal_weight > 0.f;
    const int grid_blocks = fused_fit_grid_size(eik, true);
    const int gmax = eik ? 0 : fit_group_max(vw.L, J);

    if (cudaMemsetAsync(grad, 0, (size_t)n * 4, s) != cudaSuccess) return cuda_fail();
    // both sort buffers (and staging buffers) are free once the caller's earlier work is done
    for (int b = 0; b < 2; ++b) {
        if (cudaEventRecord(pipe->consumed[b], s) != cudaSuccess) return cuda_fail();
        if (q_host && cudaEventRecord(pipe->freed[b], s) != cudaSuccess) return cuda_fail();
    }
    auto issue_sort = [&](int32_t k) -> bool {
        const int b = k & 1;
        const float *src = batch(k);
        if (q_host) {
            if (cudaStreamWaitEvent(pipe->stream, pipe->freed[b], 0) != cudaSuccess ||
                cudaMemcpyAsync(vw.stage(b, J), src, batch_bytes, cudaMemcpyHostToDevice, pipe->stream) !=
                    cudaSuccess ||
                cudaEventRecord(pipe->copied[b], pipe->stream) != cudaSuccess ||
                cudaStreamWaitEvent(ss, pipe->copied[b], 0) != cudaSuccess)
                return false;
            src = reinterpret_cast<const float *>(vw.stage(b, J));
        }
        if (cudaStreamWaitEvent(ss, pipe->consumed[b], 0) != cudaSuccess) return false;
        // one sort block per SM: the default kernel's steps are long enough to
        // hide it, and more sort traffic slows the kernel beside it
        if (sort_into_buf(sort_buf(vw, b), vw.L, R, src, J, 4, ss, 1, gmax) != cudaSuccess) return false;
        if (q_host && cudaEventRecord(pipe->freed[b], ss) != cudaSuccess) return false;
        return cudaEventRecord(pipe->sorted[b], ss) == cudaSuccess;
    };

    if (!issue_sort(0)) return cuda_fail();
    for (int32_t it = 0; it < steps; ++it) {
        const int b = it & 1;
        const SortBuf sb = sort_buf(vw, b);
        if (cudaStreamWaitEvent(s, pipe->sorted[b], 0) != cudaSuccess) return cuda_fail();
        if (pack_keys(vw, grid, params, s) != cudaSuccess) return cuda_fail();
        // the next sort starts once this step's fused kernel is about to start
        if (it + 1 < steps) {
            if (cudaEventRecord(pipe->packed, s) != cudaSuccess ||
                cudaStreamWaitEvent(ss, pipe->packed, 0) != cudaSuccess || !issue_sort(it + 1))
                return cuda_fail();
        }
        FusedArgs f = fused_args(vw, grid);
        f.sorted = sb.sorted;
        f.items = sb.items;
        f.ctrl = sb.ctrl;
        f.perm = nullptr;
        f.grad = grad;
        f.loss = loss;
        f.inv_J = (float)(1.0 / (double)J);
        f.eik_weight = eikonal_weight;
        if (launch_fused_fit(f, eik, grid_blocks, s) != cudaSuccess) return cuda_fail();
        if (gmax && launch_grouped(f, BatchArgs{}, sb.gtop, false, s) != cudaSuccess) return cuda_fail();
        float *stats_dev = reinterpret_cast<float *>(sb.ctrl) + 16;
        AdamArgs a = adam_args(adam, n, params, grad, m, v, step0 + it + 1);
        a.ctrl = sb.ctrl;
        a.inv_J = f.inv_J;
        a.stats = stats ? (stats_host ? stats_dev : stats + 2 * (size_t)it) : nullptr;
        if (launch_adam(a, s) != cudaSuccess) return cuda_fail();
        if (stats_host && cudaMemcpyAsync(stats + 2 * (size_t)it, stats_dev, 8, cudaMemcpyDeviceToHost, s) !=
                              cudaSuccess)
            return cuda_fail();
        if (cudaEventRecord(pipe->consumed[b], s) != cudaSuccess) return cuda_fail();
    }
    if (stats_host && cudaStreamSynchronize(s) != cudaSuccess) return cuda_fail();
    return EFUNC_OK;
}

// fit_pipelined's schedule replayed from a CUDA graph.  One period of
// P = lcm(2, n_batches) steps repeats exactly (sort buffer it & 1, batch
// it % n_batches, the same kernels and arguments) except for Adam's step
// number, which lives in device memory (AdamClock in the first sort
// buffer's control block, past the loss sums and the statistics slot).  The
// call seeds the clock, sorts batch 0, captures one period on a library
// stream (its last step sorts batch P = batch 0 into buffer 0 for the next
// replay), launches the graph on the caller's stream (steps - 1) / P times
// and issues the remaining 1..P steps one by one.
// Inside the captured period the first step waits for nothing: the sort of
// its batch ran before the graph launch on the same stream (or inside the
// previous replay), and both sort buffers are free when a replay starts.
efunc_status fit_graph(const efunc_grid *grid, const efunc_adam *adam, int32_t loss, float eikonal_weight,
                       float *params, float *m, float *v, const float *qo, int64_t J, int32_t n_batches,
                       int32_t steps, int64_t step0, float *stats, void *workspace, cudaStream_t s)
{
    const int R = grid->R;
    Views vw{make_layout(R, J, kKeyRecords, kSlots, true), static_cast<char *>(workspace)};
    const int64_t n = (int64_t)R * R * R * kSlots;
    float *grad = vw.grad();
    CopyPipe *pipe = nullptr;
    if (copy_pipe(&pipe) != cudaSuccess) return cuda_fail();
    std::lock_guard<std::mutex> pipe_lock(pipe->mu);   // fits on one device enqueue one at a time
    cudaStream_t ss = pipe->sort_stream;
    auto batch = [&](int32_t it) { return qo + (size_t)(it % n_batches) * (size_t)J * 4; };
    const bool eik = eikonal_weight > 0.f;
    const int grid_blocks = fused_fit_grid_size(eik, true);
    const int gmax = eik ? 0 : fit_group_max(vw.L, J);
    const int32_t period = (n_batches % 2 == 0) ? n_batches : 2 * n_batches;
    static_assert(sizeof(Ctrl) <= 64 && sizeof(AdamClock) <= 128, "control block layout");
    AdamClock *clk = reinterpret_cast<AdamClock *>(reinterpret_cast<char *>(vw.ctrl()) + 128);
    const AdamArgs base = adam_args(adam, n, params, grad, m, v, step0 + 1);

    if (cudaMemsetAsync(grad, 0, (size_t)n * 4, s) != cudaSuccess) return cuda_fail();
    if (launch_adam_clock_seed(clk, adam_clock_init(adam->lr, adam->beta1, adam->beta2, step0 + 1), s) !=
        cudaSuccess)
        return cuda_fail();
    for (int b = 0; b < 2; ++b)
        if (cudaEventRecord(pipe->consumed[b], s) != cudaSuccess) return cuda_fail();
    auto issue_sort = [&](int32_t k, bool wait_consumed) -> bool {
        const int b = k & 1;
        if (wait_consumed && cudaStreamWaitEvent(ss, pipe->consumed[b], 0) != cudaSuccess) return false;
        if (sort_into_buf(sort_buf(vw, b), vw.L, R, batch(k), J, 4, ss, 1, gmax) != cudaSuccess) return false;
        return cudaEventRecord(pipe->sorted[b], ss) == cudaSuccess;
    };
    // one step on stream st; `head` marks the first step of a captured period
    auto issue_step = [&](int32_t it, bool head, bool sort_next, cudaStream_t st) -> bool {
        const int b = it & 1;
        const SortBuf sb = sort_buf(vw, b);
        if (!head && cudaStreamWaitEvent(st, pipe->sorted[b], 0) != cudaSuccess) return false;
        if (pack_keys(vw, grid, params, st) != cudaSuccess) return false;
        if (sort_next) {
            if (cudaEventRecord(pipe->packed, st) != cudaSuccess ||
                cudaStreamWaitEvent(ss, pipe->packed, 0) != cudaSuccess || !issue_sort(it + 1, !head))
                return false;
        }
        FusedArgs f = fused_args(vw, grid);
        f.sorted = sb.sorted;
        f.items = sb.items;
        f.ctrl = sb.ctrl;
        f.perm = nullptr;
        f.grad = grad;
        f.loss = loss;
        f.inv_J = (float)(1.0 / (double)J);
        f.eik_weight = eikonal_weight;
        if (launch_fused_fit(f, eik, grid_blocks, st) != cudaSuccess) return false;
        if (gmax && launch_grouped(f, BatchArgs{}, sb.gtop, false, st) != cudaSuccess) return false;
        AdamArgs a = base;
        a.ctrl = sb.ctrl;
        a.inv_J = f.inv_J;
        a.stats = stats;
        if (launch_adam_clocked(a, clk, st) != cudaSuccess) return false;
        return cudaEventRecord(pipe->consumed[b], st) == cudaSuccess;
    };

    if (!issue_sort(0, true) || cudaStreamWaitEvent(s, pipe->sorted[0], 0) != cudaSuccess) return cuda_fail();
    const int32_t replays = (steps - 1) / period;
    if (replays > 0) {
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        cudaStream_t cs = pipe->capture_stream;
        if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return cuda_fail();
        g_captured = 0;
        g_in_capture = true;
        bool ok = true;
        for (int32_t it = 0; it < period && ok; ++it) ok = issue_step(it, it == 0, true, cs);
        // the sort stream rejoins the capturing stream
        ok = ok && cudaEventRecord(pipe->joined, ss) == cudaSuccess &&
             cudaStreamWaitEvent(cs, pipe->joined, 0) == cudaSuccess;
        g_in_capture = false;
        const cudaError_t ce = cudaStreamEndCapture(cs, &graph);
        const int64_t captured = g_captured;
        cudaError_t e = ce;
        if (ok && e == cudaSuccess && graph) e = cudaGraphInstantiate(&exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        for (int32_t r = 0; ok && exec && r < replays && e == cudaSuccess; ++r) e = cudaGraphLaunch(exec, s);
        if (exec) cudaGraphExecDestroy(exec);   // deferred by the driver until the launches complete
        // the events recorded during the capture stand for graph nodes, not
        // for work on a stream: record them again after the replays, on the
        // caller's stream, before anything outside the graph waits for them
        for (cudaEvent_t ev : {pipe->sorted[0], pipe->sorted[1], pipe->consumed[0], pipe->consumed[1], pipe->packed,
                               pipe->joined})
            if (cudaEventRecord(ev, s) != cudaSuccess && e == cudaSuccess) e = cudaErrorUnknown;
        if (!ok || e != cudaSuccess) return cuda_fail(ok ? e : cudaSuccess);
        std::lock_guard<std::mutex> lk(g_prof_mu);
        g_launches += captured * replays;
    }
    for (int32_t it = replays * period; it < steps; ++it)
        if (!issue_step(it, false, it + 1 < steps, s)) return cuda_fail();
    return EFUNC_OK;
}

// The sort-ahead schedule of fit_pipelined for device batches, shared by the
// variant and cosine fits: pack(stream) issues a step's key pack,
// compute(step, sort buffer, stream) its fused kernel and Adam step.
template <class Pack, class Compute>
efunc_status pipelined_device_fit(const Views &vw, int R, const float *qo, int64_t J, int32_t n_batches,
                                  int32_t steps, cudaStream_t s, Pack pack, Compute compute)
{
    CopyPipe *pipe = nullptr;
    if (copy_pipe(&pipe) != cudaSuccess) return cuda_fail();
    std::lock_guard<std::mutex> pipe_lock(pipe->mu);   // fits on one device enqueue one at a time
    cudaStream_t ss = pipe->sort_stream;
    auto batch = [&](int32_t it) { return qo + (size_t)(it % n_batches) * (size_t)J * 4; };
    for (int b = 0; b < 2; ++b)
        if (cudaEventRecord(pipe->consumed[b], s) != cudaSuccess) return cuda_fail();
    auto issue_sort = [&](int32_t k) -> bool {
        const int b = k & 1;
        if (cudaStreamWaitEvent(ss, pipe->consumed[b], 0) != cudaSuccess) return false;
        // two sort blocks per SM (the room the persistent grids leave): the
        // variant and cosine kernels are shorter than the default one
        if (sort_into_buf(sort_buf(vw, b), vw.L, R, batch(k), J, 4, ss, 2) != cudaSuccess) return false;
        return cudaEventRecord(pipe->sorted[b], ss) == cudaSuccess;
    };
    if (!issue_sort(0)) return cuda_fail();
    for (int32_t it = 0; it < steps; ++it) {
        const int b = it & 1;
        if (cudaStreamWaitEvent(s, pipe->sorted[b], 0) != cudaSuccess) return cuda_fail();
        if (pack(s) != cudaSuccess) return cuda_fail();
        if (it + 1 < steps) {
            if (cudaEventRecord(pipe->packed, s) != cudaSuccess ||
                cudaStreamWaitEvent(ss, pipe->packed, 0) != cudaSuccess || !issue_sort(it + 1))
                return cuda_fail();
        }
        if (compute(it, sort_buf(vw, b), s) != cudaSuccess) return cuda_fail();
        if (cudaEventRecord(pipe->consumed[b], s) != cudaSuccess) return cuda_fail();
    }
    return EFUNC_OK;
}

}  // namespace

extern "C" {

int64_t efunc_param_count(int32_t R)
{
    if (R < 1 || R > kMaxR) return -1;
    return (int64_t)R * R * R * kSlots;
}

float efunc_default_log_beta0(int32_t R)
{
    if (R < 1) return NAN;
    return (float)(7.0 + 2.0 * log((double)R / 32.0));
}

const char *efunc_status_str(efunc_status s)
{
    switch (s) {
    case EFUNC_OK: return "ok";
    case EFUNC_ERR_ARG: return "invalid argument";
    case EFUNC_ERR_CUDA: return "CUDA runtime error";
    case EFUNC_ERR_IO: return "checkpoint file missing, unwritable, short or corrupt";
    case EFUNC_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
    case EFUNC_ERR_NONFINITE: return "non-finite hyper-parameter";
    case EFUNC_ERR_UNSUPPORTED: return "unsupported configuration";
    case EFUNC_ERR_TIMEOUT: return "a bounded wait inside a kernel ran out";
    }
    return "unknown status";
}

size_t efunc_workspace_bytes(const efunc_grid *grid, int64_t J)
{
    if (!grid_ok(grid) || J < 0 || J > kMaxJ) return 0;
    return make_layout(grid->R, J).total;
}

size_t efunc_eval_workspace_bytes(const efunc_grid *grid, int64_t J)
{
    if (!grid_ok(grid) || J < 0 || J > kMaxJ) return 0;
    return eval_layout(grid->R, J).total;
}

size_t efunc_fit_workspace_bytes(const efunc_grid *grid, int64_t J)
{
    if (!grid_ok(grid) || J < 0 || J > kMaxJ) return 0;
    return make_layout(grid->R, J, kKeyRecords, kSlots, true).total;
}

efunc_status efunc_cell_sort(const efunc_grid *grid, const float *q, int64_t J, int32_t q_stride, float *q_sorted,
                             int32_t *perm, void *workspace, size_t workspace_bytes, efunc_stream_t stream)
{
    efunc_status st = check_grid(grid);
    if (st) return st;
    if (J < 0 || J > kMaxJ || (q_stride != 3 && q_stride != 4)) return EFUNC_ERR_ARG;
    if (J == 0) return EFUNC_OK;
    if (!q || !q_sorted || !perm || (reinterpret_cast<uintptr_t>(q_sorted) & 15u)) return EFUNC_ERR_ARG;
    if ((st = check_workspace(grid, J, workspace, workspace_bytes))) return st;
    Views v{eval_layout(grid->R, J), static_cast<char *>(workspace)};
    return cuda_status(sort_into(v, grid->R, q, J, q_stride, reinterpret_cast<float4 *>(q_sorted), perm,
                                 (cudaStream_t)stream));
}

efunc_status efunc_forward(const efunc_grid *grid, const float *params, const float *q, int64_t J, int32_t q_stride,
                           float *O, float *lse, float *dOdq, void *workspace, size_t workspace_bytes,
                           efunc_stream_t stream)
{
    efunc_status st = check_grid(grid);
    if (st) return st;
    if (J < 0 || J > kMaxJ || (q_stride != 3 && q_stride != 4) || !params) return EFUNC_ERR_ARG;
    if (J == 0) return EFUNC_OK;
    if (!q || !O) return EFUNC_ERR_ARG;
    if ((st = check_workspace(grid, J, workspace, workspace_bytes))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    Views v{eval_layout(grid->R, J), static_cast<char *>(workspace)};
    cudaError_t e = sort_into(v, grid->R, q, J, q_stride, v.sorted(), v.perm(), s);
    if (e == cudaSuccess) e = pack_keys(v, grid, params, s);
    if (e != cudaSuccess) return cuda_fail();
    FusedArgs f = fused_args(v, grid);
    f.O = O;
    f.lse = lse;
    f.dq = dOdq;
    return cuda_status(launch_forward(f, dOdq != nullptr, fused_grid_size(), s));
}

efunc_status efunc_backward(const efunc_grid *grid, const float *params, const float *q, int64_t J,
                            int32_t q_stride, const float *gO, float *grad, float *gq, void *workspace,
                            size_t workspace_bytes, efunc_stream_t stream)
{
    efunc_status st = check_grid(grid);
    if (st) return st;
    if (J < 0 || J > kMaxJ || (q_stride != 3 && q_stride != 4) || !params || !grad) return EFUNC_ERR_ARG;
    if (J == 0) return EFUNC_OK;
    if (!q || !gO) return EFUNC_ERR_ARG;
    if ((st = check_workspace(grid, J, workspace, workspace_bytes))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    Views v{eval_layout(grid->R, J), static_cast<char *>(workspace)};
    cudaError_t e = sort_into(v, grid->R, q, J, q_stride, v.sorted(), v.perm(), s);
    if (e == cudaSuccess) e = pack_keys(v, grid, params, s);
    if (e != cudaSuccess) return cuda_fail();
    FusedArgs f = fused_args(v, grid);
    f.gO = gO;
    f.grad = grad;
    f.gq = gq;
    return cuda_status(launch_fused_backward(f, gq != nullptr, false, fused_grid_size(), s));
}

efunc_status efunc_backward_grad(const efunc_grid *grid, const float *params, const float *q, int64_t J,
                                 int32_t q_stride, const float *gO, const float *gG, float *grad, void *workspace,
                                 size_t workspace_bytes, efunc_stream_t stream)
{
    efunc_status st = check_grid(grid);
    if (st) return st;
    if (J < 0 || J > kMaxJ || (q_stride != 3 && q_stride != 4) || !params || !grad) return EFUNC_ERR_ARG;
    if (J == 0) return EFUNC_OK;
    if (!q || (!gO && !gG)) return EFUNC_ERR_ARG;
    if ((st = check_workspace(grid, J, workspace, workspace_bytes))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    Views v{eval_layout(grid->R, J), static_cast<char *>(workspace)};
    cudaError_t e = sort_into(v, grid->R, q, J, q_stride, v.sorted(), v.perm(), s);
    if (e == cudaSuccess) e = pack_keys(v, grid, params, s);
    if (e != cudaSuccess) return cuda_fail();
    FusedArgs f = fused_args(v, grid);
    f.gO = gO;
    f.gG = gG;
    f.grad = grad;
    if (!gG) return cuda_status(launch_fused_backward(f, false, false, fused_grid_size(), s));
    return cuda_status(launch_fused_backward(f, false, true, fused_grid_size(), s));
}

efunc_status efunc_eval_loss(const efunc_grid *grid, const float *params, const float *qo, int64_t J, float *out,
                             void *workspace, size_t workspace_bytes, efunc_stream_t stream)
{
    efunc_status st = check_grid(grid);
    if (st) return st;
    if (J < 1 || J > kMaxJ || !params || !qo || !out) return EFUNC_ERR_ARG;
    if ((st = check_workspace(grid, J, workspace, workspace_bytes))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    Views v{eval_layout(grid->R, J), static_cast<char *>(workspace)};
    // a sum over queries: no permutation back to the caller's order
    cudaError_t e = sort_into(v, grid->R, qo, J, 4, v.sorted(), nullptr, s);
    if (e == cudaSuccess) e = pack_keys(v, grid, params, s);
    if (e != cudaSuccess) return cuda_fail();
    FusedArgs f = fused_args(v, grid);
    f.perm = nullptr;
    if ((e = launch_fused_eval(f, fused_grid_size(), s)) != cudaSuccess) return cuda_fail(e);
    return cuda_status(launch_eval_finish(v.ctrl(), 1.0 / (double)J, out, s));
}

size_t efunc_f64_workspace_bytes(const efunc_grid *grid, int64_t J)
{
    if (!grid_ok(grid) || J < 0 || J > kMaxJ) return 0;
    return layout64(grid->R, J).total;
}

}  // extern "C"

namespace {

// The FP64 forward / backward: round the queries to FP32 rows (the windows
// are chosen from them, as in the FP32 path), sort those rows with the
// permutation, gather the FP64 rows in sorted order, pack FP64 key records,
// then run the FP64 instantiation of the fused kernel.
efunc_status run_f64(const efunc_grid *grid, const double *params, const double *q, int64_t J, int32_t q_stride,
                     double *O, double *lse, double *dOdq, const double *gO, double *grad, double *gq,
                     void *workspace, size_t workspace_bytes, cudaStream_t s, bool backward)
{
    const Layout64 X = layout64(grid->R, J);
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255u) || workspace_bytes < X.total)
        return EFUNC_ERR_WORKSPACE;
    char *base = static_cast<char *>(workspace);
    Views v{X.L, base};
    float4 *rows32 = reinterpret_cast<float4 *>(base + X.rows32);
    Double4 *rows64 = reinterpret_cast<Double4 *>(base + X.rows64);
    Double4 *keys64 = reinterpret_cast<Double4 *>(base + X.keys64);
    cudaError_t e = launch_round_queries(q, J, q_stride, rows32, s);
    if (e == cudaSuccess) e = sort_into(v, grid->R, reinterpret_cast<const float *>(rows32), J, 4, v.sorted(),
                                        v.perm(), s);
    if (e == cudaSuccess) e = launch_gather_queries64(q, J, q_stride, v.perm(), rows64, s);
    PackArgs64 pk{};
    pk.params = params;
    pk.keys = keys64;
    pk.R = grid->R;
    pk.log_beta0 = (double)grid->log_beta0;
    if (e == cudaSuccess) e = launch_pack_keys64(pk, s);
    if (e != cudaSuccess) return cuda_fail(e);
    FusedArgs64 f{};
    f.keys = keys64;
    f.R = grid->R;
    f.sorted = rows64;
    f.perm = v.perm();
    f.items = v.items();
    f.ctrl = v.ctrl();
    f.O = O;
    f.lse = lse;
    f.dq = dOdq;
    f.gO = gO;
    f.grad = grad;
    f.gq = gq;
    if (backward) return cuda_status(launch_fused_backward64(f, gq != nullptr, fused_grid_size64(), s));
    return cuda_status(launch_forward64(f, dOdq != nullptr, fused_grid_size64(), s));
}

}  // namespace

extern "C" {

efunc_status efunc_forward_f64(const efunc_grid *grid, const double *params, const double *q, int64_t J,
                               int32_t q_stride, double *O, double *lse, double *dOdq, void *workspace,
                               size_t workspace_bytes, efunc_stream_t stream)
{
    efunc_status st = check_grid(grid);
    if (st) return st;
    if (J < 0 || J > kMaxJ || (q_stride != 3 && q_stride != 4) || !params) return EFUNC_ERR_ARG;
    if (J == 0) return EFUNC_OK;
    if (!q || !O) return EFUNC_ERR_ARG;
    return run_f64(grid, params, q, J, q_stride, O, lse, dOdq, nullptr, nullptr, nullptr, workspace,
                   workspace_bytes, (cudaStream_t)stream, false);
}

efunc_status efunc_backward_f64(const efunc_grid *grid, const double *params, const double *q, int64_t J,
                                int32_t q_stride, const double *gO, double *grad, double *gq, void *workspace,
                                size_t workspace_bytes, efunc_stream_t stream)
{
    efunc_status st = check_grid(grid);
    if (st) return st;
    if (J < 0 || J > kMaxJ || (q_stride != 3 && q_stride != 4) || !params || !grad) return EFUNC_ERR_ARG;
    if (J == 0) return EFUNC_OK;
    if (!q || !gO) return EFUNC_ERR_ARG;
    return run_f64(grid, params, q, J, q_stride, nullptr, nullptr, nullptr, gO, grad, gq, workspace,
                   workspace_bytes, (cudaStream_t)stream, true);
}

efunc_status efunc_adam_step(const efunc_adam *adam, int64_t n, float *params, float *grad, float *m, float *v,
                             int64_t step, efunc_stream_t stream)
{
    efunc_status st = check_adam(adam);
    if (st) return st;
    if (n < 0 || step < 1) return EFUNC_ERR_ARG;
    if (n == 0) return EFUNC_OK;
    if (!params || !grad || !m || !v) return EFUNC_ERR_ARG;
    AdamArgs a = adam_args(adam, n, params, grad, m, v, step);
    return cuda_status(launch_adam(a, (cudaStream_t)stream));
}

efunc_status efunc_fit(const efunc_grid *grid, const efunc_adam *adam, int32_t loss, float eikonal_weight,
                       float *params, float *m, float *v, const float *qo, int64_t J, int32_t n_batches, int32_t steps,
                       int64_t step0, float *stats, void *workspace, size_t workspace_bytes, efunc_stream_t stream)
{
    efunc_status st = check_grid(grid);
    if (st) return st;
    if ((st = check_adam(adam))) return st;
    if (loss != EFUNC_LOSS_L1 && loss != EFUNC_LOSS_MSE) return EFUNC_ERR_ARG;
    if (!isfinite(eikonal_weight)) return EFUNC_ERR_NONFINITE;
    if (eikonal_weight < 0.f) return EFUNC_ERR_ARG;
    if (J < 1 || J > kMaxJ || n_batches < 1 || steps < 0 || step0 < 0) return EFUNC_ERR_ARG;
    if (!params || !m || !v || !qo) return EFUNC_ERR_ARG;
    if ((st = check_workspace(grid, J, workspace, workspace_bytes, true))) return st;
    if (steps == 0) return EFUNC_OK;
    if (workspace_bytes >= make_layout(grid->R, J, kKeyRecords, kSlots, true).total)
        return fit_pipelined(grid, adam, loss, eikonal_weight, params, m, v, qo, J, n_batches, steps, step0, stats,
                             workspace, (cudaStream_t)stream);
    cudaStream_t s = (cudaStream_t)stream;
    Views vw{make_layout(grid->R, J), static_cast<char *>(workspace)};
    const bool q_host = is_host_pointer(qo);
    const bool stats_host = stats && is_host_pointer(stats);
    const int64_t n = efunc_param_count(grid->R);
    float *grad = vw.grad();
    // scratch for the per-step statistics when the caller's array is on the host
    float *stats_dev = reinterpret_cast<float *>(vw.ctrl()) + 16;
    static_assert(sizeof(Ctrl) <= 64, "control block must leave room for the statistics slot");

    cudaError_t e = cudaMemsetAsync(grad, 0, (size_t)n * 4, s);
    if (e != cudaSuccess) return cuda_fail();
    const int grid_blocks = fused_grid_size();
    const int gmax = eikonal_weight > 0.f ? 0 : fit_group_max(vw.L, J);
    const size_t batch_bytes = (size_t)J * 16;
    auto batch = [&](int32_t it) { return qo + (size_t)(it % n_batches) * (size_t)J * 4; };

    // Host batches: copies run on the library's copy stream into two staging
    // buffers, batch it+1 landing while batch it is computed.
    CopyPipe *pipe = nullptr;
    std::unique_lock<std::mutex> pipe_lock;
    if (q_host) {
        if (copy_pipe(&pipe) != cudaSuccess) return cuda_fail();
        pipe_lock = std::unique_lock<std::mutex>(pipe->mu);   // fits on one device enqueue one at a time
        for (int b = 0; b < 2; ++b)   // buffers free once the caller's earlier work is done
            if (cudaEventRecord(pipe->freed[b], s) != cudaSuccess) return cuda_fail();
        if (cudaStreamWaitEvent(pipe->stream, pipe->freed[0], 0) != cudaSuccess ||
            cudaMemcpyAsync(vw.stage(0, J), batch(0), batch_bytes, cudaMemcpyHostToDevice, pipe->stream) != cudaSuccess ||
            cudaEventRecord(pipe->copied[0], pipe->stream) != cudaSuccess)
            return cuda_fail();
    }
    for (int32_t it = 0; it < steps; ++it) {
        const int b = it & 1;
        const float *qdev = batch(it);
        if (q_host) {
            if (it + 1 < steps &&
                (cudaStreamWaitEvent(pipe->stream, pipe->freed[b ^ 1], 0) != cudaSuccess ||
                 cudaMemcpyAsync(vw.stage(b ^ 1, J), batch(it + 1), batch_bytes, cudaMemcpyHostToDevice,
                                 pipe->stream) != cudaSuccess ||
                 cudaEventRecord(pipe->copied[b ^ 1], pipe->stream) != cudaSuccess))
                return cuda_fail();
            if (cudaStreamWaitEvent(s, pipe->copied[b], 0) != cudaSuccess) return cuda_fail();
            qdev = reinterpret_cast<const float *>(vw.stage(b, J));
        }
        // the fit reduces over queries: no permutation back to the caller's order
        e = sort_into(vw, grid->R, qdev, J, 4, vw.sorted(), nullptr, s, gmax);
        if (e == cudaSuccess && q_host) e = cudaEventRecord(pipe->freed[b], s);   // staging buffer consumed
        if (e == cudaSuccess) e = pack_keys(vw, grid, params, s);
        if (e != cudaSuccess) return cuda_fail();
        FusedArgs f = fused_args(vw, grid);
        f.grad = grad;
        f.loss = loss;
        f.inv_J = (float)(1.0 / (double)J);
        f.eik_weight = eikonal_weight;
        e = launch_fused_fit(f, eikonal_weight > 0.f, grid_blocks, s);
        if (e == cudaSuccess && gmax) e = launch_grouped(f, BatchArgs{}, vw.items() + vw.L.max_items - 1, false, s);
        if (e != cudaSuccess) return cuda_fail();
        AdamArgs a = adam_args(adam, n, params, grad, m, v, step0 + it + 1);
        a.ctrl = vw.ctrl();
        a.inv_J = f.inv_J;
        a.stats = stats ? (stats_host ? stats_dev : stats + 2 * (size_t)it) : nullptr;
        e = launch_adam(a, s);
        if (e != cudaSuccess) return cuda_fail();
        if (stats_host) {
            e = cudaMemcpyAsync(stats + 2 * (size_t)it, stats_dev, 8, cudaMemcpyDeviceToHost, s);
            if (e != cudaSuccess) return cuda_fail();
        }
    }
    if (stats_host && cudaStreamSynchronize(s) != cudaSuccess) return cuda_fail();
    return EFUNC_OK;
}

efunc_status efunc_fit_graph(const efunc_grid *grid, const efunc_adam *adam, int32_t loss, float eikonal_weight,
                             float *params, float *m, float *v, const float *qo, int64_t J, int32_t n_batches,
                             int32_t steps, int64_t step0, float *stats, void *workspace, size_t workspace_bytes,
                             efunc_stream_t stream)
{
    efunc_status st = check_grid(grid);
    if (st) return st;
    if ((st = check_adam(adam))) return st;
    if (loss != EFUNC_LOSS_L1 && loss != EFUNC_LOSS_MSE) return EFUNC_ERR_ARG;
    if (!isfinite(eikonal_weight)) return EFUNC_ERR_NONFINITE;
    if (eikonal_weight < 0.f) return EFUNC_ERR_ARG;
    if (J < 1 || J > kMaxJ || n_batches < 1 || n_batches > kMaxGraphBatches || steps < 0 || step0 < 0)
        return EFUNC_ERR_ARG;
    if (!params || !m || !v || !qo) return EFUNC_ERR_ARG;
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255u) ||
        workspace_bytes < make_layout(grid->R, J, kKeyRecords, kSlots, true).total)
        return EFUNC_ERR_WORKSPACE;
    if (steps == 0) return EFUNC_OK;
    if (is_host_pointer(qo) || (stats && is_host_pointer(stats))) return EFUNC_ERR_ARG;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing((cudaStream_t)stream, &cs) != cudaSuccess) return cuda_fail();
    if (cs != cudaStreamCaptureStatusNone) return EFUNC_ERR_ARG;
    return fit_graph(grid, adam, loss, eikonal_weight, params, m, v, qo, J, n_batches, steps, step0, stats,
                     workspace, (cudaStream_t)stream);
}

efunc_status efunc_mean_shift_init(const efunc_grid *grid, const float *pts, int64_t N, float bandwidth,
                                   float *params, efunc_stream_t stream)
{
    efunc_status st = check_grid(grid);
    if (st) return st;
    if (!isfinite(bandwidth)) return EFUNC_ERR_NONFINITE;
    if (N < 1 || N > kMaxJ || !(bandwidth > 0.f) || !pts || !params) return EFUNC_ERR_ARG;
    MeanShiftArgs a{};
    a.pts = pts;
    a.N = N;
    a.R = grid->R;
    a.sigma = (float)sqrt((double)bandwidth * 1.4426950408889634);
    a.params = params;
    return cuda_status(launch_mean_shift(a, (cudaStream_t)stream));
}

int32_t efunc_variant_channels(const efunc_variant *variant)
{
    if (!variant_ok(variant)) return -1;
    const int ns = (variant->sets & 1) + ((variant->sets >> 1) & 1);
    return ((variant->sets & 2) ? 3 : 0) + variant->learn_scale * ns + kVariantNV[variant->degree] * ns;
}

size_t efunc_variant_workspace_bytes(const efunc_grid *grid, const efunc_variant *variant, int64_t J)
{
    if (!grid_ok(grid) || !variant_ok(variant) || J < 0 || J > kMaxJ) return 0;
    return variant_layout(grid, variant, J, true).total;
}

efunc_status efunc_variant_forward(const efunc_grid *grid, const efunc_variant *variant, const float *params,
                                   const float *q, int64_t J, int32_t q_stride, float *O, float *lse,
                                   void *workspace, size_t workspace_bytes, efunc_stream_t stream)
{
    efunc_status st = check_grid(grid);
    if (st) return st;
    if (!variant_ok(variant)) return EFUNC_ERR_ARG;
    if (J < 0 || J > kMaxJ || (q_stride != 3 && q_stride != 4) || !params) return EFUNC_ERR_ARG;
    if (J == 0) return EFUNC_OK;
    if (!q || !O) return EFUNC_ERR_ARG;
    if ((st = check_variant_workspace(grid, variant, J, workspace, workspace_bytes))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    Views v{variant_layout(grid, variant, J), static_cast<char *>(workspace)};
    cudaError_t e = sort_into(v, grid->R, q, J, q_stride, v.sorted(), v.perm(), s);
    VariantArgs a = variant_args(v, grid, variant, params);
    if (e == cudaSuccess) e = launch_variant_pack(a, s);
    if (e != cudaSuccess) return cuda_fail();
    a.O = O;
    a.lse = lse;
    return cuda_status(launch_variant(a, VAR_FORWARD, s));
}

efunc_status efunc_variant_backward(const efunc_grid *grid, const efunc_variant *variant, const float *params,
                                    const float *q, int64_t J, int32_t q_stride, const float *gO, float *grad,
                                    void *workspace, size_t workspace_bytes, efunc_stream_t stream)
{
    efunc_status st = check_grid(grid);
    if (st) return st;
    if (!variant_ok(variant)) return EFUNC_ERR_ARG;
    if (J < 0 || J > kMaxJ || (q_stride != 3 && q_stride != 4) || !params || !grad) return EFUNC_ERR_ARG;
    if (J == 0) return EFUNC_OK;
    if (!q || !gO) return EFUNC_ERR_ARG;
    if ((st = check_variant_workspace(grid, variant, J, workspace, workspace_bytes))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    Views v{variant_layout(grid, variant, J), static_cast<char *>(workspace)};
    cudaError_t e = sort_into(v, grid->R, q, J, q_stride, v.sorted(), v.perm(), s);
    VariantArgs a = variant_args(v, grid, variant, params);
    if (e == cudaSuccess) e = launch_variant_pack(a, s);
    if (e != cudaSuccess) return cuda_fail();
    a.gO = gO;
    a.grad = grad;
    return cuda_status(launch_variant(a, VAR_BACKWARD, s));
}

efunc_status efunc_variant_fit(const efunc_grid *grid, const efunc_variant *variant, const efunc_adam *adam,
                               int32_t loss, float *params, float *m, float *v, const float *qo, int64_t J,
                               int32_t n_batches, int32_t steps, int64_t step0, float *stats, void *workspace,
                               size_t workspace_bytes, efunc_stream_t stream)
{
    efunc_status st = check_grid(grid);
    if (st) return st;
    if (!variant_ok(variant)) return EFUNC_ERR_ARG;
    if ((st = check_adam(adam))) return st;
    if (loss != EFUNC_LOSS_L1 && loss != EFUNC_LOSS_MSE) return EFUNC_ERR_ARG;
    if (J < 1 || J > kMaxJ || n_batches < 1 || steps < 0 || step0 < 0) return EFUNC_ERR_ARG;
    if (!params || !m || !v || !qo) return EFUNC_ERR_ARG;
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255u) ||
        workspace_bytes < variant_layout(grid, variant, J, true).total)
        return EFUNC_ERR_WORKSPACE;
    if (steps == 0) return EFUNC_OK;
    if (is_host_pointer(qo) || (stats && is_host_pointer(stats))) return EFUNC_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = (int64_t)grid->R * grid->R * grid->R * efunc_variant_channels(variant);
    const float inv_J = (float)(1.0 / (double)J);
    {
        Views vp{variant_layout(grid, variant, J, true), static_cast<char *>(workspace)};
        float *gp = vp.grad();
        if (cudaMemsetAsync(gp, 0, (size_t)n * 4, s) != cudaSuccess) return cuda_fail();
        return pipelined_device_fit(
            vp, grid->R, qo, J, n_batches, steps, s,
            [&](cudaStream_t st) { return launch_variant_pack(variant_args(vp, grid, variant, params), st); },
            [&](int32_t it, const SortBuf &sb, cudaStream_t st) {
                VariantArgs a = variant_args(vp, grid, variant, params);
                a.sorted = sb.sorted;
                a.items = sb.items;
                a.ctrl = sb.ctrl;
                a.perm = nullptr;
                a.grad = gp;
                a.loss = loss;
                a.inv_J = inv_J;
                a.leave_room = 1;
                cudaError_t e = launch_variant(a, VAR_FIT, st);
                if (e != cudaSuccess) return e;
                AdamArgs ad = adam_args(adam, n, params, gp, m, v, step0 + it + 1);
                ad.ctrl = sb.ctrl;
                ad.inv_J = inv_J;
                ad.stats = stats ? stats + 2 * (size_t)it : nullptr;
                return launch_adam(ad, st);
            });
    }
}

size_t efunc_cosine_workspace_bytes(const efunc_grid *grid, int32_t bands, int64_t J)
{
    if (!grid_ok(grid) || !bands_ok(bands) || J < 0 || J > kMaxJ) return 0;
    return cosine_layout(grid, bands, J, true).total;
}

efunc_status efunc_cosine_forward(const efunc_grid *grid, int32_t bands, const float *params, const float *q,
                                  int64_t J, int32_t q_stride, float *S, void *workspace, size_t workspace_bytes,
                                  efunc_stream_t stream)
{
    efunc_status st = check_grid(grid);
    if (st) return st;
    if (!bands_ok(bands)) return EFUNC_ERR_ARG;
    if (J < 0 || J > kMaxJ || (q_stride != 3 && q_stride != 4) || !params) return EFUNC_ERR_ARG;
    if (J == 0) return EFUNC_OK;
    if (!q || !S) return EFUNC_ERR_ARG;
    if ((st = check_cosine_workspace(grid, bands, J, workspace, workspace_bytes))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    Views v{cosine_layout(grid, bands, J), static_cast<char *>(workspace)};
    cudaError_t e = sort_into(v, grid->R, q, J, q_stride, v.sorted(), v.perm(), s);
    CosineArgs a = cosine_args(v, grid, bands, params);
    if (e == cudaSuccess) e = launch_cosine_pack(a, s);
    if (e != cudaSuccess) return cuda_fail();
    a.S = S;
    return cuda_status(launch_cosine(a, VAR_FORWARD, s));
}

efunc_status efunc_cosine_backward(const efunc_grid *grid, int32_t bands, const float *params, const float *q,
                                   int64_t J, int32_t q_stride, const float *gS, float *grad, void *workspace,
                                   size_t workspace_bytes, efunc_stream_t stream)
{
    efunc_status st = check_grid(grid);
    if (st) return st;
    if (!bands_ok(bands)) return EFUNC_ERR_ARG;
    if (J < 0 || J > kMaxJ || (q_stride != 3 && q_stride != 4) || !params || !grad) return EFUNC_ERR_ARG;
    if (J == 0) return EFUNC_OK;
    if (!q || !gS) return EFUNC_ERR_ARG;
    if ((st = check_cosine_workspace(grid, bands, J, workspace, workspace_bytes))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    Views v{cosine_layout(grid, bands, J), static_cast<char *>(workspace)};
    cudaError_t e = sort_into(v, grid->R, q, J, q_stride, v.sorted(), v.perm(), s);
    CosineArgs a = cosine_args(v, grid, bands, params);
    if (e == cudaSuccess) e = launch_cosine_pack(a, s);
    if (e != cudaSuccess) return cuda_fail();
    a.gS = gS;
    a.grad = grad;
    return cuda_status(launch_cosine(a, VAR_BACKWARD, s));
}

efunc_status efunc_cosine_fit(const efunc_grid *grid, int32_t bands, const efunc_adam *adam, int32_t loss,
                              float *params, float *m, float *v, const float *qo, int64_t J, int32_t n_batches,
                              int32_t steps, int64_t step0, float *stats, void *workspace, size_t workspace_bytes,
                              efunc_stream_t stream)
{
    efunc_status st = check_grid(grid);
    if (st) return st;
    if (!bands_ok(bands)) return EFUNC_ERR_ARG;
    if ((st = check_adam(adam))) return st;
    if (loss != EFUNC_LOSS_L1 && loss != EFUNC_LOSS_MSE) return EFUNC_ERR_ARG;
    if (J < 1 || J > kMaxJ || n_batches < 1 || steps < 0 || step0 < 0) return EFUNC_ERR_ARG;
    if (!params || !m || !v || !qo) return EFUNC_ERR_ARG;
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255u) ||
        workspace_bytes < cosine_layout(grid, bands, J, true).total)
        return EFUNC_ERR_WORKSPACE;
    if (steps == 0) return EFUNC_OK;
    if (is_host_pointer(qo) || (stats && is_host_pointer(stats))) return EFUNC_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = (int64_t)grid->R * grid->R * grid->R * 5 * bands;
    const float inv_J = (float)(1.0 / (double)J);
    {
        Views vp{cosine_layout(grid, bands, J, true), static_cast<char *>(workspace)};
        float *gp = vp.grad();
        if (cudaMemsetAsync(gp, 0, (size_t)n * 4, s) != cudaSuccess) return cuda_fail();
        return pipelined_device_fit(
            vp, grid->R, qo, J, n_batches, steps, s,
            [&](cudaStream_t st) { return launch_cosine_pack(cosine_args(vp, grid, bands, params), st); },
            [&](int32_t it, const SortBuf &sb, cudaStream_t st) {
                CosineArgs a = cosine_args(vp, grid, bands, params);
                a.sorted = sb.sorted;
                a.items = sb.items;
                a.ctrl = sb.ctrl;
                a.perm = nullptr;
                a.grad = gp;
                a.loss = loss;
                a.inv_J = inv_J;
                a.leave_room = 1;
                cudaError_t e = launch_cosine(a, VAR_FIT, st);
                if (e != cudaSuccess) return e;
                AdamArgs ad = adam_args(adam, n, params, gp, m, v, step0 + it + 1);
                ad.ctrl = sb.ctrl;
                ad.inv_J = inv_J;
                ad.stats = stats ? stats + 2 * (size_t)it : nullptr;
                return launch_adam(ad, st);
            });
    }
}

}  // extern "C"

// ------------------------------------------------------------ batched fit

namespace {

constexpr int kMinChunk = 32;

bool shapes_ok(const efunc_shape *shapes, int32_t S)
{
    if (!shapes || S < 1 || S > kMaxShapes) return false;
    int64_t jt = 0;
    for (int32_t i = 0; i < S; ++i) {
        if (shapes[i].R < 1 || shapes[i].R > kMaxR || shapes[i].J < 1 || !isfinite(shapes[i].log_beta0)) return false;
        jt += shapes[i].J;
        if (jt > kMaxJ) return false;
    }
    return true;
}

bool tuning_ok(const efunc_tuning &t)
{
    return t.chunk >= kMinChunk && t.chunk <= kChunk && t.lanes4_max >= 0 && t.lanes4_max <= t.lanes2_max &&
           t.lanes2_max <= kChunk && t.sort_blocks >= 1 && t.sort_blocks <= 16 && t.group_max >= 0 &&
           t.group_max <= kChunk;
}

efunc_tuning default_tuning() { return efunc_tuning{kChunk, 64, 32, 8, kGroupMax}; }

// Layout of a batched fit's workspace: control block (with the Adam clock
// at +128), shape table, per-shape loss sums, the sort of one batch of all
// shapes (histogram over every shape's bins), key records and gradient of the
// concatenated grids.
struct BatchedLayout {
    int64_t Jt = 0, centres = 0, nbins = 0, nscan_blocks = 0, max_items = 0;
    size_t ctrl, table, sums, hist, blocksum, rank, sorted, items, keys, grad, total;
    std::vector<BatchShape> table_host;
};

BatchedLayout batched_layout(const efunc_shape *shapes, int32_t S)
{
    BatchedLayout L;
    L.table_host.resize(S);
    for (int32_t i = 0; i < S; ++i) {
        const int R = shapes[i].R, P = (R + 1 + kBrick - 1) / kBrick;
        const int64_t nb = (int64_t)P * P * P * 64;
        BatchShape &b = L.table_host[i];
        b.R = R;
        b.P = P;
        b.q_off = L.Jt;
        b.J = shapes[i].J;
        b.bin_off = L.nbins;
        b.c_off = L.centres;
        b.log_beta0 = (double)shapes[i].log_beta0;
        b.inv_J = (float)(1.0 / (double)shapes[i].J);
        b.pad = 0;
        L.max_items += (shapes[i].J + kMinChunk - 1) / kMinChunk + (shapes[i].J < nb ? shapes[i].J : nb);
        L.Jt += shapes[i].J;
        L.nbins += nb;
        L.centres += (int64_t)R * R * R;
    }
    L.nscan_blocks = (L.nbins + kScanSegment - 1) / kScanSegment;
    const size_t A = 256;
    size_t off = 0;
    L.ctrl = off;     off = align_up(off + 256, A);   // Ctrl, then the AdamClock at +128
    L.table = off;    off = align_up(off + (size_t)S * sizeof(BatchShape), A);
    L.sums = off;     off = align_up(off + (size_t)S * 16, A);
    L.hist = off;     off = align_up(off + (size_t)L.nbins * 4, A);
    L.blocksum = off; off = align_up(off + (size_t)L.nscan_blocks * 8, A);
    L.rank = off;     off = align_up(off + (size_t)L.Jt * 4, A);
    L.sorted = off;   off = align_up(off + (size_t)L.Jt * 16, A);
    L.items = off;    off = align_up(off + (size_t)L.max_items * 16, A);
    L.keys = off;     off = align_up(off + (size_t)L.centres * kKeyRecords * 16, A);
    L.grad = off;     off = align_up(off + (size_t)L.centres * kSlots * 4, A);
    L.total = off;
    return L;
}

struct BatchedRun {
    const BatchedLayout *L;
    char *base;
    int32_t S;
    efunc_tuning tune;
    Ctrl *ctrl() const { return reinterpret_cast<Ctrl *>(base + L->ctrl); }
    AdamClock *clock() const { return reinterpret_cast<AdamClock *>(base + L->ctrl + 128); }
    BatchShape *table() const { return reinterpret_cast<BatchShape *>(base + L->table); }
    double *sums() const { return reinterpret_cast<double *>(base + L->sums); }
    float *grad() const { return reinterpret_cast<float *>(base + L->grad); }
    float4 *keys() const { return reinterpret_cast<float4 *>(base + L->keys); }

    // sort of one batch of every shape, key pack, fused kernel (FIT or EVAL)
    cudaError_t forward_backward(const float *params, const float *q, int32_t loss, bool eval, cudaStream_t s) const
    {
        cudaError_t e = cudaMemsetAsync(ctrl(), 0, sizeof(Ctrl), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(base + L->hist, 0, (size_t)L->nbins * 4, s);
        if (e != cudaSuccess) return e;
        SortArgs a{};
        a.q = q;
        a.J = L->Jt;
        a.q_stride = 4;
        a.nbins = L->nbins;
        a.hist = reinterpret_cast<uint32_t *>(base + L->hist);
        a.blocksum = reinterpret_cast<unsigned long long *>(base + L->blocksum);
        a.rank = reinterpret_cast<uint32_t *>(base + L->rank);
        a.sorted = reinterpret_cast<float4 *>(base + L->sorted);
        a.items = reinterpret_cast<Item *>(base + L->items);
        a.ctrl = ctrl();
        a.shapes = table();
        a.S = S;
        a.chunk = tune.chunk;
        a.group_max = tune.group_max;
        a.gtop = a.items + L->max_items - 1;
        if ((e = launch_sort_batched(a, s, tune.sort_blocks)) != cudaSuccess) return e;
        BatchedPackArgs pk{params, keys(), table(), S, L->centres};
        if ((e = launch_pack_keys_batched(pk, s)) != cudaSuccess) return e;
        FusedArgs f{};
        f.keys = keys();
        f.sorted = a.sorted;
        f.items = a.items;
        f.ctrl = ctrl();
        f.grad = grad();
        f.loss = loss;
        BatchArgs b{table(), sums(), tune.lanes2_max, tune.lanes4_max};
        if ((e = launch_fused_batched(f, b, eval, fused_batched_grid_size(), s)) != cudaSuccess) return e;
        return tune.group_max ? launch_grouped(f, b, a.gtop, eval, s) : cudaSuccess;
    }

    cudaError_t step(const efunc_adam *adam, int32_t loss, float *params, float *m, float *v, const float *q,
                     float *stats, cudaStream_t s) const
    {
        cudaError_t e = forward_backward(params, q, loss, false, s);
        if (e != cudaSuccess) return e;
        BatchedStatsArgs st{table(), S, sums(), stats, clock(), nullptr};
        if ((e = launch_batched_stats(st, s)) != cudaSuccess) return e;
        AdamArgs ad = adam_args(adam, L->centres * kSlots, params, grad(), m, v, 1);
        return launch_adam_clocked(ad, clock(), s);
    }
};

efunc_status check_batched(const efunc_shape *shapes, int32_t S, const efunc_tuning *tuning, void *workspace,
                           size_t workspace_bytes, BatchedLayout &L, efunc_tuning &t)
{
    if (!shapes_ok(shapes, S)) return EFUNC_ERR_ARG;
    t = tuning ? *tuning : default_tuning();
    if (!tuning_ok(t)) return EFUNC_ERR_ARG;
    L = batched_layout(shapes, S);
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255u) || workspace_bytes < L.total)
        return EFUNC_ERR_WORKSPACE;
    return EFUNC_OK;
}

// The batched fit's steps on stream s: seeds the Adam clock, uploads the
// shape table, then issues the steps one by one or replays one period of
// n_batches steps from a CUDA graph.
efunc_status fit_batched(const BatchedRun &run, const efunc_adam *adam, int32_t loss, float *params, float *m,
                         float *v, const float *qo, int32_t n_batches, int32_t steps, int64_t step0, float *stats,
                         bool graph, cudaStream_t s)
{
    const BatchedLayout &L = *run.L;
    const size_t batch_floats = (size_t)L.Jt * 4;
    auto batch = [&](int32_t it) { return qo + (size_t)(it % n_batches) * batch_floats; };
    if (cudaMemcpyAsync(run.table(), L.table_host.data(), L.table_host.size() * sizeof(BatchShape),
                        cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(run.sums(), 0, (size_t)run.S * 16, s) != cudaSuccess ||
        cudaMemsetAsync(run.grad(), 0, (size_t)L.centres * kSlots * 4, s) != cudaSuccess ||
        launch_adam_clock_seed(run.clock(), adam_clock_init(adam->lr, adam->beta1, adam->beta2, step0 + 1), s) !=
            cudaSuccess)
        return cuda_fail();
    int32_t done = 0;
    if (graph && steps > n_batches) {
        CopyPipe *pipe = nullptr;
        if (copy_pipe(&pipe) != cudaSuccess) return cuda_fail();
        std::lock_guard<std::mutex> pipe_lock(pipe->mu);
        cudaStream_t cs = pipe->capture_stream;
        cudaGraph_t g = nullptr;
        cudaGraphExec_t exec = nullptr;
        if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return cuda_fail();
        g_captured = 0;
        g_in_capture = true;
        bool ok = true;
        for (int32_t it = 0; it < n_batches && ok; ++it) ok = run.step(adam, loss, params, m, v, batch(it), stats, cs) == cudaSuccess;
        g_in_capture = false;
        cudaError_t e = cudaStreamEndCapture(cs, &g);
        const int64_t captured = g_captured;
        if (ok && e == cudaSuccess && g) e = cudaGraphInstantiate(&exec, g, 0);
        if (g) cudaGraphDestroy(g);
        const int32_t replays = steps / n_batches;
        for (int32_t r = 0; ok && exec && r < replays && e == cudaSuccess; ++r) e = cudaGraphLaunch(exec, s);
        if (exec) cudaGraphExecDestroy(exec);
        if (!ok || e != cudaSuccess) return cuda_fail(ok ? e : cudaSuccess);
        {
            std::lock_guard<std::mutex> lk(g_prof_mu);
            g_launches += captured * replays;
        }
        done = replays * n_batches;
    }
    for (int32_t it = done; it < steps; ++it)
        if (run.step(adam, loss, params, m, v, batch(it), stats, s) != cudaSuccess) return cuda_fail();
    return EFUNC_OK;
}

}  // namespace

extern "C" {

int64_t efunc_batched_param_count(const efunc_shape *shapes, int32_t S)
{
    if (!shapes_ok(shapes, S)) return -1;
    int64_t n = 0;
    for (int32_t i = 0; i < S; ++i) n += (int64_t)shapes[i].R * shapes[i].R * shapes[i].R * kSlots;
    return n;
}

int64_t efunc_batched_query_count(const efunc_shape *shapes, int32_t S)
{
    if (!shapes_ok(shapes, S)) return -1;
    int64_t n = 0;
    for (int32_t i = 0; i < S; ++i) n += shapes[i].J;
    return n;
}

size_t efunc_batched_workspace_bytes(const efunc_shape *shapes, int32_t S)
{
    if (!shapes_ok(shapes, S)) return 0;
    return batched_layout(shapes, S).total;
}

void efunc_default_tuning(efunc_tuning *out)
{
    if (out) *out = default_tuning();
}

efunc_status efunc_fit_batched(const efunc_shape *shapes, int32_t S, const efunc_adam *adam, int32_t loss,
                               float *params, float *m, float *v, const float *qo, int32_t n_batches, int32_t steps,
                               int64_t step0, float *stats, const efunc_tuning *tuning, int32_t graph,
                               void *workspace, size_t workspace_bytes, efunc_stream_t stream)
{
    efunc_status st = check_adam(adam);
    if (st) return st;
    if (loss != EFUNC_LOSS_L1 && loss != EFUNC_LOSS_MSE) return EFUNC_ERR_ARG;
    if (n_batches < 1 || n_batches > kMaxGraphBatches || steps < 0 || step0 < 0 || (graph != 0 && graph != 1))
        return EFUNC_ERR_ARG;
    if (!params || !m || !v || !qo) return EFUNC_ERR_ARG;
    BatchedLayout L;
    efunc_tuning t;
    if ((st = check_batched(shapes, S, tuning, workspace, workspace_bytes, L, t))) return st;
    if (steps == 0) return EFUNC_OK;
    if (is_host_pointer(qo) || (stats && is_host_pointer(stats))) return EFUNC_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (graph) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) return cuda_fail();
        if (cs != cudaStreamCaptureStatusNone) return EFUNC_ERR_ARG;
    }
    BatchedRun run{&L, static_cast<char *>(workspace), S, t};
    return fit_batched(run, adam, loss, params, m, v, qo, n_batches, steps, step0, stats, graph != 0, s);
}

efunc_status efunc_eval_batched(const efunc_shape *shapes, int32_t S, const float *params, const float *qo,
                                float *out, const efunc_tuning *tuning, void *workspace, size_t workspace_bytes,
                                efunc_stream_t stream)
{
    if (!params || !qo || !out) return EFUNC_ERR_ARG;
    BatchedLayout L;
    efunc_tuning t;
    efunc_status st = check_batched(shapes, S, tuning, workspace, workspace_bytes, L, t);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    BatchedRun run{&L, static_cast<char *>(workspace), S, t};
    if (cudaMemcpyAsync(run.table(), L.table_host.data(), L.table_host.size() * sizeof(BatchShape),
                        cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(run.sums(), 0, (size_t)S * 16, s) != cudaSuccess)
        return cuda_fail();
    cudaError_t e = run.forward_backward(params, qo, EFUNC_LOSS_MSE, true, s);
    if (e != cudaSuccess) return cuda_fail(e);
    BatchedStatsArgs sa{run.table(), S, run.sums(), nullptr, nullptr, out};
    return cuda_status(launch_batched_stats(sa, s));
}

efunc_status efunc_tune_batched(const efunc_shape *shapes, int32_t S, int32_t loss, float *params, float *m,
                                float *v, const float *qo, int32_t n_batches, int32_t trial_steps,
                                efunc_tuning *best, double *best_ms_per_step, void *workspace,
                                size_t workspace_bytes, efunc_stream_t stream)
{
    if (!best || trial_steps < 1 || trial_steps > 1000 || n_batches < 1 || n_batches > kMaxGraphBatches)
        return EFUNC_ERR_ARG;
    if (loss != EFUNC_LOSS_L1 && loss != EFUNC_LOSS_MSE) return EFUNC_ERR_ARG;
    if (!params || !m || !v || !qo) return EFUNC_ERR_ARG;
    BatchedLayout L;
    efunc_tuning t;
    efunc_status st = check_batched(shapes, S, nullptr, workspace, workspace_bytes, L, t);
    if (st) return st;
    if (is_host_pointer(qo)) return EFUNC_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    // trial steps take Adam steps with learning rate 0: the parameters stay
    // as they are; the moments are cleared afterwards
    const efunc_adam frozen{0.0, 0.9, 0.999, 1e-8, 0.0, 0};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return cuda_fail();
    }
    double best_ms = 1e300;
    efunc_tuning best_t = default_tuning();
    efunc_status rc = EFUNC_OK;
    const int chunks[] = {128, 256};
    const int lanes[][2] = {{64, 32}, {96, 48}, {64, 0}, {96, 0}};
    const int sorts[] = {4, 8};
    const int groups[] = {0, 64, 128};
    for (int c : chunks)
        for (const auto &ln : lanes)
            for (int sb : sorts)
                for (int gm : groups) {
                BatchedRun run{&L, static_cast<char *>(workspace), S, efunc_tuning{c, ln[0], ln[1], sb, gm}};
                // one untimed step, then trial_steps timed
                if ((rc = fit_batched(run, &frozen, loss, params, m, v, qo, n_batches, 1, 0, nullptr, false, s)))
                    goto done;
                if (cudaEventRecord(e0, s) != cudaSuccess) { rc = cuda_fail(); goto done; }
                if ((rc = fit_batched(run, &frozen, loss, params, m, v, qo, n_batches, trial_steps, 1, nullptr,
                                      false, s)))
                    goto done;
                float ms = 0.f;
                if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                    cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                    rc = cuda_fail();
                    goto done;
                }
                if (ms / trial_steps < best_ms) {
                    best_ms = ms / trial_steps;
                    best_t = run.tune;
                }
            }
    if (cudaMemsetAsync(m, 0, (size_t)L.centres * kSlots * 4, s) != cudaSuccess ||
        cudaMemsetAsync(v, 0, (size_t)L.centres * kSlots * 4, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
        rc = cuda_fail();
done:
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc == EFUNC_OK) {
        *best = best_t;
        if (best_ms_per_step) *best_ms_per_step = best_ms;
    }
    return rc;
}

void efunc_profile_enable(int32_t enable)
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_on = enable != 0;
}

int32_t efunc_profile_read(const char *name, double *total_ms, int64_t *launches)
{
    if (!name) return -1;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    int rc = drain_pending();
    for (int k = 0; k < K_COUNT; ++k) {
        if (strcmp(name, kKernelNames[k]) == 0) {
            if (total_ms) *total_ms = g_ms[k];
            if (launches) *launches = g_count[k];
            return rc;
        }
    }
    return -1;
}

efunc_status efunc_debug_bounds(int32_t *code)
{
    if (!code) return EFUNC_ERR_ARG;
    *code = 0;
#ifdef EFUNC_DEBUG_BOUNDS
    const cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e);
    const int a = bounds_code_fused(), b = bounds_code_sort();
    if (a < 0 || b < 0) return cuda_fail(cudaGetLastError());
    *code = a != 0 ? a : b;
    return EFUNC_OK;
#else
    return EFUNC_ERR_UNSUPPORTED;
#endif
}

void efunc_profile_reset(void)
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (Pending &p : g_pending) {
        if (p.start) g_free_events.push_back(p.start);
        if (p.stop) g_free_events.push_back(p.stop);
    }
    g_pending.clear();
    for (int k = 0; k < K_COUNT; ++k) {
        g_ms[k] = 0.0;
        g_count[k] = 0;
    }
}

int32_t efunc_last_cuda_error(void) { return g_last_cuda; }

const char *efunc_cuda_error_name(int32_t code) { return cudaGetErrorName((cudaError_t)code); }

int64_t efunc_launch_count(void)
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    return g_launches;
}

}  // extern "C"
