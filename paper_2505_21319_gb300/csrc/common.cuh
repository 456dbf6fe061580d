// Internal definitions shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "efunc.h"

namespace efunc {

constexpr int kMaxDevices = 64;

// Device ordinal of the calling thread's current device (0 if the runtime
// cannot tell).
int current_device();
// Multiprocessor count of the current device, looked up once per device.
int device_sm_count();
// Values derived from a device's properties (occupancy, persistent grid
// sizes, kernel attributes) are cached per (device, key, tag): the first
// call on a device runs compute() under one process-wide lock, so threads
// and devices never see each other's values.  A result <= 0 is not cached.
std::recursive_mutex &device_cache_mutex();
int &device_cache_slot(int dev, const void *key, int tag);   // caller holds the lock
template <class F>
int per_device_cached(const void *key, int tag, F compute)
{
    const int dev = current_device();
    std::lock_guard<std::recursive_mutex> lk(device_cache_mutex());
    int &v = device_cache_slot(dev, key, tag);
    if (v <= 0) v = compute();
    return v;
}

constexpr int kSlots = 13;        // floats per centre (Eq. func-offset, f^1)
constexpr int kW = 2;             // window half-width
constexpr int kCentres = 64;      // (2W)^3 centres per window
constexpr int kThreads = 128;     // threads of the fused kernel = keys per window
constexpr int kChunk = 256;       // queries per work item at most
constexpr int kMaxR = 256;
constexpr int kBrick = 4;         // cells per brick edge in the sort order
constexpr int kSortThreads = 128; // block size of every sort kernel (small, so that the
                                  // sort of the next batch fits beside the fit kernel)
constexpr int kScanSegment = 512; // bins per scan block

// Work item: one window-base cell and a contiguous slice of its sorted queries.
//   x = first sorted row, y = number of rows (1..kChunk),
//   z = packed cell (ux | uy << 10 | uz << 20) with u = c + 1 in [0, R],
//   w = shape of the item in a batched fit (0 otherwise).
using Item = int4;

// One shape of a batched fit (many grids of uneven resolution and query
// count fitted together).  Its queries are rows [q_off, q_off + J) of every
// batch, its histogram bins [bin_off, bin_off + P^3 * 64), its centres
// [c_off, c_off + R^3) of the concatenated grids (key records at 4 c_off,
// parameters and gradient at 13 c_off).
struct BatchShape {
    int R, P;
    int64_t q_off, J;
    int64_t bin_off, c_off;
    double log_beta0;
    float inv_J;
    int pad;
};
constexpr int kMaxShapes = 1024;

// Per-call control block at the start of the workspace.
struct Ctrl {
    int n_items;        // work items produced by the sort (one cell each)
    int next_item;      // dynamic work counter of the fused kernel
    int n_groups;       // grouped work items (sparse 2x2x2 cell octets), stored from the top of the item array down
    int next_group;     // dynamic work counter of the grouped kernel
    double loss_sum;    // sum over queries of |O-o| (L1) or (O-o)^2 (MSE), plus the Eikonal term
    double abs_sum;     // sum over queries of |O-o|
};

struct Layout {
    int P;              // bricks per axis, ceil((R+1)/4)
    int64_t nbins;      // P^3 * 64
    int64_t nscan_blocks;
    int64_t max_items;
    size_t ctrl, hist, blocksum, rank, sorted, perm, items, keys, grad, stage;
    // second sort buffer (the fit sorts batch s+1 while batch s is computed)
    size_t ctrl2, hist2, blocksum2, rank2, sorted2, items2;
    bool two_sort_buffers;
    size_t total;
};

// Workspace layout for R^3 centres and J queries; key_records (float4) and
// channels (floats) per centre size the key-record and gradient regions
// (the default model: 4 and 13; the ablation variants need other sizes).
// fit_regions = false leaves out what only the fits use (the gradient grid
// and the two host-batch staging buffers): the layout of the sort, forward
// and backward calls.
Layout make_layout(int R, int64_t J, int key_records = 4, int channels = 13, bool two_sort_buffers = false,
                   bool fit_regions = true);
inline Layout eval_layout(int R, int64_t J) { return make_layout(R, J, 4, 13, false, false); }

// Sort configuration passed to kernels.
struct SortArgs {
    const float *q;
    int64_t J;
    int q_stride;
    int R;
    int P;
    int64_t nbins;
    uint32_t *hist;      // counts, then exclusive offsets (in place)
    unsigned long long *blocksum;
    uint32_t *rank;
    float4 *sorted;
    int *perm;
    Item *items;
    Ctrl *ctrl;
    // batched sort (shapes != NULL): S shapes, queries of shape s binned on
    // its own grid into bins bin_off + [0, P^3 * 64); R / P above unused
    const BatchShape *shapes;
    int S;
    int chunk;           // queries per work item at most (batched sort; kChunk otherwise)
    // sparse cells: an aligned 2x2x2 octet of bins (8 consecutive bins of the
    // brick-Morton order) with at least two non-empty cells and at most
    // group_max queries becomes one grouped item, written to gtop[-g] for the
    // g-th group (the top end of the item array); 0 disables grouping
    int group_max;
    Item *gtop;
};

// Four doubles in one 32-byte aligned record: the FP64 counterpart of a
// float4 key record or query row.
struct alignas(32) Double4 {
    double x, y, z, w;
};

// Vector types of the scalar type a kernel computes in.
template <typename T> struct VecOf;
template <> struct VecOf<float> { using V4 = float4; using V2 = float2; };
template <> struct VecOf<double> { using V4 = Double4; using V2 = double2; };
template <typename T> using V4Of = typename VecOf<T>::V4;

// Key records of one centre, 4 float4 (64 bytes), built once per call by the
// pack kernel from the 13 parameters:
//   [0] (0, 0, 0, -beta log2(e))        [1] (o, d)
//   [2] (Delta, -beta' log2(e))         [3] (o', d')
// The scales are formed in FP64 and rounded once.  Key positions are not
// stored: the fused kernel forms them in window-local coordinates,
// (i - c) h for the grid key and (i - c) h + Delta for the offset key, so that
// no absolute position near +-1 is ever rounded.
constexpr int kKeyRecords = 4;

template <typename T>
struct PackArgsT {
    const T *params;
    V4Of<T> *keys;
    int R;
    double log_beta0;
};
using PackArgs = PackArgsT<float>;
using PackArgs64 = PackArgsT<double>;


// Fused-kernel arguments, for the scalar type T of its arithmetic (float:
// the hot path; double: the same kernels in FP64 for finite-difference
// checks).
template <typename T>
struct FusedArgsT {
    const V4Of<T> *keys;  // packed key records, R^3 * 4
    int R;
    const V4Of<T> *sorted;
    const int *perm;
    const Item *items;
    Ctrl *ctrl;
    // forward outputs (user order)
    T *O;
    T *lse;
    T *dq;
    // backward inputs / outputs
    const T *gO;         // user order, or NULL (no value term) in second-order mode
    const T *gG;         // user order J x 3: dL/d(dO/dq) (second-order backward)
    T *grad;
    T *gq;               // user order
    // fit / evaluation
    int loss;
    float inv_J;
    float eik_weight;    // weight of the Eikonal term (|dO/dq|^2 - 1)^2 in the fit
};
using FusedArgs = FusedArgsT<float>;
using FusedArgs64 = FusedArgsT<double>;

struct AdamArgs {
    float *p, *g, *m, *v;
    int64_t n;
    // FP32 constants formed in FP64 on the host
    float beta1, one_minus_beta1, beta2, one_minus_beta2, eps, wd;
    float decay;            // 1 - lr*wd (AdamW)
    int decoupled;
    float step_size;        // lr / (1 - beta1^t)
    float inv_sqrt_bc2;     // 1 / sqrt(1 - beta2^t)
    // optional fit statistics: stats[0] = loss_sum * inv_J, stats[1] = abs_sum * inv_J
    const Ctrl *ctrl;
    float *stats;
    float inv_J;
};

struct MeanShiftArgs {
    const float *pts;    // N x 3 surface points
    int64_t N;
    int R;
    float sigma;         // sqrt(bandwidth * log2(e)): coordinate scale of the base-2 exponent
    float *params;       // R^3 x 13, slots 0..2 written
};

// Ablation variants (Table tab:ablation): key sets, value degree, learnable
// scales.  One persistent kernel per (mode, sets, degree) over the same
// cell-sorted work items as the default model.
struct VariantArgs {
    int sets;            // 1 grid keys, 2 offset keys, 3 both
    int deg;             // value polynomial degree 0..3
    int learn;           // learnable log-scales
    int channels;        // floats per centre
    const float *params; // R^3 x channels
    double log_beta0;
    float4 *keys;        // packed records: R^3 x nsets x (1 + ceil(nv / 4)) float4
    int R;
    const float4 *sorted;
    const int *perm;
    const Item *items;
    Ctrl *ctrl;
    float *O;            // forward outputs (user order)
    float *lse;
    const float *gO;     // backward input (user order)
    float *grad;         // R^3 x channels, accumulated
    int loss;            // fit
    float inv_J;
    int leave_room;      // persistent grid leaves room for the next batch's sort (pipelined fit)
};

enum VariantMode { VAR_FORWARD = 0, VAR_BACKWARD = 1, VAR_FIT = 2 };

// Cosine-series decomposition (Sec. 4.4): B bands of Config-G-6 grids
// (5 floats per centre: b, o, d), S(q) = sum_b w_b(q) O_b(q).
constexpr int kMaxBands = 16;

struct CosineArgs {
    int B;               // bands, 1..kMaxBands
    const float *params; // B x R^3 x 5, band-major
    double log_beta0;
    float4 *keys;        // packed records: B x R^3 x 2 float4
    int R;
    const float4 *sorted;
    const int *perm;
    const Item *items;
    Ctrl *ctrl;
    float *S;            // forward output (user order)
    const float *gS;     // backward input (user order)
    float *grad;         // B x R^3 x 5, accumulated
    int loss;
    float inv_J;
    int leave_room;      // persistent grid leaves room for the next batch's sort (pipelined fit)
};

// Extra arguments of the batched fused kernel (a second kernel parameter, so
// that the other instantiations keep their argument layout): per-item shape
// (Item.w) -> R, key records, gradient, 1/J; loss sums per shape in
// shape_sums[2 s + {0, 1}]; lane thresholds of the forward (items of at most
// lanes2_max / lanes4_max queries use 2 / 4 lanes per query).
struct BatchArgs {
    const BatchShape *shapes;
    double *shape_sums;
    int lanes2_max, lanes4_max;
};

// Batched fit (many shapes, one launch per kernel per step).
struct BatchedPackArgs {
    const float *params;   // concatenated grids, 13 floats per centre
    float4 *keys;
    const BatchShape *shapes;
    int S;
    int64_t n_centres;
};
struct BatchedStatsArgs {
    const BatchShape *shapes;
    int S;
    double *sums;          // 2 S loss / |error| sums, zeroed after reading
    float *stats;          // steps x S x 2 (loss, MAE) or NULL
    const void *clk;       // AdamClock: statistics row t - t_first
    float *out;            // S x 2 (mean squared, mean absolute error) of an evaluation, or NULL
};

// Kernel identifiers for the profiler.
enum KernelId { K_BIN = 0, K_SCAN_REDUCE, K_SCAN_TOP, K_SCAN_EMIT, K_SCATTER, K_PACK_KEYS, K_FORWARD, K_FUSED_BWD,
                K_FUSED_FIT, K_ADAM, K_MEAN_SHIFT, K_VAR_PACK, K_VAR_FORWARD, K_VAR_BACKWARD, K_VAR_FIT, K_COS_PACK, K_COS_FORWARD, K_COS_BACKWARD,
                K_COS_FIT, K_EVAL, K_F64, K_BATCHED, K_BATCHED_STATS, K_ENC_CONV, K_ENC_WGRAD, K_ENC_AUX, K_GROUPED,
                K_EVAL_FINISH, K_COUNT };

// Launch bookkeeping (launch counter and optional CUDA-event profiling).
void launch_begin(int kid, cudaStream_t s);
void launch_end(int kid, cudaStream_t s);

// Launchers (defined in sort.cu, fused.cu, adam.cu).  They return the CUDA
// error of the launch.
// narrow_blocks > 0: bin and scatter with that many 128-thread blocks per SM
// (the pipelined fits run them beside a persistent fit kernel); 0: wide grids
cudaError_t launch_sort(const SortArgs &a, cudaStream_t s, int narrow_blocks = 0);
cudaError_t launch_pack_keys(const PackArgs &a, cudaStream_t s);
cudaError_t launch_forward(const FusedArgs &a, bool with_dq, int grid, cudaStream_t s);
cudaError_t launch_fused_backward(const FusedArgs &a, bool with_gq, bool second_order, int grid, cudaStream_t s);
cudaError_t launch_fused_fit(const FusedArgs &a, bool eikonal, int grid, cudaStream_t s);
// Forward over a batch of (x, y, z, target) rows that only sums the loss:
// ctrl->loss_sum += sum (O - o)^2, ctrl->abs_sum += sum |O - o|.
cudaError_t launch_fused_eval(const FusedArgs &a, int grid, cudaStream_t s);
// out[0] = loss_sum * inv_J, out[1] = abs_sum * inv_J (FP32, device)
cudaError_t launch_eval_finish(const Ctrl *ctrl, double inv_J, float *out, cudaStream_t s);
// FP64 instantiations (no fast paths: exp2 / log2 in double) of the pack,
// forward and backward kernels, and the gather of FP64 query rows in sorted
// order (rows64[i] = q64[perm[i]], q_stride 3 or 4, w = 0 for stride 3).
cudaError_t launch_pack_keys64(const PackArgs64 &a, cudaStream_t s);
cudaError_t launch_forward64(const FusedArgs64 &a, bool with_dq, int grid, cudaStream_t s);
cudaError_t launch_fused_backward64(const FusedArgs64 &a, bool with_gq, int grid, cudaStream_t s);
cudaError_t launch_round_queries(const double *q64, int64_t J, int q_stride, float4 *rows32, cudaStream_t s);
cudaError_t launch_gather_queries64(const double *q64, int64_t J, int q_stride, const int *perm, Double4 *rows64,
                                    cudaStream_t s);
int fused_grid_size64();
// batched fit: sort of all shapes' queries (bins per shape), key pack over
// all grids, fused fit / evaluation kernel with per-item shapes, per-shape
// statistics
cudaError_t launch_sort_batched(const SortArgs &a, cudaStream_t s, int blocks_per_sm);
// Grouped items (sparse cell octets): the union window of the octet is staged
// once; FIT and EVAL modes, single-shape or batched (b.shapes != NULL).
cudaError_t launch_grouped(const FusedArgs &a, const BatchArgs &b, const Item *gtop, bool eval, cudaStream_t s);
constexpr int kGroupMax = 128;   // default queries per grouped octet at most
cudaError_t launch_pack_keys_batched(const BatchedPackArgs &a, cudaStream_t s);
cudaError_t launch_fused_batched(const FusedArgs &a, const BatchArgs &b, bool eval, int grid, cudaStream_t s);
cudaError_t launch_batched_stats(const BatchedStatsArgs &a, cudaStream_t s);
int fused_batched_grid_size();
int fused_fit_grid_size(bool eikonal, bool leave_room);   // persistent grid of the fit kernel
// CTAs per SM of a persistent kernel reduced until the registers of
// sort_blocks sort blocks (kSortThreads x 32 each) stay free on every SM.
// Two by default: with exactly one block's worth free, a sort started
// together with the persistent kernel did not fit beside it (variant and
// second-order fits measured: the sort ran after the kernel).
int leave_sort_room(const void *kernel, int per_sm, int sort_blocks = 2);
cudaError_t launch_adam(const AdamArgs &a, cudaStream_t s);
cudaError_t launch_mean_shift(const MeanShiftArgs &a, cudaStream_t s);
cudaError_t launch_variant_pack(const VariantArgs &a, cudaStream_t s);
cudaError_t launch_variant(const VariantArgs &a, int mode, cudaStream_t s);
int variant_key_records(int sets, int deg);   // float4 records per centre
cudaError_t launch_cosine_pack(const CosineArgs &a, cudaStream_t s);
cudaError_t launch_cosine(const CosineArgs &a, int mode, cudaStream_t s);   // mode: VariantMode
int fused_grid_size();   // persistent grid: SMs x resident blocks per SM

// Window-base index along one axis: clamp(floor((q+1)*R/2 - 1/2), -1, R-1),
// in FP32 with every operation rounded separately (no contraction into FMA).
__device__ __forceinline__ int window_base(float q, float half_r, float rmax)
{
    float t = __fmul_rn(__fadd_rn(q, 1.0f), half_r);
    float u = __fsub_rn(t, 0.5f);
    u = (u >= -1.0f) ? u : -1.0f;   // NaN -> -1
    u = fminf(u, rmax);
    return (int)floorf(u);
}

// Brick-Morton bin of a cell u = (ux, uy, uz) in [0, R]^3: bricks of 4^3
// cells in row-major order, Morton order of the 64 cells inside a brick.
__device__ __forceinline__ uint32_t bin_of(int ux, int uy, int uz, int P)
{
    uint32_t brick = ((uint32_t)(ux >> 2) * P + (uint32_t)(uy >> 2)) * P + (uint32_t)(uz >> 2);
    uint32_t lx = ux & 3, ly = uy & 3, lz = uz & 3;
    uint32_t m = (lx & 1) << 2 | (ly & 1) << 1 | (lz & 1) | (lx & 2) << 4 | (ly & 2) << 3 | (lz & 2) << 2;
    return brick * 64u + m;
}

__device__ __forceinline__ void cell_of_bin(uint32_t bin, int P, int &ux, int &uy, int &uz)
{
    uint32_t brick = bin >> 6, m = bin & 63u;
    int bz = brick % P, by = (brick / P) % P, bx = brick / (P * P);
    int lx = ((m >> 2) & 1) | ((m >> 4) & 2);
    int ly = ((m >> 1) & 1) | ((m >> 3) & 2);
    int lz = (m & 1) | ((m >> 2) & 2);
    ux = bx * 4 + lx;
    uy = by * 4 + ly;
    uz = bz * 4 + lz;
}

// Bounds-check build (-DEFUNC_DEBUG_BOUNDS): the hot gathers and scatters
// test their indices with bounds_ok(condition, code); a failing test records
// its code in a device flag of the translation unit (the first one wins) and
// the caller skips the access.  In the normal build the test is the constant
// true and compiles away.  Codes: 1 staged key outside the grid, 2 staged
// query outside its item's cell, 3 union key outside the grid, 4 staged
// query outside its octet, 5 paired-row slot past its buffer, 6 bin past the
// bin count, 7 sorted position past J, 8 work item with a bad range.
#ifdef EFUNC_DEBUG_BOUNDS
static __device__ int g_bounds_code;
__device__ __forceinline__ bool bounds_ok(bool ok, int code)
{
    if (!ok) atomicCAS(&g_bounds_code, 0, code);
    return ok;
}
#else
__device__ __forceinline__ bool bounds_ok(bool, int) { return true; }
#endif
// first code recorded by fused.cu / sort.cu on the current device, cleared
// (0 without a failure or in the normal build, -1 on a CUDA error)
int bounds_code_fused();
int bounds_code_sort();

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float lg2_approx(float x)
{
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

}  // namespace efunc
