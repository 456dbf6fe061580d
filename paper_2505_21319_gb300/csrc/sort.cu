// Cell sort of the query batch (hot-path step a1).
//
// Every query is binned by its window-base cell u = c + 1 in [0, R]^3 (the
// cell whose 4x4x4 centre window the query blends), so that all queries of a
// bin share one window.  Bins are ordered in 4x4x4 bricks (row-major) with
// Morton order inside a brick.  A counting sort:
//   bin      histogram by atomics; each query keeps its arrival rank inside
//            its bin (batches arrive in random order, so lanes of a warp rarely
//            share a bin and warp aggregation would not pay)
//   scan     exclusive scan of (count, work items) pairs over all bins
//            (reduce per block / scan of block sums / scan + emit)
//   scatter  query -> position offset[bin] + rank: float4 row + permutation
//            (the permutation only when a caller needs outputs in its order)
// The scan also emits the work items of the fused kernel: every non-empty bin
// yields ceil(count / kChunk) slices of at most kChunk sorted queries.  On
// coarse grids the histogram has several copies (sort_copies.cuh); the
// kernels take the copy count K as a template argument.
#include "common.cuh"
#include "sort_copies.cuh"

namespace efunc {

namespace {

constexpr int kScanThreads = kSortThreads;
constexpr int kScanPerThread = kScanSegment / kScanThreads;
constexpr int kScanSeg = kScanSegment;   // bins per scan block
constexpr int kWideThreads = 256;        // bin / scatter block size when the sort runs alone
// at most 32 registers per thread, so that a kSortThreads block fits in the
// registers the persistent fit kernel leaves free on each SM
constexpr int kSortMinBlocks = 65536 / (kSortThreads * 32);
constexpr int kWideMinBlocks = 65536 / (kWideThreads * 32);
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ void load_query(const float *q, int64_t j, int stride, bool vec4, float &x, float &y,
                                           float &z, float &w)
{
    if (vec4) {
        float4 v = __ldg(reinterpret_cast<const float4 *>(q) + j);
        x = v.x; y = v.y; z = v.z; w = v.w;
    } else {
        const float *r = q + j * stride;
        x = __ldg(r); y = __ldg(r + 1); z = __ldg(r + 2);
        w = stride == 4 ? __ldg(r + 3) : 0.0f;
    }
}

__device__ __forceinline__ uint32_t query_bin(float x, float y, float z, float half_r, float rmax, int P)
{
    int ux = window_base(x, half_r, rmax) + 1;
    int uy = window_base(y, half_r, rmax) + 1;
    int uz = window_base(z, half_r, rmax) + 1;
    return bin_of(ux, uy, uz, P);
}

// Grid-stride loops take kUnroll queries per thread and iteration, so that a
// small grid (one block per SM beside the fit kernel) still keeps several
// loads and atomics in flight per thread.
constexpr int kUnroll = 4;

// The histogram copy of query j (K copies): the 32 queries of a warp's
// coalesced load share one, consecutive warps cycle through them.
template <int K>
__device__ __forceinline__ uint32_t copy_of(int64_t j)
{
    return K == 1 ? 0u : (uint32_t)(j >> 5) & (uint32_t)(K - 1);
}

template <bool VEC4, int K>
__global__ void __launch_bounds__(kWideThreads, kWideMinBlocks) bin_kernel(SortArgs a)
{
    const float half_r = (float)a.R * 0.5f, rmax = (float)(a.R - 1);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; j + (kUnroll - 1) * stride < a.J; j += kUnroll * stride) {
        uint32_t bin[kUnroll], r[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            float x, y, z, w;
            load_query(a.q, j + u * stride, a.q_stride, VEC4, x, y, z, w);
            bin[u] = query_bin(x, y, z, half_r, rmax, a.P);
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
            r[u] = atomicAdd(&a.hist[(int64_t)copy_of<K>(j + u * stride) * a.nbins + bin[u]], 1u);
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) a.rank[j + u * stride] = (copy_of<K>(j + u * stride) << kRankBits) | r[u];
    }
    for (; j < a.J; j += stride) {
        float x, y, z, w;
        load_query(a.q, j, a.q_stride, VEC4, x, y, z, w);
        const uint32_t c = copy_of<K>(j);
        a.rank[j] = (c << kRankBits) |
                    atomicAdd(&a.hist[(int64_t)c * a.nbins + query_bin(x, y, z, half_r, rmax, a.P)], 1u);
    }
}

// Coarse grids (few bins, hundreds of queries per bin) make the global
// histogram atomics contend.  There every block counts a contiguous slice of
// queries in a shared-memory histogram first (local arrival ranks), then
// reserves each non-empty bin's range with one global atomic (in histogram
// copy blockIdx mod K), then adds the reserved base to its queries' ranks.
constexpr int kSmemBinsMax = (int)kCoarseBins;   // 48 KB of counters

template <bool VEC4, int K>
__global__ void __launch_bounds__(kWideThreads, kWideMinBlocks) bin_smem_kernel(SortArgs a, int64_t slice)
{
    extern __shared__ uint32_t s_hist[];
    const float half_r = (float)a.R * 0.5f, rmax = (float)(a.R - 1);
    const int nb = (int)a.nbins;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) s_hist[i] = 0u;
    __syncthreads();
    const int64_t j0 = (int64_t)blockIdx.x * slice, j1 = min(a.J, j0 + slice);
    for (int64_t j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
        float x, y, z, w;
        load_query(a.q, j, a.q_stride, VEC4, x, y, z, w);
        a.rank[j] = atomicAdd(&s_hist[query_bin(x, y, z, half_r, rmax, a.P)], 1u);
    }
    __syncthreads();
    const uint32_t copy = K == 1 ? 0u : blockIdx.x & (uint32_t)(K - 1);
    uint32_t *h = a.hist + (int64_t)copy * a.nbins;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        const uint32_t c = s_hist[i];
        if (c) s_hist[i] = atomicAdd(&h[i], c);
    }
    __syncthreads();
    for (int64_t j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
        float x, y, z, w;
        load_query(a.q, j, a.q_stride, VEC4, x, y, z, w);
        a.rank[j] = (copy << kRankBits) | (a.rank[j] + s_hist[query_bin(x, y, z, half_r, rmax, a.P)]);
    }
}

// Packed scan value: low 32 bits = query count, high 32 bits = work items.
__device__ __forceinline__ unsigned long long pack(uint32_t count)
{
    unsigned long long items = (count + kChunk - 1) / kChunk;
    return (items << 32) | (unsigned long long)count;
}

// Exclusive block scan of one 64-bit value per thread; returns the block total.
__device__ __forceinline__ unsigned long long block_exclusive_scan(unsigned long long v, unsigned long long &total)
{
    __shared__ unsigned long long warp_tot[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    unsigned long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
        unsigned long long s = lane < nw ? warp_tot[lane] : 0ull;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long y = __shfl_up_sync(kFull, s, o);
            if (lane >= o) s += y;
        }
        warp_tot[lane] = s;
    }
    __syncthreads();
    const unsigned long long prefix = wid ? warp_tot[wid - 1] : 0ull;
    total = warp_tot[nw - 1];
    __syncthreads();   // warp_tot is reused by the next call
    return prefix + x - v;
}

// A bin's count: the sum of its K histogram copies.
template <int K>
__device__ __forceinline__ uint32_t bin_count(const SortArgs &a, int64_t b)
{
    uint32_t c = a.hist[b];
#pragma unroll
    for (int k = 1; k < K; ++k) c += a.hist[k * a.nbins + b];
    return c;
}

template <int K>
__global__ void __launch_bounds__(kScanThreads, kSortMinBlocks) scan_reduce_kernel(SortArgs a)
{
    const int64_t b0 = (int64_t)blockIdx.x * kScanSeg + (int64_t)threadIdx.x * kScanPerThread;
    unsigned long long s = 0;
#pragma unroll
    for (int k = 0; k < kScanPerThread; ++k)
        if (b0 + k < a.nbins) s += pack(bin_count<K>(a, b0 + k));
    unsigned long long total;
    block_exclusive_scan(s, total);
    if (threadIdx.x == 0) a.blocksum[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads, kSortMinBlocks) scan_top_kernel(SortArgs a, int64_t nblocks)
{
    unsigned long long carry = 0;
    for (int64_t base = 0; base < nblocks; base += kScanThreads) {
        const int64_t i = base + threadIdx.x;
        const unsigned long long v = i < nblocks ? a.blocksum[i] : 0ull;
        unsigned long long total;
        const unsigned long long ex = block_exclusive_scan(v, total);
        if (i < nblocks) a.blocksum[i] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) a.ctrl->n_items = (int)(carry >> 32);
}

template <int K>
__global__ void __launch_bounds__(kScanThreads, kSortMinBlocks) scan_emit_kernel(SortArgs a)
{
    const int64_t b0 = (int64_t)blockIdx.x * kScanSeg + (int64_t)threadIdx.x * kScanPerThread;
    uint32_t cnt[kScanPerThread];
    unsigned long long s = 0;
#pragma unroll
    for (int k = 0; k < kScanPerThread; ++k) {
        cnt[k] = b0 + k < a.nbins ? bin_count<K>(a, b0 + k) : 0u;
        s += pack(cnt[k]);
    }
    unsigned long long total;
    unsigned long long run = a.blocksum[blockIdx.x] + block_exclusive_scan(s, total);
#pragma unroll
    for (int k = 0; k < kScanPerThread; ++k) {
        if (b0 + k >= a.nbins) break;
        const uint32_t start = (uint32_t)(run & 0xffffffffull);
        const uint32_t item0 = (uint32_t)(run >> 32);
        // counts become exclusive offsets, in place: a bin's copies take
        // consecutive ranges from its start
        if (K == 1) {
            a.hist[b0 + k] = start;
        } else {
            uint32_t off = start;
#pragma unroll
            for (int c = 0; c < K; ++c) {
                const uint32_t n = a.hist[c * a.nbins + b0 + k];
                a.hist[c * a.nbins + b0 + k] = off;
                off += n;
            }
        }
        if (cnt[k]) {
            int ux, uy, uz;
            cell_of_bin((uint32_t)(b0 + k), a.P, ux, uy, uz);
            const int packed = ux | (uy << 10) | (uz << 20);
            const uint32_t nit = (cnt[k] + kChunk - 1) / kChunk;
            for (uint32_t i = 0; i < nit; ++i) {
                const uint32_t off = i * kChunk;
                const uint32_t len = min((uint32_t)kChunk, cnt[k] - off);
                a.items[item0 + i] = make_int4((int)(start + off), (int)len, packed, 0);
            }
        }
        run += pack(cnt[k]);
    }
}

template <bool VEC4, int K>
__global__ void __launch_bounds__(kWideThreads, kWideMinBlocks) scatter_kernel(SortArgs a)
{
    const float half_r = (float)a.R * 0.5f, rmax = (float)(a.R - 1);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; j + (kUnroll - 1) * stride < a.J; j += kUnroll * stride) {
        float4 v[kUnroll];
        uint32_t pos[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            load_query(a.q, j + u * stride, a.q_stride, VEC4, v[u].x, v[u].y, v[u].z, v[u].w);
            pos[u] = a.rank[j + u * stride];
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const uint32_t rk = pos[u];   // (copy, rank in the copy)
            const uint32_t bin = query_bin(v[u].x, v[u].y, v[u].z, half_r, rmax, a.P);
            if (!bounds_ok(bin < a.nbins, 6)) {
                pos[u] = 0xffffffffu;   // skipped below
                continue;
            }
            pos[u] = K == 1 ? a.hist[bin] + rk : a.hist[(int64_t)(rk >> kRankBits) * a.nbins + bin] + (rk & kRankMask);
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            if (!bounds_ok(pos[u] < a.J, 7)) continue;
            a.sorted[pos[u]] = v[u];
            if (a.perm) a.perm[pos[u]] = (int)(j + u * stride);
        }
    }
    for (; j < a.J; j += stride) {
        float x, y, z, w;
        load_query(a.q, j, a.q_stride, VEC4, x, y, z, w);
        const uint32_t bin = query_bin(x, y, z, half_r, rmax, a.P);
        if (!bounds_ok(bin < a.nbins, 6)) continue;
        const uint32_t rk = a.rank[j];
        const uint32_t pos =
            K == 1 ? a.hist[bin] + rk : a.hist[(int64_t)(rk >> kRankBits) * a.nbins + bin] + (rk & kRankMask);
        if (!bounds_ok(pos < a.J, 7)) continue;
        a.sorted[pos] = make_float4(x, y, z, w);
        if (a.perm) a.perm[pos] = (int)j;
    }
}

// Index of the last offset <= x among S ascending offsets (offs[0] = 0).
__device__ __forceinline__ int shape_of(const int64_t *offs, int S, int64_t x)
{
    int lo = 0, hi = S - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (offs[mid] <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <bool BY_BIN>
__device__ __forceinline__ void load_offsets(const SortArgs &a, int64_t *s_off)
{
    for (int i = threadIdx.x; i < a.S; i += blockDim.x) s_off[i] = BY_BIN ? a.shapes[i].bin_off : a.shapes[i].q_off;
    __syncthreads();
}

__device__ __forceinline__ uint32_t batched_bin(const BatchShape &sh, float x, float y, float z)
{
    return (uint32_t)query_bin(x, y, z, (float)sh.R * 0.5f, (float)(sh.R - 1), sh.P);
}

__device__ __forceinline__ unsigned long long pack_chunk(uint32_t count, uint32_t chunk)
{
    unsigned long long items = (count + chunk - 1) / chunk;
    return (items << 32) | (unsigned long long)count;
}

// ------------------------------------------------- grouped scan (sparse cells)
//
// The same scan over 8 bins per thread (64 threads per 512-bin segment), so
// that a thread holds one aligned octet of bins: a 2x2x2 block of cells.  An
// octet with at least two non-empty cells and at most group_max queries is
// emitted as one grouped item (appended at the top of the item array) and
// counts no per-cell item; every other octet emits its cells' items as
// usual.  The bins' offsets are the same either way (an octet's queries are
// contiguous).
constexpr int kOct = 8;
constexpr int kGrpThreads = kScanSeg / kOct;

template <bool BATCHED>
__device__ __forceinline__ uint32_t scan_chunk(const SortArgs &a) { return BATCHED ? (uint32_t)a.chunk : (uint32_t)kChunk; }

__device__ __forceinline__ bool octet_grouped(const uint32_t cnt[kOct], int group_max)
{
    uint32_t tot = 0;
    int nonempty = 0;
#pragma unroll
    for (int k = 0; k < kOct; ++k) {
        tot += cnt[k];
        nonempty += cnt[k] > 0u;
    }
    return nonempty >= 2 && tot <= (uint32_t)group_max;
}

template <int K, bool BATCHED>
__device__ __forceinline__ unsigned long long octet_value(const SortArgs &a, int64_t b0, uint32_t cnt[kOct])
{
#pragma unroll
    for (int k = 0; k < kOct; ++k) cnt[k] = b0 + k < a.nbins ? bin_count<K>(a, b0 + k) : 0u;
    const uint32_t chunk = scan_chunk<BATCHED>(a);
    unsigned long long v = 0;
    if (octet_grouped(cnt, a.group_max)) {
#pragma unroll
        for (int k = 0; k < kOct; ++k) v += cnt[k];   // queries only, no per-cell item
    } else {
#pragma unroll
        for (int k = 0; k < kOct; ++k) v += pack_chunk(cnt[k], chunk);
    }
    return v;
}

template <int K, bool BATCHED>
__global__ void __launch_bounds__(kGrpThreads) scan_reduce_grp_kernel(SortArgs a)
{
    uint32_t cnt[kOct];
    const unsigned long long v = octet_value<K, BATCHED>(a, (int64_t)blockIdx.x * kScanSeg + threadIdx.x * kOct, cnt);
    unsigned long long total;
    block_exclusive_scan(v, total);
    if (threadIdx.x == 0) a.blocksum[blockIdx.x] = total;
}

template <int K, bool BATCHED>
__global__ void __launch_bounds__(kGrpThreads) scan_emit_grp_kernel(SortArgs a)
{
    __shared__ int64_t s_off[BATCHED ? kMaxShapes : 1];
    if (BATCHED) load_offsets<true>(a, s_off);
    const int64_t b0 = (int64_t)blockIdx.x * kScanSeg + threadIdx.x * kOct;
    uint32_t cnt[kOct];
    const unsigned long long v = octet_value<K, BATCHED>(a, b0, cnt);
    unsigned long long total;
    unsigned long long run = a.blocksum[blockIdx.x] + block_exclusive_scan(v, total);
    if (b0 >= a.nbins) return;
    const bool grouped = octet_grouped(cnt, a.group_max);
    const uint32_t chunk = scan_chunk<BATCHED>(a);
    int shape = 0, P = a.P;
    int64_t local0 = b0;
    if (BATCHED) {
        shape = shape_of(s_off, a.S, b0);
        P = a.shapes[shape].P;
        local0 = b0 - s_off[shape];
    }
    if (grouped) {
        int ux, uy, uz;
        cell_of_bin((uint32_t)local0, P, ux, uy, uz);   // the octet's first cell: even coordinates
        uint32_t tot = 0;
#pragma unroll
        for (int k = 0; k < kOct; ++k) tot += cnt[k];
        const int g = atomicAdd(&a.ctrl->n_groups, 1);
        a.gtop[-g] = make_int4((int)(run & 0xffffffffull), (int)tot, ux | (uy << 10) | (uz << 20), shape);
    }
#pragma unroll
    for (int k = 0; k < kOct; ++k) {
        if (b0 + k >= a.nbins) break;
        const uint32_t start = (uint32_t)(run & 0xffffffffull);
        const uint32_t item0 = (uint32_t)(run >> 32);
        if (K == 1) {
            a.hist[b0 + k] = start;
        } else {
            uint32_t off = start;
#pragma unroll
            for (int c = 0; c < K; ++c) {
                const uint32_t n = a.hist[c * a.nbins + b0 + k];
                a.hist[c * a.nbins + b0 + k] = off;
                off += n;
            }
        }
        if (!grouped && cnt[k]) {
            int ux, uy, uz;
            cell_of_bin((uint32_t)(local0 + k), P, ux, uy, uz);
            const int packed = ux | (uy << 10) | (uz << 20);
            const uint32_t nit = (cnt[k] + chunk - 1) / chunk;
            for (uint32_t i = 0; i < nit; ++i) {
                const uint32_t off = i * chunk;
                const uint32_t len = min(chunk, cnt[k] - off);
                a.items[item0 + i] = make_int4((int)(start + off), (int)len, packed, shape);
            }
        }
        run += grouped ? (unsigned long long)cnt[k] : pack_chunk(cnt[k], chunk);
    }
}

int stream_grid(int64_t work, int threads, int blocks_per_sm)
{
    const int sms = device_sm_count();
    int64_t blocks = (work + threads - 1) / threads;
    int64_t cap = (int64_t)sms * blocks_per_sm;
    if (blocks > cap) blocks = cap;
    return (int)(blocks < 1 ? 1 : blocks);
}

// The five launches of one sort, with K histogram copies.
template <int K>
cudaError_t launch_sort_k(const SortArgs &a, cudaStream_t s, int narrow_blocks)
{
    const bool vec4 = a.q_stride == 4 && (reinterpret_cast<uintptr_t>(a.q) & 15u) == 0;
    // narrow: narrow_blocks small blocks per SM, to run beside a persistent fit kernel
    const bool narrow = narrow_blocks > 0;
    const int threads = narrow ? kSortThreads : kWideThreads;
    const int g = stream_grid(a.J, threads, narrow ? narrow_blocks : 8);
    const int64_t nblocks = (a.nbins + kScanSeg - 1) / kScanSeg;

    launch_begin(K_BIN, s);
    if (!narrow && a.nbins <= kSmemBinsMax) {
        // one slice per block, two blocks per SM (beside a fit kernel, with one
        // block per SM, the slices are too long: the global atomics win there)
        const int64_t blocks = stream_grid(a.J, kWideThreads, 2);
        const int64_t slice = (a.J + blocks - 1) / blocks;
        const size_t smem = (size_t)a.nbins * 4;
        if (vec4) bin_smem_kernel<true, K><<<(unsigned)blocks, kWideThreads, smem, s>>>(a, slice);
        else bin_smem_kernel<false, K><<<(unsigned)blocks, kWideThreads, smem, s>>>(a, slice);
    } else {
        if (vec4) bin_kernel<true, K><<<g, threads, 0, s>>>(a);
        else bin_kernel<false, K><<<g, threads, 0, s>>>(a);
    }
    launch_end(K_BIN, s);

    launch_begin(K_SCAN_REDUCE, s);
    if (a.group_max > 0) scan_reduce_grp_kernel<K, false><<<(unsigned)nblocks, kGrpThreads, 0, s>>>(a);
    else scan_reduce_kernel<K><<<(unsigned)nblocks, kScanThreads, 0, s>>>(a);
    launch_end(K_SCAN_REDUCE, s);

    launch_begin(K_SCAN_TOP, s);
    scan_top_kernel<<<1, kScanThreads, 0, s>>>(a, nblocks);
    launch_end(K_SCAN_TOP, s);

    launch_begin(K_SCAN_EMIT, s);
    if (a.group_max > 0) scan_emit_grp_kernel<K, false><<<(unsigned)nblocks, kGrpThreads, 0, s>>>(a);
    else scan_emit_kernel<K><<<(unsigned)nblocks, kScanThreads, 0, s>>>(a);
    launch_end(K_SCAN_EMIT, s);

    launch_begin(K_SCATTER, s);
    if (vec4) scatter_kernel<true, K><<<g, threads, 0, s>>>(a);
    else scatter_kernel<false, K><<<g, threads, 0, s>>>(a);
    launch_end(K_SCATTER, s);
    return cudaGetLastError();
}

// ------------------------------------------------------------ batched sort
//
// The queries of S shapes, concatenated (shape s owns rows [q_off, q_off + J)
// of the batch), are sorted in one pass of the same counting sort: a query's
// bin is its shape's bin offset plus its bin on its shape's own grid, so the
// bins of one shape are contiguous and every work item lies in one shape
// (Item.w).  Work items hold at most a.chunk queries (a tuning knob).

__global__ void __launch_bounds__(kWideThreads) bin_batched_kernel(SortArgs a)
{
    __shared__ int64_t s_off[kMaxShapes];
    load_offsets<false>(a, s_off);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < a.J; j += stride) {
        const BatchShape &sh = a.shapes[shape_of(s_off, a.S, j)];
        const float4 v = __ldg(reinterpret_cast<const float4 *>(a.q) + j);
        a.rank[j] = atomicAdd(&a.hist[sh.bin_off + batched_bin(sh, v.x, v.y, v.z)], 1u);
    }
}

__global__ void __launch_bounds__(kScanThreads) scan_reduce_batched_kernel(SortArgs a)
{
    const int64_t b0 = (int64_t)blockIdx.x * kScanSeg + (int64_t)threadIdx.x * kScanPerThread;
    unsigned long long s = 0;
#pragma unroll
    for (int k = 0; k < kScanPerThread; ++k)
        if (b0 + k < a.nbins) s += pack_chunk(a.hist[b0 + k], (uint32_t)a.chunk);
    unsigned long long total;
    block_exclusive_scan(s, total);
    if (threadIdx.x == 0) a.blocksum[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads) scan_emit_batched_kernel(SortArgs a)
{
    __shared__ int64_t s_off[kMaxShapes];
    load_offsets<true>(a, s_off);
    const uint32_t chunk = (uint32_t)a.chunk;
    const int64_t b0 = (int64_t)blockIdx.x * kScanSeg + (int64_t)threadIdx.x * kScanPerThread;
    uint32_t cnt[kScanPerThread];
    unsigned long long s = 0;
#pragma unroll
    for (int k = 0; k < kScanPerThread; ++k) {
        cnt[k] = b0 + k < a.nbins ? a.hist[b0 + k] : 0u;
        s += pack_chunk(cnt[k], chunk);
    }
    unsigned long long total;
    unsigned long long run = a.blocksum[blockIdx.x] + block_exclusive_scan(s, total);
#pragma unroll
    for (int k = 0; k < kScanPerThread; ++k) {
        if (b0 + k >= a.nbins) break;
        const uint32_t start = (uint32_t)(run & 0xffffffffull);
        const uint32_t item0 = (uint32_t)(run >> 32);
        a.hist[b0 + k] = start;
        if (cnt[k]) {
            const int sh = shape_of(s_off, a.S, b0 + k);
            int ux, uy, uz;
            cell_of_bin((uint32_t)(b0 + k - s_off[sh]), a.shapes[sh].P, ux, uy, uz);
            const int packed = ux | (uy << 10) | (uz << 20);
            const uint32_t nit = (cnt[k] + chunk - 1) / chunk;
            for (uint32_t i = 0; i < nit; ++i) {
                const uint32_t off = i * chunk;
                const uint32_t len = min(chunk, cnt[k] - off);
                a.items[item0 + i] = make_int4((int)(start + off), (int)len, packed, sh);
            }
        }
        run += pack_chunk(cnt[k], chunk);
    }
}

__global__ void __launch_bounds__(kWideThreads) scatter_batched_kernel(SortArgs a)
{
    __shared__ int64_t s_off[kMaxShapes];
    load_offsets<false>(a, s_off);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < a.J; j += stride) {
        const BatchShape &sh = a.shapes[shape_of(s_off, a.S, j)];
        const float4 v = __ldg(reinterpret_cast<const float4 *>(a.q) + j);
        const uint32_t pos = a.hist[sh.bin_off + batched_bin(sh, v.x, v.y, v.z)] + a.rank[j];
        a.sorted[pos] = v;
    }
}

}  // namespace

cudaError_t launch_sort_batched(const SortArgs &a, cudaStream_t s, int blocks_per_sm)
{
    const int g = stream_grid(a.J, kWideThreads, blocks_per_sm > 0 ? blocks_per_sm : 8);
    const int64_t nblocks = (a.nbins + kScanSeg - 1) / kScanSeg;
    launch_begin(K_BIN, s);
    bin_batched_kernel<<<g, kWideThreads, 0, s>>>(a);
    launch_end(K_BIN, s);
    launch_begin(K_SCAN_REDUCE, s);
    if (a.group_max > 0) scan_reduce_grp_kernel<1, true><<<(unsigned)nblocks, kGrpThreads, 0, s>>>(a);
    else scan_reduce_batched_kernel<<<(unsigned)nblocks, kScanThreads, 0, s>>>(a);
    launch_end(K_SCAN_REDUCE, s);
    launch_begin(K_SCAN_TOP, s);
    scan_top_kernel<<<1, kScanThreads, 0, s>>>(a, nblocks);
    launch_end(K_SCAN_TOP, s);
    launch_begin(K_SCAN_EMIT, s);
    if (a.group_max > 0) scan_emit_grp_kernel<1, true><<<(unsigned)nblocks, kGrpThreads, 0, s>>>(a);
    else scan_emit_batched_kernel<<<(unsigned)nblocks, kScanThreads, 0, s>>>(a);
    launch_end(K_SCAN_EMIT, s);
    launch_begin(K_SCATTER, s);
    scatter_batched_kernel<<<g, kWideThreads, 0, s>>>(a);
    launch_end(K_SCATTER, s);
    return cudaGetLastError();
}

// The histogram has room for hist_copies(nbins) copies; the narrow sort that
// runs beside a fit kernel uses them only on coarse grids: on finer grids its
// one block per SM does not contend on the counters, and the scatter's reads
// of four offset copies cost more than the copies save (measured at 32^3 x
// 2^22 beside the fit kernel: scatter 0.29 -> 0.35 ms with four copies).
cudaError_t launch_sort(const SortArgs &a, cudaStream_t s, int narrow_blocks)
{
    const bool copies = hist_copies(a.nbins) > 1 && (narrow_blocks <= 0 || a.nbins <= kCoarseBins);
    return copies ? launch_sort_k<kCoarseCopies>(a, s, narrow_blocks) : launch_sort_k<1>(a, s, narrow_blocks);
}


int bounds_code_sort()
{
#ifdef EFUNC_DEBUG_BOUNDS
    int c = 0, z = 0;
    if (cudaMemcpyFromSymbol(&c, g_bounds_code, sizeof c) != cudaSuccess) return -1;
    if (c != 0 && cudaMemcpyToSymbol(g_bounds_code, &z, sizeof z) != cudaSuccess) return -1;
    return c;
#else
    return 0;
#endif
}

}  // namespace efunc
