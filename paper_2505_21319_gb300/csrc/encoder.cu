// The warm-start encoder: a small BF16 3-D convolutional network that maps a
// 32^3 grid of SDF samples to a 32^3 x 13 parameter grid of the
// representation, so that a fit can start from its prediction instead of
// the N(0, 1e-3) initialisation.  The paper has no such encoder (its fits
// start from scratch, Sec. 3.4, and take ~20 minutes per shape, Sec. 5);
// the layers are
//   L1  3x3x3 conv   1 ->  32, bias, ReLU   (CUDA cores: 27 taps x 1 channel)
//   L2  3x3x3 conv  32 ->  64, bias, ReLU   (tensor cores)
//   L3  3x3x3 conv  64 -> 128, bias, ReLU   (tensor cores)
//   L4  1x1x1 conv 128 ->  13, bias         (tensor cores)
// trained on (SDF grid, fitted parameter grid) pairs with a weighted MSE.
//
// Tensor-core convolutions are implicit GEMMs (tcgen05, FP32 accumulator in
// tensor memory).  Activations are BF16, channels innermost, voxels in the
// parameter grid's order ((n, x, y, z), z fastest), channel rows padded to
// multiples of 64 (128 bytes): a tile of 128 output voxels (4 y-rows of 32
// z at one x) times one 64-channel chunk of one tap is a single TMA box of
// the input at shifted coordinates, whose out-of-range part TMA fills with
// zeros (the convolution's zero padding).  The shifts fall on the spatial
// coordinates only; the channel coordinate is always a multiple of 64.
//   forward / dgrad  D[voxel, co] += A[voxel, ci] B[co, ci] per (tap, chunk):
//                    both operands K-major (ci contiguous)
//   wgrad            D[co, ci] += dY[voxel, co] X[voxel + tap, ci] over voxel
//                    tiles: both operands MN-major (channels contiguous)
// dgrad is the forward kernel run on the output gradient with the weights
// transposed (ci <-> co) and the taps mirrored, and the ReLU of the layer
// below applied in its epilogue.
#include <cudaTypedefs.h>
#include <math.h>
#include <mutex>

#include "common.cuh"
#include "tc_conv.cuh"

namespace efunc {

efunc_status cuda_fail(cudaError_t e);

namespace {

using bf16 = __nv_bfloat16;

constexpr int kE = 32;                    // encoder grid per axis
constexpr int kEV = kE * kE * kE;         // voxels per shape
constexpr int kTileRows = 128;            // voxels per tile: 4 y-rows of 32 z
constexpr int kTilesPerShape = kEV / kTileRows;
constexpr uint32_t kTileBytes = 128 * 128;   // 128 rows of 128 bytes

enum ConvMode { CONV_RELU = 0, CONV_LINEAR_F32 = 1, CONV_DGRAD_MASK = 2 };

struct ConvArgs {
    int n_tiles;         // batch * 256
    int taps;            // 27 (3x3x3) or 1
    int cin_chunks;      // input channels / 64
    int mode;            // ConvMode
    int out_ld;          // elements per output row
    int store_cols;      // output columns stored (<= N)
    const float *bias;   // N floats (CONV_RELU, CONV_LINEAR_F32) or NULL
    const bf16 *mask;    // CONV_DGRAD_MASK: activation of the layer below, rows of out_ld
    void *out;           // BF16 (CONV_RELU, CONV_DGRAD_MASK) or FP32 (CONV_LINEAR_F32) rows
    int *err;            // set when a wait ran out
};

struct WgradArgs {
    int taps, cin_chunks, cout_blocks;   // cout_blocks = ceil(cout / 64), 1 or 2
    int n_tiles, tiles_per_cta;
    int cout, cin;                       // rows of dW written, input channels (padded)
    float *dw;                           // [cout][taps][cin], accumulated
    int *err;
};

__device__ __forceinline__ void tile_coords(int t, int &n, int &x, int &y0)
{
    n = t / kTilesPerShape;
    x = (t % kTilesPerShape) / (kE / 4);
    y0 = (t % (kE / 4)) * 4;
}

// tap = (dx + 1) * 9 + (dy + 1) * 3 + (dz + 1)
__device__ __forceinline__ void tap_offset(int tap, int taps, int &dx, int &dy, int &dz)
{
    if (taps == 1) {
        dx = dy = dz = 0;
    } else {
        dx = tap / 9 - 1;
        dy = (tap / 3) % 3 - 1;
        dz = tap % 3 - 1;
    }
}

__device__ __forceinline__ unsigned char *align1024(unsigned char *p)
{
    return reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(p) + 1023) & ~uintptr_t(1023));
}

template <int N>
constexpr int conv_stages() { return N == 128 ? 3 : 4; }

template <int N>
constexpr size_t conv_smem_bytes()
{
    return 1024 + (size_t)conv_stages<N>() * (kTileBytes + N * 128) + (2 * conv_stages<N>() + 1) * 8 + 16;
}

// Implicit-GEMM 3-D convolution over one tile of 128 output voxels and all N
// output channels: warp 0 lane 0 issues the TMA loads, warp 1 lane 0 the
// MMAs, all four warps run the epilogue (TMEM lane = tile row).
template <int N>
__global__ void __launch_bounds__(128, 1) conv_fwd_kernel(const __grid_constant__ CUtensorMap tmA,
                                                          const __grid_constant__ CUtensorMap tmB, ConvArgs a)
{
    using namespace tc;
    constexpr int S = conv_stages<N>();
    constexpr uint32_t kB = N * 128;
    constexpr uint32_t kStage = kTileBytes + kB;
    constexpr uint32_t kCols = N < 32 ? 32 : N;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = align1024(smem_raw);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + S * kStage);
    uint64_t *empty = full + S;
    uint64_t *done = empty + S;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        fence_barrier_init();
    }
    if (warp == 0) tmem_alloc(tmem_slot, kCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    int n, x, y0;
    tile_coords(blockIdx.x, n, x, y0);
    const int iters = a.taps * a.cin_chunks;

    if (warp == 0 && lane == 0) {
        for (int i = 0; i < iters; ++i) {
            const int s = i % S;
            const uint32_t ph = (uint32_t)(i / S) & 1u;
            if (!mbar_wait(&empty[s], ph ^ 1u, a.err, 1)) break;
            const int tap = i / a.cin_chunks, kc = i % a.cin_chunks;
            int dx, dy, dz;
            tap_offset(tap, a.taps, dx, dy, dz);
            unsigned char *sa = smem + s * kStage;
            mbar_expect_tx(&full[s], kStage);
            tma_load_5d(sa, &tmA, &full[s], kc * 64, dz, y0 + dy, x + dx, n);
            tma_load_2d(sa + kTileBytes, &tmB, &full[s], (tap * a.cin_chunks + kc) * 64, 0);
        }
    } else if (warp == 1 && lane == 0) {
        constexpr uint32_t idesc = idesc_bf16(128, N, 0, 0);
        for (int i = 0; i < iters; ++i) {
            const int s = i % S;
            const uint32_t ph = (uint32_t)(i / S) & 1u;
            if (!mbar_wait(&full[s], ph, a.err, 2)) break;
            tc_fence_after();
            const uint32_t sa = smem_u32(smem + s * kStage), sb = sa + kTileBytes;
#pragma unroll
            for (int k = 0; k < 4; ++k)   // K = 16 per MMA: 32 bytes along the swizzled row
                mma_bf16(tmem, smem_desc(sa + 32 * k, 16, 1024), smem_desc(sb + 32 * k, 16, 1024), idesc,
                         (i | k) != 0);
            mma_commit(&empty[s]);   // the stage is free once these MMAs have read it
        }
        mma_commit(done);
    }
    __syncwarp();
    // warp-uniform: the TMEM loads below are .sync.aligned
    const bool ok = __all_sync(0xffffffffu, mbar_wait(done, 0, a.err, 3));
    tc_fence_after();
    if (ok) {
        const int m = warp * 32 + lane;
        const size_t v = (((size_t)n * kE + x) * kE + (y0 + warp)) * kE + lane;
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
        if (a.mode == CONV_LINEAR_F32) {
            float vals[16];
            float *o = static_cast<float *>(a.out) + v * a.out_ld;
#pragma unroll
            for (int c0 = 0; c0 < N; c0 += 16) {
                tmem_ld16(trow + c0, vals);
#pragma unroll
                for (int i = 0; i < 16; ++i)
                    if (c0 + i < a.store_cols) o[c0 + i] = vals[i] + (a.bias ? a.bias[c0 + i] : 0.f);
            }
        } else {
            bf16 *o = static_cast<bf16 *>(a.out) + v * a.out_ld;
            const bf16 *mk = a.mask ? a.mask + v * a.out_ld : nullptr;
#pragma unroll 1
            for (int c0 = 0; c0 < N; c0 += 32) {
                float vals[32];
                if (N >= 32) tmem_ld32(trow + c0, vals);
                else {
                    tmem_ld16(trow + c0, vals);
#pragma unroll
                    for (int i = 16; i < 32; ++i) vals[i] = 0.f;
                }
                uint32_t packed[16];
                if (a.mode == CONV_RELU) {
#pragma unroll
                    for (int i = 0; i < 32; ++i) vals[i] = fmaxf(vals[i] + (a.bias ? a.bias[c0 + i] : 0.f), 0.f);
                } else {
                    const uint4 *mv = reinterpret_cast<const uint4 *>(mk + c0);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const uint4 w4 = mv[q];
                        const uint32_t ws[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
                        for (int h = 0; h < 4; ++h) {
                            const __nv_bfloat162 pr = *reinterpret_cast<const __nv_bfloat162 *>(&ws[h]);
                            if (!(__low2float(pr) > 0.f)) vals[q * 8 + 2 * h] = 0.f;
                            if (!(__high2float(pr) > 0.f)) vals[q * 8 + 2 * h + 1] = 0.f;
                        }
                    }
                }
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const __nv_bfloat162 pr = __floats2bfloat162_rn(vals[2 * i], vals[2 * i + 1]);
                    packed[i] = *reinterpret_cast<const uint32_t *>(&pr);
                }
                uint4 *dst = reinterpret_cast<uint4 *>(o + c0);
                const int nvec = (N >= 32 ? 32 : 16) / 8;
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (q < nvec) dst[q] = make_uint4(packed[4 * q], packed[4 * q + 1], packed[4 * q + 2], packed[4 * q + 3]);
            }
        }
        (void)m;
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, kCols);
}

constexpr int kWgradStages = 3;
constexpr uint32_t kWgradStage = 3 * kTileBytes;   // two dY blocks (co 0-63, 64-127) + one X block
constexpr size_t kWgradSmem = 1024 + (size_t)kWgradStages * kWgradStage + (2 * kWgradStages + 1) * 8 + 16;

// Weight gradient of one (tap, 64-input-channel chunk) over a range of voxel
// tiles: D[co, ci] += sum_voxels dY[voxel, co] X[voxel + tap, ci], M = 128
// output channels (two 64-channel blocks of dY; rows >= cout are not
// written), N = 64, K = 128 voxels per tile in 8 MMAs; both operands
// MN-major.  Partial sums are added to dw with FP32 atomics.
__global__ void __launch_bounds__(128, 1) conv_wgrad_kernel(const __grid_constant__ CUtensorMap tmDY,
                                                            const __grid_constant__ CUtensorMap tmX, WgradArgs a)
{
    using namespace tc;
    constexpr int S = kWgradStages;
    constexpr uint32_t kCols = 64;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = align1024(smem_raw);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + S * kWgradStage);
    uint64_t *empty = full + S;
    uint64_t *done = empty + S;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        fence_barrier_init();
    }
    if (warp == 0) tmem_alloc(tmem_slot, kCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int tap = blockIdx.x / a.cin_chunks, kc = blockIdx.x % a.cin_chunks;
    int dx, dy, dz;
    tap_offset(tap, a.taps, dx, dy, dz);
    const int t0 = blockIdx.y * a.tiles_per_cta;
    const int t1 = min(t0 + a.tiles_per_cta, a.n_tiles);
    const int iters = max(t1 - t0, 0);
    const uint32_t bytes = (uint32_t)(a.cout_blocks + 1) * kTileBytes;

    if (warp == 0 && lane == 0) {
        for (int i = 0; i < iters; ++i) {
            const int s = i % S;
            const uint32_t ph = (uint32_t)(i / S) & 1u;
            if (!mbar_wait(&empty[s], ph ^ 1u, a.err, 11)) break;
            int n, x, y0;
            tile_coords(t0 + i, n, x, y0);
            unsigned char *st = smem + s * kWgradStage;
            mbar_expect_tx(&full[s], bytes);
            for (int cb = 0; cb < a.cout_blocks; ++cb)
                tma_load_5d(st + cb * kTileBytes, &tmDY, &full[s], cb * 64, 0, y0, x, n);
            tma_load_5d(st + 2 * kTileBytes, &tmX, &full[s], kc * 64, dz, y0 + dy, x + dx, n);
        }
    } else if (warp == 1 && lane == 0) {
        constexpr uint32_t idesc = idesc_bf16(128, 64, 1, 1);
        for (int i = 0; i < iters; ++i) {
            const int s = i % S;
            const uint32_t ph = (uint32_t)(i / S) & 1u;
            if (!mbar_wait(&full[s], ph, a.err, 12)) break;
            tc_fence_after();
            const uint32_t sa = smem_u32(smem + s * kWgradStage), sb = sa + 2 * kTileBytes;
#pragma unroll
            for (int k = 0; k < 8; ++k)   // 16 voxels (rows) per MMA: two 8-row groups of 1024 bytes
                mma_bf16(tmem, smem_desc(sa + 2048 * k, kTileBytes, 1024), smem_desc(sb + 2048 * k, kTileBytes, 1024),
                         idesc, (i | k) != 0);
            mma_commit(&empty[s]);
        }
        mma_commit(done);
    }
    __syncwarp();
    const bool ok = __all_sync(0xffffffffu, mbar_wait(done, 0, a.err, 13)) && iters > 0;
    tc_fence_after();
    const int co = warp * 32 + lane;
    if (ok) {
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
        for (int c0 = 0; c0 < 64; c0 += 32) {
            float vals[32];
            tmem_ld32(trow + c0, vals);
            if (co < a.cout) {
                float *d = a.dw + ((size_t)co * a.taps + tap) * a.cin + kc * 64 + c0;
#pragma unroll
                for (int i = 0; i < 32; ++i) atomicAdd(d + i, vals[i]);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, kCols);
}

// ---------------------------------------------------------- CUDA cores

// Master FP32 weights, one flat array.
constexpr int kC1 = 32, kC2 = 64, kC3 = 128, kC4 = 13;
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kC1 * 27;
constexpr int kOffW2 = kOffB1 + kC1;
constexpr int kOffB2 = kOffW2 + kC2 * 27 * kC1;
constexpr int kOffW3 = kOffB2 + kC2;
constexpr int kOffB3 = kOffW3 + kC3 * 27 * kC2;
constexpr int kOffW4 = kOffB3 + kC3;
constexpr int kOffB4 = kOffW4 + kC4 * kC3;
constexpr int kWeights = kOffB4 + kC4;

__device__ __forceinline__ float sdf_at(const float *sdf, int n, int x, int y, int z)
{
    if ((unsigned)x >= (unsigned)kE || (unsigned)y >= (unsigned)kE || (unsigned)z >= (unsigned)kE) return 0.f;
    return __ldg(sdf + (((size_t)n * kE + x) * kE + y) * kE + z);
}

// L1: 3x3x3 conv 1 -> 32 + bias + ReLU, written as 64 BF16 channels (32..63 zero).
__global__ void __launch_bounds__(128) l1_forward_kernel(const float *w, const float *sdf, int64_t V, bf16 *out)
{
    __shared__ float sw[kC1 * 27 + kC1];
    for (int i = threadIdx.x; i < kC1 * 28; i += blockDim.x) sw[i] = w[kOffW1 + i];
    __syncthreads();
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x) {
        const int z = v % kE, y = (v / kE) % kE, x = (v / (kE * kE)) % kE, n = (int)(v / kEV);
        float s[27];
#pragma unroll
        for (int t = 0; t < 27; ++t) s[t] = sdf_at(sdf, n, x + t / 9 - 1, y + (t / 3) % 3 - 1, z + t % 3 - 1);
        uint32_t packed[32];
#pragma unroll 4
        for (int c = 0; c < kC1; c += 2) {
            float a0 = sw[kC1 * 27 + c], a1 = sw[kC1 * 27 + c + 1];
#pragma unroll
            for (int t = 0; t < 27; ++t) {
                a0 = fmaf(sw[c * 27 + t], s[t], a0);
                a1 = fmaf(sw[(c + 1) * 27 + t], s[t], a1);
            }
            const __nv_bfloat162 pr = __floats2bfloat162_rn(fmaxf(a0, 0.f), fmaxf(a1, 0.f));
            packed[c / 2] = *reinterpret_cast<const uint32_t *>(&pr);
        }
#pragma unroll
        for (int c = 16; c < 32; ++c) packed[c] = 0u;
        uint4 *dst = reinterpret_cast<uint4 *>(out + v * 64);
#pragma unroll
        for (int q = 0; q < 8; ++q) dst[q] = make_uint4(packed[4 * q], packed[4 * q + 1], packed[4 * q + 2], packed[4 * q + 3]);
    }
}

// L1 weight and bias gradients: dW1[c][t] = sum_v dPre1[v][c] sdf[v + tap t],
// db1[c] = sum_v dPre1[v][c]; one block per x-slab of one shape, in chunks
// of 4 y-rows (128 voxels) staged in shared memory, one thread per (c, t)
// pair (t = 27: the bias).
__global__ void __launch_bounds__(256) l1_wgrad_kernel(const bf16 *dpre, const float *sdf, float *grad)
{
    constexpr int kRows = 4;
    __shared__ float sd[kRows * kE][kC1 + 1];
    __shared__ float ss[3][kRows + 2][kE + 2];
    const int n = blockIdx.x / kE, x = blockIdx.x % kE;
    constexpr int kPairs = kC1 * 28;
    constexpr int kPer = (kPairs + 255) / 256;
    float acc[kPer];
#pragma unroll
    for (int k = 0; k < kPer; ++k) acc[k] = 0.f;
    for (int y0 = 0; y0 < kE; y0 += kRows) {
        __syncthreads();
        for (int i = threadIdx.x; i < kRows * kE * kC1; i += blockDim.x) {
            const int vv = i / kC1, c = i % kC1;
            sd[vv][c] = __bfloat162float(dpre[(((size_t)blockIdx.x * kE) + y0) * kE * 64 + (size_t)vv * 64 + c]);
        }
        for (int i = threadIdx.x; i < 3 * (kRows + 2) * (kE + 2); i += blockDim.x) {
            const int dx = i / ((kRows + 2) * (kE + 2)), r = i % ((kRows + 2) * (kE + 2));
            const int y = y0 + r / (kE + 2) - 1, z = r % (kE + 2) - 1;
            ss[dx][r / (kE + 2)][r % (kE + 2)] = sdf_at(sdf, n, x + dx - 1, y, z);
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const int p = threadIdx.x + 256 * k;
            if (p >= kPairs) break;
            const int c = p / 28, t = p % 28;
            float a = acc[k];
            if (t == 27) {
                for (int vv = 0; vv < kRows * kE; ++vv) a += sd[vv][c];
            } else {
                const int dx = t / 9, dy = (t / 3) % 3 - 1, dz = t % 3 - 1;
                for (int vv = 0; vv < kRows * kE; ++vv)
                    a = fmaf(sd[vv][c], ss[dx][vv / kE + dy + 1][vv % kE + dz + 1], a);
            }
            acc[k] = a;
        }
    }
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        const int p = threadIdx.x + 256 * k;
        if (p >= kPairs) break;
        const int c = p / 28, t = p % 28;
        atomicAdd(grad + (t == 27 ? kOffB1 + c : kOffW1 + c * 27 + t), acc[k]);
    }
}

// Bias gradient: grad[off + c] += sum_v dpre[v][c], c < C (rows of ld BF16).
__global__ void __launch_bounds__(256) bias_grad_kernel(const bf16 *dpre, int64_t V, int C, int ld, float *grad, int off)
{
    const int c = threadIdx.x % C;
    const int lanes = blockDim.x / C;
    const int r = threadIdx.x / C;
    float acc = 0.f;
    if (r < lanes)
        for (int64_t v = (int64_t)blockIdx.x * lanes + r; v < V; v += (int64_t)gridDim.x * lanes)
            acc += __bfloat162float(dpre[v * ld + c]);
    __shared__ float red[256];
    red[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x < C) {
        float s = 0.f;
        for (int i = 0; i < lanes; ++i) s += red[i * C + threadIdx.x];
        atomicAdd(grad + off + threadIdx.x, s);
    }
}

// Weighted MSE of the predicted parameters: L = sum_v sum_s w_s (p - t)^2 / V;
// dOut[v][s] = 2 w_s (p - t) / V in BF16 rows of 64 (s >= 13 zero); the
// output bias gradient and the loss sum (FP64) are accumulated.
__global__ void __launch_bounds__(256) loss_kernel(const float *pred, const float *target, const float *slot_w,
                                                   int64_t V, bf16 *dout, float *grad, double *loss)
{
    __shared__ float sw[kC4];
    __shared__ float sdb[kC4];
    __shared__ double sl;
    if (threadIdx.x < kC4) {
        sw[threadIdx.x] = slot_w ? slot_w[threadIdx.x] : 1.f;
        sdb[threadIdx.x] = 0.f;
    }
    if (threadIdx.x == 0) sl = 0.0;
    __syncthreads();
    const float inv = 1.f / (float)V;
    float db[kC4];
#pragma unroll
    for (int s = 0; s < kC4; ++s) db[s] = 0.f;
    double l = 0.0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x) {
        float g[16];
#pragma unroll
        for (int s = 0; s < 16; ++s) g[s] = 0.f;
#pragma unroll
        for (int s = 0; s < kC4; ++s) {
            const float d = pred[v * kC4 + s] - target[v * kC4 + s];
            l += (double)(sw[s] * d * d);
            g[s] = 2.f * sw[s] * d * inv;
            db[s] += g[s];
        }
        uint32_t packed[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const __nv_bfloat162 pr = __floats2bfloat162_rn(g[2 * i], g[2 * i + 1]);
            packed[i] = *reinterpret_cast<const uint32_t *>(&pr);
        }
        uint4 *dst = reinterpret_cast<uint4 *>(dout + v * 64);
        dst[0] = make_uint4(packed[0], packed[1], packed[2], packed[3]);
        dst[1] = make_uint4(packed[4], packed[5], packed[6], packed[7]);
#pragma unroll
        for (int q = 2; q < 8; ++q) dst[q] = make_uint4(0u, 0u, 0u, 0u);
    }
#pragma unroll
    for (int s = 0; s < kC4; ++s) atomicAdd(&sdb[s], db[s]);
    atomicAdd(&sl, l);
    __syncthreads();
    if (threadIdx.x < kC4) atomicAdd(grad + kOffB4 + threadIdx.x, sdb[threadIdx.x]);
    if (threadIdx.x == 0) atomicAdd(loss, sl * (double)inv);
}

// BF16 weight layouts of the tensor-core layers from the FP32 master weights:
//   forward  W2f [64][27][64]  (input channels 32..63 zero), W3f [128][27][64],
//            W4f [16][128] (rows 13..15 zero), b4p [16]
//   dgrad    W3d [64][27][128] = W3[co][26 - t][ci] (ci as rows, taps mirrored),
//            W2d [64][27][64]  = W2[co][26 - t][ci] (rows ci >= 32 zero),
//            W4d [128][64]     = W4[co][ci] (columns co >= 13 zero)
struct WeightViews {
    bf16 *w2f, *w3f, *w4f, *w2d, *w3d, *w4d;
    float *b4p;
};

__global__ void __launch_bounds__(256) prep_weights_kernel(const float *w, WeightViews o)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t i = t0; i < 64 * 27 * 64; i += stride) {   // W2f, W2d
        const int ci = i % 64, t = (i / 64) % 27, co = (int)(i / (64 * 27));
        o.w2f[i] = __float2bfloat16(ci < kC1 ? w[kOffW2 + (co * 27 + t) * kC1 + ci] : 0.f);
        // W2d row r = input channel of L2 (padded to 64), column (t', co)
        const int r = co, tp = t, cc = ci;   // reuse the index split: r < 64, tp < 27, cc < 64
        o.w2d[i] = __float2bfloat16(r < kC1 ? w[kOffW2 + (cc * 27 + (26 - tp)) * kC1 + r] : 0.f);
    }
    for (int64_t i = t0; i < 128 * 27 * 64; i += stride) {   // W3f [128][27][64]
        o.w3f[i] = __float2bfloat16(w[kOffW3 + i]);
    }
    for (int64_t i = t0; i < 64 * 27 * 128; i += stride) {   // W3d [64][27][128]
        const int co = i % 128, t = (i / 128) % 27, ci = (int)(i / (128 * 27));
        o.w3d[i] = __float2bfloat16(w[kOffW3 + (co * 27 + (26 - t)) * kC2 + ci]);
    }
    for (int64_t i = t0; i < 16 * 128; i += stride) {   // W4f [16][128]
        const int ci = i % 128, co = (int)(i / 128);
        o.w4f[i] = __float2bfloat16(co < kC4 ? w[kOffW4 + co * kC3 + ci] : 0.f);
    }
    for (int64_t i = t0; i < 128 * 64; i += stride) {   // W4d [128][64]
        const int co = i % 64, ci = (int)(i / 64);
        o.w4d[i] = __float2bfloat16(co < kC4 ? w[kOffW4 + co * kC3 + ci] : 0.f);
    }
    if (t0 < 16) o.b4p[t0] = t0 < kC4 ? w[kOffB4 + t0] : 0.f;
}

// Padded FP32 weight gradients -> the master gradient array.
__global__ void __launch_bounds__(256) gather_grads_kernel(const float *dw2p, const float *dw3p, const float *dw4p,
                                                           float *grad)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t i = t0; i < kC2 * 27 * kC1; i += stride) {   // dW2 [64][27][32] from [64][27][64]
        const int ci = i % kC1, rest = (int)(i / kC1);
        grad[kOffW2 + i] = dw2p[rest * 64 + ci];
    }
    for (int64_t i = t0; i < kC3 * 27 * kC2; i += stride) grad[kOffW3 + i] = dw3p[i];
    for (int64_t i = t0; i < kC4 * kC3; i += stride) grad[kOffW4 + i] = dw4p[i];
}

// ------------------------------------------------------------ host side

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static std::mutex mu;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::lock_guard<std::mutex> lk(mu);
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// 5-D map of activations [batch][32][32][32][C] BF16, box of one tile row
// block: 64 channels x 32 z x 4 y x 1 x x 1 shape, 128-byte swizzle.
bool act_map(CUtensorMap *m, const void *base, int batch, int C)
{
    auto fn = encode_fn();
    if (!fn || (reinterpret_cast<uintptr_t>(base) & 15u) || C % 64) return false;
    const cuuint64_t dims[5] = {(cuuint64_t)C, kE, kE, kE, (cuuint64_t)batch};
    const cuuint64_t strides[4] = {(cuuint64_t)C * 2, (cuuint64_t)C * 2 * kE, (cuuint64_t)C * 2 * kE * kE,
                                   (cuuint64_t)C * 2 * kE * kE * kE};
    const cuuint32_t box[5] = {64, kE, 4, 1, 1};
    const cuuint32_t es[5] = {1, 1, 1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void *>(base), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// 2-D map of weights [rows][K] BF16, box 64 x rows, 128-byte swizzle.
bool weight_map(CUtensorMap *m, const void *base, int rows, int K)
{
    auto fn = encode_fn();
    if (!fn || (reinterpret_cast<uintptr_t>(base) & 15u) || K % 64 || rows > 256) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)K * 2};
    const cuuint32_t box[2] = {64, (cuuint32_t)rows};
    const cuuint32_t es[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <class K>
cudaError_t set_smem(K kernel, size_t bytes)
{
    cudaError_t e = cudaSuccess;
    per_device_cached(reinterpret_cast<const void *>(kernel), 0, [&] {
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        return e == cudaSuccess ? 1 : 0;
    });
    return e;
}

}  // namespace

// One implicit-GEMM convolution (forward, or dgrad with transposed mirrored
// weights): x [batch][32^3][cin] BF16, w [N][taps * cin] BF16.
cudaError_t enc_conv(const bf16 *x, int batch, int cin, const bf16 *w, int N, int taps, const float *bias, int mode,
                     const bf16 *mask, void *out, int out_ld, int store_cols, int *err, cudaStream_t s)
{
    CUtensorMap ma, mb;
    if (!act_map(&ma, x, batch, cin) || !weight_map(&mb, w, N, taps * cin)) return cudaErrorInvalidValue;
    ConvArgs a{};
    a.n_tiles = batch * kTilesPerShape;
    a.taps = taps;
    a.cin_chunks = cin / 64;
    a.mode = mode;
    a.out_ld = out_ld;
    a.store_cols = store_cols;
    a.bias = bias;
    a.mask = mask;
    a.out = out;
    a.err = err;
    cudaError_t e = cudaSuccess;
    switch (N) {   // the kernels' dynamic shared-memory limits, before the launch
    case 16: e = set_smem(conv_fwd_kernel<16>, conv_smem_bytes<16>()); break;
    case 32: e = set_smem(conv_fwd_kernel<32>, conv_smem_bytes<32>()); break;
    case 64: e = set_smem(conv_fwd_kernel<64>, conv_smem_bytes<64>()); break;
    case 128: e = set_smem(conv_fwd_kernel<128>, conv_smem_bytes<128>()); break;
    default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    launch_begin(K_ENC_CONV, s);
    switch (N) {
    case 16: conv_fwd_kernel<16><<<a.n_tiles, 128, conv_smem_bytes<16>(), s>>>(ma, mb, a); break;
    case 32: conv_fwd_kernel<32><<<a.n_tiles, 128, conv_smem_bytes<32>(), s>>>(ma, mb, a); break;
    case 64: conv_fwd_kernel<64><<<a.n_tiles, 128, conv_smem_bytes<64>(), s>>>(ma, mb, a); break;
    default: conv_fwd_kernel<128><<<a.n_tiles, 128, conv_smem_bytes<128>(), s>>>(ma, mb, a); break;
    }
    launch_end(K_ENC_CONV, s);
    return cudaGetLastError();
}

// Weight gradient dw [cout][taps][cin] += sum over voxels of dy (rows of
// dy_ld >= cout channels, a multiple of 64) times x shifted by the tap.
cudaError_t enc_wgrad(const bf16 *dy, int dy_ld, int cout, const bf16 *x, int cin, int batch, int taps, float *dw,
                      int *err, cudaStream_t s)
{
    CUtensorMap md, mx;
    if (cout > 128 || !act_map(&md, dy, batch, dy_ld) || !act_map(&mx, x, batch, cin)) return cudaErrorInvalidValue;
    WgradArgs a{};
    a.taps = taps;
    a.cin_chunks = cin / 64;
    a.cout_blocks = cout > 64 ? 2 : 1;
    a.n_tiles = batch * kTilesPerShape;
    a.cout = cout;
    a.cin = cin;
    a.dw = dw;
    a.err = err;
    // split the voxel tiles so that the grid fills the GPU at least twice
    // (one CTA per SM fits) with the last wave as full as possible
    const int cells = taps * a.cin_chunks, sms = device_sm_count();
    const int split0 = max(1, min((2 * sms + cells - 1) / cells, a.n_tiles));
    int split = split0;
    double best = 0.0;
    for (int sp = split0; sp <= min(4 * split0, a.n_tiles); ++sp) {
        const int per = (a.n_tiles + sp - 1) / sp, eff = (a.n_tiles + per - 1) / per;
        const int ctas = cells * eff, waves = (ctas + sms - 1) / sms;
        const double fill = (double)ctas / ((double)waves * sms);
        if (fill > best + 1e-9) {
            best = fill;
            split = eff;
        }
    }
    a.tiles_per_cta = (a.n_tiles + split - 1) / split;
    split = (a.n_tiles + a.tiles_per_cta - 1) / a.tiles_per_cta;
    cudaError_t e = set_smem(conv_wgrad_kernel, kWgradSmem);
    if (e != cudaSuccess) return e;
    launch_begin(K_ENC_WGRAD, s);
    conv_wgrad_kernel<<<dim3(cells, split), 128, kWgradSmem, s>>>(md, mx, a);
    launch_end(K_ENC_WGRAD, s);
    return cudaGetLastError();
}

namespace {

// Workspace of the encoder calls for a batch of B shapes (V = B * 32^3).
struct EncLayout {
    size_t flags, w2f, w3f, w4f, w2d, w3d, w4d, b4p, dw2p, dw3p, dw4p, act1, act2, act3, pred, dout, dpre3, dpre2,
        dpre1, total;
};

EncLayout enc_layout(int64_t B)
{
    const int64_t V = B * kEV;
    EncLayout L{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t at = off;
        off = (off + bytes + 255) / 256 * 256;
        return at;
    };
    L.flags = take(256);   // int error flag at 0, double loss sum at 8
    L.w2f = take((size_t)64 * 27 * 64 * 2);
    L.w3f = take((size_t)128 * 27 * 64 * 2);
    L.w4f = take((size_t)16 * 128 * 2);
    L.w2d = take((size_t)64 * 27 * 64 * 2);
    L.w3d = take((size_t)64 * 27 * 128 * 2);
    L.w4d = take((size_t)128 * 64 * 2);
    L.b4p = take(16 * 4);
    L.dw2p = take((size_t)64 * 27 * 64 * 4);
    L.dw3p = take((size_t)128 * 27 * 64 * 4);
    L.dw4p = take((size_t)16 * 128 * 4);
    L.act1 = take((size_t)V * 64 * 2);
    L.act2 = take((size_t)V * 64 * 2);
    L.act3 = take((size_t)V * 128 * 2);
    L.pred = take((size_t)V * kC4 * 4);
    L.dout = take((size_t)V * 64 * 2);
    L.dpre3 = take((size_t)V * 128 * 2);
    L.dpre2 = take((size_t)V * 64 * 2);
    L.dpre1 = take((size_t)V * 64 * 2);
    L.total = off;
    return L;
}

struct Enc {
    EncLayout L;
    char *b;
    template <class T> T *at(size_t off) const { return reinterpret_cast<T *>(b + off); }
    int *err() const { return at<int>(L.flags); }
    double *loss() const { return reinterpret_cast<double *>(b + L.flags + 8); }
    WeightViews views() const
    {
        return {at<bf16>(L.w2f), at<bf16>(L.w3f), at<bf16>(L.w4f), at<bf16>(L.w2d), at<bf16>(L.w3d),
                at<bf16>(L.w4d), at<float>(L.b4p)};
    }
};

int grid_for(int64_t n, int threads)
{
    int64_t g = (n + threads - 1) / threads;
    const int64_t cap = (int64_t)device_sm_count() * 8;
    return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

__global__ void loss_finish_kernel(const double *sum, float *out) { *out = (float)*sum; }

// Forward of the encoder into params [V][13] (FP32); activations kept in
// the workspace for a backward.
cudaError_t enc_forward(const Enc &E, const float *w, const float *sdf, int B, float *params, cudaStream_t s)
{
    const int64_t V = (int64_t)B * kEV;
    launch_begin(K_ENC_AUX, s);
    prep_weights_kernel<<<grid_for(128 * 27 * 64, 256), 256, 0, s>>>(w, E.views());
    launch_end(K_ENC_AUX, s);
    launch_begin(K_ENC_AUX, s);
    l1_forward_kernel<<<grid_for(V, 128), 128, 0, s>>>(w, sdf, V, E.at<bf16>(E.L.act1));
    launch_end(K_ENC_AUX, s);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if ((e = enc_conv(E.at<bf16>(E.L.act1), B, 64, E.at<bf16>(E.L.w2f), 64, 27, w + kOffB2, CONV_RELU, nullptr,
                      E.at<bf16>(E.L.act2), 64, 64, E.err(), s)) != cudaSuccess)
        return e;
    if ((e = enc_conv(E.at<bf16>(E.L.act2), B, 64, E.at<bf16>(E.L.w3f), 128, 27, w + kOffB3, CONV_RELU, nullptr,
                      E.at<bf16>(E.L.act3), 128, 128, E.err(), s)) != cudaSuccess)
        return e;
    return enc_conv(E.at<bf16>(E.L.act3), B, 128, E.at<bf16>(E.L.w4f), 16, 1, E.at<float>(E.L.b4p),
                    CONV_LINEAR_F32, nullptr, params, kC4, kC4, E.err(), s);
}

efunc_status check_enc(const void *ws, size_t ws_bytes, int32_t batch, EncLayout &L)
{
    if (batch < 1 || batch > 4096) return EFUNC_ERR_ARG;
    L = enc_layout(batch);
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u) || ws_bytes < L.total) return EFUNC_ERR_WORKSPACE;
    if (!encode_fn()) return EFUNC_ERR_UNSUPPORTED;
    return EFUNC_OK;
}

}  // namespace
}  // namespace efunc

using namespace efunc;

extern "C" {

int64_t efunc_encoder_weight_count(void) { return kWeights; }

size_t efunc_encoder_workspace_bytes(int32_t batch)
{
    if (batch < 1 || batch > 4096) return 0;
    return enc_layout(batch).total;
}

efunc_status efunc_encoder_forward(const float *weights, const float *sdf, int32_t batch, float *params,
                                   void *workspace, size_t workspace_bytes, efunc_stream_t stream)
{
    EncLayout L;
    efunc_status st = check_enc(workspace, workspace_bytes, batch, L);
    if (st) return st;
    if (!weights || !sdf || !params) return EFUNC_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    Enc E{L, static_cast<char *>(workspace)};
    if (cudaMemsetAsync(E.err(), 0, 16, s) != cudaSuccess) return cuda_fail(cudaSuccess);
    const cudaError_t e = enc_forward(E, weights, sdf, batch, params, s);
    return e == cudaSuccess ? EFUNC_OK : cuda_fail(e);
}

efunc_status efunc_encoder_train_step(const float *weights, const float *sdf, const float *target,
                                      const float *slot_weights, int32_t batch, float *grad, float *loss,
                                      void *workspace, size_t workspace_bytes, efunc_stream_t stream)
{
    EncLayout L;
    efunc_status st = check_enc(workspace, workspace_bytes, batch, L);
    if (st) return st;
    if (!weights || !sdf || !target || !grad || !loss) return EFUNC_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    Enc E{L, static_cast<char *>(workspace)};
    const int64_t V = (int64_t)batch * kEV;
    cudaError_t e = cudaMemsetAsync(E.err(), 0, 16, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(grad, 0, (size_t)kWeights * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(E.b + L.dw2p, 0, L.act1 - L.dw2p, s);   // the padded gradients
    if (e == cudaSuccess) e = enc_forward(E, weights, sdf, batch, E.at<float>(L.pred), s);
    if (e != cudaSuccess) return cuda_fail(e);
    bf16 *dout = E.at<bf16>(L.dout), *dpre3 = E.at<bf16>(L.dpre3), *dpre2 = E.at<bf16>(L.dpre2),
         *dpre1 = E.at<bf16>(L.dpre1);
    const bf16 *act1 = E.at<bf16>(L.act1), *act2 = E.at<bf16>(L.act2), *act3 = E.at<bf16>(L.act3);
    const WeightViews W = E.views();
    launch_begin(K_ENC_AUX, s);
    loss_kernel<<<grid_for(V, 256), 256, 0, s>>>(E.at<float>(L.pred), target, slot_weights, V, dout, grad, E.loss());
    launch_end(K_ENC_AUX, s);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e);
    // L4: weight gradient, then the gradient through it with the ReLU of L3
    if ((e = enc_wgrad(dout, 64, 16, act3, 128, batch, 1, E.at<float>(L.dw4p), E.err(), s)) != cudaSuccess ||
        (e = enc_conv(dout, batch, 64, W.w4d, 128, 1, nullptr, CONV_DGRAD_MASK, act3, dpre3, 128, 128, E.err(), s)) !=
            cudaSuccess)
        return cuda_fail(e);
    launch_begin(K_ENC_AUX, s);
    bias_grad_kernel<<<grid_for(V / 64, 256), 256, 0, s>>>(dpre3, V, 128, 128, grad, kOffB3);
    launch_end(K_ENC_AUX, s);
    // L3
    if ((e = enc_wgrad(dpre3, 128, 128, act2, 64, batch, 27, E.at<float>(L.dw3p), E.err(), s)) != cudaSuccess ||
        (e = enc_conv(dpre3, batch, 128, W.w3d, 64, 27, nullptr, CONV_DGRAD_MASK, act2, dpre2, 64, 64, E.err(), s)) !=
            cudaSuccess)
        return cuda_fail(e);
    launch_begin(K_ENC_AUX, s);
    bias_grad_kernel<<<grid_for(V / 64, 256), 256, 0, s>>>(dpre2, V, 64, 64, grad, kOffB2);
    launch_end(K_ENC_AUX, s);
    // L2
    if ((e = enc_wgrad(dpre2, 64, 64, act1, 64, batch, 27, E.at<float>(L.dw2p), E.err(), s)) != cudaSuccess ||
        (e = enc_conv(dpre2, batch, 64, W.w2d, 64, 27, nullptr, CONV_DGRAD_MASK, act1, dpre1, 64, 64, E.err(), s)) !=
            cudaSuccess)
        return cuda_fail(e);
    // L1 and the gathered gradient
    launch_begin(K_ENC_AUX, s);
    l1_wgrad_kernel<<<batch * kE, 256, 0, s>>>(dpre1, sdf, grad);
    launch_end(K_ENC_AUX, s);
    launch_begin(K_ENC_AUX, s);
    gather_grads_kernel<<<grid_for(128 * 27 * 64, 256), 256, 0, s>>>(E.at<float>(L.dw2p), E.at<float>(L.dw3p),
                                                                     E.at<float>(L.dw4p), grad);
    launch_end(K_ENC_AUX, s);
    launch_begin(K_ENC_AUX, s);
    loss_finish_kernel<<<1, 1, 0, s>>>(E.loss(), loss);
    launch_end(K_ENC_AUX, s);
    return (e = cudaGetLastError()) == cudaSuccess ? EFUNC_OK : cuda_fail(e);
}

efunc_status efunc_encoder_status(const void *workspace)
{
    if (!workspace) return EFUNC_ERR_ARG;
    int flag = 0;
    if (cudaMemcpy(&flag, workspace, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return cuda_fail(cudaSuccess);
    return flag ? EFUNC_ERR_TIMEOUT : EFUNC_OK;
}

efunc_status efunc_conv3d_bf16(const void *x, int32_t batch, int32_t cin, const void *w, int32_t cout, int32_t taps,
                               const float *bias, int32_t mode, const void *mask, void *out, int32_t out_ld,
                               int32_t store_cols, int32_t *err, efunc_stream_t stream)
{
    if (!x || !w || !out || !err || batch < 1 || cin < 64 || cin % 64 || cin > 256 || (taps != 1 && taps != 27) ||
        (cout != 16 && cout != 32 && cout != 64 && cout != 128) || mode < 0 || mode > 2 || out_ld < 1 ||
        store_cols < 1 || store_cols > cout || (mode == CONV_DGRAD_MASK && !mask) ||
        (mode != CONV_LINEAR_F32 && (out_ld % 8 || out_ld < cout || store_cols != cout || cout < 32)) ||
        (mode == CONV_LINEAR_F32 && out_ld < store_cols))
        return EFUNC_ERR_ARG;
    if (!encode_fn()) return EFUNC_ERR_UNSUPPORTED;
    const cudaError_t e = enc_conv(static_cast<const bf16 *>(x), batch, cin, static_cast<const bf16 *>(w), cout,
                                   taps, bias, mode, static_cast<const bf16 *>(mask), out, out_ld, store_cols, err,
                                   (cudaStream_t)stream);
    return e == cudaSuccess ? EFUNC_OK : cuda_fail(e);
}

efunc_status efunc_conv3d_wgrad_bf16(const void *dy, int32_t dy_ld, int32_t cout, const void *x, int32_t cin,
                                     int32_t batch, int32_t taps, float *dw, int32_t *err, efunc_stream_t stream)
{
    if (!dy || !x || !dw || !err || batch < 1 || cin < 64 || cin % 64 || cin > 256 || dy_ld % 64 || dy_ld < 64 ||
        dy_ld > 128 || cout < 1 || cout > dy_ld || (taps != 1 && taps != 27))
        return EFUNC_ERR_ARG;
    if (!encode_fn()) return EFUNC_ERR_UNSUPPORTED;
    const cudaError_t e = enc_wgrad(static_cast<const bf16 *>(dy), dy_ld, cout, static_cast<const bf16 *>(x), cin,
                                    batch, taps, dw, err, (cudaStream_t)stream);
    return e == cudaSuccess ? EFUNC_OK : cuda_fail(e);
}

}  // extern "C"
