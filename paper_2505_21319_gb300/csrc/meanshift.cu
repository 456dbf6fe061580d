// Mean-shift offset initialisation (Sec. 3.3): for every grid centre k_i,
//   Delta_i = sum_n exp(-bw |k_i - s_n|^2) (s_n - k_i) / sum_n exp(-bw |k_i - s_n|^2)
// over N surface points s_n (bw = 100 in the paper).  Every (centre, point)
// pair costs one exponential and a handful of FP32 operations; there is no
// contraction to put on tensor cores, so the kernel is bound by instruction
// issue (FP32 pipe + SFU).
//
// Work split.  A warp takes 4 centres that share (a, b) and have consecutive
// c, so that the x/y part of |k - s|^2 is formed once per point for the four.
// A CTA is 8 warps (32 centres), and a cluster of 8 CTAs shares the same 32
// centres while each CTA takes 1/8 of the points; the 8 partial softmax
// states merge through distributed shared memory at the end.  At R = 32 that
// is 8192 CTAs of 65536 pairs each, fine enough that the last wave leaves
// little of the GPU idle.  Points stream through shared memory as float4
// (conflict-free 128-bit loads, every lane a different point).
//
// Arithmetic.  Coordinates are scaled by sigma = sqrt(bw log2(e)) on the way
// in, so that the base-2 exponent is e = -|sigma k - sigma s|^2 with no
// further multiply; the weighted offset sums are divided by sigma at the end.
// The softmax is shifted by a reference exponent M per centre, the largest
// exponent over the first 256 points of the CTA (warp max).  Exponents are
// never positive, so when M >= -64 every weight 2^(e - M) stays below 2^64
// and nothing can overflow: those warps run the loop with no check.  Warps
// with a centre far from the sampled points (M < -64) run the loop that
// rescales a lane's sums when a point exceeds its M by 64 (rare after the
// sample).  Lanes, then CTAs, merge their (M, Z, S) states log-sum-exp style.
// Weights multiply (s - k), not s, so the offset has no cancellation against k.
#include <cooperative_groups.h>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace efunc {

namespace {

constexpr int kMsThreads = 256;
constexpr int kMsWarps = kMsThreads / 32;
constexpr int kMsCentres = 4;        // centres per warp (consecutive c)
constexpr int kMsCluster = 8;        // CTAs sharing one set of centres
constexpr int kMsTile = 2048;        // points per shared-memory tile
constexpr int kMsSample = 256;       // points that fix the reference exponent
constexpr float kMsSlack = 64.f;     // largest weight exponent allowed above M
constexpr unsigned kFull = 0xffffffffu;

struct MsState {
    float M[kMsCentres], Z[kMsCentres], Sx[kMsCentres], Sy[kMsCentres], Sz[kMsCentres];
};

__device__ __forceinline__ float rescale_of(float M, float Mn)
{
    return M == -INFINITY ? 0.f : ex2_approx(M - Mn);
}

template <bool CHECK>
__device__ __forceinline__ void ms_point(const float4 s, float kx, float ky, const float (&kz)[kMsCentres],
                                         MsState &st)
{
    const float rx = s.x - kx, ry = s.y - ky;
    const float ce = -fmaf(rx, rx, ry * ry);
#pragma unroll
    for (int c = 0; c < kMsCentres; ++c) {
        const float rz = s.z - kz[c];
        const float e = fmaf(-rz, rz, ce);           // base-2 exponent, <= 0
        if (CHECK && e > st.M[c] + kMsSlack) {       // rescale this lane's sums to the new reference
            const float f = ex2_approx(st.M[c] - e);
            st.Z[c] *= f;
            st.Sx[c] *= f;
            st.Sy[c] *= f;
            st.Sz[c] *= f;
            st.M[c] = e;
        }
        const float l = ex2_approx(e - st.M[c]);
        st.Z[c] += l;
        st.Sx[c] = fmaf(l, rx, st.Sx[c]);
        st.Sy[c] = fmaf(l, ry, st.Sy[c]);
        st.Sz[c] = fmaf(l, rz, st.Sz[c]);
    }
}

template <bool CHECK>
__device__ __forceinline__ void ms_tile(const float4 *tile, int nt, int lane, float kx, float ky,
                                        const float (&kz)[kMsCentres], MsState &st)
{
    int p = lane;
#pragma unroll 1
    for (; p + 32 < nt; p += 64) {
        const float4 s0 = tile[p], s1 = tile[p + 32];
        ms_point<CHECK>(s0, kx, ky, kz, st);
        ms_point<CHECK>(s1, kx, ky, kz, st);
    }
    if (p < nt) ms_point<CHECK>(tile[p], kx, ky, kz, st);
}

// merge state (M2, Z2, X2, Y2, W2) into (M, Z, X, Y, W)
__device__ __forceinline__ void ms_merge(float &M, float &Z, float &X, float &Y, float &W, float M2, float Z2,
                                         float X2, float Y2, float W2)
{
    const float Mn = fmaxf(M, M2);
    const float f1 = rescale_of(M, Mn), f2 = rescale_of(M2, Mn);
    Z = fmaf(Z, f1, Z2 * f2);
    X = fmaf(X, f1, X2 * f2);
    Y = fmaf(Y, f1, Y2 * f2);
    W = fmaf(W, f1, W2 * f2);
    M = Mn;
}

__global__ void __cluster_dims__(kMsCluster, 1, 1) __launch_bounds__(kMsThreads) mean_shift_kernel(MeanShiftArgs a)
{
    __shared__ float4 tile[kMsTile];
    __shared__ float part[kMsWarps * kMsCentres][5];   // per (warp, centre): M, Z, Sx, Sy, Sz
    cg::cluster_group cluster = cg::this_cluster();
    const unsigned rank = cluster.block_rank();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int R = a.R;
    const int cgroups = (R + kMsCentres - 1) / kMsCentres;
    const int64_t g = (int64_t)(blockIdx.x / kMsCluster) * kMsWarps + warp;
    const bool active = g < (int64_t)R * R * cgroups;   // warp-uniform, the same in every CTA of the cluster
    const int ia = active ? (int)(g / ((int64_t)R * cgroups)) : 0;
    const int ib = active ? (int)((g / cgroups) % R) : 0;
    const int c0 = active ? (int)(g % cgroups) * kMsCentres : 0;
    const float sg = a.sigma, invR = 1.f / (float)R;
    const float kx = sg * ((float)(2 * ia + 1 - R) * invR);
    const float ky = sg * ((float)(2 * ib + 1 - R) * invR);
    float kz[kMsCentres];
#pragma unroll
    for (int c = 0; c < kMsCentres; ++c) kz[c] = sg * ((float)(2 * (c0 + c) + 1 - R) * invR);

    // this CTA's share of the points
    const int64_t share = (a.N + kMsCluster - 1) / kMsCluster;
    const int64_t p0 = min(a.N, (int64_t)rank * share), p1 = min(a.N, p0 + share);

    MsState st;
#pragma unroll
    for (int c = 0; c < kMsCentres; ++c) {
        st.M[c] = -INFINITY;
        st.Z[c] = st.Sx[c] = st.Sy[c] = st.Sz[c] = 0.f;
    }
    bool check = false;
    for (int64_t base = p0; base < p1; base += kMsTile) {
        const int nt = (int)min((int64_t)kMsTile, p1 - base);
        __syncthreads();   // the previous tile is consumed
        for (int p = threadIdx.x; p < nt; p += kMsThreads) {
            const float *s = a.pts + 3 * (base + p);
            tile[p] = make_float4(sg * __ldg(s), sg * __ldg(s + 1), sg * __ldg(s + 2), 0.f);
        }
        __syncthreads();
        if (!active) continue;
        if (base == p0) {   // reference exponent per centre: warp max over the first points
            const int ns = min(nt, kMsSample);
            for (int p = lane; p < ns; p += 32) {
                const float4 s = tile[p];
                const float rx = s.x - kx, ry = s.y - ky;
                const float ce = -fmaf(rx, rx, ry * ry);
#pragma unroll
                for (int c = 0; c < kMsCentres; ++c) {
                    const float rz = s.z - kz[c];
                    st.M[c] = fmaxf(st.M[c], fmaf(-rz, rz, ce));
                }
            }
#pragma unroll
            for (int c = 0; c < kMsCentres; ++c) {
#pragma unroll
                for (int o = 16; o; o >>= 1) st.M[c] = fmaxf(st.M[c], __shfl_xor_sync(kFull, st.M[c], o));
                check |= st.M[c] < -kMsSlack;
            }
        }
        if (check) ms_tile<true>(tile, nt, lane, kx, ky, kz, st);
        else ms_tile<false>(tile, nt, lane, kx, ky, kz, st);
    }

    // merge the 32 lanes (only the checking loop lets their references differ)
    if (active) {
#pragma unroll
        for (int c = 0; c < kMsCentres; ++c) {
#pragma unroll
            for (int o = 16; o; o >>= 1)
                ms_merge(st.M[c], st.Z[c], st.Sx[c], st.Sy[c], st.Sz[c], __shfl_xor_sync(kFull, st.M[c], o),
                         __shfl_xor_sync(kFull, st.Z[c], o), __shfl_xor_sync(kFull, st.Sx[c], o),
                         __shfl_xor_sync(kFull, st.Sy[c], o), __shfl_xor_sync(kFull, st.Sz[c], o));
            if (lane == c) {
                float *q = part[warp * kMsCentres + c];
                q[0] = st.M[c];
                q[1] = st.Z[c];
                q[2] = st.Sx[c];
                q[3] = st.Sy[c];
                q[4] = st.Sz[c];
            }
        }
    }
    cluster.sync();   // every CTA's partial states are visible cluster-wide

    // rank 0 merges the cluster's partial states and writes the offsets
    if (rank == 0 && threadIdx.x < kMsWarps * kMsCentres) {
        const int w = threadIdx.x / kMsCentres, c = threadIdx.x % kMsCentres;
        const int64_t gw = (int64_t)(blockIdx.x / kMsCluster) * kMsWarps + w;
        const int cz = (int)(gw % cgroups) * kMsCentres + c;
        if (gw < (int64_t)R * R * cgroups && cz < R) {
            float M = -INFINITY, Z = 0.f, X = 0.f, Y = 0.f, W = 0.f;
            for (unsigned r = 0; r < kMsCluster; ++r) {
                const float *q = cluster.map_shared_rank(&part[threadIdx.x][0], r);
                ms_merge(M, Z, X, Y, W, q[0], q[1], q[2], q[3], q[4]);
            }
            const int wa = (int)(gw / ((int64_t)R * cgroups)), wb = (int)((gw / cgroups) % R);
            float *d = a.params + ((size_t)((int64_t)wa * R + wb) * R + cz) * kSlots;
            const float inv = 1.f / (Z * sg);
            d[0] = X * inv;
            d[1] = Y * inv;
            d[2] = W * inv;
        }
    }
    cluster.sync();   // peers keep their shared memory until rank 0 has read it
}

}  // namespace

cudaError_t launch_mean_shift(const MeanShiftArgs &a, cudaStream_t s)
{
    const int64_t groups = (int64_t)a.R * a.R * ((a.R + kMsCentres - 1) / kMsCentres);
    const int64_t blocks = (groups + kMsWarps - 1) / kMsWarps * kMsCluster;
    launch_begin(K_MEAN_SHIFT, s);
    mean_shift_kernel<<<(unsigned)blocks, kMsThreads, 0, s>>>(a);
    launch_end(K_MEAN_SHIFT, s);
    return cudaGetLastError();
}

}  // namespace efunc
