// Fused evaluation / differentiation of the O^{+Delta} representation over
// cell-sorted queries (hot-path steps a2-a4).
//
// One work item = one window-base cell and up to kChunk of its sorted
// queries.  Every query of the item blends the same 4x4x4 window of centres,
// i.e. the same 128 keys (64 grid keys k_i and 64 offset keys k_i + Delta_i,
// one softmax over their union, Eq. func-offset).  A persistent CTA of 128
// threads takes items from a device counter and, per item:
//   1. stages the window's packed key records in shared memory (the records
//      are L2-resident: 64 bytes per centre), with key positions in
//      window-local coordinates (origin at the centre of index c, the window
//      base); queries are shifted into the same frame when loaded;
//   2. forward, thread per query (2 or 4 threads per query for sparse cells):
//      e = sum 2^{s}, m = sum 2^{s} f with s = -beta log2(e) ||q - key||^2,
//      O = m / e, lse2 = log2 e (Algorithm 1 in base 2).  The keys are summed
//      in four interleaved classes combined in a fixed tree, so a query's
//      result does not depend on how many threads share it.  If e underflows
//      (every key far away in units of its scale) the query is recomputed
//      with the maximum exponent subtracted;
//   3. backward, thread per key (Algorithm 2 turned around: each key loops
//      over the item's queries held in shared memory), recomputing the
//      normalised weight 2^{s - lse2} instead of storing it.  A thread keeps
//      its key's 5 (grid) or 8 (offset) gradient sums in registers and
//      issues one FP32 atomic per slot per item.
// No per-query intermediate leaves the CTA: the only outputs are O / lse /
// dO/dq (forward), the gradient grid and dL/dq (backward), and the loss sums
// (fit).
#include "common.cuh"

namespace efunc {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr float kLn2 = 0.69314718055994531f;
constexpr int kClasses = 4;   // interleaved summation classes of the forward

enum Mode { FORWARD = 0, BACKWARD = 1, FIT = 2 };

// --------------------------------------------------------------- pack

__global__ void __launch_bounds__(256) pack_keys_kernel(PackArgs a)
{
    const int I = a.R * a.R * a.R;
    const double log2e = 1.4426950408889634;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < I; i += gridDim.x * blockDim.x) {
        const float *th = a.params + (size_t)i * kSlots;
        float v[kSlots];
#pragma unroll
        for (int s = 0; s < kSlots; ++s) v[s] = __ldg(th + s);
        const float nbl_g = (float)(-exp(a.log_beta0 + (double)v[3]) * log2e);
        const float nbl_o = (float)(-exp(a.log_beta0 + (double)v[4]) * log2e);
        float4 *k = a.keys + (size_t)i * kKeyRecords;
        k[0] = make_float4(0.f, 0.f, 0.f, nbl_g);
        k[1] = make_float4(v[5], v[6], v[7], v[8]);
        k[2] = make_float4(v[0], v[1], v[2], nbl_o);
        k[3] = make_float4(v[9], v[10], v[11], v[12]);
    }
}

// ------------------------------------------------------------ forward

// One key's contribution to (e, m) for a query at (x, y, z), shifted by M2.
__device__ __forceinline__ void fwd_key(const float4 A, const float4 B, float x, float y, float z, float M2,
                                        float &e, float &m)
{
    const float rx = x - A.x, ry = y - A.y, rz = z - A.z;
    const float d2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
    const float l = ex2_approx(fmaf(A.w, d2, -M2));
    const float f = fmaf(B.y, rx, fmaf(B.z, ry, fmaf(B.w, rz, B.x)));
    e += l;
    m = fmaf(l, f, m);
}

__device__ __forceinline__ float key_exponent(const float4 A, float x, float y, float z)
{
    const float rx = x - A.x, ry = y - A.y, rz = z - A.z;
    return A.w * fmaf(rx, rx, fmaf(ry, ry, rz * rz));
}

// Combines the per-class partial sums of a query held by KQ lanes in the
// fixed order ((c0 + c1) + (c2 + c3)).  Lane `part` holds classes
// part + KQ*i, i < 4/KQ.
template <int KQ>
__device__ __forceinline__ float combine_classes(const float *v)
{
    if (KQ == 1) return (v[0] + v[1]) + (v[2] + v[3]);
    if (KQ == 2) {
        const float lo = v[0] + __shfl_xor_sync(kFull, v[0], 1);
        const float hi = v[1] + __shfl_xor_sync(kFull, v[1], 1);
        return lo + hi;
    }
    const float s1 = v[0] + __shfl_xor_sync(kFull, v[0], 1);
    return s1 + __shfl_xor_sync(kFull, s1, 2);
}

// (e, m) of one query over the window's keys, classes as above.
template <int KQ>
__device__ __forceinline__ void fwd_sums(const float4 *skA, const float4 *skB, int nc, int part, float x, float y,
                                         float z, float M2, float &e, float &m)
{
    constexpr int CPL = kClasses / KQ;
    float ev[CPL], mv[CPL];
#pragma unroll
    for (int i = 0; i < CPL; ++i) ev[i] = mv[i] = 0.f;
#pragma unroll
    for (int set = 0; set < 2; ++set) {
        const float4 *A = skA + set * kCentres, *B = skB + set * kCentres;
        for (int base = 0; base < nc; base += kClasses) {
#pragma unroll
            for (int i = 0; i < CPL; ++i) {
                const int k = base + part + KQ * i;
                if (k < nc) fwd_key(A[k], B[k], x, y, z, M2, ev[i], mv[i]);
            }
        }
    }
    e = combine_classes<KQ>(ev);
    m = combine_classes<KQ>(mv);
}

// Eq. func-normal: dO/dq = sum w (d + 2 beta (q - key)(O - f)), same classes.
template <int KQ>
__device__ __forceinline__ void dq_sums(const float4 *skA, const float4 *skB, int nc, int part, float x, float y,
                                        float z, float lse2, float O, float &gx, float &gy, float &gz)
{
    constexpr int CPL = kClasses / KQ;
    float ax[CPL], ay[CPL], az[CPL];
#pragma unroll
    for (int i = 0; i < CPL; ++i) ax[i] = ay[i] = az[i] = 0.f;
#pragma unroll
    for (int set = 0; set < 2; ++set) {
        const float4 *A = skA + set * kCentres, *B = skB + set * kCentres;
        for (int base = 0; base < nc; base += kClasses) {
#pragma unroll
            for (int i = 0; i < CPL; ++i) {
                const int k = base + part + KQ * i;
                if (k < nc) {
                    const float4 a = A[k], b = B[k];
                    const float rx = x - a.x, ry = y - a.y, rz = z - a.z;
                    const float d2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
                    const float w = ex2_approx(fmaf(a.w, d2, -lse2));
                    const float f = fmaf(b.y, rx, fmaf(b.z, ry, fmaf(b.w, rz, b.x)));
                    const float c = w * (-2.f * kLn2) * a.w * (O - f);   // 2 beta w (O - f)
                    ax[i] = fmaf(w, b.y, fmaf(c, rx, ax[i]));
                    ay[i] = fmaf(w, b.z, fmaf(c, ry, ay[i]));
                    az[i] = fmaf(w, b.w, fmaf(c, rz, az[i]));
                }
            }
        }
    }
    gx = combine_classes<KQ>(ax);
    gy = combine_classes<KQ>(ay);
    gz = combine_classes<KQ>(az);
}

struct FwdOut {
    float O, lse2;
};

// Forward of the query held by this lane group: fast path without shift,
// shifted recomputation for groups whose sum underflowed.
template <int KQ>
__device__ __forceinline__ FwdOut forward_query(const float4 *skA, const float4 *skB, int nc, int part, float4 q)
{
    float e, m;
    fwd_sums<KQ>(skA, skB, nc, part, q.x, q.y, q.z, 0.f, e, m);
    float M2 = 0.f;
    const bool tiny = !(e >= 0x1p-60f);   // identical in every lane of the group
    if (__any_sync(kFull, tiny)) {
        float mx = -INFINITY;
        for (int k = part; k < nc; k += KQ) {
            mx = fmaxf(mx, key_exponent(skA[k], q.x, q.y, q.z));
            mx = fmaxf(mx, key_exponent(skA[kCentres + k], q.x, q.y, q.z));
        }
#pragma unroll
        for (int o = 1; o < KQ; o <<= 1) mx = fmaxf(mx, __shfl_xor_sync(kFull, mx, o));
        float e2, m2;
        fwd_sums<KQ>(skA, skB, nc, part, q.x, q.y, q.z, mx, e2, m2);
        if (tiny) {
            e = e2;
            m = m2;
            M2 = mx;
        }
    }
    return {m / e, M2 + lg2_approx(e)};
}

// ----------------------------------------------------------- backward

// Thread-per-key loop over the item's queries.
template <bool OFFSET>
__device__ __forceinline__ void bwd_key_loop(const float4 A, const float4 B, const float4 *__restrict__ sq0,
                                             const float2 *__restrict__ sq1, int n, float acc[8])
{
    float ag = 0.f, arx = 0.f, ary = 0.f, arz = 0.f, ab = 0.f, adx = 0.f, ady = 0.f, adz = 0.f;
#pragma unroll 4
    for (int j = 0; j < n; ++j) {
        const float4 Q = sq0[j];
        const float2 S = sq1[j];
        const float rx = Q.x - A.x, ry = Q.y - A.y, rz = Q.z - A.z;
        const float d2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
        const float w = ex2_approx(fmaf(A.w, d2, -Q.w));
        const float g = w * S.y;
        const float f = fmaf(B.y, rx, fmaf(B.z, ry, fmaf(B.w, rz, B.x)));
        const float gd = g * (f - S.x);
        ag += g;
        arx = fmaf(g, rx, arx);
        ary = fmaf(g, ry, ary);
        arz = fmaf(g, rz, arz);
        ab = fmaf(gd, d2, ab);
        if (OFFSET) {
            adx = fmaf(gd, rx, adx);
            ady = fmaf(gd, ry, ady);
            adz = fmaf(gd, rz, adz);
        }
    }
    acc[0] = ag; acc[1] = arx; acc[2] = ary; acc[3] = arz; acc[4] = ab;
    acc[5] = adx; acc[6] = ady; acc[7] = adz;
}

// ------------------------------------------------------------- kernel

template <int MODE, bool DQ, int KQ>
__device__ __forceinline__ void forward_phase(const FusedArgs &a, const float4 *skA, const float4 *skB, float4 *sq0,
                                              float2 *sq1, int start, int n, int nc, float3 orig, float &loss_acc,
                                              float &abs_acc)
{
    constexpr int LG = KQ == 1 ? 0 : (KQ == 2 ? 1 : 2);
    const int t = threadIdx.x;
    const int part = t & (KQ - 1);
    constexpr int per_round = kThreads / KQ;
    for (int base = 0; base < n; base += per_round) {
        const int qi = base + (t >> LG);
        const bool valid = qi < n;
        float4 q = a.sorted[start + (valid ? qi : 0)];
        q.x -= orig.x;   // window-local coordinates
        q.y -= orig.y;
        q.z -= orig.z;
        const FwdOut r = forward_query<KQ>(skA, skB, nc, part, q);
        const float O = r.O, lse2 = r.lse2;

        float gO = 0.f;
        int j_user = 0;
        if (MODE != FIT) j_user = valid ? a.perm[start + qi] : 0;
        if (MODE == FIT) {
            const float diff = O - q.w;
            if (a.loss == EFUNC_LOSS_L1) gO = diff > 0.f ? a.inv_J : (diff < 0.f ? -a.inv_J : 0.f);
            else gO = 2.f * diff * a.inv_J;
            if (valid && part == 0) {
                loss_acc += a.loss == EFUNC_LOSS_L1 ? fabsf(diff) : diff * diff;
                abs_acc += fabsf(diff);
            }
        } else if (MODE == BACKWARD) {
            gO = valid ? __ldg(a.gO + j_user) : 0.f;
        } else if (valid && part == 0) {
            a.O[j_user] = O;
            if (a.lse) a.lse[j_user] = lse2 * kLn2;
        }
        if (DQ) {
            float gx, gy, gz;
            dq_sums<KQ>(skA, skB, nc, part, q.x, q.y, q.z, lse2, O, gx, gy, gz);
            if (valid && part == 0) {
                float *dst = MODE == FORWARD ? a.dq : a.gq;
                const float s = MODE == FORWARD ? 1.f : gO;
                dst[3 * (size_t)j_user + 0] = s * gx;
                dst[3 * (size_t)j_user + 1] = s * gy;
                dst[3 * (size_t)j_user + 2] = s * gz;
            }
        }
        if (MODE != FORWARD && valid && part == 0) {
            sq0[qi] = make_float4(q.x, q.y, q.z, lse2);
            sq1[qi] = make_float2(O, gO);
        }
    }
}

template <int MODE, bool DQ>
__global__ void __launch_bounds__(kThreads) fused_kernel(FusedArgs a)
{
    __shared__ float4 skA[2 * kCentres];   // key position, -beta*log2(e)
    __shared__ float4 skB[2 * kCentres];   // value constant, value linear term
    __shared__ float4 sq0[MODE == FORWARD ? 1 : kChunk];   // query, lse2
    __shared__ float2 sq1[MODE == FORWARD ? 1 : kChunk];   // O, dL/dO
    __shared__ int s_item;
    __shared__ float s_red[2][kThreads / 32];

    const int t = threadIdx.x;
    const int R = a.R;
    float loss_acc = 0.f, abs_acc = 0.f;

    for (;;) {
        __syncthreads();   // the previous item is fully consumed
        if (t == 0) s_item = atomicAdd(&a.ctrl->next_item, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= a.ctrl->n_items) break;
        const Item item = a.items[it];
        const int start = item.x, n = item.y;
        const int cx = (item.z & 1023) - 1, cy = ((item.z >> 10) & 1023) - 1, cz = ((item.z >> 20) & 1023) - 1;
        const int lox = max(cx - kW + 1, 0), loy = max(cy - kW + 1, 0), loz = max(cz - kW + 1, 0);
        const int nx = min(cx + kW, R - 1) - lox + 1;
        const int ny = min(cy + kW, R - 1) - loy + 1;
        const int nz = min(cz + kW, R - 1) - loz + 1;
        const int nc = nx * ny * nz;

        // window origin: centre of index (cx, cy, cz), exact for power-of-two R
        const float fR = (float)R;
        const float3 orig = make_float3((float)(2 * cx + 1 - R) / fR, (float)(2 * cy + 1 - R) / fR,
                                        (float)(2 * cz + 1 - R) / fR);

        // ---- 1. stage the window's key records, positions relative to orig
        if (t < nc) {
            const int oz = t % nz, oy = (t / nz) % ny, ox = t / (ny * nz);
            const int ia = lox + ox, ib = loy + oy, ic = loz + oz;
            const float4 *k = a.keys + (((size_t)ia * R + ib) * R + ic) * kKeyRecords;
            const float gx = (float)(2 * (ia - cx)) / fR, gy = (float)(2 * (ib - cy)) / fR,
                        gz = (float)(2 * (ic - cz)) / fR;
            const float4 k0 = k[0], k2 = k[2];
            skA[t] = make_float4(gx, gy, gz, k0.w);
            skB[t] = k[1];
            skA[kCentres + t] = make_float4(gx + k2.x, gy + k2.y, gz + k2.z, k2.w);
            skB[kCentres + t] = k[3];
        }
        __syncthreads();

        // ---- 2. forward, one (or 2 / 4) threads per query
        if (n > 64) forward_phase<MODE, DQ, 1>(a, skA, skB, sq0, sq1, start, n, nc, orig, loss_acc, abs_acc);
        else if (n > 32) forward_phase<MODE, DQ, 2>(a, skA, skB, sq0, sq1, start, n, nc, orig, loss_acc, abs_acc);
        else forward_phase<MODE, DQ, 4>(a, skA, skB, sq0, sq1, start, n, nc, orig, loss_acc, abs_acc);

        if (MODE == FORWARD) continue;

        // ---- 3. backward, one thread per key
        __syncthreads();
        const int c = t & (kCentres - 1);
        if (c < nc) {
            const bool offset = t >= kCentres;
            const float4 A = skA[t], B = skB[t];
            float acc[8];
            if (offset) bwd_key_loop<true>(A, B, sq0, sq1, n, acc);
            else bwd_key_loop<false>(A, B, sq0, sq1, n, acc);
            const int oz = c % nz, oy = (c / nz) % ny, ox = c / (ny * nz);
            float *gr = a.grad + (((size_t)(lox + ox) * R + (loy + oy)) * R + (loz + oz)) * kSlots;
            const float beta = -A.w * kLn2;
            if (!offset) {
                atomicAdd(gr + 5, acc[0]);
                atomicAdd(gr + 6, acc[1]);
                atomicAdd(gr + 7, acc[2]);
                atomicAdd(gr + 8, acc[3]);
                atomicAdd(gr + 3, -beta * acc[4]);
            } else {
                atomicAdd(gr + 9, acc[0]);
                atomicAdd(gr + 10, acc[1]);
                atomicAdd(gr + 11, acc[2]);
                atomicAdd(gr + 12, acc[3]);
                atomicAdd(gr + 4, -beta * acc[4]);
                // dO/dDelta = w (-d' + 2 beta' (q - key)(f' - O))
                atomicAdd(gr + 0, fmaf(-B.y, acc[0], 2.f * beta * acc[5]));
                atomicAdd(gr + 1, fmaf(-B.z, acc[0], 2.f * beta * acc[6]));
                atomicAdd(gr + 2, fmaf(-B.w, acc[0], 2.f * beta * acc[7]));
            }
        }
    }

    if (MODE == FIT) {
        // loss sums: warp shuffle, then one double atomic per CTA
        for (int o = 16; o > 0; o >>= 1) {
            loss_acc += __shfl_xor_sync(kFull, loss_acc, o);
            abs_acc += __shfl_xor_sync(kFull, abs_acc, o);
        }
        if ((t & 31) == 0) {
            s_red[0][t >> 5] = loss_acc;
            s_red[1][t >> 5] = abs_acc;
        }
        __syncthreads();
        if (t == 0) {
            double l = 0.0, ab = 0.0;
            for (int w = 0; w < kThreads / 32; ++w) {
                l += s_red[0][w];
                ab += s_red[1][w];
            }
            atomicAdd(&a.ctrl->loss_sum, l);
            atomicAdd(&a.ctrl->abs_sum, ab);
        }
    }
}

int sm_count()
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

}  // namespace

int fused_grid_size()
{
    static int g = 0;
    if (!g) {
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fused_kernel<FIT, false>, kThreads, 0);
        if (per_sm <= 0) per_sm = 1;
        g = sm_count() * per_sm;
    }
    return g;
}

cudaError_t launch_pack_keys(const PackArgs &a, cudaStream_t s)
{
    const int I = a.R * a.R * a.R;
    int blocks = (I + 255) / 256;
    if (blocks > sm_count() * 8) blocks = sm_count() * 8;
    launch_begin(K_PACK_KEYS, s);
    pack_keys_kernel<<<blocks, 256, 0, s>>>(a);
    launch_end(K_PACK_KEYS, s);
    return cudaGetLastError();
}

cudaError_t launch_forward(const FusedArgs &a, bool with_dq, int grid, cudaStream_t s)
{
    launch_begin(K_FORWARD, s);
    if (with_dq) fused_kernel<FORWARD, true><<<grid, kThreads, 0, s>>>(a);
    else fused_kernel<FORWARD, false><<<grid, kThreads, 0, s>>>(a);
    launch_end(K_FORWARD, s);
    return cudaGetLastError();
}

cudaError_t launch_fused_backward(const FusedArgs &a, bool with_gq, int grid, cudaStream_t s)
{
    launch_begin(K_FUSED_BWD, s);
    if (with_gq) fused_kernel<BACKWARD, true><<<grid, kThreads, 0, s>>>(a);
    else fused_kernel<BACKWARD, false><<<grid, kThreads, 0, s>>>(a);
    launch_end(K_FUSED_BWD, s);
    return cudaGetLastError();
}

cudaError_t launch_fused_fit(const FusedArgs &a, int grid, cudaStream_t s)
{
    launch_begin(K_FUSED_FIT, s);
    fused_kernel<FIT, false><<<grid, kThreads, 0, s>>>(a);
    launch_end(K_FUSED_FIT, s);
    return cudaGetLastError();
}

}  // namespace efunc
