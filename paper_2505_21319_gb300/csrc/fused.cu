// Fused evaluation / differentiation of the O^{+Delta} representation over
// cell-sorted queries (hot-path steps a2-a4).
//
// One work item = one window-base cell and up to kChunk of its sorted
// queries.  Every query of the item blends the same 4x4x4 window of centres,
// i.e. the same 128 keys (64 grid keys k_i and 64 offset keys k_i + Delta_i,
// one softmax over their union, Eq. func-offset).  A persistent CTA of 128
// threads takes items from a device counter and, per item:
//   1. stages the window's keys in shared memory (params are L2-resident):
//      key position, -beta*log2(e), value constant and linear term;
//   2. forward, thread per query (2 or 4 threads per query for sparse cells):
//      e = sum 2^{s}, m = sum 2^{s} f with s = -beta log2(e) ||q - key||^2,
//      O = m / e, lse2 = log2 e (Algorithm 1 in base 2).  If e underflows
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

enum Mode { FORWARD = 0, BACKWARD = 1, FIT = 2 };

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

// Thread-per-key backward loop over the item's queries.
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
    const float fR = (float)R;
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

        // ---- 1. stage the window's keys
        if (t < nc) {
            const int oz = t % nz, oy = (t / nz) % ny, ox = t / (ny * nz);
            const int ia = lox + ox, ib = loy + oy, ic = loz + oz;
            const float *th = a.params + ((size_t)((size_t)ia * R + ib) * R + ic) * kSlots;
            float v[kSlots];
#pragma unroll
            for (int s = 0; s < kSlots; ++s) v[s] = __ldg(th + s);
            const float kx = (float)(2 * ia + 1 - R) / fR;
            const float ky = (float)(2 * ib + 1 - R) / fR;
            const float kz = (float)(2 * ic + 1 - R) / fR;
            // -beta*log2(e) = (-exp(log_beta0)*log2(e)) * exp(b); the first
            // factor is folded on the host in double precision.
            skA[t] = make_float4(kx, ky, kz, a.nbl0 * expf(v[3]));
            skB[t] = make_float4(v[5], v[6], v[7], v[8]);
            skA[kCentres + t] = make_float4(kx + v[0], ky + v[1], kz + v[2], a.nbl0 * expf(v[4]));
            skB[kCentres + t] = make_float4(v[9], v[10], v[11], v[12]);
        }
        __syncthreads();

        // ---- 2. forward, one (or 2 / 4) threads per query
        const int lg = n > 64 ? 0 : (n > 32 ? 1 : 2);
        const int kq = 1 << lg;
        const int part = t & (kq - 1);
        const int per_round = kThreads >> lg;
        for (int base = 0; base < n; base += per_round) {
            const int qi = base + (t >> lg);
            const bool valid = qi < n;
            const float4 q = a.sorted[start + (valid ? qi : 0)];
            float e = 0.f, m = 0.f, M2 = 0.f;
            for (int k = part; k < nc; k += kq) fwd_key(skA[k], skB[k], q.x, q.y, q.z, 0.f, e, m);
            for (int k = part; k < nc; k += kq) fwd_key(skA[kCentres + k], skB[kCentres + k], q.x, q.y, q.z, 0.f, e, m);
            for (int o = 1; o < kq; o <<= 1) {
                e += __shfl_xor_sync(kFull, e, o);
                m += __shfl_xor_sync(kFull, m, o);
            }
            const bool tiny = !(e >= 0x1p-60f);
            if (__any_sync(kFull, tiny)) {
                // every key far away in units of its scale: subtract the max exponent
                float mx = -INFINITY;
                for (int k = part; k < nc; k += kq) {
                    mx = fmaxf(mx, key_exponent(skA[k], q.x, q.y, q.z));
                    mx = fmaxf(mx, key_exponent(skA[kCentres + k], q.x, q.y, q.z));
                }
                for (int o = 1; o < kq; o <<= 1) mx = fmaxf(mx, __shfl_xor_sync(kFull, mx, o));
                M2 = mx;
                e = 0.f;
                m = 0.f;
                for (int k = part; k < nc; k += kq) fwd_key(skA[k], skB[k], q.x, q.y, q.z, M2, e, m);
                for (int k = part; k < nc; k += kq)
                    fwd_key(skA[kCentres + k], skB[kCentres + k], q.x, q.y, q.z, M2, e, m);
                for (int o = 1; o < kq; o <<= 1) {
                    e += __shfl_xor_sync(kFull, e, o);
                    m += __shfl_xor_sync(kFull, m, o);
                }
            }
            const float O = m / e;
            const float lse2 = M2 + lg2_approx(e);

            float gO = 0.f;
            int j_user = 0;
            if (MODE != FIT) j_user = valid ? a.perm[start + qi] : 0;
            if (MODE == FIT) {
                const float diff = O - q.w;
                if (a.loss == EFUNC_LOSS_L1)
                    gO = diff > 0.f ? a.inv_J : (diff < 0.f ? -a.inv_J : 0.f);
                else
                    gO = 2.f * diff * a.inv_J;
                if (valid && part == 0) {
                    loss_acc += a.loss == EFUNC_LOSS_L1 ? fabsf(diff) : diff * diff;
                    abs_acc += fabsf(diff);
                }
            } else if (MODE == BACKWARD) {
                gO = valid ? __ldg(a.gO + j_user) : 0.f;
            } else {
                if (valid && part == 0) {
                    a.O[j_user] = O;
                    if (a.lse) a.lse[j_user] = lse2 * kLn2;
                }
            }

            if (DQ) {
                // Eq. func-normal: dO/dq = sum w (d + 2 beta (q - key)(O - f))
                float gx = 0.f, gy = 0.f, gz = 0.f;
                for (int s = 0; s < 2; ++s) {
                    for (int k = part; k < nc; k += kq) {
                        const float4 A = skA[s * kCentres + k], B = skB[s * kCentres + k];
                        const float rx = q.x - A.x, ry = q.y - A.y, rz = q.z - A.z;
                        const float d2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
                        const float w = ex2_approx(fmaf(A.w, d2, -lse2));
                        const float f = fmaf(B.y, rx, fmaf(B.z, ry, fmaf(B.w, rz, B.x)));
                        // 2 beta = -2 ln2 * A.w
                        const float c = w * (-2.f * kLn2) * A.w * (O - f);
                        gx = fmaf(w, B.y, fmaf(c, rx, gx));
                        gy = fmaf(w, B.z, fmaf(c, ry, gy));
                        gz = fmaf(w, B.w, fmaf(c, rz, gz));
                    }
                }
                for (int o = 1; o < kq; o <<= 1) {
                    gx += __shfl_xor_sync(kFull, gx, o);
                    gy += __shfl_xor_sync(kFull, gy, o);
                    gz += __shfl_xor_sync(kFull, gz, o);
                }
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
            float *gr = a.grad + ((size_t)((size_t)(lox + ox) * R + (loy + oy)) * R + (loz + oz)) * kSlots;
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

}  // namespace

int fused_grid_size()
{
    static int g = 0;
    if (!g) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fused_kernel<FIT, false>, kThreads, 0);
        if (sms <= 0) sms = 1;
        if (per_sm <= 0) per_sm = 1;
        g = sms * per_sm;
    }
    return g;
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
