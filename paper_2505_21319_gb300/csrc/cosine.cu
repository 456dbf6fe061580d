// Cosine-series decomposition (Sec. 4.4, Eq. o-as-value / Eq. cosine-series):
//   S(q) = sum_{b < B} w_b(q) O_b(q),  w_b(q) = cos(b pi q_x) cos(b pi q_y) cos(b pi q_z),
// where every band b is a Config-G-6 representation (fixed grid keys,
// first-order values, learnable log-scales: b, o, d per centre).
//
// All bands share the grid, so a work item's window is the same for every
// band: the kernel stages the window's records of all B bands once, and per
// query evaluates the B softmaxes (forward thread-per-query) and the weighted
// sum.  The backward loops thread-per-(key, band) over the item's queries with
// the band's upstream gS_j w_b(q_j), one atomic per parameter per item.  The
// band weights are formed in FP32 from the exact split of b q (cos_factor);
// FP64 cospi, exact but slow on this GPU, cost a third of the one-band kernel.
#include "common.cuh"

namespace efunc {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr float kLn2 = 0.69314718055994531f;

__global__ void __launch_bounds__(256) cos_pack_kernel(CosineArgs a)
{
    const int64_t I = (int64_t)a.R * a.R * a.R;
    const double log2e = 1.4426950408889634;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < I * a.B;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float *th = a.params + (size_t)i * 5;
        const float s = (float)(-exp(a.log_beta0 + (double)__ldg(th)) * log2e);
        a.keys[2 * i] = make_float4(0.f, 0.f, 0.f, s);
        a.keys[2 * i + 1] = make_float4(__ldg(th + 1), __ldg(th + 2), __ldg(th + 3), __ldg(th + 4));
    }
}

struct CWin {
    int cx, cy, cz, lox, loy, loz, nx, ny, nz, nc;
};

__device__ __forceinline__ CWin cwindow_of(const Item item, int R)
{
    CWin w;
    w.cx = (item.z & 1023) - 1;
    w.cy = ((item.z >> 10) & 1023) - 1;
    w.cz = ((item.z >> 20) & 1023) - 1;
    w.lox = max(w.cx - kW + 1, 0);
    w.loy = max(w.cy - kW + 1, 0);
    w.loz = max(w.cz - kW + 1, 0);
    w.nx = min(w.cx + kW, R - 1) - w.lox + 1;
    w.ny = min(w.cy + kW, R - 1) - w.loy + 1;
    w.nz = min(w.cz + kW, R - 1) - w.loz + 1;
    w.nc = w.nx * w.ny * w.nz;
    return w;
}

// cos(b pi x) in FP32 from the exact split b x = hi + lo (lo = fma(b, x, -hi),
// |lo| <= ulp(hi) / 2): cos(pi hi) - pi lo sin(pi hi), the neglected terms
// O(lo^2) far below FP32 rounding; sincospif is accurate to about one ulp.
__device__ __forceinline__ float cos_factor(int b, float x)
{
    const float fb = (float)b;
    const float hi = fb * x;
    const float lo = fmaf(fb, x, -hi);
    float s, c;
    sincospif(hi, &s, &c);
    return fmaf(-3.14159265358979f * lo, s, c);
}

// (e, m) of one query over one band's window keys, exponents shifted by M2.
__device__ __forceinline__ void band_sums(const float4 *rec, int nc, float x, float y, float z, float M2, float &e,
                                          float &m)
{
    e = 0.f;
    m = 0.f;
#pragma unroll 4
    for (int c = 0; c < nc; ++c) {
        const float4 A = rec[2 * c], V = rec[2 * c + 1];
        const float rx = x - A.x, ry = y - A.y, rz = z - A.z;
        const float d2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
        const float l = ex2_approx(fmaf(A.w, d2, -M2));
        e += l;
        m = fmaf(l, fmaf(V.y, rx, fmaf(V.z, ry, fmaf(V.w, rz, V.x))), m);
    }
}

// band_sums over a full window (64 centres): the grid keys sit on the lattice
// (i - c) h, so d2 = (x2 + y2) + z2 from per-axis terms formed once per query
// (ry, y2, rz, z2 for the four offsets of each axis); same key order.
__device__ __forceinline__ void band_sums_lattice(const float4 *rec, float h, float x, const float (&ry)[4],
                                                  const float (&y2)[4], const float (&rz)[4], const float (&z2)[4],
                                                  float &e, float &m)
{
    e = 0.f;
    m = 0.f;
#pragma unroll 1
    for (int ox = 0; ox < 4; ++ox) {
        const float rx = x - (float)(ox - 1) * h;
        const float x2 = rx * rx;
#pragma unroll
        for (int oy = 0; oy < 4; ++oy) {
            const float xy = x2 + y2[oy];
#pragma unroll
            for (int oz = 0; oz < 4; ++oz) {
                const int c = 16 * ox + 4 * oy + oz;
                const float nbl = rec[2 * c].w;
                const float4 V = rec[2 * c + 1];
                const float l = ex2_approx(nbl * (xy + z2[oz]));
                e += l;
                m = fmaf(l, fmaf(V.y, rx, fmaf(V.z, ry[oy], fmaf(V.w, rz[oz], V.x))), m);
            }
        }
    }
}

size_t cos_smem_bytes(int B, int mode)
{
    return (size_t)(B * kCentres * 2 + kChunk + (mode == VAR_FORWARD ? 0 : kChunk * B)) * sizeof(float4);
}

template <int MODE>
__global__ void __launch_bounds__(kThreads) cosine_kernel(CosineArgs a)
{
    extern __shared__ float4 smem[];
    const int B = a.B;
    float4 *s_rec = smem;                       // [band][centre][2]
    float4 *s_qt = s_rec + B * kCentres * 2;    // [query]: (x, y, z, target), then (local q, 0)
    float4 *s_qb = s_qt + kChunk;               // [query][band]: (lse2_b, O_b, gS w_b, 0)
    __shared__ int s_item;
    __shared__ float s_red[2][kThreads / 32];

    const int t = threadIdx.x;
    const int R = a.R;
    const int64_t I = (int64_t)R * R * R;
    const float invR = 1.f / (float)R;
    const int n_items = a.ctrl->n_items;
    float loss_acc = 0.f, abs_acc = 0.f;

    for (;;) {
        __syncthreads();   // the previous item is consumed
        if (t == 0) s_item = atomicAdd(&a.ctrl->next_item, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= n_items) break;
        const Item item = a.items[it];
        const CWin w = cwindow_of(item, R);
        const int start = item.x, n = item.y, nc = w.nc;
        const float3 orig = make_float3((float)(2 * w.cx + 1 - R) * invR, (float)(2 * w.cy + 1 - R) * invR,
                                        (float)(2 * w.cz + 1 - R) * invR);
        // ---- 1. stage every band's window records (window-local key positions) and the queries
        for (int k = t; k < nc * B; k += kThreads) {
            const int c = k % nc, b = k / nc;
            const int oz = c % w.nz, oy = (c / w.nz) % w.ny, ox = c / (w.ny * w.nz);
            const int64_t i = ((int64_t)(w.lox + ox) * R + (w.loy + oy)) * R + (w.loz + oz);
            const float4 A = a.keys[2 * (b * I + i)];
            s_rec[(b * kCentres + c) * 2] =
                make_float4((float)(2 * (w.lox + ox - w.cx)) * invR, (float)(2 * (w.loy + oy - w.cy)) * invR,
                            (float)(2 * (w.loz + oz - w.cz)) * invR, A.w);
            s_rec[(b * kCentres + c) * 2 + 1] = a.keys[2 * (b * I + i) + 1];
        }
        for (int qi = t; qi < n; qi += kThreads) s_qt[qi] = a.sorted[start + qi];
        __syncthreads();

        // ---- 2. forward: B softmaxes and the cosine-weighted sum per query
        //         (full windows: lattice distances, per-axis terms shared by the bands)
        const bool full = nc == kCentres;
        const float h = 2.f * invR;
        for (int qi = t; qi < n; qi += kThreads) {
            const float4 q4 = s_qt[qi];
            const float x = q4.x - orig.x, y = q4.y - orig.y, z = q4.z - orig.z;
            float ry[4], y2[4], rz[4], z2[4];
#pragma unroll
            for (int o = 0; o < 4; ++o) {
                ry[o] = y - (float)(o - 1) * h;
                y2[o] = ry[o] * ry[o];
                rz[o] = z - (float)(o - 1) * h;
                z2[o] = rz[o] * rz[o];
            }
            float S = 0.f;
            for (int b = 0; b < B; ++b) {
                const float4 *rec = s_rec + b * kCentres * 2;
                float e, m, M2 = 0.f;
                if (full) band_sums_lattice(rec, h, x, ry, y2, rz, z2, e, m);
                else band_sums(rec, nc, x, y, z, 0.f, e, m);
                if (!(e >= 0x1p-60f)) {   // every key far in units of its scale: shift by the largest exponent
                    float mx = -INFINITY;
                    for (int c = 0; c < nc; ++c) {
                        const float4 A = rec[2 * c];
                        const float rx = x - A.x, ry = y - A.y, rz = z - A.z;
                        mx = fmaxf(mx, A.w * fmaf(rx, rx, fmaf(ry, ry, rz * rz)));
                    }
                    M2 = mx;
                    band_sums(rec, nc, x, y, z, M2, e, m);
                }
                const float O = m / e;
                const float wb = cos_factor(b, q4.x) * cos_factor(b, q4.y) * cos_factor(b, q4.z);
                S = fmaf(wb, O, S);
                if (MODE != VAR_FORWARD) s_qb[qi * B + b] = make_float4(M2 + lg2_approx(e), O, wb, 0.f);
            }
            float gS = 0.f;
            if (MODE == VAR_FIT) {
                const float diff = S - q4.w;
                if (a.loss == EFUNC_LOSS_L1) gS = diff > 0.f ? a.inv_J : (diff < 0.f ? -a.inv_J : 0.f);
                else gS = 2.f * diff * a.inv_J;
                loss_acc += a.loss == EFUNC_LOSS_L1 ? fabsf(diff) : diff * diff;
                abs_acc += fabsf(diff);
            } else {
                const int j = __ldg(a.perm + start + qi);
                if (MODE == VAR_FORWARD) a.S[j] = S;
                else gS = __ldg(a.gS + j);
            }
            if (MODE != VAR_FORWARD) {
                for (int b = 0; b < B; ++b) s_qb[qi * B + b].z *= gS;
                s_qt[qi] = make_float4(x, y, z, 0.f);
            }
        }
        if (MODE == VAR_FORWARD) continue;

        // ---- 3. backward: thread per (key, band) over the item's queries;
        //         with at most 64 keys (one band) two threads share a key,
        //         each over every second query
        __syncthreads();
        const int nkeys = nc * B;
        const int split = nkeys <= kThreads / 2 ? 2 : 1;
        for (int kk = t; kk < nkeys * split; kk += kThreads) {
            const int k = kk / split, part = kk - k * split;
            const int c = k % nc, b = k / nc;
            const float4 A = s_rec[(b * kCentres + c) * 2], V = s_rec[(b * kCentres + c) * 2 + 1];
            float ao = 0.f, adx = 0.f, ady = 0.f, adz = 0.f, ab = 0.f;
#pragma unroll 2
            for (int j = part; j < n; j += split) {
                const float4 Q = s_qt[j], P = s_qb[j * B + b];
                const float rx = Q.x - A.x, ry = Q.y - A.y, rz = Q.z - A.z;
                const float d2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
                const float g = ex2_approx(fmaf(A.w, d2, -P.x)) * P.z;
                const float f = fmaf(V.y, rx, fmaf(V.z, ry, fmaf(V.w, rz, V.x)));
                ao += g;
                adx = fmaf(g, rx, adx);
                ady = fmaf(g, ry, ady);
                adz = fmaf(g, rz, adz);
                ab = fmaf(g * (f - P.y), d2, ab);
            }
            const int oz = c % w.nz, oy = (c / w.nz) % w.ny, ox = c / (w.ny * w.nz);
            const int64_t i = ((int64_t)(w.lox + ox) * R + (w.loy + oy)) * R + (w.loz + oz);
            float *gr = a.grad + (size_t)(b * I + i) * 5;
            atomicAdd(gr + 0, A.w * kLn2 * ab);   // dO/db = w (f - O)(-beta |r|^2), beta = -A.w ln 2
            atomicAdd(gr + 1, ao);
            atomicAdd(gr + 2, adx);
            atomicAdd(gr + 3, ady);
            atomicAdd(gr + 4, adz);
        }
    }

    if (MODE == VAR_FIT) {
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
            for (int wi = 0; wi < kThreads / 32; ++wi) {
                l += s_red[0][wi];
                ab += s_red[1][wi];
            }
            atomicAdd(&a.ctrl->loss_sum, l);
            atomicAdd(&a.ctrl->abs_sum, ab);
        }
    }
}

int cos_sm_count() { return device_sm_count(); }

template <int MODE>
cudaError_t launch_mode(const CosineArgs &a, int kid, cudaStream_t s)
{
    const size_t smem = cos_smem_bytes(a.B, MODE);
    // the dynamic shared-memory limit is a per-device attribute of the kernel
    cudaError_t e = cudaSuccess;
    per_device_cached(reinterpret_cast<const void *>(cosine_kernel<MODE>), 0, [&e] {
        e = cudaFuncSetAttribute(cosine_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)cos_smem_bytes(kMaxBands, VAR_FIT));
        return e == cudaSuccess ? 1 : 0;   // a failure is not cached
    });
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cosine_kernel<MODE>, kThreads, smem);
    if (per_sm <= 0) per_sm = 1;
    if (a.leave_room) per_sm = leave_sort_room(reinterpret_cast<const void *>(cosine_kernel<MODE>), per_sm);
    launch_begin(kid, s);
    cosine_kernel<MODE><<<cos_sm_count() * per_sm, kThreads, smem, s>>>(a);
    launch_end(kid, s);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_cosine_pack(const CosineArgs &a, cudaStream_t s)
{
    const int64_t n = (int64_t)a.R * a.R * a.R * a.B;
    int64_t blocks = (n + 255) / 256;
    if (blocks > cos_sm_count() * 8) blocks = cos_sm_count() * 8;
    launch_begin(K_COS_PACK, s);
    cos_pack_kernel<<<(unsigned)blocks, 256, 0, s>>>(a);
    launch_end(K_COS_PACK, s);
    return cudaGetLastError();
}

cudaError_t launch_cosine(const CosineArgs &a, int mode, cudaStream_t s)
{
    if (mode == VAR_FORWARD) return launch_mode<VAR_FORWARD>(a, K_COS_FORWARD, s);
    if (mode == VAR_BACKWARD) return launch_mode<VAR_BACKWARD>(a, K_COS_BACKWARD, s);
    return launch_mode<VAR_FIT>(a, K_COS_FIT, s);
}

}  // namespace efunc
