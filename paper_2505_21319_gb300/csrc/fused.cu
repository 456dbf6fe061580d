// Fused evaluation / differentiation of the O^{+Delta} representation over
// cell-sorted queries (hot-path steps a2-a4).
//
// One work item = one window-base cell and up to kChunk of its sorted
// queries.  Every query of the item blends the same 4x4x4 window of centres,
// i.e. the same 128 keys (64 grid keys k_i and 64 offset keys k_i + Delta_i,
// one softmax over their union, Eq. func-offset).  A persistent CTA of 128
// threads takes items from a device counter and, per item:
//   1. stages the item's query tile and the window's key records (L2-resident,
//      64 bytes per centre) in shared memory, key positions rewritten into
//      window-local coordinates (origin at the centre of index c, the window
//      base; queries are shifted into the same frame);
//   2. forward, thread per query (2 threads per query in items of at most 64
//      queries; 4 in a batched fit whose tuning asks for it):
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
//
// Every function is templated on the scalar type T of the arithmetic.  The
// hot path is T = float with the SFU's ex2.approx / lg2.approx; T = double
// runs the same kernels (same staging, windows, summation classes and
// branches) with exp2 / log2 in double, so that finite differences of the
// FP64 results check the very code the FP32 path runs.
#include <type_traits>

#include "adam_clock.cuh"
#include "common.cuh"

namespace efunc {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kClasses = 4;   // interleaved summation classes of the forward

enum Mode { FORWARD = 0, BACKWARD = 1, FIT = 2, EVAL = 3 };

// Scalar arithmetic of the kernels for T = float (fast SFU exponentials) and
// T = double (exp2 / log2 in double).
template <typename T> struct Num;
template <> struct Num<float> {
    using V4 = float4;
    using V2 = float2;
    static constexpr float kLn2 = 0.69314718055994531f;
    __device__ static __forceinline__ float fma(float a, float b, float c) { return fmaf(a, b, c); }
    __device__ static __forceinline__ float ex2(float x) { return ex2_approx(x); }
    __device__ static __forceinline__ float lg2(float x) { return lg2_approx(x); }
    __device__ static __forceinline__ float4 v4(float x, float y, float z, float w) { return make_float4(x, y, z, w); }
    __device__ static __forceinline__ float2 v2(float x, float y) { return make_float2(x, y); }
};
template <> struct Num<double> {
    using V4 = Double4;
    using V2 = double2;
    static constexpr double kLn2 = 0.69314718055994531;
    __device__ static __forceinline__ double fma(double a, double b, double c) { return ::fma(a, b, c); }
    __device__ static __forceinline__ double ex2(double x) { return exp2(x); }
    __device__ static __forceinline__ double lg2(double x) { return log2(x); }
    __device__ static __forceinline__ Double4 v4(double x, double y, double z, double w) { return {x, y, z, w}; }
    __device__ static __forceinline__ double2 v2(double x, double y) { return make_double2(x, y); }
};

// Shared key tile of one window: centre c holds 4 records of 4 scalars,
//   rec[4c + 0] = (grid key position, -beta log2 e)    rec[4c + 1] = (o, d)
//   rec[4c + 2] = (offset key position, -beta' log2 e) rec[4c + 3] = (o', d')
// with positions in window-local coordinates; set 0 = grid keys, 1 = offset keys.
template <typename V>
__device__ __forceinline__ V keyA(const V *rec, int set, int k) { return rec[4 * k + 2 * set]; }
template <typename V>
__device__ __forceinline__ V keyB(const V *rec, int set, int k) { return rec[4 * k + 2 * set + 1]; }

struct Window {
    int cx, cy, cz, lox, loy, loz, nx, ny, nz, nc;
};

__device__ __forceinline__ Window window_of(const Item item, int R)
{
    Window w;
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

// --------------------------------------------------------------- pack

template <typename T>
__global__ void __launch_bounds__(256) pack_keys_kernel(PackArgsT<T> a)
{
    using N = Num<T>;
    const int I = a.R * a.R * a.R;
    const double log2e = 1.4426950408889634;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < I; i += gridDim.x * blockDim.x) {
        const T *th = a.params + (size_t)i * kSlots;
        T v[kSlots];
#pragma unroll
        for (int s = 0; s < kSlots; ++s) v[s] = __ldg(th + s);
        const T nbl_g = (T)(-exp(a.log_beta0 + (double)v[3]) * log2e);
        const T nbl_o = (T)(-exp(a.log_beta0 + (double)v[4]) * log2e);
        typename N::V4 *k = a.keys + (size_t)i * kKeyRecords;
        k[0] = N::v4(T(0), T(0), T(0), nbl_g);
        k[1] = N::v4(v[5], v[6], v[7], v[8]);
        k[2] = N::v4(v[0], v[1], v[2], nbl_o);
        k[3] = N::v4(v[9], v[10], v[11], v[12]);
    }
}

// FP32 rows (x, y, z, 0) of FP64 queries: the rounding that picks windows.
__global__ void __launch_bounds__(256) round_queries_kernel(const double *q64, int64_t J, int stride, float4 *rows)
{
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < J; j += (int64_t)gridDim.x * blockDim.x) {
        const double *r = q64 + j * stride;
        rows[j] = make_float4((float)r[0], (float)r[1], (float)r[2], 0.f);
    }
}

// FP64 query rows in sorted order: rows64[i] = q64[perm[i]].
__global__ void __launch_bounds__(256) gather_queries64_kernel(const double *q64, int64_t J, int stride,
                                                               const int *perm, Double4 *rows)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < J; i += (int64_t)gridDim.x * blockDim.x) {
        const double *r = q64 + (int64_t)perm[i] * stride;
        rows[i] = Double4{r[0], r[1], r[2], stride == 4 ? r[3] : 0.0};
    }
}

// ------------------------------------------------------------ forward

// One key's contribution to (e, m) for a query at (x, y, z), shifted by M2.
template <typename T, typename V>
__device__ __forceinline__ void fwd_key(const V A, const V B, T x, T y, T z, T M2, T &e, T &m)
{
    using N = Num<T>;
    const T rx = x - A.x, ry = y - A.y, rz = z - A.z;
    const T d2 = N::fma(rx, rx, N::fma(ry, ry, rz * rz));
    const T l = N::ex2(N::fma(A.w, d2, -M2));
    const T f = N::fma(B.y, rx, N::fma(B.z, ry, N::fma(B.w, rz, B.x)));
    e += l;
    m = N::fma(l, f, m);
}

template <typename T, typename V>
__device__ __forceinline__ T key_exponent(const V A, T x, T y, T z)
{
    using N = Num<T>;
    const T rx = x - A.x, ry = y - A.y, rz = z - A.z;
    return A.w * N::fma(rx, rx, N::fma(ry, ry, rz * rz));
}

// Combines the per-class partial sums of a query held by KQ lanes in the
// fixed order ((c0 + c1) + (c2 + c3)).  Lane `part` holds classes
// part + KQ*i, i < 4/KQ.
template <int KQ, typename T>
__device__ __forceinline__ T combine_classes(const T *v)
{
    if (KQ == 1) return (v[0] + v[1]) + (v[2] + v[3]);
    if (KQ == 2) {
        const T lo = v[0] + __shfl_xor_sync(kFull, v[0], 1);
        const T hi = v[1] + __shfl_xor_sync(kFull, v[1], 1);
        return lo + hi;
    }
    const T s1 = v[0] + __shfl_xor_sync(kFull, v[0], 1);
    return s1 + __shfl_xor_sync(kFull, s1, 2);
}

// (e, m) of one query over the window's keys, classes as above.
template <int KQ, typename T, typename V>
__device__ __forceinline__ void fwd_sums(const V *rec, int nc, int part, T x, T y, T z, T M2, T &e, T &m)
{
    constexpr int CPL = kClasses / KQ;
    T ev[CPL], mv[CPL];
#pragma unroll
    for (int i = 0; i < CPL; ++i) ev[i] = mv[i] = T(0);
#pragma unroll
    for (int set = 0; set < 2; ++set) {
        for (int base = 0; base < nc; base += kClasses) {
#pragma unroll
            for (int i = 0; i < CPL; ++i) {
                const int k = base + part + KQ * i;
                if (k < nc) fwd_key(keyA(rec, set, k), keyB(rec, set, k), x, y, z, M2, ev[i], mv[i]);
            }
        }
    }
    e = combine_classes<KQ>(ev);
    m = combine_classes<KQ>(mv);
}

// Full window (nc = 64, the interior case).  Grid keys sit on the lattice
// (i - c) h, i - c in {-1, 0, 1, 2} per axis, so their distance terms are
// formed once per query and axis: d2 = (X2[ox] + Y2[oy]) + Z2[oz].  Offset
// keys take the generic path.  Classes as in fwd_sums: class i of lane `part`
// is the z offset oz = part + KQ i.
template <int KQ, typename T, typename V>
__device__ __forceinline__ void fwd_sums_full(const V *rec, int part, T h, T x, T y, T z, T &e, T &m)
{
    using N = Num<T>;
    constexpr int CPL = kClasses / KQ;
    T ev[CPL], mv[CPL];
    T ry[4], y2[4], rz[CPL], z2[CPL];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        ry[a] = y - (T)(a - 1) * h;
        y2[a] = ry[a] * ry[a];
    }
#pragma unroll
    for (int i = 0; i < CPL; ++i) {
        rz[i] = z - (T)(part + KQ * i - 1) * h;
        z2[i] = rz[i] * rz[i];
        ev[i] = mv[i] = T(0);
    }
    const V *P = rec + 4 * part;
#pragma unroll 1
    for (int ox = 0; ox < 4; ++ox) {
        const T rx = x - (T)(ox - 1) * h;
        const T x2 = rx * rx;
        const V *Po = P + 4 * 16 * ox;
#pragma unroll
        for (int oy = 0; oy < 4; ++oy) {
            const T xy = x2 + y2[oy];
#pragma unroll
            for (int i = 0; i < CPL; ++i) {
                const int k = oy * 4 + KQ * i;
                const T nbl = Po[4 * k].w;
                const V b = Po[4 * k + 1];
                const T l = N::ex2(nbl * (xy + z2[i]));
                const T f = N::fma(b.y, rx, N::fma(b.z, ry[oy], N::fma(b.w, rz[i], b.x)));
                ev[i] += l;
                mv[i] = N::fma(l, f, mv[i]);
            }
        }
    }
#pragma unroll 1
    for (int k0 = 0; k0 < kCentres; k0 += 16) {
#pragma unroll
        for (int kk = 0; kk < 16; kk += kClasses) {
#pragma unroll
            for (int i = 0; i < CPL; ++i) {
                const int k = k0 + kk + KQ * i;
                fwd_key(P[4 * k + 2], P[4 * k + 3], x, y, z, T(0), ev[i], mv[i]);
            }
        }
    }
    e = combine_classes<KQ>(ev);
    m = combine_classes<KQ>(mv);
}

// Eq. func-normal: dO/dq = sum w (d + 2 beta (q - key)(O - f)), same classes.
template <int KQ, typename T, typename V>
__device__ __forceinline__ void dq_sums(const V *rec, int nc, int part, T x, T y, T z, T lse2, T O, T &gx, T &gy,
                                        T &gz)
{
    using N = Num<T>;
    constexpr int CPL = kClasses / KQ;
    T ax[CPL], ay[CPL], az[CPL];
#pragma unroll
    for (int i = 0; i < CPL; ++i) ax[i] = ay[i] = az[i] = T(0);
#pragma unroll
    for (int set = 0; set < 2; ++set) {
        for (int base = 0; base < nc; base += kClasses) {
#pragma unroll
            for (int i = 0; i < CPL; ++i) {
                const int k = base + part + KQ * i;
                if (k < nc) {
                    const V a = keyA(rec, set, k), b = keyB(rec, set, k);
                    const T rx = x - a.x, ry = y - a.y, rz = z - a.z;
                    const T d2 = N::fma(rx, rx, N::fma(ry, ry, rz * rz));
                    const T w = N::ex2(N::fma(a.w, d2, -lse2));
                    const T f = N::fma(b.y, rx, N::fma(b.z, ry, N::fma(b.w, rz, b.x)));
                    const T c = w * (T(-2) * N::kLn2) * a.w * (O - f);   // 2 beta w (O - f)
                    ax[i] = N::fma(w, b.y, N::fma(c, rx, ax[i]));
                    ay[i] = N::fma(w, b.z, N::fma(c, ry, ay[i]));
                    az[i] = N::fma(w, b.w, N::fma(c, rz, az[i]));
                }
            }
        }
    }
    gx = combine_classes<KQ>(ax);
    gy = combine_classes<KQ>(ay);
    gz = combine_classes<KQ>(az);
}

// dO/dq (as dq_sums) together with V = sum w beta (q - key), the two
// per-query sums the backward through dO/dq needs; same classes.
template <int KQ>
__device__ __forceinline__ void gv_sums(const float4 *rec, int nc, int part, float x, float y, float z, float lse2,
                                        float O, float G[3], float V[3])
{
    constexpr int CPL = kClasses / KQ;
    float ax[CPL], ay[CPL], az[CPL], vx[CPL], vy[CPL], vz[CPL];
#pragma unroll
    for (int i = 0; i < CPL; ++i) ax[i] = ay[i] = az[i] = vx[i] = vy[i] = vz[i] = 0.f;
#pragma unroll
    for (int set = 0; set < 2; ++set) {
        for (int base = 0; base < nc; base += kClasses) {
#pragma unroll
            for (int i = 0; i < CPL; ++i) {
                const int k = base + part + KQ * i;
                if (k < nc) {
                    const float4 a = keyA(rec, set, k), b = keyB(rec, set, k);
                    const float rx = x - a.x, ry = y - a.y, rz = z - a.z;
                    const float d2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
                    const float w = ex2_approx(fmaf(a.w, d2, -lse2));
                    const float f = fmaf(b.y, rx, fmaf(b.z, ry, fmaf(b.w, rz, b.x)));
                    const float wb = w * (-Num<float>::kLn2) * a.w;   // w beta
                    const float c = 2.f * wb * (O - f);                // 2 beta w (O - f)
                    ax[i] = fmaf(w, b.y, fmaf(c, rx, ax[i]));
                    ay[i] = fmaf(w, b.z, fmaf(c, ry, ay[i]));
                    az[i] = fmaf(w, b.w, fmaf(c, rz, az[i]));
                    vx[i] = fmaf(wb, rx, vx[i]);
                    vy[i] = fmaf(wb, ry, vy[i]);
                    vz[i] = fmaf(wb, rz, vz[i]);
                }
            }
        }
    }
    G[0] = combine_classes<KQ>(ax);
    G[1] = combine_classes<KQ>(ay);
    G[2] = combine_classes<KQ>(az);
    V[0] = combine_classes<KQ>(vx);
    V[1] = combine_classes<KQ>(vy);
    V[2] = combine_classes<KQ>(vz);
}

template <typename T>
struct FwdOut {
    T O, lse2;
};

// Forward of the query held by this lane group: fast path without shift,
// shifted recomputation for groups whose sum underflowed.
template <int KQ, bool FULL, typename T, typename V>
__device__ __forceinline__ FwdOut<T> forward_query(const V *rec, int nc, int part, T h, V q)
{
    T e, m;
    if (FULL) fwd_sums_full<KQ>(rec, part, h, q.x, q.y, q.z, e, m);
    else fwd_sums<KQ>(rec, nc, part, q.x, q.y, q.z, T(0), e, m);
    T M2 = T(0);
    const bool tiny = !(e >= T(0x1p-60));   // identical in every lane of the group
    if (__any_sync(kFull, tiny)) {
        T mx = -INFINITY;
        for (int k = part; k < nc; k += KQ) {
            mx = fmax(mx, key_exponent(keyA(rec, 0, k), q.x, q.y, q.z));
            mx = fmax(mx, key_exponent(keyA(rec, 1, k), q.x, q.y, q.z));
        }
#pragma unroll
        for (int o = 1; o < KQ; o <<= 1) mx = fmax(mx, __shfl_xor_sync(kFull, mx, o));
        // the shifted sums take the generic path in every window shape
        T e2, m2;
        fwd_sums<KQ>(rec, nc, part, q.x, q.y, q.z, mx, e2, m2);
        if (tiny) {
            e = e2;
            m = m2;
            M2 = mx;
        }
    }
    return {m / e, M2 + Num<T>::lg2(e)};
}

// ----------------------------------------------------------- backward

// Thread-per-key loop over the item's queries, two queries per iteration:
// sqA[j] = (q_j local, lse2_j), sqB[j/2] = (O_j, gO_j, O_j+1, gO_j+1); an odd
// count is padded with a copy of the last query carrying dL/dO = 0.
template <bool OFFSET, typename T, typename V>
__device__ __forceinline__ void bwd_key_loop(const V A, const V B, const V *__restrict__ sqA,
                                             const V *__restrict__ sqB, int n, T acc[8])
{
    using N = Num<T>;
    T ag = 0, arx = 0, ary = 0, arz = 0, ab = 0, adx = 0, ady = 0, adz = 0;
    auto one = [&](const V Q, T O, T gO) {
        const T rx = Q.x - A.x, ry = Q.y - A.y, rz = Q.z - A.z;
        const T d2 = N::fma(rx, rx, N::fma(ry, ry, rz * rz));
        const T w = N::ex2(N::fma(A.w, d2, -Q.w));
        const T g = w * gO;
        const T f = N::fma(B.y, rx, N::fma(B.z, ry, N::fma(B.w, rz, B.x)));
        const T gd = g * (f - O);
        ag += g;
        arx = N::fma(g, rx, arx);
        ary = N::fma(g, ry, ary);
        arz = N::fma(g, rz, arz);
        ab = N::fma(gd, d2, ab);
        if (OFFSET) {
            adx = N::fma(gd, rx, adx);
            ady = N::fma(gd, ry, ady);
            adz = N::fma(gd, rz, adz);
        }
    };
    const int pairs = (n + 1) >> 1;
#pragma unroll 2
    for (int jp = 0; jp < pairs; ++jp) {
        const V Q0 = sqA[2 * jp], Q1 = sqA[2 * jp + 1], S = sqB[jp];
        one(Q0, S.x, S.y);
        one(Q1, S.z, S.w);
    }
    acc[0] = ag; acc[1] = arx; acc[2] = ary; acc[3] = arz; acc[4] = ab;
    acc[5] = adx; acc[6] = ady; acc[7] = adz;
}

// Thread-per-key loop of the second-order backward: the value term (as
// bwd_key_loop, dL/dO = gO) plus the gradient of u . dO/dq per query, with
// per-query rows sqA[j] = (q local, lse2), sqE[j] = (O, gO, H, T),
// sqU[j] = (u, 0), H = u . dO/dq, T = -2 u . sum w beta (q - key).  For one
// key (w its weight, r = q - key, dlt = f - O, t = -2 beta r):
//   d(u.G)/do    = w (u.t - T)
//   d(u.G)/dd    = w (r (u.t - T) + u)
//   d(u.G)/dbeta = w (-|r|^2 [(h - H) - dlt T] - 2 dlt u.r),  h = u.d + dlt u.t
//   d(u.G)/dkey  = w (2 beta r [(h - H) - dlt T] - d (u.t - T) + 2 beta dlt u)
// Accumulators: acc[0..7] value term as bwd_key_loop; acc[8] sum w (u.t - T),
// acc[9..11] sum w (u.t - T) r + w u, acc[12] sum w (...) of dbeta,
// acc[13..15] sum w [(h - H) - dlt T] r, acc[16..18] sum w dlt u.
template <bool OFFSET>
__device__ __forceinline__ void bwd2_key_loop(const float4 A, const float4 B, const float4 *__restrict__ sqA,
                                              const float4 *__restrict__ sqE, const float4 *__restrict__ sqU, int n,
                                              float acc[19])
{
    const float beta = -A.w * Num<float>::kLn2;
    float v0 = 0.f, v1 = 0.f, v2 = 0.f, v3 = 0.f, v4 = 0.f, v5 = 0.f, v6 = 0.f, v7 = 0.f;
    float e0 = 0.f, ex = 0.f, ey = 0.f, ez = 0.f, eb = 0.f, px = 0.f, py = 0.f, pz = 0.f, qx = 0.f, qy = 0.f,
          qz = 0.f;
#pragma unroll 2
    for (int j = 0; j < n; ++j) {
        const float4 Q = sqA[j], E = sqE[j], U = sqU[j];
        const float rx = Q.x - A.x, ry = Q.y - A.y, rz = Q.z - A.z;
        const float d2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
        const float w = ex2_approx(fmaf(A.w, d2, -Q.w));
        const float f = fmaf(B.y, rx, fmaf(B.z, ry, fmaf(B.w, rz, B.x)));
        const float dlt = f - E.x;
        // value term
        const float g = w * E.y;
        const float gd = g * dlt;
        v0 += g;
        v1 = fmaf(g, rx, v1);
        v2 = fmaf(g, ry, v2);
        v3 = fmaf(g, rz, v3);
        v4 = fmaf(gd, d2, v4);
        if (OFFSET) {
            v5 = fmaf(gd, rx, v5);
            v6 = fmaf(gd, ry, v6);
            v7 = fmaf(gd, rz, v7);
        }
        // gradient term
        const float ur = fmaf(U.x, rx, fmaf(U.y, ry, U.z * rz));
        const float ut = -2.f * beta * ur;
        const float ua = fmaf(U.x, B.y, fmaf(U.y, B.z, U.z * B.w));
        const float h = fmaf(dlt, ut, ua);
        const float we1 = w * (ut - E.w);
        const float hH = fmaf(-dlt, E.w, h - E.z);
        e0 += we1;
        ex = fmaf(we1, rx, fmaf(w, U.x, ex));
        ey = fmaf(we1, ry, fmaf(w, U.y, ey));
        ez = fmaf(we1, rz, fmaf(w, U.z, ez));
        eb = fmaf(w, fmaf(-d2, hH, -2.f * dlt * ur), eb);
        if (OFFSET) {
            const float whH = w * hH, wd = w * dlt;
            px = fmaf(whH, rx, px);
            py = fmaf(whH, ry, py);
            pz = fmaf(whH, rz, pz);
            qx = fmaf(wd, U.x, qx);
            qy = fmaf(wd, U.y, qy);
            qz = fmaf(wd, U.z, qz);
        }
    }
    acc[0] = v0; acc[1] = v1; acc[2] = v2; acc[3] = v3; acc[4] = v4; acc[5] = v5; acc[6] = v6; acc[7] = v7;
    acc[8] = e0; acc[9] = ex; acc[10] = ey; acc[11] = ez; acc[12] = eb;
    acc[13] = px; acc[14] = py; acc[15] = pz; acc[16] = qx; acc[17] = qy; acc[18] = qz;
}

// ------------------------------------------ packed FP32 (f32x2) forms
//
// The SMs of this GPU issue two FP32 operations per f32x2 instruction (each
// half rounds exactly as the scalar instruction; the FMA pipe's rate is the
// same, the issue slots are halved).  The FP32 kernels are issue bound, so
// their forward blends two keys per instruction (summation classes j and
// j + 2 of one query) and their backward two queries per instruction (one
// key).  Every operation is written with its rounding (_rn, no contraction).

__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b)
{
    unsigned long long r, x, y;
    asm("mov.b64 %0, {%1, %2};" : "=l"(x) : "f"(a.x), "f"(a.y));
    asm("mov.b64 %0, {%1, %2};" : "=l"(y) : "f"(b.x), "f"(b.y));
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(x), "l"(y));
    float2 v;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
    return v;
}
__device__ __forceinline__ float2 dup2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 lo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ float2 ex2_2(float2 a) { return make_float2(ex2_approx(a.x), ex2_approx(a.y)); }

// Paired key tile (FP32): pair p = 2 r + j of set s (0 grid keys, 1 offset
// keys) interleaves keys 4 r + j and 4 r + j + 2 of the window, classes j
// and j + 2:
//   P[0] = (x, x', y, y')   P[1] = (z, z', -beta log2 e, ...')
//   P[2] = (o, o', dx, dx') P[3] = (dy, dy', dz, dz')
// at rec2 + 4 (32 s + p), positions window-local.  Keys from the window's
// last centre up to a multiple of 4 are neutral (position 1e18, scale -1,
// values 0): their weight is exactly 0 and they add exact zeros.
constexpr int kPairs = kCentres / 2;

__device__ __forceinline__ const float4 *pair_of(const float4 *rec2, int set, int p)
{
    return rec2 + 4 * (kPairs * set + p);
}

__device__ __forceinline__ float *pair_slot(float4 *rec2, int set, int k)
{
    return reinterpret_cast<float *>(rec2 + 4 * (kPairs * set + 2 * (k >> 2) + (k & 1))) + ((k >> 1) & 1);
}

// Stages key k (this lane) and key k ^ 2 (lane ^ 2: the other class of the
// same pair) into their pair's four rows: the lane of class j writes P[0],
// P[1], its partner P[2], P[3], each after one swap of half a key record, so
// that the tile is written with conflict-free 16-byte stores.  Every lane of
// the warp calls it; store = the pair is part of the tile.
__device__ __forceinline__ void stage_pair_keys(float4 *rec2, int set, int k, bool store, float4 A, float4 B)
{
    const bool hi = (k >> 1) & 1;   // class j + 2 of its pair
    const float4 s = hi ? A : B;
    const float4 r = make_float4(__shfl_xor_sync(kFull, s.x, 2), __shfl_xor_sync(kFull, s.y, 2),
                                 __shfl_xor_sync(kFull, s.z, 2), __shfl_xor_sync(kFull, s.w, 2));
    if (!store) return;
    float4 *P = rec2 + 4 * (kPairs * set + 2 * (k >> 2) + (k & 1));
    if (!hi) {
        P[0] = make_float4(A.x, r.x, A.y, r.y);
        P[1] = make_float4(A.z, r.z, A.w, r.w);
    } else {
        P[2] = make_float4(r.x, B.x, r.y, B.y);
        P[3] = make_float4(r.z, B.z, r.w, B.w);
    }
}

__device__ __forceinline__ float4 pair_keyA(const float4 *rec2, int set, int k)
{
    const float *f = pair_slot(const_cast<float4 *>(rec2), set, k);
    return make_float4(f[0], f[2], f[4], f[6]);
}

// Per-lane sums -> (e or m) of the query in the fixed order ((c0 + c1) +
// (c2 + c3)) of combine_classes.  KQ = 1: v[0] = (c0, c2), v[1] = (c1, c3);
// KQ = 2: lane `part` holds (c_part, c_part+2); KQ = 4: lanes `part` and
// `part ^ 2` blend the same pair, lane `part` keeps class `part`.
template <int KQ>
__device__ __forceinline__ float combine_x2(const float2 *v, int part)
{
    if (KQ == 1) return (v[0].x + v[1].x) + (v[0].y + v[1].y);
    if (KQ == 2) {
        const float lo = v[0].x + __shfl_xor_sync(kFull, v[0].x, 1);
        const float hi = v[0].y + __shfl_xor_sync(kFull, v[0].y, 1);
        return lo + hi;
    }
    const float c = (part & 2) ? v[0].y : v[0].x;
    const float s1 = c + __shfl_xor_sync(kFull, c, 1);
    return s1 + __shfl_xor_sync(kFull, s1, 2);
}

// Two keys of one pair for a query at (x, y, z) (duplicated in both halves):
// the generic key form of fwd_key, exponent shifted by nm = -M2.
__device__ __forceinline__ void fwd_pair(const float4 *P, float2 xd, float2 yd, float2 zd, float2 nm, float2 &ev,
                                         float2 &mv)
{
    const float4 P0 = P[0], P1 = P[1], P2 = P[2], P3 = P[3];
    const float2 rx = sub2(xd, lo2(P0)), ry = sub2(yd, hi2(P0)), rz = sub2(zd, lo2(P1));
    const float2 d2 = fma2(rx, rx, fma2(ry, ry, mul2(rz, rz)));
    const float2 l = ex2_2(fma2(hi2(P1), d2, nm));
    const float2 f = fma2(hi2(P2), rx, fma2(lo2(P3), ry, fma2(hi2(P3), rz, lo2(P2))));
    ev = add2(ev, l);
    mv = fma2(l, f, mv);
}

// (e, m) of one query over a window of nc keys per set from the paired tile
// (any window shape; the shifted recomputation after an underflow).
template <int KQ>
__device__ __forceinline__ void fwd_sums_x2(const float4 *rec2, int nc, int part, float x, float y, float z,
                                            float nM2, float &e, float &m)
{
    constexpr int NP = KQ == 1 ? 2 : 1;   // pairs per lane and row
    const int j0 = KQ == 1 ? 0 : (part & 1);
    float2 ev[NP], mv[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) ev[i] = mv[i] = make_float2(0.f, 0.f);
    const float2 xd = dup2(x), yd = dup2(y), zd = dup2(z), nm = dup2(nM2);
    const int rows = (nc + 3) >> 2;
#pragma unroll
    for (int set = 0; set < 2; ++set)
        for (int r = 0; r < rows; ++r)
#pragma unroll
            for (int i = 0; i < NP; ++i) fwd_pair(pair_of(rec2, set, 2 * r + j0 + i), xd, yd, zd, nm, ev[i], mv[i]);
    e = combine_x2<KQ>(ev, part);
    m = combine_x2<KQ>(mv, part);
}

// Full window (nc = 64): grid keys on the lattice, d2 = (rx^2 + ry^2) + rz^2
// formed per row and pair without their positions (as fwd_sums_full); offset
// keys in the generic form.
template <int KQ>
__device__ __forceinline__ void fwd_sums_full_x2(const float4 *rec2, int part, float h, float x, float y, float z,
                                                 float &e, float &m)
{
    constexpr int NP = KQ == 1 ? 2 : 1;
    const int j0 = KQ == 1 ? 0 : (part & 1);
    float2 ev[NP], mv[NP], rz[NP], ry[4], y2[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        ry[a] = dup2(__fsub_rn(y, (float)(a - 1) * h));
        y2[a] = mul2(ry[a], ry[a]);
    }
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        const int j = j0 + i;
        rz[i] = make_float2(__fsub_rn(z, (float)(j - 1) * h), __fsub_rn(z, (float)(j + 1) * h));
        ev[i] = mv[i] = make_float2(0.f, 0.f);
    }
#pragma unroll 1
    for (int ox = 0; ox < 4; ++ox) {
        const float2 rx = dup2(__fsub_rn(x, (float)(ox - 1) * h));
#pragma unroll
        for (int oy = 0; oy < 4; ++oy) {
            const float2 xy = fma2(rx, rx, y2[oy]);
#pragma unroll
            for (int i = 0; i < NP; ++i) {
                const float4 *P = pair_of(rec2, 0, 2 * (4 * ox + oy) + j0 + i);
                const float4 P1 = P[1], P2 = P[2], P3 = P[3];
                const float2 l = ex2_2(mul2(hi2(P1), fma2(rz[i], rz[i], xy)));
                const float2 f = fma2(hi2(P2), rx, fma2(lo2(P3), ry[oy], fma2(hi2(P3), rz[i], lo2(P2))));
                ev[i] = add2(ev[i], l);
                mv[i] = fma2(l, f, mv[i]);
            }
        }
    }
    const float2 xd = dup2(x), yd = dup2(y), zd = dup2(z), nm = dup2(-0.f);
#pragma unroll 1
    for (int r0 = 0; r0 < kCentres / 4; r0 += 4)
#pragma unroll
        for (int rr = 0; rr < 4; ++rr)
#pragma unroll
            for (int i = 0; i < NP; ++i)
                fwd_pair(pair_of(rec2, 1, 2 * (r0 + rr) + j0 + i), xd, yd, zd, nm, ev[i], mv[i]);
    e = combine_x2<KQ>(ev, part);
    m = combine_x2<KQ>(mv, part);
}

// fwd_pair for two queries a and b from one load of the pair: the forward
// is bound by these broadcast 16-byte shared loads (two wavefronts each), so
// the threads of a pair in one-lane-per-query items share them (below).
__device__ __forceinline__ void fwd_pair_2q(const float4 *P, float2 xa, float2 ya, float2 za, float2 xb, float2 yb,
                                            float2 zb, float2 nm, float2 &eva, float2 &mva, float2 &evb, float2 &mvb)
{
    const float4 P0 = P[0], P1 = P[1], P2 = P[2], P3 = P[3];
    {
        const float2 rx = sub2(xa, lo2(P0)), ry = sub2(ya, hi2(P0)), rz = sub2(za, lo2(P1));
        const float2 d2 = fma2(rx, rx, fma2(ry, ry, mul2(rz, rz)));
        const float2 l = ex2_2(fma2(hi2(P1), d2, nm));
        const float2 f = fma2(hi2(P2), rx, fma2(lo2(P3), ry, fma2(hi2(P3), rz, lo2(P2))));
        eva = add2(eva, l);
        mva = fma2(l, f, mva);
    }
    {
        const float2 rx = sub2(xb, lo2(P0)), ry = sub2(yb, hi2(P0)), rz = sub2(zb, lo2(P1));
        const float2 d2 = fma2(rx, rx, fma2(ry, ry, mul2(rz, rz)));
        const float2 l = ex2_2(fma2(hi2(P1), d2, nm));
        const float2 f = fma2(hi2(P2), rx, fma2(lo2(P3), ry, fma2(hi2(P3), rz, lo2(P2))));
        evb = add2(evb, l);
        mvb = fma2(l, f, mvb);
    }
}

// Full window, own query q of thread t (a for even, b for odd t): grid keys
// on the lattice for the own query over all classes (as fwd_sums_full_x2<1>),
// then the offset keys for both queries of the thread pair over the classes
// j0, j0 + 2 of this thread, the class sums handed over by shuffles so that
// every class is summed in row order as in the other lane counts.
__device__ __forceinline__ void fwd_sums_full_o2q(const float4 *rec2, float h, float4 qa, float4 qb, float4 q, float &e,
                                                  float &m)
{
    const int j0 = threadIdx.x & 1;
    float2 ev[2], mv[2], rz[2], ry[4], y2[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        ry[a] = dup2(__fsub_rn(q.y, (float)(a - 1) * h));
        y2[a] = mul2(ry[a], ry[a]);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        rz[i] = make_float2(__fsub_rn(q.z, (float)(i - 1) * h), __fsub_rn(q.z, (float)(i + 1) * h));
        ev[i] = mv[i] = make_float2(0.f, 0.f);
    }
#pragma unroll 1
    for (int ox = 0; ox < 4; ++ox) {
        const float2 rx = dup2(__fsub_rn(q.x, (float)(ox - 1) * h));
#pragma unroll
        for (int oy = 0; oy < 4; ++oy) {
            const float2 xy = fma2(rx, rx, y2[oy]);
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const float4 *P = pair_of(rec2, 0, 2 * (4 * ox + oy) + i);
                const float4 P1 = P[1], P2 = P[2], P3 = P[3];
                const float2 l = ex2_2(mul2(hi2(P1), fma2(rz[i], rz[i], xy)));
                const float2 f = fma2(hi2(P2), rx, fma2(lo2(P3), ry[oy], fma2(hi2(P3), rz[i], lo2(P2))));
                ev[i] = add2(ev[i], l);
                mv[i] = fma2(l, f, mv[i]);
            }
        }
    }
    // hand the partner the classes it continues for this thread's query
    const float2 mine_e = j0 ? ev[1] : ev[0], mine_m = j0 ? mv[1] : mv[0];
    const float2 send_e = j0 ? ev[0] : ev[1], send_m = j0 ? mv[0] : mv[1];
    const float2 got_e = make_float2(__shfl_xor_sync(kFull, send_e.x, 1), __shfl_xor_sync(kFull, send_e.y, 1));
    const float2 got_m = make_float2(__shfl_xor_sync(kFull, send_m.x, 1), __shfl_xor_sync(kFull, send_m.y, 1));
    float2 eva = j0 ? got_e : mine_e, mva = j0 ? got_m : mine_m;
    float2 evb = j0 ? mine_e : got_e, mvb = j0 ? mine_m : got_m;
    const float2 xa = dup2(qa.x), ya = dup2(qa.y), za = dup2(qa.z);
    const float2 xb = dup2(qb.x), yb = dup2(qb.y), zb = dup2(qb.z), nm = dup2(-0.f);
#pragma unroll 1
    for (int r0 = 0; r0 < kCentres / 4; r0 += 4)
#pragma unroll
        for (int rr = 0; rr < 4; ++rr)
            fwd_pair_2q(pair_of(rec2, 1, 2 * (r0 + rr) + j0), xa, ya, za, xb, yb, zb, nm, eva, mva, evb, mvb);
    // back: the own query's classes of the partner
    const float2 se = j0 ? eva : evb, sm = j0 ? mva : mvb;
    const float2 me = j0 ? evb : eva, mm = j0 ? mvb : mva;
    const float re0 = __shfl_xor_sync(kFull, se.x, 1), re1 = __shfl_xor_sync(kFull, se.y, 1);
    const float rm0 = __shfl_xor_sync(kFull, sm.x, 1), rm1 = __shfl_xor_sync(kFull, sm.y, 1);
    e = (me.x + re0) + (me.y + re1);
    m = (mm.x + rm0) + (mm.y + rm1);
}

// Forward of one query from the paired tile (as forward_query).  qa and qb
// are the two queries of this thread's pair (even and odd thread), used by
// full windows with one lane per query; q is this thread's own.
template <int KQ, bool FULL>
__device__ __forceinline__ FwdOut<float> forward_query_x2(const float4 *rec2, int nc, int part, float h, float4 q,
                                                          float4 qa, float4 qb)
{
    float e, m;
    if (FULL && KQ == 1) fwd_sums_full_o2q(rec2, h, qa, qb, q, e, m);
    else if (FULL) fwd_sums_full_x2<KQ>(rec2, part, h, q.x, q.y, q.z, e, m);
    else fwd_sums_x2<KQ>(rec2, nc, part, q.x, q.y, q.z, -0.f, e, m);
    float M2 = 0.f;
    const bool tiny = !(e >= 0x1p-60f);
    if (__any_sync(kFull, tiny)) {
        float mx = -INFINITY;
        for (int k = part; k < nc; k += KQ) {
            mx = fmaxf(mx, key_exponent(pair_keyA(rec2, 0, k), q.x, q.y, q.z));
            mx = fmaxf(mx, key_exponent(pair_keyA(rec2, 1, k), q.x, q.y, q.z));
        }
#pragma unroll
        for (int o = 1; o < KQ; o <<= 1) mx = fmaxf(mx, __shfl_xor_sync(kFull, mx, o));
        float e2, m2;
        fwd_sums_x2<KQ>(rec2, nc, part, q.x, q.y, q.z, -mx, e2, m2);
        if (tiny) {
            e = e2;
            m = m2;
            M2 = mx;
        }
    }
    return {m / e, M2 + lg2_approx(e)};
}

// Paired query rows of the backward: pair jp = queries 2 jp, 2 jp + 1 at
// sq2 + 3 jp,
//   [0] = (x, x', y, y')  [1] = (z, z', -lse2, -lse2')  [2] = (-O, -O', gO, gO')
// (window-local positions); an odd count is padded with a copy of the last
// query carrying dL/dO = 0.
__device__ __forceinline__ void store_pair_query(float4 *sq2, int qi, float4 q, float lse2, float O, float gO)
{
    float *f = reinterpret_cast<float *>(sq2 + 3 * (qi >> 1)) + (qi & 1);
    f[0] = q.x; f[2] = q.y; f[4] = q.z; f[6] = -lse2; f[8] = -O; f[10] = gO;
}

// Thread-per-key loop of the backward, two queries per instruction: the sums
// of bwd_key_loop over the even and the odd queries, added at the end.
template <bool OFFSET>
__device__ __forceinline__ void bwd_key_loop_x2(const float4 A, const float4 B, const float4 *__restrict__ sq2,
                                                int pairs, float acc[8])
{
    const float2 ax = dup2(A.x), ay = dup2(A.y), az = dup2(A.z), nbl = dup2(A.w);
    const float2 bo = dup2(B.x), bx = dup2(B.y), by = dup2(B.z), bz = dup2(B.w);
    const float2 z2 = make_float2(0.f, 0.f);
    float2 ag = z2, arx = z2, ary = z2, arz = z2, ab = z2, adx = z2, ady = z2, adz = z2;
#pragma unroll 2
    for (int jp = 0; jp < pairs; ++jp) {
        const float4 Q0 = sq2[3 * jp], Q1 = sq2[3 * jp + 1], S = sq2[3 * jp + 2];
        const float2 rx = sub2(lo2(Q0), ax), ry = sub2(hi2(Q0), ay), rz = sub2(lo2(Q1), az);
        const float2 d2 = fma2(rx, rx, fma2(ry, ry, mul2(rz, rz)));
        const float2 w = ex2_2(fma2(nbl, d2, hi2(Q1)));
        const float2 g = mul2(w, hi2(S));
        const float2 f = fma2(bx, rx, fma2(by, ry, fma2(bz, rz, bo)));
        const float2 gd = mul2(g, add2(f, lo2(S)));
        ag = add2(ag, g);
        arx = fma2(g, rx, arx);
        ary = fma2(g, ry, ary);
        arz = fma2(g, rz, arz);
        ab = fma2(gd, d2, ab);
        if (OFFSET) {
            adx = fma2(gd, rx, adx);
            ady = fma2(gd, ry, ady);
            adz = fma2(gd, rz, adz);
        }
    }
    acc[0] = ag.x + ag.y; acc[1] = arx.x + arx.y; acc[2] = ary.x + ary.y; acc[3] = arz.x + arz.y;
    acc[4] = ab.x + ab.y; acc[5] = adx.x + adx.y; acc[6] = ady.x + ady.y; acc[7] = adz.x + adz.y;
}

// ------------------------------------------------------------- kernel

// Forward over the item's queries.  qt holds the raw query tile (x, y, z,
// target); a query's row is rewritten in place with (local position, lse2)
// by the lane that owns it, after every lane of its group has read it.
template <int MODE, bool DQ, bool GEIK, int KQ, bool FULL, typename T>
__device__ __forceinline__ void forward_phase(const FusedArgsT<T> &a, const V4Of<T> *rec, const float4 *rec2,
                                              V4Of<T> *qt, V4Of<T> *sqB, float4 *sq2, float4 *sqE, float4 *sqU,
                                              int start, int n, int nc, V4Of<T> orig, T h, T &loss_acc, T &abs_acc)
{
    using N = Num<T>;
    using V = V4Of<T>;
    constexpr bool PAIRS = std::is_same<T, float>::value;   // packed FP32 forward
    constexpr bool PAIRQ = PAIRS && !GEIK;                 // packed FP32 backward
    constexpr int LG = KQ == 1 ? 0 : (KQ == 2 ? 1 : 2);
    const int t = threadIdx.x;
    const int part = t & (KQ - 1);
    constexpr int per_round = kThreads / KQ;
    for (int base = 0; base < n; base += per_round) {
        // a warp without a query in this round leaves its issue slots to the other CTAs
        if (base + ((t & ~31) >> LG) >= n) continue;
        const int qi = base + (t >> LG);
        const bool valid = qi < n;
        int j_user = 0;
        if (MODE != FIT && MODE != EVAL) j_user = valid ? __ldg(a.perm + start + qi) : 0;   // issued before the long compute
        auto local_query = [&](int i) {
            V v = N::v4(T(0.5) * h, T(0.5) * h, T(0.5) * h, T(0));
            if (i < n) {
                v = qt[i];
                v.x -= orig.x;
                v.y -= orig.y;
                v.z -= orig.z;
            }
            return v;
        };
        V q;
        FwdOut<T> r;
        if constexpr (PAIRS) {
            if constexpr (KQ == 1 && FULL) {
                const V qa = local_query(qi & ~1), qb = local_query(qi | 1);
                q = (t & 1) ? qb : qa;
                r = forward_query_x2<KQ, FULL>(rec2, nc, part, h, q, qa, qb);
            } else {
                q = local_query(valid ? qi : n);
                r = forward_query_x2<KQ, FULL>(rec2, nc, part, h, q, q, q);
            }
        } else {
            q = local_query(valid ? qi : n);
            r = forward_query<KQ, FULL>(rec, nc, part, h, q);
        }
        const T O = r.O, lse2 = r.lse2;

        T gO = T(0);
        if (MODE == FIT) {
            const T diff = O - q.w;
            if (a.loss == EFUNC_LOSS_L1) gO = diff > T(0) ? (T)a.inv_J : (diff < T(0) ? -(T)a.inv_J : T(0));
            else gO = T(2) * diff * (T)a.inv_J;
            if (valid && part == 0) {
                loss_acc += a.loss == EFUNC_LOSS_L1 ? fabs(diff) : diff * diff;
                abs_acc += fabs(diff);
            }
        } else if (MODE == EVAL) {
            const T diff = O - q.w;
            if (valid && part == 0) {
                loss_acc += diff * diff;
                abs_acc += fabs(diff);
            }
        } else if (MODE == BACKWARD) {
            gO = (valid && a.gO) ? __ldg(a.gO + j_user) : T(0);
        } else if (valid && part == 0) {
            a.O[j_user] = O;
            if (a.lse) a.lse[j_user] = lse2 * N::kLn2;
        }
        if (DQ) {
            T gx, gy, gz;
            dq_sums<KQ>(rec, nc, part, q.x, q.y, q.z, lse2, O, gx, gy, gz);
            if (valid && part == 0) {
                T *dst = MODE == FORWARD ? a.dq : a.gq;
                const T s = MODE == FORWARD ? T(1) : gO;
                dst[3 * (size_t)j_user + 0] = s * gx;
                dst[3 * (size_t)j_user + 1] = s * gy;
                dst[3 * (size_t)j_user + 2] = s * gz;
            }
        }
        if (GEIK) {
            // second order (FP32 only): u = dL/d(dO/dq), H = u . dO/dq,
            // T = -2 u . sum w beta (q - key)
            float G[3], Vs[3];
            gv_sums<KQ>(reinterpret_cast<const float4 *>(rec), nc, part, (float)q.x, (float)q.y, (float)q.z,
                        (float)lse2, (float)O, G, Vs);
            float u0 = 0.f, u1 = 0.f, u2 = 0.f;
            if (MODE == FIT) {
                // Eikonal term of Sec. 3.2 in the squared form: weight (|G|^2 - 1)^2 / J
                const float res = fmaf(G[0], G[0], fmaf(G[1], G[1], fmaf(G[2], G[2], -1.f)));
                const float c = 4.f * a.eik_weight * res * a.inv_J;
                u0 = c * G[0]; u1 = c * G[1]; u2 = c * G[2];
                if (valid && part == 0) loss_acc += a.eik_weight * res * res;
            } else if (valid) {
                u0 = __ldg(a.gG + 3 * (size_t)j_user);
                u1 = __ldg(a.gG + 3 * (size_t)j_user + 1);
                u2 = __ldg(a.gG + 3 * (size_t)j_user + 2);
            }
            const float H = fmaf(u0, G[0], fmaf(u1, G[1], u2 * G[2]));
            const float Tt = -2.f * fmaf(u0, Vs[0], fmaf(u1, Vs[1], u2 * Vs[2]));
            if (valid && part == 0) {
                sqE[qi] = make_float4((float)O, (float)gO, H, Tt);
                sqU[qi] = make_float4(u0, u1, u2, 0.f);
            }
        }
        if constexpr (PAIRQ && (MODE == BACKWARD || MODE == FIT)) {
            if (valid && part == 0) {
                store_pair_query(sq2, qi, q, lse2, O, gO);
                if (qi == n - 1 && (n & 1)) store_pair_query(sq2, n, q, lse2, O, 0.f);
            }
        } else if (MODE == BACKWARD || MODE == FIT) {
            __syncwarp();   // every lane of the group has read its row of qt
            if (valid && part == 0) {
                const V qa = N::v4(q.x, q.y, q.z, lse2);
                typename N::V2 *sqB2 = reinterpret_cast<typename N::V2 *>(sqB);
                qt[qi] = qa;
                sqB2[qi] = N::v2(O, gO);
                if (qi == n - 1 && (n & 1)) {   // pad the last pair: same query, no gradient
                    qt[n] = qa;
                    sqB2[n] = N::v2(O, T(0));
                }
            }
        }
    }
}

// Resident CTAs per SM asked of the compiler: the FP32 kernels run 8 CTAs
// of 64 registers (7 beside a block of the next batch's sort in the
// pipelined fit); the second-order and FP64 kernels need more registers.
template <bool GEIK, typename T>
constexpr int min_ctas() { return sizeof(T) == 8 ? 2 : (GEIK ? 5 : 8); }

// One work item: stage, forward, backward.  ai carries the item's grid
// (R, key records, gradient, 1/J): the kernel's own arguments, or in a
// batched launch those of the item's shape.
template <int MODE, bool DQ, bool GEIK, typename T, bool BATCHED>
__device__ __forceinline__ void item_body(const FusedArgsT<T> &a, const FusedArgsT<T> &ai, const BatchArgs &b, const Item item,
                                          const int R, const T invR, const T h, V4Of<T> *rec, float4 *rec2,
                                          float4 *keyT, V4Of<T> *qt, V4Of<T> *qB, float4 *sq2, float4 *s_sqE,
                                          float4 *s_sqU, T &loss_acc, T &abs_acc)
{
    using N = Num<T>;
    using V = V4Of<T>;
    constexpr bool BWD = MODE == BACKWARD || MODE == FIT;
    constexpr bool PAIRS = std::is_same<T, float>::value;   // paired key tile, packed forward
    constexpr bool NEED_REC = !PAIRS || DQ || GEIK;        // the per-key tile (dO/dq sums, FP64)
    constexpr bool PAIRQ = PAIRS && !GEIK;                 // paired query rows, packed backward
    const int t = threadIdx.x;
    if (!bounds_ok(item.x >= 0 && item.y >= 1 && item.y <= kChunk, 8)) return;   // uniform in the CTA
    const Window w = window_of(item, R);
    const int start = item.x, n = item.y, nc = w.nc;
    const bool full = nc == kCentres;
    const V orig = N::v4((T)(2 * w.cx + 1 - R) * invR, (T)(2 * w.cy + 1 - R) * invR,
                         (T)(2 * w.cz + 1 - R) * invR, T(0));
    // ---- 1. stage the key records (positions made window-local) and
    // queries: thread t stages key t (set t / 64 of centre t mod 64)
    const int kc = t & (kCentres - 1), kset = t / kCentres;
    // keys past the window's last centre (up to a multiple of 4) are neutral
    V A = N::v4(T(1e18), T(1e18), T(1e18), T(-1)), B = N::v4(T(0), T(0), T(0), T(0));
    if (kc < nc) {
        int ox, oy, oz;
        if (full) { ox = kc >> 4; oy = (kc >> 2) & 3; oz = kc & 3; }
        else { oz = kc % w.nz; oy = (kc / w.nz) % w.ny; ox = kc / (w.ny * w.nz); }
        int ix = w.lox + ox, iy = w.loy + oy, iz = w.loz + oz;
        if (!bounds_ok((unsigned)ix < (unsigned)R && (unsigned)iy < (unsigned)R && (unsigned)iz < (unsigned)R, 1))
            ix = iy = iz = 0;   // read centre 0 instead
        const V *k = ai.keys + (((size_t)ix * R + iy) * R + iz) * kKeyRecords;
        const T gx = (T)(2 * (w.lox + ox - w.cx)) * invR, gy = (T)(2 * (w.loy + oy - w.cy)) * invR,
                gz = (T)(2 * (w.loz + oz - w.cz)) * invR;
        const V p = k[2 * kset];
        B = k[2 * kset + 1];
        A = kset ? N::v4(gx + p.x, gy + p.y, gz + p.z, p.w) : N::v4(gx, gy, gz, p.w);
        if constexpr (NEED_REC) {
            rec[4 * kc + 2 * kset] = A;
            rec[4 * kc + 2 * kset + 1] = B;
        }
        if constexpr (PAIRS) {
            keyT[2 * t] = A;
            keyT[2 * t + 1] = B;
        }
    }
    if constexpr (PAIRS) stage_pair_keys(rec2, kset, kc, kc < ((nc + 3) & ~3), A, B);
    for (int qi = t; qi < n; qi += kThreads) {
        qt[qi] = a.sorted[start + qi];
#ifdef EFUNC_DEBUG_BOUNDS
        if constexpr (std::is_same<T, float>::value) {
            const float half_r = (float)R * 0.5f, rmax = (float)(R - 1);
            const float4 q = qt[qi];
            bounds_ok(window_base(q.x, half_r, rmax) == w.cx && window_base(q.y, half_r, rmax) == w.cy &&
                          window_base(q.z, half_r, rmax) == w.cz, 2);
        }
#endif
    }
    __syncthreads();

    // ---- 2. forward, one (or 2 / 4) threads per query
    // single grids: no four-lane items (those lanes would blend every pair twice;
    // two lanes per query are faster, same-process A/B at 64^3 x 2^24: -3.6 %)
    const int l2 = BATCHED ? b.lanes2_max : 64, l4 = BATCHED ? b.lanes4_max : 0;
    if (full) {
        if (n > l2) forward_phase<MODE, DQ, GEIK, 1, true>(ai, rec, rec2, qt, qB, sq2, s_sqE, s_sqU, start, n, nc, orig, h, loss_acc, abs_acc);
        else if (n > l4) forward_phase<MODE, DQ, GEIK, 2, true>(ai, rec, rec2, qt, qB, sq2, s_sqE, s_sqU, start, n, nc, orig, h, loss_acc, abs_acc);
        else forward_phase<MODE, DQ, GEIK, 4, true>(ai, rec, rec2, qt, qB, sq2, s_sqE, s_sqU, start, n, nc, orig, h, loss_acc, abs_acc);
    } else {
        if (n > l2) forward_phase<MODE, DQ, GEIK, 1, false>(ai, rec, rec2, qt, qB, sq2, s_sqE, s_sqU, start, n, nc, orig, h, loss_acc, abs_acc);
        else if (n > l4) forward_phase<MODE, DQ, GEIK, 2, false>(ai, rec, rec2, qt, qB, sq2, s_sqE, s_sqU, start, n, nc, orig, h, loss_acc, abs_acc);
        else forward_phase<MODE, DQ, GEIK, 4, false>(ai, rec, rec2, qt, qB, sq2, s_sqE, s_sqU, start, n, nc, orig, h, loss_acc, abs_acc);
    }
    if (BWD) {
        // ---- 3. backward, one thread per key (the window is formed again
        // from the item instead of being held through the forward)
        __syncthreads();
        const int c = t & (kCentres - 1);
        const Window w = window_of(item, R);
        const bool full = w.nc == kCentres;
        if (c < w.nc) {
            const bool offset = t >= kCentres;
            V A, B;
            if constexpr (PAIRS) {
                A = keyT[2 * t];   // staged by this thread
                B = keyT[2 * t + 1];
            } else {
                A = keyA(rec, offset, c);
                B = keyB(rec, offset, c);
            }
            T acc[19];
            if constexpr (PAIRQ) {
                float accf[8];
                if (offset) bwd_key_loop_x2<true>(A, B, sq2, (n + 1) >> 1, accf);
                else bwd_key_loop_x2<false>(A, B, sq2, (n + 1) >> 1, accf);
                for (int i = 0; i < 8; ++i) acc[i] = accf[i];
                for (int i = 8; i < 19; ++i) acc[i] = T(0);
            } else if (GEIK) {
                float accf[19];
                const float4 Af = make_float4((float)A.x, (float)A.y, (float)A.z, (float)A.w);
                const float4 Bf = make_float4((float)B.x, (float)B.y, (float)B.z, (float)B.w);
                const float4 *qtf = reinterpret_cast<const float4 *>(qt);
                if (offset) bwd2_key_loop<true>(Af, Bf, qtf, s_sqE, s_sqU, n, accf);
                else bwd2_key_loop<false>(Af, Bf, qtf, s_sqE, s_sqU, n, accf);
                for (int i = 0; i < 19; ++i) acc[i] = accf[i];
            } else {
                if (offset) bwd_key_loop<true>(A, B, qt, qB, n, acc);
                else bwd_key_loop<false>(A, B, qt, qB, n, acc);
                for (int i = 8; i < 19; ++i) acc[i] = T(0);
            }
            int ox, oy, oz;
            if (full) { ox = c >> 4; oy = (c >> 2) & 3; oz = c & 3; }
            else { oz = c % w.nz; oy = (c / w.nz) % w.ny; ox = c / (w.ny * w.nz); }
            const bool in_grid = bounds_ok((unsigned)(w.lox + ox) < (unsigned)R && (unsigned)(w.loy + oy) < (unsigned)R &&
                                               (unsigned)(w.loz + oz) < (unsigned)R, 1);
            T *gr = ai.grad + (((size_t)(w.lox + ox) * R + (w.loy + oy)) * R + (w.loz + oz)) * kSlots;
            const T beta = -A.w * N::kLn2;
            // value term (dO/dtheta) plus, in second-order mode, the
            // gradient term d(u . dO/dq)/dtheta
            const T go = acc[0] + acc[8];
            const T gdx = acc[1] + acc[9], gdy = acc[2] + acc[10], gdz = acc[3] + acc[11];
            const T gb = beta * (-acc[4] + acc[12]);
            if (!in_grid) {
                // skipped (bounds-check build)
            } else if (!offset) {
                atomicAdd(gr + 5, go);
                atomicAdd(gr + 6, gdx);
                atomicAdd(gr + 7, gdy);
                atomicAdd(gr + 8, gdz);
                atomicAdd(gr + 3, gb);
            } else {
                atomicAdd(gr + 9, go);
                atomicAdd(gr + 10, gdx);
                atomicAdd(gr + 11, gdy);
                atomicAdd(gr + 12, gdz);
                atomicAdd(gr + 4, gb);
                // dO/dDelta = w (-d' + 2 beta' (q - key)(f' - O)); d(u.G)/dDelta as above
                const T tb = T(2) * beta;
                atomicAdd(gr + 0, N::fma(-B.y, go, tb * (acc[5] + acc[13] + acc[16])));
                atomicAdd(gr + 1, N::fma(-B.z, go, tb * (acc[6] + acc[14] + acc[17])));
                atomicAdd(gr + 2, N::fma(-B.w, go, tb * (acc[7] + acc[15] + acc[18])));
            }
        }
    }
}

// BATCHED: the items of many shapes in one launch; an item's shape (Item.w)
// selects its grid (R, key records, gradient, 1/J) and the loss sums go to
// that shape's pair in a.shape_sums after every item.
template <int MODE, bool DQ, bool GEIK, typename T = float, bool BATCHED = false>
__global__ void __launch_bounds__(kThreads, min_ctas<GEIK, T>()) fused_kernel(FusedArgsT<T> a, BatchArgs b)
{
    using V = V4Of<T>;
    constexpr bool BWD = MODE == BACKWARD || MODE == FIT;
    constexpr bool PAIRS = std::is_same<T, float>::value;
    constexpr bool NEED_REC = !PAIRS || DQ || GEIK;
    constexpr bool PAIRQ = PAIRS && !GEIK && BWD;
    __shared__ V s_rec[NEED_REC ? kCentres * kKeyRecords : 1];      // key records of the window
    __shared__ float4 s_rec2[PAIRS ? 2 * kPairs * 4 : 1];           // the same keys, paired (FP32)
    __shared__ float4 s_keyT[PAIRS ? 2 * kThreads : 1];             // (A, B) of thread t's key (FP32)
    __shared__ V s_qt[kChunk];                                      // query tile
    __shared__ V s_sqB[BWD && !PAIRQ ? kChunk / 2 : 1];
    __shared__ float4 s_sq2[PAIRQ ? 3 * kChunk / 2 : 1];            // paired query rows (FP32 backward)
    __shared__ float4 s_sqE[GEIK ? kChunk : 1];               // (O, gO, H, T) per query
    __shared__ float4 s_sqU[GEIK ? kChunk : 1];               // (u, 0) per query
    __shared__ int s_item;
    __shared__ T s_red[2][kThreads / 32];

    const int t = threadIdx.x;
    const int R = a.R;
    const T invR = T(1) / (T)R;    // exact for power-of-two R
    const T h = T(2) * invR;
    const int n_items = a.ctrl->n_items;
    T loss_acc = T(0), abs_acc = T(0);

    if (t == 0) s_item = atomicAdd(&a.ctrl->next_item, 1);
    for (;;) {
        __syncthreads();   // s_item published; the previous item is consumed
        const int it = s_item;
        if (it >= n_items) break;
        const Item item = a.items[it];
        if constexpr (BATCHED) {
            const BatchShape sh = b.shapes[item.w];
            FusedArgsT<T> ai = a;
            ai.R = sh.R;
            ai.keys = a.keys + sh.c_off * kKeyRecords;
            ai.grad = a.grad + sh.c_off * kSlots;
            ai.inv_J = sh.inv_J;
            const T invRb = T(1) / (T)sh.R;
            item_body<MODE, DQ, GEIK, T, BATCHED>(a, ai, b, item, sh.R, invRb, T(2) * invRb, s_rec, s_rec2, s_keyT,
                                                  s_qt, s_sqB, s_sq2, s_sqE, s_sqU, loss_acc, abs_acc);
            if (MODE == FIT || MODE == EVAL) {
                // this item's loss sums to its shape: one double atomic pair per warp
                for (int o = 16; o > 0; o >>= 1) {
                    loss_acc += __shfl_xor_sync(kFull, loss_acc, o);
                    abs_acc += __shfl_xor_sync(kFull, abs_acc, o);
                }
                if ((t & 31) == 0 && (loss_acc != T(0) || abs_acc != T(0))) {
                    atomicAdd(b.shape_sums + 2 * item.w, (double)loss_acc);
                    atomicAdd(b.shape_sums + 2 * item.w + 1, (double)abs_acc);
                }
                loss_acc = abs_acc = T(0);
            }
        } else {
            item_body<MODE, DQ, GEIK, T, BATCHED>(a, a, b, item, R, invR, h, s_rec, s_rec2, s_keyT, s_qt, s_sqB,
                                                  s_sq2, s_sqE, s_sqU, loss_acc, abs_acc);
        }
        // thread 0 has done its share of the item: claim the next one while
        // the other warps finish theirs (every thread read s_item before the
        // staging barrier of this item)
        if (t == 0) s_item = atomicAdd(&a.ctrl->next_item, 1);
    }

    if (!BATCHED && (MODE == FIT || MODE == EVAL)) {
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
            for (int wi = 0; wi < kThreads / 32; ++wi) {
                l += s_red[0][wi];
                ab += s_red[1][wi];
            }
            atomicAdd(&a.ctrl->loss_sum, l);
            atomicAdd(&a.ctrl->abs_sum, ab);
        }
    }
}

int sm_count() { return device_sm_count(); }

}  // namespace

int fused_grid_size()
{
    const void *k = reinterpret_cast<const void *>(fused_kernel<FIT, false, false>);
    return per_device_cached(k, 0, [k] {
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kThreads, 0);
        if (per_sm <= 0) per_sm = 1;
        return sm_count() * per_sm;
    });
}

int fused_fit_grid_size(bool eikonal, bool leave_room)
{
    const void *k = eikonal ? reinterpret_cast<const void *>(fused_kernel<FIT, false, true>)
                            : reinterpret_cast<const void *>(fused_kernel<FIT, false, false>);
    return per_device_cached(k, leave_room ? 2 : 1, [k, leave_room] {
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kThreads, 0);
        if (per_sm <= 0) per_sm = 1;
        if (leave_room) per_sm = leave_sort_room(k, per_sm);
        return sm_count() * per_sm;
    });
}

int leave_sort_room(const void *kernel, int per_sm, int sort_blocks)
{
    cudaFuncAttributes fa{};
    int dev = 0, regs_sm = 65536;
    cudaFuncGetAttributes(&fa, kernel);
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    const int per_cta = (fa.numRegs + 7) / 8 * 8 * kThreads;
    while (per_sm > 1 && per_sm * per_cta > regs_sm - sort_blocks * kSortThreads * 32) --per_sm;
    return per_sm;
}

cudaError_t launch_pack_keys(const PackArgs &a, cudaStream_t s)
{
    const int I = a.R * a.R * a.R;
    int blocks = (I + 255) / 256;
    if (blocks > sm_count() * 8) blocks = sm_count() * 8;
    launch_begin(K_PACK_KEYS, s);
    pack_keys_kernel<float><<<blocks, 256, 0, s>>>(a);
    launch_end(K_PACK_KEYS, s);
    return cudaGetLastError();
}

cudaError_t launch_forward(const FusedArgs &a, bool with_dq, int grid, cudaStream_t s)
{
    launch_begin(K_FORWARD, s);
    if (with_dq) fused_kernel<FORWARD, true, false><<<grid, kThreads, 0, s>>>(a, BatchArgs{});
    else fused_kernel<FORWARD, false, false><<<grid, kThreads, 0, s>>>(a, BatchArgs{});
    launch_end(K_FORWARD, s);
    return cudaGetLastError();
}

cudaError_t launch_fused_backward(const FusedArgs &a, bool with_gq, bool second_order, int grid, cudaStream_t s)
{
    launch_begin(K_FUSED_BWD, s);
    if (second_order) fused_kernel<BACKWARD, false, true><<<grid, kThreads, 0, s>>>(a, BatchArgs{});
    else if (with_gq) fused_kernel<BACKWARD, true, false><<<grid, kThreads, 0, s>>>(a, BatchArgs{});
    else fused_kernel<BACKWARD, false, false><<<grid, kThreads, 0, s>>>(a, BatchArgs{});
    launch_end(K_FUSED_BWD, s);
    return cudaGetLastError();
}

cudaError_t launch_fused_fit(const FusedArgs &a, bool eikonal, int grid, cudaStream_t s)
{
    launch_begin(K_FUSED_FIT, s);
    if (eikonal) fused_kernel<FIT, false, true><<<grid, kThreads, 0, s>>>(a, BatchArgs{});
    else fused_kernel<FIT, false, false><<<grid, kThreads, 0, s>>>(a, BatchArgs{});
    launch_end(K_FUSED_FIT, s);
    return cudaGetLastError();
}

cudaError_t launch_fused_eval(const FusedArgs &a, int grid, cudaStream_t s)
{
    launch_begin(K_EVAL, s);
    fused_kernel<EVAL, false, false><<<grid, kThreads, 0, s>>>(a, BatchArgs{});
    launch_end(K_EVAL, s);
    return cudaGetLastError();
}

namespace {
__global__ void eval_finish_kernel(const Ctrl *ctrl, double inv_J, float *out)
{
    out[0] = (float)(ctrl->loss_sum * inv_J);
    out[1] = (float)(ctrl->abs_sum * inv_J);
}
}  // namespace

cudaError_t launch_eval_finish(const Ctrl *ctrl, double inv_J, float *out, cudaStream_t s)
{
    launch_begin(K_EVAL_FINISH, s);
    eval_finish_kernel<<<1, 1, 0, s>>>(ctrl, inv_J, out);
    launch_end(K_EVAL_FINISH, s);
    return cudaGetLastError();
}

// ------------------------------------------------------------ grouped items
//
// A grouped item is an aligned 2x2x2 octet of window-base cells holding few
// queries (the sort groups sparse octets).  The union of the octet's
// windows, at most 5x5x5 centres, is staged once; every query blends its own
// 4x4x4 sub-window (the same keys, in the same order and summation classes
// as the generic path of fused_kernel).  The backward walks the octet's
// sub-cells in turn: for each, all 128 threads take the 128 keys of its
// window over its queries (two per instruction), so that no lane idles on
// another lane's queries, and add their sums to a shared gradient tile of
// the union; the tile then goes to the gradient with one atomic per non-zero
// entry, consecutive threads on consecutive floats of a z-row.  Compared
// with one item per cell, the window is staged and each key's gradient is
// added once per octet instead of once per cell.

namespace {

constexpr int kGU = 5;                      // union window per axis
constexpr int kGCentres = kGU * kGU * kGU;  // 125

struct GroupWin {
    int c0x, c0y, c0z;      // window base of the octet's first cell
    int lox, loy, loz;      // first centre of the union window
    int nx, ny, nz, nc;     // its extent (clipped to the grid)
};

// t / n for 1 <= n <= 5 and 0 <= t < 13107, exact: (t * ceil(2^16 / n)) >> 16
// (the error t (ceil(2^16 / n) - 2^16 / n) / 2^16 stays below 1 / n).
__device__ __forceinline__ int small_div(int t, int n) { return (t * ((65536 + n - 1) / n)) >> 16; }

// Union key tile of a grouped item: four arrays of kGCentres records
// (grid A, grid B, offset A, offset B), so that lanes reading different
// centres fall on consecutive 16-byte bank groups.
__device__ __forceinline__ float4 gA(const float4 *rec, int set, int c) { return rec[2 * set * kGCentres + c]; }
__device__ __forceinline__ float4 gB(const float4 *rec, int set, int c) { return rec[(2 * set + 1) * kGCentres + c]; }

__device__ __forceinline__ GroupWin group_window(const Item item, int R)
{
    GroupWin g;
    g.c0x = (item.z & 1023) - 1;
    g.c0y = ((item.z >> 10) & 1023) - 1;
    g.c0z = ((item.z >> 20) & 1023) - 1;
    g.lox = max(g.c0x - 1, 0);
    g.loy = max(g.c0y - 1, 0);
    g.loz = max(g.c0z - 1, 0);
    g.nx = min(g.c0x + 3, R - 1) - g.lox + 1;
    g.ny = min(g.c0y + 3, R - 1) - g.loy + 1;
    g.nz = min(g.c0z + 3, R - 1) - g.loz + 1;
    g.nc = g.nx * g.ny * g.nz;
    return g;
}

// (e, m) of one query over its own window inside the staged union: axis
// ranges [w0, w0 + wn) of the union's centre indices, keys in the order of
// fwd_sums (set outer, then x, y, z with z fastest), class of key k = k mod 4.
// A full window (4 along y and z) is walked row by row without divisions.
template <int KQ>
__device__ __forceinline__ void grp_fwd_sums(const float4 *rec, const GroupWin &g, int w0x, int w0y, int w0z,
                                             int wnx, int wny, int wnz, int part, float x, float y, float z, float M2,
                                             float &e, float &m)
{
    constexpr int CPL = kClasses / KQ;
    float ev[CPL], mv[CPL];
#pragma unroll
    for (int i = 0; i < CPL; ++i) ev[i] = mv[i] = 0.f;
    const int nq = wnx * wny * wnz;
    const int cbase = (w0x * g.ny + w0y) * g.nz + w0z;
    if (wny == 4 && wnz == 4) {
#pragma unroll
        for (int set = 0; set < 2; ++set) {
            for (int base = 0; base < nq; base += kClasses) {
                const int r = base >> 2;   // row (kx, ky) = (r >> 2, r & 3)
                const int row = cbase + (r >> 2) * (g.ny * g.nz) + (r & 3) * g.nz;
#pragma unroll
                for (int i = 0; i < CPL; ++i) {
                    const int c = row + part + KQ * i;
                    fwd_key(gA(rec, set, c), gB(rec, set, c), x, y, z, M2, ev[i], mv[i]);
                }
            }
        }
    } else {
        // clipped window: walk the keys k = part, part + KQ, ... with their
        // union index c, carrying z into y and y into x
#pragma unroll
        for (int set = 0; set < 2; ++set) {
            int kz = part, ky = 0, c = cbase + part;
            while (kz >= wnz) {
                kz -= wnz;
                c += g.nz - wnz;
                if (++ky == wny) {
                    ky = 0;
                    c += (g.ny - wny) * g.nz;
                }
            }
            for (int base = 0; base < nq; base += kClasses) {
#pragma unroll
                for (int i = 0; i < CPL; ++i) {
                    const int k = base + part + KQ * i;
                    if (k < nq) fwd_key(gA(rec, set, c), gB(rec, set, c), x, y, z, M2, ev[i], mv[i]);
                    kz += KQ;
                    c += KQ;
                    while (kz >= wnz) {
                        kz -= wnz;
                        c += g.nz - wnz;
                        if (++ky == wny) {
                            ky = 0;
                            c += (g.ny - wny) * g.nz;
                        }
                    }
                }
            }
        }
    }
    e = combine_classes<KQ>(ev);
    m = combine_classes<KQ>(mv);
}

template <int MODE, int KQ, bool BATCHED>
__device__ __forceinline__ void grp_forward(const int loss, const float inv_J, const float4 *rec, const float4 *qt,
                                            float4 *sq2,
                                            const unsigned char *qoff, const int *beg, const int *pbeg,
                                            const GroupWin &g, int n, int R, float h, float3 orig, float &loss_acc,
                                            float &abs_acc)
{
    constexpr int LG = KQ == 1 ? 0 : (KQ == 2 ? 1 : 2);
    const int t = threadIdx.x;
    const int part = t & (KQ - 1);
    for (int base = 0; base < n; base += kThreads / KQ) {
        const int qi = base + (t >> LG);
        const bool valid = qi < n;
        float4 q = valid ? qt[qi] : make_float4(0.f, 0.f, 0.f, 0.f);
        const int off = valid ? qoff[qi] : 0;
        // the query's window base c = c0 + offset (sub-cell id ox << 2 | oy << 1
        // | oz), its window [c - 1, c + 2] clipped to the grid, relative to
        // the union's first centre
        const int cx = g.c0x + ((off >> 2) & 1), cy = g.c0y + ((off >> 1) & 1), cz = g.c0z + (off & 1);
        const int w0x = max(cx - 1, 0) - g.lox, w0y = max(cy - 1, 0) - g.loy, w0z = max(cz - 1, 0) - g.loz;
        const int wnx = min(cx + 2, R - 1) - g.lox - w0x + 1, wny = min(cy + 2, R - 1) - g.loy - w0y + 1,
                  wnz = min(cz + 2, R - 1) - g.loz - w0z + 1;
        if (valid) {
            q.x -= orig.x;
            q.y -= orig.y;
            q.z -= orig.z;
        } else {
            q.x = q.y = q.z = 0.5f * h;
        }
        float e, m;
        grp_fwd_sums<KQ>(rec, g, w0x, w0y, w0z, wnx, wny, wnz, part, q.x, q.y, q.z, 0.f, e, m);
        float M2 = 0.f;
        const bool tiny = !(e >= 0x1p-60f);
        if (__any_sync(kFull, tiny)) {
            float mx = -INFINITY;
            const int nq = wnx * wny * wnz;
            for (int k = part; k < nq; k += KQ) {
                const int kz = k % wnz, ky = (k / wnz) % wny, kx = k / (wny * wnz);
                const int c = ((w0x + kx) * g.ny + (w0y + ky)) * g.nz + (w0z + kz);
                mx = fmaxf(mx, key_exponent(gA(rec, 0, c), q.x, q.y, q.z));
                mx = fmaxf(mx, key_exponent(gA(rec, 1, c), q.x, q.y, q.z));
            }
#pragma unroll
            for (int o = 1; o < KQ; o <<= 1) mx = fmaxf(mx, __shfl_xor_sync(kFull, mx, o));
            float e2, m2;
            grp_fwd_sums<KQ>(rec, g, w0x, w0y, w0z, wnx, wny, wnz, part, q.x, q.y, q.z, mx, e2, m2);
            if (tiny) {
                e = e2;
                m = m2;
                M2 = mx;
            }
        }
        const float O = m / e, lse2 = M2 + lg2_approx(e);
        const float diff = O - q.w;
        float gO = 0.f;
        if (MODE == FIT) {
            if (loss == EFUNC_LOSS_L1) gO = diff > 0.f ? inv_J : (diff < 0.f ? -inv_J : 0.f);
            else gO = 2.f * diff * inv_J;
            if (valid && part == 0) {
                loss_acc += loss == EFUNC_LOSS_L1 ? fabsf(diff) : diff * diff;
                abs_acc += fabsf(diff);
            }
        } else if (valid && part == 0) {
            loss_acc += diff * diff;
            abs_acc += fabsf(diff);
        }
        if (MODE == FIT && valid && part == 0) {
            // paired rows of the query's sub-cell, an odd last one padded
            const int r = qi - beg[off], p = 2 * pbeg[off] + r;
            if (bounds_ok(p + 1 < 2 * (kChunk / 2 + 8), 5)) {
                store_pair_query(sq2, p, q, lse2, O, gO);
                if (qi == beg[off + 1] - 1 && (r & 1) == 0) store_pair_query(sq2, p + 1, q, lse2, O, 0.f);
            }
        }
    }
}

template <int MODE, bool BATCHED>
__global__ void __launch_bounds__(kThreads, 7) grouped_kernel(FusedArgs a, BatchArgs b, const Item *gtop)
{
    __shared__ float4 s_rec[kGCentres * kKeyRecords];
    __shared__ float4 s_qt[kChunk];
    __shared__ float4 s_sq2[MODE == FIT ? 3 * (kChunk / 2 + 8) : 1];   // paired rows, per sub-cell
    __shared__ float s_grad[MODE == FIT ? kGCentres * kSlots : 1];     // the union's gradient tile
    __shared__ unsigned char s_off[kChunk];
    __shared__ int s_beg[9];          // query range of sub-cell o: [s_beg[o], s_beg[o + 1])
    __shared__ int s_pbeg[9];         // its pairs from s_pbeg[o]
    __shared__ int s_item[2];
    __shared__ float s_red[2][kThreads / 32];
    const int t = threadIdx.x;
    const int n_groups = a.ctrl->n_groups;
    float loss_acc = 0.f, abs_acc = 0.f;
    if (MODE == FIT)
        for (int i = t; i < kGCentres * kSlots; i += kThreads) s_grad[i] = 0.f;
    if (t == 0) s_item[0] = atomicAdd(&a.ctrl->next_group, 1);
    int cur = 0;

    for (;;) {
        __syncthreads();   // the previous item is consumed; s_item[cur] is visible
        const int gi = s_item[cur];
        if (gi >= n_groups) break;
        int next = 0;
        if (t == 0) next = atomicAdd(&a.ctrl->next_group, 1);   // the next item, published at the end
        if (t < 9) s_beg[t] = 0;
        const Item item = gtop[-gi];
        const float4 *keys = a.keys;
        float *grad = a.grad;
        float inv_J = a.inv_J;
        int R = a.R;
        if (BATCHED) {
            const BatchShape sh = b.shapes[item.w];
            R = sh.R;
            keys = a.keys + sh.c_off * kKeyRecords;
            grad = a.grad + sh.c_off * kSlots;
            inv_J = sh.inv_J;
        }
        const float invR = 1.f / (float)R, h = 2.f * invR;
        const float half_r = (float)R * 0.5f, rmax = (float)(R - 1);
        const GroupWin g = group_window(item, R);
        const int start = item.x, n = bounds_ok(item.x >= 0 && item.y >= 1 && item.y <= kChunk, 8) ? item.y : 0;
        const float3 orig = make_float3((float)(2 * g.c0x + 1 - R) * invR, (float)(2 * g.c0y + 1 - R) * invR,
                                        (float)(2 * g.c0z + 1 - R) * invR);
        __syncthreads();   // s_beg cleared
        // ---- stage the union window's key records (window-local) and the queries
        if (t < g.nc) {
            const int rowi = small_div(t, g.nz), oz = t - rowi * g.nz;
            const int ox = small_div(rowi, g.ny), oy = rowi - ox * g.ny;
            int ix = g.lox + ox, iy = g.loy + oy, iz = g.loz + oz;
            if (!bounds_ok((unsigned)ix < (unsigned)R && (unsigned)iy < (unsigned)R && (unsigned)iz < (unsigned)R, 3))
                ix = iy = iz = 0;   // read centre 0 instead
            const float4 *k = keys + (((size_t)ix * R + iy) * R + iz) * kKeyRecords;
            const float gx = (float)(2 * (g.lox + ox - g.c0x)) * invR, gy = (float)(2 * (g.loy + oy - g.c0y)) * invR,
                        gz = (float)(2 * (g.loz + oz - g.c0z)) * invR;
            const float4 kg = k[0], ko = k[2];
            s_rec[t] = make_float4(gx, gy, gz, kg.w);
            s_rec[kGCentres + t] = k[1];
            s_rec[2 * kGCentres + t] = make_float4(gx + ko.x, gy + ko.y, gz + ko.z, ko.w);
            s_rec[3 * kGCentres + t] = k[3];
        }
        for (int qi = t; qi < n; qi += kThreads) {
            const float4 q = a.sorted[start + qi];
            const int cx = window_base(q.x, half_r, rmax), cy = window_base(q.y, half_r, rmax),
                      cz = window_base(q.z, half_r, rmax);
            int o = ((cx - g.c0x) << 2) | ((cy - g.c0y) << 1) | (cz - g.c0z);
            if (!bounds_ok((unsigned)(cx - g.c0x) < 2u && (unsigned)(cy - g.c0y) < 2u && (unsigned)(cz - g.c0z) < 2u, 4))
                o = 0;
            s_qt[qi] = q;
            s_off[qi] = (unsigned char)o;
            atomicAdd(&s_beg[o + 1], 1);
        }
        __syncthreads();
        if (t == 0) {
            // the queries are sorted by sub-cell; pair ranges padded to even counts
            s_pbeg[0] = 0;
            for (int o = 1; o <= 8; ++o) {
                s_pbeg[o] = s_pbeg[o - 1] + ((s_beg[o] + 1) >> 1);
                s_beg[o] += s_beg[o - 1];
            }
        }
        __syncthreads();
        // ---- forward
        if (n > 64) grp_forward<MODE, 1, BATCHED>(a.loss, inv_J, s_rec, s_qt, s_sq2, s_off, s_beg, s_pbeg, g, n, R, h, orig, loss_acc, abs_acc);
        else if (n > 32) grp_forward<MODE, 2, BATCHED>(a.loss, inv_J, s_rec, s_qt, s_sq2, s_off, s_beg, s_pbeg, g, n, R, h, orig, loss_acc, abs_acc);
        else grp_forward<MODE, 4, BATCHED>(a.loss, inv_J, s_rec, s_qt, s_sq2, s_off, s_beg, s_pbeg, g, n, R, h, orig, loss_acc, abs_acc);
        if (MODE == FIT) {
            // ---- backward, sub-cell by sub-cell: thread t takes key t of the
            // sub-cell's window (set t / 64) over the sub-cell's query pairs
            // and adds its sums to the union's gradient tile
            const int kc = t & (kCentres - 1), kset = t / kCentres;
            __syncthreads();   // the paired rows are written
            for (int o = 0; o < 8; ++o) {
                const int npairs = s_pbeg[o + 1] - s_pbeg[o];
                if (npairs == 0) continue;   // uniform
                const int cx = g.c0x + ((o >> 2) & 1), cy = g.c0y + ((o >> 1) & 1), cz = g.c0z + (o & 1);
                const int w0x = max(cx - 1, 0), w0y = max(cy - 1, 0), w0z = max(cz - 1, 0);
                const int wnx = min(cx + 2, R - 1) - w0x + 1, wny = min(cy + 2, R - 1) - w0y + 1,
                          wnz = min(cz + 2, R - 1) - w0z + 1;
                if (kc < wnx * wny * wnz) {
                const int kr = small_div(kc, wnz), kz = kc - kr * wnz;
                const int kx = small_div(kr, wny), ky = kr - kx * wny;
                const int u = ((w0x - g.lox + kx) * g.ny + (w0y - g.loy + ky)) * g.nz + (w0z - g.loz + kz);
                const float4 A = gA(s_rec, kset, u), B = gB(s_rec, kset, u);
                float acc[8];
                if (kset) bwd_key_loop_x2<true>(A, B, s_sq2 + 3 * s_pbeg[o], npairs, acc);
                else bwd_key_loop_x2<false>(A, B, s_sq2 + 3 * s_pbeg[o], npairs, acc);
                float *gt = s_grad + u * kSlots;
                const float beta = -A.w * Num<float>::kLn2;
                if (!kset) {
                    gt[5] += acc[0];
                    gt[6] += acc[1];
                    gt[7] += acc[2];
                    gt[8] += acc[3];
                    gt[3] += -beta * acc[4];
                } else {
                    gt[9] += acc[0];
                    gt[10] += acc[1];
                    gt[11] += acc[2];
                    gt[12] += acc[3];
                    gt[4] += -beta * acc[4];
                    const float tb = 2.f * beta;
                    gt[0] += fmaf(-B.y, acc[0], tb * acc[5]);
                    gt[1] += fmaf(-B.z, acc[0], tb * acc[6]);
                    gt[2] += fmaf(-B.w, acc[0], tb * acc[7]);
                }
                }
                __syncthreads();   // this sub-cell's adds are done
            }
            // ---- the tile to the gradient: rows of nz centres along z are
            // contiguous in the grid, so consecutive threads add consecutive
            // floats; the tile is cleared for the next item
            const int row = g.nz * kSlots, lane = t & 31;
            for (int r = t >> 5; r < g.nx * g.ny; r += kThreads / 32) {
                const int ox = small_div(r, g.ny), oy = r - ox * g.ny;
                float *dst = grad + (((size_t)(g.lox + ox) * R + (g.loy + oy)) * R + g.loz) * kSlots;
                float *src = s_grad + r * row;
                const bool in_grid = bounds_ok((unsigned)(g.lox + ox) < (unsigned)R && (unsigned)(g.loy + oy) < (unsigned)R &&
                                                   (unsigned)g.loz + (unsigned)g.nz <= (unsigned)R, 3);
                for (int f = lane; f < row && in_grid; f += 32) {
                    const float v = src[f];
                    if (v != 0.f) {
                        atomicAdd(dst + f, v);
                        src[f] = 0.f;
                    }
                }
            }
        }
        if (BATCHED) {
            for (int o = 16; o > 0; o >>= 1) {
                loss_acc += __shfl_xor_sync(kFull, loss_acc, o);
                abs_acc += __shfl_xor_sync(kFull, abs_acc, o);
            }
            if ((t & 31) == 0 && (loss_acc != 0.f || abs_acc != 0.f)) {
                atomicAdd(b.shape_sums + 2 * item.w, (double)loss_acc);
                atomicAdd(b.shape_sums + 2 * item.w + 1, (double)abs_acc);
            }
            loss_acc = abs_acc = 0.f;
        }
        if (t == 0) s_item[cur ^ 1] = next;
        cur ^= 1;
    }
    if (!BATCHED) {
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

}  // namespace


int bounds_code_fused()
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

cudaError_t launch_grouped(const FusedArgs &a, const BatchArgs &b, const Item *gtop, bool eval, cudaStream_t s)
{
    const bool batched = b.shapes != nullptr;
    const void *k = batched ? (eval ? reinterpret_cast<const void *>(grouped_kernel<EVAL, true>)
                                    : reinterpret_cast<const void *>(grouped_kernel<FIT, true>))
                            : (eval ? reinterpret_cast<const void *>(grouped_kernel<EVAL, false>)
                                    : reinterpret_cast<const void *>(grouped_kernel<FIT, false>));
    const int grid = per_device_cached(k, 0, [k] {
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kThreads, 0);
        if (per_sm <= 0) per_sm = 1;
        return sm_count() * per_sm;
    });
    launch_begin(K_GROUPED, s);
    if (batched) {
        if (eval) grouped_kernel<EVAL, true><<<grid, kThreads, 0, s>>>(a, b, gtop);
        else grouped_kernel<FIT, true><<<grid, kThreads, 0, s>>>(a, b, gtop);
    } else {
        if (eval) grouped_kernel<EVAL, false><<<grid, kThreads, 0, s>>>(a, b, gtop);
        else grouped_kernel<FIT, false><<<grid, kThreads, 0, s>>>(a, b, gtop);
    }
    launch_end(K_GROUPED, s);
    return cudaGetLastError();
}

// ------------------------------------------------------------ batched fit

namespace {

// Key records of every centre of the concatenated grids (pack_keys_kernel
// per shape: each shape's own log_beta0).
__global__ void __launch_bounds__(256) pack_keys_batched_kernel(BatchedPackArgs a)
{
    __shared__ int64_t s_off[kMaxShapes];
    for (int i = threadIdx.x; i < a.S; i += blockDim.x) s_off[i] = a.shapes[i].c_off;
    __syncthreads();
    const double log2e = 1.4426950408889634;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n_centres;
         i += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = a.S - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_off[mid] <= i) lo = mid;
            else hi = mid - 1;
        }
        const double lb = a.shapes[lo].log_beta0;
        const float *th = a.params + i * kSlots;
        float v[kSlots];
#pragma unroll
        for (int s = 0; s < kSlots; ++s) v[s] = __ldg(th + s);
        float4 *k = a.keys + i * kKeyRecords;
        k[0] = make_float4(0.f, 0.f, 0.f, (float)(-exp(lb + (double)v[3]) * log2e));
        k[1] = make_float4(v[5], v[6], v[7], v[8]);
        k[2] = make_float4(v[0], v[1], v[2], (float)(-exp(lb + (double)v[4]) * log2e));
        k[3] = make_float4(v[9], v[10], v[11], v[12]);
    }
}

// Per-shape statistics of a batched step (loss, MAE per shape, in the row of
// the step held by the Adam clock), or of an evaluation (MSE, MAE), and the
// sums cleared for the next step.
__global__ void batched_stats_kernel(BatchedStatsArgs a)
{
    const AdamClock *clk = static_cast<const AdamClock *>(a.clk);
    const int64_t row = clk ? clk->t - clk->t_first : 0;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < a.S; s += gridDim.x * blockDim.x) {
        const double inv_J = (double)a.shapes[s].inv_J;
        const float l = (float)(a.sums[2 * s] * inv_J), ab = (float)(a.sums[2 * s + 1] * inv_J);
        if (a.stats) {
            a.stats[(row * a.S + s) * 2] = l;
            a.stats[(row * a.S + s) * 2 + 1] = ab;
        }
        if (a.out) {
            a.out[2 * s] = l;
            a.out[2 * s + 1] = ab;
        }
        a.sums[2 * s] = 0.0;
        a.sums[2 * s + 1] = 0.0;
    }
}

}  // namespace

int fused_batched_grid_size()
{
    const void *k = reinterpret_cast<const void *>(fused_kernel<FIT, false, false, float, true>);
    return per_device_cached(k, 0, [k] {
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kThreads, 0);
        if (per_sm <= 0) per_sm = 1;
        return sm_count() * per_sm;
    });
}

cudaError_t launch_pack_keys_batched(const BatchedPackArgs &a, cudaStream_t s)
{
    int64_t blocks = (a.n_centres + 255) / 256;
    if (blocks > (int64_t)sm_count() * 8) blocks = (int64_t)sm_count() * 8;
    launch_begin(K_PACK_KEYS, s);
    pack_keys_batched_kernel<<<(unsigned)(blocks < 1 ? 1 : blocks), 256, 0, s>>>(a);
    launch_end(K_PACK_KEYS, s);
    return cudaGetLastError();
}

cudaError_t launch_fused_batched(const FusedArgs &a, const BatchArgs &b, bool eval, int grid, cudaStream_t s)
{
    launch_begin(eval ? K_EVAL : K_BATCHED, s);
    if (eval) fused_kernel<EVAL, false, false, float, true><<<grid, kThreads, 0, s>>>(a, b);
    else fused_kernel<FIT, false, false, float, true><<<grid, kThreads, 0, s>>>(a, b);
    launch_end(eval ? K_EVAL : K_BATCHED, s);
    return cudaGetLastError();
}

cudaError_t launch_batched_stats(const BatchedStatsArgs &a, cudaStream_t s)
{
    launch_begin(K_BATCHED_STATS, s);
    batched_stats_kernel<<<(a.S + 127) / 128, 128, 0, s>>>(a);
    launch_end(K_BATCHED_STATS, s);
    return cudaGetLastError();
}

// ------------------------------------------------------------ FP64 path

int fused_grid_size64()
{
    const void *k = reinterpret_cast<const void *>(fused_kernel<BACKWARD, true, false, double>);
    return per_device_cached(k, 0, [k] {
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kThreads, 0);
        if (per_sm <= 0) per_sm = 1;
        return sm_count() * per_sm;
    });
}

namespace {
int stream_blocks(int64_t n)
{
    int64_t blocks = (n + 255) / 256;
    if (blocks > (int64_t)sm_count() * 8) blocks = (int64_t)sm_count() * 8;
    return blocks < 1 ? 1 : (int)blocks;
}
}  // namespace

cudaError_t launch_pack_keys64(const PackArgs64 &a, cudaStream_t s)
{
    launch_begin(K_F64, s);
    pack_keys_kernel<double><<<stream_blocks((int64_t)a.R * a.R * a.R), 256, 0, s>>>(a);
    launch_end(K_F64, s);
    return cudaGetLastError();
}

cudaError_t launch_round_queries(const double *q64, int64_t J, int q_stride, float4 *rows32, cudaStream_t s)
{
    launch_begin(K_F64, s);
    round_queries_kernel<<<stream_blocks(J), 256, 0, s>>>(q64, J, q_stride, rows32);
    launch_end(K_F64, s);
    return cudaGetLastError();
}

cudaError_t launch_gather_queries64(const double *q64, int64_t J, int q_stride, const int *perm, Double4 *rows64,
                                    cudaStream_t s)
{
    launch_begin(K_F64, s);
    gather_queries64_kernel<<<stream_blocks(J), 256, 0, s>>>(q64, J, q_stride, perm, rows64);
    launch_end(K_F64, s);
    return cudaGetLastError();
}

cudaError_t launch_forward64(const FusedArgs64 &a, bool with_dq, int grid, cudaStream_t s)
{
    launch_begin(K_F64, s);
    if (with_dq) fused_kernel<FORWARD, true, false, double><<<grid, kThreads, 0, s>>>(a, BatchArgs{});
    else fused_kernel<FORWARD, false, false, double><<<grid, kThreads, 0, s>>>(a, BatchArgs{});
    launch_end(K_F64, s);
    return cudaGetLastError();
}

cudaError_t launch_fused_backward64(const FusedArgs64 &a, bool with_gq, int grid, cudaStream_t s)
{
    launch_begin(K_F64, s);
    if (with_gq) fused_kernel<BACKWARD, true, false, double><<<grid, kThreads, 0, s>>>(a, BatchArgs{});
    else fused_kernel<BACKWARD, false, false, double><<<grid, kThreads, 0, s>>>(a, BatchArgs{});
    launch_end(K_F64, s);
    return cudaGetLastError();
}

}  // namespace efunc
