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

// Shared key tile of one window: centre c holds 4 float4 records,
//   rec[4c + 0] = (grid key position, -beta log2 e)    rec[4c + 1] = (o, d)
//   rec[4c + 2] = (offset key position, -beta' log2 e) rec[4c + 3] = (o', d')
// with positions in window-local coordinates; set 0 = grid keys, 1 = offset keys.
__device__ __forceinline__ float4 keyA(const float4 *rec, int set, int k) { return rec[4 * k + 2 * set]; }
__device__ __forceinline__ float4 keyB(const float4 *rec, int set, int k) { return rec[4 * k + 2 * set + 1]; }

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
__device__ __forceinline__ void fwd_sums(const float4 *rec, int nc, int part, float x, float y, float z, float M2,
                                         float &e, float &m)
{
    constexpr int CPL = kClasses / KQ;
    float ev[CPL], mv[CPL];
#pragma unroll
    for (int i = 0; i < CPL; ++i) ev[i] = mv[i] = 0.f;
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
template <int KQ>
__device__ __forceinline__ void fwd_sums_full(const float4 *rec, int part, float h, float x, float y, float z,
                                              float &e, float &m)
{
    constexpr int CPL = kClasses / KQ;
    float ev[CPL], mv[CPL];
    float ry[4], y2[4], rz[CPL], z2[CPL];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        ry[a] = y - (float)(a - 1) * h;
        y2[a] = ry[a] * ry[a];
    }
#pragma unroll
    for (int i = 0; i < CPL; ++i) {
        rz[i] = z - (float)(part + KQ * i - 1) * h;
        z2[i] = rz[i] * rz[i];
        ev[i] = mv[i] = 0.f;
    }
    const float4 *P = rec + 4 * part;
#pragma unroll 1
    for (int ox = 0; ox < 4; ++ox) {
        const float rx = x - (float)(ox - 1) * h;
        const float x2 = rx * rx;
        const float4 *Po = P + 4 * 16 * ox;
#pragma unroll
        for (int oy = 0; oy < 4; ++oy) {
            const float xy = x2 + y2[oy];
#pragma unroll
            for (int i = 0; i < CPL; ++i) {
                const int k = oy * 4 + KQ * i;
                const float nbl = Po[4 * k].w;
                const float4 b = Po[4 * k + 1];
                const float l = ex2_approx(nbl * (xy + z2[i]));
                const float f = fmaf(b.y, rx, fmaf(b.z, ry[oy], fmaf(b.w, rz[i], b.x)));
                ev[i] += l;
                mv[i] = fmaf(l, f, mv[i]);
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
                fwd_key(P[4 * k + 2], P[4 * k + 3], x, y, z, 0.f, ev[i], mv[i]);
            }
        }
    }
    e = combine_classes<KQ>(ev);
    m = combine_classes<KQ>(mv);
}

// Eq. func-normal: dO/dq = sum w (d + 2 beta (q - key)(O - f)), same classes.
template <int KQ>
__device__ __forceinline__ void dq_sums(const float4 *rec, int nc, int part, float x, float y, float z, float lse2,
                                        float O, float &gx, float &gy, float &gz)
{
    constexpr int CPL = kClasses / KQ;
    float ax[CPL], ay[CPL], az[CPL];
#pragma unroll
    for (int i = 0; i < CPL; ++i) ax[i] = ay[i] = az[i] = 0.f;
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
                    const float wb = w * (-kLn2) * a.w;               // w beta
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

struct FwdOut {
    float O, lse2;
};

// Forward of the query held by this lane group: fast path without shift,
// shifted recomputation for groups whose sum underflowed.
template <int KQ, bool FULL>
__device__ __forceinline__ FwdOut forward_query(const float4 *rec, int nc, int part, float h, float4 q)
{
    float e, m;
    if (FULL) fwd_sums_full<KQ>(rec, part, h, q.x, q.y, q.z, e, m);
    else fwd_sums<KQ>(rec, nc, part, q.x, q.y, q.z, 0.f, e, m);
    float M2 = 0.f;
    const bool tiny = !(e >= 0x1p-60f);   // identical in every lane of the group
    if (__any_sync(kFull, tiny)) {
        float mx = -INFINITY;
        for (int k = part; k < nc; k += KQ) {
            mx = fmaxf(mx, key_exponent(keyA(rec, 0, k), q.x, q.y, q.z));
            mx = fmaxf(mx, key_exponent(keyA(rec, 1, k), q.x, q.y, q.z));
        }
#pragma unroll
        for (int o = 1; o < KQ; o <<= 1) mx = fmaxf(mx, __shfl_xor_sync(kFull, mx, o));
        // the shifted sums take the generic path in every window shape
        float e2, m2;
        fwd_sums<KQ>(rec, nc, part, q.x, q.y, q.z, mx, e2, m2);
        if (tiny) {
            e = e2;
            m = m2;
            M2 = mx;
        }
    }
    return {m / e, M2 + lg2_approx(e)};
}

// ----------------------------------------------------------- backward

// Thread-per-key loop over the item's queries, two queries per iteration:
// sqA[j] = (q_j local, lse2_j), sqB[j/2] = (O_j, gO_j, O_j+1, gO_j+1); an odd
// count is padded with a copy of the last query carrying dL/dO = 0.
template <bool OFFSET>
__device__ __forceinline__ void bwd_key_loop(const float4 A, const float4 B, const float4 *__restrict__ sqA,
                                             const float4 *__restrict__ sqB, int n, float acc[8])
{
    float ag = 0.f, arx = 0.f, ary = 0.f, arz = 0.f, ab = 0.f, adx = 0.f, ady = 0.f, adz = 0.f;
    auto one = [&](const float4 Q, float O, float gO) {
        const float rx = Q.x - A.x, ry = Q.y - A.y, rz = Q.z - A.z;
        const float d2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
        const float w = ex2_approx(fmaf(A.w, d2, -Q.w));
        const float g = w * gO;
        const float f = fmaf(B.y, rx, fmaf(B.z, ry, fmaf(B.w, rz, B.x)));
        const float gd = g * (f - O);
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
    };
    const int pairs = (n + 1) >> 1;
#pragma unroll 2
    for (int jp = 0; jp < pairs; ++jp) {
        const float4 Q0 = sqA[2 * jp], Q1 = sqA[2 * jp + 1], S = sqB[jp];
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
    const float beta = -A.w * kLn2;
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

// ------------------------------------------------------------- kernel

// Forward over the item's queries.  qt holds the raw query tile (x, y, z,
// target); a query's row is rewritten in place with (local position, lse2)
// by the lane that owns it, after every lane of its group has read it.
template <int MODE, bool DQ, bool GEIK, int KQ, bool FULL>
__device__ __forceinline__ void forward_phase(const FusedArgs &a, const float4 *rec, float4 *qt, float4 *sqB,
                                              float4 *sqE, float4 *sqU, int start, int n, int nc, float3 orig,
                                              float h, float &loss_acc, float &abs_acc)
{
    constexpr int LG = KQ == 1 ? 0 : (KQ == 2 ? 1 : 2);
    const int t = threadIdx.x;
    const int part = t & (KQ - 1);
    constexpr int per_round = kThreads / KQ;
    for (int base = 0; base < n; base += per_round) {
        const int qi = base + (t >> LG);
        const bool valid = qi < n;
        int j_user = 0;
        if (MODE != FIT) j_user = valid ? __ldg(a.perm + start + qi) : 0;   // issued before the long compute
        float4 q;
        if (valid) {
            q = qt[qi];
            q.x -= orig.x;   // window-local coordinates
            q.y -= orig.y;
            q.z -= orig.z;
        } else {
            // lanes without a query evaluate the window centre (never stored)
            q = make_float4(0.5f * h, 0.5f * h, 0.5f * h, 0.f);
        }
        const FwdOut r = forward_query<KQ, FULL>(rec, nc, part, h, q);
        const float O = r.O, lse2 = r.lse2;

        float gO = 0.f;
        if (MODE == FIT) {
            const float diff = O - q.w;
            if (a.loss == EFUNC_LOSS_L1) gO = diff > 0.f ? a.inv_J : (diff < 0.f ? -a.inv_J : 0.f);
            else gO = 2.f * diff * a.inv_J;
            if (valid && part == 0) {
                loss_acc += a.loss == EFUNC_LOSS_L1 ? fabsf(diff) : diff * diff;
                abs_acc += fabsf(diff);
            }
        } else if (MODE == BACKWARD) {
            gO = (valid && a.gO) ? __ldg(a.gO + j_user) : 0.f;
        } else if (valid && part == 0) {
            a.O[j_user] = O;
            if (a.lse) a.lse[j_user] = lse2 * kLn2;
        }
        if (DQ) {
            float gx, gy, gz;
            dq_sums<KQ>(rec, nc, part, q.x, q.y, q.z, lse2, O, gx, gy, gz);
            if (valid && part == 0) {
                float *dst = MODE == FORWARD ? a.dq : a.gq;
                const float s = MODE == FORWARD ? 1.f : gO;
                dst[3 * (size_t)j_user + 0] = s * gx;
                dst[3 * (size_t)j_user + 1] = s * gy;
                dst[3 * (size_t)j_user + 2] = s * gz;
            }
        }
        float4 rowE = make_float4(O, gO, 0.f, 0.f), rowU = make_float4(0.f, 0.f, 0.f, 0.f);
        if (GEIK) {
            // second order: u = dL/d(dO/dq), H = u . dO/dq, T = -2 u . sum w beta (q - key)
            float G[3], V[3];
            gv_sums<KQ>(rec, nc, part, q.x, q.y, q.z, lse2, O, G, V);
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
            const float T = -2.f * fmaf(u0, V[0], fmaf(u1, V[1], u2 * V[2]));
            rowE = make_float4(O, gO, H, T);
            rowU = make_float4(u0, u1, u2, 0.f);
        }
        if (GEIK && valid && part == 0) {
            sqE[qi] = rowE;
            sqU[qi] = rowU;
        }
        if (MODE != FORWARD) {
            __syncwarp();   // every lane of the group has read its row of qt
            if (valid && part == 0) {
                const float4 qa = make_float4(q.x, q.y, q.z, lse2);
                float2 *sqB2 = reinterpret_cast<float2 *>(sqB);
                qt[qi] = qa;
                sqB2[qi] = make_float2(O, gO);
                if (qi == n - 1 && (n & 1)) {   // pad the last pair: same query, no gradient
                    qt[n] = qa;
                    sqB2[n] = make_float2(O, 0.f);
                }
            }
        }
    }
}

template <int MODE, bool DQ, bool GEIK>
__global__ void __launch_bounds__(kThreads, GEIK ? 5 : 9) fused_kernel(FusedArgs a)
{
    __shared__ float4 s_rec[kCentres * kKeyRecords];          // key records of the window
    __shared__ float4 s_qt[kChunk];                           // query tile
    __shared__ float4 s_sqB[MODE == FORWARD ? 1 : kChunk / 2];
    __shared__ float4 s_sqE[GEIK ? kChunk : 1];               // (O, gO, H, T) per query
    __shared__ float4 s_sqU[GEIK ? kChunk : 1];               // (u, 0) per query
    __shared__ int s_item;
    __shared__ float s_red[2][kThreads / 32];

    const int t = threadIdx.x;
    const int R = a.R;
    const float invR = 1.f / (float)R;    // exact for power-of-two R
    const float h = 2.f * invR;
    const int n_items = a.ctrl->n_items;
    float loss_acc = 0.f, abs_acc = 0.f;

    for (;;) {
        __syncthreads();   // the previous item is consumed
        if (t == 0) s_item = atomicAdd(&a.ctrl->next_item, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= n_items) break;
        const Item item = a.items[it];
        const Window w = window_of(item, R);
        const int start = item.x, n = item.y, nc = w.nc;
        const bool full = nc == kCentres;
        float4 *rec = s_rec, *qt = s_qt, *qB = s_sqB;
        const float3 orig = make_float3((float)(2 * w.cx + 1 - R) * invR, (float)(2 * w.cy + 1 - R) * invR,
                                        (float)(2 * w.cz + 1 - R) * invR);
        // ---- 1. stage the key records (positions made window-local) and queries
        if (t < nc) {
            int ox, oy, oz;
            if (full) { ox = t >> 4; oy = (t >> 2) & 3; oz = t & 3; }
            else { oz = t % w.nz; oy = (t / w.nz) % w.ny; ox = t / (w.ny * w.nz); }
            const float4 *k = a.keys + (((size_t)(w.lox + ox) * R + (w.loy + oy)) * R + (w.loz + oz)) * kKeyRecords;
            const float gx = (float)(2 * (w.lox + ox - w.cx)) * invR, gy = (float)(2 * (w.loy + oy - w.cy)) * invR,
                        gz = (float)(2 * (w.loz + oz - w.cz)) * invR;
            const float4 g = k[0], o = k[2];
            float4 *r = rec + 4 * t;
            r[0] = make_float4(gx, gy, gz, g.w);
            r[1] = k[1];
            r[2] = make_float4(gx + o.x, gy + o.y, gz + o.z, o.w);
            r[3] = k[3];
        }
        for (int qi = t; qi < n; qi += kThreads) qt[qi] = a.sorted[start + qi];
        __syncthreads();

        // ---- 2. forward, one (or 2 / 4) threads per query
        if (full) {
            if (n > 64) forward_phase<MODE, DQ, GEIK, 1, true>(a, rec, qt, qB, s_sqE, s_sqU, start, n, nc, orig, h, loss_acc, abs_acc);
            else if (n > 32) forward_phase<MODE, DQ, GEIK, 2, true>(a, rec, qt, qB, s_sqE, s_sqU, start, n, nc, orig, h, loss_acc, abs_acc);
            else forward_phase<MODE, DQ, GEIK, 4, true>(a, rec, qt, qB, s_sqE, s_sqU, start, n, nc, orig, h, loss_acc, abs_acc);
        } else {
            if (n > 64) forward_phase<MODE, DQ, GEIK, 1, false>(a, rec, qt, qB, s_sqE, s_sqU, start, n, nc, orig, h, loss_acc, abs_acc);
            else if (n > 32) forward_phase<MODE, DQ, GEIK, 2, false>(a, rec, qt, qB, s_sqE, s_sqU, start, n, nc, orig, h, loss_acc, abs_acc);
            else forward_phase<MODE, DQ, GEIK, 4, false>(a, rec, qt, qB, s_sqE, s_sqU, start, n, nc, orig, h, loss_acc, abs_acc);
        }
        if (MODE != FORWARD) {
            // ---- 3. backward, one thread per key
            __syncthreads();
            const int c = t & (kCentres - 1);
            if (c < nc) {
                const bool offset = t >= kCentres;
                const float4 A = keyA(rec, offset, c), B = keyB(rec, offset, c);
                float acc[19];
                if (GEIK) {
                    if (offset) bwd2_key_loop<true>(A, B, qt, s_sqE, s_sqU, n, acc);
                    else bwd2_key_loop<false>(A, B, qt, s_sqE, s_sqU, n, acc);
                } else {
                    if (offset) bwd_key_loop<true>(A, B, qt, qB, n, acc);
                    else bwd_key_loop<false>(A, B, qt, qB, n, acc);
                    for (int i = 8; i < 19; ++i) acc[i] = 0.f;
                }
                int ox, oy, oz;
                    if (full) { ox = c >> 4; oy = (c >> 2) & 3; oz = c & 3; }
                else { oz = c % w.nz; oy = (c / w.nz) % w.ny; ox = c / (w.ny * w.nz); }
                float *gr = a.grad + (((size_t)(w.lox + ox) * R + (w.loy + oy)) * R + (w.loz + oz)) * kSlots;
                const float beta = -A.w * kLn2;
                // value term (dO/dtheta) plus, in second-order mode, the
                // gradient term d(u . dO/dq)/dtheta
                const float go = acc[0] + acc[8];
                const float gdx = acc[1] + acc[9], gdy = acc[2] + acc[10], gdz = acc[3] + acc[11];
                const float gb = beta * (-acc[4] + acc[12]);
                if (!offset) {
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
                    const float tb = 2.f * beta;
                    atomicAdd(gr + 0, fmaf(-B.y, go, tb * (acc[5] + acc[13] + acc[16])));
                    atomicAdd(gr + 1, fmaf(-B.z, go, tb * (acc[6] + acc[14] + acc[17])));
                    atomicAdd(gr + 2, fmaf(-B.w, go, tb * (acc[7] + acc[15] + acc[18])));
                }
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
    pack_keys_kernel<<<blocks, 256, 0, s>>>(a);
    launch_end(K_PACK_KEYS, s);
    return cudaGetLastError();
}

cudaError_t launch_forward(const FusedArgs &a, bool with_dq, int grid, cudaStream_t s)
{
    launch_begin(K_FORWARD, s);
    if (with_dq) fused_kernel<FORWARD, true, false><<<grid, kThreads, 0, s>>>(a);
    else fused_kernel<FORWARD, false, false><<<grid, kThreads, 0, s>>>(a);
    launch_end(K_FORWARD, s);
    return cudaGetLastError();
}

cudaError_t launch_fused_backward(const FusedArgs &a, bool with_gq, bool second_order, int grid, cudaStream_t s)
{
    launch_begin(K_FUSED_BWD, s);
    if (second_order) fused_kernel<BACKWARD, false, true><<<grid, kThreads, 0, s>>>(a);
    else if (with_gq) fused_kernel<BACKWARD, true, false><<<grid, kThreads, 0, s>>>(a);
    else fused_kernel<BACKWARD, false, false><<<grid, kThreads, 0, s>>>(a);
    launch_end(K_FUSED_BWD, s);
    return cudaGetLastError();
}

cudaError_t launch_fused_fit(const FusedArgs &a, bool eikonal, int grid, cudaStream_t s)
{
    launch_begin(K_FUSED_FIT, s);
    if (eikonal) fused_kernel<FIT, false, true><<<grid, kThreads, 0, s>>>(a);
    else fused_kernel<FIT, false, false><<<grid, kThreads, 0, s>>>(a);
    launch_end(K_FUSED_FIT, s);
    return cudaGetLastError();
}

}  // namespace efunc
