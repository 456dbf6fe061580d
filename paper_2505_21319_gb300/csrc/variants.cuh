// Ablation variants of the representation (Table tab:ablation): grid keys
// only (Config-G-*), offset keys only (Config-Full-1/2) or both under one
// softmax (Full-3/4); values are polynomials of degree 0..3 in Taylor form
// (Sec. 3.2 Eq. poly-func)
//   f(x) = o + d.x + 1/2 x^T S x + 1/6 T[x, x, x],  S, T symmetric,
// stored per key as phi = (o, d_xyz, S_xx, S_yy, S_zz, S_xy, S_xz, S_yz,
// T_xxx, T_yyy, T_zzz, T_xxy, T_xxz, T_xyy, T_yyz, T_xzz, T_yzz, T_xyz)
// truncated to 1 / 4 / 10 / 20 entries; scales are learnable log offsets or
// fixed at exp(log_beta0).  Channels per centre, in the tuple order of
// Eq. func-offset: [Delta if offset keys] [b per key set if learnable]
// [phi per key set], grid set first.
//
// The kernels follow the default model's fused kernel (same cell-sorted work
// items, persistent CTAs, key records staged per window in shared memory,
// forward thread-per-query, backward thread-per-key with one atomic per
// parameter per item) without its degree-1 specialisations.  The pack kernel
// folds the Taylor factors and the symmetric multiplicities into the
// coefficients, so the kernels evaluate f = sum_m c_m mono_m(x) over the
// monomials (1, x, y, z, xx, yy, zz, xy, xz, yz, xxx, yyy, zzz, xxy, xxz, xyy,
// yyz, xzz, yzz, xyz).
#pragma once

#include "common.cuh"

namespace efunc {
namespace variant {

constexpr unsigned kFull = 0xffffffffu;
constexpr float kLn2 = 0.69314718055994531f;

__host__ __device__ constexpr int nv_of(int deg) { return deg == 0 ? 1 : deg == 1 ? 4 : deg == 2 ? 10 : 20; }
__host__ __device__ constexpr int nrec_of(int deg) { return 1 + (nv_of(deg) + 3) / 4; }
__host__ __device__ constexpr int nsets_of(int sets) { return (sets & 1) + ((sets >> 1) & 1); }

// Taylor factor times symmetric multiplicity of coefficient m: 1/2 for the
// diagonal of S, 1 off it; 1/6 for T_aaa, 1/2 for T_aab, 1 for T_xyz.
__host__ __device__ constexpr float coef_factor(int m)
{
    return m < 4 ? 1.f : m < 7 ? 0.5f : m < 10 ? 1.f : m < 13 ? (1.f / 6.f) : m < 19 ? 0.5f : 1.f;
}

template <int DEG>
__device__ __forceinline__ void monomials(float x, float y, float z, float (&mo)[nv_of(DEG)])
{
    mo[0] = 1.f;
    if constexpr (DEG >= 1) {
        mo[1] = x; mo[2] = y; mo[3] = z;
    }
    if constexpr (DEG >= 2) {
        mo[4] = x * x; mo[5] = y * y; mo[6] = z * z;
        mo[7] = x * y; mo[8] = x * z; mo[9] = y * z;
    }
    if constexpr (DEG >= 3) {
        mo[10] = mo[4] * x; mo[11] = mo[5] * y; mo[12] = mo[6] * z;
        mo[13] = mo[4] * y; mo[14] = mo[4] * z; mo[15] = x * mo[5];
        mo[16] = mo[5] * z; mo[17] = x * mo[6]; mo[18] = y * mo[6];
        mo[19] = mo[7] * z;
    }
}

// Value coefficients of one key, read from its staged records.
template <int DEG>
__device__ __forceinline__ void load_coefs(const float4 *r, float (&c)[nv_of(DEG)])
{
#pragma unroll
    for (int i = 0; i < (nv_of(DEG) + 3) / 4; ++i) {
        const float4 v = r[1 + i];
        if (4 * i + 0 < nv_of(DEG)) c[4 * i + 0] = v.x;
        if (4 * i + 1 < nv_of(DEG)) c[4 * i + 1] = v.y;
        if (4 * i + 2 < nv_of(DEG)) c[4 * i + 2] = v.z;
        if (4 * i + 3 < nv_of(DEG)) c[4 * i + 3] = v.w;
    }
}

template <int DEG>
__device__ __forceinline__ float poly(const float (&c)[nv_of(DEG)], const float (&mo)[nv_of(DEG)])
{
    float f = c[0];
#pragma unroll
    for (int m = 1; m < nv_of(DEG); ++m) f = fmaf(c[m], mo[m], f);
    return f;
}

// grad f(x) for DEG >= 2 (DEG <= 1: the constant (c1, c2, c3))
template <int DEG>
__device__ __forceinline__ void poly_grad(const float (&c)[nv_of(DEG)], const float (&mo)[nv_of(DEG)], float &gx,
                                          float &gy, float &gz)
{
    const float x = mo[1], y = mo[2], z = mo[3];
    gx = fmaf(2.f * c[4], x, fmaf(c[7], y, fmaf(c[8], z, c[1])));
    gy = fmaf(2.f * c[5], y, fmaf(c[7], x, fmaf(c[9], z, c[2])));
    gz = fmaf(2.f * c[6], z, fmaf(c[8], x, fmaf(c[9], y, c[3])));
    if constexpr (DEG >= 3) {
        // xxx yyy zzz xxy xxz xyy yyz xzz yzz xyz
        gx += 3.f * c[10] * mo[4] + 2.f * c[13] * mo[7] + 2.f * c[14] * mo[8] + c[15] * mo[5] + c[17] * mo[6] +
              c[19] * mo[9];
        gy += 3.f * c[11] * mo[5] + c[13] * mo[4] + 2.f * c[15] * mo[7] + 2.f * c[16] * mo[9] + c[18] * mo[6] +
              c[19] * mo[8];
        gz += 3.f * c[12] * mo[6] + c[14] * mo[4] + c[16] * mo[5] + 2.f * c[17] * mo[8] + 2.f * c[18] * mo[9] +
              c[19] * mo[7];
    }
}

// ------------------------------------------------------------------ pack

// Per centre and key set: record 0 = (Delta or 0, -beta log2 e) with the
// scale formed in FP64, records 1.. = c_m = factor_m phi_m, zero padded.
template <int SETS, int DEG>
__global__ void __launch_bounds__(256) pack_kernel(VariantArgs a)
{
    constexpr int NV = nv_of(DEG), NREC = nrec_of(DEG), NS = nsets_of(SETS);
    const int I = a.R * a.R * a.R;
    const double log2e = 1.4426950408889634;
    const int base = (SETS & 2) ? 3 : 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < I; i += gridDim.x * blockDim.x) {
        const float *th = a.params + (size_t)i * a.channels;
        float4 *k = a.keys + (size_t)i * NS * NREC;
#pragma unroll
        for (int si = 0; si < NS; ++si) {
            const bool offset = (SETS == 2) || si == 1;
            const double b = a.learn ? (double)__ldg(th + base + si) : 0.0;
            const float s = (float)(-exp(a.log_beta0 + b) * log2e);
            float4 *r = k + si * NREC;
            r[0] = offset ? make_float4(__ldg(th), __ldg(th + 1), __ldg(th + 2), s) : make_float4(0.f, 0.f, 0.f, s);
            const float *phi = th + base + a.learn * NS + si * NV;
            float c[4 * (NREC - 1)];
#pragma unroll
            for (int m = 0; m < 4 * (NREC - 1); ++m) c[m] = m < NV ? coef_factor(m) * __ldg(phi + m) : 0.f;
#pragma unroll
            for (int j = 0; j < NREC - 1; ++j) r[1 + j] = make_float4(c[4 * j], c[4 * j + 1], c[4 * j + 2], c[4 * j + 3]);
        }
    }
}

// ---------------------------------------------------------------- kernel

struct Win {
    int cx, cy, cz, lox, loy, loz, nx, ny, nz, nc;
};

__device__ __forceinline__ Win window_of(const Item item, int R)
{
    Win w;
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

constexpr int kClasses = 4;   // interleaved summation classes of the forward

// Combines per-class partial sums of a query held by KQ lanes in the fixed
// order ((c0 + c1) + (c2 + c3)); lane `part` holds classes part + KQ i.
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

// (e, m) of one query over the window's keys, exponents shifted by M2.  Key k
// goes to class k mod 4, summed in key order, the classes combined in a
// fixed tree: the result does not depend on how many lanes share the query.
template <int DEG, int KQ>
__device__ __forceinline__ void fwd_sums(const float4 *rec, int nk, int part, float x, float y, float z, float M2,
                                         float &e, float &m)
{
    constexpr int NREC = nrec_of(DEG);
    constexpr int CPL = kClasses / KQ;
    float ev[CPL], mv[CPL];
#pragma unroll
    for (int i = 0; i < CPL; ++i) ev[i] = mv[i] = 0.f;
#pragma unroll 1
    for (int base = 0; base < nk; base += kClasses) {
#pragma unroll
        for (int i = 0; i < CPL; ++i) {
            const int k = base + part + KQ * i;
            if (k < nk) {
                const float4 *r = rec + k * NREC;
                const float4 A = r[0];
                const float rx = x - A.x, ry = y - A.y, rz = z - A.z;
                const float d2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
                const float l = ex2_approx(fmaf(A.w, d2, -M2));
                float c[nv_of(DEG)], mo[nv_of(DEG)];
                load_coefs<DEG>(r, c);
                monomials<DEG>(rx, ry, rz, mo);
                ev[i] += l;
                mv[i] = fmaf(l, poly<DEG>(c, mo), mv[i]);
            }
        }
    }
    e = combine_classes<KQ>(ev);
    m = combine_classes<KQ>(mv);
}

// (e, m) over a full window (64 centres) of grid keys only: the keys sit on
// the lattice (i - c) h, so the per-axis differences and squares are formed
// once per query and axis and d2 = (x2 + y2) + z2.  Key k = 16 ox + 4 oy + oz
// is in class oz, summed in the same key order as fwd_sums.
template <int DEG, int KQ>
__device__ __forceinline__ void fwd_sums_lattice(const float4 *rec, int part, float h, float x, float y, float z,
                                                 float &e, float &m)
{
    constexpr int NREC = nrec_of(DEG);
    constexpr int CPL = kClasses / KQ;
    float ev[CPL], mv[CPL], ry[4], y2[4], rz[CPL], z2[CPL];
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        ry[b] = y - (float)(b - 1) * h;
        y2[b] = ry[b] * ry[b];
    }
#pragma unroll
    for (int i = 0; i < CPL; ++i) {
        rz[i] = z - (float)(part + KQ * i - 1) * h;
        z2[i] = rz[i] * rz[i];
        ev[i] = mv[i] = 0.f;
    }
#pragma unroll 1
    for (int ox = 0; ox < 4; ++ox) {
        const float rx = x - (float)(ox - 1) * h;
        const float x2 = rx * rx;
#pragma unroll
        for (int oy = 0; oy < 4; ++oy) {
            const float xy = x2 + y2[oy];
#pragma unroll
            for (int i = 0; i < CPL; ++i) {
                const float4 *r = rec + (16 * ox + 4 * oy + part + KQ * i) * NREC;
                const float l = ex2_approx(r[0].w * (xy + z2[i]));
                float c[nv_of(DEG)], mo[nv_of(DEG)];
                load_coefs<DEG>(r, c);
                monomials<DEG>(rx, ry[oy], rz[i], mo);
                ev[i] += l;
                mv[i] = fmaf(l, poly<DEG>(c, mo), mv[i]);
            }
        }
    }
    e = combine_classes<KQ>(ev);
    m = combine_classes<KQ>(mv);
}

// Forward of the item's queries with KQ lanes per query; stores, for the
// backward, (local q, lse2) and (O, dL/dO) per query.
template <int MODE, int DEG, int KQ, bool LATTICE>
__device__ __forceinline__ void forward_phase(const VariantArgs &a, const float4 *rec, float4 *qt, float2 *og,
                                              int start, int n, int nk, float3 orig, float h, float &loss_acc,
                                              float &abs_acc)
{
    constexpr int NREC = nrec_of(DEG);
    constexpr int LG = KQ == 1 ? 0 : (KQ == 2 ? 1 : 2);
    const int t = threadIdx.x;
    const int part = t & (KQ - 1);
    for (int base = 0; base < n; base += kThreads / KQ) {
        const int qi = base + (t >> LG);
        const bool valid = qi < n;
        // lanes without a query evaluate the window origin (never stored)
        const float4 q4 = valid ? qt[qi] : make_float4(orig.x, orig.y, orig.z, 0.f);
        const float x = q4.x - orig.x, y = q4.y - orig.y, z = q4.z - orig.z;
        float e, m, M2 = 0.f;
        if (LATTICE) fwd_sums_lattice<DEG, KQ>(rec, part, h, x, y, z, e, m);
        else fwd_sums<DEG, KQ>(rec, nk, part, x, y, z, 0.f, e, m);
        const bool tiny = !(e >= 0x1p-60f);   // the same in every lane of the group
        if (__any_sync(kFull, tiny)) {        // every key far in units of its scale: shift by the largest exponent
            float mx = -INFINITY;
            for (int k = part; k < nk; k += KQ) {
                const float4 A = rec[k * NREC];
                const float rx = x - A.x, ry = y - A.y, rz = z - A.z;
                mx = fmaxf(mx, A.w * fmaf(rx, rx, fmaf(ry, ry, rz * rz)));
            }
#pragma unroll
            for (int o = 1; o < KQ; o <<= 1) mx = fmaxf(mx, __shfl_xor_sync(kFull, mx, o));
            float e2, m2;
            fwd_sums<DEG, KQ>(rec, nk, part, x, y, z, mx, e2, m2);
            if (tiny) {
                e = e2;
                m = m2;
                M2 = mx;
            }
        }
        const float O = m / e, lse2 = M2 + lg2_approx(e);
        float gO = 0.f;
        if (MODE == VAR_FIT) {
            const float diff = O - q4.w;
            if (a.loss == EFUNC_LOSS_L1) gO = diff > 0.f ? a.inv_J : (diff < 0.f ? -a.inv_J : 0.f);
            else gO = 2.f * diff * a.inv_J;
            if (valid && part == 0) {
                loss_acc += a.loss == EFUNC_LOSS_L1 ? fabsf(diff) : diff * diff;
                abs_acc += fabsf(diff);
            }
        } else if (valid && part == 0) {
            const int j = __ldg(a.perm + start + qi);
            if (MODE == VAR_FORWARD) {
                a.O[j] = O;
                if (a.lse) a.lse[j] = lse2 * kLn2;
            } else {
                gO = __ldg(a.gO + j);
            }
        }
        if (MODE != VAR_FORWARD) {
            __syncwarp();   // every lane of the group has read its row of qt
            if (valid && part == 0) {
                const float4 row = make_float4(x, y, z, lse2);
                qt[qi] = row;
                og[qi] = make_float2(O, gO);
                if (qi == n - 1 && (n & 1)) {   // pad the last pair: the same query without gradient
                    qt[n] = row;
                    og[n] = make_float2(O, 0.f);
                }
            }
        }
    }
}

template <int MODE, int SETS, int DEG>
__global__ void __launch_bounds__(kThreads, DEG <= 1 ? 7 : (DEG == 2 ? 5 : 4)) variant_kernel(VariantArgs a)
{
    constexpr int NV = nv_of(DEG), NREC = nrec_of(DEG), NS = nsets_of(SETS);
    __shared__ float4 s_rec[kCentres * NS * NREC];   // window key records, key-major
    __shared__ float4 s_qt[kChunk];                   // queries: (x, y, z, target), then (local q, lse2)
    __shared__ float4 s_og[kChunk / 2];               // (O, dL/dO) of query pairs 2i, 2i + 1
    __shared__ int s_item;
    __shared__ float s_red[2][kThreads / 32];

    const int t = threadIdx.x;
    const int R = a.R;
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
        const Win w = window_of(item, R);
        const int start = item.x, n = item.y, nc = w.nc, nk = nc * NS;
        const float3 orig = make_float3((float)(2 * w.cx + 1 - R) * invR, (float)(2 * w.cy + 1 - R) * invR,
                                        (float)(2 * w.cz + 1 - R) * invR);
        // ---- 1. stage key records (window-local positions) and queries
        if (t < nc) {
            const int oz = t % w.nz, oy = (t / w.nz) % w.ny, ox = t / (w.ny * w.nz);
            const float4 *k =
                a.keys + (((size_t)(w.lox + ox) * R + (w.loy + oy)) * R + (w.loz + oz)) * (size_t)(NS * NREC);
            const float gx = (float)(2 * (w.lox + ox - w.cx)) * invR, gy = (float)(2 * (w.loy + oy - w.cy)) * invR,
                        gz = (float)(2 * (w.loz + oz - w.cz)) * invR;
#pragma unroll
            for (int si = 0; si < NS; ++si) {
                float4 *r = s_rec + (t * NS + si) * NREC;
                const float4 A = k[si * NREC];
                r[0] = make_float4(gx + A.x, gy + A.y, gz + A.z, A.w);
#pragma unroll
                for (int j = 1; j < NREC; ++j) r[j] = k[si * NREC + j];
            }
        }
        for (int qi = t; qi < n; qi += kThreads) s_qt[qi] = a.sorted[start + qi];
        __syncthreads();

        // ---- 2. forward, 1, 2 or 4 lanes per query (sparse items use more)
        //         (grid keys of a full window, degree <= 1: lattice distances;
        //         for higher degrees the per-axis arrays cost more registers
        //         than the distances save)
        const float h = 2.f * invR;
        float2 *og2 = reinterpret_cast<float2 *>(s_og);
        if (SETS == 1 && DEG <= 1 && nc == kCentres) {
            if (n > 64) forward_phase<MODE, DEG, 1, true>(a, s_rec, s_qt, og2, start, n, nk, orig, h, loss_acc, abs_acc);
            else if (n > 32) forward_phase<MODE, DEG, 2, true>(a, s_rec, s_qt, og2, start, n, nk, orig, h, loss_acc, abs_acc);
            else forward_phase<MODE, DEG, 4, true>(a, s_rec, s_qt, og2, start, n, nk, orig, h, loss_acc, abs_acc);
        } else {
            if (n > 64) forward_phase<MODE, DEG, 1, false>(a, s_rec, s_qt, og2, start, n, nk, orig, h, loss_acc, abs_acc);
            else if (n > 32) forward_phase<MODE, DEG, 2, false>(a, s_rec, s_qt, og2, start, n, nk, orig, h, loss_acc, abs_acc);
            else forward_phase<MODE, DEG, 4, false>(a, s_rec, s_qt, og2, start, n, nk, orig, h, loss_acc, abs_acc);
        }
        if (MODE == VAR_FORWARD) continue;

        // ---- 3. backward, one thread per key (two threads per key, each
        //         over every second pair of queries, when there is one key
        //         set); a pair's two query rows and its (O, dL/dO) float4 are
        //         loaded together
        __syncthreads();
        const int kk = NS == 2 ? t : (t & (kCentres - 1));
        const int half = NS == 2 ? 0 : (t >> 6);
        const int qstep = NS == 2 ? 1 : 2;
        const int cidx = kk % kCentres;   // NS == 2: keys t and t + 64 share centre t & 63
        const int si = NS == 2 ? kk / kCentres : 0;
        if (cidx < nc) {
            const int key = cidx * NS + si;
            const float4 *r = s_rec + key * NREC;
            const float4 A = r[0];
            float c[NV];
            load_coefs<DEG>(r, c);
            const bool offset = (SETS == 2) || si == 1;
            float acc[NV];
#pragma unroll
            for (int i = 0; i < NV; ++i) acc[i] = 0.f;
            float ab = 0.f, adx = 0.f, ady = 0.f, adz = 0.f, agx = 0.f, agy = 0.f, agz = 0.f;
            // one query: Q = (local q, lse2), O and dL/dO
            auto one = [&](const float4 Q, float O, float gO) {
                const float rx = Q.x - A.x, ry = Q.y - A.y, rz = Q.z - A.z;
                const float d2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
                const float g = ex2_approx(fmaf(A.w, d2, -Q.w)) * gO;
                float mo[NV];
                monomials<DEG>(rx, ry, rz, mo);
#pragma unroll
                for (int i = 0; i < NV; ++i) acc[i] = fmaf(g, mo[i], acc[i]);
                if (a.learn || offset) {
                    const float gd = g * (poly<DEG>(c, mo) - O);
                    ab = fmaf(gd, d2, ab);
                    if (offset) {
                        adx = fmaf(gd, rx, adx);
                        ady = fmaf(gd, ry, ady);
                        adz = fmaf(gd, rz, adz);
                        if constexpr (DEG >= 2) {
                            float gx, gy, gz;
                            poly_grad<DEG>(c, mo, gx, gy, gz);
                            agx = fmaf(g, gx, agx);
                            agy = fmaf(g, gy, agy);
                            agz = fmaf(g, gz, agz);
                        }
                    }
                }
            };
            const int pairs = (n + 1) >> 1;
#pragma unroll 1
            for (int jp = half; jp < pairs; jp += qstep) {
                const float4 Q0 = s_qt[2 * jp], Q1 = s_qt[2 * jp + 1], G = s_og[jp];
                one(Q0, G.x, G.y);
                one(Q1, G.z, G.w);
            }
            const int oz = cidx % w.nz, oy = (cidx / w.nz) % w.ny, ox = cidx / (w.ny * w.nz);
            float *gr = a.grad + (((size_t)(w.lox + ox) * R + (w.loy + oy)) * R + (w.loz + oz)) * a.channels;
            const int base = (SETS & 2) ? 3 : 0;
            float *gphi = gr + base + a.learn * NS + si * NV;
#pragma unroll
            for (int i = 0; i < NV; ++i) atomicAdd(gphi + i, coef_factor(i) * acc[i]);
            const float beta = -A.w * kLn2;
            if (a.learn) atomicAdd(gr + base + si, -beta * ab);
            if (offset) {
                // dO/dDelta = w (2 beta (q - key)(f - O) - grad f)
                if constexpr (DEG <= 1) {
                    if constexpr (DEG == 1) {
                        agx = c[1] * acc[0];
                        agy = c[2] * acc[0];
                        agz = c[3] * acc[0];
                    }
                }
                atomicAdd(gr + 0, fmaf(2.f * beta, adx, -agx));
                atomicAdd(gr + 1, fmaf(2.f * beta, ady, -agy));
                atomicAdd(gr + 2, fmaf(2.f * beta, adz, -agz));
            }
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

int sm_count();

template <int MODE, int SETS, int DEG>
int persistent_grid(bool leave_room)
{
    const void *k = reinterpret_cast<const void *>(variant_kernel<MODE, SETS, DEG>);
    return per_device_cached(k, leave_room ? 2 : 1, [k, leave_room] {
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kThreads, 0);
        if (per_sm <= 0) per_sm = 1;
        if (leave_room) per_sm = leave_sort_room(k, per_sm);
        return sm_count() * per_sm;
    });
}

template <int SETS, int DEG>
cudaError_t launch_sets_deg(const VariantArgs &a, int mode, cudaStream_t s)
{
    if (mode == VAR_FORWARD) {
        launch_begin(K_VAR_FORWARD, s);
        variant_kernel<VAR_FORWARD, SETS, DEG><<<persistent_grid<VAR_FORWARD, SETS, DEG>(a.leave_room), kThreads, 0, s>>>(a);
        launch_end(K_VAR_FORWARD, s);
    } else if (mode == VAR_BACKWARD) {
        launch_begin(K_VAR_BACKWARD, s);
        variant_kernel<VAR_BACKWARD, SETS, DEG><<<persistent_grid<VAR_BACKWARD, SETS, DEG>(a.leave_room), kThreads, 0, s>>>(a);
        launch_end(K_VAR_BACKWARD, s);
    } else {
        launch_begin(K_VAR_FIT, s);
        variant_kernel<VAR_FIT, SETS, DEG><<<persistent_grid<VAR_FIT, SETS, DEG>(a.leave_room), kThreads, 0, s>>>(a);
        launch_end(K_VAR_FIT, s);
    }
    return cudaGetLastError();
}

template <int SETS, int DEG>
cudaError_t launch_pack_sets_deg(const VariantArgs &a, cudaStream_t s)
{
    const int I = a.R * a.R * a.R;
    int blocks = (I + 255) / 256;
    if (blocks > sm_count() * 8) blocks = sm_count() * 8;
    launch_begin(K_VAR_PACK, s);
    pack_kernel<SETS, DEG><<<blocks, 256, 0, s>>>(a);
    launch_end(K_VAR_PACK, s);
    return cudaGetLastError();
}

// one translation unit per degree (variants_d<DEG>.cu) defines these
cudaError_t launch_deg0(const VariantArgs &a, int mode, cudaStream_t s);
cudaError_t launch_deg1(const VariantArgs &a, int mode, cudaStream_t s);
cudaError_t launch_deg2(const VariantArgs &a, int mode, cudaStream_t s);
cudaError_t launch_deg3(const VariantArgs &a, int mode, cudaStream_t s);
cudaError_t launch_pack_deg0(const VariantArgs &a, cudaStream_t s);
cudaError_t launch_pack_deg1(const VariantArgs &a, cudaStream_t s);
cudaError_t launch_pack_deg2(const VariantArgs &a, cudaStream_t s);
cudaError_t launch_pack_deg3(const VariantArgs &a, cudaStream_t s);

#define EFUNC_VARIANT_DEGREE(DEG)                                                     \
    cudaError_t launch_deg##DEG(const VariantArgs &a, int mode, cudaStream_t s)       \
    {                                                                                 \
        if (a.sets == 1) return launch_sets_deg<1, DEG>(a, mode, s);                  \
        if (a.sets == 2) return launch_sets_deg<2, DEG>(a, mode, s);                  \
        return launch_sets_deg<3, DEG>(a, mode, s);                                   \
    }                                                                                 \
    cudaError_t launch_pack_deg##DEG(const VariantArgs &a, cudaStream_t s)            \
    {                                                                                 \
        if (a.sets == 1) return launch_pack_sets_deg<1, DEG>(a, s);                   \
        if (a.sets == 2) return launch_pack_sets_deg<2, DEG>(a, s);                   \
        return launch_pack_sets_deg<3, DEG>(a, s);                                    \
    }

}  // namespace variant
}  // namespace efunc
