/*
 * efunc_oracle.c -- plain, slow FP64 CPU oracle for the O^{+Delta} representation
 * of "efunc: An Efficient Function Representation without Neural Networks"
 * (arXiv 2505.21319).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this file.  It shares no code, header,
 * table or constant with the CUDA library; the two meet only through the seeded
 * input generators.
 *
 * What it computes (paper notation):
 *   Keys      (Sec. 3.3, Eq. func-offset): every grid centre k_i carries a fixed
 *             grid key k_i and a learnable offset key k_i + Delta_i; both key sets
 *             enter ONE softmax (the union in Eq. func-offset).
 *   Weights   (Sec. 3.1, Eq. nrbf): softmax over -beta ||q - key||^2.
 *   Values    (Sec. 3.2, Eq. func-interp, Eq. poly-func, first order f^1):
 *             f(q - key; phi) = o + dot(d, q - key), shift-invariant.
 *   Forward   (Sec. 3.5, Algorithm 1): e_j = sum_i l, m_j = sum_i l f, O = m/e.
 *   Backward  (Sec. 3.6, Algorithm 2 and the closed-form dO/dk, dO/dbeta,
 *             dO/dphi that follow it).
 *   dO/dq     (Sec. 3.2, Eq. func-normal), and the backward through it (the
 *             parameter gradient of a loss on dO/dq, e.g. the Eikonal term).
 *   Loss      (Sec. 3.4, Eq. loss: MSE) and the L1 variant.
 *   Offsets   (Sec. 3.3, mean-shift initialisation from surface points).
 *   Adam      (Sec. 3.4 / Sec. 4.2 name Adam / AdamW; torch.optim semantics).
 *
 * Readings of the paper that this file fixes (the paper is silent on them):
 *   - Domain [-1,1]^3, R centres per axis, spacing h = 2/R, centre of index
 *     (a,b,c) at k = -1 + ((a,b,c) + 0.5) h.  Parameters are stored as
 *     params[((a*R + b)*R + c)*13 + slot].
 *   - Slot order follows the parameter tuple of Eq. func-offset
 *     {k_i, Delta_i, beta_i, beta'_i, phi_i, phi'_i} with k_i implicit:
 *       0..2  Delta       3  b  (grid key log-scale)   4  b' (offset key log-scale)
 *       5     o  (grid value constant)     6..8   d  (grid value linear term)
 *       9     o' (offset value constant)   10..12 d' (offset value linear term)
 *   - Scales are stored as log offsets: beta = exp(log_beta0 + b).  Sec. 4.3
 *     initialises every scale to exp(7); log_beta0 carries that constant.
 *   - Support: the paper's sum is global (Algorithm 1 loops over all I keys).
 *     The hot path truncates it to a window of (2W)^3 centres around the query;
 *     W >= R gives the paper's global model exactly.  The window base index per
 *     axis is c = clamp(floor((q + 1) * (R/2) - 0.5), -1, R-1), evaluated in
 *     FP32 on the FP32 query with no fused multiply-add (this file must be built
 *     with -ffp-contract=off); the window holds the centres with index in
 *     [c - W + 1, c + W], dropping indices outside [0, R-1].
 *   - Softmax is evaluated with the maximum exponent subtracted (log-sum-exp);
 *     mathematically identical to Algorithm 1, which has no shift.
 *   - L1 loss uses sign(0) = 0.
 *
 * All arithmetic after the window choice is FP64.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <string.h>

#define NSLOT 13

/* ---------------------------------------------------------------- window */

/* Window base index along one axis (see header).  FP32 on purpose: the CUDA
 * path takes the same integer decision in the same precision. */
int ora_window_base(float q, int R)
{
    float scale = (float)R * 0.5f;
    float t = (q + 1.0f) * scale;
    float u = t - 0.5f;
    float lo = -1.0f, hi = (float)(R - 1);
    if (!(u >= lo)) u = lo; /* also maps NaN to the first window */
    if (u > hi) u = hi;
    return (int)floorf(u);
}

static void window_range(const double *q, int R, int W, int lo[3], int hi[3])
{
    for (int a = 0; a < 3; ++a) {
        int c = ora_window_base((float)q[a], R);
        int l = c - W + 1, h = c + W;
        lo[a] = l < 0 ? 0 : l;
        hi[a] = h > R - 1 ? R - 1 : h;
    }
}

/* ------------------------------------------------------------- the keys */

/* One key of the union in Eq. func-offset: position, scale beta and the
 * first-order value f(x) = o + dot(d, x) with x = q - position. */
typedef struct {
    double p[3];
    double beta;
    double o;
    double d[3];
} key_t_;

static double centre_coord(int idx, int R) { return -1.0 + ((double)idx + 0.5) * (2.0 / (double)R); }

/* which = 0: grid key k_i; which = 1: offset key k_i + Delta_i. */
static key_t_ make_key(const double *params, int R, double log_beta0, int a, int b, int c, int which)
{
    const double *th = params + ((size_t)((size_t)a * R + b) * R + c) * NSLOT;
    key_t_ k;
    k.p[0] = centre_coord(a, R);
    k.p[1] = centre_coord(b, R);
    k.p[2] = centre_coord(c, R);
    if (which == 0) {
        k.beta = exp(log_beta0 + th[3]);
        k.o = th[5];
        k.d[0] = th[6]; k.d[1] = th[7]; k.d[2] = th[8];
    } else {
        k.p[0] += th[0]; k.p[1] += th[1]; k.p[2] += th[2];
        k.beta = exp(log_beta0 + th[4]);
        k.o = th[9];
        k.d[0] = th[10]; k.d[1] = th[11]; k.d[2] = th[12];
    }
    return k;
}

/* exponent -beta ||q - p||^2 (Eq. nrbf) and value f(q - p) (Eq. poly-func, f^1) */
static void eval_key(const key_t_ *k, const double *q, double r[3], double *d2, double *expo, double *f)
{
    r[0] = q[0] - k->p[0];
    r[1] = q[1] - k->p[1];
    r[2] = q[2] - k->p[2];
    *d2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
    *expo = -k->beta * (*d2);
    *f = k->o + k->d[0] * r[0] + k->d[1] * r[1] + k->d[2] * r[2];
}

/* --------------------------------------------------------------- forward */

/* Algorithm 1 for one query over the windowed key set.  Returns O, the
 * log-normaliser lse = log(sum exp(expo)), if dq != NULL dO/dq from
 * Eq. func-normal, and if kappa != NULL the condition number of O with respect
 * to relative perturbations of the exponents and of the individual weights,
 *     kappa = sum_keys softmax * (|expo| + 1) * |f - O|
 * (dO/dexpo_i = softmax_i (f_i - O)): an evaluation that perturbs every
 * exponent and every weight by a relative error u is off by about u * kappa. */
static void forward_one(const double *params, int R, int W, double log_beta0, const double *q,
                        double *O_out, double *lse_out, double *dq, double *kappa, double *dq_sens)
{
    int lo[3], hi[3];
    window_range(q, R, W, lo, hi);
    double r[3], d2, expo, f;

    /* maximum exponent (the stabilising shift) */
    double M = -INFINITY;
    for (int a = lo[0]; a <= hi[0]; ++a)
        for (int b = lo[1]; b <= hi[1]; ++b)
            for (int c = lo[2]; c <= hi[2]; ++c)
                for (int s = 0; s < 2; ++s) {
                    key_t_ k = make_key(params, R, log_beta0, a, b, c, s);
                    eval_key(&k, q, r, &d2, &expo, &f);
                    if (expo > M) M = expo;
                }

    /* e_j = sum l, m_j = sum l f  (Algorithm 1, with l scaled by exp(-M)) */
    double e = 0.0, m = 0.0;
    for (int a = lo[0]; a <= hi[0]; ++a)
        for (int b = lo[1]; b <= hi[1]; ++b)
            for (int c = lo[2]; c <= hi[2]; ++c)
                for (int s = 0; s < 2; ++s) {
                    key_t_ k = make_key(params, R, log_beta0, a, b, c, s);
                    eval_key(&k, q, r, &d2, &expo, &f);
                    double l = exp(expo - M);
                    e += l;
                    m += l * f;
                }
    double O = m / e;
    *O_out = O;
    if (lse_out) *lse_out = M + log(e);

    if (kappa) {
        double k_sum = 0.0;
        for (int a = lo[0]; a <= hi[0]; ++a)
            for (int b = lo[1]; b <= hi[1]; ++b)
                for (int c = lo[2]; c <= hi[2]; ++c)
                    for (int s = 0; s < 2; ++s) {
                        key_t_ k = make_key(params, R, log_beta0, a, b, c, s);
                        eval_key(&k, q, r, &d2, &expo, &f);
                        k_sum += exp(expo - M) / e * (fabs(expo) + 1.0) * fabs(f - O);
                    }
        *kappa = k_sum;
    }

    if (dq_sens) {
        /* dO/dq contains 2 O sum softmax beta (q - p): an error in O moves it by
         * that error times 2 ||sum softmax beta (q - p)||. */
        double v[3] = {0.0, 0.0, 0.0};
        for (int a = lo[0]; a <= hi[0]; ++a)
            for (int b = lo[1]; b <= hi[1]; ++b)
                for (int c = lo[2]; c <= hi[2]; ++c)
                    for (int s = 0; s < 2; ++s) {
                        key_t_ k = make_key(params, R, log_beta0, a, b, c, s);
                        eval_key(&k, q, r, &d2, &expo, &f);
                        double w = exp(expo - M) / e;
                        for (int x = 0; x < 3; ++x) v[x] += w * k.beta * r[x];
                    }
        *dq_sens = 2.0 * sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    }

    if (dq) {
        /* Eq. func-normal: dO/dq = sum softmax * (df/dq + 2 beta (q - p)(O - f)),
         * df/dq = d for the first-order value. */
        double g[3] = {0.0, 0.0, 0.0};
        for (int a = lo[0]; a <= hi[0]; ++a)
            for (int b = lo[1]; b <= hi[1]; ++b)
                for (int c = lo[2]; c <= hi[2]; ++c)
                    for (int s = 0; s < 2; ++s) {
                        key_t_ k = make_key(params, R, log_beta0, a, b, c, s);
                        eval_key(&k, q, r, &d2, &expo, &f);
                        double w = exp(expo - M) / e;
                        for (int x = 0; x < 3; ++x)
                            g[x] += w * (k.d[x] + 2.0 * k.beta * r[x] * (O - f));
                    }
        dq[0] = g[0]; dq[1] = g[1]; dq[2] = g[2];
    }
}

/* Forward over J queries.  q: J rows of q_stride doubles (x, y, z first).
 * O, lse: J doubles each (lse may be NULL).  dq: J*3 doubles or NULL.
 * kappa, dq_sens: J doubles or NULL (diagnostics, see forward_one). */
void ora_forward(int R, int W, double log_beta0, const double *params, const double *q, int64_t J,
                 int q_stride, double *O, double *lse, double *dq, double *kappa, double *dq_sens)
{
    for (int64_t j = 0; j < J; ++j)
        forward_one(params, R, W, log_beta0, q + j * q_stride, &O[j], lse ? &lse[j] : NULL,
                    dq ? dq + 3 * j : NULL, kappa ? &kappa[j] : NULL, dq_sens ? &dq_sens[j] : NULL);
}

/* Error terms of dO/dq (Eq. func-normal) for its floating-point tolerance.
 * With g_i = d_i + 2 beta_i (q - p_i)(O - f_i) the term of key i,
 * G = dO/dq = sum softmax_i g_i:
 *   kappa_G = sum softmax * (|expo| + 1) * ||g - G||
 *     multiplying every weight by (1 + eps_i) moves G, to first order, by
 *     sum softmax_i eps_i (g_i - G) (plus the change of O, which enters with
 *     the factor dq_sens of forward_one): at most eps kappa_G when each
 *     exponent and weight carries a relative error eps;
 *   fabs = sum softmax * (|o| + |d_x r_x| + |d_y r_y| + |d_z r_z|)
 *     relative errors eps in every term of every value f move O by at most
 *     eps fabs;
 *   gabs = sum softmax * ||(|d_a| + 2 beta |r_a| |O - f|)_a||
 *     the same for the terms of G. */
static void err_terms_one(const double *params, int R, int W, double log_beta0, const double *q, double *kappa_G,
                          double *fabs_out, double *gabs_out)
{
    double O, lse, G[3];
    forward_one(params, R, W, log_beta0, q, &O, &lse, G, NULL, NULL);
    int lo[3], hi[3];
    window_range(q, R, W, lo, hi);
    double r[3], d2, expo, f, k_sum = 0.0, fa = 0.0, ga = 0.0;
    for (int a = lo[0]; a <= hi[0]; ++a)
        for (int b = lo[1]; b <= hi[1]; ++b)
            for (int c = lo[2]; c <= hi[2]; ++c)
                for (int s = 0; s < 2; ++s) {
                    key_t_ k = make_key(params, R, log_beta0, a, b, c, s);
                    eval_key(&k, q, r, &d2, &expo, &f);
                    const double w = exp(expo - lse);
                    double dev2 = 0.0, gab2 = 0.0;
                    for (int x = 0; x < 3; ++x) {
                        const double gx = k.d[x] + 2.0 * k.beta * r[x] * (O - f) - G[x];
                        dev2 += gx * gx;
                        const double ax = fabs(k.d[x]) + 2.0 * k.beta * fabs(r[x]) * fabs(O - f);
                        gab2 += ax * ax;
                    }
                    k_sum += w * (fabs(expo) + 1.0) * sqrt(dev2);
                    fa += w * (fabs(k.o) + fabs(k.d[0] * r[0]) + fabs(k.d[1] * r[1]) + fabs(k.d[2] * r[2]));
                    ga += w * sqrt(gab2);
                }
    *kappa_G = k_sum;
    *fabs_out = fa;
    *gabs_out = ga;
}

/* The error terms of J queries (q: J rows of q_stride doubles); diagnostics
 * for the floating-point tolerance of dO/dq. */
void ora_forward_err_terms(int R, int W, double log_beta0, const double *params, const double *q, int64_t J,
                           int q_stride, double *kappa_G, double *fabs_out, double *gabs_out)
{
    for (int64_t j = 0; j < J; ++j)
        err_terms_one(params, R, W, log_beta0, q + j * q_stride, &kappa_G[j], &fabs_out[j], &gabs_out[j]);
}

/* -------------------------------------------------------------- backward */

/* Algorithm 2 with the closed-form gradients of Sec. 3.6.  For every query j
 * and every key of its window:
 *   l            = exp(-beta ||q - p||^2) / e_j                     (softmax)
 *   dO/dphi      = l * df/dphi        (df/do = 1, df/dd = q - p)
 *   dO/dbeta     = l * ( -||q - p||^2 (f - O) )
 *   dO/dkey      = l * ( df/dkey + 2 beta (q - p)(f - O) ),  df/dkey = -d
 * and dL/dtheta += dL/dO_j * dO_j/dtheta.  The stored scale is the log offset
 * b (beta = exp(log_beta0 + b)), so dO/db = beta dO/dbeta; the offset key is
 * k_i + Delta_i with k_i fixed, so dO/dDelta = dO/dkey of the offset key.
 * Grid keys are fixed (configuration Full-4 of the ablation table): no
 * gradient for k_i.
 * grad: R^3*13 doubles, ACCUMULATED into.  gq: J*3 doubles or NULL, set to
 * dL/dO_j * dO_j/dq. */
void ora_backward(int R, int W, double log_beta0, const double *params, const double *q, int64_t J,
                  int q_stride, const double *gO, double *grad, double *gq)
{
    for (int64_t j = 0; j < J; ++j) {
        const double *qj = q + j * q_stride;
        double O, lse, dq[3];
        forward_one(params, R, W, log_beta0, qj, &O, &lse, gq ? dq : NULL, NULL, NULL);
        if (gq) {
            gq[3 * j + 0] = gO[j] * dq[0];
            gq[3 * j + 1] = gO[j] * dq[1];
            gq[3 * j + 2] = gO[j] * dq[2];
        }
        int lo[3], hi[3];
        window_range(qj, R, W, lo, hi);
        double r[3], d2, expo, f;
        for (int a = lo[0]; a <= hi[0]; ++a)
            for (int b = lo[1]; b <= hi[1]; ++b)
                for (int c = lo[2]; c <= hi[2]; ++c)
                    for (int s = 0; s < 2; ++s) {
                        key_t_ k = make_key(params, R, log_beta0, a, b, c, s);
                        eval_key(&k, qj, r, &d2, &expo, &f);
                        double l = exp(expo - lse);
                        double gl = gO[j] * l;
                        double *gr = grad + ((size_t)((size_t)a * R + b) * R + c) * NSLOT;
                        double dbeta = gl * (-d2 * (f - O));
                        if (s == 0) {
                            gr[5] += gl;
                            gr[6] += gl * r[0];
                            gr[7] += gl * r[1];
                            gr[8] += gl * r[2];
                            gr[3] += k.beta * dbeta;
                        } else {
                            gr[9] += gl;
                            gr[10] += gl * r[0];
                            gr[11] += gl * r[1];
                            gr[12] += gl * r[2];
                            gr[4] += k.beta * dbeta;
                            for (int x = 0; x < 3; ++x)
                                gr[x] += gl * (-k.d[x] + 2.0 * k.beta * r[x] * (f - O));
                        }
                    }
    }
}

/* Error terms of Algorithm 2's gradients for their floating-point
 * tolerance.  Every gradient entry is a sum over queries and keys of terms
 * t = dL/dO_j * softmax * (a slot's factor); where the terms cancel the sum
 * is small against them, so its rounding is bounded by the terms'
 * magnitudes, not by the sum:
 *   abs0[i, s] = sum |t|                         (rounding of the products and sums)
 *   abs1[i, s] = sum |t| * (|expo| + 1)          (relative error of the weight)
 * with every factor taken term by term in magnitude: o: 1, d: |q - p|,
 * b: beta ||q - p||^2 |f - O|, Delta: |d| + 2 beta |q - p| |f - O|.
 * abs0, abs1: R^3 * 13 doubles each, ACCUMULATED into. */
void ora_backward_err_terms(int R, int W, double log_beta0, const double *params, const double *q, int64_t J,
                            int q_stride, const double *gO, double *abs0, double *abs1)
{
    for (int64_t j = 0; j < J; ++j) {
        const double *qj = q + j * q_stride;
        double O, lse;
        forward_one(params, R, W, log_beta0, qj, &O, &lse, NULL, NULL, NULL);
        int lo[3], hi[3];
        window_range(qj, R, W, lo, hi);
        double r[3], d2, expo, f;
        for (int a = lo[0]; a <= hi[0]; ++a)
            for (int b = lo[1]; b <= hi[1]; ++b)
                for (int c = lo[2]; c <= hi[2]; ++c)
                    for (int s = 0; s < 2; ++s) {
                        key_t_ k = make_key(params, R, log_beta0, a, b, c, s);
                        eval_key(&k, qj, r, &d2, &expo, &f);
                        const double gl = fabs(gO[j]) * exp(expo - lse);
                        const double we = fabs(expo) + 1.0;
                        const size_t base = ((size_t)((size_t)a * R + b) * R + c) * NSLOT;
                        double t[NSLOT];
                        int slots[8], ns = 0;
                        const int so = s == 0 ? 5 : 9, sb = s == 0 ? 3 : 4;
                        t[so] = gl;
                        t[so + 1] = gl * fabs(r[0]);
                        t[so + 2] = gl * fabs(r[1]);
                        t[so + 3] = gl * fabs(r[2]);
                        t[sb] = gl * k.beta * d2 * fabs(f - O);
                        slots[ns++] = so; slots[ns++] = so + 1; slots[ns++] = so + 2; slots[ns++] = so + 3;
                        slots[ns++] = sb;
                        if (s == 1)
                            for (int x = 0; x < 3; ++x) {
                                t[x] = gl * (fabs(k.d[x]) + 2.0 * k.beta * fabs(r[x]) * fabs(f - O));
                                slots[ns++] = x;
                            }
                        for (int i = 0; i < ns; ++i) {
                            abs0[base + slots[i]] += t[slots[i]];
                            abs1[base + slots[i]] += t[slots[i]] * we;
                        }
                    }
    }
}

/* ------------------------------------------- backward through dO/dq */

/* Gradient of L = sum_j [ gO_j O(q_j) + gG_j . G(q_j) ] with respect to the
 * parameters, G = dO/dq of Eq. func-normal.  The second term is what a loss
 * on the query gradient (the Eikonal condition |dO/dq|^2 = 1 of Sec. 3.2, or
 * a normal-alignment loss) needs.  Derivation (per query, u = gG_j): write
 * every key's contribution to G as w (a + (f - O) t) with a = d (the value's
 * linear term), t = ds/dq = -2 beta (q - p), w the softmax weight.  With
 * h = u.a + (f - O)(u.t), H = u.G = sum w h and T = sum w (u.t), a change of
 * one key's exponent s, value f, slope a and gradient t gives
 *   d(u.G) = w { ds [(h - H) - (f - O) T] + df [(u.t) - T] + u.da + (f - O) u.dt }
 * (the normaliser and O are differentiated through; O changes by
 * w [ds (f - O) + df]).  Per parameter of a key:
 *   o:      df = 1
 *   d:      df = q - p,  da = unit vector
 *   beta:   ds = -|q - p|^2,  dt = -2 (q - p)        (chain rule to b: * beta)
 *   key p:  ds = 2 beta (q - p),  df = -d,  dt = 2 beta I   (Delta of offset keys)
 * gO may be NULL (no value term); gG may be NULL (plain backward).
 * grad: R^3*13 doubles, ACCUMULATED into. */
void ora_backward_grad(int R, int W, double log_beta0, const double *params, const double *q, int64_t J,
                       int q_stride, const double *gO, const double *gG, double *grad)
{
    for (int64_t j = 0; j < J; ++j) {
        const double *qj = q + j * q_stride;
        double O, lse, G[3];
        forward_one(params, R, W, log_beta0, qj, &O, &lse, G, NULL, NULL);
        const double go = gO ? gO[j] : 0.0;
        const double u[3] = {gG ? gG[3 * j] : 0.0, gG ? gG[3 * j + 1] : 0.0, gG ? gG[3 * j + 2] : 0.0};
        int lo[3], hi[3];
        window_range(qj, R, W, lo, hi);
        double r[3], d2, expo, f;
        /* V = sum w beta (q - p), T = -2 u.V, H = u.G */
        double V[3] = {0.0, 0.0, 0.0};
        for (int a = lo[0]; a <= hi[0]; ++a)
            for (int b = lo[1]; b <= hi[1]; ++b)
                for (int c = lo[2]; c <= hi[2]; ++c)
                    for (int s = 0; s < 2; ++s) {
                        key_t_ k = make_key(params, R, log_beta0, a, b, c, s);
                        eval_key(&k, qj, r, &d2, &expo, &f);
                        double w = exp(expo - lse);
                        for (int x = 0; x < 3; ++x) V[x] += w * k.beta * r[x];
                    }
        const double T = -2.0 * (u[0] * V[0] + u[1] * V[1] + u[2] * V[2]);
        const double H = u[0] * G[0] + u[1] * G[1] + u[2] * G[2];
        for (int a = lo[0]; a <= hi[0]; ++a)
            for (int b = lo[1]; b <= hi[1]; ++b)
                for (int c = lo[2]; c <= hi[2]; ++c)
                    for (int s = 0; s < 2; ++s) {
                        key_t_ k = make_key(params, R, log_beta0, a, b, c, s);
                        eval_key(&k, qj, r, &d2, &expo, &f);
                        const double w = exp(expo - lse);
                        const double dlt = f - O;
                        double ut = 0.0, ua = 0.0, ur = 0.0;
                        for (int x = 0; x < 3; ++x) {
                            ut += u[x] * (-2.0 * k.beta * r[x]);
                            ua += u[x] * k.d[x];
                            ur += u[x] * r[x];
                        }
                        const double h = ua + dlt * ut;
                        const double e1 = ut - T;
                        const double hH = (h - H) - dlt * T;
                        /* d(u.G) and d O per parameter, then weighted by u / gO */
                        const double g_o = w * e1 + go * w;
                        double g_d[3], g_p[3];
                        for (int x = 0; x < 3; ++x) {
                            g_d[x] = w * (r[x] * e1 + u[x]) + go * w * r[x];
                            g_p[x] = w * (2.0 * k.beta * r[x] * hH - k.d[x] * e1 + 2.0 * k.beta * dlt * u[x]) +
                                     go * w * (-k.d[x] + 2.0 * k.beta * r[x] * dlt);
                        }
                        const double g_beta = w * (-d2 * hH - 2.0 * dlt * ur) + go * w * (-d2 * dlt);
                        double *gr = grad + ((size_t)((size_t)a * R + b) * R + c) * NSLOT;
                        if (s == 0) {
                            gr[5] += g_o;
                            gr[6] += g_d[0]; gr[7] += g_d[1]; gr[8] += g_d[2];
                            gr[3] += k.beta * g_beta;
                        } else {
                            gr[9] += g_o;
                            gr[10] += g_d[0]; gr[11] += g_d[1]; gr[12] += g_d[2];
                            gr[4] += k.beta * g_beta;
                            gr[0] += g_p[0]; gr[1] += g_p[1]; gr[2] += g_p[2];
                        }
                    }
    }
}

/* ------------------------------------------------ global-support brute force */

/* The paper's global model (Algorithm 1 over ALL I centres, both key sets),
 * written as an explicit table of the 2I key exponents and values followed by
 * a two-pass softmax.  No window is involved; it pins the windowed oracle.
 * scratch: 4*R^3 doubles. */
void ora_forward_global(int R, double log_beta0, const double *params, const double *q, int64_t J,
                        int q_stride, double *O, double *scratch)
{
    int64_t I = (int64_t)R * R * R;
    double *ex = scratch, *fv = scratch + 2 * I;
    for (int64_t j = 0; j < J; ++j) {
        const double *qj = q + j * q_stride;
        double M = -INFINITY;
        for (int64_t i = 0; i < I; ++i) {
            int a = (int)(i / ((int64_t)R * R)), b = (int)((i / R) % R), c = (int)(i % R);
            for (int s = 0; s < 2; ++s) {
                key_t_ k = make_key(params, R, log_beta0, a, b, c, s);
                double r[3], d2;
                eval_key(&k, qj, r, &d2, &ex[2 * i + s], &fv[2 * i + s]);
                if (ex[2 * i + s] > M) M = ex[2 * i + s];
            }
        }
        double e = 0.0, m = 0.0;
        for (int64_t t = 0; t < 2 * I; ++t) {
            double l = exp(ex[t] - M);
            e += l;
            m += l * fv[t];
        }
        O[j] = m / e;
    }
}

/* ---------------------------------------------------- mean-shift init */

/* Offset initialisation of Sec. 3.3: for every grid centre k_i
 *   Delta_i = sum_n exp(-bw ||k_i - s_n||^2) s_n / sum_n exp(-bw ||k_i - s_n||^2) - k_i
 * over N surface points s_n (bw = 100 in the paper), evaluated with the
 * largest exponent subtracted (the ratio is unchanged and stays defined for
 * centres far from every point).  pts: N x 3 doubles; delta: R^3 x 3 doubles. */
void ora_mean_shift(int R, double bw, const double *pts, int64_t N, double *delta)
{
    for (int a = 0; a < R; ++a)
        for (int b = 0; b < R; ++b)
            for (int c = 0; c < R; ++c) {
                const double k[3] = {centre_coord(a, R), centre_coord(b, R), centre_coord(c, R)};
                double M = -INFINITY;
                for (int64_t n = 0; n < N; ++n) {
                    double d2 = 0.0;
                    for (int x = 0; x < 3; ++x) d2 += (k[x] - pts[3 * n + x]) * (k[x] - pts[3 * n + x]);
                    if (-bw * d2 > M) M = -bw * d2;
                }
                double Z = 0.0, S[3] = {0.0, 0.0, 0.0};
                for (int64_t n = 0; n < N; ++n) {
                    double d2 = 0.0;
                    for (int x = 0; x < 3; ++x) d2 += (k[x] - pts[3 * n + x]) * (k[x] - pts[3 * n + x]);
                    const double w = exp(-bw * d2 - M);
                    Z += w;
                    for (int x = 0; x < 3; ++x) S[x] += w * pts[3 * n + x];
                }
                double *dl = delta + 3 * ((size_t)((size_t)a * R + b) * R + c);
                for (int x = 0; x < 3; ++x) dl[x] = S[x] / Z - k[x];
            }
}

/* ------------------------------------------------- ablation variants */

/* The configurations of Table tab:ablation as one family (Sec. 3.2
 * Eq. func-interp and Eq. poly-func, Sec. 3.3 Eq. func-offset):
 *   sets   1 = grid keys k_i only (Config-G-*), 2 = offset keys k_i + Delta_i
 *          only (Config-Full-1/2), 3 = both under one softmax (Full-3/4)
 *   deg    degree of the value polynomial, 0..3, in Taylor form
 *            f(x) = o + sum_a d_a x_a + 1/2 sum_ab S_ab x_a x_b
 *                   + 1/6 sum_abc T_abc x_a x_b x_c
 *          with S and T symmetric (the "..." of Eq. poly-func read as the
 *          next Taylor term)
 *   learn  1: a log-scale b per key, beta = exp(log_beta0 + b);
 *          0: beta = exp(log_beta0) fixed (Config-G-1..4)
 * Channels per centre, in the tuple order of Eq. func-offset:
 *   [Delta (3) if offset keys] [b of each key set if learn] [phi of each key set]
 * phi = (o, d_x, d_y, d_z, S_xx, S_yy, S_zz, S_xy, S_xz, S_yz, T_xxx, T_yyy,
 * T_zzz, T_xxy, T_xxz, T_xyy, T_yyz, T_xzz, T_yzz, T_xyz) truncated to 1, 4,
 * 10 or 20 entries; grid set first.  sets = 3, deg = 1, learn = 1 is the
 * 13-float layout above.  Only the offset keys move (grid keys are fixed in
 * every configuration of the table). */

static const int VAR_NV[4] = {1, 4, 10, 20};

static int var_nsets(int sets) { return (sets & 1) + ((sets >> 1) & 1); }

int ora_variant_channels(int sets, int deg, int learn)
{
    if (sets < 1 || sets > 3 || deg < 0 || deg > 3 || (learn != 0 && learn != 1)) return -1;
    return ((sets & 2) ? 3 : 0) + learn * var_nsets(sets) + VAR_NV[deg] * var_nsets(sets);
}

/* channel of key set s's log-scale (-1 if fixed) and of its first phi entry */
static void var_channels_of(int sets, int deg, int learn, int s, int *i_b, int *i_phi)
{
    int base = (sets & 2) ? 3 : 0;
    int rank = (s == 1 && (sets & 1)) ? 1 : 0;   /* position among the present sets */
    *i_b = learn ? base + rank : -1;
    *i_phi = base + learn * var_nsets(sets) + VAR_NV[deg] * rank;
}

/* index into phi of the symmetric cubic coefficient T_abc */
static int var_cubic_index(int a, int b, int c)
{
    int t;
    if (a > b) { t = a; a = b; b = t; }
    if (b > c) { t = b; b = c; c = t; }
    if (a > b) { t = a; a = b; b = t; }
    if (a == b && b == c) return 10 + a;                       /* xxx yyy zzz */
    if (a == 0 && b == 0) return c == 1 ? 13 : 14;             /* xxy xxz */
    if (a == 0 && b == 1 && c == 1) return 15;                 /* xyy */
    if (a == 1 && b == 1) return 16;                           /* yyz */
    if (a == 0 && b == 2) return 17;                           /* xzz */
    if (a == 1 && b == 2) return 18;                           /* yzz */
    return 19;                                                 /* xyz */
}

/* f(x) and grad f(x) of the Taylor-form polynomial of degree deg */
static void var_poly(int deg, const double *phi, const double x[3], double *f, double g[3])
{
    double S[3][3] = {{0}}, T[3][3][3] = {{{0}}};
    if (deg >= 2) {
        S[0][0] = phi[4]; S[1][1] = phi[5]; S[2][2] = phi[6];
        S[0][1] = S[1][0] = phi[7];
        S[0][2] = S[2][0] = phi[8];
        S[1][2] = S[2][1] = phi[9];
    }
    if (deg >= 3)
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                for (int c = 0; c < 3; ++c) T[a][b][c] = phi[var_cubic_index(a, b, c)];
    double v = phi[0];
    for (int a = 0; a < 3; ++a) g[a] = 0.0;
    if (deg >= 1)
        for (int a = 0; a < 3; ++a) {
            v += phi[1 + a] * x[a];
            g[a] += phi[1 + a];
        }
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            v += 0.5 * S[a][b] * x[a] * x[b];
            g[a] += S[a][b] * x[b];
            for (int c = 0; c < 3; ++c) {
                v += T[a][b][c] * x[a] * x[b] * x[c] / 6.0;
                g[a] += 0.5 * T[a][b][c] * x[b] * x[c];
            }
        }
    *f = v;
}

typedef struct {
    double p[3];
    double beta;
    const double *phi;
    double *grad_phi;   /* NULL in the forward */
    double *grad_b;     /* NULL if the scale is fixed */
    double *grad_delta; /* NULL for grid keys */
} var_key_t;

static var_key_t var_make_key(const double *params, double *grad, int R, double log_beta0, int sets, int deg,
                              int learn, int a, int b, int c, int s)
{
    int ch = ora_variant_channels(sets, deg, learn), i_b, i_phi;
    var_channels_of(sets, deg, learn, s, &i_b, &i_phi);
    size_t row = ((size_t)((size_t)a * R + b) * R + c) * (size_t)ch;
    const double *th = params + row;
    var_key_t k;
    k.p[0] = centre_coord(a, R);
    k.p[1] = centre_coord(b, R);
    k.p[2] = centre_coord(c, R);
    if (s == 1) {
        k.p[0] += th[0]; k.p[1] += th[1]; k.p[2] += th[2];
    }
    k.beta = exp(log_beta0 + (learn ? th[i_b] : 0.0));
    k.phi = th + i_phi;
    k.grad_phi = grad ? grad + row + i_phi : NULL;
    k.grad_b = (grad && learn) ? grad + row + i_b : NULL;
    k.grad_delta = (grad && s == 1) ? grad + row : NULL;
    return k;
}

/* O and lse of one query (Algorithm 1 with the maximum exponent subtracted);
 * with grad != NULL also accumulates gO * dO/dtheta into grad (Algorithm 2):
 *   dO/dphi_m   = softmax * df/dphi_m (f is linear in phi: f evaluated at the
 *                 unit vector e_m)
 *   dO/db       = softmax * beta * (-||x||^2 (f - O))
 *   dO/dDelta   = softmax * (-grad f(x) + 2 beta x (f - O)),  x = q - key */
static void variant_one(const double *params, double *grad, double gO, int R, int W, double log_beta0, int sets,
                        int deg, int learn, const double *q, double *O_out, double *lse_out, double *kappa,
                        double *fabs_out)
{
    int lo[3], hi[3];
    window_range(q, R, W, lo, hi);
    double M = -INFINITY, O = 0.0, lse = 0.0;
    /* pass 0: maximum exponent; pass 1: e_j, m_j; pass 2: gradients */
    for (int pass = 0; pass < 3; ++pass) {
        double e = 0.0, m = 0.0;
        for (int a = lo[0]; a <= hi[0]; ++a)
            for (int b = lo[1]; b <= hi[1]; ++b)
                for (int c = lo[2]; c <= hi[2]; ++c)
                    for (int s = 0; s < 2; ++s) {
                        if (!(sets & (1 << s))) continue;
                        var_key_t k = var_make_key(params, pass == 2 ? grad : NULL, R, log_beta0, sets, deg, learn,
                                                   a, b, c, s);
                        double x[3] = {q[0] - k.p[0], q[1] - k.p[1], q[2] - k.p[2]};
                        double d2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
                        double expo = -k.beta * d2;
                        double f, g[3];
                        var_poly(deg, k.phi, x, &f, g);
                        if (pass == 0) {
                            if (expo > M) M = expo;
                        } else if (pass == 1) {
                            double l = exp(expo - M);
                            e += l;
                            m += l * f;
                        } else if (!grad) {
                            /* diagnostics: kappa as in forward_one; fabs = sum softmax *
                             * sum_m |phi_m df/dphi_m|, the scale of the rounding of f */
                            double w = exp(expo - lse), fa = 0.0;
                            for (int i = 0; i < VAR_NV[deg]; ++i) {
                                double unit[20] = {0}, fu, gu[3];
                                unit[i] = 1.0;
                                var_poly(deg, unit, x, &fu, gu);
                                fa += fabs(k.phi[i] * fu);
                            }
                            *kappa += w * (fabs(expo) + 1.0) * fabs(f - O);
                            *fabs_out += w * fa;
                        } else {
                            double gl = gO * exp(expo - lse);
                            for (int i = 0; i < VAR_NV[deg]; ++i) {
                                double unit[20] = {0}, fu, gu[3];
                                unit[i] = 1.0;
                                var_poly(deg, unit, x, &fu, gu);
                                k.grad_phi[i] += gl * fu;
                            }
                            if (k.grad_b) *k.grad_b += gl * k.beta * (-d2 * (f - O));
                            if (k.grad_delta)
                                for (int i = 0; i < 3; ++i)
                                    k.grad_delta[i] += gl * (-g[i] + 2.0 * k.beta * x[i] * (f - O));
                        }
                    }
        if (pass == 1) {
            O = m / e;
            lse = M + log(e);
            *O_out = O;
            if (lse_out) *lse_out = lse;
            if (!grad && !kappa) return;
            if (kappa) *kappa = *fabs_out = 0.0;
        }
    }
}

/* Forward of a variant over J queries (rows of q_stride doubles).
 * O, lse: J doubles (lse may be NULL).  kappa, fabs: J doubles or both NULL
 * (diagnostics for FP32 tolerances: kappa as in ora_forward, fabs = sum of
 * softmax times the sum of the absolute terms of f). */
void ora_variant_forward(int R, int W, double log_beta0, int sets, int deg, int learn, const double *params,
                         const double *q, int64_t J, int q_stride, double *O, double *lse, double *kappa,
                         double *fabs_out)
{
    for (int64_t j = 0; j < J; ++j)
        variant_one(params, NULL, 0.0, R, W, log_beta0, sets, deg, learn, q + j * q_stride, &O[j],
                    lse ? &lse[j] : NULL, kappa ? &kappa[j] : NULL, kappa ? &fabs_out[j] : NULL);
}

/* Backward of a variant: grad (R^3 * channels doubles) ACCUMULATES
 * sum_j gO_j dO_j/dtheta. */
void ora_variant_backward(int R, int W, double log_beta0, int sets, int deg, int learn, const double *params,
                          const double *q, int64_t J, int q_stride, const double *gO, double *grad)
{
    for (int64_t j = 0; j < J; ++j) {
        double O;
        variant_one(params, grad, gO[j], R, W, log_beta0, sets, deg, learn, q + j * q_stride, &O, NULL, NULL, NULL);
    }
}

/* ---------------------------------------------- cosine-series decomposition */

/* Sec. 4.4 Eq. o-as-value / Eq. cosine-series: S(q) = sum_b w_b(q) O_b(q)
 * with cosine weights and one Config-G-6 representation per band (grid keys,
 * first-order values, learnable scales: 5 floats per centre).  Readings: the
 * weight of band b at a 3-D query is the separable cosine
 *   w_b(q) = cos(b pi q_x) cos(b pi q_y) cos(b pi q_z),
 * and there are B bands b = 0 .. B-1 (20480 B parameters at 16^3, and B = 1
 * is Config-G-6).  params: B blocks of R^3 x 5 floats, band-major. */
static double cosine_weight(int b, const double *q)
{
    const double pi = 3.14159265358979323846;
    return cos(b * pi * q[0]) * cos(b * pi * q[1]) * cos(b * pi * q[2]);
}

void ora_cosine_forward(int R, int W, double log_beta0, int B, const double *params, const double *q, int64_t J,
                        int q_stride, double *S)
{
    const size_t band = (size_t)R * R * R * 5;
    for (int64_t j = 0; j < J; ++j) {
        const double *qj = q + j * q_stride;
        double s = 0.0;
        for (int b = 0; b < B; ++b) {
            double O;
            variant_one(params + b * band, NULL, 0.0, R, W, log_beta0, 1, 1, 1, qj, &O, NULL, NULL, NULL);
            s += cosine_weight(b, qj) * O;
        }
        S[j] = s;
    }
}

/* dS/dtheta_b = w_b(q) dO_b/dtheta_b: each band's backward with upstream
 * gS_j w_b(q_j).  grad (B x R^3 x 5) is ACCUMULATED into. */
void ora_cosine_backward(int R, int W, double log_beta0, int B, const double *params, const double *q, int64_t J,
                         int q_stride, const double *gS, double *grad)
{
    const size_t band = (size_t)R * R * R * 5;
    for (int64_t j = 0; j < J; ++j) {
        const double *qj = q + j * q_stride;
        for (int b = 0; b < B; ++b) {
            double O;
            variant_one(params + b * band, grad + b * band, gS[j] * cosine_weight(b, qj), R, W, log_beta0, 1, 1, 1,
                        qj, &O, NULL, NULL, NULL);
        }
    }
}

/* ------------------------------------------------------------------ loss */

/* Eq. loss (MSE) and the L1 variant: the upstream gradient dL/dO_j and the
 * loss value.  loss_kind 0 = L1 (sign(0) = 0), 1 = MSE.  target: J doubles. */
void ora_loss_grad(int loss_kind, const double *O, const double *target, int64_t J, double *gO,
                   double *loss_out, double *mae_out)
{
    double L = 0.0, mae = 0.0;
    for (int64_t j = 0; j < J; ++j) {
        double diff = O[j] - target[j];
        mae += fabs(diff);
        if (loss_kind == 0) {
            L += fabs(diff);
            gO[j] = (diff > 0.0 ? 1.0 : (diff < 0.0 ? -1.0 : 0.0)) / (double)J;
        } else {
            L += diff * diff;
            gO[j] = 2.0 * diff / (double)J;
        }
    }
    if (loss_out) *loss_out = J > 0 ? L / (double)J : 0.0;
    if (mae_out) *mae_out = J > 0 ? mae / (double)J : 0.0;
}

/* ------------------------------------------------------------------ Adam */

/* One Adam / AdamW step with torch.optim semantics (Adam: L2 penalty added to
 * the gradient; AdamW: decoupled decay p *= 1 - lr*wd).  step is 1-based.  The
 * gradient is left untouched. */
void ora_adam(int64_t n, double *p, const double *g, double *m, double *v, int64_t step, double lr,
              double beta1, double beta2, double eps, double wd, int decoupled)
{
    double bc1 = 1.0 - pow(beta1, (double)step);
    double bc2 = 1.0 - pow(beta2, (double)step);
    for (int64_t i = 0; i < n; ++i) {
        double gi = g[i];
        if (decoupled)
            p[i] *= 1.0 - lr * wd;
        else
            gi += wd * p[i];
        m[i] = beta1 * m[i] + (1.0 - beta1) * gi;
        v[i] = beta2 * v[i] + (1.0 - beta2) * gi * gi;
        double mhat = m[i] / bc1;
        double vhat = v[i] / bc2;
        p[i] -= lr * mhat / (sqrt(vhat) + eps);
    }
}
