/*
 * efunc.h -- C ABI of the GB300 (sm_103a) library for the O^{+Delta}
 * representation of "efunc: An Efficient Function Representation without
 * Neural Networks" (arXiv 2505.21319).
 *
 * Representation (Sec. 3.3, Eq. func-offset, first-order values of Sec. 3.2):
 *   an R x R x R grid of centres k_i = -1 + (idx + 0.5) * 2/R on [-1,1]^3, each
 *   holding 13 FP32 parameters, stored row-major as
 *       params[((a*R + b)*R + c)*13 + slot]      (a = x index, slowest)
 *   slot  0..2  Delta       offset of the second key, k_i + Delta_i
 *         3     b           grid-key log-scale,   beta  = exp(log_beta0 + b)
 *         4     b'          offset-key log-scale, beta' = exp(log_beta0 + b')
 *         5     o           grid-key value constant
 *         6..8  d           grid-key value linear term, f = o + d.(q - k)
 *         9     o'          offset-key value constant
 *         10..12 d'         offset-key value linear term, f' = o' + d'.(q - k - Delta)
 *   O(q) = sum over keys of softmax(-beta ||q - key||^2) * f(q - key), one
 *   softmax over the union of grid keys and offset keys (Eq. func-offset).
 *
 * Support: each query blends the (2W)^3 centres whose index lies in
 * [c - W + 1, c + W] per axis, with c = clamp(floor((q+1)*R/2 - 1/2), -1, R-1)
 * evaluated in FP32 without fused multiply-add; indices outside [0, R-1] are
 * dropped.  W = 2 (64 centres, 128 keys) is the implemented width.  The
 * paper's own sum is global (Algorithm 1); at the initial scale a truncated
 * key weighs at most exp(-3.25 * beta h^2) ~ 1e-6 of the nearest one.
 *
 * Conventions for every call:
 *   - Pointers marked [device] are device pointers owned by the caller; the
 *     library never frees or keeps them.  [host|device] accepts either.
 *   - Calls are asynchronous on `stream` (a cudaStream_t; NULL = legacy
 *     default stream) unless stated otherwise.
 *   - Work memory comes from the caller: `workspace` [device] of at least
 *     efunc_eval_workspace_bytes(grid, J) bytes for the sort, forward and
 *     backward, efunc_workspace_bytes(grid, J) for efunc_fit (or the
 *     variant / cosine / pipelined-fit sizes below), 256-byte aligned.  Concurrent calls must not share a workspace.
 *     The library allocates no device memory; it creates, once per device,
 *     the copy and sort streams and events of efunc_fit.
 *   - Arguments are validated on the host before anything is launched; an
 *     invalid argument returns EFUNC_ERR_ARG (or _WORKSPACE / _NONFINITE /
 *     _UNSUPPORTED) and enqueues nothing.  A failing CUDA call returns
 *     EFUNC_ERR_CUDA.  Nothing aborts the process.
 *   - Queries: q holds J rows of q_stride floats (q_stride 3 or 4), x,y,z
 *     first, J in [0, 2^30] (J = 0 enqueues nothing and returns EFUNC_OK;
 *     the fitting loops need J >= 1).  Outputs indexed by query are in the
 *     caller's query order.
 *   - Non-finite parameters or queries give non-finite outputs; they are not
 *     checked.
 */
#ifndef EFUNC_H
#define EFUNC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *efunc_stream_t; /* same handle as cudaStream_t */

typedef enum {
    EFUNC_OK = 0,
    EFUNC_ERR_ARG = 1,         /* invalid argument, nothing enqueued */
    EFUNC_ERR_CUDA = 2,        /* a CUDA runtime call failed */
    EFUNC_ERR_WORKSPACE = 3,   /* workspace NULL, misaligned or too small */
    EFUNC_ERR_NONFINITE = 4,   /* a hyper-parameter is NaN or infinite */
    EFUNC_ERR_UNSUPPORTED = 5, /* valid request outside the implemented set */
    EFUNC_ERR_IO = 6,          /* checkpoint file missing, unwritable, short or corrupt */
    EFUNC_ERR_TIMEOUT = 7      /* a bounded wait inside a kernel ran out (efunc_encoder_status) */
} efunc_status;

/* Grid description.  R in [1, 256]; W must be 2; log_beta0 is the log-scale
 * that b = 0 stands for (Sec. 4.3 initialises scales to exp(7) at R = 32;
 * efunc_default_log_beta0 keeps beta*h^2 fixed across R). */
typedef struct {
    int32_t R;
    int32_t W;
    float log_beta0;
} efunc_grid;

typedef enum { EFUNC_LOSS_L1 = 0, EFUNC_LOSS_MSE = 1 } efunc_loss;

/* Adam (decoupled = 0: weight_decay added to the gradient) or AdamW
 * (decoupled = 1: p *= 1 - lr*weight_decay), torch.optim semantics.
 * Sec. 3.4 fits with Adam; Sec. 4.2 uses AdamW with lr 6e-4.  The
 * hyper-parameters are double so that 1 - beta2 and the bias corrections are
 * formed before rounding to the FP32 arithmetic of the kernel. */
typedef struct {
    double lr, beta1, beta2, eps, weight_decay;
    int32_t decoupled;
} efunc_adam;

/* Ablation variant of the representation (Table tab:ablation, Sec. 4.3).
 *   sets         EFUNC_KEYS_GRID: fixed grid keys only (Config-G-*);
 *                EFUNC_KEYS_OFFSET: offset keys k_i + Delta_i only
 *                (Config-Full-1/2, learnable key positions);
 *                EFUNC_KEYS_BOTH: both under one softmax (Full-3/4,
 *                Eq. func-offset)
 *   degree       0..3, degree of the value polynomial of Sec. 3.2
 *                Eq. poly-func in Taylor form
 *                  f(x) = o + d.x + 1/2 x^T S x + 1/6 T[x, x, x]
 *                with S, T symmetric
 *   learn_scale  1: a log-scale b per key, beta = exp(log_beta0 + b);
 *                0: beta = exp(log_beta0) (Config-G-1..4)
 * Parameter layout per centre (row of efunc_variant_channels floats), in the
 * tuple order of Eq. func-offset: [Delta (3), if offset keys] [b of each key
 * set, if learn_scale] [phi of each key set], grid set first, with
 *   phi = (o, d_x, d_y, d_z, S_xx, S_yy, S_zz, S_xy, S_xz, S_yz, T_xxx,
 *          T_yyy, T_zzz, T_xxy, T_xxz, T_xyy, T_yyz, T_xzz, T_yzz, T_xyz)
 * truncated to 1, 4, 10 or 20 entries.  {EFUNC_KEYS_BOTH, 1, 1} is the
 * 13-float layout of the default model. */
typedef enum { EFUNC_KEYS_GRID = 1, EFUNC_KEYS_OFFSET = 2, EFUNC_KEYS_BOTH = 3 } efunc_key_sets;

typedef struct {
    int32_t sets;
    int32_t degree;
    int32_t learn_scale;
} efunc_variant;

/* ---------------------------------------------------------------- helpers */

/* Number of floats in the parameter grid, R^3 * 13 (Sec. 3.3: theta in
 * R^{R^3 x (5 + |phi| + |phi'|)}).  -1 if R is outside [1, 256]. */
int64_t efunc_param_count(int32_t R);

/* 7 + 2 ln(R/32): exp(7) at R = 32 (Sec. 4.3), beta*h^2 constant in R. */
float efunc_default_log_beta0(int32_t R);

/* Static description of a status code.  Never NULL. */
const char *efunc_status_str(efunc_status s);

/* Bytes of workspace that suffice for every call of the default model below
 * for J queries on this grid, including the in-line efunc_fit (efunc_fit can
 * use more, see efunc_fit_workspace_bytes; the sort, forward and backward
 * need only efunc_eval_workspace_bytes; the variant and cosine calls have
 * their own sizes).  0 if the grid is invalid. */
size_t efunc_workspace_bytes(const efunc_grid *grid, int64_t J);

/* Bytes of workspace that suffice for efunc_cell_sort, efunc_forward,
 * efunc_backward and efunc_backward_grad for J queries on this grid: the
 * sort buffers and key records, without the gradient grid and host-batch
 * staging buffers that only efunc_fit uses (about 32 bytes per query and
 * 52 R^3 bytes less than efunc_workspace_bytes).  0 if the grid is
 * invalid. */
size_t efunc_eval_workspace_bytes(const efunc_grid *grid, int64_t J);

/* Bytes of workspace with which efunc_fit pipelines its steps: the sort of
 * batch s+1 runs on a library-owned stream, into a second sort buffer, while
 * batch s is computed on the caller's stream (about 20 bytes per query more
 * than efunc_workspace_bytes).  With less (but at least
 * efunc_workspace_bytes) efunc_fit sorts each batch in line.  0 if the grid
 * is invalid. */
size_t efunc_fit_workspace_bytes(const efunc_grid *grid, int64_t J);

/* ------------------------------------------------------------ entry points */

/* Cell sort (hot-path step a1; not in the paper, whose Algorithm 1 visits
 * every key): groups the J queries by window base cell, cells in 4x4x4 bricks,
 * Morton order inside a brick.
 *   q        [device] J rows of q_stride floats
 *   q_sorted [device] J x 4 floats, 16-byte aligned: (x, y, z, w) with w the
 *            4th input column when q_stride == 4, else 0
 *   perm     [device] J int32: q_sorted row i is input row perm[i]
 * The order of queries inside a cell is unspecified (atomic arrival order). */
efunc_status efunc_cell_sort(const efunc_grid *grid, const float *q, int64_t J, int32_t q_stride,
                             float *q_sorted, int32_t *perm, void *workspace, size_t workspace_bytes,
                             efunc_stream_t stream);

/* Forward (Sec. 3.5, Algorithm 1; Eq. func-offset): O(q_j) for J queries.
 *   params   [device] R^3*13 floats (layout above)
 *   q        [device] J rows of q_stride floats
 *   O        [device] J floats, written
 *   lse      [device] J floats or NULL: natural log of the softmax
 *            normaliser, log(sum_keys exp(-beta ||q - key||^2)) (the e_j of
 *            Algorithm 1, in log form)
 *   dOdq     [device] J*3 floats or NULL: dO/dq (Eq. func-normal) */
efunc_status efunc_forward(const efunc_grid *grid, const float *params, const float *q, int64_t J,
                           int32_t q_stride, float *O, float *lse, float *dOdq, void *workspace,
                           size_t workspace_bytes, efunc_stream_t stream);

/* Backward (Sec. 3.6, Algorithm 2 and the closed-form dO/dk, dO/dbeta,
 * dO/dphi): recomputes the weights from params (no per-query state is kept
 * between forward and backward) and ACCUMULATES
 *   grad[i*13 + s] += sum_j gO_j * dO(q_j)/dtheta_{i,s}
 * with the chain rule to the stored log-scales (dO/db = beta dO/dbeta) and to
 * Delta (the offset key's dO/dk).  Grid keys are fixed.
 *   gO       [device] J floats: dL/dO_j
 *   grad     [device] R^3*13 floats, accumulated into (FP32 atomics: the
 *            summation order is not deterministic)
 *   gq       [device] J*3 floats or NULL: written with gO_j * dO/dq_j */
efunc_status efunc_backward(const efunc_grid *grid, const float *params, const float *q, int64_t J,
                            int32_t q_stride, const float *gO, float *grad, float *gq, void *workspace,
                            size_t workspace_bytes, efunc_stream_t stream);

/* Backward through the value and its query gradient: ACCUMULATES
 *   grad[i*13 + s] += sum_j [ gO_j dO(q_j)/dtheta + gG_j . d(dO/dq)(q_j)/dtheta ]
 * where dO/dq is Eq. func-normal (Sec. 3.2).  The second term is what a loss
 * on the query gradient needs: the Eikonal condition |dO/dq|^2 = 1 that
 * Sec. 3.2 states for signed distance functions, or a normal-alignment loss
 * (Sec. 4.6 uses dO/dq as the surface normal).  Per query it needs, besides
 * the forward, H = gG . dO/dq and T = -2 gG . sum softmax beta (q - key); the
 * per-key gradient then follows from differentiating every key's
 * contribution w (d + (f - O) ds/dq) to dO/dq once more.
 *   gO       [device] J floats or NULL (no value term)
 *   gG       [device] J x 3 floats or NULL (then this is efunc_backward)
 *   grad     [device] R^3*13 floats, accumulated into
 * At least one of gO, gG must be given. */
efunc_status efunc_backward_grad(const efunc_grid *grid, const float *params, const float *q, int64_t J,
                                 int32_t q_stride, const float *gO, const float *gG, float *grad, void *workspace,
                                 size_t workspace_bytes, efunc_stream_t stream);

/* Loss of the representation on a batch of J rows (x, y, z, target SDF),
 * without any gradient: the forward of Algorithm 1 at every row, then
 *   out[0] = mean_j (O_j - o_j)^2     (Eq. loss)
 *   out[1] = mean_j |O_j - o_j|       (the absolute error the paper reports
 *                                      as its AE metrics, Sec. 4.1)
 * summed in FP64 and written as FP32.  For held-out error curves of a fit.
 *   qo       [device] J x 4 floats, J >= 1
 *   out      [device] 2 floats
 *   workspace  at least efunc_eval_workspace_bytes(grid, J) */
efunc_status efunc_eval_loss(const efunc_grid *grid, const float *params, const float *qo, int64_t J, float *out,
                             void *workspace, size_t workspace_bytes, efunc_stream_t stream);

/* ------------------------------------------------------------- FP64 path */

/* The forward and backward above in FP64 (Algorithm 1, Algorithm 2, Eq.
 * func-normal), for finite-difference checks of the implementation: the same
 * fused kernels instantiated for double, with exp2 / log2 in double instead
 * of the SFU approximations.  The window of a query is chosen, as in the
 * FP32 path, from its coordinates rounded to FP32; everything after that is
 * FP64.  Not a hot path (FP64 runs far below the FP32 rate on this GPU).
 *   params   [device] R^3*13 doubles; q [device] J rows of q_stride doubles;
 *   O, lse, dOdq, gO, grad, gq as efunc_forward / efunc_backward, in double
 *   workspace  at least efunc_f64_workspace_bytes(grid, J) */
size_t efunc_f64_workspace_bytes(const efunc_grid *grid, int64_t J);

efunc_status efunc_forward_f64(const efunc_grid *grid, const double *params, const double *q, int64_t J,
                               int32_t q_stride, double *O, double *lse, double *dOdq, void *workspace,
                               size_t workspace_bytes, efunc_stream_t stream);

/* ACCUMULATES grad[i*13 + s] += sum_j gO_j dO(q_j)/dtheta_{i,s} (double
 * atomics); gq (or NULL) is written with gO_j dO/dq_j. */
efunc_status efunc_backward_f64(const efunc_grid *grid, const double *params, const double *q, int64_t J,
                                int32_t q_stride, const double *gO, double *grad, double *gq, void *workspace,
                                size_t workspace_bytes, efunc_stream_t stream);

/* One Adam/AdamW step over n floats (Sec. 3.4), step is 1-based (bias
 * correction).  params, m, v are updated in place; grad is read and then
 * zeroed.  All four [device], n >= 0. */
efunc_status efunc_adam_step(const efunc_adam *adam, int64_t n, float *params, float *grad, float *m,
                             float *v, int64_t step, efunc_stream_t stream);

/* Fitting loop (Sec. 3.4): for s in [0, steps): take batch (s mod n_batches)
 * of J rows (x, y, z, target SDF) from qo, cell-sort it, run the fused
 * forward + loss gradient + backward, then one Adam step with step number
 * step0 + s + 1.
 *   loss     EFUNC_LOSS_L1 (dL/dO = sign(O - o)/J, sign(0) = 0) or
 *            EFUNC_LOSS_MSE (Eq. loss, 2(O - o)/J)
 *   eikonal_weight  >= 0: adds weight * mean_j (|dO/dq(q_j)|^2 - 1)^2, the
 *            Eikonal condition of Sec. 3.2 in its squared form, whose
 *            gradient goes through efunc_backward_grad's second-order term
 *            inside the fused kernel; 0 disables it
 *   params, m, v  [device] R^3*13 floats each, updated
 *   qo       [host|device] n_batches*J*4 floats.  Host memory is copied
 *            to the device inside every step; the copy of batch s+1 runs on
 *            a copy stream of the library (created on the first such call on
 *            a device) while batch s is computed, so with pinned memory the
 *            copies overlap the computation.
 *   stats    [host|device] steps*2 floats or NULL: (loss including the
 *            Eikonal term, mean |O - o|) of every step, evaluated at the
 *            parameters before that step's
 *            update.  If stats is host memory the call synchronises the
 *            stream before returning.
 *   workspace  at least efunc_workspace_bytes; with efunc_fit_workspace_bytes
 *            the sort of batch s+1 runs on a sort stream of the library
 *            alongside batch s (the copy and sort streams and their events
 *            are shared per device; fits called on one device from several
 *            host threads enqueue their steps one call at a time). */
efunc_status efunc_fit(const efunc_grid *grid, const efunc_adam *adam, int32_t loss, float eikonal_weight,
                       float *params, float *m, float *v, const float *qo, int64_t J, int32_t n_batches,
                       int32_t steps, int64_t step0, float *stats, void *workspace, size_t workspace_bytes,
                       efunc_stream_t stream);

/* efunc_fit replayed from a CUDA graph (Sec. 3.4 as efunc_fit; same
 * arguments and results).  The schedule of efunc_fit with the second sort
 * buffer repeats every P = lcm(2, n_batches) steps, apart from Adam's step
 * number; here that number and the bias corrections 1 - beta^t live in
 * device memory (in the workspace) and advance on the GPU, so the call
 * captures one period of P steps (sort of the next batch, key pack, fused
 * kernel, Adam) into a graph, launches it (steps - 1) / P times and issues
 * the remaining steps one by one.  It removes the per-step host launch cost,
 * which exceeds the GPU time for small batches (tens of thousands of
 * queries); for large batches it matches efunc_fit.
 *   qo, stats  [device] only (stats may be NULL; a host pointer returns
 *              EFUNC_ERR_ARG); n_batches in [1, 64]
 *   workspace  at least efunc_fit_workspace_bytes(grid, J)
 *   - The graph is built and destroyed inside the call (its instantiation
 *     costs about a few steps' host time).  The call itself must not be made
 *     while `stream` is being captured (EFUNC_ERR_ARG).
 *   - efunc_launch_count counts every kernel the replays run; the event
 *     profiler (efunc_profile_*) times only the steps issued one by one.
 *   - Bias corrections come from running products beta^t in FP64 instead
 *     of pow: they agree with efunc_fit's to FP64 rounding. */
efunc_status efunc_fit_graph(const efunc_grid *grid, const efunc_adam *adam, int32_t loss, float eikonal_weight,
                             float *params, float *m, float *v, const float *qo, int64_t J, int32_t n_batches,
                             int32_t steps, int64_t step0, float *stats, void *workspace, size_t workspace_bytes,
                             efunc_stream_t stream);

/* Forward without any device allocation by the caller.  The paper has no
 * counterpart: this entry point exists for callers that cannot allocate
 * device memory themselves, for example code running inside a host
 * framework that owns every device allocation through its own pool, or a
 * latency-critical caller that must not trigger the implicit device
 * synchronisation of cudaMalloc.  It computes exactly what efunc_forward
 * computes, with the same arguments minus the workspace: the scratch is a
 * fixed 32 MiB array inside this library (every GPU that loads the library
 * keeps it until the process exits).
 *   - Limit: requests whose efunc_eval_workspace_bytes(grid, J) exceeds
 *     32 MiB return EFUNC_ERR_WORKSPACE with nothing enqueued.  That admits
 *     up to 1,245,200 queries at R = 32, 1,372,896 at R = 16 and 435,648 at
 *     R = 64; larger requests need efunc_forward with a caller workspace.
 *   - The first call on a device looks up the array's device address (once
 *     per device, with that device current); make that first call before
 *     any stream capture.
 *   - It calls no cudaMalloc, cudaFree or other allocating routine.
 *   - All calls share the one array and it keeps the last call's contents;
 *     every call clears what it reads before use.  Calls that overlap on the
 *     GPU (other streams, other host threads) race on the array: serialise
 *     them. */
efunc_status efunc_forward_noalloc(const efunc_grid *grid, const float *params, const float *q, int64_t J,
                                   int32_t q_stride, float *O, float *lse, float *dOdq, efunc_stream_t stream);

/* Mean-shift offset initialisation (Sec. 3.3): writes, for every centre,
 *   Delta_i = sum_n exp(-bw |k_i - s_n|^2) s_n / sum_n exp(-bw |k_i - s_n|^2) - k_i
 * into params slots 0..2 (the other slots are left as they are), with the
 * largest exponent subtracted so that centres far from every point still get
 * a defined offset.  The paper uses bw = 100 and N = 16384 surface points.
 *   pts      [device] N x 3 floats, N in [1, 2^30] (N = 0 is EFUNC_ERR_ARG:
 *            the offset is undefined without points)
 *   params   [device] R^3*13 floats, slots 0..2 written
 *   bandwidth > 0 and finite */
efunc_status efunc_mean_shift_init(const efunc_grid *grid, const float *pts, int64_t N, float bandwidth,
                                   float *params, efunc_stream_t stream);

/* ------------------------------------------------------- ablation variants */

/* Floats per centre of a variant (the "Ch" column of Table tab:ablation:
 * G-1..G-4 1/4/10/20, G-5..G-8 2/5/11/21, Full-1/2 8, Full-3/4 13); -1 for
 * an invalid description. */
int32_t efunc_variant_channels(const efunc_variant *variant);

/* Workspace bytes of every variant call below for J queries (the fit sorts
 * the next batch into a second sort buffer on a library stream while the
 * current one is computed, and needs all of it; forward and backward need
 * less); 0 if the grid or the variant is invalid. */
size_t efunc_variant_workspace_bytes(const efunc_grid *grid, const efunc_variant *variant, int64_t J);

/* Forward of a variant (Algorithm 1 over the windowed keys of its key sets,
 * values of its degree): O and optionally lse per query, in the caller's
 * order.  Arguments as efunc_forward; params [device] R^3 x channels. */
efunc_status efunc_variant_forward(const efunc_grid *grid, const efunc_variant *variant, const float *params,
                                   const float *q, int64_t J, int32_t q_stride, float *O, float *lse,
                                   void *workspace, size_t workspace_bytes, efunc_stream_t stream);

/* Backward of a variant (Algorithm 2): ACCUMULATES sum_j gO_j dO_j/dparams
 * into grad [device, R^3 x channels].  dO/dphi = softmax * (Taylor factor) *
 * monomial; dO/db = softmax * beta * (-|q - key|^2 (f - O)) for learnable
 * scales; dO/dDelta = softmax * (2 beta (q - key)(f - O) - grad f) for
 * offset keys.  Grid keys are fixed. */
efunc_status efunc_variant_backward(const efunc_grid *grid, const efunc_variant *variant, const float *params,
                                    const float *q, int64_t J, int32_t q_stride, const float *gO, float *grad,
                                    void *workspace, size_t workspace_bytes, efunc_stream_t stream);

/* Fitting loop of a variant (Sec. 3.4), as efunc_fit without the Eikonal
 * term: per step sort, pack, fused forward + loss + backward, Adam on
 * R^3 x channels floats, with the sort of batch s+1 beside batch s (as
 * efunc_fit with efunc_fit_workspace_bytes).  qo and stats must be device
 * memory (a host pointer returns EFUNC_ERR_ARG); workspace_bytes at least
 * efunc_variant_workspace_bytes. */
efunc_status efunc_variant_fit(const efunc_grid *grid, const efunc_variant *variant, const efunc_adam *adam,
                               int32_t loss, float *params, float *m, float *v, const float *qo, int64_t J,
                               int32_t n_batches, int32_t steps, int64_t step0, float *stats, void *workspace,
                               size_t workspace_bytes, efunc_stream_t stream);

/* ------------------------------------------- cosine-series decomposition */

/* Function decomposition of Sec. 4.4 (Eq. o-as-value, Eq. cosine-series):
 *   S(q) = sum_{b=0}^{B-1} w_b(q) O_b(q),
 *   w_b(q) = cos(b pi q_x) cos(b pi q_y) cos(b pi q_z),
 * with every band O_b a Config-G-6 representation (fixed grid keys, first
 * order values, learnable log-scale: 5 floats per centre, (b, o, d_x, d_y,
 * d_z)).  The paper's 3-D weight "cos(b pi q)" is read as the separable
 * product, and its B bands as b = 0 .. B-1 (20480 B floats at 16^3; B = 1
 * is Config-G-6).  bands in [1, 16].
 *   params  [device] B x R^3 x 5 floats, band-major
 * Workspace: efunc_cosine_workspace_bytes (0 for an invalid grid, band count
 * or J; the fit needs all of it, forward and backward less). */
size_t efunc_cosine_workspace_bytes(const efunc_grid *grid, int32_t bands, int64_t J);

/* S at J queries (caller's order), arguments as efunc_forward. */
efunc_status efunc_cosine_forward(const efunc_grid *grid, int32_t bands, const float *params, const float *q,
                                  int64_t J, int32_t q_stride, float *S, void *workspace, size_t workspace_bytes,
                                  efunc_stream_t stream);

/* ACCUMULATES sum_j gS_j dS_j/dparams into grad [device, B x R^3 x 5]:
 * band b's backward (Algorithm 2) with upstream gS_j w_b(q_j). */
efunc_status efunc_cosine_backward(const efunc_grid *grid, int32_t bands, const float *params, const float *q,
                                   int64_t J, int32_t q_stride, const float *gS, float *grad, void *workspace,
                                   size_t workspace_bytes, efunc_stream_t stream);

/* Fitting loop of S (Sec. 4.4 optimises S as in Eq. loss), as
 * efunc_variant_fit (sort of the next batch beside the current one; device
 * batches and statistics only). */
efunc_status efunc_cosine_fit(const efunc_grid *grid, int32_t bands, const efunc_adam *adam, int32_t loss,
                              float *params, float *m, float *v, const float *qo, int64_t J, int32_t n_batches,
                              int32_t steps, int64_t step0, float *stats, void *workspace, size_t workspace_bytes,
                              efunc_stream_t stream);

/* ------------------------------------------------------------ batched fit */

/* Many shapes of uneven grid resolution and query count fitted together.
 * The paper fits one shape in about 20 minutes (Sec. 5, limitations); this
 * call fits S shapes at once, every step one launch of each kernel for all
 * of them: the cell sort of all shapes' queries (a shape's queries binned
 * on its own grid), the key pack of all grids, the fused forward + loss +
 * backward over the work items of every shape (an item's shape selects its
 * grid), per-shape loss statistics, and one Adam step over the concatenated
 * grids (Sec. 3.4 for each shape; one shared step count and learning rate).
 *
 * Shape s has an R_s^3 grid (13 floats per centre, layout of efunc_forward)
 * stored at float offset 13 * sum_{s' < s} R_s'^3 of params / m / v, and J_s
 * queries per batch; a batch holds the rows (x, y, z, target SDF) of every
 * shape in shape order, sum_s J_s rows.  S in [1, 1024], J_s >= 1,
 * sum_s J_s <= 2^30. */
typedef struct {
    int32_t R;           /* grid resolution, [1, 256] */
    float log_beta0;     /* log-scale of b = 0 (efunc_default_log_beta0(R) by default) */
    int64_t J;           /* queries per batch */
} efunc_shape;

/* Launch configuration of the batched fit, chosen by efunc_tune_batched:
 *   chunk        queries per work item at most, [32, 256]
 *   lanes2_max   work items of at most this many queries take 2 lanes per
 *   lanes4_max   query in the forward, of at most lanes4_max 4 lanes
 *                (lanes4_max <= lanes2_max <= 256)
 *   sort_blocks  blocks per SM of the sort's bin and scatter kernels, [1, 16]
 *   group_max    sparse cells: an aligned 2x2x2 block of window cells with at
 *                least two occupied cells and at most group_max queries is
 *                one work item (its 5x5x5 union window staged once, each key's
 *                gradient added once); 0 disables grouping, at most 256 */
typedef struct {
    int32_t chunk;
    int32_t lanes2_max;
    int32_t lanes4_max;
    int32_t sort_blocks;
    int32_t group_max;
} efunc_tuning;

/* The configuration used when none is given: {256, 64, 32, 8, 128}. */
void efunc_default_tuning(efunc_tuning *out);

/* Floats per array (params, m, v) of S shapes, sum 13 R_s^3; -1 if a shape
 * is invalid. */
int64_t efunc_batched_param_count(const efunc_shape *shapes, int32_t S);

/* Rows of one batch, sum J_s; -1 if a shape is invalid. */
int64_t efunc_batched_query_count(const efunc_shape *shapes, int32_t S);

/* Workspace bytes of efunc_fit_batched / efunc_eval_batched /
 * efunc_tune_batched for these shapes (any tuning); 0 if a shape is invalid. */
size_t efunc_batched_workspace_bytes(const efunc_shape *shapes, int32_t S);

/* Batched fitting loop: for it in [0, steps), batch (it mod n_batches) of
 * qo, the step above, with Adam step number step0 + it + 1.
 *   shapes   [host] S shape descriptions
 *   params, m, v  [device] efunc_batched_param_count floats each, updated
 *   qo       [device] n_batches * efunc_batched_query_count rows of 4 floats
 *   stats    [device] steps x S x 2 floats or NULL: (loss, MAE) of every
 *            shape at every step, at the parameters before the step
 *   tuning   [host] or NULL (efunc_default_tuning)
 *   graph    1: one period of n_batches steps is captured into a CUDA graph
 *            and replayed (steps / n_batches) times, the rest issued one by
 *            one (Adam's step number and the statistics row advance on the
 *            device); 0: every step issued one by one.  With graph = 1 the
 *            call must not be made while `stream` is being captured.
 * n_batches in [1, 64].  The shape table is copied from host memory to the
 * workspace at the start of the call (the call returns after that copy). */
efunc_status efunc_fit_batched(const efunc_shape *shapes, int32_t S, const efunc_adam *adam, int32_t loss,
                               float *params, float *m, float *v, const float *qo, int32_t n_batches, int32_t steps,
                               int64_t step0, float *stats, const efunc_tuning *tuning, int32_t graph,
                               void *workspace, size_t workspace_bytes, efunc_stream_t stream);

/* Per-shape loss of S shapes on one batch (efunc_eval_loss for each shape,
 * in one sort and one launch): out[2 s] = mean (O - o)^2 and
 * out[2 s + 1] = mean |O - o| over shape s's rows.
 *   qo  [device] efunc_batched_query_count rows of 4 floats
 *   out [device] 2 S floats */
efunc_status efunc_eval_batched(const efunc_shape *shapes, int32_t S, const float *params, const float *qo,
                                float *out, const efunc_tuning *tuning, void *workspace, size_t workspace_bytes,
                                efunc_stream_t stream);

/* Autotuner of the batched fit: times trial_steps steps of efunc_fit_batched
 * (after one untimed step) for each of 24 configurations (chunk 128 / 256,
 * lane thresholds 64 / 32 and 96 / 48, 4 / 8 sort blocks per SM, grouping
 * of sparse cells off / 64 / 128 queries) on these shapes and batches, with CUDA events on `stream`, and writes the
 * fastest to *best (and its milliseconds per step to *best_ms_per_step, or
 * NULL).  The trial steps are Adam steps with learning rate 0: params are
 * left as they are and m, v are zeroed at the end (tune before fitting).
 * Synchronises the stream.  trial_steps in [1, 1000]. */
efunc_status efunc_tune_batched(const efunc_shape *shapes, int32_t S, int32_t loss, float *params, float *m,
                                float *v, const float *qo, int32_t n_batches, int32_t trial_steps,
                                efunc_tuning *best, double *best_ms_per_step, void *workspace,
                                size_t workspace_bytes, efunc_stream_t stream);

/* ------------------------------------------------------ warm-start encoder */

/* A small BF16 3-D convolutional network that predicts a fit's starting
 * parameter grid from the shape's SDF sampled at the 32^3 cell centres (the
 * paper starts every fit from scratch, Sec. 3.4; it has no such encoder):
 *   L1 3x3x3 conv 1 -> 32 + ReLU, L2 3x3x3 conv 32 -> 64 + ReLU,
 *   L3 3x3x3 conv 64 -> 128 + ReLU, L4 1x1x1 conv 128 -> 13,
 * zero padding, BF16 activations, FP32 accumulation; L2-L4 and their
 * gradients run on the tensor cores (implicit GEMM, tcgen05).  It is
 * trained on (SDF grid, fitted parameter grid) pairs with the weighted MSE
 *   L = (1/V) sum_voxels sum_slots w_s (pred_s - target_s)^2
 * and its FP32 master weights are updated with efunc_adam_step.
 * Weights, one FP32 array of efunc_encoder_weight_count floats:
 *   W1 [32][27], b1 [32], W2 [64][27][32], b2 [64], W3 [128][27][64],
 *   b3 [128], W4 [13][128], b4 [13]
 * with W[co][tap][ci], tap = 9 (dx + 1) + 3 (dy + 1) + (dz + 1) the offset
 * of the input voxel read for an output voxel.
 * Volumes: sdf [device] batch x 32^3 floats, params / target [device]
 * batch x 32^3 x 13 floats, voxels in the order of the parameter grid
 * (x slowest).  batch in [1, 4096].  The kernels' waits are bounded; a wait
 * that runs out marks the workspace (efunc_encoder_status). */
int64_t efunc_encoder_weight_count(void);

/* Workspace bytes of the encoder calls for a batch (about 1.2 KB per voxel:
 * BF16 activations and their gradients); 0 for an invalid batch. */
size_t efunc_encoder_workspace_bytes(int32_t batch);

/* params = encoder(sdf). */
efunc_status efunc_encoder_forward(const float *weights, const float *sdf, int32_t batch, float *params,
                                   void *workspace, size_t workspace_bytes, efunc_stream_t stream);

/* One training step's forward and backward: grad [device,
 * efunc_encoder_weight_count floats] is written with dL/dweights, *loss
 * [device, 1 float] with L.  slot_weights [device] 13 floats or NULL (all 1). */
efunc_status efunc_encoder_train_step(const float *weights, const float *sdf, const float *target,
                                      const float *slot_weights, int32_t batch, float *grad, float *loss,
                                      void *workspace, size_t workspace_bytes, efunc_stream_t stream);

/* EFUNC_ERR_TIMEOUT if a wait inside an encoder kernel of the last call on
 * this workspace ran out (its outputs are then invalid), else EFUNC_OK.
 * Synchronises with the device. */
efunc_status efunc_encoder_status(const void *workspace);

/* The encoder's tensor-core convolution on its own (for tests): BF16
 * activations x [batch][32^3][cin] (cin a multiple of 64, at most 256),
 * weights w [cout][taps][cin] BF16 (taps 27 = 3x3x3 with zero padding, or
 * 1), cout in {16, 32, 64, 128}:
 *   out[v][co] = sum_{tap, ci} w[co][tap][ci] x[v + offset(tap)][ci]
 * then per mode: 0 bias + ReLU -> BF16 rows of out_ld; 1 bias -> FP32 rows
 * of out_ld, the first store_cols columns; 2 zeroed where mask (BF16 rows of
 * out_ld) is <= 0 -> BF16 (the gradient through the ReLU of the layer
 * below).  bias [device] cout floats or NULL.  err [device] int, set if a
 * wait ran out. */
efunc_status efunc_conv3d_bf16(const void *x, int32_t batch, int32_t cin, const void *w, int32_t cout, int32_t taps,
                               const float *bias, int32_t mode, const void *mask, void *out, int32_t out_ld,
                               int32_t store_cols, int32_t *err, efunc_stream_t stream);

/* Its weight gradient: dw [cout][taps][cin] FP32 += sum_v dy[v][co]
 * x[v + offset(tap)][ci], dy [batch][32^3][dy_ld] BF16 (dy_ld 64 or 128,
 * cout <= dy_ld), FP32 atomics. */
efunc_status efunc_conv3d_wgrad_bf16(const void *dy, int32_t dy_ld, int32_t cout, const void *x, int32_t cin,
                                     int32_t batch, int32_t taps, float *dw, int32_t *err, efunc_stream_t stream);

/* ---------------------------------------------------- checkpoint / resume */

/* A fit's state is its parameter grid, Adam's two moments and the number of
 * steps taken (the representation is its own checkpoint: 13 R^3 floats,
 * Sec. 3.1); with the configuration below, a later efunc_fit with
 * step0 = step continues the same trajectory (up to the order of the FP32
 * gradient atomics).  The file is flat and little-endian: a 128-byte header
 * (magic "EFUNCCKP", format version 1, these fields, an FNV-1a 64 checksum of
 * the header), params, m, v as n floats each, and an FNV-1a 64 checksum of
 * those 12 n bytes.  Host code only: the arrays are HOST memory. */
typedef struct {
    int32_t R;          /* grid resolution */
    int32_t W;          /* window half-width */
    float log_beta0;
    int32_t channels;   /* floats per centre: 13, efunc_variant_channels, or 5 B for B cosine bands */
    int64_t n;          /* floats per array: R^3 * channels */
    int64_t step;       /* Adam steps taken */
    uint64_t seed;      /* the caller's sampling seed, stored as given */
    int32_t loss;       /* efunc_loss */
    efunc_adam adam;
} efunc_checkpoint_info;

/* Writes params, m, v ([host], info->n floats each) and info to path, through
 * a temporary file renamed over path once complete (an interrupted save
 * leaves the previous file).  EFUNC_ERR_ARG for an inconsistent info
 * (n != R^3 * channels, step < 0, ...), EFUNC_ERR_IO if the file cannot be
 * written. */
efunc_status efunc_checkpoint_save(const char *path, const efunc_checkpoint_info *info, const float *params,
                                   const float *m, const float *v);

/* Reads and checks the header only (to size the arrays of a load).
 * EFUNC_ERR_IO if the file is missing or its header is not a valid
 * version-1 header (magic, sizes, checksum). */
efunc_status efunc_checkpoint_info_read(const char *path, efunc_checkpoint_info *info);

/* Reads a checkpoint into params, m, v ([host], capacity floats each) and
 * info.  EFUNC_ERR_ARG if capacity < n; EFUNC_ERR_IO if the file is
 * missing, short, longer than its contents, or a checksum does not match
 * (the arrays' contents are then unspecified and info is not written). */
efunc_status efunc_checkpoint_load(const char *path, efunc_checkpoint_info *info, float *params, float *m, float *v,
                                   int64_t capacity);

/* ------------------------------------------------------------ measurement */

/* When enabled, every kernel launch of the library is bracketed by CUDA
 * events recorded on its launch stream.  Events are created lazily (this is
 * the one place the library asks the runtime for resources). */
void efunc_profile_enable(int32_t enable);

/* Waits for the recorded events and folds them into per-kernel totals.
 * Writes the total milliseconds and launch count of kernel `name` (one of
 * "bin", "scan_reduce", "scan_top", "scan_emit", "scatter", "pack_keys",
 * "forward", "fused_backward", "fused_fit", "adam", "mean_shift", "variant_pack",
 * "variant_forward", "variant_backward", "variant_fit", "cosine_pack",
 * "cosine_forward", "cosine_backward", "cosine_fit", "eval" (the fused
 * kernel of efunc_eval_loss and efunc_eval_batched), "eval_finish" (the
 * one-thread kernel that turns their sums into means), "f64" (every kernel
 * of the FP64 calls), "batched" (the batched fit's fused kernel),
 * "batched_stats" (its per-shape statistics), "enc_conv" / "enc_wgrad" (the
 * encoder's tensor-core convolutions and weight gradients), "enc_aux" (its
 * other kernels) or "grouped" (the grouped-item kernel)).  Returns 0 on
 * success, -1 for an unknown name or a CUDA error. */
int32_t efunc_profile_read(const char *name, double *total_ms, int64_t *launches);

/* Clears the per-kernel totals (pending events are discarded). */
void efunc_profile_reset(void);

/* Kernels launched by this library since it was loaded. */
int64_t efunc_launch_count(void);

/* Bounds-check build (the sources compiled with -DEFUNC_DEBUG_BOUNDS into
 * lib/libefunc_debug.so): the kernels test the indices of their hot gathers
 * and scatters - staged key records and gradient rows inside the grid, each
 * staged query inside its work item's cell or octet, paired-row slots
 * inside their buffer, the sort's bins and sorted positions - and on a
 * failing test record its code in a device flag and skip the access (no
 * trap, no abort).  Waits for the current device, writes the first code
 * recorded there since the last call to *code (0: none; 1 staged key outside
 * the grid, 2 staged query outside its item's cell, 3 union key outside the
 * grid, 4 staged query outside its octet, 5 paired-row slot past its buffer,
 * 6 bin past the bin count, 7 sorted position past J, 8 work item with a bad
 * range) and clears it.  The normal build writes 0 and returns
 * EFUNC_ERR_UNSUPPORTED; code NULL is EFUNC_ERR_ARG. */
efunc_status efunc_debug_bounds(int32_t *code);

/* The cudaError_t of the CUDA call behind the calling thread's most recent
 * EFUNC_ERR_CUDA (0 before any).  The library clears the runtime's pending
 * error when it reports one, so a failure never resurfaces in a later call. */
int32_t efunc_last_cuda_error(void);

/* Name of a cudaError_t value ("cudaErrorInvalidValue", ...); a static
 * string owned by the CUDA runtime. */
const char *efunc_cuda_error_name(int32_t code);

#ifdef __cplusplus
}
#endif

#endif /* EFUNC_H */
