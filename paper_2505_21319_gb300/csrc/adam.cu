// Adam / AdamW step over the parameter grid (hot-path step a5; Sec. 3.4,
// Sec. 4.2), torch.optim semantics:
//   g' = g + wd*p (Adam) | p *= 1 - lr*wd (AdamW)
//   m = b1 m + (1-b1) g';  v = b2 v + (1-b2) g'^2
//   p -= (lr / (1 - b1^t)) * m / (sqrt(v) / sqrt(1 - b2^t) + eps)
// and the gradient is zeroed for the next accumulation.  Memory-bound: 16
// bytes read and 16 bytes written per parameter, float4-vectorised.
#include <math.h>

#include "adam_clock.cuh"

namespace efunc {

namespace {

__device__ __forceinline__ void adam_one(const AdamArgs &a, float &p, float &g, float &m, float &v)
{
    float gi = g;
    if (a.decoupled) p *= a.decay;
    else gi = fmaf(a.wd, p, gi);
    m = fmaf(a.beta1, m, a.one_minus_beta1 * gi);
    v = fmaf(a.beta2, v, a.one_minus_beta2 * gi * gi);
    const float denom = sqrtf(v) * a.inv_sqrt_bc2 + a.eps;
    p -= a.step_size * m / denom;
    g = 0.0f;
}

// The update over all n parameters: float4 rows when every array is 16-byte
// aligned, then the scalar tail.
template <bool VEC>
__device__ __forceinline__ void adam_all(const AdamArgs &a)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t tail = 0;
    if (VEC) {
        const int64_t n4 = a.n >> 2;
        float4 *p4 = reinterpret_cast<float4 *>(a.p), *g4 = reinterpret_cast<float4 *>(a.g);
        float4 *m4 = reinterpret_cast<float4 *>(a.m), *v4 = reinterpret_cast<float4 *>(a.v);
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
            float4 p = p4[i], g = g4[i], m = m4[i], v = v4[i];
            adam_one(a, p.x, g.x, m.x, v.x);
            adam_one(a, p.y, g.y, m.y, v.y);
            adam_one(a, p.z, g.z, m.z, v.z);
            adam_one(a, p.w, g.w, m.w, v.w);
            p4[i] = p; g4[i] = g; m4[i] = m; v4[i] = v;
        }
        tail = n4 << 2;
    }
    for (int64_t i = tail + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride)
        adam_one(a, a.p[i], a.g[i], a.m[i], a.v[i]);
}

__device__ __forceinline__ void write_stats(const AdamArgs &a, float *dst)
{
    dst[0] = (float)(a.ctrl->loss_sum * (double)a.inv_J);
    dst[1] = (float)(a.ctrl->abs_sum * (double)a.inv_J);
}

__global__ void __launch_bounds__(256) adam_kernel_vec(AdamArgs a)
{
    adam_all<true>(a);
    if (a.stats && blockIdx.x == 0 && threadIdx.x == 0) write_stats(a, a.stats);
}

__global__ void __launch_bounds__(256) adam_kernel_scalar(AdamArgs a)
{
    adam_all<false>(a);
    if (a.stats && blockIdx.x == 0 && threadIdx.x == 0) write_stats(a, a.stats);
}

template <bool VEC>
__global__ void __launch_bounds__(256) adam_kernel_clocked(AdamArgs a, AdamClock *clk)
{
    // every block reads step t's constants before it counts itself done, and
    // the clock advances only after the last block has counted itself
    AdamArgs b = a;
    b.step_size = clk->step_size;
    b.inv_sqrt_bc2 = clk->inv_sqrt_bc2;
    const int64_t row = clk->t - clk->t_first;
    adam_all<VEC>(b);
    if (a.stats && blockIdx.x == 0 && threadIdx.x == 0) write_stats(a, a.stats + 2 * row);
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&clk->done, 1u) == gridDim.x - 1) {
            const double b1t = clk->b1t * clk->beta1, b2t = clk->b2t * clk->beta2;
            clk->t += 1;
            clk->b1t = b1t;
            clk->b2t = b2t;
            clk->step_size = (float)(clk->lr / (1.0 - b1t));
            clk->inv_sqrt_bc2 = (float)(1.0 / sqrt(1.0 - b2t));
            clk->done = 0;
        }
    }
}

__global__ void adam_clock_seed_kernel(AdamClock *clk, AdamClock init) { *clk = init; }

int adam_blocks(const AdamArgs &a, bool &vec)
{
    const int sms = device_sm_count();
    const uintptr_t mis = reinterpret_cast<uintptr_t>(a.p) | reinterpret_cast<uintptr_t>(a.g) |
                          reinterpret_cast<uintptr_t>(a.m) | reinterpret_cast<uintptr_t>(a.v);
    vec = (mis & 15u) == 0;
    const int64_t work = vec ? (a.n + 3) / 4 : a.n;
    int64_t blocks = (work + 255) / 256;
    if (blocks > (int64_t)sms * 8) blocks = (int64_t)sms * 8;
    if (blocks < 1) blocks = 1;
    return (int)blocks;
}

}  // namespace

AdamClock adam_clock_init(double lr, double beta1, double beta2, int64_t t_first)
{
    AdamClock c{};
    c.t = t_first;
    c.t_first = t_first;
    c.beta1 = beta1;
    c.beta2 = beta2;
    c.lr = lr;
    c.b1t = pow(beta1, (double)t_first);
    c.b2t = pow(beta2, (double)t_first);
    c.step_size = (float)(lr / (1.0 - c.b1t));
    c.inv_sqrt_bc2 = (float)(1.0 / sqrt(1.0 - c.b2t));
    c.done = 0;
    return c;
}

cudaError_t launch_adam_clock_seed(AdamClock *clk, const AdamClock &init, cudaStream_t s)
{
    launch_begin(K_ADAM, s);
    adam_clock_seed_kernel<<<1, 1, 0, s>>>(clk, init);
    launch_end(K_ADAM, s);
    return cudaGetLastError();
}

cudaError_t launch_adam_clocked(const AdamArgs &a, AdamClock *clk, cudaStream_t s)
{
    bool vec = false;
    const int blocks = adam_blocks(a, vec);
    launch_begin(K_ADAM, s);
    if (vec) adam_kernel_clocked<true><<<(unsigned)blocks, 256, 0, s>>>(a, clk);
    else adam_kernel_clocked<false><<<(unsigned)blocks, 256, 0, s>>>(a, clk);
    launch_end(K_ADAM, s);
    return cudaGetLastError();
}

cudaError_t launch_adam(const AdamArgs &a, cudaStream_t s)
{
    bool vec = false;
    const int blocks = adam_blocks(a, vec);
    launch_begin(K_ADAM, s);
    if (vec) adam_kernel_vec<<<(unsigned)blocks, 256, 0, s>>>(a);
    else adam_kernel_scalar<<<(unsigned)blocks, 256, 0, s>>>(a);
    launch_end(K_ADAM, s);
    return cudaGetLastError();
}

}  // namespace efunc
