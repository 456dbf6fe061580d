// Adam / AdamW step over the parameter grid (hot-path step a5; Sec. 3.4,
// Sec. 4.2), torch.optim semantics:
//   g' = g + wd*p (Adam) | p *= 1 - lr*wd (AdamW)
//   m = b1 m + (1-b1) g';  v = b2 v + (1-b2) g'^2
//   p -= (lr / (1 - b1^t)) * m / (sqrt(v) / sqrt(1 - b2^t) + eps)
// and the gradient is zeroed for the next accumulation.  Memory-bound: 16
// bytes read and 16 bytes written per parameter, float4-vectorised.
#include "common.cuh"

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

__global__ void __launch_bounds__(256) adam_kernel_vec(AdamArgs a)
{
    const int64_t n4 = a.n >> 2;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
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
    // scalar tail
    for (int64_t i = (n4 << 2) + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride)
        adam_one(a, a.p[i], a.g[i], a.m[i], a.v[i]);
    if (a.stats && blockIdx.x == 0 && threadIdx.x == 0) {
        a.stats[0] = (float)(a.ctrl->loss_sum * (double)a.inv_J);
        a.stats[1] = (float)(a.ctrl->abs_sum * (double)a.inv_J);
    }
}

__global__ void __launch_bounds__(256) adam_kernel_scalar(AdamArgs a)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride)
        adam_one(a, a.p[i], a.g[i], a.m[i], a.v[i]);
    if (a.stats && blockIdx.x == 0 && threadIdx.x == 0) {
        a.stats[0] = (float)(a.ctrl->loss_sum * (double)a.inv_J);
        a.stats[1] = (float)(a.ctrl->abs_sum * (double)a.inv_J);
    }
}

}  // namespace

cudaError_t launch_adam(const AdamArgs &a, cudaStream_t s)
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    const uintptr_t mis = reinterpret_cast<uintptr_t>(a.p) | reinterpret_cast<uintptr_t>(a.g) |
                          reinterpret_cast<uintptr_t>(a.m) | reinterpret_cast<uintptr_t>(a.v);
    const bool vec = (mis & 15u) == 0;
    const int64_t work = vec ? (a.n + 3) / 4 : a.n;
    int64_t blocks = (work + 255) / 256;
    if (blocks > (int64_t)sms * 8) blocks = (int64_t)sms * 8;
    if (blocks < 1) blocks = 1;
    launch_begin(K_ADAM, s);
    if (vec) adam_kernel_vec<<<(unsigned)blocks, 256, 0, s>>>(a);
    else adam_kernel_scalar<<<(unsigned)blocks, 256, 0, s>>>(a);
    launch_end(K_ADAM, s);
    return cudaGetLastError();
}

}  // namespace efunc
