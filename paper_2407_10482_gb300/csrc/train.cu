// train.cu -- the rest of a training step around the render's reverse pass:
// photometric L2 loss with its gradient, and a fused Adam update (Sec. S2.4 uses
// Adam with beta = (0.9, 0.99), eps = 1e-8).  Both are streaming kernels over
// contiguous arrays (grid-stride loops, float4 where the length allows).
#include "common.cuh"

namespace ngprt {
namespace {

__global__ void l2_loss_kernel(const float* __restrict__ rgb, const float* __restrict__ target, int64_t n,
                               float scale, float* __restrict__ loss, float* __restrict__ d_rgb) {
    float acc = 0.0f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float e = rgb[i] - target[i];
        acc = fmaf(e, e, acc);
        if (d_rgb) d_rgb[i] = 2.0f * scale * e;
    }
    __shared__ float red[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        float v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0 && loss) atomicAdd(loss, scale * v);
    }
}

// Huber loss of Sec. S2.4 (L_color): h(e) = e^2 / 2 for |e| <= delta, else
// delta (|e| - delta / 2); h'(e) = e, or delta sign(e).
__global__ void huber_loss_kernel(const float* __restrict__ rgb, const float* __restrict__ target, int64_t n,
                                  float delta, float scale, float* __restrict__ loss, float* __restrict__ d_rgb) {
    float acc = 0.0f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float e = rgb[i] - target[i];
        const float a = fabsf(e);
        const bool quad = a <= delta;
        acc += quad ? 0.5f * e * e : delta * (a - 0.5f * delta);
        if (d_rgb) d_rgb[i] = scale * (quad ? e : copysignf(delta, e));
    }
    __shared__ float red[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        float v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0 && loss) atomicAdd(loss, scale * v);
    }
}

// Mean of the per-ray sample counts (second int of each ray_stats pair) into *out.
__global__ void mean_samples_kernel(const int2* __restrict__ stats, int64_t n, float* __restrict__ out) {
    unsigned long long acc = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc += (unsigned long long)stats[i].y;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd(out, (float)((double)acc / (double)n));
}

// Count of the values that are NaN or infinite (the guard after fault injection).
__global__ void nonfinite_kernel(const float* __restrict__ x, int64_t n, int32_t* __restrict__ count) {
    int c = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        c += isfinite(x[i]) ? 0 : 1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

__global__ void adam_kernel(float* __restrict__ p, float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float c1,
                            float c2, int zero_grad) {
    const int64_t n4 = n / 4;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
        float4 pp = reinterpret_cast<float4*>(p)[i], gg = reinterpret_cast<float4*>(g)[i];
        float4 mm = reinterpret_cast<float4*>(m)[i], vv = reinterpret_cast<float4*>(v)[i];
        float* pa = &pp.x; float* ga = &gg.x; float* ma = &mm.x; float* va = &vv.x;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            ma[k] = b1 * ma[k] + (1.0f - b1) * ga[k];
            va[k] = b2 * va[k] + (1.0f - b2) * ga[k] * ga[k];
            pa[k] -= lr * (ma[k] / c1) / (sqrtf(va[k] / c2) + eps);
        }
        reinterpret_cast<float4*>(p)[i] = pp;
        reinterpret_cast<float4*>(m)[i] = mm;
        reinterpret_cast<float4*>(v)[i] = vv;
        if (zero_grad) reinterpret_cast<float4*>(g)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    for (int64_t i = n4 * 4 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        m[i] = b1 * m[i] + (1.0f - b1) * g[i];
        v[i] = b2 * v[i] + (1.0f - b2) * g[i] * g[i];
        p[i] -= lr * (m[i] / c1) / (sqrtf(v[i] / c2) + eps);
        if (zero_grad) g[i] = 0.0f;
    }
}

unsigned grid_for(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    const int64_t cap = 152 * 16;
    return (unsigned)(b < 1 ? 1 : (b > cap ? cap : b));
}

}  // namespace
}  // namespace ngprt

using namespace ngprt;

extern "C" int32_t ngprt_l2_loss(const float* rgb, const float* target, int64_t n, float scale, float* loss,
                                 float* d_rgb, void* stream) {
    const char* fn = "ngprt_l2_loss";
    NGPRT_REQUIRE(n >= 0, "%s: n=%lld", fn, (long long)n);
    if (n == 0) return NGPRT_OK;
    NGPRT_REQUIRE(rgb && target && (loss || d_rgb), "%s: NULL buffer", fn);
    l2_loss_kernel<<<grid_for(n, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(rgb, target, n, scale, loss, d_rgb);
    return cuda_status(fn);
}

extern "C" int32_t ngprt_adam_step(float* param, float* grad, float* m, float* v, int64_t n, float lr, float beta1,
                                   float beta2, float eps, int32_t step, int32_t zero_grad, void* stream) {
    const char* fn = "ngprt_adam_step";
    NGPRT_REQUIRE(n >= 0 && step >= 1, "%s: n=%lld step=%d", fn, (long long)n, step);
    if (n == 0) return NGPRT_OK;
    NGPRT_REQUIRE(param && grad && m && v, "%s: NULL buffer", fn);
    NGPRT_REQUIRE((((uintptr_t)param | (uintptr_t)grad | (uintptr_t)m | (uintptr_t)v) & 15) == 0,
                  "%s: buffers must be 16-byte aligned", fn);
    const float c1 = (float)(1.0 - pow((double)beta1, step)), c2 = (float)(1.0 - pow((double)beta2, step));
    adam_kernel<<<grid_for(n / 4 + 1, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(param, grad, m, v, n, lr,
                                                                                        beta1, beta2, eps, c1, c2,
                                                                                        zero_grad);
    return cuda_status(fn);
}

extern "C" int32_t ngprt_huber_loss(const float* rgb, const float* target, int64_t n, float delta, float scale,
                                    float* loss, float* d_rgb, void* stream) {
    const char* fn = "ngprt_huber_loss";
    NGPRT_REQUIRE(n >= 0, "%s: n=%lld", fn, (long long)n);
    NGPRT_REQUIRE(delta > 0.0f, "%s: delta=%g must be > 0", fn, (double)delta);
    if (n == 0) return NGPRT_OK;
    NGPRT_REQUIRE(rgb && target && (loss || d_rgb), "%s: NULL buffer", fn);
    huber_loss_kernel<<<grid_for(n, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(rgb, target, n, delta, scale,
                                                                                      loss, d_rgb);
    return cuda_status(fn);
}

extern "C" int32_t ngprt_mean_samples(const int32_t* ray_stats, int64_t n_rays, float* out, void* stream) {
    const char* fn = "ngprt_mean_samples";
    NGPRT_REQUIRE(n_rays >= 0 && out != nullptr, "%s: bad arguments", fn);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(out, 0, sizeof(float), st) != cudaSuccess) return cuda_status(fn);
    if (n_rays == 0) return cuda_status(fn);
    NGPRT_REQUIRE(ray_stats != nullptr && ((uintptr_t)ray_stats & 7) == 0, "%s: ray_stats must be 8-byte aligned", fn);
    mean_samples_kernel<<<grid_for(n_rays, 256), 256, 0, st>>>(reinterpret_cast<const int2*>(ray_stats), n_rays, out);
    return cuda_status(fn);
}

extern "C" float ngprt_step_autotune(float gamma, float n_mean, float n_min, float kappa, float gamma_min) {
    // Eq. S3: grow gamma by (1 + kappa) up to 1 while the batch keeps n_min samples
    // per ray on average, else shrink it by (1 - kappa) down to gamma_min
    if (n_mean >= n_min) return fminf(1.0f, (1.0f + kappa) * gamma);
    return fmaxf(gamma_min, (1.0f - kappa) * gamma);
}

extern "C" int32_t ngprt_count_nonfinite(const float* x, int64_t n, int32_t* count, void* stream) {
    const char* fn = "ngprt_count_nonfinite";
    NGPRT_REQUIRE(n >= 0 && count != nullptr && (n == 0 || x != nullptr), "%s: bad arguments", fn);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(count, 0, sizeof(int32_t), st) != cudaSuccess) return cuda_status(fn);
    if (n > 0) nonfinite_kernel<<<grid_for(n, 256), 256, 0, st>>>(x, n, count);
    return cuda_status(fn);
}
