// propose.cu -- learned per-ray proposal: a small MLP on (o / in_scale, d) that
// predicts the interval [t_near, t_far] holding the ray's significant weights and
// its opacity A^.  Not in the paper (Sec. 2 calls adaptive sampling orthogonal to
// NGP-RT); the renderer marches only inside the interval, and a fallback pass
// re-marches rays whose interval missed more than 1% of the predicted opacity.
//   h1 = relu(W0 e + b0), h2 = relu(W1 h1 + b1), z = W2 h2 + b2,
//   t_near = t_scale sigmoid(z0), t_far = t_scale sigmoid(z1), A^ = sigmoid(z2)
// Parameters, flat float: W0 [32][6], b0 [32], W1 [32][32], b1 [32], W2 [3][32], b2 [3].
#include "march.cuh"

namespace ngprt {
namespace {

constexpr int kPW = 32;
constexpr int kPIn = 6;
constexpr int kPParams = kPW * kPIn + kPW + kPW * kPW + kPW + 3 * kPW + 3;

struct PropParams {
    MarchParams m;  // ray source only
    const float* w;
    const __half* w16;  // propose with FP16 weights (widened to FP32 in shared memory)
    float in_scale, t_scale, margin_near, margin_far, a_min;
    float* interval;
    float* a_hat;
    const float* targets;
    float* g_w;
    float* loss;
};

__device__ __forceinline__ float psig(float x) { return 1.0f / (1.0f + expf(-x)); }

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// e = (o / in_scale, d / |d|) of this thread's ray; false when the lane has none.
__device__ __forceinline__ bool prop_input(const PropParams& p, int64_t& ray, float e[kPIn]) {
    float o[3], d[3];
    df dd[3];
    if (!thread_ray(p.m, ray, o, dd)) return false;
#pragma unroll
    for (int a = 0; a < 3; ++a) d[a] = df_float(dd[a]);
    const float n = sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        e[a] = o[a] / p.in_scale;
        e[3 + a] = d[a] / n;
    }
    return true;
}

__device__ __forceinline__ void prop_mlp(const float* w, const float e[kPIn], float a1[kPW], float a2[kPW],
                                         float z[3]) {
    const float *W0 = w, *b0 = W0 + kPW * kPIn, *W1 = b0 + kPW, *b1 = W1 + kPW * kPW, *W2 = b1 + kPW, *b2 = W2 + 3 * kPW;
#pragma unroll
    for (int o = 0; o < kPW; ++o) {
        float a = b0[o];
#pragma unroll
        for (int k = 0; k < kPIn; ++k) a = fmaf(W0[o * kPIn + k], e[k], a);
        a1[o] = a;
    }
#pragma unroll 4
    for (int o = 0; o < kPW; ++o) {
        float a = b1[o];
#pragma unroll
        for (int k = 0; k < kPW; ++k) a = fmaf(W1[o * kPW + k], fmaxf(a1[k], 0.0f), a);
        a2[o] = a;
    }
#pragma unroll
    for (int o = 0; o < 3; ++o) {
        float a = b2[o];
#pragma unroll
        for (int k = 0; k < kPW; ++k) a = fmaf(W2[o * kPW + k], fmaxf(a2[k], 0.0f), a);
        z[o] = a;
    }
}

__global__ void __launch_bounds__(128) propose_kernel(const __grid_constant__ PropParams p) {
    __shared__ float ws[kPParams];
    for (int i = threadIdx.x; i < kPParams; i += blockDim.x) ws[i] = p.w16 ? __half2float(p.w16[i]) : p.w[i];
    __syncthreads();
    int64_t ray;
    float e[kPIn];
    if (!prop_input(p, ray, e)) return;
    float a1[kPW], a2[kPW], z[3];
    prop_mlp(ws, e, a1, a2, z);
    const float tn = p.t_scale * psig(z[0]), tf = p.t_scale * psig(z[1]), ah = psig(z[2]);
    float lo, hi;
    if (ah < p.a_min) {
        lo = INFINITY;   // predicted empty: march nothing
        hi = -INFINITY;
    } else if (!(tf > tn)) {
        lo = -INFINITY;  // no usable interval: march the whole ray
        hi = INFINITY;
    } else {
        lo = tn - p.margin_near;
        hi = tf + p.margin_far;  // +inf: no far clip (termination ends the ray)
    }
    p.interval[2 * ray] = lo;
    p.interval[2 * ray + 1] = hi;
    if (p.a_hat) p.a_hat[ray] = ah;
}

__device__ __forceinline__ float sl1_grad(float x, float beta) {
    const float ax = fabsf(x);
    return ax < beta ? x / beta : (x > 0.0f ? 1.0f : -1.0f);
}

__device__ __forceinline__ float sl1(float x, float beta) {
    const float ax = fabsf(x);
    return ax < beta ? 0.5f * x * x / beta : ax - 0.5f * beta;
}

// Loss and gradient, mean over n rays; weight gradients are reduced per warp
// (shuffles), per block (shared memory) and added to g_w once per block.
__global__ void __launch_bounds__(128) propose_backward_kernel(const __grid_constant__ PropParams p) {
    __shared__ float ws[kPParams];
    __shared__ float gws[kPParams];
    for (int i = threadIdx.x; i < kPParams; i += blockDim.x) {
        ws[i] = p.w[i];
        gws[i] = 0.0f;
    }
    __syncthreads();
    int64_t ray = 0;
    float e[kPIn];
    const bool active = prop_input(p, ray, e);
    if (!active)
        for (int k = 0; k < kPIn; ++k) e[k] = 0.0f;
    float a1[kPW], a2[kPW], z[3];
    prop_mlp(ws, e, a1, a2, z);
    const float inv_n = 1.0f / (float)p.m.n_rays;
    const float beta = 0.01f;
    float gz[3] = {0.0f, 0.0f, 0.0f}, L = 0.0f;
    if (active) {
        const float t0 = p.targets[3 * ray], t1 = p.targets[3 * ray + 1], A = p.targets[3 * ray + 2];
        const float s0 = psig(z[0]), s1 = psig(z[1]), s2 = psig(z[2]);
        const float x0 = (p.t_scale * s0 - t0) / p.t_scale, x1 = (p.t_scale * s1 - t1) / p.t_scale;
        // conservative intervals: a late t_near or an early t_far costs 4x
        const float a0 = x0 > 0.0f ? 4.0f : 1.0f, a1 = x1 < 0.0f ? 4.0f : 1.0f;
        L = inv_n * (A * (a0 * sl1(x0, beta) + a1 * sl1(x1, beta)) + (s2 - A) * (s2 - A));
        gz[0] = inv_n * A * a0 * sl1_grad(x0, beta) * s0 * (1.0f - s0);
        gz[1] = inv_n * A * a1 * sl1_grad(x1, beta) * s1 * (1.0f - s1);
        gz[2] = inv_n * 2.0f * (s2 - A) * s2 * (1.0f - s2);
    }
    const int lane = threadIdx.x & 31;
    const float *W1 = ws + kPW * kPIn + kPW, *W2 = W1 + kPW * kPW + kPW;
    float *gW0 = gws, *gb0 = gW0 + kPW * kPIn, *gW1 = gb0 + kPW, *gb1 = gW1 + kPW * kPW, *gW2 = gb1 + kPW,
          *gb2 = gW2 + 3 * kPW;
    float ga2[kPW];
#pragma unroll
    for (int k = 0; k < kPW; ++k) {
        const float h = fmaxf(a2[k], 0.0f);
        float g = 0.0f;
#pragma unroll
        for (int o = 0; o < 3; ++o) {
            const float s = warp_sum(gz[o] * h);
            if (lane == 0) atomicAdd(&gW2[o * kPW + k], s);
            g = fmaf(W2[o * kPW + k], gz[o], g);
        }
        ga2[k] = a2[k] > 0.0f ? g : 0.0f;
    }
#pragma unroll
    for (int o = 0; o < 3; ++o) {
        const float s = warp_sum(gz[o]);
        if (lane == 0) atomicAdd(&gb2[o], s);
    }
    float ga1[kPW];
#pragma unroll
    for (int k = 0; k < kPW; ++k) ga1[k] = 0.0f;
#pragma unroll 2
    for (int o = 0; o < kPW; ++o) {
        const float sb = warp_sum(ga2[o]);
        if (lane == 0) atomicAdd(&gb1[o], sb);
#pragma unroll
        for (int k = 0; k < kPW; ++k) {
            const float s = warp_sum(ga2[o] * fmaxf(a1[k], 0.0f));
            if (lane == 0) atomicAdd(&gW1[o * kPW + k], s);
            ga1[k] = fmaf(W1[o * kPW + k], ga2[o], ga1[k]);
        }
    }
#pragma unroll
    for (int o = 0; o < kPW; ++o) {
        const float g = a1[o] > 0.0f ? ga1[o] : 0.0f;
        const float sb = warp_sum(g);
        if (lane == 0) atomicAdd(&gb0[o], sb);
#pragma unroll
        for (int k = 0; k < kPIn; ++k) {
            const float s = warp_sum(g * e[k]);
            if (lane == 0) atomicAdd(&gW0[o * kPIn + k], s);
        }
    }
    const float ls = warp_sum(L);
    if (lane == 0 && p.loss) atomicAdd(p.loss, ls);
    __syncthreads();
    for (int i = threadIdx.x; i < kPParams; i += blockDim.x) {
        const float v = gws[i];
        if (v != 0.0f) atomicAdd(&p.g_w[i], v);
    }
}

}  // namespace

int32_t setup_rays(MarchParams& p, const ngprt_camera* cams, int32_t n_cams, const int32_t* pixel_ids,
                   const float* rays_o, const float* rays_d, int64_t n_rays, dim3& grid, const char* fn);

}  // namespace ngprt

using namespace ngprt;

extern "C" int32_t ngprt_proposal_param_count(void) { return kPParams; }

extern "C" int32_t ngprt_propose(const void* prop_w, int32_t prop_dtype, const ngprt_camera* cams, int32_t n_cams,
                                 const int32_t* pixel_ids, const float* rays_o, const float* rays_d, int64_t n_rays,
                                 float in_scale, float t_scale, float margin_near, float margin_far, float a_min,
                                 float* t_interval_out, float* a_hat_out, void* stream) {
    const char* fn = "ngprt_propose";
    PropParams p;
    memset(&p, 0, sizeof p);
    NGPRT_REQUIRE(prop_w != nullptr, "%s: prop_w is NULL", fn);
    NGPRT_REQUIRE(prop_dtype == NGPRT_F32 || prop_dtype == NGPRT_F16, "%s: prop_dtype=%d (F32 or F16)", fn,
                  prop_dtype);
    NGPRT_REQUIRE(n_rays >= 0 && in_scale > 0.0f && t_scale > 0.0f && margin_near >= 0.0f && margin_far >= 0.0f,
                  "%s: bad scalar argument", fn);
    dim3 grid;
    int32_t rc;
    if ((rc = setup_rays(p.m, cams, n_cams, pixel_ids, rays_o, rays_d, n_rays, grid, fn)) != NGPRT_OK) return rc;
    if (n_rays == 0) return NGPRT_OK;
    NGPRT_REQUIRE(t_interval_out != nullptr, "%s: t_interval_out is NULL", fn);
    p.w = prop_dtype == NGPRT_F32 ? static_cast<const float*>(prop_w) : nullptr;
    p.w16 = prop_dtype == NGPRT_F16 ? static_cast<const __half*>(prop_w) : nullptr;
    p.in_scale = in_scale;
    p.t_scale = t_scale;
    p.margin_near = margin_near;
    p.margin_far = margin_far;
    p.a_min = a_min;
    p.interval = t_interval_out;
    p.a_hat = a_hat_out;
    propose_kernel<<<grid, 128, 0, static_cast<cudaStream_t>(stream)>>>(p);
    return cuda_status(fn);
}

extern "C" int32_t ngprt_propose_backward(const float* prop_w, const ngprt_camera* cams, int32_t n_cams,
                                          const int32_t* pixel_ids, const float* rays_o, const float* rays_d,
                                          int64_t n_rays, float in_scale, float t_scale, const float* targets,
                                          float* g_prop_w, float* loss, void* stream) {
    const char* fn = "ngprt_propose_backward";
    PropParams p;
    memset(&p, 0, sizeof p);
    NGPRT_REQUIRE(prop_w != nullptr && g_prop_w != nullptr, "%s: NULL weights or gradient", fn);
    NGPRT_REQUIRE(n_rays >= 0 && in_scale > 0.0f && t_scale > 0.0f, "%s: bad scalar argument", fn);
    dim3 grid;
    int32_t rc;
    if ((rc = setup_rays(p.m, cams, n_cams, pixel_ids, rays_o, rays_d, n_rays, grid, fn)) != NGPRT_OK) return rc;
    if (n_rays == 0) return NGPRT_OK;
    NGPRT_REQUIRE(targets != nullptr, "%s: targets is NULL", fn);
    p.w = prop_w;
    p.in_scale = in_scale;
    p.t_scale = t_scale;
    p.targets = targets;
    p.g_w = g_prop_w;
    p.loss = loss;
    propose_backward_kernel<<<grid, 128, 0, static_cast<cudaStream_t>(stream)>>>(p);
    return cuda_status(fn);
}
