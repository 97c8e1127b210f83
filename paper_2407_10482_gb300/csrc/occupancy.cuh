// occupancy.cuh -- kernels of the render-time occupancy pipeline (Sec. S2.5):
// occupancy from the model's own density at voxel centres and visibility marks of
// training rays, templated on the aggregation form so that occupancy.cu (Eq. 8) and
// occupancy_agg.cu (the other forms of Table 3) build in parallel.
#pragma once
#include "march.cuh"

namespace ngprt {

struct DensityOccParams {
    Grid g;
    int32_t R;
    int32_t attn_mode;
    float sigma_thr;
    uint8_t* occ;
    float* sigma;
};

// One voxel per thread: sigma = exp(sigma_raw) at the voxel centre (Eq. 6-8).
template <int L, int DT, int AGG>
__global__ void __launch_bounds__(128) density_occ_kernel(const __grid_constant__ DensityOccParams p) {
    extern __shared__ float gate_smem[];
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t R = p.R;
    if (v >= R * R * R) return;
    const int i = (int)(v % R), j = (int)((v / R) % R), k = (int)(v / (R * R));
    const float inv = fdiv(1.0f, (float)R);  // R is a power of two: exact
    const float u[3] = {fmul(fadd((float)i, 0.5f), inv), fmul(fadd((float)j, 0.5f), inv),
                        fmul(fadd((float)k, 0.5f), inv)};
    float f[8];
    sample_features<L, DT, AGG>(p.g, u, p.attn_mode, f, gate_smem + threadIdx.x, blockDim.x);
    const float sg = expf(f[0]);
    p.occ[v] = sg > p.sigma_thr ? 1 : 0;
    if (p.sigma) p.sigma[v] = sg;
}

// Composites like the forward render and marks the voxel (R^3 grid) of every sample
// whose weight exceeds w_thr.  All writers store 1, so concurrent marks agree.
template <int L, int DT, int AGG>
struct VisibilitySampler {
    ForwardSampler<L, DT, AGG> fw;
    float w_thr;
    int32_t R;
    uint8_t* vis;
    __device__ __forceinline__ bool sample(const float u[3], float t, float delta) {
        const bool stop = fw.sample(u, t, delta);
        if (fw.w_last > w_thr) {
            const uint32_t v = (uint32_t)occ_vox(u[0], R) +
                               (uint32_t)R * ((uint32_t)occ_vox(u[1], R) + (uint32_t)R * (uint32_t)occ_vox(u[2], R));
            vis[v] = 1;
        }
        return stop;
    }
};

template <int L, int DT, int AGG>
__global__ void __launch_bounds__(128, march_min_blocks<L, DT, AGG>())
    visibility_kernel(const __grid_constant__ MarchParams p, float w_thr, int32_t R, uint8_t* vis) {
    int64_t ray;
    Ray ry;
    bool hit;
    extern __shared__ float gate_smem[];
    if (!ray_setup(p, ray, ry, hit)) return;
    VisibilitySampler<L, DT, AGG> smp{
        ForwardSampler<L, DT, AGG>(p.g, p.opts.attn_mode, p.opts.t_term, gate_smem + threadIdx.x), w_thr, R, vis};
    int n_march = 0, n_samp = 0;
    if (hit) march_loop(p, ry, smp, n_march, n_samp);
}

template <int L, int AGG>
void launch_density(int dt, const DensityOccParams& p, cudaStream_t st) {
    const int64_t n = (int64_t)p.R * p.R * p.R;
    const unsigned blocks = (unsigned)((n + 127) / 128);
    const size_t shm = (size_t)2 * L * 128 * sizeof(float);
    if (dt == NGPRT_F32) density_occ_kernel<L, NGPRT_F32, AGG><<<blocks, 128, shm, st>>>(p);
    else if (dt == NGPRT_F16) density_occ_kernel<L, NGPRT_F16, AGG><<<blocks, 128, shm, st>>>(p);
    else density_occ_kernel<L, NGPRT_BF16, AGG><<<blocks, 128, shm, st>>>(p);
}

template <int L, int AGG>
void launch_visibility(int dt, const MarchParams& p, dim3 grid, float w_thr, int32_t R, uint8_t* vis,
                       cudaStream_t st) {
    const size_t shm = (size_t)2 * L * 128 * sizeof(float);
    if (dt == NGPRT_F32) visibility_kernel<L, NGPRT_F32, AGG><<<grid, 128, shm, st>>>(p, w_thr, R, vis);
    else if (dt == NGPRT_F16) visibility_kernel<L, NGPRT_F16, AGG><<<grid, 128, shm, st>>>(p, w_thr, R, vis);
    else visibility_kernel<L, NGPRT_BF16, AGG><<<grid, 128, shm, st>>>(p, w_thr, R, vis);
}

// The forms of Table 3 other than Eq. 8 (occupancy_agg.cu): L = 2, 4, 16.
bool occupancy_agg_supports(int L);
void launch_density_agg(int L, int agg, int dt, const DensityOccParams& p, cudaStream_t st);
void launch_visibility_agg(int L, int agg, int dt, const MarchParams& p, dim3 grid, float w_thr, int32_t R,
                           uint8_t* vis, cudaStream_t st);

}  // namespace ngprt
