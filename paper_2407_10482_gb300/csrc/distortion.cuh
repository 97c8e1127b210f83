// distortion.cuh -- the distortion regulariser's forward kernel (Eq. S2), templated
// on the aggregation form: distortion.cu builds Eq. 8, distortion_agg.cu the other
// forms of Table 3 (whose reverse pass is the reverse march in distortion mode).
#pragma once
#include "backward_march.cuh"

namespace ngprt {

struct DistParams {
    MarchParams m;
    float* dist_state;       // forward: [n][4] = (L_dist, W, S, 0) out; backward: in
    float scale;             // forward: loss += scale L_dist; backward: dL_total/dL_dist per ray
    float* loss;
    float* g_tables;
    float* g_coarse;
};

template <int L, int AGG>
struct DistSampler {
    ForwardSampler<L, NGPRT_F32, AGG> fw;
    float W, S, Lp, Ls;
    __device__ __forceinline__ bool sample(const float u[3], float t, float delta) {
        const bool stop = fw.sample(u, t, delta);
        const float w = fw.w_last;
        const float m = fmaf(0.5f, delta, t);
        Lp = fmaf(2.0f * w, fmaf(m, W, -S), Lp);
        Ls = fmaf(w * w, delta * (1.0f / 3.0f), Ls);
        W += w;
        S = fmaf(w, m, S);
        return stop;
    }
};

template <int L, int AGG>
__global__ void __launch_bounds__(128) distortion_kernel(const __grid_constant__ DistParams p) {
    extern __shared__ float gate_smem[];
    int64_t ray = 0;
    Ray ry;
    bool hit = false;
    const bool has_ray = ray_setup(p.m, ray, ry, hit);
    float Ld = 0.0f;
    if (has_ray) {
        DistSampler<L, AGG> smp{ForwardSampler<L, NGPRT_F32, AGG>(p.m.g, p.m.opts.attn_mode, p.m.opts.t_term,
                                                                  gate_smem + threadIdx.x),
                                0.0f, 0.0f, 0.0f, 0.0f};
        int n_march = 0, n_samp = 0;
        if (hit) march_loop(p.m, ry, smp, n_march, n_samp);
        Ld = smp.Lp + smp.Ls;
        reinterpret_cast<float4*>(p.dist_state)[ray] = make_float4(Ld, smp.W, smp.S, 0.0f);
    }
    if (p.loss) {
        __syncwarp();
        float v = Ld;
#pragma unroll
        for (int k = 16; k > 0; k >>= 1) v += __shfl_xor_sync(0xffffffffu, v, k);
        if ((threadIdx.x & 31) == 0 && v != 0.0f) atomicAdd(p.loss, p.scale * v);
    }
}

// The forms of Table 3 other than Eq. 8 (distortion_agg.cu): L = 2, 4, 16.
void launch_dist_fwd_agg(int L, int agg, const DistParams& p, dim3 grid, cudaStream_t st);
void launch_dist_bwd_agg(int L, int agg, const MarchBwdParams& p, dim3 grid, cudaStream_t st);

}  // namespace ngprt
