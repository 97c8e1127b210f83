// backward_march.cuh -- the reverse march (Eq. 2, 5 and the gate forms of Eq. 8 and
// Table 3): per ray, the same march as the forward (same decisions: march_loop), and
// at each sample i the derivative of the composite sums Q = sum_j w_j q_j:
//     dQ/dq_i = w_i,   dQ/dsigma_i = delta_i (T_{i+1} q_i - sum_{j>i} w_j q_j),
// where the suffix sum is the stored total minus the running prefix.  The density
// activation exp has the truncated derivative exp(min(sigma_raw, 15)).  Through the
// gates and the trilinear weights the gradient reaches 8 entries of each fine level
// and 8 coarse vertices; it is added with 16-byte vector atomics.  Templated on the
// gate form, so that backward.cu (Eq. 8) and backward_agg.cu (the other forms) build
// in parallel.
#pragma once
#include "march.cuh"

namespace ngprt {

constexpr int kCotFloats = 12;  // g_Cd(3), g_F(4), g_A, g_depth, S_total, pad(2)

struct MarchBwdParams {
    MarchParams m;
    const float* state;
    const float* cot;
    float* g_tables;
    float* g_coarse;
    float* g_attn_inv;  // constant gate logits' gradient (SEPARATE_INV, SHARED_INV)
};

__device__ __forceinline__ void atomic_add4(float* p, float a, float b, float c, float d) {
#ifdef NGPRT_SCALAR_ATOMICS
    atomicAdd(p, a);
    atomicAdd(p + 1, b);
    atomicAdd(p + 2, c);
    atomicAdd(p + 3, d);
#else
    atomicAdd(reinterpret_cast<float4*>(p), make_float4(a, b, c, d));
#endif
}

// Gate logits the reverse pass accumulates per thread (in shared memory) and adds
// once per block: the spatially invariant forms' 2L or L constants.
template <int L, int AGG>
__host__ __device__ constexpr int n_inv_logits() {
    return AGG == NGPRT_AGG_SEPARATE_INV ? 2 * L : (AGG == NGPRT_AGG_SHARED_INV ? L : 0);
}

// Shared-memory floats per thread of the reverse march: the gates omega^l, beta^l
// ([0, 2L)), sigma^l and q^l ([2L, 4L)) and the invariant logits' sums.
template <int L, int AGG>
__host__ __device__ constexpr int bwd_slots() {
    return 4 * L + n_inv_logits<L, AGG>();
}

// Reverse of sample_features at u.  The sample's feature cotangent is
// gf = [gs, w gq] (gs = dL/dsigma_raw, w the sample's weight, gq the ray's colour
// cotangents); the forward half of the sampler left in the thread's slots the gates
// omega^l, beta^l ([0, 2L)) and sigma^l, q^l = f^l[1..7] . gq ([2L, 4L)), so no
// entry is read again: each level only recomputes its 8 corner rows and adds
//     d entry = cw [omega^l gs, beta^l w gq]
// (omega = beta = 1 for the plain sum).  The gate-logit gradients are
//     d omega-logit = sigma^l gs omega (1 - omega),  d beta-logit = w q^l beta (1 - beta),
// summed onto one logit where omega and beta are one gate.  Spatial logits go with gf
// to the 8 coarse vertices (Eq. 8: slots [0, 2L) -> channels 8 + [0, 2L); one gate per
// level: slot l -> channel 8 + l); invariant ones add to the thread's sums.
template <int L, int AGG>
__device__ __forceinline__ void scatter_features(const Grid& g, const float u[3], int attn_mode, float gs, float w,
                                                 const float gq[7], float* slots, int stride, float* g_tables,
                                                 float* g_coarse) {
    constexpr int NC = coarse_channels(L, AGG);
    constexpr int NLOG = NC - kNFeat;  // spatial logits stored in the coarse grid
    float gw[7];
#pragma unroll
    for (int k = 0; k < 7; ++k) gw[k] = w * gq[k];
#pragma unroll kLevelUnroll
    for (int l = 0; l < L; ++l) {
        float om = 1.0f, be = 1.0f;
        if constexpr (AGG != NGPRT_AGG_SUM) {
            om = slots[(2 * l) * stride];
            be = slots[(2 * l + 1) * stride];
        }
        const float sh = slots[(2 * L + 2 * l) * stride], q = slots[(2 * L + 2 * l + 1) * stride];
        int bl[3];
        float wl[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) grid_cell(u[a], g.N[l], bl[a], wl[a]);
        const float s0 = om * gs;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const uint32_t row = level_row(g, l, (uint32_t)(bl[0] + (c & 1)), (uint32_t)(bl[1] + ((c >> 1) & 1)),
                                           (uint32_t)(bl[2] + ((c >> 2) & 1)));
            const float cw = corner_w(wl, c);
            const float cb = cw * be;
            float* gp = g_tables + (size_t)row * 8;
            atomic_add4(gp, cw * s0, cb * gw[0], cb * gw[1], cb * gw[2]);
            atomic_add4(gp + 4, cb * gw[3], cb * gw[4], cb * gw[5], cb * gw[6]);
        }
        if constexpr (AGG == NGPRT_AGG_SEPARATE_V) {
            float go = 0.0f, gb = 0.0f;
            if (attn_mode == 0) {
                go = sh * gs * om * (1.0f - om);
                gb = w * q * be * (1.0f - be);
            } else if (attn_mode == 2) {
                go = (sh * gs + w * q) * om * (1.0f - om);
            }
            slots[(2 * l) * stride] = go;
            slots[(2 * l + 1) * stride] = gb;
        } else if constexpr (AGG == NGPRT_AGG_SHARED_V) {
            // slot l is below every slot a later level still reads (2l' >= 2l + 2)
            slots[l * stride] = (sh * gs + w * q) * om * (1.0f - om);
        } else if constexpr (AGG == NGPRT_AGG_SEPARATE_INV) {
            slots[(4 * L + 2 * l) * stride] += sh * gs * om * (1.0f - om);
            slots[(4 * L + 2 * l + 1) * stride] += w * q * be * (1.0f - be);
        } else if constexpr (AGG == NGPRT_AGG_SHARED_INV) {
            slots[(4 * L + l) * stride] += (sh * gs + w * q) * om * (1.0f - om);
        }
    }
    // coarse vertices: [gf(8), spatial logit grads(NLOG)] times the corner weight
    const bool logits = NLOG > 0 && (AGG != NGPRT_AGG_SEPARATE_V || attn_mode != 1);
    int b[3];
    float wc[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) grid_cell(u[a], g.R_C, b[a], wc[a]);
    const uint32_t R = (uint32_t)g.R_C;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const uint32_t cv = (uint32_t)(b[0] + (c & 1)) + R * ((uint32_t)(b[1] + ((c >> 1) & 1)) + R * (uint32_t)(b[2] + ((c >> 2) & 1)));
        const float cw = corner_w(wc, c);
        float* gp = g_coarse + (size_t)cv * NC;
        if constexpr (NC % 4 == 0) {
            atomic_add4(gp, cw * gs, cw * gw[0], cw * gw[1], cw * gw[2]);
            atomic_add4(gp + 4, cw * gw[3], cw * gw[4], cw * gw[5], cw * gw[6]);
            if (logits) {
#pragma unroll 4
                for (int k = 0; k < NLOG; k += 4)
                    atomic_add4(gp + 8 + k, cw * slots[k * stride], cw * slots[(k + 1) * stride],
                                cw * slots[(k + 2) * stride], cw * slots[(k + 3) * stride]);
            }
        } else {
            atomicAdd(gp, cw * gs);
#pragma unroll
            for (int ch = 0; ch < 7; ++ch) atomicAdd(gp + 1 + ch, cw * gw[ch]);
            if (logits) {
#pragma unroll
                for (int k = 0; k < NLOG; ++k) atomicAdd(gp + 8 + k, cw * slots[k * stride]);
            }
        }
    }
}

template <int L, int AGG>
struct BackwardSampler {
    const Grid& g;
    int attn_mode;
    float t_term;
    float T, S_le, S_tot;
    float gCd[3], gF[4], gA, gD;
    float* g_tables;
    float* g_coarse;
    float* gates;
    __device__ __forceinline__ bool sample(const float u[3], float t, float delta) {
        float f[8];
        const float gq[7] = {gCd[0], gCd[1], gCd[2], gF[0], gF[1], gF[2], gF[3]};
        sample_features<L, NGPRT_F32, AGG, true>(g, u, attn_mode, f, gates, blockDim.x, gq);
        const float sigma = expf(f[0]);
        const float trans = expf(-sigma * delta);
        const float w = T * (1.0f - trans);
        const float T_next = T * trans;
        float qg = fmaf(gD, t, gA);
#pragma unroll
        for (int k = 0; k < 3; ++k) qg = fmaf(gCd[k], f[1 + k], qg);
#pragma unroll
        for (int k = 0; k < 4; ++k) qg = fmaf(gF[k], f[4 + k], qg);
        S_le = fmaf(w, qg, S_le);
        const float g_sigma = delta * (T_next * qg - (S_tot - S_le));
        const float gs = g_sigma * expf(fminf(f[0], 15.0f));
        scatter_features<L, AGG>(g, u, attn_mode, gs, w, gq, gates, blockDim.x, g_tables, g_coarse);
        T = T_next;
        return T < t_term;
    }
};

// Resident blocks the reverse march's register allocation must allow.  1 lets it
// take 255 registers (about 7 warps per SM) and was the fastest measured: 4..8
// blocks (fewer registers, more warps) made a 2^18-ray training step 5-10% slower.
#ifndef NGPRT_BWD_MIN_BLOCKS
#define NGPRT_BWD_MIN_BLOCKS 1
#endif

template <int L, int AGG>
__global__ void __launch_bounds__(128, NGPRT_BWD_MIN_BLOCKS) march_backward_kernel(const __grid_constant__ MarchBwdParams p) {
    extern __shared__ float gate_smem[];
    constexpr int NI = n_inv_logits<L, AGG>();
    float* slots = gate_smem + threadIdx.x;
    const int stride = blockDim.x;
    if constexpr (NI > 0) {
#pragma unroll
        for (int k = 0; k < NI; ++k) slots[(4 * L + k) * stride] = 0.0f;
    }
    int64_t ray;
    float o[3], d[3], t, t_out;
    bool hit = false;
    const bool live = ray_setup(p.m, ray, o, d, t, t_out, hit) && hit;
    if constexpr (NI == 0) {
        if (!live) return;
    }
    if (live) {
        const float4* c4 = reinterpret_cast<const float4*>(p.cot + ray * kCotFloats);
        const float4 q0 = c4[0], q1 = c4[1], q2 = c4[2];
        BackwardSampler<L, AGG> smp{p.m.g, p.m.opts.attn_mode, p.m.opts.t_term, 1.0f, 0.0f, q2.y,
                                    {q0.x, q0.y, q0.z}, {q0.w, q1.x, q1.y, q1.z}, q1.w, q2.x, p.g_tables,
                                    p.g_coarse, slots};
        int n_march = 0, n_samp = 0;
        march_loop(p.m, o, d, t, t_out, smp, n_march, n_samp);
    }
    if constexpr (NI > 0) {
        // the block's sums of the invariant logits' gradients: thread k < NI adds
        // column k over the block's threads, then one atomic per logit and block
        __syncthreads();
        if ((int)threadIdx.x < NI) {
            const float* col = gate_smem + (size_t)(4 * L + threadIdx.x) * stride;
            float s = 0.0f;
            for (int k = 0; k < stride; ++k) s += col[k];
            atomicAdd(p.g_attn_inv + threadIdx.x, s);
        }
    }
}

template <int L, int AGG>
void launch_bwd(const MarchBwdParams& p, dim3 grid, cudaStream_t st) {
    const size_t smem = (size_t)bwd_slots<L, AGG>() * 128 * sizeof(float);
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(march_backward_kernel<L, AGG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    march_backward_kernel<L, AGG><<<grid, 128, smem, st>>>(p);
}

// The gate forms other than Eq. 8 (backward_agg.cu): L = 2, 4, 16.
bool march_bwd_agg_supports(int L);
void launch_bwd_agg(int L, int agg, const MarchBwdParams& p, dim3 grid, cudaStream_t st);

}  // namespace ngprt
