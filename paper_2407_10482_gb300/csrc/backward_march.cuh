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
    float* records;     // MLP form: per-sample (f^1..f^L, g_f) records for the weight gradient
    int32_t* n_records; // their count (device)
    int64_t rec_capacity;
    const float* dist_state;  // distortion mode: per ray (L_dist, W, S, 0) of the forward
    float dist_scale;         // distortion mode: dL_total / dL_dist
};

// Floats of one MLP-form sample record: the level features x (8L) and the feature
// cotangent g_f (8).
template <int L>
__host__ __device__ constexpr int mlp_record_floats() {
    return kNFeat * L + kNFeat;
}

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
    return AGG == NGPRT_AGG_MLP ? kNFeat * L + NGPRT_AGG_MLP_HIDDEN : 4 * L + n_inv_logits<L, AGG>();
}

// Reverse of the tiny-MLP aggregation f = f~ + W2 relu(W1 x) at one sample, x =
// [f^1..f^L] and the pre-activations h left in the slots by the forward half:
// g_h = (W2^T g_f) where h > 0 (written over h), then each level's g_x^l = W1^T g_h
// restricted to its 8 inputs, added to its 8 corner entries times the corner weight.
template <int L>
__device__ __forceinline__ void scatter_mlp_levels(const Grid& g, const float u[3], const float gf[8], float* slots,
                                                   int stride, float* g_tables) {
    constexpr int kHid = NGPRT_AGG_MLP_HIDDEN;
    constexpr int NX = kNFeat * L;
    const float4* w2 = reinterpret_cast<const float4*>(g.agg_mlp + (size_t)kHid * NX);
#pragma unroll 2
    for (int j4 = 0; j4 < kHid / 4; ++j4) {
        float4 ga = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll
        for (int k = 0; k < kNFeat; ++k) {
            const float4 a = __ldg(w2 + k * (kHid / 4) + j4);
            ga.x = fmaf(a.x, gf[k], ga.x);
            ga.y = fmaf(a.y, gf[k], ga.y);
            ga.z = fmaf(a.z, gf[k], ga.z);
            ga.w = fmaf(a.w, gf[k], ga.w);
        }
        float* hp = slots + (size_t)(NX + 4 * j4) * stride;
        hp[0] = hp[0] > 0.0f ? ga.x : 0.0f;
        hp[stride] = hp[stride] > 0.0f ? ga.y : 0.0f;
        hp[2 * stride] = hp[2 * stride] > 0.0f ? ga.z : 0.0f;
        hp[3 * stride] = hp[3 * stride] > 0.0f ? ga.w : 0.0f;
    }
    const float4* w1 = reinterpret_cast<const float4*>(g.agg_mlp);
#pragma unroll 1
    for (int l = 0; l < L; ++l) {
        float gx[8] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll 4
        for (int j = 0; j < kHid; ++j) {
            const float gh = slots[(NX + j) * stride];
            const float4 a = __ldg(w1 + 2 * (L * j + l)), b = __ldg(w1 + 2 * (L * j + l) + 1);
            gx[0] = fmaf(a.x, gh, gx[0]);
            gx[1] = fmaf(a.y, gh, gx[1]);
            gx[2] = fmaf(a.z, gh, gx[2]);
            gx[3] = fmaf(a.w, gh, gx[3]);
            gx[4] = fmaf(b.x, gh, gx[4]);
            gx[5] = fmaf(b.y, gh, gx[5]);
            gx[6] = fmaf(b.z, gh, gx[6]);
            gx[7] = fmaf(b.w, gh, gx[7]);
        }
        int bl[3];
        float wl[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) grid_cell(u[a], g.N[l], bl[a], wl[a]);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const uint32_t row = level_row(g, l, (uint32_t)(bl[0] + (c & 1)), (uint32_t)(bl[1] + ((c >> 1) & 1)),
                                           (uint32_t)(bl[2] + ((c >> 2) & 1)));
            const float cw = corner_w(wl, c);
            float* gp = g_tables + (size_t)row * 8;
            atomic_add4(gp, cw * gx[0], cw * gx[1], cw * gx[2], cw * gx[3]);
            atomic_add4(gp + 4, cw * gx[4], cw * gx[5], cw * gx[6], cw * gx[7]);
        }
    }
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
// kDensityOnly (the distortion regulariser, whose cotangent is [gs, 0, ...]): the
// gated forms and the sum add nothing to the colour channels, so only the density
// channel of each entry and vertex (and the logits) are written.
template <int L, int AGG, bool kDensityOnly = false>
__device__ __forceinline__ void scatter_features(const Grid& g, const float u[3], int attn_mode, float gs, float w,
                                                 const float gq[7], float* slots, int stride, float* g_tables,
                                                 float* g_coarse) {
    constexpr int NC = coarse_channels(L, AGG);
    constexpr int NLOG = NC - kNFeat;  // spatial logits stored in the coarse grid
    float gw[7];
#pragma unroll
    for (int k = 0; k < 7; ++k) gw[k] = w * gq[k];
    if constexpr (AGG == NGPRT_AGG_MLP) {
        const float gf[8] = {gs, gw[0], gw[1], gw[2], gw[3], gw[4], gw[5], gw[6]};
        scatter_mlp_levels<L>(g, u, gf, slots, stride, g_tables);
    }
#pragma unroll kScatterUnroll
    for (int l = 0; l < (AGG == NGPRT_AGG_MLP ? 0 : L); ++l) {
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
            if constexpr (kDensityOnly) {
                atomicAdd(gp, cw * s0);
            } else {
                atomic_add4(gp, cw * s0, cb * gw[0], cb * gw[1], cb * gw[2]);
                atomic_add4(gp + 4, cb * gw[3], cb * gw[4], cb * gw[5], cb * gw[6]);
            }
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
        if constexpr (kDensityOnly) {
            atomicAdd(gp, cw * gs);
            if (logits) {
#pragma unroll
                for (int k = 0; k < NLOG; ++k) atomicAdd(gp + 8 + k, cw * slots[k * stride]);
            }
        } else if constexpr (NC % 4 == 0) {
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

// kDist: the distortion regulariser's reverse pass (Eq. S2): the colour cotangents
// stay 0 and each sample's dL/dsigma comes from the running sums W, S, G against the
// ray's totals, as in the regulariser's own reverse pass.
template <int L, int AGG, bool kDist = false>
struct BackwardSampler {
    const Grid& g;
    int attn_mode;
    float t_term;
    float T, S_le, S_tot;
    float gCd[3], gF[4], gA, gD;
    float* g_tables;
    float* g_coarse;
    float* gates;
    float* records;
    int32_t* n_records;
    int64_t rec_capacity;
    float dW = 0.0f, dS = 0.0f, dG = 0.0f;                         // distortion running sums
    float dW_tot = 0.0f, dS_tot = 0.0f, dG_tot = 0.0f, d_scale = 0.0f;  // and the ray's totals
    __device__ __forceinline__ bool sample(const float u[3], float t, float delta) {
        float f[8];
        const float gq[7] = {gCd[0], gCd[1], gCd[2], gF[0], gF[1], gF[2], gF[3]};
        sample_features<L, NGPRT_F32, AGG, true>(g, u, attn_mode, f, gates, blockDim.x, gq);
        const float sigma = expf(f[0]);
        const float trans = expf(-sigma * delta);
        const float w = T * (1.0f - trans);
        const float T_next = T * trans;
        float gs;
        if constexpr (kDist) {
            const float m = fmaf(0.5f, delta, t);
            const float W_lt = dW, S_lt = dS;
            dW += w;
            dS = fmaf(w, m, dS);
            const float gw = 2.0f * (fmaf(m, W_lt, -S_lt) + (dS_tot - dS) - m * (dW_tot - dW)) +
                             (2.0f / 3.0f) * w * delta;
            dG = fmaf(w, gw, dG);
            const float g_sigma = delta * (T_next * gw - (dG_tot - dG));
            gs = d_scale * g_sigma * expf(fminf(f[0], 15.0f));
        } else {
            float qg = fmaf(gD, t, gA);
#pragma unroll
            for (int k = 0; k < 3; ++k) qg = fmaf(gCd[k], f[1 + k], qg);
#pragma unroll
            for (int k = 0; k < 4; ++k) qg = fmaf(gF[k], f[4 + k], qg);
            S_le = fmaf(w, qg, S_le);
            const float g_sigma = delta * (T_next * qg - (S_tot - S_le));
            gs = g_sigma * expf(fminf(f[0], 15.0f));
        }
        scatter_features<L, AGG, kDist>(g, u, attn_mode, gs, w, gq, gates, blockDim.x, g_tables, g_coarse);
        if constexpr (AGG == NGPRT_AGG_MLP) {
            // (x, g_f) of this sample for the weight gradient; capacity n_rays x
            // max_samples is never exceeded, the bound only guards the buffer
            const int64_t r = atomicAdd(n_records, 1);
            if (r < rec_capacity) {
                float4* rp = reinterpret_cast<float4*>(records + r * mlp_record_floats<L>());
                const int st = blockDim.x;
#pragma unroll 4
                for (int q = 0; q < 2 * L; ++q)
                    rp[q] = make_float4(gates[(4 * q) * st], gates[(4 * q + 1) * st], gates[(4 * q + 2) * st],
                                        gates[(4 * q + 3) * st]);
                rp[2 * L] = make_float4(gs, w * gq[0], w * gq[1], w * gq[2]);
                rp[2 * L + 1] = make_float4(w * gq[3], w * gq[4], w * gq[5], w * gq[6]);
            }
        }
        T = T_next;
        return T < t_term;
    }
};

// Resident blocks the reverse march's register allocation must allow: 3 (168
// registers, no spills) was the fastest measured on a 2^18-ray training step of
// the fitted hd scene (33.4 ms against 34.5 at 1, 255 registers; 34.4 at 4; 35.6 at
// 5 and 37.7 at 6, where it spills).
#ifndef NGPRT_BWD_MIN_BLOCKS
#define NGPRT_BWD_MIN_BLOCKS 3
#endif

template <int L, int AGG, bool kDist = false>
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
    Ray ry;
    bool hit = false;
    const bool live = ray_setup(p.m, ray, ry, hit) && hit;
    if constexpr (NI == 0) {
        if (!live) return;
    }
    if (live) {
        int n_march = 0, n_samp = 0;
        if constexpr (kDist) {
            const float4 ds = reinterpret_cast<const float4*>(p.dist_state)[ray];
            BackwardSampler<L, AGG, true> smp{p.m.g, p.m.opts.attn_mode, p.m.opts.t_term, 1.0f, 0.0f, 0.0f,
                                              {0.0f, 0.0f, 0.0f}, {0.0f, 0.0f, 0.0f, 0.0f}, 0.0f, 0.0f,
                                              p.g_tables, p.g_coarse, slots, p.records, p.n_records,
                                              p.rec_capacity, 0.0f, 0.0f, 0.0f, ds.y, ds.z, 2.0f * ds.x,
                                              p.dist_scale};
            march_loop(p.m, ry, smp, n_march, n_samp);
        } else {
            const float4* c4 = reinterpret_cast<const float4*>(p.cot + ray * kCotFloats);
            const float4 q0 = c4[0], q1 = c4[1], q2 = c4[2];
            BackwardSampler<L, AGG> smp{p.m.g, p.m.opts.attn_mode, p.m.opts.t_term, 1.0f, 0.0f, q2.y,
                                        {q0.x, q0.y, q0.z}, {q0.w, q1.x, q1.y, q1.z}, q1.w, q2.x, p.g_tables,
                                        p.g_coarse, slots, p.records, p.n_records, p.rec_capacity};
            march_loop(p.m, ry, smp, n_march, n_samp);
        }
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

// Weight gradient of the tiny-MLP aggregation from the sample records: per record
// h = W1 x, a = relu(h), g_h = (W2^T g_f) on h > 0, then dW1 += g_h x^T and dW2 +=
// g_f a^T.  Each block takes tiles of 128 records (one per thread), stages x, g_f,
// a, g_h in shared memory and sums its share of the outputs over the tile in
// registers (thread t owns outputs t, t + 128, ...); one atomic per output and block.
template <int L>
__global__ void __launch_bounds__(128) agg_mlp_wgrad_kernel(const float* __restrict__ records,
                                                            const int32_t* __restrict__ n_records, int64_t capacity,
                                                            const float* __restrict__ w, float* __restrict__ g_w) {
    constexpr int kHid = NGPRT_AGG_MLP_HIDDEN;
    constexpr int NX = kNFeat * L;
    constexpr int RF = mlp_record_floats<L>();
    constexpr int NOUT = kHid * NX + kNFeat * kHid;
    constexpr int PER = (NOUT + 127) / 128;
    extern __shared__ float sm[];
    float* X = sm;                  // [128][NX + 1]
    float* GF = X + 128 * (NX + 1);  // [128][9]
    float* A = GF + 128 * 9;         // [128][kHid + 1]
    float* GH = A + 128 * (kHid + 1); // [128][kHid + 1]
    const int64_t n = min((int64_t)*n_records, capacity);
    float acc[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) acc[k] = 0.0f;
    const int t = threadIdx.x;
    for (int64_t base = (int64_t)blockIdx.x * 128; base < n; base += (int64_t)gridDim.x * 128) {
        const int64_t r = base + t;
        // this thread's record into its rows of X and GF (zeros past the last record)
        float* xr = X + t * (NX + 1);
        float* gr = GF + t * 9;
        const float4* rp = reinterpret_cast<const float4*>(records + r * RF);
#pragma unroll 4
        for (int q = 0; q < NX / 4; ++q) {
            const float4 v = r < n ? rp[q] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            xr[4 * q] = v.x; xr[4 * q + 1] = v.y; xr[4 * q + 2] = v.z; xr[4 * q + 3] = v.w;
        }
        float gf[kNFeat];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const float4 v = r < n ? rp[NX / 4 + q] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            gf[4 * q] = v.x; gf[4 * q + 1] = v.y; gf[4 * q + 2] = v.z; gf[4 * q + 3] = v.w;
        }
#pragma unroll
        for (int k = 0; k < kNFeat; ++k) gr[k] = gf[k];
        const float4* w1 = reinterpret_cast<const float4*>(w);
        const float* w2 = w + (size_t)kHid * NX;
#pragma unroll 1
        for (int j = 0; j < kHid; ++j) {
            float h = 0.0f;
#pragma unroll 4
            for (int q = 0; q < NX / 4; ++q) {
                const float4 a = __ldg(w1 + j * (NX / 4) + q);
                h = fmaf(a.x, xr[4 * q], h);
                h = fmaf(a.y, xr[4 * q + 1], h);
                h = fmaf(a.z, xr[4 * q + 2], h);
                h = fmaf(a.w, xr[4 * q + 3], h);
            }
            float ga = 0.0f;
#pragma unroll
            for (int k = 0; k < kNFeat; ++k) ga = fmaf(__ldg(w2 + k * kHid + j), gf[k], ga);
            A[t * (kHid + 1) + j] = fmaxf(h, 0.0f);
            GH[t * (kHid + 1) + j] = h > 0.0f ? ga : 0.0f;
        }
        __syncthreads();
        // one pass over the tile per owned output (acc may live in local memory: it
        // is touched once per 128 multiply-adds)
#pragma unroll 1
        for (int k = 0; k < PER; ++k) {
            const int o = t + 128 * k;
            if (o < NOUT) {
                float s = acc[k];
                if (o < kHid * NX) {
                    const int j = o / NX, q = o - j * NX;
                    for (int rr = 0; rr < 128; ++rr) s = fmaf(GH[rr * (kHid + 1) + j], X[rr * (NX + 1) + q], s);
                } else {
                    const int o2 = o - kHid * NX, k2 = o2 / kHid, j = o2 - k2 * kHid;
                    for (int rr = 0; rr < 128; ++rr) s = fmaf(GF[rr * 9 + k2], A[rr * (kHid + 1) + j], s);
                }
                acc[k] = s;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int o = t + 128 * k;
        if (o < NOUT && acc[k] != 0.0f) atomicAdd(g_w + o, acc[k]);
    }
}

template <int L>
void launch_agg_mlp_wgrad(const MarchBwdParams& p, const float* w, float* g_w, cudaStream_t st) {
    constexpr int NX = kNFeat * L;
    const size_t smem = (size_t)128 * ((NX + 1) + 9 + 2 * (NGPRT_AGG_MLP_HIDDEN + 1)) * sizeof(float);
    cudaFuncSetAttribute(agg_mlp_wgrad_kernel<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int64_t tiles = (p.rec_capacity + 127) / 128;
    const unsigned blocks = (unsigned)(tiles < 152 * 2 ? (tiles < 1 ? 1 : tiles) : 152 * 2);
    agg_mlp_wgrad_kernel<L><<<blocks, 128, smem, st>>>(p.records, p.n_records, p.rec_capacity, w, g_w);
}

template <int L, int AGG, bool kDist = false>
void launch_bwd(const MarchBwdParams& p, dim3 grid, cudaStream_t st) {
    const size_t smem = (size_t)bwd_slots<L, AGG>() * 128 * sizeof(float);
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(march_backward_kernel<L, AGG, kDist>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    march_backward_kernel<L, AGG, kDist><<<grid, 128, smem, st>>>(p);
}

// The gate forms other than Eq. 8 and the tiny MLP (backward_agg.cu): L = 2, 4, 16.
bool march_bwd_agg_supports(int L);
void launch_bwd_agg(int L, int agg, const MarchBwdParams& p, dim3 grid, cudaStream_t st);
void launch_bwd_agg_mlp_wgrad(int L, const MarchBwdParams& p, const float* w, float* g_w, cudaStream_t st);

}  // namespace ngprt
