// distortion.cu -- the distortion regulariser of Mip-NeRF 360 in NGP-RT's training
// loss (Eq. S2), over the samples the render composites:
//     L_dist = sum_{i,j} w_i w_j |m_i - m_j| + 1/3 sum_i w_i^2 delta_i,
// m_i = t_i + delta_i / 2 the midpoint of sample i's interval (delta_i as in the
// render).  The midpoints increase along the ray, so the double sum is
// 2 sum_i w_i (m_i W_<i - S_<i) with the running sums W_<i = sum_{j<i} w_j and
// S_<i = sum_{j<i} w_j m_j: one pass, O(N) per ray.
//
// Reverse pass.  g_i = dL/dw_i = 2 (m_i W_<i - S_<i + S_>i - m_i W_>i) + 2/3 w_i delta_i,
// and through the weights (the identity the render's reverse pass uses for any
// weighted sum) dL/dsigma_i = delta_i (T_{i+1} g_i - sum_{j>i} w_j g_j).  The suffix
// sums come from per-ray totals stored by the forward kernel: W and S, and
// sum_j w_j g_j = 2 L_dist because L_dist is homogeneous of degree 2 in w.  Only
// the density path carries a gradient: sigma~ of the coarse grid, the omega logits
// and the density channel of each fine level.
#include "distortion.cuh"

namespace ngprt {
namespace {

// Density-only reverse of sample_features (Eq. 6-8) for d(loss)/d(sigma_raw) = gs.
template <int L>
__device__ __forceinline__ void scatter_density(const Grid& g, const float u[3], int attn_mode, float gs,
                                                float* g_tables, float* g_coarse) {
    constexpr int NC = kNFeat + 2 * L;
    int b[3];
    float w[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) grid_cell(u[a], g.R_C, b[a], w[a]);
    const uint32_t R = (uint32_t)g.R_C;
    uint32_t cv[8];
    float om_logit[L];
#pragma unroll
    for (int l = 0; l < L; ++l) om_logit[l] = 0.0f;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        cv[c] = (uint32_t)(b[0] + (c & 1)) + R * ((uint32_t)(b[1] + ((c >> 1) & 1)) + R * (uint32_t)(b[2] + ((c >> 2) & 1)));
        const float cw = corner_w(w, c);
        const float* row = static_cast<const float*>(g.coarse) + (size_t)cv[c] * NC;
#pragma unroll
        for (int l = 0; l < L; ++l) om_logit[l] = fmaf(cw, __ldg(row + kNFeat + 2 * l), om_logit[l]);
    }
    float glog[L];
#pragma unroll
    for (int l = 0; l < L; ++l) {
        const float om = attn_mode == 1 ? 1.0f : sigmoidf_(om_logit[l]);
        int bl[3];
        float wl[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) grid_cell(u[a], g.N[l], bl[a], wl[a]);
        uint32_t rows[8];
        float sh = 0.0f;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            rows[c] = level_row(g, l, (uint32_t)(bl[0] + (c & 1)), (uint32_t)(bl[1] + ((c >> 1) & 1)),
                                (uint32_t)(bl[2] + ((c >> 2) & 1)));
            sh = fmaf(corner_w(wl, c), __ldg(static_cast<const float*>(g.tables) + (size_t)rows[c] * 8), sh);
        }
        glog[l] = attn_mode == 1 ? 0.0f : gs * sh * om * (1.0f - om);
        const float s0 = om * gs;
#pragma unroll
        for (int c = 0; c < 8; ++c) atomicAdd(g_tables + (size_t)rows[c] * 8, corner_w(wl, c) * s0);
    }
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const float cw = corner_w(w, c);
        float* gp = g_coarse + (size_t)cv[c] * NC;
        atomicAdd(gp, cw * gs);
#pragma unroll
        for (int l = 0; l < L; ++l)
            if (attn_mode != 1) atomicAdd(gp + kNFeat + 2 * l, cw * glog[l]);
    }
}

template <int L>
struct DistBwdSampler {
    const Grid& g;
    int attn_mode;
    float t_term;
    float* gates;
    float T, W, S, G;
    float W_tot, S_tot, G_tot, scale;
    float* g_tables;
    float* g_coarse;
    __device__ __forceinline__ bool sample(const float u[3], float t, float delta) {
        float f[8];
        sample_features<L, NGPRT_F32>(g, u, attn_mode, f, gates, blockDim.x);
        const float sigma = expf(f[0]);
        const float trans = expf(-sigma * delta);
        const float w = T * (1.0f - trans);
        const float T_next = T * trans;
        const float m = fmaf(0.5f, delta, t);
        const float W_lt = W, S_lt = S;
        W += w;
        S = fmaf(w, m, S);
        const float gw = 2.0f * (fmaf(m, W_lt, -S_lt) + (S_tot - S) - m * (W_tot - W)) + (2.0f / 3.0f) * w * delta;
        G = fmaf(w, gw, G);
        const float g_sigma = delta * (T_next * gw - (G_tot - G));
        scatter_density<L>(g, u, attn_mode, scale * g_sigma * expf(fminf(f[0], 15.0f)), g_tables, g_coarse);
        T = T_next;
        return T < t_term;
    }
};

template <int L>
__global__ void __launch_bounds__(128) distortion_backward_kernel(const __grid_constant__ DistParams p) {
    extern __shared__ float gate_smem[];
    int64_t ray;
    Ray ry;
    bool hit;
    if (!ray_setup(p.m, ray, ry, hit)) return;
    if (!hit) return;
    const float4 ds = reinterpret_cast<const float4*>(p.dist_state)[ray];
    DistBwdSampler<L> smp{p.m.g, p.m.opts.attn_mode, p.m.opts.t_term, gate_smem + threadIdx.x, 1.0f, 0.0f, 0.0f,
                          0.0f, ds.y, ds.z, 2.0f * ds.x, p.scale, p.g_tables, p.g_coarse};
    int n_march = 0, n_samp = 0;
    march_loop(p.m, ry, smp, n_march, n_samp);
}

template <int L>
void launch_dist(bool backward, const DistParams& p, dim3 grid, cudaStream_t st) {
    const size_t shm = (size_t)2 * L * 128 * sizeof(float);
    if (backward) distortion_backward_kernel<L><<<grid, 128, shm, st>>>(p);
    else distortion_kernel<L, NGPRT_AGG_SEPARATE_V><<<grid, 128, shm, st>>>(p);
}

}  // namespace

int32_t make_grid(const ngprt_scene* s, Grid& g, const char* fn);
int32_t make_occ(const ngprt_occ* o, OccView& v, const char* fn);
int32_t check_opts(const ngprt_render_opts* o, const char* fn);
int32_t check_agg(const ngprt_scene* s, const ngprt_render_opts* o, bool forward_only_ok, const char* fn);
int32_t setup_rays(MarchParams& p, const ngprt_camera* cams, int32_t n_cams, const int32_t* pixel_ids,
                   const float* rays_o, const float* rays_d, int64_t n_rays, dim3& grid, const char* fn);

static int32_t run_distortion(bool backward, const ngprt_scene* scene, const ngprt_occ* occ, const ngprt_camera* cams,
                              int32_t n_cams, const int32_t* pixel_ids, const float* rays_o, const float* rays_d,
                              int64_t n_rays, const ngprt_render_opts* opts, float* dist_state, float scale,
                              float* loss, float* g_tables, float* g_coarse, float* g_attn_inv, float* g_agg_mlp,
                              void* workspace, size_t ws_bytes, void* stream, const char* fn) {
    DistParams p;
    memset(&p, 0, sizeof p);
    int32_t rc;
    if ((rc = make_grid(scene, p.m.g, fn)) != NGPRT_OK) return rc;
    NGPRT_REQUIRE(scene->coarse_index == nullptr, "%s: gradients need the dense coarse grid (coarse_index is set)", fn);
    if ((rc = make_occ(occ, p.m.occ, fn)) != NGPRT_OK) return rc;
    if ((rc = check_opts(opts, fn)) != NGPRT_OK) return rc;
    if ((rc = check_agg(scene, opts, true, fn)) != NGPRT_OK) return rc;
    NGPRT_REQUIRE(n_rays >= 0, "%s: n_rays=%lld", fn, (long long)n_rays);
    NGPRT_REQUIRE(scene->table_dtype == NGPRT_F32, "%s: needs F32 tables", fn);
    const int agg = scene->aggregation;
    const int L = scene->L;
    if (!(L == 1 || L == 2 || L == 3 || L == 4 || L == 8 || L == 16) ||
        (agg != NGPRT_AGG_SEPARATE_V && !(L == 2 || L == 4 || L == 16))) {
        set_error("%s: no kernel for L=%d (built: 1, 2, 3, 4, 8, 16)", fn, L);
        return NGPRT_ERR_UNSUPPORTED;
    }
    dim3 grid;
    if ((rc = setup_rays(p.m, cams, n_cams, pixel_ids, rays_o, rays_d, n_rays, grid, fn)) != NGPRT_OK) return rc;
    if (n_rays == 0) return NGPRT_OK;
    NGPRT_REQUIRE(dist_state != nullptr && ((uintptr_t)dist_state & 15) == 0,
                  "%s: dist_state must be a 16-byte aligned [n][4] buffer", fn);
    const bool inv = agg == NGPRT_AGG_SEPARATE_INV || agg == NGPRT_AGG_SHARED_INV;
    if (backward) {
        NGPRT_REQUIRE(g_tables && g_coarse, "%s: g_tables and g_coarse are required", fn);
        NGPRT_REQUIRE(!inv || g_attn_inv, "%s: g_attn_inv is NULL (aggregation %d)", fn, agg);
        NGPRT_REQUIRE(agg != NGPRT_AGG_MLP || g_agg_mlp, "%s: g_agg_mlp is NULL (the MLP aggregation)", fn);
        const size_t need = ngprt_distortion_backward_workspace_bytes(scene, opts, n_rays);
        if (need > 0 && (!workspace || ws_bytes < need || ((uintptr_t)workspace & 15) != 0)) {
            set_error("%s: workspace %zu bytes < %zu needed (16-byte aligned)", fn, ws_bytes, need);
            return NGPRT_ERR_WORKSPACE;
        }
    }
    p.m.opts = *opts;
    p.dist_state = dist_state;
    p.scale = scale;
    p.loss = loss;
    p.g_tables = g_tables;
    p.g_coarse = g_coarse;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (agg != NGPRT_AGG_SEPARATE_V) {
        if (!backward) {
            launch_dist_fwd_agg(L, agg, p, grid, st);
            return cuda_status(fn);
        }
        // the reverse march in distortion mode: colour cotangents 0, dL/dsigma from Eq. S2
        MarchBwdParams b;
        memset(&b, 0, sizeof b);
        b.m = p.m;
        b.g_tables = g_tables;
        b.g_coarse = g_coarse;
        b.g_attn_inv = inv ? g_attn_inv : nullptr;
        b.dist_state = dist_state;
        b.dist_scale = scale;
        if (agg == NGPRT_AGG_MLP) {
            char* w = static_cast<char*>(workspace);
            b.n_records = reinterpret_cast<int32_t*>(w);
            b.records = reinterpret_cast<float*>(w + 256);
            b.rec_capacity = n_rays * (int64_t)opts->max_samples;
            cudaMemsetAsync(b.n_records, 0, sizeof(int32_t), st);
        }
        launch_dist_bwd_agg(L, agg, b, grid, st);
        if (agg == NGPRT_AGG_MLP) launch_bwd_agg_mlp_wgrad(L, b, scene->agg_mlp, g_agg_mlp, st);
        return cuda_status(fn);
    }
    switch (L) {
        case 1: launch_dist<1>(backward, p, grid, st); break;
        case 2: launch_dist<2>(backward, p, grid, st); break;
        case 3: launch_dist<3>(backward, p, grid, st); break;
        case 4: launch_dist<4>(backward, p, grid, st); break;
        case 8: launch_dist<8>(backward, p, grid, st); break;
        default: launch_dist<16>(backward, p, grid, st); break;
    }
    return cuda_status(fn);
}

}  // namespace ngprt

using namespace ngprt;

extern "C" int32_t ngprt_distortion_loss(const ngprt_scene* scene, const ngprt_occ* occ, const ngprt_camera* cams,
                                         int32_t n_cams, const int32_t* pixel_ids, const float* rays_o,
                                         const float* rays_d, int64_t n_rays, const ngprt_render_opts* opts,
                                         float scale, float* dist_state, float* loss, void* stream) {
    return run_distortion(false, scene, occ, cams, n_cams, pixel_ids, rays_o, rays_d, n_rays, opts, dist_state, scale,
                          loss, nullptr, nullptr, nullptr, nullptr, nullptr, 0, stream, "ngprt_distortion_loss");
}

extern "C" size_t ngprt_distortion_backward_workspace_bytes(const ngprt_scene* scene, const ngprt_render_opts* opts,
                                                            int64_t n_rays) {
    if (!scene || n_rays < 0 || scene->aggregation != NGPRT_AGG_MLP) return 0;
    const int64_t ms = opts && opts->max_samples > 0 ? opts->max_samples : 0;
    return 256 + (size_t)n_rays * (size_t)ms * (size_t)(kNFeat * (scene->L + 1)) * sizeof(float);
}

extern "C" int32_t ngprt_distortion_backward(const ngprt_scene* scene, const ngprt_occ* occ, const ngprt_camera* cams,
                                             int32_t n_cams, const int32_t* pixel_ids, const float* rays_o,
                                             const float* rays_d, int64_t n_rays, const ngprt_render_opts* opts,
                                             const float* dist_state, float scale, float* g_tables, float* g_coarse,
                                             float* g_attn_inv, float* g_agg_mlp, void* workspace, size_t ws_bytes,
                                             void* stream) {
    return run_distortion(true, scene, occ, cams, n_cams, pixel_ids, rays_o, rays_d, n_rays, opts,
                          const_cast<float*>(dist_state), scale, nullptr, g_tables, g_coarse, g_attn_inv, g_agg_mlp,
                          workspace, ws_bytes, stream, "ngprt_distortion_backward");
}
