// backward.cu -- reverse pass of the render (Eq. 2, 5, 8; Sec. S2.1 activations).
//
// Kernel 1 (shade_backward_kernel): per ray, the deferred MLP_psi and colour
// sigmoid again from the stored composite state, then their reverse pass: the
// cotangents of C_d, F, A and depth go to a per-ray record, and the MLP weight
// gradients, sums over rays of outer products, are formed tile by tile from shared
// memory and added to g_mlp once per block.
// Kernel 2 (march_backward_kernel, backward_march.cuh): per ray, the march again
// and the reverse of compositing, gates and trilinear gathers, added atomically to
// the table, coarse-grid and invariant-logit gradients.
#include "backward_march.cuh"

namespace ngprt {
namespace {

struct ShadeBwdParams {
    const float* state;
    const float* w;
    const float* d_rgb;
    const float* d_depth;
    const float* d_opacity;
    float bg[3];
    int64_t n;
    float* cot;
    float* g_mlp;
};

// Shared-memory layout of the tiled deferred-MLP reverse pass: the weights, then
// per tile of 128 rays the inputs X [128][25] and the hidden activations (later
// their gradients) H1, H2 [128][W + 1] (odd row strides: a thread reading its own
// row and a thread reading one column of all rows are both bank-conflict free), and
// the colour-logit gradients GZ [128][4].
template <int WIDTH, int LAYERS>
struct ShadeTile {
    static constexpr int n_w0 = WIDTH * kMlpIn;
    static constexpr int n_mid = (LAYERS - 2) * WIDTH * WIDTH;
    static constexpr int n_last = 3 * WIDTH;
    static constexpr int n_all = n_w0 + n_mid + n_last;
    static constexpr int kRays = 128;
    static constexpr int kXs = 25;
    static constexpr int kHs = WIDTH + 1;
    static constexpr int n_smem = n_all + kRays * kXs + kRays * kHs * (LAYERS - 1) + kRays * 4;
    static constexpr int TO = WIDTH / 16, TI = WIDTH / 8;  // dW_mid tile per thread (16 x 8 tiles)
    static constexpr int T0 = WIDTH / 16;                  // dW0 tile per thread: T0 outputs x 3 inputs
};

// Kernel 1: per ray (one thread), the deferred MLP_psi and colour sigmoid again from
// the stored composite state, then their reverse pass; the cotangents of C_d, F, A
// and depth go to a per-ray record.  The weight gradients are sums over rays of
// outer products, dW = sum_r g_r h_r^T: after each layer's per-ray phase the block
// multiplies the tile's gradients and activations from shared memory, each thread
// accumulating a fixed tile of dW in registers over all the block's ray tiles, and
// adds it to g_mlp once at the end.
template <int WIDTH, int LAYERS>
__global__ void __launch_bounds__(128) shade_backward_kernel(const __grid_constant__ ShadeBwdParams p) {
    using K = ShadeTile<WIDTH, LAYERS>;
    extern __shared__ __align__(16) float sm[];
    float* ws = sm;
    float* X = ws + K::n_all;
    float* H1 = X + K::kRays * K::kXs;
    float* H2 = H1 + K::kRays * K::kHs;  // used when LAYERS == 3
    float* GZ = H1 + K::kRays * K::kHs * (LAYERS - 1);
    float* Hl = LAYERS == 3 ? H2 : H1;   // input of the last layer
    for (int i = threadIdx.x; i < K::n_all; i += blockDim.x) ws[i] = p.w[i];
    const float* w0 = ws;
    const float* wm = ws + K::n_w0;
    const float* wl = ws + K::n_w0 + K::n_mid;
    const int t = threadIdx.x;
    const int ob = t >> 3, ib = t & 7;
    float dmid[K::TO][K::TI];
    float d0[K::T0][3];
    float dl[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int a = 0; a < K::TO; ++a)
#pragma unroll
        for (int b = 0; b < K::TI; ++b) dmid[a][b] = 0.0f;
#pragma unroll
    for (int a = 0; a < K::T0; ++a) d0[a][0] = d0[a][1] = d0[a][2] = 0.0f;
    const int64_t n_tiles = (p.n + K::kRays - 1) / K::kRays;
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        __syncthreads();  // weights loaded; the previous tile's readers are done
        const int64_t ray = tile * K::kRays + t;
        const bool active = ray < p.n;
        // ---- forward again (inactive rays carry zeros: they add nothing to dW)
        float x[23];
        float A = 0.0f, depth = 0.0f;
        float Cd[3] = {0.0f, 0.0f, 0.0f}, F[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int i = 0; i < 23; ++i) x[i] = 0.0f;
        if (active) {
            const float4* s4 = reinterpret_cast<const float4*>(p.state + ray * NGPRT_STATE_FLOATS);
            const float4 q0 = s4[0], q1 = s4[1], q2 = s4[2];
            Cd[0] = q0.x; Cd[1] = q0.y; Cd[2] = q0.z;
            F[0] = q0.w; F[1] = q1.x; F[2] = q1.y; F[3] = q1.z;
            A = q1.w;
            depth = q2.x;
            x[0] = Cd[0]; x[1] = Cd[1]; x[2] = Cd[2];
            x[3] = F[0]; x[4] = F[1]; x[5] = F[2]; x[6] = F[3];
            sh16(q2.y, q2.z, q2.w, x + 7);
        }
#pragma unroll
        for (int i = 0; i < 23; ++i) X[t * K::kXs + i] = x[i];
        float h[WIDTH];
#pragma unroll
        for (int o = 0; o < WIDTH; ++o) {
            float acc = 0.0f;
#pragma unroll
            for (int i = 0; i < 23; ++i) acc = fmaf(w0[o * kMlpIn + i], x[i], acc);
            h[o] = fmaxf(acc, 0.0f);
            H1[t * K::kHs + o] = h[o];
        }
        float out[3] = {0.0f, 0.0f, 0.0f};
        if constexpr (LAYERS == 3) {
#pragma unroll 4
            for (int o = 0; o < WIDTH; ++o) {
                float acc = 0.0f;
#pragma unroll
                for (int i = 0; i < WIDTH; ++i) acc = fmaf(wm[o * WIDTH + i], h[i], acc);
                const float h2 = fmaxf(acc, 0.0f);
                H2[t * K::kHs + o] = h2;
#pragma unroll
                for (int k = 0; k < 3; ++k) out[k] = fmaf(wl[k * WIDTH + o], h2, out[k]);
            }
        } else {
#pragma unroll
            for (int o = 0; o < WIDTH; ++o)
#pragma unroll
                for (int k = 0; k < 3; ++k) out[k] = fmaf(wl[k * WIDTH + o], h[o], out[k]);
        }
        // ---- colour: rgb = A sigmoid(z) + (1 - A) bg, z = C_d + out
        float gz[3] = {0.0f, 0.0f, 0.0f}, gA = 0.0f;
        if (active) {
            gA = p.d_opacity ? p.d_opacity[ray] : 0.0f;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float sg = sigmoidf_(Cd[k] + out[k]);
                const float gr = p.d_rgb[3 * ray + k];
                gz[k] = gr * A * sg * (1.0f - sg);
                gA += gr * (sg - p.bg[k]);
            }
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) GZ[t * 4 + k] = gz[k];
        __syncthreads();
        // ---- dW_last[k][i] += sum_r gz_r[k] h_r[i] (thread i < WIDTH owns column i)
        if (t < WIDTH) {
#pragma unroll 4
            for (int r = 0; r < K::kRays; ++r) {
                const float hv = Hl[r * K::kHs + t];
#pragma unroll
                for (int k = 0; k < 3; ++k) dl[k] = fmaf(GZ[r * 4 + k], hv, dl[k]);
            }
        }
        __syncthreads();
        // ---- gradient of the last hidden pre-activation, into the thread's own row
        float g[WIDTH];
#pragma unroll
        for (int i = 0; i < WIDTH; ++i) {
            float acc = 0.0f;
#pragma unroll
            for (int k = 0; k < 3; ++k) acc = fmaf(wl[k * WIDTH + i], gz[k], acc);
            g[i] = Hl[t * K::kHs + i] > 0.0f ? acc : 0.0f;
        }
        if constexpr (LAYERS == 3) {
#pragma unroll
            for (int i = 0; i < WIDTH; ++i) H2[t * K::kHs + i] = g[i];
            __syncthreads();
            // dW_mid[o][i] += sum_r g2_r[o] h1_r[i] over this thread's TO x TI tile
#pragma unroll 2
            for (int r = 0; r < K::kRays; ++r) {
                float go[K::TO], hi[K::TI];
#pragma unroll
                for (int a = 0; a < K::TO; ++a) go[a] = H2[r * K::kHs + ob * K::TO + a];
#pragma unroll
                for (int b = 0; b < K::TI; ++b) hi[b] = H1[r * K::kHs + ib * K::TI + b];
#pragma unroll
                for (int a = 0; a < K::TO; ++a)
#pragma unroll
                    for (int b = 0; b < K::TI; ++b) dmid[a][b] = fmaf(go[a], hi[b], dmid[a][b]);
            }
            __syncthreads();
            // g1 = (W_mid^T g2) * [a1 > 0]
            float g1[WIDTH];
#pragma unroll
            for (int i = 0; i < WIDTH; ++i) g1[i] = 0.0f;
#pragma unroll 4
            for (int o = 0; o < WIDTH; ++o)
#pragma unroll
                for (int i = 0; i < WIDTH; ++i) g1[i] = fmaf(wm[o * WIDTH + i], g[o], g1[i]);
#pragma unroll
            for (int i = 0; i < WIDTH; ++i) g[i] = H1[t * K::kHs + i] > 0.0f ? g1[i] : 0.0f;
        }
        // first-layer gradient into the thread's own H1 row (its readers passed a barrier)
#pragma unroll
        for (int i = 0; i < WIDTH; ++i) H1[t * K::kHs + i] = g[i];
        if (active) {
            float gx[7];
#pragma unroll
            for (int i = 0; i < 7; ++i) {
                float acc = 0.0f;
#pragma unroll
                for (int o = 0; o < WIDTH; ++o) acc = fmaf(w0[o * kMlpIn + i], g[o], acc);
                gx[i] = acc;
            }
            const float gCd[3] = {gz[0] + gx[0], gz[1] + gx[1], gz[2] + gx[2]};
            const float gD = p.d_depth ? p.d_depth[ray] : 0.0f;
            const float S = gCd[0] * Cd[0] + gCd[1] * Cd[1] + gCd[2] * Cd[2] + gx[3] * F[0] + gx[4] * F[1] +
                            gx[5] * F[2] + gx[6] * F[3] + gA * A + gD * depth;
            float4* c4 = reinterpret_cast<float4*>(p.cot + ray * kCotFloats);
            c4[0] = make_float4(gCd[0], gCd[1], gCd[2], gx[3]);
            c4[1] = make_float4(gx[4], gx[5], gx[6], gA);
            c4[2] = make_float4(gD, S, 0.0f, 0.0f);
        }
        __syncthreads();
        // ---- dW0[o][i] += sum_r g1_r[o] x_r[i], i < 23 (T0 outputs x 3 inputs per thread)
#pragma unroll 2
        for (int r = 0; r < K::kRays; ++r) {
            float go[K::T0];
#pragma unroll
            for (int a = 0; a < K::T0; ++a) go[a] = H1[r * K::kHs + ob * K::T0 + a];
            const float x0 = X[r * K::kXs + ib * 3], x1 = X[r * K::kXs + ib * 3 + 1],
                        x2 = X[r * K::kXs + ib * 3 + 2];
#pragma unroll
            for (int a = 0; a < K::T0; ++a) {
                d0[a][0] = fmaf(go[a], x0, d0[a][0]);
                d0[a][1] = fmaf(go[a], x1, d0[a][1]);
                d0[a][2] = fmaf(go[a], x2, d0[a][2]);
            }
        }
    }
    // ---- the block's sums into g_mlp
    if constexpr (LAYERS == 3) {
#pragma unroll
        for (int a = 0; a < K::TO; ++a)
#pragma unroll
            for (int b = 0; b < K::TI; ++b)
                atomicAdd(&p.g_mlp[K::n_w0 + (ob * K::TO + a) * WIDTH + ib * K::TI + b], dmid[a][b]);
    }
#pragma unroll
    for (int a = 0; a < K::T0; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
            if (ib * 3 + b < 23) atomicAdd(&p.g_mlp[(ob * K::T0 + a) * kMlpIn + ib * 3 + b], d0[a][b]);
    if (t < WIDTH) {
#pragma unroll
        for (int k = 0; k < 3; ++k) atomicAdd(&p.g_mlp[K::n_w0 + K::n_mid + k * WIDTH + t], dl[k]);
    }
}

template <int WIDTH, int LAYERS>
void launch_shade_bwd(const ShadeBwdParams& s, cudaStream_t st) {
    using K = ShadeTile<WIDTH, LAYERS>;
    const size_t smem = (size_t)K::n_smem * sizeof(float);
    // the opt-in shared-memory size (over 48 KB) is a per-device function attribute
    cudaFuncSetAttribute(shade_backward_kernel<WIDTH, LAYERS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int64_t tiles = (s.n + K::kRays - 1) / K::kRays;
    const unsigned blocks = (unsigned)(tiles < 152 * 2 ? tiles : 152 * 2);
    shade_backward_kernel<WIDTH, LAYERS><<<blocks, 128, smem, st>>>(s);
}

}  // namespace

int32_t make_grid(const ngprt_scene* s, Grid& g, const char* fn);
int32_t make_occ(const ngprt_occ* o, OccView& v, const char* fn);
int32_t check_opts(const ngprt_render_opts* o, const char* fn);
int32_t setup_rays(MarchParams& p, const ngprt_camera* cams, int32_t n_cams, const int32_t* pixel_ids,
                   const float* rays_o, const float* rays_d, int64_t n_rays, dim3& grid, const char* fn);
bool march_supports(int L);
bool mlp_supports(int width, int layers);

}  // namespace ngprt

using namespace ngprt;

// Per-ray cotangent records at the head of the reverse pass's workspace (256-byte
// rounded, plus 256 bytes of slack as for the forward's state).
static size_t cot_bytes(int64_t n) {
    return ((size_t)n * kCotFloats * sizeof(float) + 255) / 256 * 256 + 256;
}

extern "C" size_t ngprt_render_backward_workspace_bytes(const ngprt_scene* scene, const ngprt_render_opts* opts,
                                                        int64_t n_rays) {
    if (!scene || n_rays < 0) return 0;
    size_t b = cot_bytes(n_rays);
    if (scene->aggregation == NGPRT_AGG_MLP) {
        const int64_t ms = opts && opts->max_samples > 0 ? opts->max_samples : 0;
        b += 256 + (size_t)n_rays * (size_t)ms * (size_t)(kNFeat * (scene->L + 1)) * sizeof(float);
    }
    return b;
}

extern "C" int32_t ngprt_render_backward(const ngprt_scene* scene, const ngprt_occ* occ, const ngprt_camera* cams,
                                         int32_t n_cams, const int32_t* pixel_ids, const float* rays_o,
                                         const float* rays_d, int64_t n_rays, const ngprt_render_opts* opts,
                                         const float* ray_state, const float* d_rgb, const float* d_depth,
                                         const float* d_opacity, float* g_tables, float* g_coarse, float* g_mlp,
                                         float* g_attn_inv, float* g_agg_mlp, void* workspace, size_t ws_bytes,
                                         void* stream) {
    const char* fn = "ngprt_render_backward";
    MarchBwdParams p;
    memset(&p, 0, sizeof p);
    int32_t rc;
    if ((rc = make_grid(scene, p.m.g, fn)) != NGPRT_OK) return rc;
    NGPRT_REQUIRE(scene->coarse_index == nullptr, "%s: gradients need the dense coarse grid (coarse_index is set)", fn);
    if ((rc = make_occ(occ, p.m.occ, fn)) != NGPRT_OK) return rc;
    if ((rc = check_opts(opts, fn)) != NGPRT_OK) return rc;
    NGPRT_REQUIRE(n_rays >= 0, "%s: n_rays=%lld", fn, (long long)n_rays);
    NGPRT_REQUIRE(scene->table_dtype == NGPRT_F32 && scene->mlp_dtype == NGPRT_F32,
                  "%s: gradients need F32 tables and F32 MLP weights", fn);
    const int agg = scene->aggregation;
    if (agg == NGPRT_AGG_SEPARATE_V) {
        if (!march_supports(scene->L)) {
            set_error("%s: no backward kernel for L=%d (built: 1, 2, 3, 4, 8, 16)", fn, scene->L);
            return NGPRT_ERR_UNSUPPORTED;
        }
    } else {
        NGPRT_REQUIRE(opts->attn_mode == 0, "%s: attn_mode=%d applies to the SEPARATE_V aggregation only", fn,
                      opts->attn_mode);
        if (!march_bwd_agg_supports(scene->L)) {
            set_error("%s: aggregation %d has no backward kernel for L=%d (built: 2, 4, 16)", fn, agg, scene->L);
            return NGPRT_ERR_UNSUPPORTED;
        }
    }
    if (!mlp_supports(scene->mlp_width, scene->mlp_layers)) {
        set_error("%s: MLP %d layers x %d not built", fn, scene->mlp_layers, scene->mlp_width);
        return NGPRT_ERR_UNSUPPORTED;
    }
    dim3 grid;
    if ((rc = setup_rays(p.m, cams, n_cams, pixel_ids, rays_o, rays_d, n_rays, grid, fn)) != NGPRT_OK) return rc;
    if (n_rays == 0) return NGPRT_OK;
    NGPRT_REQUIRE(ray_state && d_rgb && g_tables && g_coarse && g_mlp, "%s: NULL buffer", fn);
    const bool inv = agg == NGPRT_AGG_SEPARATE_INV || agg == NGPRT_AGG_SHARED_INV;
    NGPRT_REQUIRE(!inv || g_attn_inv, "%s: g_attn_inv is NULL (aggregation %d)", fn, agg);
    NGPRT_REQUIRE(agg != NGPRT_AGG_MLP || (g_agg_mlp && ((uintptr_t)g_agg_mlp & 3) == 0),
                  "%s: g_agg_mlp is NULL (the MLP aggregation)", fn);
    NGPRT_REQUIRE(((uintptr_t)g_tables & 15) == 0 && ((uintptr_t)g_coarse & 15) == 0 && ((uintptr_t)ray_state & 15) == 0,
                  "%s: g_tables, g_coarse, ray_state must be 16-byte aligned", fn);
    const size_t need = ngprt_render_backward_workspace_bytes(scene, opts, n_rays);
    if (!workspace || ws_bytes < need) {
        set_error("%s: workspace %zu bytes < %zu needed", fn, ws_bytes, need);
        return NGPRT_ERR_WORKSPACE;
    }
    NGPRT_REQUIRE(((uintptr_t)workspace & 15) == 0, "%s: workspace must be 16-byte aligned", fn);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    float* cot = static_cast<float*>(workspace);
    ShadeBwdParams s;
    s.state = ray_state;
    s.w = static_cast<const float*>(scene->mlp_w);
    s.d_rgb = d_rgb;
    s.d_depth = d_depth;
    s.d_opacity = d_opacity;
    s.bg[0] = opts->bg[0];
    s.bg[1] = opts->bg[1];
    s.bg[2] = opts->bg[2];
    s.n = n_rays;
    s.cot = cot;
    s.g_mlp = g_mlp;
    const int W = scene->mlp_width, Ly = scene->mlp_layers;
    if (Ly == 2) {
        if (W == 16) launch_shade_bwd<16, 2>(s, st);
        else if (W == 32) launch_shade_bwd<32, 2>(s, st);
        else launch_shade_bwd<64, 2>(s, st);
    } else {
        if (W == 16) launch_shade_bwd<16, 3>(s, st);
        else if (W == 32) launch_shade_bwd<32, 3>(s, st);
        else launch_shade_bwd<64, 3>(s, st);
    }
    p.m.opts = *opts;
    p.m.t_interval = nullptr;
    p.state = ray_state;
    p.cot = cot;
    p.g_tables = g_tables;
    p.g_coarse = g_coarse;
    p.g_attn_inv = inv ? g_attn_inv : nullptr;
    if (agg == NGPRT_AGG_MLP) {
        // after the per-ray cotangents: the record count, then n_rays x max_samples records
        char* w = static_cast<char*>(workspace) + cot_bytes(n_rays);
        p.n_records = reinterpret_cast<int32_t*>(w);
        p.records = reinterpret_cast<float*>(w + 256);
        p.rec_capacity = n_rays * (int64_t)opts->max_samples;
        cudaMemsetAsync(p.n_records, 0, sizeof(int32_t), st);
    }
    if (agg != NGPRT_AGG_SEPARATE_V) {
        launch_bwd_agg(scene->L, agg, p, grid, st);
        if (agg == NGPRT_AGG_MLP)
            launch_bwd_agg_mlp_wgrad(scene->L, p, scene->agg_mlp, g_agg_mlp, st);
        return cuda_status(fn);
    }
    switch (scene->L) {
        case 1: launch_bwd<1, NGPRT_AGG_SEPARATE_V>(p, grid, st); break;
        case 2: launch_bwd<2, NGPRT_AGG_SEPARATE_V>(p, grid, st); break;
        case 3: launch_bwd<3, NGPRT_AGG_SEPARATE_V>(p, grid, st); break;
        case 4: launch_bwd<4, NGPRT_AGG_SEPARATE_V>(p, grid, st); break;
        case 8: launch_bwd<8, NGPRT_AGG_SEPARATE_V>(p, grid, st); break;
        default: launch_bwd<16, NGPRT_AGG_SEPARATE_V>(p, grid, st); break;
    }
    return cuda_status(fn);
}
