// render.cu -- forward render of NGP-RT (Eq. 2, 5, 6, 8, 9; Sec. 3.3, S2.5).
//
// Kernel 1 (march_kernel): one ray per thread, warps laid over small pixel tiles so
// that a warp's rays sample neighbouring points (shared cache lines at the coarse
// and middle levels).  Per marching point: coarse-to-fine occupancy test; empty ->
// occupancy step s_O or distance step v*G (Eq. 9); occupied -> coarse fetch of
// F~ and the attention logits, 8-corner gathers of every fine level, attention
// fusion (Eq. 8), alpha compositing (Eq. 2/5) and early termination.  The per-ray
// composite state goes to `state`.
// Kernel 2 (mlp_kernel): the deferred MLP_psi (Eq. 5) per ray with the weights in
// shared memory, colour sigmoid, background.
#include "march.cuh"

namespace ngprt {

// Proposal training targets (per ray): with the final opacity A of the plain
// render, the position of the first sample whose cumulative weight exceeds
// 0.005 A, the end (t + delta) of the first sample whose cumulative weight reaches
// 0.995 A, and A.  The samples are the forward's (same march, same compositing).
template <int L, int DT>
struct TargetSampler {
    ForwardSampler<L, DT> fw;
    float A_final, t_near, t_far;
    bool got_near, got_far;
    __device__ __forceinline__ bool sample(const float u[3], float t, float delta) {
        const bool stop = fw.sample(u, t, delta);
        if (!got_near && fw.A > 0.005f * A_final) {
            t_near = t;
            got_near = true;
        }
        if (!got_far && fw.A >= 0.995f * A_final) {
            t_far = t + delta;
            got_far = true;
        }
        t_far = got_far ? t_far : t + delta;
        return stop;
    }
};

template <int L, int DT>
__global__ void __launch_bounds__(128, march_min_blocks<L, DT>()) targets_kernel(const __grid_constant__ MarchParams p,
                                                                                float* targets) {
    extern __shared__ float gate_smem[];
    int64_t ray;
    Ray ry;
    bool hit;
    if (!ray_setup(p, ray, ry, hit)) return;
    const float A = p.state[ray * NGPRT_STATE_FLOATS + 7];
    TargetSampler<L, DT> smp{ForwardSampler<L, DT>(p.g, p.opts.attn_mode, p.opts.t_term, gate_smem + threadIdx.x), A,
                             0.0f, 0.0f, false, false};
    int n_march = 0, n_samp = 0;
    if (hit) march_loop(p, ry, smp, n_march, n_samp);
    if (n_samp == 0) smp.t_far = 0.0f;
    targets[3 * ray] = smp.t_near;
    targets[3 * ray + 1] = smp.t_far;
    targets[3 * ray + 2] = A;
}

// ---------------------------------------------------------------- deferred MLP

struct MlpParams {
    const float* state;
    const float* w;
    float bg[3];
    int64_t n;
    float* rgb;
    float* depth;
    float* opacity;
};

template <int WIDTH, int LAYERS>
__global__ void __launch_bounds__(128) mlp_f32_kernel(const __grid_constant__ MlpParams p) {
    constexpr int n_w0 = WIDTH * kMlpIn;
    constexpr int n_mid = (LAYERS - 2) * WIDTH * WIDTH;
    constexpr int n_last = 3 * WIDTH;
    constexpr int n_all = n_w0 + n_mid + n_last;
    __shared__ __align__(16) float ws[n_all];
    for (int i = threadIdx.x; i < n_all / 4; i += blockDim.x)
        reinterpret_cast<float4*>(ws)[i] = __ldg(reinterpret_cast<const float4*>(p.w) + i);
    __syncthreads();
    const int64_t ray = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (ray >= p.n) return;
    const float4* s4 = reinterpret_cast<const float4*>(p.state + ray * NGPRT_STATE_FLOATS);
    const float4 q0 = s4[0], q1 = s4[1], q2 = s4[2];
    float x[24];
    x[0] = q0.x; x[1] = q0.y; x[2] = q0.z; x[3] = q0.w;
    x[4] = q1.x; x[5] = q1.y; x[6] = q1.z;
    const float A = q1.w, depth = q2.x;
    sh16(q2.y, q2.z, q2.w, x + 7);
    x[23] = 0.0f;
    // layer 0: 23 real inputs (the zero padding contributes nothing)
    float h[WIDTH];
#pragma unroll
    for (int o = 0; o < WIDTH; ++o) {
        const float4* wr = reinterpret_cast<const float4*>(ws + o * kMlpIn);
        float acc = 0.0f;
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            const float4 wv = wr[i];
            acc = fmaf(wv.x, x[4 * i], acc);
            acc = fmaf(wv.y, x[4 * i + 1], acc);
            acc = fmaf(wv.z, x[4 * i + 2], acc);
            acc = fmaf(wv.w, x[4 * i + 3], acc);
        }
        h[o] = fmaxf(acc, 0.0f);
    }
    float out[3] = {0.0f, 0.0f, 0.0f};
    const float* wl = ws + n_w0 + n_mid;
    if constexpr (LAYERS == 2) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            float acc = 0.0f;
#pragma unroll
            for (int i = 0; i < WIDTH; ++i) acc = fmaf(wl[k * WIDTH + i], h[i], acc);
            out[k] = acc;
        }
    } else {
        static_assert(LAYERS == 3, "MLP depth 2 or 3");
        const float* wm = ws + n_w0;
#pragma unroll 4
        for (int o = 0; o < WIDTH; ++o) {
            const float4* wr = reinterpret_cast<const float4*>(wm + o * WIDTH);
            float acc = 0.0f;
#pragma unroll
            for (int i = 0; i < WIDTH / 4; ++i) {
                const float4 wv = wr[i];
                acc = fmaf(wv.x, h[4 * i], acc);
                acc = fmaf(wv.y, h[4 * i + 1], acc);
                acc = fmaf(wv.z, h[4 * i + 2], acc);
                acc = fmaf(wv.w, h[4 * i + 3], acc);
            }
            acc = fmaxf(acc, 0.0f);
#pragma unroll
            for (int k = 0; k < 3; ++k) out[k] = fmaf(wl[k * WIDTH + o], acc, out[k]);
        }
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float z = x[k] + out[k];
        const float sg = sigmoidf_(z);
        p.rgb[3 * ray + k] = A * sg + (1.0f - A) * p.bg[k];
    }
    if (p.depth) p.depth[ray] = depth;
    if (p.opacity) p.opacity[ray] = A;
}

// ---------------------------------------------------------------- test hook

struct IndexParams {
    Grid g;
    const float* u;
    int64_t n;
    uint32_t* out;
};

__global__ void grid_indices_kernel(const __grid_constant__ IndexParams p) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.n) return;
    const float u[3] = {p.u[3 * i], p.u[3 * i + 1], p.u[3 * i + 2]};
    for (int l = 0; l < p.g.L; ++l) {
        int b[3];
        float w[3];
        for (int a = 0; a < 3; ++a) grid_cell(u[a], p.g.N[l], b[a], w[a]);
        for (int c = 0; c < 8; ++c)
            p.out[(i * p.g.L + l) * 8 + c] = level_row(p.g, l, (uint32_t)(b[0] + (c & 1)), (uint32_t)(b[1] + ((c >> 1) & 1)),
                                                       (uint32_t)(b[2] + ((c >> 2) & 1)));
    }
}

// ------------------------------------------------------------------- host side

int32_t make_grid(const ngprt_scene* s, Grid& g, const char* fn);
int32_t make_occ(const ngprt_occ* o, OccView& v, const char* fn);

template <int L>
void launch_march(int dt, const MarchParams& p, dim3 grid, cudaStream_t st) {
    launch_march_kernel<L, NGPRT_AGG_SEPARATE_V>(dt, p, grid, st);
}

template <int L>
void launch_targets(int dt, const MarchParams& p, dim3 grid, cudaStream_t st, float* targets) {
    const size_t shm = (size_t)2 * L * 128 * sizeof(float);
    if (dt == NGPRT_F32) targets_kernel<L, NGPRT_F32><<<grid, 128, shm, st>>>(p, targets);
    else if (dt == NGPRT_F16) targets_kernel<L, NGPRT_F16><<<grid, 128, shm, st>>>(p, targets);
    else targets_kernel<L, NGPRT_BF16><<<grid, 128, shm, st>>>(p, targets);
}

bool march_agg_supports(int L);
int32_t launch_march_agg(int L, int dt, int agg, const MarchParams& p, dim3 grid, cudaStream_t st);

bool march_supports(int L, int agg) {
    if (agg != NGPRT_AGG_SEPARATE_V) return march_agg_supports(L);
    return L == 1 || L == 2 || L == 3 || L == 4 || L == 8 || L == 16;
}
bool march_supports(int L) { return march_supports(L, NGPRT_AGG_SEPARATE_V); }

int32_t launch_march_any(int L, int dt, int agg, const MarchParams& p, dim3 grid, cudaStream_t st) {
    if (agg != NGPRT_AGG_SEPARATE_V) return launch_march_agg(L, dt, agg, p, grid, st);
    switch (L) {
        case 1: launch_march<1>(dt, p, grid, st); break;
        case 2: launch_march<2>(dt, p, grid, st); break;
        case 3: launch_march<3>(dt, p, grid, st); break;
        case 4: launch_march<4>(dt, p, grid, st); break;
        case 8: launch_march<8>(dt, p, grid, st); break;
        case 16: launch_march<16>(dt, p, grid, st); break;
        default: set_error("march kernel not built for L=%d", L); return NGPRT_ERR_UNSUPPORTED;
    }
    return NGPRT_OK;
}

bool mlp_supports(int width, int layers) {
    return (layers == 2 || layers == 3) && (width == 16 || width == 32 || width == 64);
}

void launch_mlp(int width, int layers, const MlpParams& p, cudaStream_t st) {
    const unsigned blocks = (unsigned)((p.n + 127) / 128);
    if (layers == 2) {
        if (width == 16) mlp_f32_kernel<16, 2><<<blocks, 128, 0, st>>>(p);
        else if (width == 32) mlp_f32_kernel<32, 2><<<blocks, 128, 0, st>>>(p);
        else mlp_f32_kernel<64, 2><<<blocks, 128, 0, st>>>(p);
    } else {
        if (width == 16) mlp_f32_kernel<16, 3><<<blocks, 128, 0, st>>>(p);
        else if (width == 32) mlp_f32_kernel<32, 3><<<blocks, 128, 0, st>>>(p);
        else mlp_f32_kernel<64, 3><<<blocks, 128, 0, st>>>(p);
    }
}

bool mlp_tc_supports(int width, int layers);
void launch_mlp_tc(int width, int layers, const float* state, const void* w, const float bg[3], int64_t n, float* rgb,
                   float* depth, float* opacity, cudaStream_t st);

// Deferred MLP stage: FP32 weights on the CUDA cores, FP16 weights on the tensor cores.
int32_t launch_shade(const ngprt_scene* scene, const float* state, int64_t n, const float bg[3], float* rgb,
                     float* depth, float* opacity, cudaStream_t st, const char* fn) {
    if (scene->mlp_dtype == NGPRT_F16) {
        if (!mlp_tc_supports(scene->mlp_width, scene->mlp_layers)) {
            set_error("%s: FP16 MLP %d layers x %d not built (2 or 3 layers, width 16/32/64)", fn, scene->mlp_layers,
                      scene->mlp_width);
            return NGPRT_ERR_UNSUPPORTED;
        }
        launch_mlp_tc(scene->mlp_width, scene->mlp_layers, state, scene->mlp_w, bg, n, rgb, depth, opacity, st);
        return NGPRT_OK;
    }
    if (scene->mlp_dtype != NGPRT_F32) {
        set_error("%s: mlp_dtype=%d (F32 or F16)", fn, scene->mlp_dtype);
        return NGPRT_ERR_INVALID_ARG;
    }
    if (!mlp_supports(scene->mlp_width, scene->mlp_layers)) {
        set_error("%s: MLP %d layers x %d not built (2 or 3 layers, width 16/32/64)", fn, scene->mlp_layers,
                  scene->mlp_width);
        return NGPRT_ERR_UNSUPPORTED;
    }
    MlpParams m;
    m.state = state;
    m.w = static_cast<const float*>(scene->mlp_w);
    m.bg[0] = bg[0];
    m.bg[1] = bg[1];
    m.bg[2] = bg[2];
    m.n = n;
    m.rgb = rgb;
    m.depth = depth;
    m.opacity = opacity;
    launch_mlp(scene->mlp_width, scene->mlp_layers, m, st);
    return NGPRT_OK;
}

// Shared by the forward and backward entry points: validates the ray source and
// fills the ray part of MarchParams; returns the launch grid.
int32_t setup_rays(MarchParams& p, const ngprt_camera* cams, int32_t n_cams, const int32_t* pixel_ids,
                   const float* rays_o, const float* rays_d, int64_t n_rays, dim3& grid, const char* fn) {
    p.n_rays = n_rays;
    p.pixel_ids = pixel_ids;
    p.rays_o = rays_o;
    p.rays_d = rays_d;
    p.n_cams = 0;
    p.W = p.H = 1;
    if (cams) {
        NGPRT_REQUIRE(n_cams >= 1 && n_cams <= NGPRT_MAX_CAMERAS, "%s: n_cams=%d not in [1, %d]", fn, n_cams,
                      NGPRT_MAX_CAMERAS);
        const int W = cams[0].W, H = cams[0].H;
        NGPRT_REQUIRE(W > 0 && H > 0, "%s: camera size %dx%d", fn, W, H);
        for (int i = 0; i < n_cams; ++i) {
            NGPRT_REQUIRE(cams[i].W == W && cams[i].H == H, "%s: cameras must share W and H", fn);
            NGPRT_REQUIRE(cams[i].fx != 0.0f && cams[i].fy != 0.0f, "%s: camera %d has a zero focal length", fn, i);
            p.cams.c[i] = cams[i];
        }
        p.n_cams = n_cams;
        p.W = W;
        p.H = H;
        if (pixel_ids) {
            p.mode = 1;
            grid = dim3((unsigned)((n_rays + 127) / 128));
        } else {
            NGPRT_REQUIRE(n_rays == (int64_t)n_cams * W * H, "%s: n_rays=%lld must equal n_cams*W*H=%lld without pixel_ids",
                          fn, (long long)n_rays, (long long)n_cams * W * H);
            p.mode = 0;
            p.tiles_x = (W + kTileW - 1) / kTileW;
            p.tiles_per_view = p.tiles_x * ((H + kTileH - 1) / kTileH);
            const int64_t warps = (int64_t)p.tiles_per_view * n_cams;
            grid = dim3((unsigned)((warps + 3) / 4));
        }
    } else {
        NGPRT_REQUIRE(n_rays == 0 || (rays_o != nullptr && rays_d != nullptr), "%s: need cams or rays_o and rays_d",
                      fn);
        p.mode = 2;
        grid = dim3((unsigned)((n_rays + 127) / 128));
    }
    return NGPRT_OK;
}

// The aggregation forms other than Eq. 8 take attn_mode 0 and are built for L = 2,
// 4, 16; callers passing forward_only_ok = false (the proposal's training targets)
// serve Eq. 8 only.
int32_t check_agg(const ngprt_scene* s, const ngprt_render_opts* o, bool forward_only_ok, const char* fn) {
    if (s->aggregation == NGPRT_AGG_SEPARATE_V) return NGPRT_OK;
    NGPRT_REQUIRE(o->attn_mode == 0, "%s: attn_mode=%d applies to the SEPARATE_V aggregation only", fn, o->attn_mode);
    if (!forward_only_ok) {
        set_error("%s: aggregation %d is not served here (Eq. 8 only)", fn, s->aggregation);
        return NGPRT_ERR_UNSUPPORTED;
    }
    if (!march_supports(s->L, s->aggregation)) {
        set_error("%s: aggregation %d not built for L=%d (built: 2, 4, 16)", fn, s->aggregation, s->L);
        return NGPRT_ERR_UNSUPPORTED;
    }
    return NGPRT_OK;
}

int32_t check_opts(const ngprt_render_opts* o, const char* fn) {
    NGPRT_REQUIRE(o != nullptr, "%s: opts is NULL", fn);
    NGPRT_REQUIRE(o->step_base > 0.0f && o->step_gamma > 0.0f, "%s: step_base and step_gamma must be > 0", fn);
    NGPRT_REQUIRE(o->max_march >= 0 && o->max_samples >= 0, "%s: negative caps", fn);
    NGPRT_REQUIRE(o->attn_mode >= 0 && o->attn_mode <= 2, "%s: attn_mode=%d", fn, o->attn_mode);
    NGPRT_REQUIRE(o->dist_rule == 0 || o->dist_rule == 1, "%s: dist_rule=%d", fn, o->dist_rule);
    return NGPRT_OK;
}

}  // namespace ngprt

using namespace ngprt;

namespace ngprt {
static size_t state_bytes(int64_t n) { return ((size_t)n * NGPRT_STATE_FLOATS * sizeof(float) + 255) / 256 * 256; }
}  // namespace ngprt

extern "C" size_t ngprt_render_workspace_bytes(const ngprt_scene* scene, int64_t n_rays) {
    (void)scene;
    if (n_rays < 0) return 0;
    return state_bytes(n_rays) + 256;
}

extern "C" int32_t ngprt_render(const ngprt_scene* scene, const ngprt_occ* occ, const ngprt_camera* cams,
                                int32_t n_cams, const int32_t* pixel_ids, const float* rays_o, const float* rays_d,
                                int64_t n_rays, const float* t_interval, const ngprt_render_opts* opts, float* rgb,
                                float* depth, float* opacity, int32_t* ray_stats, float* ray_state, void* workspace,
                                size_t ws_bytes, void* stream) {
    const char* fn = "ngprt_render";
    MarchParams p;
    memset(&p, 0, sizeof p);
    int32_t rc;
    if ((rc = make_grid(scene, p.g, fn)) != NGPRT_OK) return rc;
    if ((rc = make_occ(occ, p.occ, fn)) != NGPRT_OK) return rc;
    if ((rc = check_opts(opts, fn)) != NGPRT_OK) return rc;
    if ((rc = check_agg(scene, opts, true, fn)) != NGPRT_OK) return rc;
    NGPRT_REQUIRE(n_rays >= 0, "%s: n_rays=%lld", fn, (long long)n_rays);
    NGPRT_REQUIRE(n_rays == 0 || rgb != nullptr || ray_state != nullptr, "%s: rgb and ray_state both NULL", fn);
    NGPRT_REQUIRE(march_supports(scene->L), "%s: no kernel for L=%d (built: 1, 2, 3, 4, 8, 16)", fn, scene->L);
    if (!march_supports(scene->L)) return NGPRT_ERR_UNSUPPORTED;
    NGPRT_REQUIRE(scene->mlp_dtype == NGPRT_F32 || scene->mlp_dtype == NGPRT_F16, "%s: mlp_dtype=%d", fn,
                  scene->mlp_dtype);
    dim3 grid;
    if ((rc = setup_rays(p, cams, n_cams, pixel_ids, rays_o, rays_d, n_rays, grid, fn)) != NGPRT_OK) return rc;
    if (n_rays == 0) return NGPRT_OK;
    // the per-ray state goes to ray_state, or else to the workspace
    float* state = ray_state;
    char* ws = static_cast<char*>(workspace);
    const size_t need_state = ray_state ? 0 : state_bytes(n_rays);
    if (!state) {
        if (!ws || ws_bytes < need_state) {
            set_error("%s: workspace %zu bytes < %zu needed", fn, ws_bytes, ngprt_render_workspace_bytes(scene, n_rays));
            return NGPRT_ERR_WORKSPACE;
        }
        state = reinterpret_cast<float*>(ws);
    }
    NGPRT_REQUIRE(((uintptr_t)state & 15) == 0, "%s: ray_state/workspace must be 16-byte aligned", fn);
    NGPRT_REQUIRE(!ws || ((uintptr_t)ws & 255) == 0, "%s: workspace must be 256-byte aligned", fn);
    p.opts = *opts;
    p.t_interval = t_interval;
    p.state = state;
    p.stats = ray_stats;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // tiles (runs of 32 rays for ray lists) are handed out at run time from a counter
    // in the workspace's bytes past the state (the static tile-per-warp grid without)
    if (ws && ws_bytes >= state_bytes(n_rays) + sizeof(unsigned long long)) {
        p.tile_counter = reinterpret_cast<unsigned long long*>(ws + state_bytes(n_rays));
        cudaMemsetAsync(p.tile_counter, 0, sizeof(unsigned long long), st);
    }
    if ((rc = launch_march_any(scene->L, scene->table_dtype, scene->aggregation, p, grid, st)) != NGPRT_OK)
        return rc;
    if (!rgb) return cuda_status(fn);
    if ((rc = launch_shade(scene, state, n_rays, opts->bg, rgb, depth, opacity, st, fn)) != NGPRT_OK) return rc;
    return cuda_status(fn);
}

extern "C" int32_t ngprt_grid_indices(const ngprt_scene* scene, const float* u, int64_t n, uint32_t* idx_out,
                                      void* stream) {
    const char* fn = "ngprt_grid_indices";
    IndexParams p;
    memset(&p, 0, sizeof p);
    int32_t rc;
    if ((rc = make_grid(scene, p.g, fn)) != NGPRT_OK) return rc;
    NGPRT_REQUIRE(n >= 0 && (n == 0 || (u && idx_out)), "%s: bad buffers", fn);
    if (n == 0) return NGPRT_OK;
    p.u = u;
    p.n = n;
    p.out = idx_out;
    grid_indices_kernel<<<(unsigned)((n + 127) / 128), 128, 0, static_cast<cudaStream_t>(stream)>>>(p);
    return cuda_status(fn);
}

extern "C" int32_t ngprt_shade(const ngprt_scene* scene, const float* ray_state, int64_t n_rays, const float bg[3],
                               float* rgb, float* depth, float* opacity, void* stream) {
    const char* fn = "ngprt_shade";
    NGPRT_REQUIRE(scene != nullptr && scene->mlp_w != nullptr, "%s: scene or mlp_w is NULL", fn);
    NGPRT_REQUIRE(n_rays >= 0, "%s: n_rays=%lld", fn, (long long)n_rays);
    NGPRT_REQUIRE(n_rays == 0 || (ray_state && rgb), "%s: ray_state and rgb required", fn);
    NGPRT_REQUIRE(bg != nullptr, "%s: bg is NULL", fn);
    NGPRT_REQUIRE(((uintptr_t)scene->mlp_w & 15) == 0 && ((uintptr_t)ray_state & 15) == 0,
                  "%s: mlp_w and ray_state must be 16-byte aligned", fn);
    if (n_rays == 0) return NGPRT_OK;
    int32_t rc = launch_shade(scene, ray_state, n_rays, bg, rgb, depth, opacity, static_cast<cudaStream_t>(stream), fn);
    if (rc != NGPRT_OK) return rc;
    return cuda_status(fn);
}

extern "C" int32_t ngprt_render_fallback(const ngprt_scene* scene, const ngprt_occ* occ, const ngprt_camera* cams,
                                         int32_t n_cams, const int32_t* pixel_ids, const float* rays_o,
                                         const float* rays_d, int64_t n_rays, const float* t_interval,
                                         const float* a_hat, float threshold, const ngprt_render_opts* opts,
                                         float* ray_state, int32_t* ray_stats, void* stream) {
    const char* fn = "ngprt_render_fallback";
    MarchParams p;
    memset(&p, 0, sizeof p);
    int32_t rc;
    if ((rc = make_grid(scene, p.g, fn)) != NGPRT_OK) return rc;
    if ((rc = make_occ(occ, p.occ, fn)) != NGPRT_OK) return rc;
    if ((rc = check_opts(opts, fn)) != NGPRT_OK) return rc;
    if ((rc = check_agg(scene, opts, true, fn)) != NGPRT_OK) return rc;
    NGPRT_REQUIRE(n_rays >= 0, "%s: n_rays=%lld", fn, (long long)n_rays);
    if (!march_supports(scene->L, scene->aggregation)) {
        set_error("%s: no kernel for L=%d", fn, scene->L);
        return NGPRT_ERR_UNSUPPORTED;
    }
    dim3 grid;
    if ((rc = setup_rays(p, cams, n_cams, pixel_ids, rays_o, rays_d, n_rays, grid, fn)) != NGPRT_OK) return rc;
    if (n_rays == 0) return NGPRT_OK;
    NGPRT_REQUIRE(t_interval && a_hat && ray_state, "%s: t_interval, a_hat and ray_state are required", fn);
    NGPRT_REQUIRE(((uintptr_t)ray_state & 15) == 0, "%s: ray_state must be 16-byte aligned", fn);
    p.opts = *opts;
    p.t_interval = t_interval;
    p.state = ray_state;
    p.stats = ray_stats;
    p.fb_a_hat = a_hat;
    p.fb_thr = threshold;
    if ((rc = launch_march_any(scene->L, scene->table_dtype, scene->aggregation, p, grid,
                               static_cast<cudaStream_t>(stream))) != NGPRT_OK)
        return rc;
    return cuda_status(fn);
}

extern "C" int32_t ngprt_proposal_targets(const ngprt_scene* scene, const ngprt_occ* occ, const ngprt_camera* cams,
                                          int32_t n_cams, const int32_t* pixel_ids, const float* rays_o,
                                          const float* rays_d, int64_t n_rays, const ngprt_render_opts* opts,
                                          const float* ray_state, float* targets, void* stream) {
    const char* fn = "ngprt_proposal_targets";
    MarchParams p;
    memset(&p, 0, sizeof p);
    int32_t rc;
    if ((rc = make_grid(scene, p.g, fn)) != NGPRT_OK) return rc;
    if ((rc = make_occ(occ, p.occ, fn)) != NGPRT_OK) return rc;
    if ((rc = check_opts(opts, fn)) != NGPRT_OK) return rc;
    if ((rc = check_agg(scene, opts, false, fn)) != NGPRT_OK) return rc;
    NGPRT_REQUIRE(n_rays >= 0, "%s: n_rays=%lld", fn, (long long)n_rays);
    dim3 grid;
    if ((rc = setup_rays(p, cams, n_cams, pixel_ids, rays_o, rays_d, n_rays, grid, fn)) != NGPRT_OK) return rc;
    if (n_rays == 0) return NGPRT_OK;
    NGPRT_REQUIRE(ray_state && targets, "%s: ray_state and targets are required", fn);
    p.opts = *opts;
    p.state = const_cast<float*>(ray_state);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    switch (scene->L) {
        case 1: launch_targets<1>(scene->table_dtype, p, grid, st, targets); break;
        case 2: launch_targets<2>(scene->table_dtype, p, grid, st, targets); break;
        case 3: launch_targets<3>(scene->table_dtype, p, grid, st, targets); break;
        case 4: launch_targets<4>(scene->table_dtype, p, grid, st, targets); break;
        case 8: launch_targets<8>(scene->table_dtype, p, grid, st, targets); break;
        case 16: launch_targets<16>(scene->table_dtype, p, grid, st, targets); break;
        default: set_error("%s: no kernel for L=%d", fn, scene->L); return NGPRT_ERR_UNSUPPORTED;
    }
    return cuda_status(fn);
}
