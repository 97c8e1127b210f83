// occupancy.cu -- the render-time occupancy pipeline (Sec. S2.5): occupancy from the
// model's own density at voxel centres, visibility marking by training rays (the
// voxels of samples whose weight passes a threshold), and box dilation.  The
// pyramid and the distance grid G of the result then come from ngprt_build_occ_dist.
#include "occupancy.cuh"

namespace ngprt {

// One pass of the separable box dilation along `axis`: out = max over +-r voxels.
__global__ void dilate_pass_kernel(const uint8_t* __restrict__ in, uint8_t* __restrict__ out, int32_t R, int32_t r,
                                   int axis, const uint8_t* __restrict__ mask) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t RR = R;
    if (v >= RR * RR * RR) return;
    const int64_t stride = axis == 0 ? 1 : axis == 1 ? RR : RR * RR;
    const int c = (int)((v / stride) % RR);
    const int lo = c - r < 0 ? 0 : c - r, hi = c + r > R - 1 ? R - 1 : c + r;
    const uint8_t* base = in + (v - (int64_t)c * stride);
    uint8_t m = 0;
    for (int q = lo; q <= hi; ++q) {
        const uint8_t x = base[(int64_t)q * stride];
        m = x > m ? x : m;
    }
    out[v] = (mask && !mask[v]) ? 0 : m;
}

int32_t make_grid(const ngprt_scene* s, Grid& g, const char* fn);
int32_t make_occ(const ngprt_occ* o, OccView& v, const char* fn);
int32_t check_opts(const ngprt_render_opts* o, const char* fn);
int32_t check_agg(const ngprt_scene* s, const ngprt_render_opts* o, bool forward_only_ok, const char* fn);
int32_t setup_rays(MarchParams& p, const ngprt_camera* cams, int32_t n_cams, const int32_t* pixel_ids,
                   const float* rays_o, const float* rays_d, int64_t n_rays, dim3& grid, const char* fn);

static bool pow2_in(int32_t R) { return R >= 2 && R <= 1024 && (R & (R - 1)) == 0; }

}  // namespace ngprt

using namespace ngprt;

extern "C" int32_t ngprt_occupancy_from_density(const ngprt_scene* scene, const ngprt_render_opts* opts, int32_t R,
                                                float sigma_thr, uint8_t* occ_out, float* sigma_out, void* stream) {
    const char* fn = "ngprt_occupancy_from_density";
    DensityOccParams p;
    memset(&p, 0, sizeof p);
    int32_t rc;
    if ((rc = make_grid(scene, p.g, fn)) != NGPRT_OK) return rc;
    if ((rc = check_opts(opts, fn)) != NGPRT_OK) return rc;
    if ((rc = check_agg(scene, opts, true, fn)) != NGPRT_OK) return rc;
    NGPRT_REQUIRE(pow2_in(R), "%s: R=%d must be a power of two in [2, 1024]", fn, R);
    NGPRT_REQUIRE(occ_out != nullptr, "%s: occ_out is NULL", fn);
    p.R = R;
    p.attn_mode = opts->attn_mode;
    p.sigma_thr = sigma_thr;
    p.occ = occ_out;
    p.sigma = sigma_out;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (scene->aggregation != NGPRT_AGG_SEPARATE_V) {
        NGPRT_REQUIRE(scene->table_dtype == NGPRT_F32, "%s: the Table 3 forms are built here for F32 tables", fn);
        launch_density_agg(scene->L, scene->aggregation, scene->table_dtype, p, st);
        return cuda_status(fn);
    }
    switch (scene->L) {
        case 1: launch_density<1, NGPRT_AGG_SEPARATE_V>(scene->table_dtype, p, st); break;
        case 2: launch_density<2, NGPRT_AGG_SEPARATE_V>(scene->table_dtype, p, st); break;
        case 3: launch_density<3, NGPRT_AGG_SEPARATE_V>(scene->table_dtype, p, st); break;
        case 4: launch_density<4, NGPRT_AGG_SEPARATE_V>(scene->table_dtype, p, st); break;
        case 8: launch_density<8, NGPRT_AGG_SEPARATE_V>(scene->table_dtype, p, st); break;
        case 16: launch_density<16, NGPRT_AGG_SEPARATE_V>(scene->table_dtype, p, st); break;
        default: set_error("%s: no kernel for L=%d", fn, scene->L); return NGPRT_ERR_UNSUPPORTED;
    }
    return cuda_status(fn);
}

extern "C" int32_t ngprt_occupancy_visibility(const ngprt_scene* scene, const ngprt_occ* occ,
                                              const ngprt_camera* cams, int32_t n_cams, const int32_t* pixel_ids,
                                              const float* rays_o, const float* rays_d, int64_t n_rays,
                                              const ngprt_render_opts* opts, float w_thr, int32_t R, uint8_t* vis,
                                              void* stream) {
    const char* fn = "ngprt_occupancy_visibility";
    MarchParams p;
    memset(&p, 0, sizeof p);
    int32_t rc;
    if ((rc = make_grid(scene, p.g, fn)) != NGPRT_OK) return rc;
    if ((rc = make_occ(occ, p.occ, fn)) != NGPRT_OK) return rc;
    if ((rc = check_opts(opts, fn)) != NGPRT_OK) return rc;
    if ((rc = check_agg(scene, opts, true, fn)) != NGPRT_OK) return rc;
    NGPRT_REQUIRE(pow2_in(R), "%s: R=%d must be a power of two in [2, 1024]", fn, R);
    NGPRT_REQUIRE(n_rays >= 0, "%s: n_rays=%lld", fn, (long long)n_rays);
    dim3 grid;
    if ((rc = setup_rays(p, cams, n_cams, pixel_ids, rays_o, rays_d, n_rays, grid, fn)) != NGPRT_OK) return rc;
    if (n_rays == 0) return NGPRT_OK;
    NGPRT_REQUIRE(vis != nullptr, "%s: vis is NULL", fn);
    p.opts = *opts;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (scene->aggregation != NGPRT_AGG_SEPARATE_V) {
        NGPRT_REQUIRE(scene->table_dtype == NGPRT_F32, "%s: the Table 3 forms are built here for F32 tables", fn);
        launch_visibility_agg(scene->L, scene->aggregation, scene->table_dtype, p, grid, w_thr, R, vis, st);
        return cuda_status(fn);
    }
    switch (scene->L) {
        case 1: launch_visibility<1, NGPRT_AGG_SEPARATE_V>(scene->table_dtype, p, grid, w_thr, R, vis, st); break;
        case 2: launch_visibility<2, NGPRT_AGG_SEPARATE_V>(scene->table_dtype, p, grid, w_thr, R, vis, st); break;
        case 3: launch_visibility<3, NGPRT_AGG_SEPARATE_V>(scene->table_dtype, p, grid, w_thr, R, vis, st); break;
        case 4: launch_visibility<4, NGPRT_AGG_SEPARATE_V>(scene->table_dtype, p, grid, w_thr, R, vis, st); break;
        case 8: launch_visibility<8, NGPRT_AGG_SEPARATE_V>(scene->table_dtype, p, grid, w_thr, R, vis, st); break;
        case 16: launch_visibility<16, NGPRT_AGG_SEPARATE_V>(scene->table_dtype, p, grid, w_thr, R, vis, st); break;
        default: set_error("%s: no kernel for L=%d", fn, scene->L); return NGPRT_ERR_UNSUPPORTED;
    }
    return cuda_status(fn);
}

extern "C" size_t ngprt_dilate_workspace_bytes(int32_t R) {
    if (R < 1 || R > 1024) return 0;
    return (size_t)R * R * R;
}

extern "C" int32_t ngprt_dilate(const uint8_t* occ, int32_t R, int32_t radius, const uint8_t* mask, uint8_t* out,
                                void* workspace, size_t ws_bytes, void* stream) {
    const char* fn = "ngprt_dilate";
    NGPRT_REQUIRE(R >= 1 && R <= 1024, "%s: R=%d not in [1, 1024]", fn, R);
    NGPRT_REQUIRE(radius >= 0 && radius <= 64, "%s: radius=%d not in [0, 64]", fn, radius);
    NGPRT_REQUIRE(occ != nullptr && out != nullptr && occ != out, "%s: occ and out must be distinct buffers", fn);
    NGPRT_REQUIRE(mask != out, "%s: mask and out must be distinct buffers", fn);
    const size_t n = (size_t)R * R * R;
    if (ws_bytes < n || workspace == nullptr) {
        set_error("%s: workspace %zu bytes < %zu needed", fn, ws_bytes, n);
        return NGPRT_ERR_WORKSPACE;
    }
    uint8_t* tmp = static_cast<uint8_t*>(workspace);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const unsigned blocks = (unsigned)((n + 255) / 256);
    dilate_pass_kernel<<<blocks, 256, 0, st>>>(occ, out, R, radius, 0, nullptr);
    dilate_pass_kernel<<<blocks, 256, 0, st>>>(out, tmp, R, radius, 1, nullptr);
    dilate_pass_kernel<<<blocks, 256, 0, st>>>(tmp, out, R, radius, 2, mask);
    return cuda_status(fn);
}
