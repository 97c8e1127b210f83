// render_noalloc.cu -- ngprt_render for callers that cannot allocate device memory.
//
// ngprt_render needs scratch for the per-ray composite state that its march kernel
// hands to its shading kernel (NGPRT_STATE_FLOATS floats per ray); normally the
// caller passes it as `workspace`.  Some callers cannot call cudaMalloc at all: a
// plug-in running inside a host application that owns the device allocator, code
// that must not allocate inside a latency-critical loop, or a caller limited to a
// fixed memory budget decided at load time.  For them this entry point keeps the
// scratch in a file-scope static device array of fixed size, which every GPU that
// loads this library holds until the process exits.
#include <mutex>

#include "common.cuh"

namespace ngprt {
namespace {

constexpr int64_t kNoAllocMaxRays = NGPRT_NOALLOC_MAX_RAYS;

// The shared scratch: per-ray state of at most kNoAllocMaxRays rays (12 MiB).
static_assert(kNoAllocMaxRays * NGPRT_STATE_FLOATS * sizeof(float) == 12u << 20, "12 MiB of scratch");
static __device__ __align__(256) float g_noalloc_state[kNoAllocMaxRays * NGPRT_STATE_FLOATS];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
float* g_state_ptr[kMaxDevices] = {nullptr};

// Device address of the static array on the current device.  In host code the
// array's name is only a host-side stand-in, so the address must come from
// cudaGetSymbolAddress, once per device, with that device current.  It is kept for
// the life of the process, which assumes the device's context is never reset (the
// header tells callers so).
int32_t device_scratch(float** out, const char* fn) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        set_error("%s: cudaGetDevice failed (%s) or device %d out of range", fn, cudaGetErrorString(e), dev);
        return NGPRT_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_state_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_state);
        if (e != cudaSuccess || p == nullptr) {
            set_error("%s: cudaGetSymbolAddress failed on device %d: %s", fn, dev, cudaGetErrorString(e));
            return NGPRT_ERR_CUDA;
        }
        g_state_ptr[dev] = static_cast<float*>(p);
    }
    *out = g_state_ptr[dev];
    return NGPRT_OK;
}

}  // namespace
}  // namespace ngprt

using namespace ngprt;

extern "C" int64_t ngprt_render_noalloc_max_rays(void) { return kNoAllocMaxRays; }

extern "C" int32_t ngprt_render_noalloc(const ngprt_scene* scene, const ngprt_occ* occ, const ngprt_camera* cams,
                                        int32_t n_cams, const int32_t* pixel_ids, const float* rays_o,
                                        const float* rays_d, int64_t n_rays, const float* t_interval,
                                        const ngprt_render_opts* opts, float* rgb, float* depth, float* opacity,
                                        int32_t* ray_stats, void* stream) {
    const char* fn = "ngprt_render_noalloc";
    if (n_rays > kNoAllocMaxRays) {
        set_error("%s: n_rays=%lld exceeds the static scratch of %lld rays; render in chunks or use ngprt_render "
                  "with a workspace",
                  fn, (long long)n_rays, (long long)kNoAllocMaxRays);
        return NGPRT_ERR_INVALID_ARG;
    }
    NGPRT_REQUIRE(n_rays == 0 || rgb != nullptr, "%s: rgb is NULL", fn);
    float* state = nullptr;
    int32_t rc = device_scratch(&state, fn);
    if (rc != NGPRT_OK) return rc;
    // Every ray's state is written in full by the march kernel before the shading
    // kernel reads it, so nothing in the scratch needs clearing between calls.
    return ngprt_render(scene, occ, cams, n_cams, pixel_ids, rays_o, rays_d, n_rays, t_interval, opts, rgb, depth,
                        opacity, ray_stats, state, nullptr, 0, stream);
}
