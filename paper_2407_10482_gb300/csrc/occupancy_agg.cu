// occupancy_agg.cu -- the occupancy pipeline's density and visibility kernels for the
// forms of Table 3 other than Eq. 8 (shared or invariant gates, the sum, the tiny
// MLP), on FP32 tables (the training-time master) for L = 2, 4 and 16.
#include "occupancy.cuh"

namespace ngprt {

template <int L, int AGG>
static void density_f32(const DensityOccParams& p, cudaStream_t st) {
    const int64_t n = (int64_t)p.R * p.R * p.R;
    const size_t shm = (size_t)2 * L * 128 * sizeof(float);
    density_occ_kernel<L, NGPRT_F32, AGG><<<(unsigned)((n + 127) / 128), 128, shm, st>>>(p);
}

template <int L, int AGG>
static void visibility_f32(const MarchParams& p, dim3 grid, float w_thr, int32_t R, uint8_t* vis, cudaStream_t st) {
    const size_t shm = (size_t)2 * L * 128 * sizeof(float);
    visibility_kernel<L, NGPRT_F32, AGG><<<grid, 128, shm, st>>>(p, w_thr, R, vis);
}

template <int L>
static void density_l(int agg, const DensityOccParams& p, cudaStream_t st) {
    switch (agg) {
        case NGPRT_AGG_SHARED_V: density_f32<L, NGPRT_AGG_SHARED_V>(p, st); break;
        case NGPRT_AGG_SEPARATE_INV: density_f32<L, NGPRT_AGG_SEPARATE_INV>(p, st); break;
        case NGPRT_AGG_SHARED_INV: density_f32<L, NGPRT_AGG_SHARED_INV>(p, st); break;
        case NGPRT_AGG_SUM: density_f32<L, NGPRT_AGG_SUM>(p, st); break;
        default: density_f32<L, NGPRT_AGG_MLP>(p, st); break;
    }
}

template <int L>
static void visibility_l(int agg, const MarchParams& p, dim3 grid, float w_thr, int32_t R, uint8_t* vis,
                         cudaStream_t st) {
    switch (agg) {
        case NGPRT_AGG_SHARED_V: visibility_f32<L, NGPRT_AGG_SHARED_V>(p, grid, w_thr, R, vis, st); break;
        case NGPRT_AGG_SEPARATE_INV: visibility_f32<L, NGPRT_AGG_SEPARATE_INV>(p, grid, w_thr, R, vis, st); break;
        case NGPRT_AGG_SHARED_INV: visibility_f32<L, NGPRT_AGG_SHARED_INV>(p, grid, w_thr, R, vis, st); break;
        case NGPRT_AGG_SUM: visibility_f32<L, NGPRT_AGG_SUM>(p, grid, w_thr, R, vis, st); break;
        default: visibility_f32<L, NGPRT_AGG_MLP>(p, grid, w_thr, R, vis, st); break;
    }
}

bool occupancy_agg_supports(int L) { return L == 2 || L == 4 || L == 16; }

void launch_density_agg(int L, int agg, int dt, const DensityOccParams& p, cudaStream_t st) {
    (void)dt;
    switch (L) {
        case 2: density_l<2>(agg, p, st); break;
        case 4: density_l<4>(agg, p, st); break;
        default: density_l<16>(agg, p, st); break;
    }
}

void launch_visibility_agg(int L, int agg, int dt, const MarchParams& p, dim3 grid, float w_thr, int32_t R,
                           uint8_t* vis, cudaStream_t st) {
    (void)dt;
    switch (L) {
        case 2: visibility_l<2>(agg, p, grid, w_thr, R, vis, st); break;
        case 4: visibility_l<4>(agg, p, grid, w_thr, R, vis, st); break;
        default: visibility_l<16>(agg, p, grid, w_thr, R, vis, st); break;
    }
}

}  // namespace ngprt
