// render_agg.cu -- the fused march kernel for the aggregation forms of Table 3 other
// than Eq. 8: one gate per level (SHARED_V), spatially invariant gates (SEPARATE_INV,
// SHARED_INV), the plain sum (SUM) and the Instant-NGP-style tiny MLP (MLP).  Built
// for L = 2 and 4 here and L = 16 in render_agg16.cu (two translation units, so
// that the build compiles them in parallel).
#include "march.cuh"

namespace ngprt {

template <int L>
void launch_agg_l(int dt, int agg, const MarchParams& p, dim3 grid, cudaStream_t st) {
    switch (agg) {
        case NGPRT_AGG_SHARED_V: launch_march_kernel<L, NGPRT_AGG_SHARED_V>(dt, p, grid, st); break;
        case NGPRT_AGG_SEPARATE_INV: launch_march_kernel<L, NGPRT_AGG_SEPARATE_INV>(dt, p, grid, st); break;
        case NGPRT_AGG_SHARED_INV: launch_march_kernel<L, NGPRT_AGG_SHARED_INV>(dt, p, grid, st); break;
        case NGPRT_AGG_SUM: launch_march_kernel<L, NGPRT_AGG_SUM>(dt, p, grid, st); break;
        default: launch_march_kernel<L, NGPRT_AGG_MLP>(dt, p, grid, st); break;
    }
}

#ifdef NGPRT_AGG_L16_UNIT
void launch_agg_l16(int dt, int agg, const MarchParams& p, dim3 grid, cudaStream_t st) {
    launch_agg_l<16>(dt, agg, p, grid, st);
}
#else
void launch_agg_l16(int dt, int agg, const MarchParams& p, dim3 grid, cudaStream_t st);

bool march_agg_supports(int L) { return L == 2 || L == 4 || L == 16; }

int32_t launch_march_agg(int L, int dt, int agg, const MarchParams& p, dim3 grid, cudaStream_t st) {
    switch (L) {
        case 2: launch_agg_l<2>(dt, agg, p, grid, st); break;
        case 4: launch_agg_l<4>(dt, agg, p, grid, st); break;
        case 16: launch_agg_l16(dt, agg, p, grid, st); break;
        default: set_error("aggregation %d not built for L=%d", agg, L); return NGPRT_ERR_UNSUPPORTED;
    }
    return NGPRT_OK;
}
#endif

}  // namespace ngprt
