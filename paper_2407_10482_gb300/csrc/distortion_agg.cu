// distortion_agg.cu -- the distortion regulariser (Eq. S2) for the forms of Table 3
// other than Eq. 8: the forward kernel per form, and the reverse pass as the reverse
// march in distortion mode (density-only scatter, the forms' logits or MLP weights),
// for L = 2, 4 and 16.
#include "distortion.cuh"

namespace ngprt {

template <int L>
static void dist_fwd_l(int agg, const DistParams& p, dim3 grid, cudaStream_t st) {
    const size_t shm = (size_t)2 * L * 128 * sizeof(float);
    switch (agg) {
        case NGPRT_AGG_SHARED_V: distortion_kernel<L, NGPRT_AGG_SHARED_V><<<grid, 128, shm, st>>>(p); break;
        case NGPRT_AGG_SEPARATE_INV: distortion_kernel<L, NGPRT_AGG_SEPARATE_INV><<<grid, 128, shm, st>>>(p); break;
        case NGPRT_AGG_SHARED_INV: distortion_kernel<L, NGPRT_AGG_SHARED_INV><<<grid, 128, shm, st>>>(p); break;
        case NGPRT_AGG_SUM: distortion_kernel<L, NGPRT_AGG_SUM><<<grid, 128, shm, st>>>(p); break;
        default: distortion_kernel<L, NGPRT_AGG_MLP><<<grid, 128, shm, st>>>(p); break;
    }
}

template <int L>
static void dist_bwd_l(int agg, const MarchBwdParams& p, dim3 grid, cudaStream_t st) {
    switch (agg) {
        case NGPRT_AGG_SHARED_V: launch_bwd<L, NGPRT_AGG_SHARED_V, true>(p, grid, st); break;
        case NGPRT_AGG_SEPARATE_INV: launch_bwd<L, NGPRT_AGG_SEPARATE_INV, true>(p, grid, st); break;
        case NGPRT_AGG_SHARED_INV: launch_bwd<L, NGPRT_AGG_SHARED_INV, true>(p, grid, st); break;
        case NGPRT_AGG_SUM: launch_bwd<L, NGPRT_AGG_SUM, true>(p, grid, st); break;
        default: launch_bwd<L, NGPRT_AGG_MLP, true>(p, grid, st); break;
    }
}

void launch_dist_fwd_agg(int L, int agg, const DistParams& p, dim3 grid, cudaStream_t st) {
    switch (L) {
        case 2: dist_fwd_l<2>(agg, p, grid, st); break;
        case 4: dist_fwd_l<4>(agg, p, grid, st); break;
        default: dist_fwd_l<16>(agg, p, grid, st); break;
    }
}

void launch_dist_bwd_agg(int L, int agg, const MarchBwdParams& p, dim3 grid, cudaStream_t st) {
    switch (L) {
        case 2: dist_bwd_l<2>(agg, p, grid, st); break;
        case 4: dist_bwd_l<4>(agg, p, grid, st); break;
        default: dist_bwd_l<16>(agg, p, grid, st); break;
    }
}

}  // namespace ngprt
