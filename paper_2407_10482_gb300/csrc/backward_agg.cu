// backward_agg.cu -- the reverse march for the forms of Table 3 other than Eq. 8:
// one spatial gate per level (SHARED_V), spatially invariant gates (SEPARATE_INV,
// SHARED_INV), the plain sum (SUM) and the tiny MLP (with its weight gradient from
// per-sample records), for L = 2, 4 and 16.
#include "backward_march.cuh"

namespace ngprt {

template <int L>
static void launch_bwd_agg_l(int agg, const MarchBwdParams& p, dim3 grid, cudaStream_t st) {
    switch (agg) {
        case NGPRT_AGG_SHARED_V: launch_bwd<L, NGPRT_AGG_SHARED_V>(p, grid, st); break;
        case NGPRT_AGG_SEPARATE_INV: launch_bwd<L, NGPRT_AGG_SEPARATE_INV>(p, grid, st); break;
        case NGPRT_AGG_SHARED_INV: launch_bwd<L, NGPRT_AGG_SHARED_INV>(p, grid, st); break;
        case NGPRT_AGG_SUM: launch_bwd<L, NGPRT_AGG_SUM>(p, grid, st); break;
        default: launch_bwd<L, NGPRT_AGG_MLP>(p, grid, st); break;
    }
}

void launch_bwd_agg_mlp_wgrad(int L, const MarchBwdParams& p, const float* w, float* g_w, cudaStream_t st) {
    switch (L) {
        case 2: launch_agg_mlp_wgrad<2>(p, w, g_w, st); break;
        case 4: launch_agg_mlp_wgrad<4>(p, w, g_w, st); break;
        default: launch_agg_mlp_wgrad<16>(p, w, g_w, st); break;
    }
}

bool march_bwd_agg_supports(int L) { return L == 2 || L == 4 || L == 16; }

void launch_bwd_agg(int L, int agg, const MarchBwdParams& p, dim3 grid, cudaStream_t st) {
    switch (L) {
        case 2: launch_bwd_agg_l<2>(agg, p, grid, st); break;
        case 4: launch_bwd_agg_l<4>(agg, p, grid, st); break;
        default: launch_bwd_agg_l<16>(agg, p, grid, st); break;
    }
}

}  // namespace ngprt
