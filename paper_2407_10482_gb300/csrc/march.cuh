// march.cuh -- the ray march shared by the forward render and its reverse pass.
//
// march_loop() walks one ray: coarse-to-fine occupancy test at each marching point,
// the empty-space step s_O or the distance step v*G (Eq. 9; Sec. 3.3), and at each
// occupied point a call to the sampler, which composites (forward) or scatters
// gradients (backward) and reports early termination (Sec. S2.5).  Both passes run
// this one function, so they visit the same samples.
#pragma once

#include <math.h>

#include <type_traits>

#include "common.cuh"

// Occupancy hint for the march kernels (blocks of 128 threads per SM the register
// allocation must allow; 0 = per shape, see march_min_blocks) and the warp's pixel
// tile (TILE_W x 32/TILE_W).
#ifndef NGPRT_MARCH_MIN_BLOCKS
#define NGPRT_MARCH_MIN_BLOCKS 0
#endif
#ifndef NGPRT_TILE_W
#define NGPRT_TILE_W 4
#endif

namespace ngprt {

constexpr int kTileW = NGPRT_TILE_W;
constexpr int kTileH = 32 / NGPRT_TILE_W;

struct Cams {
    ngprt_camera c[NGPRT_MAX_CAMERAS];
};

struct MarchParams {
    Grid g;
    OccView occ;
    ngprt_render_opts opts;
    Cams cams;
    int32_t mode;  // 0: camera pixels in warp tiles, 1: camera pixel ids, 2: explicit rays
    int32_t n_cams, W, H, tiles_x, tiles_per_view;
    const int32_t* pixel_ids;
    const float* rays_o;
    const float* rays_d;
    const float* t_interval;
    int64_t n_rays;
    float* state;
    int32_t* stats;
    const float* fb_a_hat;  // fallback pass: predicted opacity per ray (NULL otherwise)
    float fb_thr;           // re-march a ray when a_hat - A(interval) > fb_thr
    // camera tiles handed out at run time (zeroed before the launch), or NULL: each
    // warp takes the tile of its own index
    unsigned long long* tile_counter;
};

// Ray of this thread (false if the lane has none): origin and unnormalised
// double-float direction.
// tile_of_warp: the warp's camera tile (mode 0) or run of 32 rays (modes 1, 2), or
// -1 for the one of its own index.
__device__ __forceinline__ bool thread_ray(const MarchParams& p, int64_t& ray, float o[3], df d[3],
                                           int64_t tile_of_warp = -1) {
    if (p.mode == 0) {
        const int64_t warp =
            tile_of_warp >= 0 ? tile_of_warp : (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
        const int lane = threadIdx.x & 31;
        const int64_t view = warp / p.tiles_per_view;
        if (view >= p.n_cams) return false;
        const int tile = (int)(warp - view * p.tiles_per_view);
        const int col = (tile % p.tiles_x) * kTileW + (lane % kTileW);
        const int row = (tile / p.tiles_x) * kTileH + (lane / kTileW);
        if (col >= p.W || row >= p.H) return false;
        ray = view * (int64_t)p.W * p.H + (int64_t)row * p.W + col;
        camera_ray_df(p.cams.c[view], col, row, o, d);
        return true;
    }
    ray = tile_of_warp >= 0 ? tile_of_warp * 32 + (threadIdx.x & 31) : (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (ray >= p.n_rays) return false;
    if (p.mode == 1) {
        int64_t id = p.pixel_ids[ray];
        if (id < 0) id = 0;
        const int64_t wh = (int64_t)p.W * p.H;
        int64_t view = id / wh;
        if (view >= p.n_cams) view = p.n_cams - 1;
        const int64_t rem = id - (id / wh) * wh;
        camera_ray_df(p.cams.c[view], (int)(rem % p.W), (int)(rem / p.W), o, d);
    } else {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            o[a] = p.rays_o[3 * ray + a];
            d[a] = df{p.rays_d[3 * ray + a], 0.0f};
        }
    }
    return true;
}

// Origin and (unnormalised) double-float direction of ray `ray` of the batch.
__device__ __forceinline__ void ray_of(const MarchParams& p, int64_t ray, float o[3], df d[3]) {
    if (p.mode == 2) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            o[a] = p.rays_o[3 * ray + a];
            d[a] = df{p.rays_d[3 * ray + a], 0.0f};
        }
        return;
    }
    int64_t id = p.mode == 1 ? (int64_t)p.pixel_ids[ray] : ray;
    if (id < 0) id = 0;
    const int64_t wh = (int64_t)p.W * p.H;
    int64_t view = id / wh;
    const int64_t rem = id - view * wh;
    if (view >= p.n_cams) view = p.n_cams - 1;
    camera_ray_df(p.cams.c[view], (int)(rem % p.W), (int)(rem / p.W), o, d);
}

// Trilinear cell of a table lattice: the exact FP32 floor for FP32 tables (the
// parity form), the fixed-point cell (ufx = unit_fx(u)) for the 16-bit forms.
template <int DT>
__device__ __forceinline__ void table_cell(float u, uint32_t ufx, int N, int& b, float& w) {
    if constexpr (DT == NGPRT_F32) grid_cell(u, N, b, w);
    else grid_cell_fx(ufx, N, b, w);
}

__device__ __forceinline__ float corner_w(const float w[3], int c) {
    const float wx = (c & 1) ? w[0] : 1.0f - w[0];
    const float wy = (c & 2) ? w[1] : 1.0f - w[1];
    const float wz = (c & 4) ? w[2] : 1.0f - w[2];
    return wx * wy * wz;
}

// Packed FP32 multiply-add on a pair of lanes (Blackwell fma.rn.f32x2): each
// half is exactly fmaf(a, b, c), so the result equals the scalar form bit for bit.
#ifndef NGPRT_FFMA2
#define NGPRT_FFMA2 1
#endif

__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
#if !NGPRT_FFMA2
    return make_float2(fmaf(a.x, b.x, c.x), fmaf(a.y, b.y, c.y));
#endif
    unsigned long long A, Bv, Cv, D;
    A = *reinterpret_cast<unsigned long long*>(&a);
    Bv = *reinterpret_cast<unsigned long long*>(&b);
    Cv = *reinterpret_cast<unsigned long long*>(&c);
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(D) : "l"(A), "l"(Bv), "l"(Cv));
    return *reinterpret_cast<float2*>(&D);
}

// Unroll of the level loops: the forward's gathers (1: measured fastest on the
// fitted hd scene at 1080p, FP16 9.5 ms against 10.9 at 2) and the reverse pass's
// scatter.
#ifndef NGPRT_LEVEL_UNROLL
#define NGPRT_LEVEL_UNROLL 1
#endif
#ifndef NGPRT_SCATTER_UNROLL
#define NGPRT_SCATTER_UNROLL 2
#endif
constexpr int kLevelUnroll = NGPRT_LEVEL_UNROLL;
constexpr int kScatterUnroll = NGPRT_SCATTER_UNROLL;

// Eq. 6-8 at unit-cube position u: f = f~ + Att(f^1..f^L; a), or one of the
// aggregations of Table 3 (AGG, an ngprt_aggregation).  The coarse fetch
// interpolates the coarse grid's channels (f~ and, for the spatially variant forms,
// the attention logits); the 2L gates (sigmoid of the interpolated or constant
// logits) are parked in shared memory, gates[k*stride], so that the level loop need
// not be unrolled.  FP32 and BF16 tables interpolate in FP32; FP16 tables
// interpolate in packed half2 FMAs with FP16 corner weights (FP16 products and
// sums, one conversion per channel), the rest of the sample in FP32.  The 16-bit
// forms take their cells with the conversion-free floor (grid_cell_fast).  The MLP form accumulates its 64 hidden
// units level by level (W1 columns of level l against f^l), then applies W2.
// With kKeep (reverse pass), level l also leaves sigma^l and q^l = sum over the
// colour channels of f^l times gq (the ray's colour cotangents) in the slots
// gates[(2L + 2l) * stride] and gates[(2L + 2l + 1) * stride]; the MLP form leaves
// f^l in the slots [8l, 8l + 8) and its 64 hidden pre-activations in [8L, 8L + 64).
template <int L, int DT, int AGG = NGPRT_AGG_SEPARATE_V, bool kKeep = false>
__device__ __forceinline__ void sample_features(const Grid& g, const float u[3], int attn_mode, float f[8],
                                                float* gates, int stride, const float* gq = nullptr) {
    constexpr int NC = coarse_channels(L, AGG);
    static_assert(NC % 2 == 0, "coarse channels are fetched in pairs");
    constexpr bool kGated = AGG != NGPRT_AGG_SUM && AGG != NGPRT_AGG_MLP;
    // FP16 tables with per-level gate pairs: the gates stay in FP16 (one word per
    // level) and each level's gated sum is taken in mixed precision (FP16 factors,
    // FP32 sum), without converting the level's features
    constexpr bool kHalfGates = DT == NGPRT_F16 && AGG == NGPRT_AGG_SEPARATE_V && !kKeep;
    uint32_t ufx[3] = {0u, 0u, 0u};
    if constexpr (DT != NGPRT_F32) {
#pragma unroll
        for (int a = 0; a < 3; ++a) ufx[a] = unit_fx(u[a]);
    }
    int b[3];
    float w[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) table_cell<DT>(u[a], ufx[a], g.R_C, b[a], w[a]);
    float2 acc[NC / 2];
    uint32_t cb, sy, sz;
    coarse_base(g, b, cb, sy, sz);
    if constexpr (DT == NGPRT_F16) {
        // FP16 tables: trilinear sums in packed half2 FMAs, converted once
        __half2 hacc[NC / 2], cw[4];
        corner_w_h2(w, cw);
#pragma unroll
        for (int ch = 0; ch < NC / 2; ++ch) hacc[ch] = __float2half2_rn(0.0f);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const uint32_t v = cb + (uint32_t)(c & 1) + sy * (uint32_t)((c >> 1) & 1) + sz * (uint32_t)((c >> 2) & 1);
            uint32_t q[NC / 2];
            load_pairs<NC>(static_cast<const uint16_t*>(g.coarse) + (size_t)v * NC, q);
            const __half2 cw2 = corner_h2(cw, c);
#pragma unroll
            for (int ch = 0; ch < NC / 2; ++ch)
                hacc[ch] = __hfma2(cw2, *reinterpret_cast<const __half2*>(&q[ch]), hacc[ch]);
        }
#pragma unroll
        for (int ch = 0; ch < (kHalfGates ? kNFeat / 2 : NC / 2); ++ch) acc[ch] = __half22float2(hacc[ch]);
        if constexpr (kHalfGates) {
#pragma unroll
            for (int l = 0; l < L; ++l) {
                const __half2 lg = hacc[kNFeat / 2 + l];
                const __half2 gp = attn_mode == 1 ? __float2half2_rn(1.0f)
                                                  : gate_sigmoid_h2(attn_mode == 2 ? __low2half2(lg) : lg);
                reinterpret_cast<__half2*>(gates)[l * stride] = gp;
            }
        }
    } else {
#pragma unroll
        for (int ch = 0; ch < NC / 2; ++ch) acc[ch] = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const uint32_t v = cb + (uint32_t)(c & 1) + sy * (uint32_t)((c >> 1) & 1) + sz * (uint32_t)((c >> 2) & 1);
            float val[NC];
            load_channels<DT, NC>(g.coarse, v, val);
            const float cw = corner_w(w, c);
            const float2 cw2 = make_float2(cw, cw);
#pragma unroll
            for (int ch = 0; ch < NC / 2; ++ch) acc[ch] = ffma2(cw2, make_float2(val[2 * ch], val[2 * ch + 1]), acc[ch]);
        }
    }
#pragma unroll
    for (int ch = 0; ch < kNFeat / 2; ++ch) {
        f[2 * ch] = acc[ch].x;
        f[2 * ch + 1] = acc[ch].y;
    }
    if constexpr (kGated && !kHalfGates) {
#pragma unroll
        for (int l = 0; l < L; ++l) {
            float om, be;
            if constexpr (AGG == NGPRT_AGG_SEPARATE_V) {
                const float2 lg = acc[kNFeat / 2 + l];
                if (attn_mode == 1) {
                    om = 1.0f;
                    be = 1.0f;
                } else if (attn_mode == 2) {
                    om = gate_sigmoid(lg.x);
                    be = om;
                } else {
                    om = gate_sigmoid(lg.x);
                    be = gate_sigmoid(lg.y);
                }
            } else if constexpr (AGG == NGPRT_AGG_SHARED_V) {
                const float2 lg = acc[(kNFeat + l) / 2];
                om = gate_sigmoid((l & 1) ? lg.y : lg.x);
                be = om;
            } else if constexpr (AGG == NGPRT_AGG_SEPARATE_INV) {
                om = gate_sigmoid(__ldg(g.attn_inv + 2 * l));
                be = gate_sigmoid(__ldg(g.attn_inv + 2 * l + 1));
            } else {
                om = gate_sigmoid(__ldg(g.attn_inv + l));
                be = om;
            }
            gates[(2 * l) * stride] = om;
            gates[(2 * l + 1) * stride] = be;
        }
    }
    constexpr int kHid = AGG == NGPRT_AGG_MLP ? NGPRT_AGG_MLP_HIDDEN : 1;
    float hid[kHid];
    if constexpr (AGG == NGPRT_AGG_MLP) {
#pragma unroll
        for (int j = 0; j < kHid; ++j) hid[j] = 0.0f;
    }
    // one level's gathers and sums; kind: 1 dense, 2 hashed, 0 by the mask
    auto level = [&](const int l, auto kind) {
        constexpr int kKind = decltype(kind)::value;
        int bl[3];
        float wl[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) table_cell<DT>(u[a], ufx[a], g.N[l], bl[a], wl[a]);
        // rows within the level, against the level's first entry
        uint32_t rows[8];
#pragma unroll
        for (int c = 0; c < 8; ++c)
            rows[c] = level_index_k<kKind>(g, l, (uint32_t)(bl[0] + (c & 1)), (uint32_t)(bl[1] + ((c >> 1) & 1)),
                                           (uint32_t)(bl[2] + ((c >> 2) & 1)));
        const void* tl = static_cast<const char*>(g.tables) + (size_t)g.level_off[l] * (DT == NGPRT_F32 ? 32 : 16);
        [[maybe_unused]] float2 fl[4];
        if constexpr (DT == NGPRT_F16) {
            uint4 q[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) q[c] = __ldg(static_cast<const uint4*>(tl) + rows[c]);
            __half2 h[4], cw[4];
            corner_w_h2(wl, cw);
#pragma unroll
            for (int ch = 0; ch < 4; ++ch) h[ch] = __float2half2_rn(0.0f);
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const __half2 cw2 = corner_h2(cw, c);
                const __half2* e2 = reinterpret_cast<const __half2*>(&q[c]);
#pragma unroll
                for (int ch = 0; ch < 4; ++ch) h[ch] = __hfma2(cw2, e2[ch], h[ch]);
            }
            if constexpr (kHalfGates) {
                const __half2 gp = reinterpret_cast<const __half2*>(gates)[l * stride];
                const __half om = __low2half(gp), be = __high2half(gp);
                f[0] = fma_f16_f32(om, __low2half(h[0]), f[0]);
                f[1] = fma_f16_f32(be, __high2half(h[0]), f[1]);
#pragma unroll
                for (int ch = 1; ch < 4; ++ch) {
                    f[2 * ch] = fma_f16_f32(be, __low2half(h[ch]), f[2 * ch]);
                    f[2 * ch + 1] = fma_f16_f32(be, __high2half(h[ch]), f[2 * ch + 1]);
                }
            } else {
#pragma unroll
                for (int ch = 0; ch < 4; ++ch) fl[ch] = __half22float2(h[ch]);
            }
        } else {
            float e[8][8];
            // FP32: large levels bypass L1 allocation (16-bit entries share sectors
            // and gain from L1: they keep the default path)
            const bool na = DT == NGPRT_F32 && ((g.na_mask >> l) & 1u);
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                if (na) load_entry_f32_na(tl, rows[c], e[c]);
                else load_entry<DT>(tl, rows[c], e[c]);
            }
#pragma unroll
            for (int ch = 0; ch < 4; ++ch) fl[ch] = make_float2(0.0f, 0.0f);
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const float cw = corner_w(wl, c);
                const float2 cw2 = make_float2(cw, cw);
#pragma unroll
                for (int ch = 0; ch < 4; ++ch) fl[ch] = ffma2(cw2, make_float2(e[c][2 * ch], e[c][2 * ch + 1]), fl[ch]);
            }
        }
        if constexpr (kKeep && AGG == NGPRT_AGG_MLP) {
#pragma unroll
            for (int ch = 0; ch < 4; ++ch) {
                gates[(kNFeat * l + 2 * ch) * stride] = fl[ch].x;
                gates[(kNFeat * l + 2 * ch + 1) * stride] = fl[ch].y;
            }
        } else if constexpr (kKeep) {
            float q = fl[0].y * gq[0];
            q = fmaf(fl[1].x, gq[1], q);
            q = fmaf(fl[1].y, gq[2], q);
            q = fmaf(fl[2].x, gq[3], q);
            q = fmaf(fl[2].y, gq[4], q);
            q = fmaf(fl[3].x, gq[5], q);
            q = fmaf(fl[3].y, gq[6], q);
            gates[(2 * L + 2 * l) * stride] = fl[0].x;
            gates[(2 * L + 2 * l + 1) * stride] = q;
        }
        if constexpr (AGG == NGPRT_AGG_SUM) {
#pragma unroll
            for (int ch = 0; ch < 4; ++ch) {
                f[2 * ch] += fl[ch].x;
                f[2 * ch + 1] += fl[ch].y;
            }
        } else if constexpr (AGG == NGPRT_AGG_MLP) {
            // W1 row j holds 8L inputs; level l's 8 columns are float4s 2(jL + l), +1
            const float4* w1 = reinterpret_cast<const float4*>(g.agg_mlp) + 2 * l;
#pragma unroll
            for (int j = 0; j < kHid; ++j) {
                const float4 a = __ldg(w1 + 2 * L * j), c = __ldg(w1 + 2 * L * j + 1);
                float h = hid[j];
                h = fmaf(a.x, fl[0].x, h);
                h = fmaf(a.y, fl[0].y, h);
                h = fmaf(a.z, fl[1].x, h);
                h = fmaf(a.w, fl[1].y, h);
                h = fmaf(c.x, fl[2].x, h);
                h = fmaf(c.y, fl[2].y, h);
                h = fmaf(c.z, fl[3].x, h);
                h = fmaf(c.w, fl[3].y, h);
                hid[j] = h;
            }
        } else if constexpr (!kHalfGates) {
            // packed pairs: each half is the scalar fmaf, bit for bit
            const float om = gates[(2 * l) * stride], be = gates[(2 * l + 1) * stride];
#pragma unroll
            for (int ch = 0; ch < 4; ++ch) {
                const float2 r = ffma2(make_float2(ch == 0 ? om : be, be), fl[ch], make_float2(f[2 * ch], f[2 * ch + 1]));
                f[2 * ch] = r.x;
                f[2 * ch + 1] = r.y;
            }
        }
    };
    // the dense levels first when they are a prefix (each loop's kind fixed)
    if (g.n_dense >= 0) {
        const int nd = min(g.n_dense, L);
#pragma unroll kLevelUnroll
        for (int l = 0; l < nd; ++l) level(l, std::integral_constant<int, 1>{});
#pragma unroll kLevelUnroll
        for (int l = nd; l < L; ++l) level(l, std::integral_constant<int, 2>{});
    } else {
#pragma unroll kLevelUnroll
        for (int l = 0; l < L; ++l) level(l, std::integral_constant<int, 0>{});
    }
    if constexpr (AGG == NGPRT_AGG_MLP) {
        if constexpr (kKeep) {
#pragma unroll
            for (int j = 0; j < kHid; ++j) gates[(kNFeat * L + j) * stride] = hid[j];
        }
        const float4* w2 = reinterpret_cast<const float4*>(g.agg_mlp + (size_t)kHid * kNFeat * L);
#pragma unroll
        for (int k = 0; k < kNFeat; ++k) {
            float o = 0.0f;
#pragma unroll
            for (int j = 0; j < kHid / 4; ++j) {
                const float4 a = __ldg(w2 + k * (kHid / 4) + j);
                o = fmaf(a.x, fmaxf(hid[4 * j], 0.0f), o);
                o = fmaf(a.y, fmaxf(hid[4 * j + 1], 0.0f), o);
                o = fmaf(a.z, fmaxf(hid[4 * j + 2], 0.0f), o);
                o = fmaf(a.w, fmaxf(hid[4 * j + 3], 0.0f), o);
            }
            f[k] += o;
        }
    }
}

// World length of a step whose contracted image stays within rho of its start (so
// a step of rho = v G cannot enter an occupied voxel, Eq. 9).  Within the box or
// the unit ball, and as a floor, rho itself (the contraction is 1-Lipschitz).
// Beyond the unit ball the image moves at |J d| <= sqrt(1/r^4 + (2r-1)^2 b^2 / r^6)
// with b = |x x d| (the ray's distance from the origin); that bound falls with r,
// and a step of at most (r-1)/2 keeps the radius >= max((r+1)/2, b).
__device__ __forceinline__ float dist_step(int bounded, const float x[3], const float d[3], float r, float rho) {
    if (bounded || !(r > 1.0f)) return rho;
    const float cx = fsub(fmul(x[1], d[2]), fmul(x[2], d[1]));
    const float cy = fsub(fmul(x[2], d[0]), fmul(x[0], d[2]));
    const float cz = fsub(fmul(x[0], d[1]), fmul(x[1], d[0]));
    const float b2 = fadd(fadd(fmul(cx, cx), fmul(cy, cy)), fmul(cz, cz));
    const float rl = fmaxf(fmul(fadd(r, 1.0f), 0.5f), fsqrt(b2));
    const float q = fdiv(fsub(fmul(2.0f, rl), 1.0f), rl);
    const float s_dir = fdiv(fmul(rho, fmul(rl, rl)), fsqrt(fadd(1.0f, fmul(fmul(q, q), b2))));
    const float cap = fmul(fsub(r, 1.0f), 0.5f);
    return fmaxf(rho, fminf(s_dir, cap));
}

// Position of a ray's march between calls: the current point t, the domain end,
// the lattice origin (all double-float) and index (lattice_snap), and the counters.
struct MarchState {
    df t, t_out, t_start;
    int lat_k, n_march, n_samp;
};

__device__ __forceinline__ MarchState march_state(const Ray& ry) {
    MarchState st;
    st.t = ry.t;
    st.t_out = ry.t_out;
    st.t_start = ry.t;
    st.lat_k = 0;
    st.n_march = 0;
    st.n_samp = 0;
    return st;
}

// Image speed J(x) d of the contraction along the ray (r = |x| > 1):
// J d = k d + m x with k = (2 - 1/r)/r and m = (x.d) 2 (1 - r) / r^4.
__device__ __forceinline__ void contracted_dir(const float x[3], const float d[3], float r, float v[3]) {
    const float ir = fdiv(1.0f, r);
    const float kk = fmul(fsub(2.0f, ir), ir);
    const float px = dot3(x, d);
    const float ir2 = fmul(ir, ir);
    const float m = fmul(fmul(px, fmul(2.0f, fsub(1.0f, r))), fmul(ir2, ir2));
#pragma unroll
    for (int a = 0; a < 3; ++a) v[a] = fadd(fmul(kk, d[a]), fmul(m, x[a]));
}

// Fraction of a finest occupancy voxel that an empty-space step carries the image
// past the exit face of its voxel.
constexpr float kEmptyGuard = 0.02f;

// s_O (Sec. 3.3): the step that leaves empty voxel ev of resolution Rk.  The image
// of the ray is aimed at the plane kEmptyGuard finest voxels (side 2B / R_O) beyond
// the voxel's exit face: along the image's local direction v = J(x) d first, which
// picks the exit axis; beyond the unit ball the image curves, and one Newton step on
// that axis, from the image's position and direction at the first estimate (the
// correction clamped to half of it), corrects the length.
__device__ __forceinline__ float empty_step(int bounded, const float x[3], const float y[3], const float d[3],
                                            float r, const int ev[3], int Rk, int R_O) {
    const float B = bounded ? 1.0f : 2.0f;
    const bool curved = !bounded && r > 1.0f;
    float v[3];
    if (curved) contracted_dir(x, d, r, v);
    else {
        v[0] = d[0]; v[1] = d[1]; v[2] = d[2];
    }
    const float vk = fdiv(2.0f * B, (float)Rk);
    const float g = fmul(kEmptyGuard, fdiv(2.0f * B, (float)R_O));
    // the exit axis's values are carried by selection (no array indexed at run time)
    float s0 = INFINITY, target = 0.0f, v_ax = 0.0f, d_ax = 0.0f, x_ax = 0.0f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float lo = fsub(fmul((float)ev[a], vk), B);
        float plane = 0.0f;
        bool moving = true;
        if (v[a] > 0.0f) plane = fadd(fadd(lo, vk), g);
        else if (v[a] < 0.0f) plane = fsub(lo, g);
        else moving = false;
        const float ta = moving ? fdiv(fsub(plane, y[a]), v[a]) : INFINITY;
        if (ta < s0) {
            s0 = ta;
            target = plane;
            v_ax = v[a];
            d_ax = d[a];
            x_ax = x[a];
        }
    }
    if (!(s0 < INFINITY)) return INFINITY;
    s0 = fmaxf(s0, 0.0f);
    if (!curved) return s0;
    float x1[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) x1[a] = fadd(x[a], fmul(s0, d[a]));
    const float x1_ax = fadd(x_ax, fmul(s0, d_ax));
    const float r1 = fsqrt(dot3(x1, x1));
    float y1, v1;
    if (r1 > 1.0f) {
        const float ir = fdiv(1.0f, r1);
        const float kk = fmul(fsub(2.0f, ir), ir);
        const float ir2 = fmul(ir, ir);
        const float m = fmul(fmul(dot3(x1, d), fmul(2.0f, fsub(1.0f, r1))), fmul(ir2, ir2));
        y1 = fmul(x1_ax, kk);
        v1 = fadd(fmul(kk, d_ax), fmul(m, x1_ax));
    } else {
        y1 = x1_ax;
        v1 = d_ax;
    }
    if (!(fmul(v1, v_ax) > 0.0f)) return s0;
    const float c = fdiv(fsub(target, y1), v1);
    const float h = fmul(0.5f, s0);
    return fadd(s0, fminf(fmaxf(c, -h), h));
}

// Advance from st.t through empty space to the next occupied marching point.
// Returns true with u (unit-cube position), delta (clipped sample step) and dt (the
// sample step) of the point at st.t, or false when the ray is exhausted (t_out or a
// cap reached).
__device__ __forceinline__ bool march_advance(const MarchParams& p, const Ray& ry, MarchState& st, float u[3],
                                              float& delta, float& dt) {
    const ngprt_render_opts& op = p.opts;
    const int bounded = p.g.bounded;
    const float B = bounded ? 1.0f : 2.0f;
    const float dt0 = fmul(op.step_base, op.step_gamma);
    const int R_O = p.occ.R_O;
    const int R_G = p.occ.R_G;
    const float vG = fdiv(2.0f * B, (float)R_G);
    const bool snap = op.lattice_snap && bounded;
    while (df_lt(st.t, st.t_out) && st.n_march < op.max_march && st.n_samp < op.max_samples) {
        ++st.n_march;
        float x[3], y[3], r;
        march_point(bounded, ry, st.t, x, y, u, r);
        int empty_level = -1, ev[3] = {0, 0, 0};
        // the finest level's voxel, once: R_O is a power of two, so u R_k = u R_O / 2^k
        // exactly and a coarser level's voxel is the finest one's shifted right by k
        const int f0 = occ_vox(u[0], R_O), f1 = occ_vox(u[1], R_O), f2 = occ_vox(u[2], R_O);
        for (int k = p.occ.n_levels - 1; k >= 0; --k) {
            const int Rk = R_O >> k;
            const int c0 = f0 >> k, c1 = f1 >> k, c2 = f2 >> k;
            const uint32_t bi = (uint32_t)c0 + (uint32_t)Rk * ((uint32_t)c1 + (uint32_t)Rk * (uint32_t)c2);
            const uint32_t word = __ldg(p.occ.bits + p.occ.word_off[k] + (bi >> 5));
            if (!((word >> (bi & 31)) & 1u)) {
                empty_level = k;
                ev[0] = c0; ev[1] = c1; ev[2] = c2;
                break;
            }
        }
        if (empty_level < 0) {
            dt = bounded ? dt0 : fmul(dt0, fmaxf(1.0f, r));
            delta = fminf(dt, fadd(fsub(st.t_out.hi, st.t.hi), fsub(st.t_out.lo, st.t.lo)));
            return true;
        }
        const float s_O = empty_step(bounded, x, y, ry.dh, r, ev, R_O >> empty_level, R_O);
        float step = s_O;
        if (op.use_dist && p.occ.dist && empty_level > p.occ.g_shift) {
            const int gs = p.occ.g_shift;
            const int g0 = f0 >> gs, g1 = f1 >> gs, g2 = f2 >> gs;
            const int gv = __ldg(p.occ.dist + ((size_t)g0 + (size_t)R_G * ((size_t)g1 + (size_t)R_G * g2)));
            if (gv > 0) {
                const float sg = dist_step(bounded, x, ry.dh, r, fmul((float)gv, vG));
                step = op.dist_rule == 1 ? fmaxf(sg, s_O) : sg;
            }
        }
        if (snap) {
            // the first lattice point t_start + k dt0 at or beyond t + step
            const df rel = df_add(df_add_f(st.t, step), df_neg(st.t_start));
            const int kk = (int)floorf(fdiv(df_float(rel), dt0));
            st.lat_k = kk > st.lat_k + 1 ? kk : st.lat_k + 1;
            st.t = df_add(st.t_start, df_prod((float)st.lat_k, dt0));
        } else {
            st.t = df_add_f(st.t, step);
        }
    }
    return false;
}

// Move past the sample just taken at st.t (sample step dt, or the next lattice point).
__device__ __forceinline__ void march_after_sample(const MarchParams& p, MarchState& st, float dt) {
    ++st.n_samp;
    if (p.opts.lattice_snap && p.g.bounded) {
        st.lat_k += 1;
        st.t = df_add(st.t_start, df_prod((float)st.lat_k, fmul(p.opts.step_base, p.opts.step_gamma)));
    } else {
        st.t = df_add_f(st.t, dt);
    }
}

// Walk one ray from its state; smp.sample(u, t, delta) is called at every occupied
// marching point and returns true when the ray terminates.  The lanes of a warp
// first advance through empty space each to its own next sample, then sample
// together.
template <class Sampler>
__device__ __forceinline__ void march_loop_from(const MarchParams& p, const Ray& ry, MarchState& st, Sampler& smp) {
    float u[3], delta, dt;
    while (march_advance(p, ry, st, u, delta, dt)) {
        const bool stop = smp.sample(u, df_float(st.t), delta);
        if (stop) {
            ++st.n_samp;
            break;
        }
        march_after_sample(p, st, dt);
    }
}

template <class Sampler>
__device__ __forceinline__ void march_loop(const MarchParams& p, const Ray& ry, Sampler& smp, int& n_march,
                                           int& n_samp) {
    MarchState st = march_state(ry);
    march_loop_from(p, ry, st, smp);
    n_march = st.n_march;
    n_samp = st.n_samp;
}

// Forward sampler: features (Eq. 6-8), alpha compositing (Eq. 2, Eq. 5).
template <int L, int DT, int AGG = NGPRT_AGG_SEPARATE_V>
struct ForwardSampler {
    const Grid& g;
    int attn_mode;
    float t_term;
    float* gates;
    float T, A, depth;
    float w_last;  // weight of the last composited sample
    float Cd[3], F[4];
    __device__ __forceinline__ ForwardSampler(const Grid& g_, int mode, float term, float* gate_buf)
        : g(g_), attn_mode(mode), t_term(term), gates(gate_buf), T(1.0f), A(0.0f), depth(0.0f), w_last(0.0f) {
        Cd[0] = Cd[1] = Cd[2] = 0.0f;
        F[0] = F[1] = F[2] = F[3] = 0.0f;
    }
    __device__ __forceinline__ void reset() {
        T = 1.0f;
        A = 0.0f;
        depth = 0.0f;
        Cd[0] = Cd[1] = Cd[2] = 0.0f;
        F[0] = F[1] = F[2] = F[3] = 0.0f;
    }
    // Resume from a stored state [C_d(3), F(4), A, depth, ...] and transmittance.
    __device__ __forceinline__ void resume(const float* s, float T_) {
        Cd[0] = s[0]; Cd[1] = s[1]; Cd[2] = s[2];
        F[0] = s[3]; F[1] = s[4]; F[2] = s[5]; F[3] = s[6];
        A = s[7];
        depth = s[8];
        T = T_;
    }
    // One composited sample from its features (the arithmetic of sample()).
    __device__ __forceinline__ bool composite(const float f[8], float t, float delta) {
        const float sigma = expf(f[0]);
        const float trans = expf(-sigma * delta);
        const float w = T * (1.0f - trans);
        w_last = w;
#pragma unroll
        for (int k = 0; k < 3; ++k) Cd[k] = fmaf(w, f[1 + k], Cd[k]);
#pragma unroll
        for (int k = 0; k < 4; ++k) F[k] = fmaf(w, f[4 + k], F[k]);
        A += w;
        depth = fmaf(w, t, depth);
        T *= trans;
        return T < t_term;
    }
    __device__ __forceinline__ bool sample(const float u[3], float t, float delta) {
        float f[8];
        sample_features<L, DT, AGG>(g, u, attn_mode, f, gates, blockDim.x);
        return composite(f, t, delta);
    }
};

// Ray set-up shared by every pass: this thread's ray and its domain interval
// (false if the lane has no ray; hit = the interval is not empty).
__device__ __forceinline__ bool ray_setup(const MarchParams& p, int64_t& ray, Ray& ry, bool& hit,
                                          int64_t tile_of_warp = -1) {
    float o[3];
    df d[3];
    if (!thread_ray(p, ray, o, d, tile_of_warp)) return false;
    float t_lo = -INFINITY, t_hi = INFINITY;
    if (p.t_interval && !p.fb_a_hat) {
        t_lo = p.t_interval[2 * ray];
        t_hi = p.t_interval[2 * ray + 1];
    }
    hit = ray_interval(p.g.bounded, o, d, p.opts.t_min, p.opts.r_far, t_lo, t_hi, ry);
    return true;
}

// The fused forward kernel: one ray per thread over the warp's pixel tile (or one
// ray id / explicit ray per thread), march + features + compositing, the per-ray
// composite state written to `state`.  In the fallback pass it re-marches only the
// rays whose interval result missed the predicted opacity.  With p.tile_counter the
// grid holds only the resident blocks and each warp takes camera tiles (or runs of
// 32 listed rays) from the counter until none are left: a warp that finishes early
// starts another tile instead of idling until its block's slowest warp ends (fitted
// hd scene, 1080p: FP16 9.46 -> 8.98 ms, FP32 16.05 -> 15.60 ms).
// Blocks per SM the register allocation must allow (measured at 1080p on the
// fitted hd scene, L = 16, and earlier on the paper shape, L = 4): FP32 tables with
// 4 or more levels are fastest at 5 (102 registers; 16.1 ms against 16.2 at 6 and
// 18.0 at 8), FP16 tables at 8 (64 registers; 9.5 ms against 9.6 at 7 and 9.9 at
// 6), BF16 tables (interpolated in FP32) at 7; FP32 with fewer levels keeps 8.  The
// MLP aggregation keeps its 64 hidden units in registers.
template <int L, int DT, int AGG = NGPRT_AGG_SEPARATE_V>
constexpr int march_min_blocks() {
    if (AGG == NGPRT_AGG_MLP) return 3;
    if (NGPRT_MARCH_MIN_BLOCKS > 0) return NGPRT_MARCH_MIN_BLOCKS;
    if (DT == NGPRT_F32) return L >= 4 ? 5 : 8;
    return DT == NGPRT_F16 ? 8 : 7;
}

template <int L, int DT, int AGG>
__global__ void __launch_bounds__(128, march_min_blocks<L, DT, AGG>())
    march_kernel(const __grid_constant__ MarchParams p) {
    extern __shared__ float gate_smem[];
    // one ray of this thread (of the warp's tile `tile`, or -1: by the thread index)
    auto one_ray = [&](int64_t tile) {
        int64_t ray;
        Ray ry;
        bool hit;
        if (!ray_setup(p, ray, ry, hit, tile)) return;
        float* s = p.state + ray * NGPRT_STATE_FLOATS;
        if (p.fb_a_hat) {
            // fallback pass: keep the interval result unless it missed predicted opacity
            const float lo = p.t_interval[2 * ray], hi = p.t_interval[2 * ray + 1];
            const bool was_full = lo == -INFINITY && hi == INFINITY;
            if (was_full || !(p.fb_a_hat[ray] - s[7] > p.fb_thr)) return;
        }
        ForwardSampler<L, DT, AGG> smp(p.g, p.opts.attn_mode, p.opts.t_term, gate_smem + threadIdx.x);
        int n_march = 0, n_samp = 0;
        if (hit) march_loop(p, ry, smp, n_march, n_samp);
        reinterpret_cast<float4*>(s)[0] = make_float4(smp.Cd[0], smp.Cd[1], smp.Cd[2], smp.F[0]);
        reinterpret_cast<float4*>(s)[1] = make_float4(smp.F[1], smp.F[2], smp.F[3], smp.A);
        reinterpret_cast<float4*>(s)[2] = make_float4(smp.depth, ry.dh[0], ry.dh[1], ry.dh[2]);
        if (p.stats) {
            int2* st = reinterpret_cast<int2*>(p.stats) + ray;
            if (p.fb_a_hat) {
                const int2 prev = *st;
                *st = make_int2(prev.x + n_march, prev.y + n_samp);
            } else {
                *st = make_int2(n_march, n_samp);
            }
        }
    };
    if (!p.tile_counter) {
        one_ray(-1);
        return;
    }
    const int64_t tiles = p.mode == 0 ? (int64_t)p.tiles_per_view * p.n_cams : (p.n_rays + 31) / 32;
    const int lane = threadIdx.x & 31;
    for (;;) {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(p.tile_counter, 1ull);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= (unsigned long long)tiles) break;
        one_ray((int64_t)t);
        __syncwarp();
    }
}

// Blocks of kernel k resident on the current device at 128 threads and `shm` bytes
// of dynamic shared memory.
template <class Kernel>
int resident_blocks(Kernel k, size_t shm) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, 128, shm);
    return (sms > 0 ? sms : 1) * (per > 0 ? per : 1);
}

template <int L, int DT, int AGG>
void launch_march_dt(const MarchParams& p, dim3 grid, cudaStream_t st) {
    const size_t shm = (size_t)2 * L * 128 * sizeof(float);  // attention gates of the block's rays
    if (p.tile_counter) {
        // this instantiation's resident blocks, per device, found once
        static int cache[16] = {0};
        int dev = 0;
        cudaGetDevice(&dev);
        if (dev < 0 || dev >= 16) dev = 0;
        if (!cache[dev]) cache[dev] = resident_blocks(march_kernel<L, DT, AGG>, shm);
        if (grid.x > (unsigned)cache[dev]) grid.x = (unsigned)cache[dev];
    }
    march_kernel<L, DT, AGG><<<grid, 128, shm, st>>>(p);
}

template <int L, int AGG>
void launch_march_kernel(int dt, const MarchParams& p, dim3 grid, cudaStream_t st) {
    if (dt == NGPRT_F32) launch_march_dt<L, NGPRT_F32, AGG>(p, grid, st);
    else if (dt == NGPRT_F16) launch_march_dt<L, NGPRT_F16, AGG>(p, grid, st);
    else launch_march_dt<L, NGPRT_BF16, AGG>(p, grid, st);
}

}  // namespace ngprt
