// common.cuh -- device helpers shared by the NGP-RT kernels (sm_103a).
//
// The march is a recurrence whose results are integers (which voxel is tested,
// which point is sampled).  It takes its voxel decisions on FP32 unit-cube
// coordinates; the ray set-up and the running parameter t are carried in
// double-float, so a position is exact to about the rounding of its last
// operations.  Its operations go through the explicitly rounded intrinsics below:
// no multiply-add is fused behind the code's back, which the error-free
// transformations of the double-float arithmetic rely on.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "ngprt.h"

namespace ngprt {

constexpr int kMaxL = NGPRT_MAX_LEVELS;
constexpr int kMaxOccLevels = 16;
constexpr int kMlpIn = 32;
constexpr int kNFeat = 8;

// ------------------------------------------------------------ host-side errors
void set_error(const char* fmt, ...);
int32_t cuda_status(const char* what);   // NGPRT_OK or NGPRT_ERR_CUDA with message

#define NGPRT_REQUIRE(cond, ...)                    \
    do {                                            \
        if (!(cond)) {                              \
            ::ngprt::set_error(__VA_ARGS__);        \
            return NGPRT_ERR_INVALID_ARG;           \
        }                                           \
    } while (0)

// ------------------------------------------------------- kernel-side scene view
struct Grid {
    const void* tables;
    const void* coarse;
    uint32_t level_off[kMaxL];   // first row of each level
    int32_t N[kMaxL];
    uint32_t dense_mask;         // bit l: level l is dense
    int32_t n_dense;             // the dense levels are levels 0 .. n_dense-1 (-1: not a prefix)
    uint32_t na_mask;            // bit l: level l's FP32 entries are read without L1 allocation
    uint32_t T_mask;             // 2^T_log2 - 1
    int32_t L;
    int32_t R_C;
    int32_t bounded;
    int32_t agg;                 // ngprt_aggregation
    const float* attn_inv;       // invariant attention logits
    const float* agg_mlp;        // MLP aggregation weights
    const int32_t* coarse_index; // sparse coarse grid: block slots [nb^3]; NULL = dense
    uint32_t coarse_nb;          // blocks per axis
    uint32_t coarse_last;        // last stored block slot
};

// Coarse-grid channels per vertex under an aggregation (f~ plus the variant's logits).
__host__ __device__ constexpr int coarse_channels(int L, int agg) {
    return agg == NGPRT_AGG_SEPARATE_V ? kNFeat + 2 * L : agg == NGPRT_AGG_SHARED_V ? kNFeat + L : kNFeat;
}

struct OccView {
    const uint32_t* bits;
    const uint8_t* dist;
    uint32_t word_off[kMaxOccLevels];  // first word of each pyramid level
    int32_t R_O;
    int32_t n_levels;
    int32_t R_G;      // resolution of dist: R_O >> g_shift
    int32_t g_shift;  // G is read when the empty pyramid level is coarser (k > g_shift)
};

// ------------------------------------------------- exactly rounded FP32 helpers
__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fdiv(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float fsqrt(float a) { return __fsqrt_rn(a); }

// ------------------------------------------------ double-float (hi + lo) values
// A value held as the unevaluated sum hi + lo of two floats (|lo| <= ulp(hi) / 2)
// carries about 48 bits.  The error-free transformations below (Knuth's two-sum,
// Dekker's fast two-sum, the FMA two-product) give the ray set-up and the march's
// running parameter t that precision, so that a sample position differs from the
// exact one by little more than the rounding of its final single-precision value.
struct df {
    float hi, lo;
};

__device__ __forceinline__ df df_two_sum(float a, float b) {
    const float s = fadd(a, b);
    const float bb = fsub(s, a);
    return {s, fadd(fsub(a, fsub(s, bb)), fsub(b, bb))};
}
// requires |a| >= |b| (or a == 0)
__device__ __forceinline__ df df_fast_sum(float a, float b) {
    const float s = fadd(a, b);
    return {s, fsub(b, fsub(s, a))};
}
__device__ __forceinline__ df df_prod(float a, float b) {
    const float q = fmul(a, b);
    return {q, __fmaf_rn(a, b, -q)};
}
__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ df df_add(df a, df b) {
    const df s = df_two_sum(a.hi, b.hi);
    return df_fast_sum(s.hi, fadd(s.lo, fadd(a.lo, b.lo)));
}
__device__ __forceinline__ df df_add_f(df a, float b) {
    const df s = df_two_sum(a.hi, b);
    return df_fast_sum(s.hi, fadd(s.lo, a.lo));
}
__device__ __forceinline__ df df_mul(df a, df b) {
    const df q = df_prod(a.hi, b.hi);
    return df_fast_sum(q.hi, __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, q.lo)));
}
__device__ __forceinline__ df df_mul_f(df a, float b) {
    const df q = df_prod(a.hi, b);
    return df_fast_sum(q.hi, __fmaf_rn(a.lo, b, q.lo));
}
__device__ __forceinline__ df df_div(df a, df b) {
    const float q1 = fdiv(a.hi, b.hi);
    const df r = df_add(a, df_neg(df_mul_f(b, q1)));  // a - q1 b
    return df_fast_sum(q1, fdiv(r.hi, b.hi));
}
__device__ __forceinline__ df df_sqrt(df a) {
    if (!(a.hi > 0.0f)) return {0.0f, 0.0f};
    const float s = fsqrt(a.hi);
    const df r = df_add(a, df_neg(df_prod(s, s)));  // a - s^2
    return df_fast_sum(s, fdiv(r.hi, fmul(2.0f, s)));
}
__device__ __forceinline__ bool df_lt(df a, df b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ df df_max(df a, df b) { return df_lt(a, b) ? b : a; }
__device__ __forceinline__ df df_min(df a, df b) { return df_lt(a, b) ? a : b; }
__device__ __forceinline__ float df_float(df a) { return fadd(a.hi, a.lo); }

// A ray as the march uses it: origin o, unit direction d = dh + dl (double-float),
// the domain interval [t, t_out) (double-float).
struct Ray {
    float o[3], dh[3], dl[3];
    df t, t_out;
};

// Pinhole ray direction (unnormalised, double-float) through the centre of pixel
// (col, row); OpenCV axes (x right, y down, z forward); origin = camera position.
__device__ __forceinline__ void camera_ray_df(const ngprt_camera& c, int col, int row, float o[3], df d[3]) {
    const df px = df_div(df_two_sum(fadd((float)col, 0.5f), -c.cx), df{c.fx, 0.0f});
    const df py = df_div(df_two_sum(fadd((float)row, 0.5f), -c.cy), df{c.fy, 0.0f});
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        d[r] = df_add_f(df_add(df_mul_f(px, c.c2w[4 * r + 0]), df_mul_f(py, c.c2w[4 * r + 1])), c.c2w[4 * r + 2]);
        o[r] = c.c2w[4 * r + 3];
    }
}

// The same ray in plain floats (the learned proposal's input).
__device__ __forceinline__ void camera_ray(const ngprt_camera& c, int col, int row, float o[3], float d[3]) {
    df dd[3];
    camera_ray_df(c, col, row, o, dd);
#pragma unroll
    for (int r = 0; r < 3; ++r) d[r] = df_float(dd[r]);
}

__device__ __forceinline__ float dot3(const float a[3], const float b[3]) {
    return fadd(fadd(fmul(a[0], b[0]), fmul(a[1], b[1])), fmul(a[2], b[2]));
}

// Normalise the direction and find the parametric interval [t, t_out) inside the
// domain (bounded: the box [-1,1]^3; unbounded: the world ball of radius r_far),
// clipped to [t_min, inf) and to the optional interval [t_lo, t_hi]; all in
// double-float.  False when the interval is empty.
__device__ __forceinline__ bool ray_interval(int bounded, const float o[3], const df din[3], float t_min, float r_far,
                                             float t_lo, float t_hi, Ray& ry) {
    const df n2 = df_add(df_add(df_mul(din[0], din[0]), df_mul(din[1], din[1])), df_mul(din[2], din[2]));
    const df nn = df_sqrt(n2);
    df d[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        d[a] = df_div(din[a], nn);
        ry.o[a] = o[a];
        ry.dh[a] = d[a].hi;
        ry.dl[a] = d[a].lo;
    }
    df t_in, t_out;
    if (bounded) {
        t_in = df{-INFINITY, 0.0f};
        t_out = df{INFINITY, 0.0f};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (d[a].hi == 0.0f) {
                if (!(o[a] >= -1.0f && o[a] <= 1.0f)) return false;
                continue;
            }
            const df t0 = df_div(df_two_sum(-1.0f, -o[a]), d[a]);
            const df t1 = df_div(df_two_sum(1.0f, -o[a]), d[a]);
            t_in = df_max(t_in, df_min(t0, t1));
            t_out = df_min(t_out, df_max(t0, t1));
        }
    } else {
        // |o + t d| = r_far
        const df b = df_add(df_add(df_mul_f(d[0], o[0]), df_mul_f(d[1], o[1])), df_mul_f(d[2], o[2]));
        const df c = df_add(df_add(df_add(df_prod(o[0], o[0]), df_prod(o[1], o[1])), df_prod(o[2], o[2])),
                            df_neg(df_prod(r_far, r_far)));
        const df disc = df_add(df_mul(b, b), df_neg(c));
        if (!(disc.hi >= 0.0f)) return false;
        const df sq = df_sqrt(disc);
        t_in = df_add(df_neg(b), df_neg(sq));
        t_out = df_add(df_neg(b), sq);
    }
    ry.t = df_max(df_max(t_in, df{t_min, 0.0f}), df{t_lo, 0.0f});
    ry.t_out = df_min(t_out, df{t_hi, 0.0f});
    return df_lt(ry.t, ry.t_out);
}

// World position x = o + t d at the double-float parameter t (products by
// two-product, one final rounding of the correction), its radius r, the
// contracted point y (mip-NeRF 360 when unbounded) and the unit-cube coordinate u.
__device__ __forceinline__ void march_point(int bounded, const Ray& ry, df t, float x[3], float y[3], float u[3],
                                            float& r) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const df q = df_prod(t.hi, ry.dh[a]);
        const df s = df_two_sum(ry.o[a], q.hi);
        const float corr = fadd(s.lo, fadd(q.lo, __fmaf_rn(t.hi, ry.dl[a], fmul(t.lo, ry.dh[a]))));
        x[a] = fadd(s.hi, corr);
    }
    r = fsqrt(dot3(x, x));
    if (!bounded && r > 1.0f) {
        const float ir = fdiv(1.0f, r);
        const float k = fmul(fsub(2.0f, ir), ir);  // (2 - 1/r) / r
#pragma unroll
        for (int a = 0; a < 3; ++a) y[a] = fmul(x[a], k);
    } else {
#pragma unroll
        for (int a = 0; a < 3; ++a) y[a] = x[a];
    }
    const float B = bounded ? 1.0f : 2.0f, hB = bounded ? 0.5f : 0.25f;
#pragma unroll
    for (int a = 0; a < 3; ++a) u[a] = fmul(fadd(y[a], B), hB);
}

__device__ __forceinline__ int occ_vox(float u, int Rk) {
    float c = floorf(fmul(u, (float)Rk));
    c = fminf(fmaxf(c, 0.0f), (float)(Rk - 1));
    return (int)c;
}

// Grid cell of a vertex grid of N per axis: base = floor(u (N-1)) of the exact
// product (the rounded product pf and its exact FMA residual e; pf can round up onto
// an integer only when e < 0), clamped to [0, N-2]; the weight w = u (N-1) - base
// carries the residual back in, so it is accurate to ~1 ulp of w.
__device__ __forceinline__ void grid_cell(float u, int N, int& base, float& w) {
    const float nm1 = (float)(N - 1);
    const float pf = fmul(u, nm1);
    const float e = __fmaf_rn(u, nm1, -pf);
    float bf = floorf(pf);
    if (bf == pf && e < 0.0f) bf = fsub(bf, 1.0f);
    bf = fminf(fmaxf(bf, 0.0f), (float)(N - 2));
    base = (int)bf;
    w = fadd(fsub(pf, bf), e);
}

// Unit-cube coordinate in 0.32 fixed point, floor(u 2^32), saturated to
// [0, 2^32 - 1] (the conversion saturates; a NaN converts to 0).
__device__ __forceinline__ uint32_t unit_fx(float u) { return __float2uint_rz(fmul(u, 4294967296.0f)); }

// The cell for the 16-bit table forms from the fixed-point coordinate U: the 64-bit
// product U (N-1) holds the cell in its high word (at most N-2, since U < 2^32, so
// no clamp) and the position within the cell in its low word, whose top 23 bits
// give the weight exactly as a float in [0, 1).  It floors u (N-1) to within 2^-32
// of u; where that differs from the FP32 floor the point lies on a vertex, where
// both cells interpolate to the same value up to rounding (trilinear
// interpolation is continuous across the vertex).
__device__ __forceinline__ void grid_cell_fx(uint32_t U, int N, int& base, float& w) {
    const uint64_t p = (uint64_t)U * (uint32_t)(N - 1);
    base = (int)(uint32_t)(p >> 32);
    w = fsub(__uint_as_float(0x3F800000u | ((uint32_t)p >> 9)), 1.0f);
}

// Trilinear weights of a cell's 8 corners for FP16 interpolation as 4 packed pairs:
// cw[j] holds corners 2j and 2j+1 (x = 0 and x = 1 at y = j & 1, z = j >> 1), the
// FP16 products of the per-axis pairs (1 - w, w).
__device__ __forceinline__ void corner_w_h2(const float w[3], __half2 cw[4]) {
    const __half2 hx = __floats2half2_rn(fsub(1.0f, w[0]), w[0]);
    const __half2 hy = __floats2half2_rn(fsub(1.0f, w[1]), w[1]);
    const __half2 hz = __floats2half2_rn(fsub(1.0f, w[2]), w[2]);
    const __half2 xy0 = __hmul2(hx, __low2half2(hy)), xy1 = __hmul2(hx, __high2half2(hy));
    cw[0] = __hmul2(xy0, __low2half2(hz));
    cw[1] = __hmul2(xy1, __low2half2(hz));
    cw[2] = __hmul2(xy0, __high2half2(hz));
    cw[3] = __hmul2(xy1, __high2half2(hz));
}

// Weight of corner c (bit 0: x, bit 1: y, bit 2: z) in both halves.
__device__ __forceinline__ __half2 corner_h2(const __half2 cw[4], int c) {
    return (c & 1) ? __high2half2(cw[c >> 1]) : __low2half2(cw[c >> 1]);
}

// Row of the coarse vertex at the base corner of cell b and the row strides of
// its y and z neighbours: dense [R_C^3] rows, or the 9^3-vertex block of the cell's
// 8^3-cell block in the sparse grid (one index lookup for all 8 corners).
__device__ __forceinline__ void coarse_base(const Grid& g, const int b[3], uint32_t& base, uint32_t& sy,
                                            uint32_t& sz) {
    if (g.coarse_index) {
        const uint32_t nb = g.coarse_nb;
        const uint32_t blk = ((uint32_t)b[0] >> 3) + nb * (((uint32_t)b[1] >> 3) + nb * ((uint32_t)b[2] >> 3));
        const uint32_t slot = min((uint32_t)__ldg(g.coarse_index + blk), g.coarse_last);
        base = slot * (uint32_t)NGPRT_COARSE_BLOCK_ROWS + (uint32_t)(b[0] & 7) +
               9u * ((uint32_t)(b[1] & 7) + 9u * (uint32_t)(b[2] & 7));
        sy = 9u;
        sz = 81u;
    } else {
        const uint32_t R = (uint32_t)g.R_C;
        base = (uint32_t)b[0] + R * ((uint32_t)b[1] + R * (uint32_t)b[2]);
        sy = R;
        sz = R * R;
    }
}

// Row of vertex (x, y, z) within level l (dense row-major or the Instant-NGP
// spatial hash), and its absolute table row.
__device__ __forceinline__ uint32_t level_index(const Grid& g, int l, uint32_t x, uint32_t y, uint32_t z) {
    if ((g.dense_mask >> l) & 1u) {
        const uint32_t n = (uint32_t)g.N[l];
        return x + n * (y + n * z);
    }
    return (x ^ (y * 2654435761u) ^ (z * 805459861u)) & g.T_mask;
}

// The same with the level's kind fixed at compile time: 1 dense, 2 hashed (0: by
// the mask).
template <int kKind>
__device__ __forceinline__ uint32_t level_index_k(const Grid& g, int l, uint32_t x, uint32_t y, uint32_t z) {
    if constexpr (kKind == 1) {
        const uint32_t n = (uint32_t)g.N[l];
        return x + n * (y + n * z);
    } else if constexpr (kKind == 2) {
        return (x ^ (y * 2654435761u) ^ (z * 805459861u)) & g.T_mask;
    } else {
        return level_index(g, l, x, y, z);
    }
}

__device__ __forceinline__ uint32_t level_row(const Grid& g, int l, uint32_t x, uint32_t y, uint32_t z) {
    return g.level_off[l] + level_index(g, l, x, y, z);
}

// ------------------------------------------------------------ vector loads
#ifndef NGPRT_COARSE_WIDE
#define NGPRT_COARSE_WIDE 1  // 0: coarse rows in 128-bit (F32) / 32-bit (16-bit) loads
#endif

// NC 16-bit channels of one row as NC/2 packed pairs, read-only path, with 128-bit
// loads when NC % 8 == 0 (rows 16-byte aligned), 64-bit when NC % 4 == 0, else 32-bit.
template <int NC>
__device__ __forceinline__ void load_pairs(const uint16_t* p, uint32_t w[NC / 2]) {
    if constexpr (NC % 8 == 0 && NGPRT_COARSE_WIDE) {
#pragma unroll
        for (int k = 0; k < NC / 8; ++k) {
            const uint4 q = __ldg(reinterpret_cast<const uint4*>(p) + k);
            w[4 * k] = q.x; w[4 * k + 1] = q.y; w[4 * k + 2] = q.z; w[4 * k + 3] = q.w;
        }
    } else if constexpr (NC % 4 == 0 && NGPRT_COARSE_WIDE) {
#pragma unroll
        for (int k = 0; k < NC / 4; ++k) {
            const uint2 q = __ldg(reinterpret_cast<const uint2*>(p) + k);
            w[2 * k] = q.x; w[2 * k + 1] = q.y;
        }
    } else {
#pragma unroll
        for (int k = 0; k < NC / 2; ++k) w[k] = __ldg(reinterpret_cast<const uint32_t*>(p) + k);
    }
}

// One 8-channel table entry, read-only path.  F32: a single 256-bit load (entries
// are 32-byte aligned); F16/BF16: a single 128-bit load.
template <int DT>
__device__ __forceinline__ void load_entry(const void* base, uint32_t row, float v[8]);

template <>
__device__ __forceinline__ void load_entry<NGPRT_F32>(const void* base, uint32_t row, float v[8]) {
    const float* p = static_cast<const float*>(base) + (size_t)row * 8;
    asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
                 : "l"(p));
}

// The same 256-bit load without allocating in L1 (entries of hashed levels are
// rarely reused; L1 is left to the coarse and dense levels).
__device__ __forceinline__ void load_entry_f32_na(const void* base, uint32_t row, float v[8]) {
    const float* p = static_cast<const float*>(base) + (size_t)row * 8;
    asm("ld.global.nc.L1::no_allocate.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
                 : "l"(p));
}

template <>
__device__ __forceinline__ void load_entry<NGPRT_F16>(const void* base, uint32_t row, float v[8]) {
    const uint4 q = __ldg(static_cast<const uint4*>(base) + row);
    const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        __half2 h = *reinterpret_cast<const __half2*>(&w[k]);
        float2 f = __half22float2(h);
        v[2 * k] = f.x;
        v[2 * k + 1] = f.y;
    }
}

template <>
__device__ __forceinline__ void load_entry<NGPRT_BF16>(const void* base, uint32_t row, float v[8]) {
    const uint4 q = __ldg(static_cast<const uint4*>(base) + row);
    const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        __nv_bfloat162 h = *reinterpret_cast<const __nv_bfloat162*>(&w[k]);
        float2 f = __bfloat1622float2(h);
        v[2 * k] = f.x;
        v[2 * k + 1] = f.y;
    }
}

// Read NC consecutive channels (NC even) of one coarse-grid vertex with the widest
// loads the row's alignment allows (the grid base is aligned like the tables: 32
// bytes for F32, 16 for F16/BF16): 256-bit (F32, NC % 8 == 0), 128-bit (F32 NC % 4,
// 16-bit NC % 8), 64-bit (16-bit NC % 4), else pairs.
template <int DT, int NC>
__device__ __forceinline__ void load_channels(const void* base, uint32_t vertex, float v[NC]) {
    if constexpr (DT == NGPRT_F32) {
        const float* p = static_cast<const float*>(base) + (size_t)vertex * NC;
        if constexpr (NC % 8 == 0 && NGPRT_COARSE_WIDE) {
#pragma unroll
            for (int k = 0; k < NC / 8; ++k) {
                float* q = v + 8 * k;
                asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                    : "=f"(q[0]), "=f"(q[1]), "=f"(q[2]), "=f"(q[3]), "=f"(q[4]), "=f"(q[5]), "=f"(q[6]), "=f"(q[7])
                    : "l"(p + 8 * k));
            }
        } else if constexpr (NC % 4 == 0) {
#pragma unroll
            for (int k = 0; k < NC / 4; ++k) {
                float4 q = __ldg(reinterpret_cast<const float4*>(p) + k);
                v[4 * k] = q.x; v[4 * k + 1] = q.y; v[4 * k + 2] = q.z; v[4 * k + 3] = q.w;
            }
        } else {
#pragma unroll
            for (int k = 0; k < NC / 2; ++k) {
                float2 q = __ldg(reinterpret_cast<const float2*>(p) + k);
                v[2 * k] = q.x; v[2 * k + 1] = q.y;
            }
        }
    } else {
        const uint16_t* p = static_cast<const uint16_t*>(base) + (size_t)vertex * NC;
        uint32_t w[NC / 2];
        load_pairs<NC>(p, w);
#pragma unroll
        for (int k = 0; k < NC / 2; ++k) {
            float2 f;
            if constexpr (DT == NGPRT_F16) f = __half22float2(*reinterpret_cast<const __half2*>(&w[k]));
            else f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w[k]));
            v[2 * k] = f.x;
            v[2 * k + 1] = f.y;
        }
    }
}

__device__ __forceinline__ float sigmoidf_(float x) { return 1.0f / (1.0f + expf(-x)); }

// Attention gate sigma(x) = 1 / (1 + e^-x) with the hardware exponential and
// reciprocal (relative error ~1e-6; the gates only scale feature values).
__device__ __forceinline__ float gate_sigmoid(float x) { return __fdividef(1.0f, 1.0f + __expf(-x)); }

// The same gate for a pair of FP16 logits, sigma(x) = (1 + tanh(x / 2)) / 2, with the
// hardware's packed FP16 tanh (absolute error of the gate about 5e-4, the size of
// the FP16 logit's own rounding).
__device__ __forceinline__ __half2 gate_sigmoid_h2(__half2 x) {
    const __half2 half = __float2half2_rn(0.5f);
    const __half2 a = __hmul2(x, half);
    uint32_t t;
    asm("tanh.approx.f16x2 %0, %1;" : "=r"(t) : "r"(*reinterpret_cast<const uint32_t*>(&a)));
    return __hfma2(*reinterpret_cast<const __half2*>(&t), half, half);
}

// c + a b with FP16 factors and an FP32 addend and result (one rounding, to FP32).
__device__ __forceinline__ float fma_f16_f32(__half a, __half b, float c) {
    float d;
    asm("fma.rn.f32.f16 %0, %1, %2, %3;" : "=f"(d) : "h"(__half_as_ushort(a)), "h"(__half_as_ushort(b)), "f"(c));
    return d;
}

// Real spherical harmonics, bands 0..3, order l^2 + l + m, no Condon-Shortley
// phase, orthonormal on the sphere (Cartesian polynomial form).
__device__ __forceinline__ void sh16(float x, float y, float z, float out[16]) {
    const float xx = x * x, yy = y * y, zz = z * z;
    out[0] = 0.28209479177387814f;
    out[1] = 0.48860251190291992f * y;
    out[2] = 0.48860251190291992f * z;
    out[3] = 0.48860251190291992f * x;
    out[4] = 1.09254843059207907f * x * y;
    out[5] = 1.09254843059207907f * y * z;
    out[6] = 0.31539156525252001f * (3.0f * zz - 1.0f);
    out[7] = 1.09254843059207907f * x * z;
    out[8] = 0.54627421529603953f * (xx - yy);
    out[9] = 0.59004358992664352f * y * (3.0f * xx - yy);
    out[10] = 2.89061144264055406f * x * y * z;
    out[11] = 0.45704579946446573f * y * (5.0f * zz - 1.0f);
    out[12] = 0.37317633259011540f * z * (5.0f * zz - 3.0f);
    out[13] = 0.45704579946446573f * x * (5.0f * zz - 1.0f);
    out[14] = 1.44530572132027735f * z * (xx - yy);
    out[15] = 0.59004358992664352f * x * (xx - 3.0f * yy);
}

}  // namespace ngprt
