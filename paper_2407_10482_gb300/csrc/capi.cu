// capi.cu -- argument validation, error reporting and small host queries of the
// C ABI (include/ngprt.h).
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include "common.cuh"

namespace ngprt {

static thread_local char g_err[1024] = "";

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
}

int32_t cuda_status(const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("%s: CUDA error %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
        return NGPRT_ERR_CUDA;
    }
    return NGPRT_OK;
}

static int64_t entries_of(const ngprt_scene* s) {
    const uint64_t T = 1ull << s->T_log2;
    uint64_t total = 0;
    for (int l = 0; l < s->L; ++l) {
        const uint64_t n = (uint64_t)s->N[l];
        const uint64_t e = n * n * n;
        total += e < T ? e : T;
    }
    return (int64_t)total;
}

// FP32 levels with at least this many entries are read without L1 allocation: their
// entries are rarely reused by nearby samples, and L1 is left to the small levels
// and the coarse grid, which are (measured: hd frame 14.5 -> 12.4 ms, paper-shaped
// L = 4 10.8 -> 9.3 ms; FP16 entries lose by it and keep L1).
#ifndef NGPRT_NA_MIN_ENTRIES
#define NGPRT_NA_MIN_ENTRIES (1u << 18)
#endif

int32_t make_grid(const ngprt_scene* s, Grid& g, const char* fn) {
    NGPRT_REQUIRE(s != nullptr, "%s: scene is NULL", fn);
    NGPRT_REQUIRE(s->L >= 1 && s->L <= kMaxL, "%s: L=%d not in [1, %d]", fn, s->L, kMaxL);
    NGPRT_REQUIRE(s->T_log2 >= 1 && s->T_log2 <= 30, "%s: T_log2=%d not in [1, 30]", fn, s->T_log2);
    NGPRT_REQUIRE(s->R_C >= 2 && s->R_C <= 1024, "%s: R_C=%d not in [2, 1024]", fn, s->R_C);
    NGPRT_REQUIRE(s->table_dtype >= NGPRT_F32 && s->table_dtype <= NGPRT_BF16, "%s: table_dtype=%d", fn,
                  s->table_dtype);
    NGPRT_REQUIRE(s->tables != nullptr && s->coarse != nullptr && s->mlp_w != nullptr, "%s: NULL scene array", fn);
    const uintptr_t align = s->table_dtype == NGPRT_F32 ? 32 : 16;
    NGPRT_REQUIRE(((uintptr_t)s->tables % align) == 0 && ((uintptr_t)s->coarse % align) == 0,
                  "%s: tables and coarse must be %d-byte aligned", fn, (int)align);
    NGPRT_REQUIRE(((uintptr_t)s->mlp_w % 16) == 0, "%s: mlp_w must be 16-byte aligned", fn);
    NGPRT_REQUIRE(s->bounded == 0 || s->bounded == 1, "%s: bounded=%d", fn, s->bounded);
    for (int l = 0; l < s->L; ++l)
        NGPRT_REQUIRE(s->N[l] >= 2 && s->N[l] <= (1 << 20), "%s: N[%d]=%d not in [2, 2^20]", fn, l, s->N[l]);
    NGPRT_REQUIRE(entries_of(s) < (int64_t)1 << 31, "%s: more than 2^31 table rows", fn);
    NGPRT_REQUIRE(s->mlp_layers >= 2 && s->mlp_width >= 1, "%s: MLP %d layers x %d", fn, s->mlp_layers, s->mlp_width);
    NGPRT_REQUIRE(s->aggregation >= NGPRT_AGG_SEPARATE_V && s->aggregation <= NGPRT_AGG_MLP, "%s: aggregation=%d", fn,
                  s->aggregation);
    const bool inv = s->aggregation == NGPRT_AGG_SEPARATE_INV || s->aggregation == NGPRT_AGG_SHARED_INV;
    NGPRT_REQUIRE(!inv || s->attn_inv != nullptr, "%s: the invariant aggregations need attn_inv", fn);
    NGPRT_REQUIRE(s->aggregation != NGPRT_AGG_MLP || (s->agg_mlp != nullptr && ((uintptr_t)s->agg_mlp % 16) == 0),
                  "%s: the MLP aggregation needs 16-byte aligned agg_mlp", fn);
    if (s->coarse_index) {
        NGPRT_REQUIRE(s->coarse_blocks >= 1 && s->coarse_blocks <= (int64_t)(0xFFFFFFFFu / NGPRT_COARSE_BLOCK_ROWS),
                      "%s: coarse_blocks=%lld", fn, (long long)s->coarse_blocks);
        NGPRT_REQUIRE(((uintptr_t)s->coarse_index & 3) == 0, "%s: coarse_index must be 4-byte aligned", fn);
    }
    memset(&g, 0, sizeof g);
    if (s->coarse_index) {
        g.coarse_index = s->coarse_index;
        g.coarse_nb = (uint32_t)((s->R_C - 1 + NGPRT_COARSE_BLOCK - 1) / NGPRT_COARSE_BLOCK);
        g.coarse_last = (uint32_t)(s->coarse_blocks - 1);
    }
    g.agg = s->aggregation;
    g.attn_inv = s->attn_inv;
    g.agg_mlp = s->agg_mlp;
    g.tables = s->tables;
    g.coarse = s->coarse;
    g.L = s->L;
    g.R_C = s->R_C;
    g.bounded = s->bounded;
    g.T_mask = (uint32_t)((1ull << s->T_log2) - 1);
    const uint64_t T = 1ull << s->T_log2;
    uint64_t off = 0;
    for (int l = 0; l < s->L; ++l) {
        const uint64_t n = (uint64_t)s->N[l];
        const uint64_t e = n * n * n;
        g.N[l] = s->N[l];
        g.level_off[l] = (uint32_t)off;
        if (e <= T) g.dense_mask |= 1u << l;
        if ((e < T ? e : T) >= (uint64_t)NGPRT_NA_MIN_ENTRIES) g.na_mask |= 1u << l;
        off += e < T ? e : T;
    }
    const int nd = __builtin_popcount(g.dense_mask);
    g.n_dense = g.dense_mask == (nd >= 32 ? 0xFFFFFFFFu : (1u << nd) - 1u) ? nd : -1;
    return NGPRT_OK;
}

int32_t make_occ(const ngprt_occ* o, OccView& v, const char* fn) {
    NGPRT_REQUIRE(o != nullptr && o->bits != nullptr, "%s: occupancy bits missing", fn);
    NGPRT_REQUIRE(o->R_O >= 2 && o->R_O <= 1024 && (o->R_O & (o->R_O - 1)) == 0, "%s: R_O=%d must be a power of two",
                  fn, o->R_O);
    NGPRT_REQUIRE(o->n_levels >= 1 && o->n_levels <= kMaxOccLevels && (o->R_O >> (o->n_levels - 1)) >= 1,
                  "%s: n_levels=%d", fn, o->n_levels);
    const int32_t RG = o->R_G == 0 ? o->R_O : o->R_G;
    int g_shift = -1;
    for (int k = 0; k < o->n_levels; ++k)
        if ((o->R_O >> k) == RG) g_shift = k;
    NGPRT_REQUIRE(g_shift >= 0, "%s: R_G=%d must be R_O >> k for a pyramid level k", fn, o->R_G);
    memset(&v, 0, sizeof v);
    v.bits = o->bits;
    v.dist = o->dist;
    v.R_O = o->R_O;
    v.n_levels = o->n_levels;
    v.R_G = RG;
    v.g_shift = g_shift;
    uint32_t off = 0;
    for (int k = 0; k < o->n_levels; ++k) {
        const uint64_t r = (uint64_t)(o->R_O >> k);
        v.word_off[k] = off;
        off += (uint32_t)((r * r * r + 31) / 32);
    }
    return NGPRT_OK;
}

}  // namespace ngprt

extern "C" const char* ngprt_last_error(void) { return ngprt::g_err; }

extern "C" int32_t ngprt_version(void) { return NGPRT_ABI_VERSION; }

extern "C" int32_t ngprt_coarse_channels(int32_t L, int32_t aggregation) {
    if (L < 1 || L > ngprt::kMaxL) return 0;
    switch (aggregation) {
        case NGPRT_AGG_SEPARATE_V: return ngprt::kNFeat + 2 * L;
        case NGPRT_AGG_SHARED_V: return ngprt::kNFeat + L;
        case NGPRT_AGG_SEPARATE_INV:
        case NGPRT_AGG_SHARED_INV:
        case NGPRT_AGG_SUM:
        case NGPRT_AGG_MLP: return ngprt::kNFeat;
        default: return 0;
    }
}

extern "C" int64_t ngprt_table_entries(const ngprt_scene* scene) {
    if (!scene || scene->L < 1 || scene->L > ngprt::kMaxL || scene->T_log2 < 1 || scene->T_log2 > 30) return -1;
    return ngprt::entries_of(scene);
}
