/*
 * ngprt_oracle.c -- plain CPU oracle of the NGP-RT render path (arXiv 2407.10482).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the package smoke check and the
 * benchmark's CPU-baseline / reference arm load this library.  It shares no code,
 * header or constant table with the CUDA library; both sides receive the same
 * seeded input arrays and nothing else.
 *
 * Precision.  Everything is computed in FP64 from the FP32 inputs: ray set-up,
 * sample positions t, the contraction, the occupancy voxel and trilinear cell
 * choices, the empty-space and distance steps, features, attention, compositing,
 * the MLP and every gradient.  The march is written from its definition and shares
 * no operation order with the kernels, which take the same decisions in FP32.  A
 * decision that FP32 rounding could take the other way is flagged: a ray is
 * "ambiguous" when one of its unit-cube coordinates came within OR_AMB_U (the FP32
 * march's position error) of a voxel face whose other side changes the march's
 * outcome, when a termination test came within OR_AMB_T
 * (relative) of t_term, or when the march came within OR_AMB_END of the domain's
 * end.  Parity tests require every ray on which the kernels differ to be flagged.
 *
 * Where each function comes from:
 *   volume rendering quadrature ........ Eq. 2 (Sec. 3, Preliminaries)
 *   deferred shading C = C_d + MLP ..... Eq. 5
 *   hash-grid encoding ................. Eq. 3 and Sec. S2.1 (the spatial hash of
 *                                         Instant-NGP, which the paper builds on)
 *   feature construction f = f~ + f^ ... Eq. 6
 *   attention a = [w1,b1,...] .......... Eq. 7;  Att(...) weighted sums ..... Eq. 8
 *   occupancy distance step ............ Eq. 9 (Sec. 3.3)
 *   5-level occupancy pyramid, T<2e-3 .. Sec. S2.5 (Real-time Rendering)
 *   activations (exp, sigmoid) ......... Sec. S2.1 (Activation Layers)
 *   SH16 view embedding ................ Sec. S2.1 (Forward Pass)
 * Readings of passages the paper leaves open are listed with the build's design
 * notes (hash function, distance metric of G, delta_i, background, contraction).
 */
#define _DEFAULT_SOURCE
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAXL 32
#define OR_NFEAT 8
#define OR_MLP_IN 32

typedef struct {
    int L;
    int T_log2;
    int N[OR_MAXL];
    const double* tables;  /* [n_entries][8] */
    int R_C;
    const double* coarse;  /* [R_C^3][8 + 2L] */
    int mlp_layers;
    int mlp_width;
    const double* mlp_w;   /* layer k: [out_k][in_k] row-major, concatenated */
    int bounded;
    int aggregation;       /* 0 Eq. 8; 1 one gate per level from the grid; 2, 3 the same
                              two with constant gates; 4 plain sum; 5 tiny MLP (Table 3) */
    const double* attn_inv;/* constant logits: [L][2] (aggregation 2) or [L] (3) */
    const double* agg_mlp; /* aggregation 5: W1 [64][8L] then W2 [8][64] */
} or_scene;

#define OR_AGG_HIDDEN 64

typedef struct {
    int R_O;
    int n_levels;
    const uint32_t* bits;  /* pyramid, finest level first */
    const uint8_t* dist;   /* R_G^3 occupancy distance grid, or NULL */
    int R_G;               /* resolution of dist: R_O >> k for a pyramid level k (0: R_O) */
} or_occ;

typedef struct {
    float step_base;
    float step_gamma;
    float t_min;
    float r_far;
    float t_term;
    double bg[3];
    int max_march;
    int max_samples;
    int use_dist;
    int lattice_snap;
    int attn_mode;  /* 0 separate (w, b per level), 1 SUM (w = b = 1), 2 shared (b = w) */
    int dist_rule;  /* 0: Eq. 9 as printed (v G when G > 0); 1: max(v G, s_O) */
} or_opts;

/* ------------------------------------------------------------------ hashing */

/* Spatial hash of Instant-NGP: XOR of the coordinates times large primes,
 * uint32 wrap-around, modulo the power-of-two table size. */
uint32_t or_hash(uint32_t x, uint32_t y, uint32_t z, uint32_t T) {
    uint32_t h = (x * 1u) ^ (y * 2654435761u) ^ (z * 805459861u);
    return h % T;
}

/* Entry of vertex (x, y, z) inside one level: dense row-major (x fastest) when
 * the level's N^3 vertices fit in T entries, else the spatial hash. */
uint64_t or_level_entry(int N, uint32_t T, int x, int y, int z) {
    uint64_t n = (uint64_t)N;
    if (n * n * n <= (uint64_t)T)
        return (uint64_t)x + n * ((uint64_t)y + n * (uint64_t)z);
    return (uint64_t)or_hash((uint32_t)x, (uint32_t)y, (uint32_t)z, T);
}

void or_hash_batch(const uint32_t* xyz, int n, uint32_t T, uint32_t* out) {
    for (int i = 0; i < n; ++i) out[i] = or_hash(xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], T);
}

uint64_t or_level_offset(const int* N, int L, int T_log2, int l) {
    uint64_t T = 1ull << T_log2, off = 0;
    for (int j = 0; j < l && j < L; ++j) {
        uint64_t n = (uint64_t)N[j];
        uint64_t e = n * n * n;
        off += e < T ? e : T;
    }
    return off;
}

/* Trilinear cell of a vertex grid of N vertices per axis covering u in [0, 1]:
 * p = u (N - 1), cell = floor(p) clamped to [0, N-2], weights p - cell.  FP64: for
 * an FP32 u the product is exact, so the cell is the exact floor. */
static void or_cell(const double u[3], int N, int base[3], double w[3]) {
    for (int a = 0; a < 3; ++a) {
        double p = u[a] * (double)(N - 1);
        double b = floor(p);
        if (b < 0.0) b = 0.0;
        if (b > (double)(N - 2)) b = (double)(N - 2);
        base[a] = (int)b;
        w[a] = p - b;
    }
}

/* For tests: per position, per level, the 8 corner entry indices (absolute row in
 * the concatenated tables) and the 3 FP64 weights.  Corner c takes +1 on x if bit0,
 * on y if bit1, on z if bit2. */
void or_grid_indices(const int* N, int L, int T_log2, const float* u, int n,
                     uint64_t* idx_out, double* w_out) {
    uint32_t T = 1u << T_log2;
    for (int i = 0; i < n; ++i) {
        for (int l = 0; l < L; ++l) {
            int base[3];
            double w[3], ud[3] = {u[3 * i], u[3 * i + 1], u[3 * i + 2]};
            or_cell(ud, N[l], base, w);
            uint64_t off = or_level_offset(N, L, T_log2, l);
            for (int c = 0; c < 8; ++c) {
                int x = base[0] + (c & 1), y = base[1] + ((c >> 1) & 1), z = base[2] + ((c >> 2) & 1);
                idx_out[((size_t)i * L + l) * 8 + c] = off + or_level_entry(N[l], T, x, y, z);
            }
            for (int a = 0; a < 3; ++a) w_out[((size_t)i * L + l) * 3 + a] = w[a];
        }
    }
}

/* --------------------------------------------------- occupancy and distance */

static size_t or_words(size_t bits) { return (bits + 31) / 32; }

size_t or_pyramid_words(int R, int n_levels) {
    size_t total = 0;
    for (int k = 0; k < n_levels; ++k) {
        size_t r = (size_t)(R >> k);
        total += or_words(r * r * r);
    }
    return total;
}

static int or_bit(const uint32_t* w, size_t i) { return (int)((w[i >> 5] >> (i & 31)) & 1u); }

/* Occupancy pyramid, finest first; a coarser voxel is occupied iff any of its
 * 8 children is (Sec. S2.5: the grid is down-sampled to coarser levels). */
void or_build_pyramid(const uint8_t* occ, int R, int n_levels, uint32_t* bits) {
    memset(bits, 0, or_pyramid_words(R, n_levels) * 4);
    size_t R3 = (size_t)R * R * R;
    for (size_t i = 0; i < R3; ++i)
        if (occ[i]) bits[i >> 5] |= 1u << (i & 31);
    size_t off_prev = 0, off = or_words(R3);
    for (int k = 1; k < n_levels; ++k) {
        int rp = R >> (k - 1), r = R >> k;
        for (int z = 0; z < r; ++z)
            for (int y = 0; y < r; ++y)
                for (int x = 0; x < r; ++x) {
                    int any = 0;
                    for (int c = 0; c < 8; ++c) {
                        size_t cx = 2 * x + (c & 1), cy = 2 * y + ((c >> 1) & 1), cz = 2 * z + ((c >> 2) & 1);
                        any |= or_bit(bits + off_prev, cx + (size_t)rp * (cy + (size_t)rp * cz));
                    }
                    size_t i = (size_t)x + (size_t)r * ((size_t)y + (size_t)r * z);
                    if (any) bits[off + (i >> 5)] |= 1u << (i & 31);
                }
        off_prev = off;
        off += or_words((size_t)r * r * r);
    }
}

static int64_t or_isqrt(int64_t v) {
    int64_t s = (int64_t)sqrt((double)v);
    while (s * s > v) --s;
    while ((s + 1) * (s + 1) <= v) ++s;
    return s;
}

/* Squared box-to-box gap along one axis between voxel p and voxel q, in voxels:
 * max(|p - q| - 1, 0)^2.  Summed over the axes it is the squared Euclidean distance
 * between the two closed voxel boxes. */
static int64_t or_gap2(int k) {
    int64_t g = (k < 0 ? -k : k) - 1;
    return g > 0 ? g * g : 0;
}

/* Occupancy distance grid G by brute force (Sec. 3.3: distance to the nearest
 * occupied voxel, rounded down, in voxel units, stored as uint8).  Distance is
 * between voxel boxes; G = min(255, floor(sqrt(D^2))); 255 when nothing is
 * occupied.  O(R^3 x occupied): for small grids. */
void or_occ_dist_brute(const uint8_t* occ, int R, uint8_t* dist) {
    size_t R3 = (size_t)R * R * R;
    for (size_t p = 0; p < R3; ++p) {
        int px = (int)(p % R), py = (int)((p / R) % R), pz = (int)(p / ((size_t)R * R));
        int64_t best = -1;
        for (size_t q = 0; q < R3; ++q) {
            if (!occ[q]) continue;
            int qx = (int)(q % R), qy = (int)((q / R) % R), qz = (int)(q / ((size_t)R * R));
            int64_t d2 = or_gap2(px - qx) + or_gap2(py - qy) + or_gap2(pz - qz);
            if (best < 0 || d2 < best) best = d2;
        }
        dist[p] = (uint8_t)(best < 0 ? 255 : (or_isqrt(best) < 255 ? or_isqrt(best) : 255));
    }
}

/* Same quantity by three exact 1-D minimisations: the squared box distance is a sum
 * of per-axis terms, so min over q of the sum = nested minima axis by axis.
 * O(R^4); used for grids too large for brute force. */
void or_occ_dist(const uint8_t* occ, int R, uint8_t* dist) {
    size_t R3 = (size_t)R * R * R;
    const int64_t INF = (int64_t)1 << 40;
    int64_t* a = (int64_t*)malloc(R3 * sizeof(int64_t));
    int64_t* b = (int64_t*)malloc(R3 * sizeof(int64_t));
    for (int z = 0; z < R; ++z)
        for (int y = 0; y < R; ++y)
            for (int x = 0; x < R; ++x) {
                int64_t best = INF;
                for (int q = 0; q < R; ++q)
                    if (occ[(size_t)q + (size_t)R * (y + (size_t)R * z)]) {
                        int64_t v = or_gap2(x - q);
                        if (v < best) best = v;
                    }
                a[(size_t)x + (size_t)R * (y + (size_t)R * z)] = best;
            }
    for (int z = 0; z < R; ++z)
        for (int y = 0; y < R; ++y)
            for (int x = 0; x < R; ++x) {
                int64_t best = INF;
                for (int q = 0; q < R; ++q) {
                    int64_t v = a[(size_t)x + (size_t)R * (q + (size_t)R * z)];
                    if (v < INF && v + or_gap2(y - q) < best) best = v + or_gap2(y - q);
                }
                b[(size_t)x + (size_t)R * (y + (size_t)R * z)] = best;
            }
    for (int z = 0; z < R; ++z)
        for (int y = 0; y < R; ++y)
            for (int x = 0; x < R; ++x) {
                int64_t best = INF;
                for (int q = 0; q < R; ++q) {
                    int64_t v = b[(size_t)x + (size_t)R * (y + (size_t)R * q)];
                    if (v < INF && v + or_gap2(z - q) < best) best = v + or_gap2(z - q);
                }
                int64_t g = best >= INF ? 255 : or_isqrt(best);
                dist[(size_t)x + (size_t)R * (y + (size_t)R * z)] = (uint8_t)(g < 255 ? g : 255);
            }
    free(a);
    free(b);
}

/* --------------------------------------------------------- view embedding */

/* Real spherical harmonics of bands 0..3 (16 values) of the unit direction d, in
 * the order l^2 + l + m, m = -l..l; Y_l^m = sqrt(2) K_l^|m| P_l^|m|(cos th) times
 * cos(m phi) (m > 0) or sin(|m| phi) (m < 0), K_l^m = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!),
 * associated Legendre functions without the Condon-Shortley phase.  Evaluated from
 * the definition by the three-term recurrence, in FP64 (Sec. S2.1). */
void or_sh16(const double d[3], double out[16]) {
    double x = d[2];                       /* cos(theta) */
    double s = sqrt(fmax(0.0, 1.0 - x * x));
    double phi = atan2(d[1], d[0]);
    double P[4][4];
    memset(P, 0, sizeof P);
    for (int m = 0; m <= 3; ++m) {
        double pmm = 1.0;
        for (int k = 1; k <= m; ++k) pmm *= (2.0 * k - 1.0) * s;
        P[m][m] = pmm;
        if (m + 1 <= 3) P[m + 1][m] = x * (2.0 * m + 1.0) * pmm;
        for (int l = m + 2; l <= 3; ++l)
            P[l][m] = (x * (2.0 * l - 1.0) * P[l - 1][m] - (l + m - 1.0) * P[l - 2][m]) / (l - m);
    }
    for (int l = 0; l <= 3; ++l)
        for (int m = -l; m <= l; ++m) {
            int am = m < 0 ? -m : m;
            double fr = 1.0;  /* (l-|m|)!/(l+|m|)! */
            for (int k = l - am + 1; k <= l + am; ++k) fr /= (double)k;
            double K = sqrt((2.0 * l + 1.0) / (4.0 * 3.14159265358979323846) * fr);
            double v;
            if (m == 0) v = K * P[l][0];
            else if (m > 0) v = sqrt(2.0) * K * cos(m * phi) * P[l][am];
            else v = sqrt(2.0) * K * sin(am * phi) * P[l][am];
            out[l * l + l + m] = v;
        }
}

void or_sh16_batch(const double* d, int n, double* out) {
    for (int i = 0; i < n; ++i) or_sh16(d + 3 * i, out + 16 * i);
}

/* ----------------------------------------------------------- deferred MLP */

static int or_mlp_out(const or_scene* s, int k) { return k == s->mlp_layers - 1 ? 3 : s->mlp_width; }
static int or_mlp_in(const or_scene* s, int k) { return k == 0 ? OR_MLP_IN : s->mlp_width; }

/* MLP_psi of Eq. 5: dense layers without bias, ReLU on hidden layers, linear
 * output of 3.  Stores every layer's pre-activation in acts (for the reverse pass). */
static void or_mlp_forward(const or_scene* s, const double* x, double* y, double* acts) {
    double h[256], g[256];
    memcpy(h, x, OR_MLP_IN * sizeof(double));
    const double* w = s->mlp_w;
    size_t ao = 0;
    for (int k = 0; k < s->mlp_layers; ++k) {
        int no = or_mlp_out(s, k), ni = or_mlp_in(s, k);
        for (int o = 0; o < no; ++o) {
            double acc = 0.0;
            for (int i = 0; i < ni; ++i) acc += w[(size_t)o * ni + i] * h[i];
            g[o] = acc;
            if (acts) acts[ao + o] = acc;
        }
        ao += no;
        w += (size_t)no * ni;
        for (int o = 0; o < no; ++o) h[o] = (k == s->mlp_layers - 1) ? g[o] : (g[o] > 0.0 ? g[o] : 0.0);
    }
    memcpy(y, h, 3 * sizeof(double));
}

void or_mlp_batch(const or_scene* s, const double* x, int n, double* y) {
    for (int i = 0; i < n; ++i) or_mlp_forward(s, x + (size_t)OR_MLP_IN * i, y + 3 * i, NULL);
}

/* ----------------------------------------------------- feature construction */

static double or_sigmoid(double v) { return 1.0 / (1.0 + exp(-v)); }

/* Per-sample quantities the reverse pass needs again. */
typedef struct {
    double t, delta, u[3];
    double sigma_raw, sigma, alpha, T_before;
    double f[OR_NFEAT];          /* fused deferred feature [sigma_raw, c_d, v_s] */
} or_sample;

/* Trilinear interpolation over one grid: 8 corners, weight prod(w or 1-w). */
static double or_corner_weight(const double w[3], int c) {
    double wx = (c & 1) ? w[0] : 1.0 - w[0];
    double wy = (c & 2) ? w[1] : 1.0 - w[1];
    double wz = (c & 4) ? w[2] : 1.0 - w[2];
    return wx * wy * wz;
}

/* Channels per coarse-grid vertex: f~ (8), then the attention logits of the
 * spatially variant forms (omega, beta per level for Eq. 8; one per level for the
 * shared form); the other forms keep f~ alone. */
int or_coarse_channels(int L, int aggregation) {
    if (aggregation == 0) return OR_NFEAT + 2 * L;
    if (aggregation == 1) return OR_NFEAT + L;
    return OR_NFEAT;
}

/* Eq. 6-8: f = f~ + Att(f^1..f^L; a), f~ and a trilinear in the coarse grid, a
 * squashed by a sigmoid after interpolation (Sec. S2.1), f^l trilinear in level l.
 * The aggregation variants of Table 3 replace Att: one gate per level for all
 * channels (shared), gates constant over space (invariant: sigmoid of a logit per
 * level), the plain sum, or Instant-NGP's tiny MLP on the concatenated levels,
 * f^ = W2 relu(W1 [f^1, ..., f^L]). */
static void or_features(const or_scene* s, const or_opts* op, const double u[3], double f[OR_NFEAT]) {
    int nch = or_coarse_channels(s->L, s->aggregation);
    double coarse[OR_NFEAT + 2 * OR_MAXL];
    double hid[OR_AGG_HIDDEN];
    int base[3];
    double w[3];
    memset(coarse, 0, sizeof coarse);
    memset(hid, 0, sizeof hid);
    or_cell(u, s->R_C, base, w);
    for (int c = 0; c < 8; ++c) {
        int x = base[0] + (c & 1), y = base[1] + ((c >> 1) & 1), z = base[2] + ((c >> 2) & 1);
        size_t v = (size_t)x + (size_t)s->R_C * ((size_t)y + (size_t)s->R_C * z);
        double cw = or_corner_weight(w, c);
        for (int ch = 0; ch < nch; ++ch) coarse[ch] += cw * s->coarse[v * nch + ch];
    }
    for (int ch = 0; ch < OR_NFEAT; ++ch) f[ch] = coarse[ch];
    uint32_t T = 1u << s->T_log2;
    for (int l = 0; l < s->L; ++l) {
        double om = 1.0, be = 1.0;
        switch (s->aggregation) {
            case 0:
                if (op->attn_mode == 1) { om = 1.0; be = 1.0; }
                else if (op->attn_mode == 2) { om = or_sigmoid(coarse[OR_NFEAT + 2 * l]); be = om; }
                else { om = or_sigmoid(coarse[OR_NFEAT + 2 * l]); be = or_sigmoid(coarse[OR_NFEAT + 2 * l + 1]); }
                break;
            case 1: om = or_sigmoid(coarse[OR_NFEAT + l]); be = om; break;
            case 2: om = or_sigmoid(s->attn_inv[2 * l]); be = or_sigmoid(s->attn_inv[2 * l + 1]); break;
            case 3: om = or_sigmoid(s->attn_inv[l]); be = om; break;
            default: break; /* 4: sum; 5: MLP below */
        }
        double fl[OR_NFEAT];
        memset(fl, 0, sizeof fl);
        or_cell(u, s->N[l], base, w);
        uint64_t off = or_level_offset(s->N, s->L, s->T_log2, l);
        for (int c = 0; c < 8; ++c) {
            int x = base[0] + (c & 1), y = base[1] + ((c >> 1) & 1), z = base[2] + ((c >> 2) & 1);
            uint64_t e = off + or_level_entry(s->N[l], T, x, y, z);
            double cw = or_corner_weight(w, c);
            for (int ch = 0; ch < OR_NFEAT; ++ch) fl[ch] += cw * s->tables[e * OR_NFEAT + ch];
        }
        if (s->aggregation == 5) {
            for (int j = 0; j < OR_AGG_HIDDEN; ++j)
                for (int ch = 0; ch < OR_NFEAT; ++ch)
                    hid[j] += s->agg_mlp[(size_t)j * OR_NFEAT * s->L + OR_NFEAT * l + ch] * fl[ch];
        } else {
            f[0] += om * fl[0];
            for (int ch = 1; ch < OR_NFEAT; ++ch) f[ch] += be * fl[ch];
        }
    }
    if (s->aggregation == 5) {
        const double* w2 = s->agg_mlp + (size_t)OR_AGG_HIDDEN * OR_NFEAT * s->L;
        for (int k = 0; k < OR_NFEAT; ++k) {
            double o = 0.0;
            for (int j = 0; j < OR_AGG_HIDDEN; ++j) o += w2[k * OR_AGG_HIDDEN + j] * fmax(hid[j], 0.0);
            f[k] += o;
        }
    }
}

/* ------------------------------------------------------------- FP64 march */

/* Ambiguity margins (see the header): unit-cube distance to a deciding voxel face,
 * and the relative distance of T to t_term or of t to the domain's end. */
#define OR_AMB_T 3e-5
/* Largest distance (unit-cube coordinates) between an FP32 march's sample positions
 * and the exact ones: a decision whose deciding face lies closer than this may go
 * either way. */
#ifndef OR_AMB_U
#define OR_AMB_U 8e-7
#endif

/* Position error the tiny-MLP form's kink flag allows for (or_set_kink_position_error):
 * OR_AMB_U, or 0 for rays whose sample positions are exact in FP32 as well. */
static double or_kink_pos_err = OR_AMB_U;
void or_set_kink_position_error(double e) { or_kink_pos_err = e; }
#define OR_AMB_END 1e-6      /* relative distance of t to the domain's end */
#define OR_AMB_LATTICE 1e-4  /* lattice units, for lattice_snap */

/* Position at parameter t: world x = o + t d, its radius r, the contracted point y
 * (mip-NeRF 360: x inside the unit ball, (2 - 1/r) x / r outside; the bounded scene
 * keeps x) and the unit-cube coordinate u = (y + B) / (2B), B = 1 bounded, 2
 * contracted. */
static void or_point(int bounded, const double o[3], const double d[3], double t,
                     double x[3], double y[3], double u[3], double* r_out) {
    for (int a = 0; a < 3; ++a) x[a] = o[a] + t * d[a];
    double r = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
    *r_out = r;
    double scale = (!bounded && r > 1.0) ? (2.0 - 1.0 / r) / r : 1.0;
    double B = bounded ? 1.0 : 2.0;
    for (int a = 0; a < 3; ++a) {
        y[a] = scale * x[a];
        u[a] = (y[a] + B) / (2.0 * B);
    }
}

/* For tests: the contraction and unit-cube position of world points x. */
void or_contract_batch(int bounded, const double* x, int n, double* y_out, double* u_out) {
    const double o[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < n; ++i) {
        double xx[3], r;
        or_point(bounded, o, x + 3 * i, 1.0, xx, y_out + 3 * i, u_out + 3 * i, &r);
    }
}

/* The contraction's Jacobian applied to d at x (radius r > 1): with
 * y = g(r) x, g(r) = 2/r - 1/r^2, J d = g d + g'(r) (x.d / r) x, g'(r) = 2/r^3 - 2/r^2. */
static void or_jacobian_dir(const double x[3], const double d[3], double r, double v[3]) {
    double g = 2.0 / r - 1.0 / (r * r);
    double gp = 2.0 / (r * r * r) - 2.0 / (r * r);
#ifdef OR_PLANT_JACOBIAN_SIGN
    gp = -gp;   /* a planted mistake, built only by the pin that must catch it */
#endif
    double xd = x[0] * d[0] + x[1] * d[1] + x[2] * d[2];
    for (int a = 0; a < 3; ++a) v[a] = g * d[a] + gp * (xd / r) * x[a];
}

/* World length of a step whose contracted image stays within distance rho of its
 * start, so that a step of rho = v G cannot enter an occupied voxel (Eq. 9 in the
 * unbounded scene).  The box and the unit ball map by the identity and the
 * contraction is 1-Lipschitz, so rho itself is always safe.  Beyond the unit ball
 * the image of the segment [x, x + s d] moves at speed |J d| with
 * |J d|^2 <= 1/r^4 + (2r - 1)^2 b^2 / r^6, b = |x x d| the ray's distance from the
 * origin (constant along it) and r the radius on the segment; that bound falls
 * with r, and with s <= (r - 1)/2 the segment stays at radius >= max((r+1)/2, b),
 * where the speed is at most sqrt(1 + q^2 b^2) / r'^2, q = (2r' - 1)/r'. */
static double or_dist_step(int bounded, const double x[3], const double d[3], double r, double rho) {
    if (bounded || !(r > 1.0)) return rho;
    double c[3] = {x[1] * d[2] - x[2] * d[1], x[2] * d[0] - x[0] * d[2], x[0] * d[1] - x[1] * d[0]};
    double b = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
    double rl = fmax(0.5 * (r + 1.0), b);
    double q = 2.0 - 1.0 / rl;
    double speed = sqrt(1.0 + q * q * b * b) / (rl * rl);
    double s = fmin(rho / speed, 0.5 * (r - 1.0));
    return fmax(rho, s);
}

void or_dist_step_batch(int bounded, const double* x, const double* d, const double* rho, int n, double* out) {
    for (int i = 0; i < n; ++i) {
        const double* xi = x + 3 * i;
        double r = sqrt(xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2]);
        out[i] = or_dist_step(bounded, xi, d + 3 * i, r, rho[i]);
    }
}

/* Voxel of coordinate u in a grid of Rk voxels over [0, 1] (clamped to the grid). */
static int or_vox(double u, int Rk) {
    double c = floor(u * (double)Rk);
    if (c < 0.0) c = 0.0;
    if (c > (double)(Rk - 1)) c = (double)(Rk - 1);
    return (int)c;
}

/* Empty-space step s_O from a point of empty voxel ev of resolution Rk (Sec. 3.3:
 * the step that leaves the voxel the empty level reports).  The contracted image
 * of the ray is aimed at a plane OR_GUARD finest voxels (2B / R_O each) beyond the
 * voxel's exit face, so that the next point lies clearly inside the next voxel:
 * first along the image's local direction v = J(x) d, which picks the exit axis
 * a (the first plane reached); beyond the unit ball the image curves, so one
 * Newton step on that axis then corrects the length with the image's position
 * and direction at the first estimate (the correction clamped to half the
 * estimate).  The bounded scene and the unit ball map straight, where the first
 * estimate is exact. */
#define OR_GUARD 2e-2
static double or_empty_step(int bounded, const double x[3], const double y[3], const double d[3], double r,
                            const int ev[3], int Rk, int R_O, double* v_exit) {
    double B = bounded ? 1.0 : 2.0;
    int curved = !bounded && r > 1.0;
    double v[3];
    if (curved) or_jacobian_dir(x, d, r, v);
    else { v[0] = d[0]; v[1] = d[1]; v[2] = d[2]; }
    double side = 2.0 * B / (double)Rk, g = OR_GUARD * 2.0 * B / (double)R_O;
    double s0 = INFINITY, target = 0.0;
    int ax = -1;
    for (int a = 0; a < 3; ++a) {
        double plane;
        if (v[a] > 0.0) plane = -B + side * (ev[a] + 1) + g;
        else if (v[a] < 0.0) plane = -B + side * ev[a] - g;
        else continue;
        double ta = (plane - y[a]) / v[a];
        if (ta < s0) { s0 = ta; ax = a; target = plane; }
    }
    if (ax < 0) return INFINITY;
    if (v_exit) *v_exit = fabs(v[ax]);
    s0 = fmax(s0, 0.0);
    if (!curved) return s0;
    /* Newton step on axis ax at the first estimate */
    double o0[3] = {0.0, 0.0, 0.0}, x1[3], y1[3], u1[3], r1, v1[3];
    double p1[3] = {x[0] + s0 * d[0], x[1] + s0 * d[1], x[2] + s0 * d[2]};
    or_point(0, o0, p1, 1.0, x1, y1, u1, &r1);
    if (r1 > 1.0) or_jacobian_dir(x1, d, r1, v1);
    else { v1[0] = d[0]; v1[1] = d[1]; v1[2] = d[2]; }
    if (!(v1[ax] * v[ax] > 0.0)) return s0;
    double c = (target - y1[ax]) / v1[ax];
    return s0 + fmin(fmax(c, -0.5 * s0), 0.5 * s0);
}

/* For tests: s_O of points x (bounded or contracted) in their empty voxel of
 * resolution Rk, with the guard of a finest resolution R_O. */
void or_empty_step_batch(int bounded, const double* x, const double* d, int Rk, int R_O, int n, double* out) {
    for (int i = 0; i < n; ++i) {
        const double o[3] = {0.0, 0.0, 0.0};
        double xx[3], y[3], u[3], r;
        or_point(bounded, o, x + 3 * i, 1.0, xx, y, u, &r);
        int ev[3] = {or_vox(u[0], Rk), or_vox(u[1], Rk), or_vox(u[2], Rk)};
        out[i] = or_empty_step(bounded, xx, y, d + 3 * i, r, ev, Rk, R_O, NULL);
    }
}

typedef struct {
    int n_march, n_samples, ambiguous, hit;
    double C_d[3], F[4], A, depth;
    double T;
} or_ray_out;

/* What one marching point decides (Sec. 3.3): the coarse-to-fine occupancy test and,
 * at an empty point, the step: s_O from the coarsest empty level, or the distance
 * step v G (Eq. 9; max(v G, s_O) with dist_rule 1) when that level is coarser than
 * G's grid and G > 0.  The voxel choices read u; the steps read the position. */
typedef struct {
    int empty_level;  /* -1: occupied at every level (a sample) */
    double step;
    double v_exit;    /* s_O: the image's speed across the exit face; 0 for a G step */
} or_decision;

static size_t or_level_word(const or_occ* oc, int k) {
    size_t off = 0;
    for (int j = 0; j < k; ++j) {
        size_t rj = (size_t)(oc->R_O >> j);
        off += or_words(rj * rj * rj);
    }
    return off;
}

static int or_g_shift(const or_occ* oc) {
    int R_G = oc->R_G ? oc->R_G : oc->R_O, g = 0;
    while ((oc->R_O >> g) > R_G) ++g;
    return g;
}

static or_decision or_decide(const or_scene* s, const or_occ* oc, const or_opts* op, const double u[3],
                             const double x[3], const double y[3], const double d[3], double r, double t) {
    or_decision dc = {-1, 0.0, 0.0};
    int ev[3] = {0, 0, 0};
    for (int k = oc->n_levels - 1; k >= 0; --k) {
        int Rk = oc->R_O >> k;
        int c[3] = {or_vox(u[0], Rk), or_vox(u[1], Rk), or_vox(u[2], Rk)};
        size_t bi = (size_t)c[0] + (size_t)Rk * ((size_t)c[1] + (size_t)Rk * (size_t)c[2]);
        if (!or_bit(oc->bits + or_level_word(oc, k), bi)) {
            dc.empty_level = k;
            ev[0] = c[0]; ev[1] = c[1]; ev[2] = c[2];
            break;
        }
    }
    if (dc.empty_level < 0) return dc;
    double s_O = or_empty_step(s->bounded, x, y, d, r, ev, oc->R_O >> dc.empty_level, oc->R_O, &dc.v_exit);
    dc.step = s_O;
    int R_G = oc->R_G ? oc->R_G : oc->R_O;
    if (op->use_dist && oc->dist && dc.empty_level > or_g_shift(oc)) {
        int g = oc->dist[(size_t)or_vox(u[0], R_G) +
                         (size_t)R_G * ((size_t)or_vox(u[1], R_G) + (size_t)R_G * (size_t)or_vox(u[2], R_G))];
        if (g > 0) {
            double B = s->bounded ? 1.0 : 2.0;
            double sg = or_dist_step(s->bounded, x, d, r, g * (2.0 * B / (double)R_G));
            dc.step = op->dist_rule == 1 ? fmax(sg, s_O) : sg;
            if (dc.step != s_O) dc.v_exit = 0.0;
        }
    }
    return dc;
}

/* 1 when a unit-cube coordinate of this point lies within `margin` of a face of the
 * voxels or G cells the decision reads and the decision on the other side of that
 * face differs (another level empty, or an empty step longer or shorter by more
 * than 1e-7 max(1, t)). */
static int or_decision_ambiguous(const or_scene* s, const or_occ* oc, const or_opts* op, const double u[3],
                                 const double x[3], const double y[3], const double d[3], double r, double t,
                                 or_decision dc, double margin) {
    int R_G = oc->R_G ? oc->R_G : oc->R_O;
    int R_max = oc->R_O > R_G ? oc->R_O : R_G;
    for (int a = 0; a < 3; ++a) {
        /* faces of every grid read are faces of the finest one (resolutions are
         * powers of two of one another) */
        double p = u[a] * (double)R_max;
        double f = floor(p + 0.5);
        if (f <= 0.0 || f >= (double)R_max) continue;
        if (fabs(p - f) >= margin * (double)R_max) continue;
        double uo[3] = {u[0], u[1], u[2]};
        double face = f / (double)R_max;
        uo[a] = p >= f ? face - 1e-12 : face + 1e-12;
        or_decision other = or_decide(s, oc, op, uo, x, y, d, r, t);
        if ((other.empty_level < 0) != (dc.empty_level < 0)) return 1;
        if (dc.empty_level >= 0 && fabs(other.step - dc.step) > 1e-7 * fmax(1.0, t)) return 1;
    }
    return 0;
}

/* March one ray and composite (Eq. 2, Eq. 5 before the MLP), in FP64.  The step
 * rule is Eq. 9 with the multi-level occupancy check of Sec. 3.3; the sample step is
 * gamma s_0 (bounded) or gamma s_0 max(1, |x|), and delta_i is that step clipped to
 * the domain's end.  If samples != NULL the per-sample records are written there
 * (capacity max_samples). */
static void or_march(const or_scene* s, const or_occ* oc, const or_opts* op,
                     const double o[3], const double din[3], double t_lo, double t_hi,
                     or_ray_out* res, or_sample* samples, double d_out[3]) {
    memset(res, 0, sizeof *res);
    res->T = 1.0;
    double nn = sqrt(din[0] * din[0] + din[1] * din[1] + din[2] * din[2]);
    double d[3] = {din[0] / nn, din[1] / nn, din[2] / nn};
    if (d_out) { d_out[0] = d[0]; d_out[1] = d[1]; d_out[2] = d[2]; }
    double t_in, t_out;
    if (s->bounded) {
        t_in = -INFINITY;
        t_out = INFINITY;
        for (int a = 0; a < 3; ++a) {
            double t0 = (-1.0 - o[a]) / d[a], t1 = (1.0 - o[a]) / d[a];
            t_in = fmax(t_in, fmin(t0, t1));
            t_out = fmin(t_out, fmax(t0, t1));
        }
    } else {
        /* |o + t d| = r_far */
        double b = o[0] * d[0] + o[1] * d[1] + o[2] * d[2];
        double c = o[0] * o[0] + o[1] * o[1] + o[2] * o[2] - (double)op->r_far * (double)op->r_far;
        double disc = b * b - c;
        if (fabs(disc) <= OR_AMB_END * fabs(c)) res->ambiguous = 1;
        if (!(disc >= 0.0)) return;
        t_in = -b - sqrt(disc);
        t_out = -b + sqrt(disc);
    }
    double t = fmax(fmax(t_in, (double)op->t_min), t_lo);
    t_out = fmin(t_out, t_hi);
    if (fabs(t - t_out) <= OR_AMB_END * fmax(1.0, fabs(t))) res->ambiguous = 1;
    if (!(t < t_out)) return;
    res->hit = 1;
    const double dt0 = (double)op->step_base * (double)op->step_gamma;
    const double t_start = t;
    long lat_k = 0;
    double T = 1.0;
    while (t < t_out && res->n_march < op->max_march && res->n_samples < op->max_samples) {
        res->n_march++;
        double x[3], y[3], u[3], r;
        or_point(s->bounded, o, d, t, x, y, u, &r);
        or_decision dc = or_decide(s, oc, op, u, x, y, d, r, t);
        if (or_decision_ambiguous(s, oc, op, u, x, y, d, r, t, dc, OR_AMB_U)) res->ambiguous = 1;
        double step;
        int sampled = 0;
        if (dc.empty_level < 0) {
            /* occupied at every level: a sample */
            double dt = s->bounded ? dt0 : dt0 * fmax(1.0, r);
            double delta = fmin(dt, t_out - t);
            double f[OR_NFEAT];
            or_features(s, op, u, f);
            double sigma = exp(f[0]);
            double alpha = 1.0 - exp(-sigma * delta);
            double w = T * alpha;
            if (samples) {
                or_sample* sp = samples + res->n_samples;
                sp->t = t; sp->delta = delta;
                sp->u[0] = u[0]; sp->u[1] = u[1]; sp->u[2] = u[2];
                sp->sigma_raw = f[0]; sp->sigma = sigma; sp->alpha = alpha; sp->T_before = T;
                memcpy(sp->f, f, sizeof f);
            }
            for (int k = 0; k < 3; ++k) res->C_d[k] += w * f[1 + k];
            for (int k = 0; k < 4; ++k) res->F[k] += w * f[4 + k];
            res->A += w;
            res->depth += w * t;
            T *= 1.0 - alpha;
            res->n_samples++;
            sampled = 1;
            step = dt;
            if (fabs(T - (double)op->t_term) <= OR_AMB_T * (double)op->t_term) res->ambiguous = 1;
            if (T < (double)op->t_term) break;   /* strict: the crossing sample is kept */
        } else {
            step = dc.step;
        }
        if (op->lattice_snap && s->bounded) {
            /* next point on the lattice t_start + k dt0: the next index after a
             * sample, else the first lattice point at or beyond t + step */
            if (sampled) lat_k += 1;
            else {
                double q = (t + step - t_start) / dt0;
                double kq = floor(q);
                if (fabs(q - floor(q + 0.5)) <= OR_AMB_LATTICE) res->ambiguous = 1;
                lat_k = (long)kq > lat_k + 1 ? (long)kq : lat_k + 1;
            }
            t = t_start + (double)lat_k * dt0;
        } else {
            t = t + step;
        }
        if (fabs(t - t_out) <= OR_AMB_END * fmax(1.0, fabs(t))) res->ambiguous = 1;
    }
    res->T = T;
}

/* Pinhole ray of pixel (col, row) of a camera [c2w(3x4) fx fy cx cy] through the
 * pixel centre; OpenCV axes (x right, y down, z forward). */
static void or_camera_ray(const float* cam, int col, int row, double o[3], double d[3]) {
    double px = ((double)col + 0.5 - (double)cam[14]) / (double)cam[12];
    double py = ((double)row + 0.5 - (double)cam[15]) / (double)cam[13];
    for (int r = 0; r < 3; ++r) {
        d[r] = (double)cam[4 * r + 0] * px + (double)cam[4 * r + 1] * py + (double)cam[4 * r + 2];
        o[r] = (double)cam[4 * r + 3];
    }
}

/* Ray i of a batch: pixel i (or pix[i]) of the cameras, view-major then row-major,
 * or the i-th explicit ray. */
static void or_ray_input(const float* cams, int n_cams, int W, int H, const int32_t* pix,
                         const float* rays_o, const float* rays_d, int i, double o[3], double d[3]) {
    if (cams) {
        int64_t id = pix ? pix[i] : i;
        int64_t v = id / ((int64_t)W * H), rem = id % ((int64_t)W * H);
        if (v >= n_cams) v = n_cams - 1;
        or_camera_ray(cams + 16 * v, (int)(rem % W), (int)(rem / W), o, d);
    } else {
        for (int a = 0; a < 3; ++a) { o[a] = rays_o[3 * i + a]; d[a] = rays_d[3 * i + a]; }
    }
}

void or_camera_rays(const float* cams, int n_cams, int W, int H, const int32_t* pix, int n,
                    double* o_out, double* d_out) {
    for (int i = 0; i < n; ++i) or_ray_input(cams, n_cams, W, H, pix, NULL, NULL, i, o_out + 3 * i, d_out + 3 * i);
}

/* Final colour: sigmoid(C_d + MLP_psi(C_d, F, SH(d))) (Eq. 5 then the colour
 * sigmoid of Sec. S2.1), composited over the background with the accumulated
 * opacity A (the paper's C when A = 1). */
static void or_shade(const or_scene* s, const or_opts* op, const or_ray_out* rr, const double d[3],
                     double rgb[3], double x_out[OR_MLP_IN], double acts[256], double z_out[3]) {
    double x[OR_MLP_IN];
    memset(x, 0, sizeof x);
    for (int k = 0; k < 3; ++k) x[k] = rr->C_d[k];
    for (int k = 0; k < 4; ++k) x[3 + k] = rr->F[k];
    or_sh16(d, x + 7);
    double y[3];
    or_mlp_forward(s, x, y, acts);
    for (int k = 0; k < 3; ++k) {
        double z = rr->C_d[k] + y[k];
        if (z_out) z_out[k] = z;
        rgb[k] = rr->A * or_sigmoid(z) + (1.0 - rr->A) * op->bg[k];
    }
    if (x_out) memcpy(x_out, x, sizeof x);
}

/* Render n rays (explicit rays, or camera pixels when cams != NULL).  Outputs:
 * rgb [n][3], depth [n] (= sum w_i t_i), opacity [n] (= sum w_i), stats [n][2]
 * (marching points, samples), ambiguous [n] (1 when a termination test came
 * within 3e-5 relative of the threshold, so FP32 may decide it otherwise), state
 * [n][9] = C_d(3), F(4), A, depth. */
void or_render(const or_scene* s, const or_occ* oc, const or_opts* op,
               const float* cams, int n_cams, int W, int H, const int32_t* pix,
               const float* rays_o, const float* rays_d, int n, const float* interval,
               double* rgb, double* depth, double* opacity, int32_t* stats,
               int32_t* ambiguous, double* state) {
    /* rays are independent: one ray per loop iteration, spread over host threads */
    #pragma omp parallel for schedule(dynamic, 16)
    for (int i = 0; i < n; ++i) {
        double o[3], dv[3], d[3];
        or_ray_input(cams, n_cams, W, H, pix, rays_o, rays_d, i, o, dv);
        double tlo = interval ? interval[2 * i] : -INFINITY, thi = interval ? interval[2 * i + 1] : INFINITY;
        or_ray_out rr;
        or_march(s, oc, op, o, dv, tlo, thi, &rr, NULL, d);
        double c[3];
        if (rr.hit) or_shade(s, op, &rr, d, c, NULL, NULL, NULL);
        else { c[0] = op->bg[0]; c[1] = op->bg[1]; c[2] = op->bg[2]; }
        for (int k = 0; k < 3; ++k) rgb[3 * i + k] = c[k];
        depth[i] = rr.depth;
        opacity[i] = rr.A;
        if (stats) { stats[2 * i] = rr.n_march; stats[2 * i + 1] = rr.n_samples; }
        if (ambiguous) ambiguous[i] = rr.ambiguous;
        if (state) {
            for (int k = 0; k < 3; ++k) state[9 * i + k] = rr.C_d[k];
            for (int k = 0; k < 4; ++k) state[9 * i + 3 + k] = rr.F[k];
            state[9 * i + 7] = rr.A;
            state[9 * i + 8] = rr.depth;
        }
    }
}

/* Per-sample dump of one ray: t, delta, u, sigma, weight (for tests). */
int or_ray_samples(const or_scene* s, const or_occ* oc, const or_opts* op, const float of[3],
                   const float df[3], int cap, double* out /* [cap][7] */) {
    const double o[3] = {of[0], of[1], of[2]}, d[3] = {df[0], df[1], df[2]};
    or_sample* sm = (or_sample*)malloc(sizeof(or_sample) * (size_t)(op->max_samples > 0 ? op->max_samples : 1));
    or_ray_out rr;
    or_march(s, oc, op, o, d, -INFINITY, INFINITY, &rr, sm, NULL);
    int n = rr.n_samples < cap ? rr.n_samples : cap;
    for (int i = 0; i < n; ++i) {
        out[7 * i + 0] = sm[i].t;
        out[7 * i + 1] = sm[i].delta;
        out[7 * i + 2] = sm[i].u[0];
        out[7 * i + 3] = sm[i].u[1];
        out[7 * i + 4] = sm[i].u[2];
        out[7 * i + 5] = sm[i].sigma;
        out[7 * i + 6] = sm[i].T_before * sm[i].alpha;
    }
    free(sm);
    return rr.n_samples;
}

/* ------------------------------------------------------------ reverse pass */

/* Reverse of Eq. 6-8 (and of Table 3's other forms) at one sample u: given the
 * sample's feature cotangent g_f = dL/d f (f = [sigma_raw, c_d(3), v_s(4)]), add the
 * gradients of the coarse vertices, the gate logits (coarse channels or the constant
 * logits) or the tiny MLP's weights, and the fine entries.  kink (may be NULL) is set
 * when a hidden unit of the MLP form lies within 1e-5 relative of its ReLU kink. */
static void or_feature_reverse(const or_scene* s, const or_opts* op, const double u[3], const double g_f[OR_NFEAT],
                               double* g_tables, double* g_coarse, double* g_attn_inv, double* g_agg_mlp,
                               int32_t* kink) {
    int nch = or_coarse_channels(s->L, s->aggregation);
    uint32_t T = 1u << s->T_log2;
    /* Eq. 6-8 reverse: coarse part, attention logits, fine levels */
    double coarse[OR_NFEAT + 2 * OR_MAXL], g_coarse_v[OR_NFEAT + 2 * OR_MAXL];
    int base[3];
    double wc[3];
    memset(coarse, 0, sizeof coarse);
    memset(g_coarse_v, 0, sizeof g_coarse_v);
    or_cell(u, s->R_C, base, wc);
    size_t cv[8];
    double cwt[8];
    for (int c = 0; c < 8; ++c) {
        int xx = base[0] + (c & 1), yy = base[1] + ((c >> 1) & 1), zz = base[2] + ((c >> 2) & 1);
        cv[c] = (size_t)xx + (size_t)s->R_C * ((size_t)yy + (size_t)s->R_C * zz);
        cwt[c] = or_corner_weight(wc, c);
        for (int ch = 0; ch < nch; ++ch) coarse[ch] += cwt[c] * s->coarse[cv[c] * nch + ch];
    }
    for (int ch = 0; ch < OR_NFEAT; ++ch) g_coarse_v[ch] = g_f[ch];
    if (s->aggregation == 5) {
        /* Instant-NGP's tiny MLP in place of the attention: f = f~ + W2 relu(W1 x),
         * x = [f^1, ..., f^L].  Its reverse: dW2 += g_f relu(h)^T, g_h = (W2^T g_f)
         * where h > 0, dW1 += g_h x^T, g_x = W1^T g_h, then each level's entries. */
        int nx = OR_NFEAT * s->L;
        const double* w1 = s->agg_mlp;
        const double* w2 = s->agg_mlp + (size_t)OR_AGG_HIDDEN * nx;
        double xs[OR_NFEAT * OR_MAXL], dxs[OR_NFEAT * OR_MAXL], h[OR_AGG_HIDDEN], gh[OR_AGG_HIDDEN];
        double gx[OR_NFEAT * OR_MAXL];
        uint64_t ents[OR_MAXL][8];
        double ews[OR_MAXL][8];
        memset(xs, 0, sizeof xs);
        memset(dxs, 0, sizeof dxs);
        for (int l = 0; l < s->L; ++l) {
            int bl[3];
            double wl[3], gd[3][OR_NFEAT];
            memset(gd, 0, sizeof gd);
            or_cell(u, s->N[l], bl, wl);
            uint64_t off = or_level_offset(s->N, s->L, s->T_log2, l);
            for (int c = 0; c < 8; ++c) {
                int xx = bl[0] + (c & 1), yy = bl[1] + ((c >> 1) & 1), zz = bl[2] + ((c >> 2) & 1);
                ents[l][c] = off + or_level_entry(s->N[l], T, xx, yy, zz);
                ews[l][c] = or_corner_weight(wl, c);
                for (int ch = 0; ch < OR_NFEAT; ++ch) {
                    double v = s->tables[ents[l][c] * OR_NFEAT + ch];
                    xs[OR_NFEAT * l + ch] += ews[l][c] * v;
                    /* d/du_a of the corner weight: +-(N-1) times the other two factors */
                    for (int a = 0; a < 3; ++a) {
                        double dw = (double)(s->N[l] - 1) * (((c >> a) & 1) ? 1.0 : -1.0);
                        for (int b = 0; b < 3; ++b)
                            if (b != a) dw *= ((c >> b) & 1) ? wl[b] : 1.0 - wl[b];
                        gd[a][ch] += dw * v;
                    }
                }
            }
            for (int ch = 0; ch < OR_NFEAT; ++ch)
                dxs[OR_NFEAT * l + ch] = (fabs(gd[0][ch]) + fabs(gd[1][ch]) + fabs(gd[2][ch])) * or_kink_pos_err;
        }
        for (int j = 0; j < OR_AGG_HIDDEN; ++j) {
            double acc = 0.0, mag = 0.0, sens = 0.0;
            for (int q = 0; q < nx; ++q) {
                acc += w1[(size_t)j * nx + q] * xs[q];
                mag += fabs(w1[(size_t)j * nx + q] * xs[q]);
                sens += fabs(w1[(size_t)j * nx + q]) * dxs[q];
            }
            h[j] = acc;
            /* a unit this close to its ReLU kink may switch sides in FP32 (its own
             * rounding, or the FP32 sample position moving the level features by up
             * to their gradient times the position error): the ray's gradient is then
             * not comparable element by element */
            if (kink && fabs(acc) <= 1e-5 * mag + sens) *kink = 1;
        }
        for (int j = 0; j < OR_AGG_HIDDEN; ++j) {
            double ga = 0.0;
            for (int k = 0; k < OR_NFEAT; ++k) ga += w2[k * OR_AGG_HIDDEN + j] * g_f[k];
            gh[j] = h[j] > 0.0 ? ga : 0.0;
        }
        if (g_agg_mlp) {
            double* gw2 = g_agg_mlp + (size_t)OR_AGG_HIDDEN * nx;
            for (int k = 0; k < OR_NFEAT; ++k)
                for (int j = 0; j < OR_AGG_HIDDEN; ++j) gw2[k * OR_AGG_HIDDEN + j] += g_f[k] * fmax(h[j], 0.0);
            for (int j = 0; j < OR_AGG_HIDDEN; ++j)
                for (int q = 0; q < nx; ++q) g_agg_mlp[(size_t)j * nx + q] += gh[j] * xs[q];
        }
        for (int q = 0; q < nx; ++q) {
            double acc = 0.0;
            for (int j = 0; j < OR_AGG_HIDDEN; ++j) acc += w1[(size_t)j * nx + q] * gh[j];
            gx[q] = acc;
        }
        for (int l = 0; l < s->L; ++l)
            for (int c = 0; c < 8; ++c)
                for (int ch = 0; ch < OR_NFEAT; ++ch)
                    g_tables[ents[l][c] * OR_NFEAT + ch] += ews[l][c] * gx[OR_NFEAT * l + ch];
    }
    for (int l = 0; l < (s->aggregation == 5 ? 0 : s->L); ++l) {
        /* the gates of this level and whether each is shared by both modalities */
        double om = 1.0, be = 1.0;
        int shared = 0;
        switch (s->aggregation) {
            case 0:
                if (op->attn_mode == 2) { om = or_sigmoid(coarse[OR_NFEAT + 2 * l]); be = om; shared = 1; }
                else if (op->attn_mode == 0) {
                    om = or_sigmoid(coarse[OR_NFEAT + 2 * l]);
                    be = or_sigmoid(coarse[OR_NFEAT + 2 * l + 1]);
                }
                break;
            case 1: om = or_sigmoid(coarse[OR_NFEAT + l]); be = om; shared = 1; break;
            case 2: om = or_sigmoid(s->attn_inv[2 * l]); be = or_sigmoid(s->attn_inv[2 * l + 1]); break;
            case 3: om = or_sigmoid(s->attn_inv[l]); be = om; shared = 1; break;
            default: break; /* 4: plain sum */
        }
        int bl[3];
        double wl[3];
        or_cell(u, s->N[l], bl, wl);
        uint64_t off = or_level_offset(s->N, s->L, s->T_log2, l);
        double fl[OR_NFEAT];
        memset(fl, 0, sizeof fl);
        uint64_t ent[8];
        double ew[8];
        for (int c = 0; c < 8; ++c) {
            int xx = bl[0] + (c & 1), yy = bl[1] + ((c >> 1) & 1), zz = bl[2] + ((c >> 2) & 1);
            ent[c] = off + or_level_entry(s->N[l], T, xx, yy, zz);
            ew[c] = or_corner_weight(wl, c);
            for (int ch = 0; ch < OR_NFEAT; ++ch) fl[ch] += ew[c] * s->tables[ent[c] * OR_NFEAT + ch];
        }
        double g_om = fl[0] * g_f[0], g_be = 0.0;
        for (int ch = 1; ch < OR_NFEAT; ++ch) g_be += fl[ch] * g_f[ch];
        /* gate gradients through the sigmoid, to the logit they come from */
        double lo_g = shared ? (g_om + g_be) * om * (1.0 - om) : g_om * om * (1.0 - om);
        double lb_g = shared ? 0.0 : g_be * be * (1.0 - be);
        if (s->aggregation == 0 && op->attn_mode == 0) {
            g_coarse_v[OR_NFEAT + 2 * l] += lo_g;
            g_coarse_v[OR_NFEAT + 2 * l + 1] += lb_g;
        } else if (s->aggregation == 0 && op->attn_mode == 2) {
            g_coarse_v[OR_NFEAT + 2 * l] += lo_g;
        } else if (s->aggregation == 1) {
            g_coarse_v[OR_NFEAT + l] += lo_g;
        } else if (s->aggregation == 2 && g_attn_inv) {
            g_attn_inv[2 * l] += lo_g;
            g_attn_inv[2 * l + 1] += lb_g;
        } else if (s->aggregation == 3 && g_attn_inv) {
            g_attn_inv[l] += lo_g;
        }
        for (int c = 0; c < 8; ++c) {
            g_tables[ent[c] * OR_NFEAT + 0] += ew[c] * om * g_f[0];
            for (int ch = 1; ch < OR_NFEAT; ++ch) g_tables[ent[c] * OR_NFEAT + ch] += ew[c] * be * g_f[ch];
        }
    }
    for (int c = 0; c < 8; ++c)
        for (int ch = 0; ch < nch; ++ch) g_coarse[cv[c] * nch + ch] += cwt[c] * g_coarse_v[ch];
}

/* Reverse-mode derivative of or_render with respect to the fine tables, the coarse
 * grid and the MLP weights, accumulated (+=) into g_tables, g_coarse, g_mlp.
 *
 * Compositing (Eq. 2 and Eq. 5): Q = sum_i w_i q_i with w_i = T_i alpha_i,
 * alpha_i = 1 - exp(-sigma_i delta_i), T_i = prod_{j<i} (1 - alpha_j), so
 *   dQ/dq_i     = w_i
 *   dQ/dsigma_i = delta_i (T_{i+1} q_i - sum_{j>i} w_j q_j),
 * the second sum written out over the later samples of the ray.  The density
 * activation exp has the truncated derivative exp(min(sigma_raw, 15))
 * (Sec. S2.1, following Instant-NGP).  The sample set itself does not depend on
 * the parameters except through the termination test, whose derivative is zero. */
void or_render_backward(const or_scene* s, const or_occ* oc, const or_opts* op,
                        const float* cams, int n_cams, int W, int H, const int32_t* pix,
                        const float* rays_o, const float* rays_d, int n,
                        const double* d_rgb, const double* d_depth, const double* d_opacity,
                        double* g_tables, double* g_coarse, double* g_mlp, double* g_attn_inv,
                        double* g_agg_mlp, int32_t* kink) {
    int cap = op->max_samples > 0 ? op->max_samples : 1;
    or_sample* sm = (or_sample*)malloc(sizeof(or_sample) * (size_t)cap);
    double* qg = (double*)malloc(sizeof(double) * (size_t)cap);
    for (int i = 0; i < n; ++i) {
        double o[3], dv[3], d[3];
        or_ray_input(cams, n_cams, W, H, pix, rays_o, rays_d, i, o, dv);
        or_ray_out rr;
        or_march(s, oc, op, o, dv, -INFINITY, INFINITY, &rr, sm, d);
        if (!rr.hit) continue;
        double x[OR_MLP_IN], acts[256], z[3], rgb[3];
        or_shade(s, op, &rr, d, rgb, x, acts, z);
        double g_z[3], g_A = d_opacity ? d_opacity[i] : 0.0;
        for (int k = 0; k < 3; ++k) {
            double sg = or_sigmoid(z[k]);
            double gr = d_rgb ? d_rgb[3 * i + k] : 0.0;
            g_z[k] = gr * rr.A * sg * (1.0 - sg);
            g_A += gr * (sg - op->bg[k]);
        }
        /* MLP reverse pass: layer inputs are x, then relu of the previous pre-activation */
        double g_cur[256], g_in[256];
        memcpy(g_cur, g_z, sizeof g_z);
        size_t woff[16], aoff[16];
        size_t wo = 0, ao = 0;
        for (int k = 0; k < s->mlp_layers; ++k) {
            woff[k] = wo; aoff[k] = ao;
            wo += (size_t)or_mlp_out(s, k) * or_mlp_in(s, k);
            ao += or_mlp_out(s, k);
        }
        for (int k = s->mlp_layers - 1; k >= 0; --k) {
            int no = or_mlp_out(s, k), ni = or_mlp_in(s, k);
            const double* Wk = s->mlp_w + woff[k];
            double hin[256];
            for (int j = 0; j < ni; ++j) {
                if (k == 0) hin[j] = x[j];
                else { double pa = acts[aoff[k - 1] + j]; hin[j] = pa > 0.0 ? pa : 0.0; }
            }
            for (int oo = 0; oo < no; ++oo)
                for (int j = 0; j < ni; ++j) g_mlp[woff[k] + (size_t)oo * ni + j] += g_cur[oo] * hin[j];
            for (int j = 0; j < ni; ++j) {
                double acc = 0.0;
                for (int oo = 0; oo < no; ++oo) acc += Wk[(size_t)oo * ni + j] * g_cur[oo];
                g_in[j] = acc;
            }
            if (k > 0)
                for (int j = 0; j < ni; ++j) g_cur[j] = acts[aoff[k - 1] + j] > 0.0 ? g_in[j] : 0.0;
        }
        double g_Cd[3], g_F[4], g_D = d_depth ? d_depth[i] : 0.0;
        for (int k = 0; k < 3; ++k) g_Cd[k] = g_z[k] + g_in[k];
        for (int k = 0; k < 4; ++k) g_F[k] = g_in[3 + k];
        /* per-sample scalar q_i . g (the gradient-weighted quantity composited) */
        int ns = rr.n_samples;
        for (int a = 0; a < ns; ++a) {
            double q = g_A + g_D * sm[a].t;
            for (int k = 0; k < 3; ++k) q += g_Cd[k] * sm[a].f[1 + k];
            for (int k = 0; k < 4; ++k) q += g_F[k] * sm[a].f[4 + k];
            qg[a] = q;
        }
        for (int a = 0; a < ns; ++a) {
            const or_sample* sp = sm + a;
            double w = sp->T_before * sp->alpha;
            double T_next = sp->T_before * (1.0 - sp->alpha);
            double later = 0.0;
            for (int b = a + 1; b < ns; ++b) later += sm[b].T_before * sm[b].alpha * qg[b];
            double g_sigma = sp->delta * (T_next * qg[a] - later);
            double g_f[OR_NFEAT];
            g_f[0] = g_sigma * exp(fmin(sp->sigma_raw, 15.0));
            for (int k = 0; k < 3; ++k) g_f[1 + k] = w * g_Cd[k];
            for (int k = 0; k < 4; ++k) g_f[4 + k] = w * g_F[k];
            or_feature_reverse(s, op, sp->u, g_f, g_tables, g_coarse, g_attn_inv, g_agg_mlp, kink ? kink + i : NULL);
        }
    }
    free(sm);
    free(qg);
}

/* Scalar loss used by the gradient tests: sum of the rendered outputs weighted by
 * fixed cotangents, L = <d_rgb, rgb> + <d_depth, depth> + <d_opacity, A>. */
double or_render_dot(const or_scene* s, const or_occ* oc, const or_opts* op,
                     const float* cams, int n_cams, int W, int H, const int32_t* pix,
                     const float* rays_o, const float* rays_d, int n,
                     const double* d_rgb, const double* d_depth, const double* d_opacity) {
    double* rgb = (double*)malloc(sizeof(double) * 3 * (size_t)n);
    double* dep = (double*)malloc(sizeof(double) * (size_t)n);
    double* opa = (double*)malloc(sizeof(double) * (size_t)n);
    or_render(s, oc, op, cams, n_cams, W, H, pix, rays_o, rays_d, n, NULL, rgb, dep, opa, NULL, NULL, NULL);
    double L = 0.0;
    for (int i = 0; i < n; ++i) {
        for (int k = 0; k < 3; ++k) L += (d_rgb ? d_rgb[3 * i + k] : 0.0) * rgb[3 * i + k];
        L += (d_depth ? d_depth[i] : 0.0) * dep[i] + (d_opacity ? d_opacity[i] : 0.0) * opa[i];
    }
    free(rgb); free(dep); free(opa);
    return L;
}

#ifdef _OPENMP
#include <omp.h>
void or_set_threads(int n) { omp_set_num_threads(n); }
int or_max_threads(void) { return omp_get_max_threads(); }
#else
void or_set_threads(int n) { (void)n; }
int or_max_threads(void) { return 1; }
#endif

/* ------------------------------------------------------------ training step */

/* Photometric L2 loss L = scale * sum (rgb - target)^2 and its gradient
 * d_rgb = 2 scale (rgb - target) (the configs' training objective). */
double or_l2_loss(const double* rgb, const double* target, int64_t n, double scale, double* d_rgb) {
    double L = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double e = rgb[i] - target[i];
        L += scale * e * e;
        if (d_rgb) d_rgb[i] = 2.0 * scale * e;
    }
    return L;
}

/* One Adam step (Kingma and Ba; the optimiser of Sec. S2.4): m = b1 m + (1-b1) g,
 * v = b2 v + (1-b2) g^2, p -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps). */
void or_adam_step(double* p, const double* g, double* m, double* v, int64_t n, double lr, double b1, double b2,
                  double eps, int step) {
    double c1 = 1.0 - pow(b1, step), c2 = 1.0 - pow(b2, step);
    for (int64_t i = 0; i < n; ++i) {
        m[i] = b1 * m[i] + (1.0 - b1) * g[i];
        v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
        p[i] -= lr * (m[i] / c1) / (sqrt(v[i] / c2) + eps);
    }
}

/* ------------------------------------------------------- learned proposal */
/* Not in the paper (it calls adaptive sampling orthogonal, Sec. 2).  A small MLP
 * maps a ray (o / in_scale, d) to [t_near, t_far] and the expected opacity A^:
 *   h1 = relu(W0 e + b0), h2 = relu(W1 h1 + b1), z = W2 h2 + b2,
 *   t_near = t_scale sigmoid(z0), t_far = t_scale sigmoid(z1), A^ = sigmoid(z2).
 * Parameters, flat: W0 [W][6], b0 [W], W1 [W][W], b1 [W], W2 [3][W], b2 [3].
 * Loss per ray: A* (a_n sl1((t_near - t_near*)/t_scale) + a_f sl1((t_far - t_far*)/t_scale))
 * + (A^ - A*)^2, sl1 = smooth L1 with beta = 0.01, a_n = 4 when t_near is late
 * (> target) else 1, a_f = 4 when t_far is early (< target) else 1: intervals err
 * on the wide side, where a miss costs marching points instead of opacity. */

#define OR_PROP_IN 6

static void or_prop_input(const float o[3], const float d[3], double in_scale, double e[OR_PROP_IN]) {
    double n = sqrt((double)d[0] * d[0] + (double)d[1] * d[1] + (double)d[2] * d[2]);
    for (int a = 0; a < 3; ++a) {
        e[a] = (double)o[a] / in_scale;
        e[3 + a] = (double)d[a] / n;
    }
}

static double or_sl1(double x, double beta) {
    double ax = fabs(x);
    return ax < beta ? 0.5 * x * x / beta : ax - 0.5 * beta;
}

static double or_sl1_grad(double x, double beta) {
    double ax = fabs(x);
    return ax < beta ? x / beta : (x > 0 ? 1.0 : -1.0);
}

/* Forward for n rays: out [n][3] = t_near, t_far, A^. */
void or_prop_forward(const double* w, int W, const float* rays_o, const float* rays_d, int n, double in_scale,
                     double t_scale, double* out) {
    const double *W0 = w, *b0 = W0 + W * OR_PROP_IN, *W1 = b0 + W, *b1 = W1 + W * W, *W2 = b1 + W, *b2 = W2 + 3 * W;
    for (int i = 0; i < n; ++i) {
        double e[OR_PROP_IN], h1[256], h2[256], z[3];
        or_prop_input(rays_o + 3 * i, rays_d + 3 * i, in_scale, e);
        for (int o = 0; o < W; ++o) {
            double a = b0[o];
            for (int k = 0; k < OR_PROP_IN; ++k) a += W0[o * OR_PROP_IN + k] * e[k];
            h1[o] = a > 0 ? a : 0;
        }
        for (int o = 0; o < W; ++o) {
            double a = b1[o];
            for (int k = 0; k < W; ++k) a += W1[o * W + k] * h1[k];
            h2[o] = a > 0 ? a : 0;
        }
        for (int o = 0; o < 3; ++o) {
            double a = b2[o];
            for (int k = 0; k < W; ++k) a += W2[o * W + k] * h2[k];
            z[o] = a;
        }
        out[3 * i + 0] = t_scale * or_sigmoid(z[0]);
        out[3 * i + 1] = t_scale * or_sigmoid(z[1]);
        out[3 * i + 2] = or_sigmoid(z[2]);
    }
}

/* Mean loss over n rays against targets [n][3] = t_near*, t_far*, A*, and its
 * gradient (accumulated into g, same layout as w). */
double or_prop_loss_grad(const double* w, int W, const float* rays_o, const float* rays_d, int n, double in_scale,
                         double t_scale, const double* targets, double* g) {
    const double *W0 = w, *b0 = W0 + W * OR_PROP_IN, *W1 = b0 + W, *b1 = W1 + W * W, *W2 = b1 + W, *b2 = W2 + 3 * W;
    double *gW0 = g, *gb0 = gW0 + W * OR_PROP_IN, *gW1 = gb0 + W, *gb1 = gW1 + W * W, *gW2 = gb1 + W, *gb2 = gW2 + 3 * W;
    double total = 0.0;
    const double beta = 0.01, inv_n = 1.0 / (double)n;
    for (int i = 0; i < n; ++i) {
        double e[OR_PROP_IN], a1[256], h1[256], a2[256], h2[256], z[3];
        or_prop_input(rays_o + 3 * i, rays_d + 3 * i, in_scale, e);
        for (int o = 0; o < W; ++o) {
            double a = b0[o];
            for (int k = 0; k < OR_PROP_IN; ++k) a += W0[o * OR_PROP_IN + k] * e[k];
            a1[o] = a;
            h1[o] = a > 0 ? a : 0;
        }
        for (int o = 0; o < W; ++o) {
            double a = b1[o];
            for (int k = 0; k < W; ++k) a += W1[o * W + k] * h1[k];
            a2[o] = a;
            h2[o] = a > 0 ? a : 0;
        }
        for (int o = 0; o < 3; ++o) {
            double a = b2[o];
            for (int k = 0; k < W; ++k) a += W2[o * W + k] * h2[k];
            z[o] = a;
        }
        const double *tg = targets + 3 * i;
        double s0 = or_sigmoid(z[0]), s1 = or_sigmoid(z[1]), s2 = or_sigmoid(z[2]);
        double x0 = (t_scale * s0 - tg[0]) / t_scale, x1 = (t_scale * s1 - tg[1]) / t_scale;
        /* conservative intervals: a late t_near or an early t_far costs 4x */
        double an = x0 > 0 ? 4.0 : 1.0, af = x1 < 0 ? 4.0 : 1.0;
        double L = tg[2] * (an * or_sl1(x0, beta) + af * or_sl1(x1, beta)) + (s2 - tg[2]) * (s2 - tg[2]);
        total += L * inv_n;
        double gz[3];
        gz[0] = inv_n * tg[2] * an * or_sl1_grad(x0, beta) * s0 * (1 - s0);
        gz[1] = inv_n * tg[2] * af * or_sl1_grad(x1, beta) * s1 * (1 - s1);
        gz[2] = inv_n * 2.0 * (s2 - tg[2]) * s2 * (1 - s2);
        double gh2[256], ga2[256], gh1[256], ga1[256];
        for (int k = 0; k < W; ++k) gh2[k] = 0.0;
        for (int o = 0; o < 3; ++o) {
            gb2[o] += gz[o];
            for (int k = 0; k < W; ++k) {
                gW2[o * W + k] += gz[o] * h2[k];
                gh2[k] += W2[o * W + k] * gz[o];
            }
        }
        for (int k = 0; k < W; ++k) { ga2[k] = a2[k] > 0 ? gh2[k] : 0.0; gh1[k] = 0.0; }
        for (int o = 0; o < W; ++o) {
            gb1[o] += ga2[o];
            for (int k = 0; k < W; ++k) {
                gW1[o * W + k] += ga2[o] * h1[k];
                gh1[k] += W1[o * W + k] * ga2[o];
            }
        }
        for (int k = 0; k < W; ++k) ga1[k] = a1[k] > 0 ? gh1[k] : 0.0;
        for (int o = 0; o < W; ++o) {
            gb0[o] += ga1[o];
            for (int k = 0; k < OR_PROP_IN; ++k) gW0[o * OR_PROP_IN + k] += ga1[o] * e[k];
        }
    }
    return total;
}

/* Training targets from the plain render (per ray): with the final opacity A,
 * t_near* = t_i of the first sample whose cumulative weight exceeds 0.005 A, and
 * t_far* = t_i + delta_i of the first sample whose cumulative weight reaches
 * 0.995 A; A* = A.  Rays without samples get (0, 0, 0). */
void or_prop_targets(const or_scene* s, const or_occ* oc, const or_opts* op, const float* cams, int n_cams, int W,
                     int H, const int32_t* pix, const float* rays_o, const float* rays_d, int n, double* targets) {
    int cap = op->max_samples > 0 ? op->max_samples : 1;
    #pragma omp parallel
    {
        or_sample* sm = (or_sample*)malloc(sizeof(or_sample) * (size_t)cap);
        #pragma omp for schedule(dynamic, 16)
        for (int i = 0; i < n; ++i) {
            double o[3], dv[3];
            or_ray_input(cams, n_cams, W, H, pix, rays_o, rays_d, i, o, dv);
            or_ray_out rr;
            or_march(s, oc, op, o, dv, -INFINITY, INFINITY, &rr, sm, NULL);
            double tn = 0.0, tf = 0.0, cum = 0.0;
            int got_near = 0, got_far = 0;
            for (int k = 0; k < rr.n_samples; ++k) {
                cum += sm[k].T_before * sm[k].alpha;
                if (!got_near && cum > 0.005 * rr.A) { tn = sm[k].t; got_near = 1; }
                if (!got_far && cum >= 0.995 * rr.A) { tf = sm[k].t + sm[k].delta; got_far = 1; }
            }
            if (rr.n_samples > 0 && !got_far) tf = sm[rr.n_samples - 1].t + sm[rr.n_samples - 1].delta;
            targets[3 * i + 0] = tn;
            targets[3 * i + 1] = tf;
            targets[3 * i + 2] = rr.A;
        }
        free(sm);
    }
}

/* ------------------------------------------------------- occupancy pipeline */

/* Occupancy from the model's own density (Sec. S2.5): voxel (i, j, k) of an R^3
 * grid over the unit cube (x fastest) is occupied when sigma = exp(sigma_raw) at
 * its centre u = ((i, j, k) + 1/2) / R exceeds sigma_thr.  sigma_out (NULL
 * allowed) receives sigma per voxel. */
void or_occupancy_density(const or_scene* s, const or_opts* op, int R, double sigma_thr, uint8_t* occ,
                          double* sigma_out) {
    long n = (long)R * R * R;
    #pragma omp parallel for schedule(static)
    for (long v = 0; v < n; ++v) {
        int i = (int)(v % R), j = (int)((v / R) % R), k = (int)(v / ((long)R * R));
        double u[3] = {(i + 0.5) / R, (j + 0.5) / R, (k + 0.5) / R};
        double f[OR_NFEAT];
        or_features(s, op, u, f);
        double sg = exp(f[0]);
        occ[v] = sg > sigma_thr ? 1 : 0;
        if (sigma_out) sigma_out[v] = sg;
    }
}

/* Visibility (Sec. S2.5, after MERF): every ray is marched and composited as in
 * the render; each sample whose weight T_i alpha_i exceeds w_thr marks the voxel
 * of its unit-cube position in an R^3 grid.  vis is only ever set (the caller
 * clears it); wmax (NULL allowed, caller-initialised) receives the largest weight
 * per voxel. */
void or_occupancy_visibility(const or_scene* s, const or_occ* oc, const or_opts* op,
                             const float* cams, int n_cams, int W, int H, const int32_t* pix,
                             const float* rays_o, const float* rays_d, int n, int R, double w_thr,
                             uint8_t* vis, double* wmax) {
    or_sample* sm = (or_sample*)malloc(sizeof(or_sample) * (size_t)(op->max_samples > 0 ? op->max_samples : 1));
    for (int i = 0; i < n; ++i) {
        double o[3], dv[3];
        or_ray_input(cams, n_cams, W, H, pix, rays_o, rays_d, i, o, dv);
        or_ray_out rr;
        or_march(s, oc, op, o, dv, -INFINITY, INFINITY, &rr, sm, NULL);
        for (int a = 0; a < rr.n_samples; ++a) {
            double w = sm[a].T_before * sm[a].alpha;
            long v = (long)or_vox(sm[a].u[0], R) + (long)R * ((long)or_vox(sm[a].u[1], R) +
                                                             (long)R * (long)or_vox(sm[a].u[2], R));
            if (w > w_thr) vis[v] = 1;
            if (wmax && w > wmax[v]) wmax[v] = w;
        }
    }
    free(sm);
}

/* Dilation by a (2r+1)^3 box: out[v] = the largest occ over the voxels within r of
 * v along every axis, the grid's faces clipping the box; with a mask, out[v] is
 * cleared wherever mask[v] is 0. */
void or_dilate(const uint8_t* occ, int R, int r, const uint8_t* mask, uint8_t* out) {
    #pragma omp parallel for schedule(static)
    for (long v = 0; v < (long)R * R * R; ++v) {
        int i = (int)(v % R), j = (int)((v / R) % R), k = (int)(v / ((long)R * R));
        uint8_t m = 0;
        for (int dz = -r; dz <= r; ++dz)
            for (int dy = -r; dy <= r; ++dy)
                for (int dx = -r; dx <= r; ++dx) {
                    int x = i + dx, y = j + dy, z = k + dz;
                    if (x < 0 || y < 0 || z < 0 || x >= R || y >= R || z >= R) continue;
                    uint8_t q = occ[(long)x + (long)R * ((long)y + (long)R * z)];
                    if (q > m) m = q;
                }
        out[v] = (mask && !mask[v]) ? 0 : m;
    }
}

/* ------------------------------------------------ training losses and controls */

/* Huber colour loss (Sec. S2.4): sum of h(e) over n values, h(e) = e^2 / 2 when
 * |e| <= delta, else delta (|e| - delta / 2); d[i] = h'(e_i) (NULL allowed). */
double or_huber_loss(const double* rgb, const double* target, long n, double delta, double* d) {
    double L = 0.0;
    for (long i = 0; i < n; ++i) {
        double e = rgb[i] - target[i];
        if (fabs(e) <= delta) { L += 0.5 * e * e; if (d) d[i] = e; }
        else { L += delta * (fabs(e) - 0.5 * delta); if (d) d[i] = e > 0 ? delta : -delta; }
    }
    return L;
}

/* Step-size auto-tuning (Eq. S3): the next gamma from the batch's mean samples. */
double or_step_autotune(double gamma, double n_mean, double n_min, double kappa, double gamma_min) {
    if (n_mean >= n_min) return fmin(1.0, (1.0 + kappa) * gamma);
    return fmax(gamma_min, (1.0 - kappa) * gamma);
}

/* Distortion regulariser (Eq. S2) of each ray, by its definition: over the
 * composited samples with weights w_i and intervals [t_i, t_i + delta_i],
 * L = sum_{i,j} w_i w_j |m_i - m_j| + 1/3 sum_i w_i^2 delta_i, m_i the midpoints.
 * out[n][4] = (L, sum w, sum w m, 0). */
void or_distortion(const or_scene* s, const or_occ* oc, const or_opts* op,
                   const float* cams, int n_cams, int W, int H, const int32_t* pix,
                   const float* rays_o, const float* rays_d, int n, double* out) {
    #pragma omp parallel
    {
        or_sample* sm = (or_sample*)malloc(sizeof(or_sample) * (size_t)(op->max_samples > 0 ? op->max_samples : 1));
        #pragma omp for schedule(dynamic, 16)
        for (int r = 0; r < n; ++r) {
            double o[3], dv[3];
            or_ray_input(cams, n_cams, W, H, pix, rays_o, rays_d, r, o, dv);
            or_ray_out rr;
            or_march(s, oc, op, o, dv, -INFINITY, INFINITY, &rr, sm, NULL);
            double pair = 0.0, self = 0.0, Ws = 0.0, Ss = 0.0;
            for (int i = 0; i < rr.n_samples; ++i) {
                double wi = sm[i].T_before * sm[i].alpha, mi = sm[i].t + 0.5 * sm[i].delta;
                for (int j = 0; j < rr.n_samples; ++j) {
                    double wj = sm[j].T_before * sm[j].alpha, mj = sm[j].t + 0.5 * sm[j].delta;
                    pair += wi * wj * fabs(mi - mj);
                }
                self += wi * wi * sm[i].delta / 3.0;
                Ws += wi;
                Ss += wi * mi;
            }
            out[4 * r + 0] = pair + self;
            out[4 * r + 1] = Ws;
            out[4 * r + 2] = Ss;
            out[4 * r + 3] = 0.0;
        }
        free(sm);
    }
}

/* Reverse of or_distortion: g_tables / g_coarse += scale * dL/d(parameter) summed
 * over rays.  g_j = dL/dw_j by differentiating the definition; w_j = T_j alpha_j
 * gives dw_j/dsigma_i = delta_i T_{i+1} (j = i), -delta_i w_j (j > i), 0 (j < i);
 * sigma = exp(sigma_raw) with the truncated derivative; then Eq. 6-8 backwards
 * for the density channel only. */
void or_distortion_backward(const or_scene* s, const or_occ* oc, const or_opts* op,
                            const float* cams, int n_cams, int W, int H, const int32_t* pix,
                            const float* rays_o, const float* rays_d, int n, double scale,
                            double* g_tables, double* g_coarse, double* g_attn_inv, double* g_agg_mlp) {
    or_sample* sm = (or_sample*)malloc(sizeof(or_sample) * (size_t)(op->max_samples > 0 ? op->max_samples : 1));
    double* g = (double*)malloc(sizeof(double) * (size_t)(op->max_samples > 0 ? op->max_samples : 1));
    for (int r = 0; r < n; ++r) {
        double o[3], dv[3];
        or_ray_input(cams, n_cams, W, H, pix, rays_o, rays_d, r, o, dv);
        or_ray_out rr;
        or_march(s, oc, op, o, dv, -INFINITY, INFINITY, &rr, sm, NULL);
        int ns = rr.n_samples;
        for (int j = 0; j < ns; ++j) {
            double mj = sm[j].t + 0.5 * sm[j].delta;
            double acc = 0.0;
            for (int k = 0; k < ns; ++k) {
                double mk = sm[k].t + 0.5 * sm[k].delta;
                acc += sm[k].T_before * sm[k].alpha * fabs(mj - mk);
            }
            double wj = sm[j].T_before * sm[j].alpha;
            g[j] = 2.0 * acc + 2.0 / 3.0 * wj * sm[j].delta;
        }
        for (int i = 0; i < ns; ++i) {
            const or_sample* sp = sm + i;
            double T_next = sp->T_before * (1.0 - sp->alpha);
            double d_sigma = sp->delta * T_next * g[i];
            for (int j = i + 1; j < ns; ++j) d_sigma -= sp->delta * sm[j].T_before * sm[j].alpha * g[j];
            /* the regulariser sees the density only: f's cotangent is [dL/d sigma_raw, 0, ...] */
            double g_f[OR_NFEAT] = {scale * d_sigma * exp(fmin(sp->sigma_raw, 15.0)), 0, 0, 0, 0, 0, 0, 0};
            or_feature_reverse(s, op, sp->u, g_f, g_tables, g_coarse, g_attn_inv, g_agg_mlp, NULL);
        }
    }
    free(g);
    free(sm);
}
