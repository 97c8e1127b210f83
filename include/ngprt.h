/*
 * ngprt.h -- C ABI of the GB300 (sm_103a) NGP-RT render path, arXiv 2407.10482.
 *
 * Conventions shared by every entry point:
 *   - Every array argument is caller-owned DEVICE memory (CUDA global memory of the
 *     current device) unless its comment says "host".  The library keeps no pointer
 *     after a call returns and allocates no device memory: scratch comes from the
 *     caller's `workspace` (size from the matching *_workspace_bytes query, 256-byte
 *     aligned).
 *   - Calls are asynchronous on `stream` (a cudaStream_t; NULL = legacy default
 *     stream).  Outputs are valid once the stream reaches the call.
 *   - The return value is an ngprt_status.  Argument errors are reported before
 *     anything is launched and leave every output untouched; NGPRT_ERR_CUDA reports
 *     a launch failure.  ngprt_last_error() returns a message for the calling host
 *     thread's last failure.
 *   - Layouts are row-major with the last index fastest.  Grids are x fastest:
 *     vertex/voxel (x, y, z) of an R-per-axis grid is element x + R*(y + R*z).
 */
#ifndef NGPRT_H
#define NGPRT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    NGPRT_OK = 0,
    NGPRT_ERR_INVALID_ARG = -1, /* bad size, null pointer, misaligned pointer, bad enum */
    NGPRT_ERR_UNSUPPORTED = -2, /* valid request this build does not implement (e.g. an L without a kernel) */
    NGPRT_ERR_CUDA = -3,        /* a CUDA launch or query failed */
    NGPRT_ERR_WORKSPACE = -4,   /* workspace missing or smaller than the query asked for */
    NGPRT_ERR_TIMEOUT = -5      /* a bounded device-side wait expired (reported by ngprt_sync_status) */
} ngprt_status;

typedef enum { NGPRT_F32 = 0, NGPRT_F16 = 1, NGPRT_BF16 = 2 } ngprt_dtype;

#define NGPRT_MAX_LEVELS 32
#define NGPRT_MAX_CAMERAS 64
#define NGPRT_STATE_FLOATS 12 /* per-ray state: C_d(3), F(4), A, depth, d(3) */

/*
 * How the L fine levels fuse into f^ (Eq. 7-8 and the variants of Table 3).  The
 * coarse grid holds f~ (8 channels) and, for the spatially variant forms, the
 * attention logits; the spatially invariant forms take one logit per level (and
 * modality) from attn_inv; gates are sigmoid(logit) in every attention form.
 *   SEPARATE_V  : Eq. 8 as printed: omega^l on sigma^l, beta^l on (c_d^l, v_s^l),
 *                 logits interpolated from the coarse grid (8 + 2L channels)
 *   SHARED_V    : one gate per level on all 8 channels, from the coarse grid (8 + L)
 *   SEPARATE_INV: omega^l, beta^l constant over space (coarse grid 8 channels)
 *   SHARED_INV  : one constant gate per level (coarse grid 8 channels)
 *   SUM         : f^ = sum of the levels (coarse grid 8 channels)
 *   MLP         : f^ = W2 relu(W1 [f^1, ..., f^L]), the tiny-MLP aggregation of
 *                 Instant-NGP (one hidden layer of NGPRT_AGG_MLP_HIDDEN, no biases;
 *                 coarse grid 8 channels)
 */
typedef enum {
    NGPRT_AGG_SEPARATE_V = 0,
    NGPRT_AGG_SHARED_V = 1,
    NGPRT_AGG_SEPARATE_INV = 2,
    NGPRT_AGG_SHARED_INV = 3,
    NGPRT_AGG_SUM = 4,
    NGPRT_AGG_MLP = 5
} ngprt_aggregation;

#define NGPRT_AGG_MLP_HIDDEN 64

/* Sparse coarse grid (the block-indexed storage of the baked 512^3 grid, Sec. 3.1,
 * Eq. S1): cells are grouped in blocks of 8^3; a stored block holds the 9^3 vertices
 * of its cells (neighbouring blocks repeat their shared face), so one index lookup
 * serves all 8 corners of a sample. */
#define NGPRT_COARSE_BLOCK 8
#define NGPRT_COARSE_BLOCK_ROWS 729

/*
 * Render-time scene (Sec. 3.1, Eq. 6): L fine levels of explicit deferred features
 * and a coarse grid holding the coarse feature and the attention logits.
 *   tables : [n_entries][8] of table_dtype; entry = [sigma^, c_d^(3), v_s^(4)].
 *            Level l owns min(N[l]^3, 2^T_log2) consecutive rows, levels in order.
 *            A level with N^3 <= 2^T_log2 is dense (row x + N*y + N^2*z); the others
 *            use the spatial hash (x*1 ^ y*2654435761 ^ z*805459861) mod 2^T_log2.
 *            32-byte aligned (F32) or 16-byte aligned (F16/BF16).
 *   coarse : [R_C^3][ngprt_coarse_channels(L, aggregation)] of table_dtype,
 *            channels [sigma~, c_d~(3), v_s~(4)] then, for SEPARATE_V, the logits
 *            omega^1, beta^1, ..., omega^L, beta^L (Eq. 7), for SHARED_V one logit
 *            per level a^1, ..., a^L.  Aligned like tables (32 bytes F32, 16 bytes
 *            F16/BF16).
 *   mlp_w  : deferred MLP_psi (Eq. 5) of mlp_layers dense layers without bias:
 *            layer k is a [out_k][in_k] matrix, in_0 = 32 (C_d, F, SH16(d), zero
 *            padding), out_k = mlp_width for hidden layers (ReLU), 3 for the last.
 *            mlp_dtype F32 (float; CUDA-core FMA) or F16 (__half; tcgen05 tensor-core
 *            MMA with FP32 accumulation, activations rounded to FP16 between layers).
 *   bounded: 1 = scene in the box [-1,1]^3; 0 = unbounded scene under the
 *            mip-NeRF-360 contraction into [-2,2]^3.
 *   aggregation: ngprt_aggregation (0 = Eq. 8).
 *   attn_inv: device FP32 logits of the invariant forms: SEPARATE_INV [L][2]
 *            (omega^l, beta^l), SHARED_INV [L]; NULL otherwise.
 *   agg_mlp: device FP32 weights of the MLP form, W1 [64][8L] then W2 [8][64]
 *            ([out][in] row-major; input = level 1's 8 channels, then level 2's, ...),
 *            16-byte aligned; NULL otherwise.
 *   coarse_index: NULL = coarse is the dense [R_C^3] grid above.  Else coarse is
 *            sparse: [coarse_blocks][NGPRT_COARSE_BLOCK_ROWS][channels], block s
 *            row i + 9 j + 81 k = vertex (8 bx + i, 8 by + j, 8 bz + k) of the block
 *            (bx, by, bz) whose index entry is s, and coarse_index is int32
 *            [NB^3] (NB = ceil((R_C - 1) / 8), entry bx + NB (by + NB bz)).  Slot 0
 *            conventionally holds zeros and serves the empty blocks.  Slots outside
 *            [0, coarse_blocks) are clamped into it.  Render paths only
 *            (ngprt_render, the occupancy builders); the reverse passes need the
 *            dense grid.  Built by ngprt_coarse_block_mask + ngprt_coarse_sparsify.
 *   coarse_blocks: stored blocks (>= 1) when coarse_index != NULL.
 * Vertex grids of N per axis cover the unit cube coordinate u in [0,1]^3 with
 * p = u (N - 1) (trilinear interpolation, Eq. 6).
 */
typedef struct {
    int32_t L;
    int32_t T_log2;
    int32_t N[NGPRT_MAX_LEVELS];
    int32_t table_dtype;
    int32_t R_C;
    int32_t mlp_layers;
    int32_t mlp_width;
    int32_t mlp_dtype;
    int32_t bounded;
    const void* tables;
    const void* coarse;
    const void* mlp_w;
    int32_t aggregation;
    const float* attn_inv;
    const float* agg_mlp;
    const int32_t* coarse_index;
    int64_t coarse_blocks;
} ngprt_scene;

/* Channels per coarse-grid vertex for L levels under `aggregation` (0 if invalid). */
int32_t ngprt_coarse_channels(int32_t L, int32_t aggregation);


/*
 * Occupancy (Sec. 3.3; Sec. S2.5).  bits: n_levels bit-packed grids, finest
 * (R_O^3 bits) first, each next level halving the resolution, each level padded
 * to whole 32-bit words (bit i of a level is word i/32, bit i%32).  dist: the
 * R_G^3 uint8 occupancy distance grid G, or NULL to march without it; R_G is the
 * resolution of one pyramid level, R_O >> k (0 means R_O; the paper's renders keep
 * G at 256^3 beside a 512^3 finest level), and G is read at an empty point only
 * when the empty level is coarser than R_G (Sec. 3.3).
 */
typedef struct {
    int32_t R_O;
    int32_t n_levels;
    const uint32_t* bits;
    const uint8_t* dist;
    int32_t R_G;
} ngprt_occ;

/*
 * Coarse blocks a render can read: block_mask (uint8 [NB^3], NB = ceil((R_C - 1) / 8),
 * written 0/1 in full) marks every block holding a cell that an occupied voxel of
 * the finest occupancy level (occ->bits, R_O^3) overlaps, widened by one cell on
 * each side.  Voxel x covers u in [x / R_O, (x + 1) / R_O] and so the coarse cells
 * floor(x (R_C - 1) / R_O) - 1 ... floor((x + 1) (R_C - 1) / R_O) + 1 (clamped to
 * [0, R_C - 2]) per axis: samples are only taken in occupied voxels, so a sparse
 * grid of the marked blocks renders exactly like the dense grid.  occ->dist unused.
 */
int32_t ngprt_coarse_block_mask(const ngprt_occ* occ, int32_t R_C, uint8_t* block_mask, void* stream);

/*
 * Sparse coarse grid from a dense one.  block_mask: device uint8 [NB^3] (e.g. from
 * ngprt_coarse_block_mask).  Writes the device index (int32 [NB^3]: marked blocks
 * numbered 1, 2, ... in index order, unmarked ones 0) and the host count
 * *n_blocks = 1 + marked blocks (slot 0 = zeros).  With blocks != NULL (device,
 * room for max_blocks blocks of NGPRT_COARSE_BLOCK_ROWS rows of row_bytes) the
 * blocks are filled from dense ([R_C^3] rows of row_bytes = channels x element
 * size, a multiple of 4; vertices past R_C - 1 are zero).  NULL blocks only counts.
 * Synchronises `stream` (the count comes back to the host).  workspace: device,
 * ngprt_coarse_sparsify_workspace_bytes(R_C) bytes, 16-byte aligned.
 */
size_t ngprt_coarse_sparsify_workspace_bytes(int32_t R_C);
int32_t ngprt_coarse_sparsify(const void* dense, int32_t R_C, int32_t row_bytes, const uint8_t* block_mask,
                              int32_t* index, void* blocks, int64_t max_blocks, int64_t* n_blocks, void* workspace,
                              size_t ws_bytes, void* stream);

/* Pinhole camera, OpenCV axes (x right, y down, z forward).  c2w: 3x4 row-major
 * camera-to-world.  Pixel (col, row) looks through (col + 0.5, row + 0.5). */
typedef struct {
    float c2w[12];
    float fx, fy, cx, cy;
    int32_t W, H;
} ngprt_camera;

/* Per-call knobs.  step_base = s_0 and step_gamma = gamma of the step s = gamma s_0
 * (Sec. S2.3); t_min = near distance; r_far = world radius of the unbounded domain;
 * t_term = transmittance threshold (2e-3 in Sec. S2.5); bg = background colour;
 * max_march / max_samples = caps on marching points / samples per ray;
 * use_dist = read G (Eq. 9); lattice_snap = (bounded only) keep samples on the
 * uniform lattice; attn_mode (SEPARATE_V scenes only; 0 for every other
 * aggregation) 0 = separate attention (Eq. 8), 1 = gates fixed at 1 (SUM over the
 * same grid), 2 = omega^l for both modalities; dist_rule 1 = max(v G, s_O) (the
 * longer of two safe steps; the rule the bindings default to), 0 = Eq. 9 as
 * printed (v G whenever G > 0). */
typedef struct {
    float step_base;
    float step_gamma;
    float t_min;
    float r_far;
    float t_term;
    float bg[3];
    int32_t max_march;
    int32_t max_samples;
    int32_t use_dist;
    int32_t lattice_snap;
    int32_t attn_mode;
    int32_t dist_rule;
} ngprt_render_opts;

/* Number of uint32 words of an occupancy pyramid (see ngprt_occ). */
size_t ngprt_occ_bits_words(int32_t R, int32_t n_levels);

/* Workspace bytes ngprt_build_occ_dist needs for an R^3 grid. */
size_t ngprt_build_occ_dist_workspace_bytes(int32_t R);

/*
 * Occupancy pyramid and occupancy distance grid G (Sec. 3.3: per voxel, the
 * distance to the nearest occupied voxel, rounded down, in voxel units, uint8;
 * Sec. S2.5: the grid down-sampled to coarser levels).
 *   occ          : [R^3] uint8, nonzero = occupied.  R a power of two, 2..1024.
 *   n_levels     : pyramid levels, 1 <= n_levels and R >> (n_levels-1) >= 1.
 *   dist_level   : G is built on pyramid level dist_level (R_G = R >> dist_level,
 *                  0 <= dist_level < n_levels): a voxel of that level is occupied when
 *                  any of its finest voxels is.
 *   occ_bits_out : [ngprt_occ_bits_words(R, n_levels)] uint32, written in full.
 *   dist_out     : [R_G^3] uint8 G, or NULL to skip it.  G = min(255, floor(D)), D the
 *                  Euclidean distance between the voxel boxes in voxels of R_G; 0 on and
 *                  next to occupied voxels; 255 everywhere if nothing is occupied.
 *   workspace    : >= ngprt_build_occ_dist_workspace_bytes(R) bytes.
 */
int32_t ngprt_build_occ_dist(const uint8_t* occ, int32_t R, int32_t n_levels, int32_t dist_level,
                             uint32_t* occ_bits_out, uint8_t* dist_out, void* workspace, size_t ws_bytes,
                             void* stream);

/*
 * Render-time occupancy pipeline (Sec. S2.5: occupancy from the trained model,
 * visibility culling and dilation as in MERF, then the pyramid and G above).
 * Grids are R^3 uint8 over the unit cube of the scene (x fastest), R a power of two
 * in [2, 1024].  The three calls are asynchronous on `stream` and need the Eq. 8
 * aggregation (SEPARATE_V).
 *
 * ngprt_occupancy_from_density: occ_out[v] = 1 when sigma = exp(sigma_raw) at the
 *   centre u = (v + 1/2) / R of voxel v exceeds sigma_thr (features of Eq. 6-8 with
 *   opts->attn_mode), else 0; sigma_out [R^3] (NULL allowed) receives sigma.
 */
int32_t ngprt_occupancy_from_density(const ngprt_scene* scene, const ngprt_render_opts* opts, int32_t R,
                                     float sigma_thr, uint8_t* occ_out, float* sigma_out, void* stream);

/*
 * ngprt_occupancy_visibility: marches and composites the given rays as ngprt_render
 *   does (occ, opts) and sets vis[v] = 1 for the voxel v (R^3 grid, voxel of the
 *   unit-cube position) of every sample whose weight T_i alpha_i exceeds w_thr.
 *   vis is only ever set: the caller clears it, and calls over several ray batches
 *   accumulate.  Rays as for ngprt_render.
 */
int32_t ngprt_occupancy_visibility(const ngprt_scene* scene, const ngprt_occ* occ, const ngprt_camera* cams,
                                   int32_t n_cams, const int32_t* pixel_ids, const float* rays_o,
                                   const float* rays_d, int64_t n_rays, const ngprt_render_opts* opts, float w_thr,
                                   int32_t R, uint8_t* vis, void* stream);

/*
 * ngprt_dilate: out[v] = max of occ over the voxels within `radius` of v along
 *   every axis (a (2 radius + 1)^3 box clipped by the grid's faces), then 0 wherever
 *   mask[v] == 0 (mask NULL: no mask; e.g. the density occupancy, so that the render
 *   grid stays inside it).  R in [1, 1024], radius in [0, 64]; out distinct from occ
 *   and mask; workspace >= ngprt_dilate_workspace_bytes(R).
 */
size_t ngprt_dilate_workspace_bytes(int32_t R);
int32_t ngprt_dilate(const uint8_t* occ, int32_t R, int32_t radius, const uint8_t* mask, uint8_t* out,
                     void* workspace, size_t ws_bytes, void* stream);

/* Rows of the concatenated fine tables (sum over levels of min(N^3, 2^T_log2)). */
int64_t ngprt_table_entries(const ngprt_scene* scene);

/* Workspace bytes of ngprt_render / ngprt_render_backward for n_rays rays. */
size_t ngprt_render_workspace_bytes(const ngprt_scene* scene, int64_t n_rays);

/*
 * Render rays (Eq. 2, 5, 6, 8, 9): occupancy-distance marching, per-sample coarse
 * fetch + per-level gathers + lightweight attention, alpha compositing, one
 * deferred MLP per ray, colour over the background.
 * Rays: with cams != NULL (host array of n_cams <= 64 cameras sharing W, H) ray i
 * is pixel pixel_ids[i] (or i if pixel_ids == NULL) of the multi-view image,
 * id = view*W*H + row*W + col; else ray i is (rays_o[i], rays_d[i]) (float [n][3],
 * d need not be unit: it is normalised).  n_rays >= 0 (0 launches nothing).
 *   t_interval : NULL or float [n][2] (t_near, t_far): march only inside it.
 *   rgb [n][3], depth [n], opacity [n] : float outputs (NULL allowed for depth/opacity).
 *                If rgb is NULL only the march kernel runs: ray_state is then required
 *                and ngprt_shade turns it into colours.
 *   ray_stats  : NULL or int32 [n][2] = (marching points, samples).
 *   ray_state  : NULL or float [n][NGPRT_STATE_FLOATS], the per-ray composite state
 *                ngprt_render_backward consumes.
 *   workspace  : 256-byte aligned, at least ngprt_render_workspace_bytes(n) bytes
 *                (the per-ray state when ray_state is NULL); NULL allowed with
 *                ray_state.  One fused march kernel runs either way.  The 8 bytes
 *                after the state's rounded size (ngprt_render_workspace_bytes(n) -
 *                256) hold a counter from which the kernel's warps take image tiles
 *                (runs of 32 rays for pixel_ids or explicit rays) at run time, zeroed
 *                on `stream` before the launch.  Without a workspace of that size,
 *                each warp renders the tile of its own index.  The counter makes
 *                concurrent calls that share one workspace race, as the state
 *                already does.
 */
int32_t ngprt_render(const ngprt_scene* scene, const ngprt_occ* occ, const ngprt_camera* cams, int32_t n_cams,
                     const int32_t* pixel_ids, const float* rays_o, const float* rays_d, int64_t n_rays,
                     const float* t_interval, const ngprt_render_opts* opts, float* rgb, float* depth,
                     float* opacity, int32_t* ray_stats, float* ray_state, void* workspace, size_t ws_bytes,
                     void* stream);

/*
 * Deferred shading of marched rays (Eq. 5 and the colour sigmoid of Sec. S2.1):
 * rgb = A sigmoid(C_d + MLP_psi(C_d, F, SH16(d))) + (1 - A) bg from ray_state
 * ([n][NGPRT_STATE_FLOATS], written by ngprt_render); depth and opacity (NULL
 * allowed) are copied out of the state.  Only scene->mlp_* fields are read.
 */
int32_t ngprt_shade(const ngprt_scene* scene, const float* ray_state, int64_t n_rays, const float bg[3],
                    float* rgb, float* depth, float* opacity, void* stream);

/*
 * Reverse pass of ngprt_render (F32 tables and F32 MLP): given dL/d rgb, depth,
 * opacity of the same rays (same cams/pixel_ids or rays, same opts, and the
 * ray_state a forward call wrote), ACCUMULATE (+=) dL/d tables into g_tables
 * ([n_entries][8] float), dL/d coarse into g_coarse ([R_C^3][ngprt_coarse_channels]
 * float), dL/d mlp_w into g_mlp (float, mlp_w's layout) and, for the spatially
 * invariant gate forms (SEPARATE_INV, SHARED_INV), dL/d attn_inv into g_attn_inv
 * (float, attn_inv's layout; ignored, and may be NULL, for the other forms) and, for
 * the MLP form, dL/d agg_mlp into g_agg_mlp (float, agg_mlp's layout; ignored, and
 * may be NULL, otherwise).
 * Aggregations: SEPARATE_V (Eq. 8, any attn_mode; L = 1, 2, 3, 4, 8, 16), and SHARED_V,
 * SEPARATE_INV, SHARED_INV, SUM and MLP (Table 3; L = 2, 4, 16).  Each ray is marched
 * again; the sample set is the forward's.  Table, grid, logit and weight gradients
 * are atomic adds, so their float summation order varies from run to run.
 *   d_rgb [n][3]; d_depth, d_opacity [n] or NULL (zero).
 *   workspace: ngprt_render_backward_workspace_bytes(scene, opts, n_rays) bytes,
 *              16-byte aligned (the MLP form keeps one (f^1..f^L, g_f) record per
 *              sample there: n_rays x opts->max_samples x (8L + 8) floats).
 */
size_t ngprt_render_backward_workspace_bytes(const ngprt_scene* scene, const ngprt_render_opts* opts,
                                             int64_t n_rays);
int32_t ngprt_render_backward(const ngprt_scene* scene, const ngprt_occ* occ, const ngprt_camera* cams,
                              int32_t n_cams, const int32_t* pixel_ids, const float* rays_o,
                              const float* rays_d, int64_t n_rays, const ngprt_render_opts* opts,
                              const float* ray_state, const float* d_rgb, const float* d_depth,
                              const float* d_opacity, float* g_tables, float* g_coarse, float* g_mlp,
                              float* g_attn_inv, float* g_agg_mlp, void* workspace, size_t ws_bytes,
                              void* stream);

/* ------------------------------------------------------------------------------
 * Learned proposal (not in the paper, which leaves adaptive sampling aside in
 * Sec. 2): a 6 -> 32 -> 32 -> 3 MLP on (o / in_scale, d / |d|) predicting the interval
 * [t_near, t_far] that holds a ray's significant weights and its opacity A^:
 *   h1 = relu(W0 e + b0), h2 = relu(W1 h1 + b1), z = W2 h2 + b2,
 *   t_near = t_scale sigmoid(z0), t_far = t_scale sigmoid(z1), A^ = sigmoid(z2).
 * prop_w: float [ngprt_proposal_param_count()] = W0 [32][6], b0 [32], W1 [32][32],
 * b1 [32], W2 [3][32], b2 [3].  Rays are given as for ngprt_render.
 * ------------------------------------------------------------------------------ */
int32_t ngprt_proposal_param_count(void);

/* Interval per ray, t_interval_out [n][2] = (t_near - margin_near, t_far + margin_far)
 * from prop_w in prop_dtype (F32, or F16 copies of the FP32 master widened to FP32 in
 * shared memory; the per-ray arithmetic is FP32)
 * (margin_far = +inf: no far clip, early termination ends the ray); a ray with
 * A^ < a_min gets an empty interval (+inf, -inf) (nothing is marched), a ray with
 * t_far <= t_near gets (-inf, +inf) (the whole ray).  a_hat_out [n] (NULL allowed). */
int32_t ngprt_propose(const void* prop_w, int32_t prop_dtype, const ngprt_camera* cams, int32_t n_cams,
                      const int32_t* pixel_ids,
                      const float* rays_o, const float* rays_d, int64_t n_rays, float in_scale, float t_scale,
                      float margin_near, float margin_far, float a_min, float* t_interval_out, float* a_hat_out,
                      void* stream);

/* Training loss of the proposal against targets [n][3] = (t_near*, t_far*, A*):
 * mean over rays of A* (a_n sl1(dt_near / t_scale) + a_f sl1(dt_far / t_scale)) +
 * (A^ - A*)^2, sl1 = smooth L1 with beta 0.01, a_n = 4 if t_near is later than its
 * target else 1, a_f = 4 if t_far is earlier than its target else 1.  ACCUMULATES the gradient into g_prop_w and the loss
 * into *loss (one device float, NULL to skip). */
int32_t ngprt_propose_backward(const float* prop_w, const ngprt_camera* cams, int32_t n_cams,
                               const int32_t* pixel_ids, const float* rays_o, const float* rays_d, int64_t n_rays,
                               float in_scale, float t_scale, const float* targets, float* g_prop_w, float* loss,
                               void* stream);

/* Proposal targets from a plain render of the same rays (ray_state from ngprt_render
 * without t_interval): targets [n][3] = t of the first sample whose cumulative weight
 * exceeds 0.005 A, t + delta of the first sample whose cumulative weight reaches
 * 0.995 A, and A (0, 0, 0 for rays without samples).  Eq. 8 scenes only
 * (NGPRT_ERR_UNSUPPORTED for the other aggregation forms). */
int32_t ngprt_proposal_targets(const ngprt_scene* scene, const ngprt_occ* occ, const ngprt_camera* cams,
                               int32_t n_cams, const int32_t* pixel_ids, const float* rays_o, const float* rays_d,
                               int64_t n_rays, const ngprt_render_opts* opts, const float* ray_state, float* targets,
                               void* stream);

/* Fallback pass after a render with t_interval: every ray whose interval was not the
 * whole ray and whose composited opacity A (ray_state) fell short of the prediction,
 * a_hat - A > threshold, is marched again over its whole domain and its ray_state
 * overwritten; ray_stats (NULL allowed) then adds the second march's counts.  Then
 * ngprt_shade gives the colours. */
int32_t ngprt_render_fallback(const ngprt_scene* scene, const ngprt_occ* occ, const ngprt_camera* cams,
                              int32_t n_cams, const int32_t* pixel_ids, const float* rays_o, const float* rays_d,
                              int64_t n_rays, const float* t_interval, const float* a_hat, float threshold,
                              const ngprt_render_opts* opts, float* ray_state, int32_t* ray_stats, void* stream);

/*
 * Photometric L2 loss of a training step: *loss += scale * sum_i (rgb_i - target_i)^2
 * (loss: one device float, NULL to skip) and d_rgb = 2 scale (rgb - target) (NULL to
 * skip), over n floats.
 */
int32_t ngprt_l2_loss(const float* rgb, const float* target, int64_t n, float scale, float* loss, float* d_rgb,
                      void* stream);

/*
 * Huber colour loss of the training objective (Sec. S2.4, L_color): per float
 * h(e) = e^2 / 2 for |e| <= delta, else delta (|e| - delta / 2), e = rgb - target;
 * *loss += scale * sum_i h(e_i) (NULL to skip) and d_rgb = scale * h'(e) (NULL to
 * skip), h'(e) = e or delta sign(e).  delta > 0.
 */
int32_t ngprt_huber_loss(const float* rgb, const float* target, int64_t n, float delta, float scale, float* loss,
                         float* d_rgb, void* stream);

/*
 * Distortion regulariser of the training objective (Eq. S2), per ray over the
 * samples the render composites (same march, same weights):
 *   L_dist = sum_{i,j} w_i w_j |m_i - m_j| + 1/3 sum_i w_i^2 delta_i,
 * m_i = t_i + delta_i / 2.  ngprt_distortion_loss writes dist_state [n][4] =
 * (L_dist, sum_i w_i, sum_i w_i m_i, 0) per ray (16-byte aligned) and adds
 * scale * sum over rays of L_dist to *loss (NULL to skip).
 * ngprt_distortion_backward ACCUMULATES scale * dL_dist/d(parameters) into g_tables
 * and g_coarse (FP32, layouts of the scene) from that dist_state: the density path
 * only (sigma~, the density logits and the fine density channel; for the tiny-MLP
 * form every channel it mixes), and for SEPARATE_INV / SHARED_INV into g_attn_inv,
 * for the MLP form into g_agg_mlp (NULL otherwise).  Both need F32 tables; L in
 * {1, 2, 3, 4, 8, 16} for Eq. 8, {2, 4, 16} for the other forms; rays as for
 * ngprt_render.  workspace: ngprt_distortion_backward_workspace_bytes(scene, opts,
 * n_rays) bytes, 16-byte aligned (0, and NULL allowed, except for the MLP form, which
 * keeps one record per sample there).
 */
size_t ngprt_distortion_backward_workspace_bytes(const ngprt_scene* scene, const ngprt_render_opts* opts,
                                                 int64_t n_rays);
int32_t ngprt_distortion_loss(const ngprt_scene* scene, const ngprt_occ* occ, const ngprt_camera* cams,
                              int32_t n_cams, const int32_t* pixel_ids, const float* rays_o, const float* rays_d,
                              int64_t n_rays, const ngprt_render_opts* opts, float scale, float* dist_state,
                              float* loss, void* stream);
int32_t ngprt_distortion_backward(const ngprt_scene* scene, const ngprt_occ* occ, const ngprt_camera* cams,
                                  int32_t n_cams, const int32_t* pixel_ids, const float* rays_o, const float* rays_d,
                                  int64_t n_rays, const ngprt_render_opts* opts, const float* dist_state, float scale,
                                  float* g_tables, float* g_coarse, float* g_attn_inv, float* g_agg_mlp,
                                  void* workspace, size_t ws_bytes, void* stream);

/*
 * Step-size auto-tuning of training (Eq. S3).  ngprt_mean_samples writes to the
 * device float *out the mean of the per-ray sample counts of ray_stats [n][2] (the
 * second int of each pair).  ngprt_step_autotune (host, no device work) returns the
 * next scaler gamma of the step s = gamma s_0: min(1, (1 + kappa) gamma) when
 * n_mean >= n_min, else max(gamma_min, (1 - kappa) gamma).
 */
int32_t ngprt_mean_samples(const int32_t* ray_stats, int64_t n_rays, float* out, void* stream);
float ngprt_step_autotune(float gamma, float n_mean, float n_min, float kappa, float gamma_min);

/*
 * One Adam step over n floats (the optimiser of Sec. S2.4): m = b1 m + (1-b1) g,
 * v = b2 v + (1-b2) g^2, param -= lr (m/(1-b1^step)) / (sqrt(v/(1-b2^step)) + eps);
 * step >= 1 counts from 1; zero_grad != 0 also clears grad.  All four arrays 16-byte
 * aligned.
 */
int32_t ngprt_adam_step(float* param, float* grad, float* m, float* v, int64_t n, float lr, float beta1, float beta2,
                        float eps, int32_t step, int32_t zero_grad, void* stream);

/* ------------------------------------------------------------------------------
 * Render without any caller-provided scratch.  The paper has no counterpart: this
 * is for callers that cannot allocate device memory (a plug-in inside a host
 * application that owns the device allocator, code that must not allocate in a
 * latency-critical loop, a fixed memory budget set at load time).  It computes
 * exactly what ngprt_render computes, with the per-ray state kept in a static device
 * array of NGPRT_NOALLOC_MAX_RAYS * NGPRT_STATE_FLOATS floats (12 MiB) that every
 * GPU loading this library holds until the process exits.
 *   - It allocates nothing (no cudaMalloc, cudaFree or allocating library call).
 *   - n_rays > NGPRT_NOALLOC_MAX_RAYS is rejected with NGPRT_ERR_INVALID_ARG: render
 *     larger batches in chunks.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call before
 *     any stream capture.  The address is kept for the life of the process: it
 *     assumes the device's context is never reset.  After cudaDeviceReset (or a
 *     primary context released and created again) the kept address is stale, so do
 *     not call this entry point on that device again in the same process.
 *   - Every call on a device shares the one array, which keeps the last call's
 *     contents (each call overwrites the state of the rays it renders before reading
 *     it).  Calls that overlap on the GPU (other streams, other host threads) race
 *     on it: serialise them.
 * Arguments are those of ngprt_render without ray_state and workspace.
 * ------------------------------------------------------------------------------ */
#define NGPRT_NOALLOC_MAX_RAYS 262144

int64_t ngprt_render_noalloc_max_rays(void);

int32_t ngprt_render_noalloc(const ngprt_scene* scene, const ngprt_occ* occ, const ngprt_camera* cams, int32_t n_cams,
                             const int32_t* pixel_ids, const float* rays_o, const float* rays_d, int64_t n_rays,
                             const float* t_interval, const ngprt_render_opts* opts, float* rgb, float* depth,
                             float* opacity, int32_t* ray_stats, void* stream);

/*
 * Test hook for the per-level indexing (Eq. 3, Eq. 6): for n positions u (float
 * [n][3] in the unit cube) write the absolute table row of each of the 8 corners
 * of each fine level, uint32 [n][L][8], corner c = +x if bit0, +y if bit1, +z if bit2.
 */
int32_t ngprt_grid_indices(const ngprt_scene* scene, const float* u, int64_t n, uint32_t* idx_out,
                           void* stream);

/* Waits for `stream` and reports what went wrong on the device since the last
 * report: NGPRT_ERR_CUDA (with the CUDA message) if the stream holds a failed
 * launch, NGPRT_ERR_TIMEOUT if a tensor-core MLP kernel gave up waiting for its MMAs
 * (its rays were left unshaded; the flag is cleared by this report), else NGPRT_OK.
 * After an expired wait the kernel waits once more, again bounded, for the MMA in
 * flight before releasing its tensor memory; if that MMA never completes it keeps
 * the memory, and the message says so: the context is then suspect and the
 * tensor-core forms should not be used in it again. */
int32_t ngprt_sync_status(void* stream);

/* Test hook of the timeout path (no counterpart in the paper): one block waits, with
 * at most `limit` polls (1..2^20), on an mbarrier nothing arrives at, the same
 * bounded wait the tensor-core MLP uses; it gives up, sets the flag and exits, so the
 * next ngprt_sync_status returns NGPRT_ERR_TIMEOUT.  Nothing faults or stays
 * running. */
int32_t ngprt_test_bounded_wait(int32_t limit, void* stream);

/* Writes to the device int *count the number of NaN or infinite values among x[0..n)
 * (a check after fault injection: a NaN in the tables makes the affected rays' colour
 * NaN; the march still ends at its caps). */
int32_t ngprt_count_nonfinite(const float* x, int64_t n, int32_t* count, void* stream);

/* 1 if a tensor-core MLP kernel (mlp_dtype F16) ever gave up waiting for its MMAs
 * (it then frees its tensor memory and leaves its rays unwritten), 0 if not, -1 if
 * the flag cannot be read.  Synchronises with the device. */
int32_t ngprt_tensor_core_error(void);

/* Message of the calling thread's last failed call ("" if none). */
const char* ngprt_last_error(void);

/* ABI version of this header (major*100 + minor); ngprt_version() returns the
 * library's, so a caller can refuse a library built from another header. */
#define NGPRT_ABI_VERSION 201
int32_t ngprt_version(void);

#ifdef __cplusplus
}
#endif

#endif /* NGPRT_H */
