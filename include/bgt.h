/*
 * bgt.h -- C ABI of the GB300 BG-Triangle differentiable rasterizer.
 *
 * Renders Bezier Gaussian Triangles (Wu et al., "BG-Triangle: Bezier Gaussian
 * Triangle for 3D Vectorization and Rendering", CVPR 2025) into images and
 * back-propagates image gradients to their parameters. The forward pass is
 * the pipeline of Sec. 3.2 / Fig. 2: tessellation + rasterization with a
 * depth test (I_id, I_uv, boundary set B), sub-primitive generation (Eq. 3-5)
 * and discontinuity-aware alpha blending (Eq. 6-8). The backward pass follows
 * the supplementary "Backward Derivative" with the rasterizer outputs held
 * fixed, as the paper does.
 *
 * Conventions
 *   - All pointers inside bgt_scene, bgt_grads and every image buffer are
 *     DEVICE pointers owned by the caller. Cameras are HOST memory.
 *   - Streams are passed as `void *` holding a cudaStream_t (NULL = default).
 *     All work is asynchronous on that stream; one handle must not be used
 *     from two streams at once.
 *   - Images of a call with n views are packed back to back in view order;
 *     view v occupies pixels [off_v, off_v + W_v H_v), row-major, 3 floats
 *     (R, G, B) per pixel, off_v = sum of the earlier views' W H.
 *   - Control points of primitive g are ctrl[g][idx][3] with idx running over
 *     (i, j, k), i + j + k = n, in the order i = n..0, then j = n-i..0; the
 *     corner p_n00 is barycentric u = 1, p_0n0 is v = 1, p_00n is w = 1.
 *   - Errors are returned, never trapped. Errors detected on the device
 *     (capacity overflow, non-finite values) set a status word that
 *     bgt_sync_status() reports; outputs of such a call are unspecified.
 *
 * The library allocates its whole workspace in bgt_create() from the
 * capacities in bgt_config and never allocates afterwards, so a sequence of
 * calls can be captured in a CUDA graph.
 */
#ifndef BGT_H
#define BGT_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  BGT_OK = 0,
  BGT_ERR_INVALID_ARG = 1, /* bad pointer, size or configuration */
  BGT_ERR_CAPACITY = 2,    /* a call or a device-side count exceeded a capacity */
  BGT_ERR_CUDA = 3,        /* a CUDA runtime call failed; see bgt_last_error */
  BGT_ERR_TIMEOUT = 4,     /* reserved: a bounded device wait gave up */
  BGT_ERR_NONFINITE = 5,   /* non-finite projected Gaussian detected */
  BGT_ERR_STATE = 6        /* backward called without a matching forward */
} bgt_status;

typedef struct bgt_handle bgt_handle;

/* Flags of bgt_config.flags */
#define BGT_FLAG_NO_BOUNDARY 1 /* w = 1 everywhere: the paper's "w/o B" ablation (Table 3) */
#define BGT_FLAG_GRAPH 2       /* capture forward and backward in CUDA graphs, replay when shapes repeat */

typedef struct {
  int degree;                   /* n of the Bezier triangles, 1..4 (paper: 2) */
  int max_prims;                /* capacity: primitives per scene */
  int max_views;                /* capacity: views per call (<= 4096) */
  long long max_pixels;         /* capacity: sum of W*H over the views of one call (<= 2^27) */
  long long max_pairs;          /* capacity: (Gaussian, tile) pairs per call */
  long long max_boundary_pairs; /* capacity: (boundary point, tile) pairs per call */
  long long max_blend_pairs;    /* capacity: (pixel, Gaussian) pairs the forward pass composites
                                   per call, recorded for the backward pass: headers get 3/4,
                                   fill records 1/64 of it; 0 = 8 per pixel, at least 2^22.
                                   Warp blocks whose records do not fit are differentiated by
                                   re-walking their tile lists (bgt_get_counts out[7]): not an
                                   error, only slower */
  int tess_level;               /* L: each primitive becomes L^2 flat triangles (1..16) */
  int tile_size;                /* screen tile edge: 8, 16 or 32 pixels */
  float k_b;                    /* boundary radius sigma = k_b fx r_b / z (Sec. 3.2) */
  float alpha_min;              /* pairs with alpha below are skipped (1/255) */
  float alpha_max;              /* alpha = min(alpha_max, o w G) (0.99) */
  float t_stop;                 /* blending stops before T would fall below (1e-4) */
  float dilation;               /* added to the diagonal of every 2D covariance, px^2 (0.3) */
  float near_z;                 /* flat triangles with a vertex nearer than this are culled */
  int flags;                    /* BGT_FLAG_* */
} bgt_config;

typedef struct {
  float R[9];           /* world -> camera rotation, row-major; camera x right, y down, z forward */
  float t[3];           /* world -> camera translation */
  float fx, fy, cx, cy; /* pinhole intrinsics in pixels; pixel (x, y) has its centre at (x, y) */
  int width, height;
} bgt_camera;

typedef struct {
  const float *ctrl;      /* [M][Ncp][3] control points p_ijk (Eq. 1), Ncp = (n+1)(n+2)/2 */
  const float *color;     /* [M][Ncp][3] colour control points p^c_ijk (Eq. 4) */
  const float *opacity;   /* [M] opacity o (Eq. 8) */
  const float *r_b;       /* [M] boundary scale r_b (Sec. 3.2) */
  const float *log_scale; /* [M][T][3] scaling attribute maps: log scales of the sub-primitive
                             Gaussians (Sec. 3.2, Eq. 5), T = R (R + 1) / 2 texels */
  const float *quat;      /* [M][T][4] rotation attribute maps, (w, x, y, z), normalised after
                             interpolation */
  int num_prims;          /* M */
  float bg[3];            /* background colour c_bg */
  int attr_res;           /* R, leg resolution of the attribute maps (1..16; 0 counts as 1).
                             Texel (i, j), i + j <= R - 1, sits at (u, v) = (i, j) / (R - 1),
                             stored in the control-point order (i = R-1..0, then
                             j = R-1-i..0); Theta interpolates linearly on the lattice
                             triangle holding I_uv (R = 1: one texel per primitive) */
  const float *sh;        /* [M][K][3] view-dependent colour: coefficients of the real spherical
                             harmonics of bands 1..D per primitive and RGB channel, K = (D+1)^2 - 1,
                             added to the diffuse colour at the direction from the camera centre
                             to S_q (Sec. 3.2, "SH coefficients"); NULL when D = 0 */
  int sh_degree;          /* D = 0..3 */
} bgt_scene;

typedef struct {
  float *ctrl;    /* [M][Ncp][3] dl/dp_ijk */
  float *color;   /* [M][Ncp][3] dl/dp^c_ijk */
  float *opacity; /* [M] dl/do */
  float *r_b;     /* [M] dl/dr_b */
  float *log_scale; /* [M][T][3] dl/d scaling map texels, or NULL (not computed) */
  float *quat;      /* [M][T][4] dl/d rotation map texels (raw quaternion), or NULL */
  float *sh;        /* [M][K][3] dl/d SH coefficients, or NULL (not computed) */
} bgt_grads;

/* Fill *cfg with the defaults named above (n = 2, L = 8, tile 16, 1/255, 0.99,
 * 1e-4, 0.3, k_b = 3, near 0.2) and capacities for one 1024x1024 view of
 * 100k primitives. Returns BGT_ERR_INVALID_ARG if cfg is NULL. */
bgt_status bgt_default_config(bgt_config *cfg);

/* Create a handle on the current CUDA device and allocate its workspace from
 * the capacities in *cfg. On success *out owns the workspace until
 * bgt_destroy. BGT_ERR_INVALID_ARG for an out-of-range field, BGT_ERR_CUDA if
 * the allocation fails. */
bgt_status bgt_create(const bgt_config *cfg, bgt_handle **out);

/* Release the handle and its workspace (synchronizes the device). NULL is a no-op. */
void bgt_destroy(bgt_handle *h);

/* Forward pass (Sec. 3.2 pipeline) of n_views cameras (host array) on
 * `stream`. images: device [sum W H][3], written entirely. The handle keeps
 * the rasterizer outputs, sorted lists, per-pixel final transmittance and
 * the blend records (which Gaussians each pixel composited, with their w and
 * most influential boundary point; capacity max_blend_pairs) for
 * bgt_render_bwd (valid until the next bgt_render_fwd on the handle).
 * BGT_ERR_INVALID_ARG / BGT_ERR_CAPACITY for bad or oversized inputs (checked
 * on the host before any launch), BGT_ERR_CUDA if a launch fails. */
bgt_status bgt_render_fwd(bgt_handle *h, const bgt_scene *scene, const bgt_camera *cams, int n_views,
                          float *images, void *stream);

/* Backward pass for the last forward on this handle: d_images is dl/dC in
 * the image layout (device). Overwrites the gradient arrays of *grads
 * (device, zeroed first; ctrl, color, opacity and r_b always, log_scale, quat
 * and sh when not NULL) with dl/dparameters summed over all views, holding
 * I_id, I_uv, B and the per-pixel survivor lists of the forward fixed
 * (supplementary "Backward Derivative"). The scene and cameras must be those
 * of the forward; BGT_ERR_STATE otherwise or without a forward. */
bgt_status bgt_render_bwd(bgt_handle *h, const bgt_scene *scene, const bgt_camera *cams, int n_views,
                          const float *d_images, const bgt_grads *grads, void *stream);

/* Wait for `stream`, then report and clear the device status word:
 * BGT_ERR_CAPACITY (pairs or boundary pairs exceeded their capacity),
 * BGT_ERR_NONFINITE, or BGT_OK. Blend records that did not fit are not an
 * error (see max_blend_pairs). */
bgt_status bgt_sync_status(bgt_handle *h, void *stream);

/* Text of the last error on this handle ("" if none). Owned by the handle. */
const char *bgt_last_error(const bgt_handle *h);

/* Counts of the last forward, after a synchronize: out[0] = foreground
 * pixels F (= Gaussians), out[1] = boundary points |B|, out[2] = Gaussian
 * tile pairs K, out[3] = boundary tile pairs Kb, out[4] = total tiles,
 * out[5] = blend-record header slots taken (capacity 3/4 max_blend_pairs),
 * out[6] = blend fill-record units taken (capacity max_blend_pairs / 64),
 * out[7] = warp blocks (32 pixels, 128 at tile 32) whose records did not
 * fit: the backward pass re-walks their tile lists instead of replaying
 * records (same gradients, slower); taken slots beyond a capacity were not
 * written. */
bgt_status bgt_get_counts(bgt_handle *h, long long out[8], void *stream);

/* Change the tile size (8, 16 or 32) used by later calls. Images do not
 * depend on it (every pixel composites the same pairs in the same order). */
bgt_status bgt_set_tile_size(bgt_handle *h, int tile_size);
int bgt_get_tile_size(const bgt_handle *h);

/* Per-stage timing: when on, forward and backward record CUDA events on their
 * stream between stages (also inside captured graphs); on = 1 also has the
 * blending kernels count their work units (a build of them with counters,
 * slightly slower), on = 2 times the kernels of the normal step without
 * counting, on = 0 turns profiling off (BGT_ERR_INVALID_ARG otherwise). bgt_get_profile
 * waits for the last backward and returns device milliseconds of the last
 * forward + backward: ms[0] clears + per-primitive prep, [1] tessellation +
 * raster, [2] resolve, [3] sub-primitive generation, [4] binning + sort,
 * [5] forward blending, [6] backward blending, [7] chain to parameters;
 * *kernels_fwd / *kernels_bwd receive the kernels each pass enqueues.
 * units (nullable) receives the work units the blending kernels counted:
 * [0] pairs inside a Gaussian's support (o G >= alpha_min), [1] pairs
 * composited, [2] boundary candidates scanned by the Eq. 6 search, [3]
 * warp visits (a warp of 32 pixels evaluating one listed Gaussian with at
 * least one pixel in its support), for the forward; for the backward, which
 * replays the forward's blend records: [4] and [5] pairs composited, [6]
 * zero, [7] records replayed.
 * BGT_ERR_STATE if profiling is off or no profiled pair has run. */
bgt_status bgt_set_profiling(bgt_handle *h, int on);
bgt_status bgt_get_profile(bgt_handle *h, float ms[8], int *kernels_fwd, int *kernels_bwd,
                           unsigned long long units[8]);

/* Scheduling of the batched launches: the tile size and the work each
 * queue dequeue or persistent block takes. No knob changes an image (every
 * pixel composites the same pairs in the same order); gradients change only
 * by the summation order of FP32 atomics. */
typedef struct {
  int tile_size;           /* screen tile edge: 8, 16 or 32 pixels */
  int raster_prims;        /* primitives each rasterizer warp takes per block, 1..64 (default 8) */
  int bwd_dequeue;         /* warp blocks a backward-blending warp takes per queue dequeue, 1..8 (default 1) */
  int chain_blocks_per_sm; /* persistent blocks per SM of the chain-rule kernels, 1..32 (default 8) */
} bgt_tuning;

/* Current scheduling of the handle. BGT_ERR_INVALID_ARG for NULL. */
bgt_status bgt_get_tuning(const bgt_handle *h, bgt_tuning *out);

/* Set the scheduling used by later calls; BGT_ERR_INVALID_ARG (nothing
 * changed) for a value out of its range. A backward must follow a forward
 * of the same tile size (changing the tile size invalidates the forward). */
bgt_status bgt_set_tuning(bgt_handle *h, const bgt_tuning *t);

/* Autotuner: time `iters` forward + backward passes of this workload at each
 * tile size in {8, 16, 32} with CUDA events on `stream`, keep the fastest and
 * return it in *best (ms per pass of each size in ms_out[3] if non-NULL);
 * then, at that tile size, time the other knobs of bgt_tuning one at a time
 * (raster_prims in {4, 8, 16}, bwd_dequeue in {1, 2, 4},
 * chain_blocks_per_sm in {4, 8, 16}) and keep each fastest value. The
 * candidates of each knob are timed in two interleaved rounds, each keeping
 * its faster time. Read the chosen tuple with bgt_get_tuning. Buffers as for
 * bgt_render_fwd / bgt_render_bwd. */
bgt_status bgt_autotune(bgt_handle *h, const bgt_scene *scene, const bgt_camera *cams, int n_views,
                        float *images, const float *d_images, const bgt_grads *grads, int iters,
                        int *best, float *ms_out, void *stream);

/* Loss helper for training loops and benchmarks: L1 loss
 * l = scale * sum |images - target| over n floats; writes dl/dC =
 * scale * sign(images - target) to d_images and atomically adds l to *loss
 * (device, may be NULL). */
bgt_status bgt_l1_loss_grad(const float *images, const float *target, long long n, float scale,
                            float *d_images, float *loss, void *stream);

/* Photometric training loss of Sec. 3.3, Eq. 9, and its gradient, fused.
 * images, target: device, the renderer's image layout ([sum W H][3] float,
 * view v an [H_v][W_v][3] block); sizes: host [n_views][2] = (W_v, H_v).
 * For each view
 *   L_v = (1 - lambda) * L2 + lambda * (1 - SSIM),
 * L2 the mean of (images - target)^2 over the view's 3 W H values and SSIM
 * the mean over its pixels and channels of the SSIM map (11 x 11 Gaussian
 * window of sigma 1.5 normalised to one, values outside the image taken as
 * zero, C1 = 0.01^2, C2 = 0.03^2, each channel on its own); the paper uses
 * lambda = 0.2. Writes scale * dL_v/dC to d_images (same layout, written
 * entirely) and atomically adds scale * sum_v L_v to *loss (device float,
 * may be NULL; the caller zeroes it). d_images must not overlap images or
 * target. BGT_ERR_INVALID_ARG for negative sizes, a view of more than
 * 2^31 / 3 pixels, lambda outside [0, 1], a non-finite scale, missing or
 * aliased buffers (checked on the host before any launch). */
bgt_status bgt_l2_dssim_loss_grad(const float *images, const float *target, int n_views, const int *sizes,
                                  float lambda, float scale, float *d_images, float *loss, void *stream);

/* Output arrays of bgt_subdivide (device memory, caller-owned), laid out like
 * the bgt_scene arrays of 4 * n_sel primitives with the input's degree,
 * attr_res and sh_degree. sh may be NULL when sh_degree = 0. */
typedef struct {
  float *ctrl;      /* [4 n_sel][Ncp][3] */
  float *color;     /* [4 n_sel][Ncp][3] */
  float *opacity;   /* [4 n_sel] */
  float *r_b;       /* [4 n_sel] */
  float *log_scale; /* [4 n_sel][T][3] */
  float *quat;      /* [4 n_sel][T][4] */
  float *sh;        /* [4 n_sel][K][3] */
} bgt_prims;

/* Measures of the pruning and splitting criteria (Sec. 3.3 "Splitting and
 * Pruning") for the num_prims degree-`degree` primitives of `scene` (device
 * arrays; only ctrl is read):
 *   area[m]   sum of the areas of the four planar triangles through the three
 *             corners and the surface points at the edge midpoints, in the
 *             pattern of the midpoint split;
 *   aspect[m] longer / shorter side of the bounding rectangle of the control
 *             points in the plane of the three corners, its first axis along
 *             the longest corner edge (+inf when the corners are collinear);
 *   grad[m]   mean over the control points of |dl/dp_ijk| from g_ctrl
 *             ([M][Ncp][3] device, e.g. bgt_grads.ctrl; may be NULL);
 *   flags[m]  bit 0 = prune (area < tau_a or aspect > tau_s; the paper uses
 *             3e-4 and 10), bit 1 = split (grad > tau_g, the paper's 0.0018,
 *             with g_ctrl; or edge_sum[m] > tau_b edge_count[m], the
 *             accumulated average of the edge prior above the paper's 13,
 *             with edge_sum / edge_count from bgt_edge_prior), bit 2 = occluded in the views
 *             (view_count[m] < tau_v n_views, the paper's 0.08), bit 3 =
 *             occluded in its visibility texture (set bits of its cell_mask
 *             words < tau_r L^2, the paper's 0.4, L = tess_level); bits 2 and
 *             3 need view_count / cell_mask (from bgt_visibility, device).
 * Each output (device, M entries) may be NULL. BGT_ERR_INVALID_ARG for a
 * degree outside 1..4, a NULL scene or ctrl with M > 0, n_views < 0, a
 * tess_level outside 1..16 with a cell_mask, or only one of edge_sum and
 * edge_count. */
bgt_status bgt_prim_metrics(int degree, const bgt_scene *scene, const float *g_ctrl, float tau_a, float tau_s,
                            float tau_g, const float *edge_sum, const int *edge_count, float tau_b,
                            const int *view_count, int n_views, const unsigned long long *cell_mask, int tess_level,
                            float tau_v, float tau_r, float *area, float *aspect, float *grad, unsigned char *flags,
                            void *stream);

/* Edge prior of the split criterion (Sec. 3.3 "Splitting and Pruning"),
 * step 1: the edge magnitude of training images, the Sobel gradient magnitude
 * sqrt(Gx^2 + Gy^2) of the 8-bit luma 255 (0.299 R + 0.587 G + 0.114 B) with
 * the unnormalised 3 x 3 Sobel pair and the border replicated. images:
 * device, the renderer's layout ([sum W H][3], view v an [H_v][W_v][3]
 * block, values in [0, 1]); sizes: host [n_views][2] = (W_v, H_v); edges:
 * device [sum W H], written entirely. BGT_ERR_INVALID_ARG for negative sizes,
 * more than 2^31 / 3 pixels or missing buffers. */
bgt_status bgt_edge_magnitude(const float *images, int n_views, const int *sizes, float *edges, void *stream);

/* Edge prior, step 2: edges ([sum W H] device, e.g. from
 * bgt_edge_magnitude of the training images of the views of the last
 * bgt_render_fwd on the handle) back-projected onto the primitives through
 * that forward's I_id: edge_sum[m] += the sum of edges over the pixels
 * primitive m owns, edge_count[m] += their number (device arrays of
 * num_prims, accumulated across calls; either may be NULL). The split
 * criterion of bgt_prim_metrics compares edge_sum / edge_count with tau_b
 * (the paper's 13). BGT_ERR_STATE without a forward. */
bgt_status bgt_edge_prior(bgt_handle *h, const float *edges, float *edge_sum, int *edge_count, void *stream);

/* Visibility measures of the pruning criteria (Sec. 3.3 "Splitting and
 * Pruning"), from the raster of the last bgt_render_fwd on the handle:
 * view_count[m] += the number of its views in which primitive m owns at
 * least one pixel of I_id; cell_mask[m * words + s / 64] |= 1 << (s % 64) for
 * every flat triangle s = 2 (a L + b) + down of its level-L lattice (the
 * raster's sub-triangles, L = tess_level) through which it owns a pixel in
 * one of the views: its visibility texture, words = ceil(2 L^2 / 64). Device
 * arrays of num_prims (cell_mask: num_prims * words) entries, accumulated
 * across calls, so that views rendered in several forwards add up (the
 * caller zeroes them when a tracking period starts); either may be NULL.
 * BGT_ERR_STATE without a forward; BGT_ERR_CUDA if a launch fails. */
bgt_status bgt_visibility(bgt_handle *h, int *view_count, unsigned long long *cell_mask, void *stream);

/* The 1 -> 4 split of Sec. 3.3 ("Splitting and Pruning"): each primitive
 * sel[s] (device int array of n_sel indices into scene) becomes the pieces
 * 4 s + p, p = U corner, V corner, W corner, middle, with corners (U, M_uv,
 * M_uw), (M_uv, V, M_vw), (M_uw, M_vw, W), (M_vw, M_uw, M_uv) of its
 * parameter domain (M the edge midpoints; every piece keeps the parent's
 * orientation). Control points and colour control points are the exact
 * restriction of the degree-n Bezier patch to the piece (its polar form at
 * the piece's corners); opacity, r_b and SH coefficients are copied; each
 * texel of a piece's rotation / scaling maps (attr_res R > 1) is the
 * parent map's Eq. 5 interpolation at the texel's node. The pieces of an
 * index outside [0, num_prims) are written as NaN. `out` must not overlap
 * the scene's arrays. BGT_ERR_INVALID_ARG for a degree outside 1..4, n_sel
 * < 0 or > 2^28, or NULL arrays that the call needs. */
bgt_status bgt_subdivide(int degree, const bgt_scene *scene, const int *sel, int n_sel, const bgt_prims *out,
                         void *stream);

/* Intermediate buffers of the last forward, copied to host memory for stage
 * tests. `which`: 0 I_id int32[P]; 1 I_uv float[P][2]; 2 Gaussian records
 * float[F][12] (off_x, off_y, K_a, K_b, K_c, o, bits(qx|qy<<16), bits(prim),
 * r, g, b, depth); 3 boundary records float[Nb][8] (pixel, prim, off_x,
 * off_y, sigma, z, 0, 0 with pixel and prim as int32 bits); 4 per-tile
 * Gaussian ranges int64[tiles+1]; 5 sorted Gaussian keys uint64[K] (bits 63..32 FP32 depth, 31..27 finer
 * depth, 26..0 Gaussian index); 6 per-tile
 * boundary ranges int64[tiles+1]; 7 sorted boundary keys uint64[Kb] (primitive << 32 | boundary index);
 * 8 final transmittance float[P]; 9 per-pixel count of list entries
 * processed int32[P]; 10 per-Gaussian gradients float[F][12] (dl/dmu x, y,
 * dl/dK a, b, c, dl/do, dl/dcolour r, g, b, 0, 0, 0);
 * 11 per-boundary-point gradients float[Nb][4]. `bytes` is the size of dst;
 * *written receives the bytes copied. Synchronizes `stream`. */
bgt_status bgt_get_stage(bgt_handle *h, int which, void *dst, long long bytes, long long *written,
                         void *stream);

/* Binning + sort stage on its own (Sec. 3.2 "Rendering Acceleration"; the
 * (tile, depth) sort): `count` projected Gaussians of one W x H view given
 * as device arrays qxy int32[count] (qx | qy << 16), off float[count][2],
 * conic float[count][3], opacity float[count], depth float[count]. The
 * Gaussians are binned to tiles of the handle's tile size by their support
 * o exp(-1/2 d^T K d) >= alpha_min and sorted inside each tile by
 * (depth, index); read the result with bgt_get_stage(4) and (5). */
bgt_status bgt_bin_sort(bgt_handle *h, int width, int height, int count, const int *qxy, const float *off,
                        const float *conic, const float *opacity, const float *depth, void *stream);

/* Binning + per-tile sort without any device allocation. The paper has no
 * counterpart: this entry exists for callers that cannot call cudaMalloc --
 * code running inside another framework's memory pool (whose allocator owns
 * the device memory), or plugins whose device memory is fixed when they are
 * loaded -- and so cannot create a handle.
 *
 * It computes what bgt_bin_sort computes (same Gaussians in, same tile
 * ranges and sorted keys out), for one width x height view with tiles of
 * tile_size (8, 16, 32) and the given alpha_min. Inputs as for bgt_bin_sort
 * (device). Outputs (device, caller-owned): out_ranges int64[tiles + 1], the
 * start of each tile's keys plus the total; out_keys uint64[key_capacity],
 * the keys of each tile sorted ascending (FP32 depth bits << 32 | 5 finer
 * depth bits << 27 | Gaussian index).
 *
 * Scratch: one static device array of about 5.4 MB, held by every GPU that
 * loads the library until the process exits. Limits: count <= 65,536
 * Gaussians, tiles <= 16,384, total keys <= 262,144; larger inputs return
 * BGT_ERR_CAPACITY (count and tiles before any work, the key total after the
 * counting pass). Every call waits for `stream` once, on the host, to read
 * the key total, and returns after the sort is enqueued. The first call on a
 * device looks up the array's device address and keeps it for the life of
 * the CUDA context (do not use the library across a cudaDeviceReset); make
 * that first call before any stream capture. Calls share the array: two
 * calls that overlap on the GPU (other streams, other threads) race and
 * corrupt each other's results. */
bgt_status bgt_bin_sort_static(int width, int height, int tile_size, int count, const int *qxy,
                               const float *off, const float *conic, const float *opacity,
                               const float *depth, float alpha_min, long long *out_ranges,
                               unsigned long long *out_keys, long long key_capacity, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* BGT_H */
