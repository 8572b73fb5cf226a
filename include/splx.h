/*
 * splx.h - C ABI of the GB300-native Splaxel hot path (libsplx.so).
 *
 * The library renders K Gaussian subsets of a 3D Gaussian Splatting scene into partial
 * pixel images (premultiplied colour C^m, transmittance T^m, alpha-weighted depth D^m;
 * Sec. 4.1 "Local Rendering", Eq. 3-4), composites them per pixel in depth order into
 * the final image (Sec. 4.1 "Global Composition", Eq. 5), back-propagates a pixel loss
 * gradient through both steps to the Gaussian parameters (Sec. 4.1 "Backward
 * Propagation", Eq. 6-7) and applies Adam (Sec. 2, step 4 "Parameter Optimization").
 * The K subsets the paper places on K GPUs are all resident on one device here.
 *
 * Conventions shared by every entry point
 *   - Pointers are DEVICE pointers unless a comment says "host".  The caller owns every
 *     buffer it passes (parameters, gradients, Adam moments, images, partials) and must
 *     keep it alive until the stream work completes.  The library owns its scratch and
 *     the opaque objects it returns.
 *   - Every call is asynchronous on `stream` (NULL = legacy default stream) unless its
 *     comment says it synchronises.  No call throws, aborts or traps; each returns a
 *     status code below.  Errors detected on the device (capacity overflow, a bounded
 *     wait that gave up) set a device status word read by splx_device_status().
 *   - Gaussian parameters are FP32 structure-of-arrays: means [n][3], log_scales [n][3],
 *     quats [n][4] as (w,x,y,z) (normalised on use), opacity_logits [n] (opacity =
 *     sigmoid), sh [n][(deg+1)^2][3] real spherical-harmonic coefficients (colour =
 *     max(0, SH(view direction) + 0.5)).  Theta_i = {mu, R, S, o, c} of Sec. 2.
 *   - Images are planar FP32: rgb [3][H][W], T [H][W]; pixel (x, y) has centre
 *     (x + 0.5, y + 0.5).  Camera space is x right, y down, z forward.
 *   - Gradients are ACCUMULATED (+=) into the caller's arrays, so K subsets and many
 *     views can share one gradient buffer; zero it before a step.
 */
#ifndef SPLX_H
#define SPLX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------------ */
#define SPLX_OK 0
#define SPLX_ERR_INVALID (-1)   /* bad argument (null pointer, size, alignment, option) */
#define SPLX_ERR_BUDGET (-2)    /* the context's HBM budget would be exceeded */
#define SPLX_ERR_CAPACITY (-3)  /* a pair buffer overflowed on the device; re-plan larger */
#define SPLX_ERR_CUDA (-4)      /* a CUDA runtime call failed (see splx_last_cuda_error) */
#define SPLX_ERR_TIMEOUT (-5)   /* a bounded device wait gave up */
#define SPLX_ERR_STATE (-6)     /* object used in the wrong state (e.g. stale forward state) */

typedef struct CUstream_st* splx_stream_t; /* a cudaStream_t */
typedef struct splx_ctx_s* splx_ctx_t;     /* library-owned context (scratch pool, budget) */
typedef struct splx_state_s* splx_state_t; /* forward state of one (view, subset) render */
typedef struct splx_batch_s* splx_batch_t; /* planned batch of V views x K subsets */
typedef struct splx_graph_s* splx_graph_t; /* captured CUDA graph of library calls */
typedef struct splx_server_s* splx_server_t; /* render server over a resident scene */

/* One Gaussian subset Q^m (read-only parameters). */
typedef struct {
  const float* means;
  const float* log_scales;
  const float* quats;
  const float* opacity_logits;
  const float* sh;
  int64_t n;          /* Gaussians in the subset, < 2^31 */
  int32_t sh_degree;  /* 0..3 */
} splx_gaussians;

/* Mutable parameter arrays with the same layout: gradients (+=), Adam moments, or the
 * parameters being optimised. */
typedef struct {
  float* means;
  float* log_scales;
  float* quats;
  float* opacity_logits;
  float* sh;
  int64_t n;
  int32_t sh_degree;
} splx_params;

/* Pinhole camera (host struct).  R is the world->camera rotation (row-major), t the
 * translation: x_cam = R x_world + t.  fx, fy, cx, cy in pixels. */
typedef struct {
  float R[9];
  float t[3];
  float fx, fy, cx, cy;
  int32_t width, height; /* 1..16384 */
  float near_plane;      /* Gaussians with camera depth <= near_plane are culled */
} splx_camera;

/* Rendering options (host struct). */
typedef struct {
  int32_t tile;    /* tile side: 8, 16 or 32; results do not depend on it */
  float eps_T;     /* a pixel stops before the Gaussian that would take T below eps_T */
  float eps_comp;  /* composition skips subsets once the prefix transmittance < eps_comp
                      (the saturation threshold, 1e-4 in Sec. 5.4) */
  float alpha_min; /* Gaussians with alpha < alpha_min are skipped (1/255) */
  float alpha_max; /* alpha is clamped to alpha_max (0.99) */
  float bg[3];     /* background colour added behind the composite */
} splx_opts;

/* Partial pixel image of one (view, subset): Eq. 3-4.  rgb = C^m premultiplied
 * [3][H][W]; T = T^m [H][W]; depth = D^m = sum_i d_i alpha_i T_i [H][W] (Eq. 4 read with
 * the alpha_i factor); last = position of the last blended entry in the subset's sorted
 * tile list, -1 if none [H][W] (used by the backward to recompute the blend). */
typedef struct {
  float* rgb;
  float* T;
  float* depth;
  int32_t* last;
} splx_partial;

/* Adam hyper-parameters (host struct); torch.optim.Adam semantics. */
typedef struct {
  float lr[6]; /* means, log_scales, quats, opacity_logits, sh degree-0, sh higher */
  float beta1, beta2, eps;
  int32_t zero_grad; /* nonzero: the gradient arrays are set to 0 after they are read */
} splx_adam;

/* ---- context ------------------------------------------------------------------ */

/* Creates a context on CUDA device `device` whose scratch never exceeds
 * `hbm_budget_bytes` (0 = no cap).  Scratch comes from a stream-ordered pool the
 * context owns.  Returns SPLX_ERR_INVALID for a bad device. */
int splx_create(splx_ctx_t* out, int device, size_t hbm_budget_bytes);
/* Synchronises the device, frees all scratch and the context. */
int splx_destroy(splx_ctx_t ctx);
/* Scratch bytes currently held by the context (host value). */
size_t splx_scratch_bytes(splx_ctx_t ctx);

/* ---- per-view entry points (Sec. 4.1) ------------------------------------------- */

/* Local rendering of one subset for one view (Sec. 4.1, Eq. 3-4; steps 1-3 of Sec. 2):
 * projection with EWA covariance, SH colour, 16x16 (opts->tile) binning, sort of each
 * tile's list by depth with the Gaussian index as tie-break, front-to-back blending into
 * `out` (sized to cam->width x cam->height).  If state_out is non-NULL the projected
 * records and sorted lists are kept for splx_backward and must be released with
 * splx_state_release.  Synchronises once (to size the pair list). */
int splx_render_partial(splx_ctx_t ctx, const splx_gaussians* subset, const splx_camera* cam,
                        const splx_opts* opts, const splx_partial* out, splx_state_t* state_out,
                        splx_stream_t stream);
/* Cross-boundary per-ray filtering on the per-view path (Sec. 8.1, appendix "Cross-boundary
 * Gaussians Handling"; the batch's splx_batch_set_cross_filter per view).  The filter of
 * one view needs every subset's visible region and depth range in that view:
 * splx_view_regions projects the K subsets (device pointers, as for a batch) for `cam` and
 * writes regions_out (host, [K][6] uint32: the visible region's tile rectangle x0, y0,
 * ~x1, ~y1 and the FP32 depth bits min, ~max of the Gaussians the projection keeps; an
 * empty subset gives 0xFFFFFFFF throughout).  Synchronises `stream`.  No device memory
 * outlives the call. */
int splx_view_regions(splx_ctx_t ctx, const splx_gaussians* subsets, int32_t K,
                      const splx_camera* cam, const splx_opts* opts, uint32_t* regions_out,
                      splx_stream_t stream);
/* splx_render_partial of subset k of K with cross-boundary filtering: cells (host, [K][6]
 * floats, the k-d boxes lo x, y, z, hi x, y, z, +-INFINITY on open sides; NaN rejected) and
 * regions (host, [K][6], from splx_view_regions for the same camera and options).  A
 * Gaussian of subset k whose support box mu +- 3 s_max meets another cell s leaves the rays
 * of every tile of its own list that lies in s's visible region when its depth lies in the
 * overlap of the two subsets' depth ranges; its pairs there sort last and stay out of the
 * tile's range, so the kept state's backward (splx_backward) follows the same lists.  The
 * partial equals the batch's filtered partial of that subset bit for bit.  K in 1..64,
 * 0 <= k < K, else SPLX_ERR_INVALID. */
int splx_render_partial_filtered(splx_ctx_t ctx, const splx_gaussians* subset, int32_t k,
                                 int32_t K, const float* cells, const uint32_t* regions,
                                 const splx_camera* cam, const splx_opts* opts,
                                 const splx_partial* out, splx_state_t* state_out,
                                 splx_stream_t stream);

/* Global composition (Sec. 4.1, Eq. 5): per pixel, orders the K partials by the
 * normalised depth D^m/(1-T^m) (ties to the lower index, empty subsets last) and
 * accumulates C = sum_m C^m prod_{k before m} T^k + bg * prod T, skipping the rest once
 * the prefix product falls below opts->eps_comp.  parts is a host array of K partials
 * (device planes).  out_rgb [3][H][W]; out_T [H][W] (nullable) = prefix product. */
int splx_composite(splx_ctx_t ctx, const splx_partial* parts, int32_t K, int32_t width,
                   int32_t height, const splx_opts* opts, float* out_rgb, float* out_T,
                   splx_stream_t stream);

/* Backward of one view (Sec. 4.1, Eq. 6-7, then the chain through Eq. 1-4 and the
 * projection): given dL/dC of the composited image [3][H][W] and optionally dL/dT of
 * out_T [H][W] (nullable), adds dL/dtheta for every Gaussian of the K subsets into
 * grads[k] (host array of K; device arrays sized like the subsets).  subsets, parts and
 * states are the host arrays used in the forward. */
int splx_backward(splx_ctx_t ctx, const splx_gaussians* subsets, int32_t K,
                  const splx_camera* cam, const splx_partial* parts, const splx_state_t* states,
                  const float* dL_drgb, const float* dL_dT, const splx_opts* opts,
                  const splx_params* grads, splx_stream_t stream);

/* Diagnostic export of a forward state (synchronises): the pair count and tile count
 * (host, either nullable), then - for each non-NULL device buffer - the per-tile
 * [start, end) ranges into the sorted list (ranges_out: n_tiles x 2 uint32), the sorted
 * keys (keys_out: n_pairs uint64, FP32 depth bits << 32 | Gaussian index, each tile's
 * segment ascending) and the 64-byte projected records
 * (rec_out: n x 16 floats: u, v, qa, qb | qc, opacity, depth, rect_x | r, g, b, rect_y |
 * 0,0,0,0 where rect_x = x0 | x1 << 16 and rect_y = y0 | y1 << 16 as bit patterns and
 * (qa, qb, qc) = -log2(e) * (A/2, B, C/2) for the conic (A, B, C); a culled Gaussian has
 * x0 = 0xFFFF > x1).  Tiles are numbered row-major. */
int splx_state_export(splx_ctx_t ctx, splx_state_t state, int64_t* n_pairs, int64_t* n_tiles,
                      uint32_t* ranges_out, uint64_t* keys_out, float* rec_out,
                      splx_stream_t stream);

/* Releases a forward state (stream-ordered). */
int splx_state_release(splx_ctx_t ctx, splx_state_t state, splx_stream_t stream);

/* Adam step on one parameter set (Sec. 2 step 4; the paper names no optimiser, torch
 * Adam semantics are used): m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
 * p -= lr * (m / (1-b1^step)) / (sqrt(v / (1-b2^step)) + eps), per-group lr. */
int splx_step(splx_ctx_t ctx, const splx_params* p, const splx_params* g, const splx_params* m,
              const splx_params* v, const splx_adam* hp, int64_t step, splx_stream_t stream);

/* splx_step with the step number on the device: *step_dev (device int64) is incremented
 * first and the update uses the new value, so a CUDA graph holding this call advances
 * the bias correction on every replay. */
int splx_step_device(splx_ctx_t ctx, const splx_params* p, const splx_params* g,
                     const splx_params* m, const splx_params* v, const splx_adam* hp,
                     int64_t* step_dev, splx_stream_t stream);

/* L1 photometric loss (Sec. 2 step 4, the L_RGB term): loss_out[0] = mean |img - target|
 * over n elements and dL_dimg = sign(img - target)/n (sign(0) = 0).  dL_dimg nullable.
 * loss_out is a device float (overwritten). */
int splx_loss_l1(splx_ctx_t ctx, const float* img, const float* target, int64_t n,
                 float* loss_out, float* dL_dimg, splx_stream_t stream);
/* Photometric loss with the structural term (Sec. 2 step 4: L = L_RGB + L_D-SSIM, read as
 * (1 - lambda) L1 + lambda (1 - SSIM); lambda = 0.2 in 3DGS practice).  SSIM per channel
 * with an 11 x 11 Gaussian window (sigma 1.5), zero padding, C1 = 0.01^2, C2 = 0.03^2; both
 * terms are means over the 3 W H elements of the image [3][H][W].  loss_out (device float)
 * is overwritten; dL_dimg [3][H][W] receives the gradient (overwritten).  lambda in [0, 1],
 * else SPLX_ERR_INVALID.  Allocates its scratch (12 floats per pixel) from the context. */
int splx_loss_l1_dssim(splx_ctx_t ctx, const float* img, const float* target, int32_t width,
                       int32_t height, float lambda, float* loss_out, float* dL_dimg,
                       splx_stream_t stream);

/* ---- batched path: V views x K subsets per launch (conflict-free view consolidation
 *      of Sec. 4.3 in spirit: many independent views run in the same kernels) ------- */

/* Plans a batch.  subsets (host array of K) share one SH degree; cams (host array of
 * V).  Each view keeps its resolution for the life of the batch; poses may change with
 * splx_batch_set_cameras.  pair_capacity = max (Gaussian, tile) pairs the batch holds;
 * 0 = measure once now (synchronises) and add 25% headroom.  The batch owns scratch for
 * V*K partial images, the projected records and the pair lists; it reads parameters
 * through the subset pointers on every run. */
int splx_batch_create(splx_ctx_t ctx, const splx_gaussians* subsets, int32_t K,
                      const splx_camera* cams, int32_t V, const splx_opts* opts,
                      int64_t pair_capacity, splx_batch_t* out, splx_stream_t stream);
/* Replaces the V camera poses (resolutions must be unchanged); host cams are copied
 * through a pinned staging buffer, so the call is capturable. */
int splx_batch_set_cameras(splx_batch_t b, const splx_camera* cams, int32_t V,
                           splx_stream_t stream);
/* Offsets (in floats) of view v's image inside the concatenated outputs: rgb at
 * rgb_off[v] (3*H_v*W_v floats), T at pix_off[v]; host arrays of V+1 entries each. */
int splx_batch_layout(splx_batch_t b, int64_t* rgb_off, int64_t* pix_off);
/* Forward of all V views: local render of every (view, subset) then composition.
 * out_rgb / out_T are the concatenated images (layout from splx_batch_layout).  Never
 * synchronises; capturable once the batch exists. */
int splx_batch_forward(splx_batch_t b, float* out_rgb, float* out_T, splx_stream_t stream);
/* Backward of the last forward: dL_drgb / dL_dT (nullable) concatenated like the
 * outputs; gradients added into grads[k] (host array of K).  Capturable. */
int splx_batch_backward(splx_batch_t b, const float* dL_drgb, const float* dL_dT,
                        const splx_params* grads, splx_stream_t stream);
/* Backward of the last forward with the Adam step fused into the projection adjoint
 * (Sec. 4.1 step 3): the same result as splx_batch_backward into zeroed gradients followed
 * by splx_step_device over every subset, but no gradient array exists; each Gaussian's
 * parameters, first and second moments are updated straight from its gradient of this
 * backward (Gaussians without one take a zero gradient, as after zero_grad).
 *   params[k]  device arrays of subset k's Gaussians, the very arrays the batch was
 *              created on (checked: SPLX_ERR_INVALID otherwise); overwritten in place.
 *   m[k], v[k] device Adam moments of subset k (same layout), updated in place.
 *   hp         learning rates, betas, eps (zero_grad is ignored: there is no gradient).
 *   step_dev   device int64 step counter, incremented first; the update uses the new value.
 * Host arrays params, m, v hold K entries each; nothing is owned by the call (the batch
 * keeps one flag byte per 128 Gaussians, allocated at the first call: blocks without any
 * gradient are updated by a second, streaming pass).  Never synchronises; capturable once
 * the batch exists.  Per-element arithmetic is that of splx_step, so both routes give
 * bit-identical parameters. */
int splx_batch_backward_adam(splx_batch_t b, const float* dL_drgb, const float* dL_dT,
                             const splx_params* params, const splx_params* m,
                             const splx_params* v, const splx_adam* hp, int64_t* step_dev,
                             splx_stream_t stream);
/* Total pairs of the last forward and the device status word (synchronises).  Returns
 * SPLX_ERR_CAPACITY if the pair list overflowed (its forward output is invalid). */
int splx_batch_status(splx_batch_t b, int64_t* pairs_out, splx_stream_t stream);
int splx_batch_destroy(splx_batch_t b);
/* Per-kernel timing (off by default).  When enabled the batch records CUDA events around
 * each of its kernels; inside a captured graph they become event nodes, so every replay
 * re-records them.  splx_batch_kernel_times waits for the last run's final event and
 * writes 9 durations in ms (host array): project, scan, fill, sort, raster_fwd,
 * composite, composite_bwd, raster_bwd, project_bwd.  With saturation skipping on and at
 * least two views, the waves of up to four view groups (about equal pixels each) run side
 * by side on their own streams; sort and raster_fwd are then the first group's stream's
 * intervals, which add up to the waves' whole span. */
int splx_batch_set_timing(splx_batch_t b, int enable);
/* Launch shape of the batch's rasterisers (the autotuner's second axis beside the tile
 * side; Sec. 4.3's aim of keeping every SM busy).  raster_ctas_per_sm = 0 launches one
 * CTA per (view, subset, tile) work item; n > 0 launches n CTAs per SM that take work
 * items in order from a device counter until none is left (persistent).  Results do not
 * depend on it except for the summation order of gradient atomics.  0..64, else
 * SPLX_ERR_INVALID.  Applies to launches issued afterwards (a captured graph keeps the
 * shape it was captured with). */
int splx_batch_set_launch(splx_batch_t b, int32_t raster_ctas_per_sm);
/* The loss of splx_loss_l1_dssim over the batch's V views: rgb and target are the
 * concatenated images (layout from splx_batch_layout), the means run over all 3 x total
 * pixels, dL_drgb is concatenated like rgb.  Scratch (12 floats per pixel) is allocated by
 * the first call, which must not be inside a stream capture (SPLX_ERR_STATE); later calls
 * are capturable. */
int splx_batch_loss_l1_dssim(splx_batch_t b, const float* rgb, const float* target,
                             float lambda, float* loss_out, float* dL_drgb, splx_stream_t stream);
/* Spatial visibility (Sec. 4.2 "spatial visibility", the region Omega_v^m of subset m in
 * view v).  On by default for batches: the projection records, per (view, subset), the
 * bounding tile rectangle of the subset's (Gaussian, tile) pairs; work items outside it
 * have no pairs, so the rasterisers skip them and the composites neither write nor read
 * their partial planes (treated as empty: C = 0, T = 1).  Results are identical with it on
 * or off.  enable = 0 turns it off for launches issued afterwards. */
int splx_batch_set_visibility(splx_batch_t b, int32_t enable);
/* Selected-prefix sort of long tile segments (the per-tile depth sort of Sec. 2 step 2,
 * restricted to what the forward reaches).  On by default for batches: a segment longer
 * than 2048 keys gets only its nearest keys (at most 2048, the keys below a depth threshold
 * read from a two-level histogram of the key's depth bits) sorted, and the forward walks
 * that prefix; a work item whose pixels are still blending at the prefix's end renders
 * nothing in that pass, and after its segment is sorted whole it is rendered again, so
 * images, transmittances and gradients are those of whole-segment sorts.  enable = 0 sorts
 * every segment whole, for launches issued afterwards (a captured graph keeps the mode it
 * was captured with).  Off while cross-boundary filtering is on, and for a pair capacity
 * of 2^31 or more. */
int splx_batch_set_prefix_sort(splx_batch_t b, int32_t enable);
/* Keeps the selected-prefix sort on only if the last eager forward handed at most a
 * quarter of its prefix items back to the whole sort (their pixels still blending at the
 * prefix's end: tiles with long lists of small or faint Gaussians), and turns it off
 * otherwise, for launches issued afterwards; call it between an eager forward and a graph
 * capture.  Synchronises `stream`; not capturable; SPLX_ERR_INVALID without a batch state. */
int splx_batch_tune_prefix_sort(splx_batch_t b, splx_stream_t stream);
/* Cross-boundary per-ray filtering (Sec. 8.1, appendix "Cross-boundary Gaussians
 * Handling").  cells (host, [K][6] floats: lo x, y, z, hi x, y, z of subset k's k-d box,
 * +-INFINITY on open sides; NaN rejected) turns it on for launches issued afterwards (and
 * spatial visibility with it); NULL turns it off.  A Gaussian of subset k whose support box
 * mu +- 3 s_max (FP32, s_max its largest activated scale exp(log_scale)) meets another
 * cell s leaves the rays of every tile of view v that lies in Omega_v^s (the visible region
 * of splx_batch_set_visibility) when its FP32 camera depth lies in the overlap of the two
 * subsets' depth ranges in view v (min and max depth of the Gaussians the projection
 * keeps).  Forward and backward take the same decisions; results change where a filtered
 * Gaussian contributed.  Device memory: 8 B per Gaussian + 8 B per (view, subset). */
int splx_batch_set_cross_filter(splx_batch_t b, const float* cells);
/* Saturation skipping (Sec. 4.2 "saturation skipping", with the composite's threshold
 * eps_comp of splx_opts).  order (host, [V][K]) is, per view, a front-to-back order of the
 * K subsets (for k-d cells: the BSP order from the camera centre).  Once set, the forward
 * renders the subsets in K waves in that order, and a subset leaves a pixel empty (C = 0,
 * T = 1, D = 0, no contributor) where the product of the transmittances of the subsets
 * rendered before it is below eps_comp: saturated pixels leave the subset's pixel set.  A
 * (view, subset, tile) work item with no open pixel is neither sorted nor rendered; the
 * backward has nothing to do at empty pixels.  The composite skips such subsets at those
 * pixels anyway, so images and gradients are unchanged wherever the per-pixel subset order
 * of Eq. 5 agrees with the given order.  NULL turns skipping off.  Each row must be a
 * permutation of 0..K-1, else SPLX_ERR_INVALID.  Synchronises; applies to launches
 * issued afterwards. */
int splx_batch_set_order(splx_batch_t b, const int32_t* order);
/* Stale saturation state (Sec. 4.2 step 2: the pixels that one visit's composition finds
 * saturated leave the subsets behind in the view's next visit).  sat (host array of V)
 * holds one device plane per view, sat[v] of H_v * W_v bytes (row-major, owned by the
 * caller, kept alive while set).  Value s at a pixel prunes the subsets of rank >= s in
 * the view's order (splx_batch_set_order): they leave the pixel empty as in the waves
 * above.  Values >= K prune nothing: fill a plane with 255 for a view's first visit.
 * While set, each forward renders with one sort and one rasteriser launch (no waves),
 * leaves out every (view, subset, tile) work item pruned at all its pixels, and after the
 * composite overwrites each plane with the state re-evaluated from this visit's partials:
 * the first rank r + 1 whose prefix (FP32 product of the partial transmittances of ranks
 * 0..r, in order) is below eps_comp, among ranks below the old state, else 255.  Pruned
 * ranks count as transparent there, so a pixel whose prefix no longer saturates gets all
 * of them back at the next visit.  A visit after an identical one renders exactly what
 * the waves render; when the scene changed in between, the pruned pixels miss what the
 * pruned subsets would now add (the price of a stale state).  The state belongs to the
 * view's pose and order: reset it (255) when either changes.  NULL turns it off.
 * SPLX_ERR_STATE without an order, SPLX_ERR_INVALID for a NULL plane.  Synchronises;
 * applies to launches issued afterwards (a captured graph reads the planes set when it
 * replays). */
int splx_batch_set_stale(splx_batch_t b, uint8_t* const* sat);
/* Largest number of persistent forward / backward rasteriser CTAs resident on one SM at
 * the batch's tile side (host outputs). */
int splx_batch_max_ctas_per_sm(splx_batch_t b, int32_t* fwd, int32_t* bwd);
int splx_batch_kernel_times(splx_batch_t b, float* ms_out);
/* The same 9 durations for the replay of graph g that took ring slot `slot` of
 * splx_graph_set_timing_ring (waits for that replay's final event only).  SPLX_ERR_INVALID
 * for a slot outside the ring. */
int splx_batch_kernel_times_slot(splx_batch_t b, splx_graph_t g, int32_t slot, float* ms_out);
/* Work counters (synchronises; host array of 11): out[0] = (Gaussian, tile) pairs of the
 * last run; then, from the last EAGER run (replays of a captured graph do not count):
 * forward rasteriser out[1] = (thread, list entry) pairs examined, out[2] = (pixel,
 * entry) alpha evaluations, out[3] = (pixel, entry) blends; backward rasteriser out[4] =
 * (thread, entry) pairs, out[5] = alpha evaluations, out[6] = contributions (alpha >=
 * alpha_min); out[7] = (view, subset, tile) work items left empty by saturation skipping
 * (no open pixel); out[8] = work items outside their subset's visible region; out[9] =
 * work items whose segment, longer than 2048 keys, the forward walked on its sorted
 * prefix of the nearest keys (at most 2048), out[10] = those of them (and those with no
 * prefix) whose pixels were still open at the prefix's end, so that the segment was
 * sorted whole and the item rendered again (the batch's results are those of whole
 * sorts either way).
 * A forward thread owns 2 pixels (8x8, 16x16 tiles) or 4 (32x32); a backward thread 2
 * (8x8), 8 (16x16: one warp per tile) or 4 (32x32). */
int splx_batch_counters(splx_batch_t b, int64_t* out, splx_stream_t stream);
/* Number of (view, Gaussian) pairs that the last forward's projection kept (a tile count
 * above zero: the Gaussians that write a record and may receive a 2-D gradient), for the
 * kernels' algorithmic byte counts.  Host output; synchronises; not capturable. */
int splx_batch_visible(splx_batch_t b, int64_t* visible_out, splx_stream_t stream);

/* ---- serving: continuous batching of render requests --------------------------- */
/* A render server keeps K resident subsets and renders requests (a camera of any
 * resolution) with the forward of the hot path: local render of every (view, subset)
 * (Sec. 4.1 "Local Rendering", Eq. 3-4) and composition (Eq. 5).  It has `slots` launch
 * slots, each with its own CUDA stream, so launches overlap on the device.  A slot that
 * is idle takes the oldest queued requests, up to `max_views` of them, as one launch
 * (the spirit of Sec. 4.3's view consolidation); requests are admitted in arrival order
 * while the launch's device footprint (records, partial planes, pair buffers estimated
 * from the largest pairs-per-pixel ratio seen so far) fits the server's budget next to
 * the launches in flight.  A launch projects and counts its pairs, and the server reads
 * the exact count behind an event before it allocates the pair buffers, so nothing here
 * blocks the host.  A request's image does not depend on the other requests of its
 * launch (every (view, subset, tile) work item is independent), so results alone and in
 * the mix are bit-identical.
 *
 * Not thread-safe: one host thread drives a server.  Results are written to the
 * caller's device buffer out_rgb [3][H][W] (keep it alive until the request finishes).
 * A request that cannot fit the budget even alone finishes with SPLX_ERR_BUDGET. */
int splx_server_create(splx_ctx_t ctx, const splx_gaussians* subsets, int32_t K,
                       const splx_opts* opts, size_t hbm_budget_bytes, int32_t slots,
                       int32_t max_views, splx_server_t* out);
/* Queues one request (host camera copied) and runs a scheduling pass; *id_out (host) is
 * its id, increasing from 0 in submission order.  order (host, K entries, nullable) is a
 * front-to-back order of the subsets for this camera (see splx_batch_set_order): a launch
 * whose requests all carry one renders with saturation skipping, which leaves the images
 * unchanged wherever a pixel's Eq. 5 order agrees with it.  SPLX_ERR_INVALID if order is
 * not a permutation of 0..K-1. */
int splx_server_submit(splx_server_t s, const splx_camera* cam, const int32_t* order,
                       float* out_rgb, int64_t* id_out);
/* Scheduling pass (never waits on the device): retires finished launches, renders
 * launches whose pair count has arrived, admits queued requests into idle slots; then
 * reports up to `cap` finished requests as (ids[i], status[i]) host arrays, *n_out of
 * them.  status is SPLX_OK or the error that ended the request. */
int splx_server_poll(splx_server_t s, int64_t* ids, int32_t* status, int32_t cap,
                     int32_t* n_out);
/* Host outputs (each nullable): queued requests, requests in flight, reserved bytes. */
int splx_server_stats(splx_server_t s, int32_t* queued, int32_t* inflight, size_t* reserved);
/* Device timeline of a finished request (of the last 65,536): times_ms (host array of 3)
 * receives, in ms after the server's creation, when its launch began on the GPU (before
 * its first kernel), when its projection and tile counts were done, and when its image
 * had been copied out.  Requests launched together share these.  SPLX_ERR_INVALID for an
 * unknown or unfinished id.  Shows how launches overlap on the device. */
int splx_server_request_times(splx_server_t s, int64_t id, float* times_ms);
/* Waits for the launches in flight, releases everything; queued requests are dropped. */
int splx_server_destroy(splx_server_t s);

/* ---- CUDA graphs of library calls --------------------------------------------- */
/* Begins capturing `stream` (thread-local mode).  Any capturable splx_* calls issued
 * until splx_graph_end become one graph. */
int splx_graph_begin(splx_ctx_t ctx, splx_stream_t stream);
int splx_graph_end(splx_ctx_t ctx, splx_stream_t stream, splx_graph_t* out);
int splx_graph_launch(splx_graph_t g, splx_stream_t stream);
/* Timing ring (measurement only; the paper has no counterpart).  With slots > 0, launch
 * number i of g records the graph's event nodes (the batch timing events of
 * splx_batch_set_timing captured into it) into ring slot i mod slots instead of the
 * captured events, so the per-kernel times of every replay of a back-to-back run can be read
 * afterwards with splx_batch_kernel_times_slot, with no host wait between replays.  Creates
 * slots x (event nodes) events, owned by g (0 removes the ring; 0..4096, else
 * SPLX_ERR_INVALID).  The next launch takes slot 0. */
int splx_graph_set_timing_ring(splx_graph_t g, int32_t slots);
int splx_graph_destroy(splx_graph_t g);

/* ---- allocation-free local render ----------------------------------------------- */
/* The paper has no counterpart to this entry point; it exists for callers that cannot
 * allocate device memory: a process whose HBM is reserved up front by another allocator
 * (an inference server's arena, a framework caching allocator that already holds the
 * device), or a latency-critical loop where the implicit device synchronisation of
 * cudaMalloc/cudaFree is not acceptable.  It computes exactly what splx_render_partial
 * computes (same kernels) but takes no context, keeps no forward state and allocates
 * nothing: its scratch is one fixed 32 MiB array that every GPU which loads libsplx holds
 * until the process exits.  The caller passes the inputs and the output planes.
 *   - Limits: subset->n <= 65536 Gaussians, at most 2^20 (Gaussian, tile) pairs and at
 *     most 65536 tiles; larger requests return SPLX_ERR_INVALID before any work, and a
 *     pair overflow found on the device returns SPLX_ERR_CAPACITY (output not valid).
 *   - The first call on a device looks up the array's device address (with that device
 *     current) and caches it; make that first call before any stream capture.
 *   - All calls share the array and leave their contents in it: calls that overlap on
 *     the GPU (other streams, other host threads) race on it and must be serialised.
 *   - Synchronises `stream` once at the end to read the device status. */
int splx_render_partial_noalloc(const splx_gaussians* subset, const splx_camera* cam,
                                const splx_opts* opts, const splx_partial* out,
                                splx_stream_t stream);

/* ---- diagnostics ---------------------------------------------------------------- */
/* Synchronises `stream`, returns and clears the context's device status word
 * (SPLX_OK, SPLX_ERR_CAPACITY or SPLX_ERR_TIMEOUT). */
int splx_device_status(splx_ctx_t ctx, splx_stream_t stream);
/* Text of a status code (static storage). */
const char* splx_strerror(int status);
/* Last CUDA error string seen by the library in this thread (static storage). */
const char* splx_last_cuda_error(void);
/* Number of kernel launches issued by the library since the context was created. */
int64_t splx_launch_count(splx_ctx_t ctx);

#ifdef __cplusplus
}
#endif
#endif /* SPLX_H */
