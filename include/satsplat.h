/*
 * satsplat.h -- C ABI of the GB300 affine 2D-Gaussian-splat (surfel) rasterizer.
 *
 * The operation is the differentiable rasterizer of SatSplat (Song, Kim, Qin):
 *   - affine camera x = F [p; 1], F split into the screen rows [B_xy | b_xy]
 *     and the fixed depth row B_z = [0 0 -1], b_z = max_altitude
 *       (Sec. 3.1 Eq. affine_camera; Sec. 3.2 Eq. decompose_affine_camera,
 *        Eq. depth_affine_camera);
 *   - per-camera learnable delta F'_xy = F_xy + dF_xy (Sec. 3.3);
 *   - 2D splats P(u,v) = p + s_u t_u u + s_v t_v v (Sec. 3.1 Eq. 2dgs_splat_param),
 *     intersected with the parallel camera rays analytically:
 *     u = Q x + q, Q = (B_xy R S')^-1, q = -Q (B_xy p + b_xy)
 *       (Sec. 3.2 Eq. affine2dgs_screen2uv, Eq. affine2dgs_Qq);
 *   - lower-bounded Gaussian max(G(u), G((x - c)/sigma)); only the screen-space
 *     term when |det(B_xy R S')| < det_eps (Sec. 3.2, degenerate solutions);
 *   - tiles, splats ordered by the height-based depth of their centres, and
 *     front-to-back alpha blending of colour, depth and normal
 *       (Sec. 3.2 Eq. rasterization; normal definition);
 *   - the sun-direction camera B_sun = B'_xy (I - [0 0 s]),
 *     s = (cos(phi)/tan(theta), sin(phi)/tan(theta), 1), rendering depth for
 *     shadow mapping (Sec. 3.3 Eq. sun_camera_Bxy; Supp. A);
 *   - per-camera 3x4 colour correction C A + c (Sec. 3.1 Eq. image_formation);
 *   - the reverse-mode adjoint of all of the above;
 *   - beside the rasterizer: the sun visibility and image formation, the depth-gradient
 *     normal, the distortion of the blending weights, the optimiser step (Adam with the
 *     3DGS-MCMC noise and relocation) and the geometry-aware DSM initialisation.
 * Constants the paper leaves open (alpha threshold, alpha clamp, early-stop
 * transmittance, sigma, det threshold) are fields of ss_raster_opts.
 *
 * Conventions for every entry point:
 *   - The caller owns all memory; the library never allocates and keeps no
 *     state between calls other than what it writes into the caller's
 *     workspace.  Device pointers must be on the current CUDA device.
 *   - Calls are asynchronous on the given stream, except where stated.  Host
 *     arguments are read during the call and may be released afterwards.
 *   - Arguments are validated on the host before anything is launched; a bad
 *     argument returns SS_ERR_INVALID_ARG and launches nothing.  A failed
 *     launch returns SS_ERR_CUDA.  No exception crosses the boundary.
 *   - Gradient outputs ACCUMULATE (+=); the caller zeroes them.
 *   - A frame is one set of (splats, cameras, passes, options, workspace).
 *     ss_project_splats, ss_bin_and_sort, ss_rasterize_fwd and
 *     ss_rasterize_bwd must be called in that order for the same frame; each
 *     reads what the previous one wrote into the workspace.
 */
#ifndef SATSPLAT_H
#define SATSPLAT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* ss_stream_t; /* a cudaStream_t; NULL = legacy default stream */

typedef enum {
  SS_OK = 0,
  SS_ERR_INVALID_ARG = 1, /* bad pointer, size, alignment, option or layout */
  SS_ERR_CAPACITY = 2,    /* the intersection list did not fit: see ss_bin_and_sort */
  SS_ERR_CUDA = 3,        /* a CUDA runtime call or launch failed */
  SS_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up */
  SS_ERR_NONFINITE = 5    /* a splat or camera value was NaN/Inf (that splat is culled) */
} ss_status;

typedef enum { SS_F32 = 0, SS_BF16 = 1 } ss_dtype;

/* Passes of a frame.  The render targets of a frame are, in this order: the main
 * view of every camera (if SS_PASS_MAIN), then the sun view of every camera (if
 * SS_PASS_SUN).  n_targets = n_cams * (number of bits set). */
enum { SS_PASS_MAIN = 1, SS_PASS_SUN = 2 };

/* Splat attributes (Sec. 3.1 Eq. 2dgs_splat_param).  DEVICE pointers to
 * component-planar arrays [C][n_pad] of `dtype` (fp32 or bf16), 16-byte aligned.
 *   means   [3][n_pad]  p = (x, y, z) in world units (normalised UTM); z is height
 *   scales  [2][n_pad]  s_u, s_v > 0 (already activated)
 *   quats   [4][n_pad]  rotation (w, x, y, z), any non-zero norm (normalised inside)
 *   opacity [n_pad]     o in (0, 1) (already activated)
 *   rgb     [3][n_pad]  per-splat colour (albedo); no spherical harmonics
 * n_pad >= n, a multiple of 8.  Entries n..n_pad-1 are never read. */
typedef struct {
  const void* means;
  const void* scales;
  const void* quats;
  const void* opacity;
  const void* rgb;
  int64_t n;
  int64_t n_pad;
  int32_t dtype; /* ss_dtype */
  int32_t reserved;
} ss_splats;

/* One affine camera (HOST memory; its fixed geometry).  F_xy maps world
 * coordinates straight to pixel coordinates: pixel (i, j) covers [i, i+1) x
 * [j, j+1) and is sampled at its centre (i + 0.5, j + 0.5).  The depth row is
 * fixed: depth = max_alt - height (Sec. 3.2 Eq. depth_affine_camera).  The sun
 * view (Sec. 3.3, Supp. A) uses B_sun = shadow_scale * B'_xy (I - [0 0 s]) and
 * b_sun = shadow_scale * b'_xy on a shadow_w x shadow_h image; its depth is the
 * same height-based depth. */
typedef struct {
  float F_xy[2][4];
  float max_alt;
  int32_t width, height;
  float sun_phi;   /* sun azimuth, radians */
  float sun_theta; /* sun elevation, radians, in (0, pi/2] */
  int32_t shadow_w, shadow_h;
  float shadow_scale;
} ss_camera;

/* Rasterizer options.  ss_default_opts() fills the defaults in brackets. */
typedef struct {
  int32_t tile_w, tile_h; /* screen tile [16 x 16]; also 32 x 8, 8 x 32 (two warps per tile) and
                             32 x 16, 16 x 32 (four warps per tile) */
  int32_t batch;          /* [256], the only value: the kernels' own staging, in which a tile
                             block copies the tile's sorted splat records into shared memory with
                             cp.async in batches (ss_staging_batches gives their sizes) */
  int32_t persistent;     /* [0] one block (one warp per 128 pixels) per tile; 1: one persistent
                             launch whose blocks pull tiles from a queue */
  float sigma_px;         /* screen-space low-pass sigma, pixels [1/sqrt(2)] */
  float det_eps;          /* |det M| threshold, px^2 [1e-6] */
  float alpha_min;        /* a splat contributes iff alpha >= alpha_min [1/255] */
  float alpha_max;        /* alpha = min(alpha_max, o G^) [0.99] */
  float t_min;            /* stop before the splat that takes T below t_min [1e-4] */
  int32_t pixels_per_thread; /* [4], the only value: each lane owns one column of four pixels
                                of a 2 x 4 sub-block.  Tile shape, batch and persistence never
                                change an output. */
  int32_t subblock_cull;  /* [1] each group of lanes walks only the staged splats whose support
                             can reach its sub-block; 0 walks every staged splat in every
                             sub-block.  The outputs are identical (the test is conservative);
                             0 is slower and serves to check that. */
  int32_t count_pairs;    /* [0] 1: ss_rasterize_fwd also counts the walked (pixel, splat) pairs
                             (alpha >= alpha_min, up to and including the stopping one) into the
                             frame status (ss_frame_status `walked`); 0 leaves that count at 0.
                             The count is the algorithmic work of the roofline; it costs one
                             reduction per warp and is left out of training steps. */
} ss_raster_opts;

/* Per render target I/O (device pointers; row-major [H][W] planes of the
 * target's own size, planar [3][H][W] for 3-channel outputs).  Caller-owned;
 * unused pointers must be NULL.
 *   rgb     corrected colour C A + c (main targets only; NULL = not written)
 *   depth   sum_i w_i z_i, z_i the depth of the ray-splat intersection, not
 *           normalised by alpha (NULL = not written)
 *   normal  sum_i w_i n_i, n_i = R[:,2] flipped to face the sensor (main only)
 *   alpha   1 - T_final (NULL = not written)
 *   T_final, last  saved state for the backward pass (REQUIRED by ss_rasterize_fwd
 *           and ss_rasterize_bwd): final transmittance and the end of the
 *           pixel's walk in the sorted intersection list
 *   d_rgb, d_depth, d_normal, d_alpha  upstream gradients (backward; NULL = 0)
 *   distort  distortion of the blending weights along the pixel's ray, the
 *           point-sample distortion that Supp. B adds to the training loss:
 *           sum over composited pairs j before i of 2 w_i w_j (z_i - z_j), with
 *           w_i the blending weight and z_i the intersection depth; it equals
 *           sum_{i,j} w_i w_j |z_i - z_j| where the compositing order is the order
 *           of z (NULL = not computed; the forward then runs without it)
 *   d_distort  its upstream gradient (backward; NULL = 0).  Requires `depth`:
 *           the adjoint reads the forward's depth plane, which must hold the
 *           values that ss_rasterize_fwd wrote for this frame (SS_ERR_INVALID_ARG
 *           when it is NULL) */
typedef struct {
  float* rgb;
  float* depth;
  float* normal;
  float* alpha;
  float* T_final;
  uint32_t* last;
  const float* d_rgb;
  const float* d_depth;
  const float* d_normal;
  const float* d_alpha;
  float* distort;
  const float* d_distort;
} ss_target_io;

/* Gradients with respect to the splat attributes: FP32 DEVICE arrays [C][n_pad]
 * laid out like ss_splats (quats: w.r.t. the unnormalised input).  Accumulated. */
typedef struct {
  float* means;
  float* scales;
  float* quats;
  float* opacity;
  float* rgb;
  int64_t n_pad;
} ss_splat_grads;

/* Fill `opts` with the defaults listed above.  Never fails. */
void ss_default_opts(ss_raster_opts* opts);

/* Human-readable name of a status code (static storage). */
const char* ss_status_string(ss_status status);

/* Records per staged batch of the forward (ss_rasterize_fwd) and the backward
 * (ss_rasterize_bwd) rasterizer kernels, for reports.  Either pointer may be
 * NULL.  Never fails; host only. */
void ss_staging_batches(int32_t* fwd, int32_t* bwd);

/* Bytes of device workspace a frame needs, for an intersection-list capacity
 * of `capacity` (tile, splat) pairs over all targets.  The workspace holds the
 * assembled cameras, the per-(target, splat) projected records, the
 * visibility order, the sorted intersection lists, per-tile ranges, the
 * per-(target, splat) gradient records and a status block.  Host only.
 * Errors: SS_ERR_INVALID_ARG for bad cameras/options/sizes. */
ss_status ss_workspace_size(const ss_splats* splats, const ss_camera* cams, int32_t n_cams,
                            int32_t passes, const ss_raster_opts* opts, int64_t capacity,
                            size_t* bytes);

/* Camera assembly and per-splat projection (K1), Sec. 3.2-3.3: for every target
 * and splat, F' = F + dF, the sun camera when the target is a sun view, the
 * normalised rotation, M = B R S', det, Q = M^-1, the projected centre, the
 * depth of the centre and its slopes along u and v, the normal flipped toward
 * the sensor, log-opacity, the conservative screen extent and the tile
 * rectangle, and zeroes the frame's gradient records of the visible pairs.
 * Splats with opacity < alpha_min are culled.  The colour correction of a main
 * view (Sec. 3.1 Eq. image_formation) is applied here to the splat colour, since
 * C (sum_i w_i rgb_i) = sum_i w_i (C rgb_i); its offset c is added per pixel by
 * ss_rasterize_fwd.
 *   dF:    DEVICE [n_cams][2][4] fp32 camera deltas, or NULL (zero).
 *   color: DEVICE [n_cams][3][4] fp32 [C | c], or NULL (identity).
 *   ws:    DEVICE workspace of ws_bytes >= ss_workspace_size(..., capacity).
 * Non-finite splat values are counted in the status block (ss_frame_status). */
ss_status ss_project_splats(const ss_splats* splats, const ss_camera* cams, int32_t n_cams,
                            int32_t passes, const float* dF, const float* color,
                            const ss_raster_opts* opts, void* ws, size_t ws_bytes, int64_t capacity,
                            ss_stream_t stream);

/* Tile binning and sorting (K2), Sec. 3.2 rasterization paragraph: one stable
 * radix sort of the splats by height (descending; ties by the smaller index)
 * serves every target, because the depth key is view independent; then every
 * (target, tile, splat) overlap is emitted in that order and stably radix
 * sorted by tile, and per-tile [start, end) ranges are built.
 *   needed: HOST out, may be NULL.  If non-NULL the call synchronises the
 *     stream, stores the number of intersections the frame needs, and returns
 *     SS_ERR_CAPACITY when it exceeds `capacity` (the lists are then
 *     truncated and the frame must be re-run with a larger workspace).  If
 *     NULL nothing is synchronised (CUDA-graph friendly) and an overflow is
 *     reported by ss_frame_status. */
ss_status ss_bin_and_sort(const ss_splats* splats, const ss_camera* cams, int32_t n_cams,
                          int32_t passes, const ss_raster_opts* opts, void* ws, size_t ws_bytes,
                          int64_t capacity, int64_t* needed, ss_stream_t stream);

/* Forward rasterization (K3), Sec. 3.2 Eq. rasterization and Sec. 3.1
 * Eq. image_formation (the C A + c part): per pixel, front to back over the
 * tile's list, alpha = min(alpha_max, o G^), contributing iff >= alpha_min,
 * stop before T would fall below t_min; outputs per ss_target_io; the colour
 * correction given to ss_project_splats completes rgb = C A + c.
 *   io:    HOST array of n_targets ss_target_io (T_final and last required). */
ss_status ss_rasterize_fwd(const ss_splats* splats, const ss_camera* cams, int32_t n_cams,
                           int32_t passes, const ss_raster_opts* opts, const ss_target_io* io,
                           void* ws, size_t ws_bytes, int64_t capacity, ss_stream_t stream);

/* Backward (K4, then K5 unless grads is NULL): the adjoint of ss_rasterize_fwd
 * and ss_project_splats for the same frame.  Per pixel the walk runs in reverse
 * from `last`, recovering the transmittance from T_final (Sec. 3.2
 * Eq. rasterization, differentiated); per-splat partials are summed over each
 * lane's four pixels and reduced across the two lanes of a 2 x 4 sub-block,
 * then added into per-(target, splat) records in the workspace with vector
 * reductions in L2; K5 (ss_project_bwd) chains them through the projection.
 * Call it once per ss_project_splats: the records start from zero there.
 *   grads:   accumulated splat gradients; NULL runs K4 only, and a later
 *            ss_project_bwd for the same frame finishes the backward.
 *   d_dF:    DEVICE [n_cams][2][4] fp32, accumulated, or NULL (used with grads).
 *   d_color: DEVICE [n_cams][3][4] fp32, accumulated, or NULL: gradient of the
 *            colour correction (Eq. image_formation): here d c = sum over pixels of
 *            d(rgb_out); d C = sum g A^T is accumulated by the projection adjoint
 *            (with grads, or ss_project_bwd) as sum_i H_i rgb_i^T, H_i = sum w_i g. */
ss_status ss_rasterize_bwd(const ss_splats* splats, const ss_camera* cams, int32_t n_cams,
                           int32_t passes, const ss_raster_opts* opts, const ss_target_io* io,
                           const ss_splat_grads* grads, float* d_dF, float* d_color, void* ws,
                           size_t ws_bytes, int64_t capacity, ss_stream_t stream);

/* Projection adjoint (K5), Sec. 3.2 Eq. affine2dgs_Qq and Sec. 3.3: chains the
 * per-(target, splat) records left by ss_rasterize_bwd(grads = NULL) through
 * Q = M^-1, M = B' R S', c = B' p + b', the depth row, the normal flip, the
 * quaternion normalisation and, for sun targets, the flattening along s; sums
 * over targets into `grads` (required, accumulated), into d_dF and into the 3x3
 * block C of d_color (both accumulated, or NULL).  d(opacity) is taken through
 * log(opacity). */
ss_status ss_project_bwd(const ss_splats* splats, const ss_camera* cams, int32_t n_cams,
                         int32_t passes, const ss_raster_opts* opts, const ss_splat_grads* grads,
                         float* d_dF, float* d_color, void* ws, size_t ws_bytes, int64_t capacity,
                         ss_stream_t stream);

/* Sun-direction shadow depth (K6), Sec. 3.3 and Supp. A: project, bin and
 * rasterize the sun view of every camera (depth and alpha only).  Equivalent
 * to the three calls above with passes = SS_PASS_SUN.  `io` holds n_cams
 * targets; `needed` as in ss_bin_and_sort. */
ss_status ss_shadow_depth(const ss_splats* splats, const ss_camera* cams, int32_t n_cams,
                          const float* dF, const ss_raster_opts* opts, const ss_target_io* io,
                          void* ws, size_t ws_bytes, int64_t capacity, int64_t* needed,
                          ss_stream_t stream);

/* Sun visibility and image formation (K7), Sec. 3.1 Eq. image_formation with the shadow
 * mapping of Sec. 3.1 and Sec. 3.3.  Per main-view pixel x = (i + 0.5, j + 0.5):
 *   z   = D / alpha                       receiver depth (alpha-normalised rendered depth)
 *   h   = max_alt - z                     its height
 *   u   = S (x - h B' s)                  where the sun ray through the receiver meets the
 *                                         view's sun view (B' = F'[:, 0:3], s the sun
 *                                         direction, S = shadow_scale; Supp. A)
 *   z_o = bilinear sample of D_sun / alpha_sun at u (texel centres at +0.5)
 *   V   = exp(-k max(z - z_o - bias, 0))  exponential shadow-map filter
 *   I   = (C A + c) (V + (1 - V) L_a)     per channel, L_a the view's ambient light
 * A pixel without a surface (alpha < alpha_eps), or whose sample needs a texel outside the sun
 * view or without a surface, is lit (V = 1).  The paper takes the filter from earlier work
 * without its constants: k, bias and alpha_eps are options. */
typedef struct {
  float esm_k;     /* filter sharpness per depth unit [2000] */
  float esm_bias;  /* depth units [0] */
  float alpha_eps; /* a pixel or texel with alpha below this has no surface [1e-3] */
} ss_shade_opts;

/* Per-view planes of the shading (device pointers, row-major, planar [3][H][W] for 3 channels):
 *   rgb, depth, alpha          the main view's rasterize_fwd outputs (C A + c, D, alpha)
 *   sun_depth, sun_alpha       the view's sun view [shadow_h][shadow_w]
 *   image                      forward out: I [3][H][W]
 *   vis                        forward out: V [H][W] (NULL = not written)
 *   d_image                    backward in: dL/dI [3][H][W]
 *   d_rgb, d_depth, d_alpha    backward: ADDED to (the main view's rasterizer upstream)
 *   d_sun_depth, d_sun_alpha   backward: ADDED to (atomically; the sun view's upstream)
 * Any backward output may be NULL (not written). */
typedef struct {
  const float* rgb;
  const float* depth;
  const float* alpha;
  const float* sun_depth;
  const float* sun_alpha;
  float* image;
  float* vis;
  const float* d_image;
  float* d_rgb;
  float* d_depth;
  float* d_alpha;
  float* d_sun_depth;
  float* d_sun_alpha;
} ss_shade_io;

void ss_default_shade_opts(ss_shade_opts* opts);

/* Forward shading of n_cams views (one launch).  cams: HOST array; dF: DEVICE [n_cams][2][4]
 * or NULL; La: DEVICE [n_cams][3]; io: HOST array of n_cams.  Errors: SS_ERR_INVALID_ARG. */
ss_status ss_shade_fwd(const ss_camera* cams, int32_t n_cams, const float* dF, const float* La,
                       const ss_shade_opts* opts, const ss_shade_io* io, ss_stream_t stream);

/* Adjoint of ss_shade_fwd for io[v].d_image: adds into the io planes listed above, into d_La
 * (DEVICE [n_cams][3], accumulated, or NULL) and into d_dF (DEVICE [n_cams][2][4], accumulated,
 * or NULL: the sun position depends on B').  The derivative of V is zero where the filter is
 * clamped at 1. */
ss_status ss_shade_bwd(const ss_camera* cams, int32_t n_cams, const float* dF, const float* La,
                       const ss_shade_opts* opts, const ss_shade_io* io, float* d_La, float* d_dF,
                       ss_stream_t stream);

/* Depth-gradient surface normal (K8), Sec. 3.2 Eq. surface_normal: the world-space normal
 * N = (grad_x p_s x grad_y p_s) / |grad_x p_s x grad_y p_s| of the point map p_s back-projected
 * from a main view's rendered depth, for the normal-consistency regulariser (the rendered
 * normal against N).  Per pixel x = (i + 0.5, j + 0.5):
 *   z = D / alpha, h = max_alt - z, p_s = (X, Y, h) with B'[:, 0:2] (X, Y) = x - b' - B'[:, 2] h
 *   grad_x p_s = p_s(i + 1, j) - p_s(i - 1, j), grad_y p_s = p_s(i, j + 1) - p_s(i, j - 1)
 * N is multiplied by sign(det B'[:, 0:2]) so that flat ground gets (0, 0, 1).  A border pixel, or
 * one whose own or a neighbour's alpha is below alpha_eps, gets N = 0 (and passes no gradient). */
typedef struct {
  const float* depth;    /* the main view's rasterize_fwd depth [H][W] */
  const float* alpha;    /* and alpha [H][W] */
  float* normal;         /* forward out: N [3][H][W] */
  const float* d_normal; /* backward in: dL/dN [3][H][W] */
  float* d_depth;        /* backward: ADDED to (atomically), the view's upstream */
  float* d_alpha;        /* backward: ADDED to (atomically) */
} ss_dnormal_io;

/* cams: HOST array; dF: DEVICE [n_cams][2][4] or NULL; io: HOST array of n_cams.
 * Errors: SS_ERR_INVALID_ARG. */
ss_status ss_depth_normal_fwd(const ss_camera* cams, int32_t n_cams, const float* dF, float alpha_eps,
                              const ss_dnormal_io* io, ss_stream_t stream);

/* Adjoint of ss_depth_normal_fwd for io[v].d_normal: adds into io[v].d_depth / d_alpha (either may
 * be NULL) and into d_dF (DEVICE [n_cams][2][4], accumulated, or NULL). */
ss_status ss_depth_normal_bwd(const ss_camera* cams, int32_t n_cams, const float* dF, float alpha_eps,
                              const ss_dnormal_io* io, float* d_dF, ss_stream_t stream);

/* ---------------------------------------------------------------------------------------
 * Optimiser step (training).  SatSplat trains with Adam at per-group learning rates (Supp. B)
 * and relocates splats with the 3DGS-MCMC strategy under a bounded splat quota (Sec. 3.5,
 * Sec. 4.4); the update rules are those of the cited works (Adam: Kingma and Ba, Algorithm 1;
 * position noise and relocation: Kheradmand et al., 3D Gaussian Splatting as Markov Chain
 * Monte Carlo).  Random numbers come from Philox4x64-10 (Salmon et al., SC'11) with key
 * (seed, 0) and counter (index, step, stream, 0): stream 0 draws the position noise of splat
 * `index`, stream 1 the source of relocation target `index`.
 * --------------------------------------------------------------------------------------- */

/* Raw (pre-activation) splat parameters, and Adam's moments laid out the same way: FP32 DEVICE
 * arrays [C][n_pad], 16-byte aligned, n_pad a multiple of 8:
 *   means [3], log_scales [2] (s = exp(x)), quats [4] (unnormalised),
 *   logit_opacity [1] (o = 1 / (1 + exp(-x))), rgb [3] (identity). */
typedef struct {
  float* means;
  float* log_scales;
  float* quats;
  float* logit_opacity;
  float* rgb;
  int64_t n_pad;
} ss_splat_params;

/* Adam options.  ss_default_adam_opts() fills the defaults in brackets (learning rates of
 * Supp. B; the opacity rate, which it does not list, and eps follow 3D Gaussian splatting). */
typedef struct {
  float lr_means, lr_scales, lr_quats, lr_opacity, lr_rgb; /* [0.075, 0.001, 0.001, 0.05, 0.0025] */
  float beta1, beta2, eps;                                 /* [0.9, 0.999, 1e-15] */
  float noise_lr; /* [5e5] scale of the position noise; 0 = no noise */
  float noise_k;  /* [100] steepness of the noise gate sigmoid(-k (o - t)) */
  float noise_t;  /* [0.005] opacity at which the gate is 1/2 */
  int32_t step;   /* Adam step t >= 1 (bias correction and the noise counter) */
  uint64_t seed;  /* [0] */
} ss_adam_opts;

void ss_default_adam_opts(ss_adam_opts* opts);

/* One fused optimiser step over the splats 0..storage->n-1, in place:
 *   - the rasterizer's gradients `grads` (with respect to the activated values) are chained
 *     through the activations (d log s = s ds, d logit o = o (1 - o) do);
 *   - Adam with bias correction on every raw parameter:
 *       m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
 *       x -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps);
 *   - then the 3DGS-MCMC position noise from the updated parameters:
 *       mu += lr_means noise_lr sigmoid(-k (o - t)) Sigma eta, eta ~ N(0, I) (Box-Muller on
 *       Philox uniforms ((x >> 40) + 0.5) 2^-24), Sigma = R diag(s_u^2, s_v^2, 0) R^T
 *       (a surfel's covariance: the noise stays in its plane);
 *   - the activated values are written to the rasterizer's storage arrays `storage` (fp32
 *     or bf16, rounded to nearest even): its pointers are WRITTEN here.
 * params, exp_avg, exp_avg_sq, grads and storage must share n_pad.  One launch, no
 * workspace.  Errors: SS_ERR_INVALID_ARG (pointers, alignment, n_pad, options). */
ss_status ss_adam_step(const ss_splat_params* params, const ss_splat_params* exp_avg,
                       const ss_splat_params* exp_avg_sq, const ss_splat_grads* grads,
                       const ss_splats* storage, const ss_adam_opts* opts, ss_stream_t stream);

/* Adam (no noise) over a flat FP32 DEVICE array of n values, in place: the per-camera deltas
 * (Supp. B: lr 1e-4) and colour corrections (lr 1e-3).  Uses beta1, beta2, eps and step of
 * `opts`.  Errors: SS_ERR_INVALID_ARG. */
ss_status ss_adam_flat(float* param, float* exp_avg, float* exp_avg_sq, const float* grad, int64_t n,
                       float lr, const ss_adam_opts* opts, ss_stream_t stream);

/* 3DGS-MCMC relocation options.  ss_default_mcmc_opts() fills the defaults in brackets. */
typedef struct {
  float min_opacity; /* [0.005] a splat is dead iff its stored opacity <= min_opacity */
  float growth;      /* [0.05] growth per call: min(cap - n, floor(n growth)) new splats */
  int32_t n_max;     /* [51] largest copy count N in the opacity and scale rule */
  int32_t step;      /* counter word of the draws (e.g. the index of this relocation) */
  uint64_t seed;     /* [0] */
} ss_mcmc_opts;

void ss_default_mcmc_opts(ss_mcmc_opts* opts);

/* Bytes of device workspace ss_mcmc_relocate needs for a budget of `cap` splats.  Host only.
 * Errors: SS_ERR_INVALID_ARG when cap < 1 or cap >= 2^31. */
ss_status ss_mcmc_workspace_size(int64_t cap, size_t* bytes);

/* 3DGS-MCMC relocation and growth, in place, for the splats 0..storage->n-1 (n = the active
 * count) under the budget `cap`:
 *   - dead splats (stored opacity <= min_opacity) and the new slots n..n_after-1,
 *     n_after = n + min(cap - n, floor(n growth)), are the targets, in that order;
 *   - target j takes a live source drawn with probability proportional to opacity: integer
 *     weights floor(o 2^24) of the stored opacities, r = floor(x W / 2^64) for the total W
 *     and the first Philox word x of counter (j, step, 1, 0), and the source is the last splat
 *     whose exclusive prefix sum of weights is <= r (exact integer arithmetic);
 *   - a source drawn c times gets, with N = min(c + 1, n_max), o' = 1 - (1 - o)^(1/N)
 *     (clamped to [min_opacity, 1 - 2^-23]) and s' = s o / sum_{j=1}^{N} (-1)^(j-1) C(N, j)
 *     o'^j / sqrt(j) (the relocation rule, its double sum collapsed), in FP64;
 *   - every target then copies its source's raw parameters, and the moments of the sources
 *     and the targets are zeroed; the storage arrays are rewritten for them.
 * When no splat is alive nothing changes and n_after = n.  params, moments and storage need
 * n_pad >= cap.  SYNCHRONISES the stream once (it reads the dead count and the total weight
 * before sizing the draws).  *n_after (host) receives the new active count.  d_stats, if not
 * NULL, is a DEVICE int64 [2] that receives (dead count, total weight W).
 * Errors: SS_ERR_INVALID_ARG (pointers, sizes, options, workspace), SS_ERR_CUDA. */
ss_status ss_mcmc_relocate(const ss_splat_params* params, const ss_splat_params* exp_avg,
                           const ss_splat_params* exp_avg_sq, const ss_splats* storage, int64_t cap,
                           const ss_mcmc_opts* opts, void* ws, size_t ws_bytes, int64_t* n_after,
                           int64_t* d_stats, ss_stream_t stream);

/* ---------------------------------------------------------------------------------------
 * Geometry-aware initialisation (Sec. 3.4): splat centres sampled from a DSM with probability
 * proportional to the local surface area, oriented by the DSM's local normal, sized by the
 * mean distance to their nearest neighbours.  Runs once, before training.
 * --------------------------------------------------------------------------------------- */

/* A DSM on a north-up grid: pixel (i, j) (column i, row j) is the point
 * (x0 + i gsd, y0 - j gsd, heights[j][i]) in world units.
 *   heights  DEVICE [height_px][width] fp32
 *   rgb      DEVICE [3][height_px][width] fp32 orthophoto colour, or NULL (0.5 grey) */
typedef struct {
  const float* heights;
  const float* rgb;
  int32_t width, height_px;
  float x0, y0, gsd;
} ss_dsm;

typedef struct {
  int32_t knn_k;   /* [3] neighbours of the scale estimate, 1..8 */
  float opacity;   /* [0.1] initial opacity, in (0, 1) */
  uint64_t seed;   /* [0] */
} ss_init_opts;

void ss_default_init_opts(ss_init_opts* opts);

/* Bytes of device workspace ss_dsm_init needs for `n` samples of `dsm`.  Host only.
 * Errors: SS_ERR_INVALID_ARG (sizes: width * height_px < 2^31, n < 2^31, gsd > 0). */
ss_status ss_init_workspace_size(const ss_dsm* dsm, int64_t n, size_t* bytes);

/* Draw out->n initial splats into the storage arrays `out` (fp32 or bf16; WRITTEN):
 *   - per DSM pixel the tangents dx = (gsd, 0, dz_x) and dy = (0, gsd, dz_y), finite
 *     differences toward +x and +y (central inside, one-sided on the border); the area
 *     weight |dx x dy| as the integer w = floor(sqrt(dz_x^2 + dz_y^2 + gsd^2) 2^16 / gsd),
 *     evaluated in fp32 with IEEE operations in that order;
 *   - sample s draws Philox4x64-10 with key (seed, 0) and counter (s, 0, 2, 0): the pixel is
 *     the last one whose exclusive prefix sum of weights is <= floor(x W / 2^64) (W the total),
 *     and the centre is the pixel's point + u dx + v dy with u, v uniform in (-1/2, 1/2);
 *   - the rotation [t_u t_v n]: t_u = dx / |dx|, t_v the Gram-Schmidt residual of dy,
 *     n = t_u x t_v (the DSM normal), as a quaternion (w, x, y, z) with w >= 0;
 *   - scales s_u = s_v = the mean distance to the knn_k nearest other samples (exact, by a
 *     ring search over a uniform grid of cells); opacity = opts->opacity; rgb from the
 *     orthophoto at the pixel.
 * Requires out->n > knn_k.  Errors: SS_ERR_INVALID_ARG, SS_ERR_CUDA. */
ss_status ss_dsm_init(const ss_dsm* dsm, const ss_init_opts* opts, const ss_splats* out, void* ws, size_t ws_bytes,
                      ss_stream_t stream);

/* Status block of a frame's workspace.  SYNCHRONISES the stream.
 *   needed:    intersections the last ss_bin_and_sort needed
 *   nonfinite: splats culled for non-finite values by the last projection
 *   walked:    (pixel, splat) pairs with alpha >= alpha_min that the forward passes since
 *              the last projection walked, the stopping pair included (algorithmic work);
 *              counted only by forward passes run with opts->count_pairs = 1, else 0
 *   flags:     bit 0 = intersection overflow, bit 1 = a bounded wait timed out
 * Any output pointer may be NULL.
 * Returns SS_ERR_CAPACITY / SS_ERR_TIMEOUT / SS_ERR_NONFINITE when set, else SS_OK. */
ss_status ss_frame_status(const void* ws, size_t ws_bytes, int64_t* needed, int64_t* nonfinite,
                          int64_t* walked, int32_t* flags, ss_stream_t stream);

/* Number of SMs of the current device and the library's compiled architecture
 * (e.g. 1030 for sm_103a); a test hook to check the build.  Host only. */
int32_t ss_device_info(int32_t* num_sms, int32_t* arch);

/* Allocation-free forward render of ONE main view (no counterpart in the paper: a
 * deployment aid).  Some callers cannot call cudaMalloc: host applications that
 * reserve their device memory once at start-up (a real-time viewer, an inference
 * service under a fixed memory budget); plug-ins handed a stream but no allocator.
 * This call needs no caller workspace: it runs ss_project_splats, ss_bin_and_sort and
 * ss_rasterize_fwd for `cam` (n_cams = 1, SS_PASS_MAIN) on a static device array of
 * ss_noalloc_scratch_bytes() bytes (64 MiB) inside this library, which every GPU that
 * loads the library holds until the process exits.  It calls no allocating routine.
 *   splats, dF (DEVICE [1][2][4] or NULL), color (DEVICE [1][3][4] or NULL), opts, io
 *     (HOST array of 1 ss_target_io): as for the calls above.
 *   needed: HOST out (may be NULL): intersections the view needed.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress,
 * with that device current); make that first call before any stream capture.  Every
 * call synchronises `stream` once, to read the intersection count.  Do not call it on a
 * device again after a cudaDeviceReset of that device in the same process.  Every call shares the array and
 * keeps the last call's contents (the status block and tile ranges are cleared on each
 * call); calls that overlap on the GPU race on it.
 * Errors: SS_ERR_INVALID_ARG when the splats (or the view's intersection lists) cannot fit
 * the array, or for bad arguments; SS_ERR_CAPACITY when the lists outgrow the capacity
 * left in the array (nothing is rasterized); SS_ERR_CUDA. */
ss_status ss_render_fwd_noalloc(const ss_splats* splats, const ss_camera* cam, const float* dF,
                                const float* color, const ss_raster_opts* opts, const ss_target_io* io,
                                int64_t* needed, ss_stream_t stream);

/* Size in bytes of the static scratch array used by ss_render_fwd_noalloc.  Never fails. */
size_t ss_noalloc_scratch_bytes(void);

/* Number of kernels this library has launched, or recorded into a CUDA graph under
 * stream capture, in this process (a host-side diagnostic counter; the paper has no
 * counterpart).  Host only; never fails. */
int64_t ss_kernel_launches(void);

#ifdef __cplusplus
}
#endif

#endif /* SATSPLAT_H */
