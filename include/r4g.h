/*
 * r4g.h -- C ABI of the GB300 (sm_103a) renderer for 4D-rotor Gaussian splatting
 * (Duan et al., "4D-Rotor Gaussian Splatting", SIGGRAPH 2024, arXiv 2402.03307).
 *
 * The library renders N anisotropic 4D Gaussians at a query time t and
 * differentiates the render:
 *   rotor normalisation F_norm            appendix A.1
 *   rotor -> 4x4 rotation F_map           appendix A.2
 *   Sigma4 = R S S^T R^T                  Sec. 3.2.1 (Eq. 5)
 *   temporal slice (Eq. 7, stable form)   Sec. 3.2.2, appendix A.3
 *   visibility cull lambda (t-mu_t)^2>16  Sec. 3.2.2
 *   EWA projection J V Sigma V^T J^T      Sec. 3.1
 *   SH colour, alpha compositing (Eq. 3)  Sec. 3.1
 * with (tile, depth) 64-bit keys, a bit-exact stable radix sort and a tiled
 * front-to-back blend, all in hand-written CUDA kernels.
 *
 * Conventions shared by every entry point:
 *  - All buffer pointers are DEVICE pointers unless a parameter says "host".
 *    The caller owns every buffer; the library never frees caller memory and
 *    allocates no device memory (a context creates one side stream and two
 *    events at its first render, and CUDA events when stage timing is on).
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Every call only enqueues work on that stream; none synchronises, except
 *    r4g_frame_status, which waits for the stream to read the frame's status.
 *  - Return value: R4G_OK, or an error code for invalid arguments detected on
 *    the host (nothing is enqueued then), or R4G_ECUDA when a launch fails
 *    (r4g_last_error gives the CUDA message). Errors that only the device can
 *    see (key-buffer overflow) are recorded in the frame and returned by
 *    r4g_frame_status.
 *  - Floating point: FP32 arithmetic; BF16 storage is accepted for the scales
 *    and SH coefficients; an FP64 debug mode computes Sigma4 and the slice in
 *    double precision.
 */
#ifndef R4G_H
#define R4G_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum r4g_status {
  R4G_OK = 0,
  R4G_EINVAL = 1,      /* a NULL pointer, a negative or oversize count, a bad enum */
  R4G_ENOMEM = 2,      /* r4g_create could not allocate its status memory */
  R4G_EWORKSPACE = 3,  /* the frame / scratch buffer is smaller than required */
  R4G_ECUDA = 4,       /* a CUDA launch or call failed; see r4g_last_error */
  R4G_ETIMEOUT = 5,    /* a bounded device-side wait gave up (see r4g_frame_status) */
  R4G_EDEVICE = 6,     /* the device reported an inconsistent state */
  R4G_EOVERFLOW = 7    /* the frame's key capacity was too small (see r4g_frame_status) */
} r4g_status;

typedef enum r4g_dtype { R4G_F32 = 0, R4G_BF16 = 1 } r4g_dtype;

/* Flags of r4g_config.flags */
#define R4G_FLAG_FP64_SLICE 0x1u   /* debug: Sigma4, the slice and Sigma3 in FP64 */
#define R4G_FLAG_NO_TEMPORAL_CULL 0x2u  /* keep Gaussians with lambda (t-mu_t)^2 > 16 */
#define R4G_FLAG_COUNT_PAIRS 0x4u  /* measurement: count composited (pixel, Gaussian) pairs
                                     (a slower, instrumented blend; see r4g_frame_stats) */
#define R4G_FLAG_FLOW 0x8u         /* optical-flow render (Sec. 3.2.2 speed V/W): out_rgb
                                     channels 0, 1 receive d(mean2d)/dt in pixels per unit of
                                     t, composited with the colour render's weights over a
                                     zero background; channel 2 is 0. No backward. */

/* Render configuration. tile_w x tile_h in {8x8, 16x16, 16x32}. */
typedef struct r4g_config {
  int32_t tile_w;      /* tile width in pixels (default 16) */
  int32_t tile_h;      /* tile height in pixels (default 16) */
  float bg[3];         /* background colour added with the final transmittance (default 0) */
  int32_t sh_degree;   /* 0..3 SH bands used (default 3) */
  uint32_t flags;      /* R4G_FLAG_* */
} r4g_config;

/* N Gaussians, one row each, all device pointers, row-major, densely packed.
 * mean [n,4] = (x, y, z, t); rotor [n,8] = (s, b01, b02, b12, b03, b13, b23, p)
 * (raw: normalised inside the render, appendix A.1); logscale [n,4] = log of
 * (s_x, s_y, s_z, s_t) stored as float or bf16 per scale_dtype; logit [n]
 * (opacity = sigmoid(logit)); sh [n,16,3] SH coefficients [coefficient][rgb]
 * stored as float or bf16 per sh_dtype. mean, rotor and logscale rows must be
 * 16-byte aligned (8-byte for bf16 logscale). */
typedef struct r4g_gaussians {
  const float* mean;
  const float* rotor;
  const void* logscale;
  const float* logit;
  const void* sh;
  int64_t n;
  int32_t scale_dtype; /* r4g_dtype */
  int32_t sh_dtype;    /* r4g_dtype */
} r4g_gaussians;

/* Pinhole camera, host struct passed by pointer. world_to_cam is the row-major
 * 3x4 [R | t] (OpenCV axes: x right, y down, z forward); pixel (i, j) samples
 * the image-plane point (i + 0.5, j + 0.5); u = fx x/z + cx, v = fy y/z + cy. */
typedef struct r4g_camera {
  float world_to_cam[12];
  float fx, fy, cx, cy;
  int32_t width, height;
} r4g_camera;

/* Parameter gradients (device pointers, FP32, same shapes as r4g_gaussians,
 * 16-byte aligned rows). The backward ADDS into them, so several views can
 * accumulate one step; the caller zeroes them.
 *
 * The last three members are optional (NULL = not kept) per-Gaussian
 * statistics of adaptive density control (Sec. 4.2: densification by the
 * view-space positional gradient, as in 3D Gaussian Splatting), each device
 * float [n], updated by r4g_render_backward and r4g_render_batch_backward
 * once per view in which the Gaussian was composited into at least one
 * pixel:
 *   vs_grad    += | (dL/du * W/2, dL/dv * H/2) |, the norm of the gradient
 *                 of the loss with respect to the projected centre (u, v) in
 *                 normalised device coordinates (pixels / (W/2, H/2)) for a
 *                 W x H view; only the blend's direct dependence on (u, v)
 *                 counts (not the conic's);
 *   vs_count   += 1;
 *   max_radius  = max(max_radius, 3 sqrt(lambda_max(Sigma'))) in pixels,
 *                 Sigma' the dilated 2D covariance.
 * r4g_regularizers ignores them. */
typedef struct r4g_grads {
  float* mean;
  float* rotor;
  float* logscale;
  float* logit;
  float* sh;
  float* vs_grad;
  float* vs_count;
  float* max_radius;
} r4g_grads;

/* One (camera, t) view of a batched call. */
typedef struct r4g_view {
  r4g_camera cam;
  float t;
} r4g_view;

/* ---- context -------------------------------------------------------------- */
typedef struct r4g_ctx r4g_ctx;

/* Create a context holding a copy of `cfg` (NULL = defaults: 16x16 tiles,
 * black background, degree 3, no flags). The context is not thread-safe;
 * use one per host thread. Returns R4G_EINVAL for an unsupported tile shape.
 * Its first render creates a side stream and two events on the device then
 * current (the tile counts run there beside the depth sort); later renders
 * on another device return R4G_EINVAL: use one context per device.
 * r4g_destroy releases them. */
r4g_status r4g_create(r4g_ctx** out, const r4g_config* cfg);
void r4g_destroy(r4g_ctx* ctx);
/* Message of the last error on this context (static storage, never NULL). */
const char* r4g_last_error(const r4g_ctx* ctx);
/* Library version as major*10000 + minor*100 + patch. */
int32_t r4g_version(void);

/* ---- frame state ------------------------------------------------------------
 * A frame is one caller-allocated device buffer holding everything a render
 * writes for its backward: per-Gaussian screen records, the sorted (tile,
 * depth) keys and Gaussian indices, per-tile ranges, per-pixel final
 * transmittance and last-contributor position, plus the sort's scratch.
 * key_capacity bounds the number of (tile, Gaussian) pairs; a render whose
 * pairs exceed it marks the frame R4G_EOVERFLOW (the image is then invalid)
 * and records the count it needed (r4g_frame_status). */
r4g_status r4g_frame_bytes(const r4g_ctx* ctx, int64_t n, int32_t width, int32_t height,
                           int64_t key_capacity, size_t* bytes /* host out */);

/* Wait for `stream`, then report the frame's device-side status: R4G_OK,
 * R4G_EOVERFLOW, R4G_ETIMEOUT when a radix-sort look-back wait reached its
 * iteration limit, or R4G_EDEVICE when device views (r4g_render_batch) had
 * other image sizes than the host views (the image of that render is then
 * invalid). *keys_needed (host, may be NULL) receives the number of (tile,
 * Gaussian) pairs of the last render into this frame. */
r4g_status r4g_frame_status(r4g_ctx* ctx, const void* frame, size_t frame_bytes,
                            int64_t* keys_needed, void* stream);

/* The same status without waiting: enqueues on `stream` a copy of the
 * frame's three status words into host_out (HOST memory, uint32 [3]; pinned
 * memory makes the copy asynchronous). Once the stream has passed that point
 * (an event, a synchronisation), r4g_frame_status_decode turns the words into
 * the r4g_frame_status result and *keys_needed (may be NULL). Lets a training
 * step check a render's key capacity without stalling the stream. */
r4g_status r4g_frame_status_async(const void* frame, size_t frame_bytes, uint32_t* host_out, void* stream);
r4g_status r4g_frame_status_decode(const uint32_t* words /* host [3] */, int64_t* keys_needed);

/* Statistics of the last render into a frame (waits for `stream`). */
typedef struct r4g_frame_info {
  int64_t n_visible;         /* (view, Gaussian) items with at least one tile */
  int64_t key_count;         /* (tile, Gaussian) pairs in the sorted list */
  int64_t key_needed;        /* pairs the render needed (> key_count after an overflow) */
  int64_t composited_pairs;  /* (pixel, Gaussian) pairs composited; -1 unless the context
                                has R4G_FLAG_COUNT_PAIRS */
  int32_t status;            /* R4G_OK, R4G_EOVERFLOW, R4G_ETIMEOUT or R4G_EDEVICE */
  int32_t reserved;
  int64_t reached_pairs;     /* (tile, Gaussian) pairs that got a gradient slot in the last
                                backward on this frame (a pixel of the tile composited them) */
  int64_t visible_gaussians; /* Gaussians visible in at least one view of the call */
} r4g_frame_info;
r4g_status r4g_frame_stats(r4g_ctx* ctx, const void* frame, size_t frame_bytes, r4g_frame_info* out,
                           void* stream);

/* Copy out of a frame (device -> device, enqueued on `stream`): the key count
 * (uint32 [1]), the sorted 64-bit keys and 32-bit values (first key_count
 * entries, key = tile_id << 32 | float_bits(depth)), per-tile ranges
 * (uint32 [tiles][2], [begin, end)), and the per-Gaussian screen records
 * (float [n][12] = mean2d.x, mean2d.y, conic a, b, c, opacity_t, depth,
 * log2(255 opacity_t), r, g, b, max(log2 opacity_t, -126); conic is the inverse 2D covariance, exponent
 * -1/2 (a dx^2 + 2 b dx dy + c dy^2); culled Gaussians have opacity_t = 0).
 * Any output pointer may be NULL. For tests and tools. */
r4g_status r4g_frame_export(r4g_ctx* ctx, const void* frame, size_t frame_bytes, int64_t n,
                            int32_t width, int32_t height,
                            uint32_t* key_count, uint64_t* keys, uint32_t* values,
                            uint32_t* ranges, float* records, void* stream);

/* ---- render -----------------------------------------------------------------
 * Forward render of `g` seen by `cam` at time `t` (Sec. 3.2.2 and Sec. 3.1):
 * out_rgb [3, height, width] (planar FP32), and, when not NULL,
 * out_T [height, width] (final transmittance) and out_last [height, width]
 * (1 + position in the tile's sorted list of the last composited Gaussian,
 * 0 when none). The frame must be at least r4g_frame_bytes(n, width, height,
 * key_capacity) bytes. An image may have at most 51,200 tiles (e.g. 3840x2160
 * with 16x16 tiles); larger ones return R4G_EINVAL. */
r4g_status r4g_render(r4g_ctx* ctx, const r4g_gaussians* g, const r4g_camera* cam, float t,
                      float* out_rgb, float* out_T, uint32_t* out_last,
                      void* frame, size_t frame_bytes, int64_t key_capacity, void* stream);

/* Backward of r4g_render for the same (g, cam, t) and the frame it filled:
 * given dL/d out_rgb (grad_rgb [3, height, width]) ADD dL/d parameters into
 * `grads`. Transmittance is recovered back to front from the stored final T,
 * no per-layer state is kept. Gradients through inactive branches (clamped
 * alpha, negative colour, the Jacobian clamp, culled Gaussians) are zero.
 * A frame whose key buffer overflowed adds nothing (its image was invalid;
 * r4g_frame_status reports it). Deterministic: the same inputs add the same
 * bits (no floating-point atomics). */
r4g_status r4g_render_backward(r4g_ctx* ctx, const r4g_gaussians* g, const r4g_camera* cam,
                               float t, const float* grad_rgb, r4g_grads* grads,
                               void* frame, size_t frame_bytes, int64_t key_capacity,
                               void* stream);

/* ---- batched views ------------------------------------------------------------
 * The training of the paper (Sec. 4.2 implementation details; the batch
 * training ablation of Sec. 4.5) renders several (camera, t) views of the
 * same Gaussians per step.
 * A batched call renders V = nviews views (1..64, of any sizes) in one launch
 * sequence: the view-independent work of a Gaussian (rotor, R, Sigma4) is
 * done once, every per-item stage runs over all V x N (view, Gaussian) items,
 * the tile ids of all views form one list sorted once, and the blend is one
 * persistent launch over the tiles of every view. Each view's image is
 * bit-identical to r4g_render of that view.
 *
 * Packed images: out_rgb (and grad_rgb) hold the views one after another,
 * view v as [3, height_v, width_v] planar FP32 starting at float offset
 * 3 * sum_{u<v} width_u height_u; out_T (NULL or [sum width_v height_v])
 * likewise. `views` is a HOST array (sizes and, when views_dev is NULL, the
 * cameras and times). `views_dev`, when not NULL, is a DEVICE array of nviews
 * r4g_view read by the kernels for the cameras and times, so a captured CUDA
 * graph can be replayed with new cameras written there; its image sizes must
 * equal the host views' (else the frame reports R4G_EDEVICE). No call
 * allocates, synchronises or copies from host memory: a render and its
 * backward can be captured in a CUDA graph (with stage timing off). */
r4g_status r4g_batch_frame_bytes(const r4g_ctx* ctx, int64_t n, const r4g_view* views, int32_t nviews,
                                 int64_t key_capacity, int32_t tile_w, int32_t tile_h,
                                 size_t* bytes /* host out */);
/* tile_w = tile_h = 0 in r4g_batch_frame_bytes means the context's tile shape. */
r4g_status r4g_render_batch(r4g_ctx* ctx, const r4g_gaussians* g, const r4g_view* views, int32_t nviews,
                            const r4g_view* views_dev, float* out_rgb, float* out_T, void* frame,
                            size_t frame_bytes, int64_t key_capacity, void* stream);
/* Backward of r4g_render_batch (same g, views and frame): adds into `grads`
 * the gradient of L given dL/d out_rgb (packed like out_rgb), summed over the
 * views. The cameras are those the render used (kept in the frame). */
r4g_status r4g_render_batch_backward(r4g_ctx* ctx, const r4g_gaussians* g, const r4g_view* views,
                                     int32_t nviews, const float* grad_rgb, r4g_grads* grads, void* frame,
                                     size_t frame_bytes, int64_t key_capacity, void* stream);

/* Tile-shape autotuner. Times r4g_render_batch (and, when grad_rgb is not
 * NULL, r4g_render_batch_backward into `grads`, which it changes) for the
 * tile shapes 8x8, 16x16 and 16x32: one warm-up call and `reps` timed calls
 * each, CUDA events on `stream`. A shape whose frame does not fit
 * frame_bytes, whose views exceed the tile limit, or whose render overflows
 * key_capacity is skipped (ms < 0). The fastest shape is set on the context
 * and returned. The images do not depend on the tile shape (the per-pixel 3
 * sigma test, Sec. 3.1). Synchronises the stream; not for graph capture. */
typedef struct r4g_tune_result {
  int32_t tile_w, tile_h;  /* the chosen shape */
  float ms[3];             /* mean ms per call for 8x8, 16x16, 16x32 (< 0: skipped) */
  int64_t keys_needed[3];  /* (tile, Gaussian) pairs of each shape (-1: not run) */
} r4g_tune_result;
r4g_status r4g_autotune_batch(r4g_ctx* ctx, const r4g_gaussians* g, const r4g_view* views, int32_t nviews,
                              float* out_rgb, const float* grad_rgb, r4g_grads* grads, void* frame,
                              size_t frame_bytes, int64_t key_capacity, int32_t reps, void* stream,
                              r4g_tune_result* out /* host */);
/* Change the context's tile shape (8x8, 16x16 or 16x32); frames sized for
 * another shape must be re-queried. */
r4g_status r4g_set_tile(r4g_ctx* ctx, int32_t tile_w, int32_t tile_h);
/* The context's current configuration (host out). */
r4g_status r4g_get_config(const r4g_ctx* ctx, r4g_config* out);

/* ---- measurement ------------------------------------------------------------
 * Stage timing: when enabled on a context, r4g_render / r4g_render_backward
 * record a CUDA event pair around each stage on the call's stream; the times
 * are accumulated when r4g_stage_times collects them (it waits for those
 * events). Launch counts are kept whether or not timing is on. */
typedef enum r4g_stage {
  R4G_STAGE_PREPROCESS = 0,   /* per-Gaussian preprocess kernel */
  R4G_STAGE_BINNING = 1,      /* block-total scan + key emission */
  R4G_STAGE_SORT = 2,         /* radix sort passes */
  R4G_STAGE_RANGES = 3,       /* tile ranges */
  R4G_STAGE_BLEND = 4,        /* forward blend */
  R4G_STAGE_BLEND_BWD = 5,    /* backward blend */
  R4G_STAGE_PREPROCESS_BWD = 6,
  R4G_NSTAGES = 7
} r4g_stage;

r4g_status r4g_set_timing(r4g_ctx* ctx, int32_t enable);
/* ms[R4G_NSTAGES] and launches[R4G_NSTAGES] (host, either may be NULL)
 * receive the accumulated stage times and kernel launch counts since the
 * last reset; reset != 0 clears them afterwards. */
r4g_status r4g_stage_times(r4g_ctx* ctx, double* ms, int64_t* launches, int32_t reset);

/* ---- regularisers (Sec. 3.3) -----------------------------------------------------
 * 4D K-nearest neighbours of the Gaussian means (Sec. 3.3 "4D Consistency
 * Loss"): Euclidean distance after dividing x, y, z by scale_xyz and t by
 * scale_t (the spatial and temporal scene scales). means: device [n, 4]
 * (16-byte aligned). out_idx: device int32 [n, k], the neighbours of each
 * point in increasing distance, ties to the smaller index, the point itself
 * excluded; out_dist2 (device float [n, k] or NULL): their squared scaled
 * distances. k in {4, 8, 16}, k < n <= 2^28. Exact (a grid search that stops
 * only when no unsearched cell can hold a closer point). scratch: device,
 * 256-byte aligned, r4g_knn_scratch_bytes(n) bytes. Deterministic. */
r4g_status r4g_knn_scratch_bytes(int64_t n, size_t* bytes /* host out */);
r4g_status r4g_knn4d(const float* means, int64_t n, float scale_xyz, float scale_t, int32_t k,
                     int32_t* out_idx, float* out_dist2, void* scratch, size_t scratch_bytes,
                     void* stream);
/* Waits for `stream`; R4G_ETIMEOUT if the last r4g_knn4d in `scratch` had a
 * radix-sort look-back wait reach its iteration limit (its result is then
 * invalid), else R4G_OK. */
r4g_status r4g_knn_status(const void* scratch, int64_t n, void* stream);

/* The entropy loss L_e = 1/N sum -o log o (o = sigmoid(logit)) and the 4D
 * consistency loss L_c = 1/N sum_i || s_i - 1/k sum_{j in knn_idx[i]} s_j ||_1
 * on the speeds s = V / W of Sigma4 (Sec. 3.2.2), for k-nearest-neighbour
 * lists knn_idx (device int32 [n, k], as r4g_knn4d writes them; an index
 * outside [0, n) counts as the point itself). out_loss (device float [2])
 * receives (L_e, L_c), unweighted. When `grads` is not NULL, ADDS
 * lambda_entropy dL_e/dlogit into grads->logit and lambda_consistency dL_c/d
 * (rotor, log-scale) into grads->rotor and grads->logscale (the neighbour
 * lists are constants). mean and sh are not used. scratch: device, 256-byte
 * aligned, r4g_regularizers_scratch_bytes(n) bytes. Deterministic. */
r4g_status r4g_regularizers_scratch_bytes(int64_t n, size_t* bytes /* host out */);
r4g_status r4g_regularizers(const r4g_gaussians* g, const int32_t* knn_idx, int32_t k,
                            float lambda_entropy, float lambda_consistency, float* out_loss,
                            r4g_grads* grads, void* scratch, size_t scratch_bytes, void* stream);

/* The image loss of the optimisation (Sec. 3.3 total loss, as in 3D Gaussian
 * Splatting): L = (1 - lambda_ssim) L1 + lambda_ssim (1 - SSIM) between a
 * rendered image and a target (device float [channels, height, width],
 * planar), L1 = mean |x - y|, SSIM the mean structural similarity over an
 * 11 x 11 Gaussian window (sigma 1.5, zero padding, C1 = 0.01^2,
 * C2 = 0.03^2). out_loss (device float [3]) receives (L, L1, SSIM);
 * grad_image (device, like the image, or NULL) receives dL/d image
 * (written, not added). scratch: device, 256-byte aligned,
 * r4g_image_loss_scratch_bytes bytes. Deterministic. */
r4g_status r4g_image_loss_scratch_bytes(int32_t channels, int32_t height, int32_t width,
                                        size_t* bytes /* host out */);
r4g_status r4g_image_loss(const float* image, const float* target, int32_t channels, int32_t height,
                          int32_t width, float lambda_ssim, float* out_loss, float* grad_image,
                          void* scratch, size_t scratch_bytes, void* stream);

/* ---- adaptive density control (Sec. 4.2 "CUDA Acceleration" and training
 * details: duplication and pruning of the 4D Gaussians on the GPU, with the
 * densification gradient threshold and the 3D Gaussian Splatting rules) ----
 * One densify-and-prune step over n Gaussians in two calls, from the
 * statistics the backward kept (r4g_grads.vs_grad / vs_count / max_radius):
 *
 *   densify  Gaussian i when vs_grad[i] >= grad_threshold * vs_count[i] and
 *            vs_count[i] > 0 (its mean view-space gradient reaches the
 *            threshold; decided exactly, in double precision);
 *   clone    a densified Gaussian whose largest spatial scale
 *            max(exp(logscale[i][0..2])) <= dense_scale: it is kept and an
 *            identical copy follows it;
 *   split    a densified Gaussian with a larger spatial scale: it is replaced
 *            by two children drawn from its own 4D distribution,
 *            mean_c = mean + R diag(s) z_c (R the rotation of the normalised
 *            rotor, s = exp(logscale), z_c = z[i][c][0..3] standard normal,
 *            c = 0, 1), log-scales logscale - ln(split_divisor) on all four
 *            axes, the same rotor, logit and SH;
 *   prune    every output row whose opacity sigmoid(logit) < min_opacity; if
 *            max_scale > 0, every row whose largest spatial scale exceeds
 *            max_scale; if max_screen_radius > 0 and max_radius is given,
 *            every row continuing a Gaussian (not a new copy or child) whose
 *            max_radius exceeds max_screen_radius.
 *
 * Output order: for i = 0..n-1, the surviving rows of Gaussian i (kept: i;
 * clone: i, then its copy; split: child 0, child 1). out_src[j] receives, for
 * output row j, i when the row continues Gaussian i (its optimiser state
 * carries over) and -(i + 1) when it is new (a copy or a child). All
 * parameters are FP32 (scale_dtype = sh_dtype = R4G_F32). */
typedef struct r4g_densify_config {
  float grad_threshold;     /* view-space gradient threshold (2e-4 Plenoptic, 5e-5 D-NeRF) */
  float dense_scale;        /* clone / split boundary on the largest spatial scale
                               (3D Gaussian Splatting: 0.01 x scene extent) */
  float split_divisor;      /* children's scale divisor (1.6); > 1 */
  float min_opacity;        /* prune below this opacity (0.005); in [0, 1) */
  float max_scale;          /* prune above this spatial scale; 0 = off */
  float max_screen_radius;  /* prune above this radius in pixels; 0 = off */
} r4g_densify_config;

/* Output parameter buffers (device, FP32, rows like r4g_gaussians, 16-byte
 * aligned), capacity rows each. */
typedef struct r4g_params_out {
  float* mean;
  float* rotor;
  float* logscale;
  float* logit;
  float* sh;
} r4g_params_out;

/* scratch of the two calls: device, 256-byte aligned, r4g_densify_scratch_bytes(n). */
r4g_status r4g_densify_scratch_bytes(int64_t n, size_t* bytes /* host out */);

/* Plan: decide every Gaussian's outputs from g (logit, logscale), vs_grad,
 * vs_count and (optional, NULL allowed) max_radius (device float [n]) and
 * write into scratch the per-Gaussian decisions and output offsets;
 * *out_count (device int64 [1]) receives the number of output rows.
 * n <= 2^28. Deterministic. */
r4g_status r4g_densify_plan(const r4g_gaussians* g, const float* vs_grad, const float* vs_count,
                            const float* max_radius, const r4g_densify_config* cfg, void* scratch,
                            size_t scratch_bytes, int64_t* out_count, void* stream);

/* Apply: write the output rows planned into `scratch` by r4g_densify_plan for
 * the same g and cfg. z: device float [n, 2, 4] standard normal draws (read
 * only for split Gaussians). Rows j >= capacity are not written: allocate
 * capacity >= *out_count (2 n always suffices). out and g must not overlap.
 * out_src: device int32 [capacity] or NULL. */
r4g_status r4g_densify_apply(const r4g_gaussians* g, const float* z, const r4g_densify_config* cfg,
                             const void* scratch, size_t scratch_bytes, r4g_params_out* out,
                             int64_t capacity, int32_t* out_src, void* stream);

/* Opacity reset of the training schedule (every 3,000 steps in Sec. 4.2's
 * settings, as in 3D Gaussian Splatting): logit[i] = min(logit[i],
 * logit(max_opacity)), logit(p) = ln(p / (1 - p)) rounded to FP32 once on
 * the host. max_opacity in (0, 1) (0.01). logit: device float [n]. */
r4g_status r4g_opacity_reset(float* logit, int64_t n, float max_opacity, void* stream);

/* ---- sort -------------------------------------------------------------------
 * Stable LSD radix sort of (uint64 key, uint32 value) pairs on key bits
 * [begin_bit, end_bit), 0 <= begin_bit < end_bit <= 64 (the key-sort step of
 * the tile rasteriser, Sec. 3.1). keys_in/values_in are read only; results go
 * to keys_out/values_out (which must not alias the inputs). scratch must hold
 * r4g_sort_scratch_bytes(n) bytes. Bit-exact and deterministic. */
r4g_status r4g_sort_scratch_bytes(int64_t n, size_t* bytes /* host out */);
r4g_status r4g_sort_pairs(const uint64_t* keys_in, const uint32_t* values_in,
                          uint64_t* keys_out, uint32_t* values_out, int64_t n,
                          int32_t begin_bit, int32_t end_bit,
                          void* scratch, size_t scratch_bytes, void* stream);

/* ---- the render's own sort ----------------------------------------------------
 * Stable LSD radix sort of (uint32 key, uint32 value) pairs on key bits
 * [0, bits), 1 <= bits <= 32, in 8-bit passes of one kernel each with a
 * decoupled look-back between 2048-item tiles: the kernels that sort the
 * render's depth keys and tile ids (the key-sort step of the tile rasteriser,
 * Sec. 3.1), as an entry point of their own. values_in may be NULL (then the
 * values are the input positions 0..n-1). keys_out/values_out must not alias
 * the inputs; n < 2^30. scratch (device, 256-byte aligned) must hold
 * r4g_sort32_scratch_bytes(n, bits) bytes; its first word is the call's
 * status, which r4g_sort32_status reads (it synchronises the stream):
 * R4G_ETIMEOUT there means a look-back wait gave up after its iteration
 * limit and the result is invalid. Bit-exact and deterministic. */
r4g_status r4g_sort32_scratch_bytes(int64_t n, int32_t bits, size_t* bytes /* host out */);
r4g_status r4g_sort32(const uint32_t* keys_in, const uint32_t* values_in, uint32_t* keys_out,
                      uint32_t* values_out, int64_t n, int32_t bits, void* scratch,
                      size_t scratch_bytes, void* stream);
r4g_status r4g_sort32_status(const void* scratch, void* stream);
/* Test hook of the failure path of the look-back wait: as r4g_sort32, but the
 * tile whose ticket is withheld_tile never publishes its counts, and every
 * wait gives up after spin_limit (1..65536) rounds without progress instead
 * of 2^22. The call then completes with R4G_ETIMEOUT in its status word and
 * an invalid result; nothing hangs or faults, and the next call on the same
 * scratch is unaffected. */
r4g_status r4g_sort32_wait_test(const uint32_t* keys_in, const uint32_t* values_in,
                                uint32_t* keys_out, uint32_t* values_out, int64_t n, int32_t bits,
                                void* scratch, size_t scratch_bytes, void* stream,
                                uint32_t withheld_tile, uint32_t spin_limit);

/* ---- sort without allocation -------------------------------------------------
 * The paper has no counterpart to this entry point; it serves callers that
 * cannot allocate device memory and therefore cannot pass the scratch buffer
 * r4g_sort_pairs needs (a plug-in inside a host application that owns the GPU
 * memory budget, a real-time loop that must not call an allocator). Same
 * result as r4g_sort_pairs, bit for bit, for n <= R4G_SORT_NOALLOC_MAX_PAIRS;
 * larger n returns R4G_EINVAL with nothing enqueued. It allocates nothing:
 * its scratch is one file-scope device array of R4G_SORT_NOALLOC_SCRATCH_BYTES
 * bytes that each GPU loading the library holds until the process exits.
 * All calls on a device share that array and it keeps the last call's
 * contents, so calls that may overlap on the GPU (unordered streams) race and
 * corrupt each other; order them on one stream or with events. The first call
 * on each device looks up the array's device address with that device current
 * and caches it; make that first call before starting any stream capture. The
 * cached address belongs to the device's primary context: after
 * cudaDeviceReset (or any teardown of that context) it is stale, so do not
 * call this entry point again in a process that has reset the device.
 * Error messages are returned by r4g_last_error(NULL). */
#define R4G_SORT_NOALLOC_MAX_PAIRS 1048576
#define R4G_SORT_NOALLOC_SCRATCH_BYTES 12894208
r4g_status r4g_sort_pairs_noalloc(const uint64_t* keys_in, const uint32_t* values_in,
                                  uint64_t* keys_out, uint32_t* values_out, int64_t n,
                                  int32_t begin_bit, int32_t end_bit, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* R4G_H */
