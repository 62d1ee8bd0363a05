/*
 * gsr.h -- C ABI of the GB300-native differentiable 3D-Gaussian rasterizer
 * of Gaussian-SLAM (arXiv 2312.10070).
 *
 * Plain C: pointers, sizes and small POD structs.  No CUDA or PyTorch type
 * appears in a signature; a CUDA stream is passed as `void *` (a
 * cudaStream_t, NULL = the legacy default stream).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - All arrays are CALLER-OWNED DEVICE memory of the current CUDA device,
 *    float32 (int32 where stated), contiguous, in the layouts stated below.
 *    Images are planar: rgb [3,H,W], single-channel maps [H,W], row major.
 *  - Gaussian parameters are structure-of-arrays (Sec. 3.1): mean [n,3],
 *    log_scale [n,3] (s = exp(log_scale)), quat [n,4] (w,x,y,z, normalised
 *    inside), opacity_logit [n] (o = sigmoid), rgb [n,3] (colour used
 *    directly, no spherical harmonics, Sec. 3.2 "Sub-map Optimization").
 *  - A pose is world-to-camera, T_wc = (R(q), t); the camera frame is x right,
 *    y down, z forward; pixel (i, j) has its centre at (i + 0.5, j + 0.5).
 *  - Pose gradients are 6-vectors d_pose6 = dL/dxi for the left perturbation
 *    T_wc(xi) = exp(xi^) T_wc, xi = (rho, phi), translation first.
 *  - Work is enqueued asynchronously on `stream`; only the calls documented
 *    as synchronising wait for the GPU.
 *  - Errors: every call returns a gsr_status; no exception or longjmp
 *    crosses the ABI.  gsr_last_error() gives a message for the last failure
 *    on a context.  Asynchronous device-side conditions (capacity overflow
 *    in fixed-capacity mode, non-finite losses) are latched in a device
 *    status word and returned by the next synchronising call.
 *  - The context owns all scratch memory (tile lists, sort buffers, per-pixel
 *    state is caller-owned).  Scratch grows on demand unless the context was
 *    created with fixed_capacity = 1.  A context is not thread safe; use one
 *    per host thread / stream.
 */
#ifndef GSR_H
#define GSR_H

#include <stdint.h>

#if defined(__GNUC__)
#define GSR_API __attribute__((visibility("default")))
#else
#define GSR_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GSR_OK = 0,
    GSR_ERR_INVALID_ARG = -1, /* a pointer, size or option is invalid */
    GSR_ERR_CUDA = -2,        /* a CUDA runtime call failed */
    GSR_ERR_OOM = -3,         /* device allocation failed */
    GSR_ERR_CAPACITY = -4,    /* fixed-capacity scratch was too small (results invalid) */
    GSR_ERR_TIMEOUT = -5,     /* a bounded device wait expired */
    GSR_ERR_NONFINITE = -6,   /* a loss became NaN or Inf */
    GSR_ERR_STATE = -7        /* call order violated (e.g. backward without a forward) */
} gsr_status;

typedef struct gsr_ctx gsr_ctx;

/* Rasterizer options fixed at context creation. */
typedef struct {
    int32_t tile_w, tile_h;  /* pixel tile: 16x16 (default), 8x8, 16x8 or 32x8 */
    int32_t batch;           /* Gaussians staged in shared memory per batch: 32, 64, 128, 256 */
    int32_t memory_saving;   /* 1: render_backward re-projects and re-bins instead of reusing
                                the tile lists saved by the last forward */
    int32_t fixed_capacity;  /* 1: never synchronise to grow scratch (CUDA-graph safe); an
                                overflow latches GSR_ERR_CAPACITY */
    int64_t max_gaussians;   /* initial scratch capacities (0 = grow on first use) */
    int64_t max_instances;   /* tile instances (Gaussian x tile pairs) */
    int64_t max_pixels;
    int32_t ppt_fwd, ppt_bwd;  /* pixels each forward / backward blend thread owns: 1 or 2
                                  (0 = defaults 1 and 2); results do not depend on them */
    int32_t rect_lists;        /* 0 (default): a tile's list holds the Gaussians whose rectangle
                                  covers it AND that may composite at one of its pixel centres
                                  (minimum of sigma over the tile's pixel-centre box below the
                                  skip threshold, with the float32 error margin); 1: every
                                  Gaussian whose rectangle covers the tile (Sec. 3.1's tiling as
                                  the prior art defines it).  Images, n_contrib and gradients are
                                  the same either way; last_idx indexes the list in use. */
} gsr_options;

/* Pinhole camera and rasterizer constants. */
typedef struct {
    int32_t width, height;
    float fx, fy, cx, cy;
    float z_near;  /* Gaussians with camera z <= z_near are culled (default 0.2 m) */
    float eps2d;   /* low-pass dilation added to the 2D covariance, px^2 (default 0.3) */
} gsr_camera;

typedef struct {
    float q[4]; /* world-to-camera rotation quaternion (w, x, y, z) */
    float t[3]; /* world-to-camera translation */
} gsr_pose;

typedef struct {
    const float *mean, *log_scale, *quat, *opacity_logit, *rgb;
    int64_t n;
} gsr_gaussians;

/* Gradient outputs, same layouts as gsr_gaussians; any pointer may be NULL. */
typedef struct {
    float *mean, *log_scale, *quat, *opacity_logit, *rgb;
} gsr_gaussian_grads;

/* Forward outputs / saved state.  rgb [3,H,W], depth [H,W] (camera z, not
 * normalised by alpha), alpha [H,W] = 1 - final_T, final_T [H,W],
 * last_idx [H,W] (position in the pixel's tile list of the last composited
 * Gaussian, -1 if none).  n_contrib [H,W] may be NULL. */
typedef struct {
    float *rgb, *depth, *alpha, *final_T;
    int32_t *last_idx, *n_contrib;
} gsr_render_out;

/* Counters of the last forward on a context (read back synchronously). */
typedef struct {
    int64_t n_visible;    /* V: Gaussians that survived culling */
    int64_t n_instances;  /* I: Gaussian x tile pairs */
    int64_t n_tiles;
    int64_t capacity_instances;
} gsr_frame_stats;

/* ------------------------------------------------------------- context */

/* Fills `opt` with the defaults (16x16 tiles, batch 256, grow on demand). */
GSR_API void gsr_default_options(gsr_options *opt);
/* Fills `cam` with z_near 0.2 and eps2d 0.3 and the given intrinsics. */
GSR_API void gsr_default_camera(gsr_camera *cam, int32_t width, int32_t height, float fx, float fy,
                        float cx, float cy);
/* Creates a context on the current CUDA device.  *out is NULL on failure. */
GSR_API gsr_status gsr_create(gsr_ctx **out, const gsr_options *opt);
/* Releases the context and its scratch (synchronises the device). */
GSR_API void gsr_destroy(gsr_ctx *ctx);
/* Message of the last failed call on `ctx` (never NULL; "" if none). */
GSR_API const char *gsr_last_error(const gsr_ctx *ctx);
/* Human-readable name of a status code. */
GSR_API const char *gsr_status_string(gsr_status s);
/* Number of CUDA kernels this context has launched so far. */
GSR_API int64_t gsr_kernel_launches(const gsr_ctx *ctx);

/* Profiling: when enabled, each call records CUDA events around its phases
 * (also inside captured graphs).  gsr_profile_read synchronises `stream` and
 * writes the elapsed milliseconds of the latest execution of each phase to
 * ms[0..n): 0 projection + binning, 1 blend forward, 2 fused loss, 3 blend
 * backward, 4 projection backward (+ pose reduction), 5 Adam; -1 if the phase
 * has not run since profiling was enabled.  For a multi-keyframe map_step the
 * per-keyframe phases report the last keyframe. */
GSR_API gsr_status gsr_profile_enable(gsr_ctx *ctx, int32_t on);
GSR_API gsr_status gsr_profile_read(gsr_ctx *ctx, float *ms, int32_t n, void *stream);

/* ------------------------------------------------------------ renderer */

/* Differentiable render (Sec. 3.1 colour blending Eq. (color_blending),
 * alpha_j = o_j exp(-sigma_j), the EWA covariance J R Sigma R^T J^T, and the
 * depth rendering D = sum mu^z alpha T of Sec. 3.4).  Writes `out`.
 * The tile lists it builds stay in the context until its next forward and are
 * reused by render_backward (unless memory_saving).  In grow-on-demand mode
 * it synchronises once to size the instance buffers. */
GSR_API gsr_status gsr_render_forward(gsr_ctx *ctx, const gsr_gaussians *g, const gsr_camera *cam,
                              const gsr_pose *pose, gsr_render_out *out, void *stream);

/* Counters of the last forward (synchronises `stream`).  Also returns, and
 * clears, a device-side condition latched since the last synchronising call
 * (GSR_ERR_CAPACITY: a fixed-capacity forward had more tile instances than
 * room, so its lists were truncated; GSR_ERR_NONFINITE; GSR_ERR_TIMEOUT);
 * `st` is filled in either case. */
GSR_API gsr_status gsr_frame_stats_get(gsr_ctx *ctx, gsr_frame_stats *st, void *stream);

/* Failure-detection check (the paper has no counterpart).  Runs, in one warp,
 * the bounded wait that the radix sort's decoupled look-back uses, on a word
 * of the context's counter block that no kernel publishes, so the wait gives
 * up after `polls` polls (1 .. 1000000: microseconds to about a second),
 * latches GSR_ERR_TIMEOUT in the context's status word and the kernel
 * returns.  The call synchronises `stream` and returns the latched status
 * (GSR_ERR_TIMEOUT, or an earlier latched condition first), clearing it, so
 * the context stays usable.  It exercises the error path of a wait that
 * expires without faulting or hanging the GPU.  GSR_ERR_INVALID_ARG for a
 * NULL context or `polls` out of range (no launch). */
GSR_API gsr_status gsr_check_wait_timeout(gsr_ctx *ctx, int32_t polls, void *stream);

/* Copies the tile lists of the last forward to HOST memory (synchronises;
 * for tests and debugging).  ranges: host uint32[2 * n_tiles] = [start, end)
 * per tile into `gids`; gids: host int32[capacity] = Gaussian index of each
 * list entry, tiles in row-major order, each list in depth order; depth_bits:
 * host uint32[n] (NULL = skip) = float bits of each Gaussian's camera depth
 * (0xffffffff if culled).  *n_instances receives the list length; if it
 * exceeds `capacity` nothing is copied into gids and GSR_ERR_CAPACITY is
 * returned. */
GSR_API gsr_status gsr_tile_lists_get(gsr_ctx *ctx, uint32_t *ranges, int32_t *gids, int64_t capacity,
                                      uint32_t *depth_bits, int64_t *n_instances, void *stream);

/* Copies the per-Gaussian image-space records of the last forward to HOST
 * memory (synchronises; for tests and debugging).  rec: host float[12 n] =
 * per Gaussian (u, v, conic a, conic b, conic c, opacity, camera depth,
 * bits of the first tile column/row, r, g, b, bits of the last tile
 * column/row) -- the projection of Sec. 3.1 (mean, inverse of the EWA
 * covariance Sigma^I, activated opacity) as the blend kernels read it;
 * visible: host uint32[n], 1 where the Gaussian survived culling (records of
 * culled Gaussians are unspecified).  n must equal the last forward's count.
 * GSR_ERR_STATE without a forward. */
GSR_API gsr_status gsr_records_get(gsr_ctx *ctx, float *rec, uint32_t *visible, int64_t n, void *stream);

/* Backward of gsr_render_forward (Sec. 3.4 adjoints, including the depth
 * adjoint dD/dalpha_j = mu^z_j T_j - sum_{u>j} mu^z_u alpha_u T_u /(1-alpha_j)).
 * `saved` must hold the final_T and last_idx of the matching forward.
 * d_rgb [3,H,W], d_depth [H,W], d_alpha [H,W] are dL/d(outputs); any may be
 * NULL (= zero).  `dg` (gradients overwritten, NULL = none wanted; NULL
 * members are skipped) and `d_pose6` (device float[6], overwritten, NULL =
 * none) receive the gradients.  With memory_saving, or if another forward ran
 * on the context since, the tile lists are rebuilt from `g` and `pose`. */
GSR_API gsr_status gsr_render_backward(gsr_ctx *ctx, const gsr_gaussians *g, const gsr_camera *cam,
                               const gsr_pose *pose, const gsr_render_out *saved,
                               const float *d_rgb, const float *d_depth, const float *d_alpha,
                               gsr_gaussian_grads *dg, float *d_pose6, void *stream);

/* Twist-perturbed render and its backward (Sec. 3.5: tracking optimises the
 * camera pose by gradient descent; here the pose is perturbed on the left by a
 * twist held in DEVICE memory, so an autograd graph over the twist needs no
 * host round trip).  gsr_render_forward_xi renders at the float pose
 * fl(exp(xi^) T), exp formed in double precision on the device from
 * xi = (rho, phi) (device float[6], caller-owned; T = *pose).
 * gsr_render_backward_xi returns the parameter gradients of that render and,
 * in d_xi (device float[6], overwritten, NULL = none), dL/dxi =
 * J_l(xi)^T g, where g is the left-perturbation pose gradient at exp(xi^) T
 * and J_l the SE(3) left Jacobian (exp((xi + e)^) = exp((J_l e)^) exp(xi^)
 * to first order).  xi must hold the same values in the backward as in the
 * matching forward.  Otherwise as gsr_render_forward / gsr_render_backward;
 * GSR_ERR_INVALID_ARG for a NULL xi. */
GSR_API gsr_status gsr_render_forward_xi(gsr_ctx *ctx, const gsr_gaussians *g, const gsr_camera *cam,
                                         const gsr_pose *pose, const float *xi, gsr_render_out *out, void *stream);
GSR_API gsr_status gsr_render_backward_xi(gsr_ctx *ctx, const gsr_gaussians *g, const gsr_camera *cam,
                                          const gsr_pose *pose, const float *xi, const gsr_render_out *saved,
                                          const float *d_rgb, const float *d_depth, const float *d_alpha,
                                          gsr_gaussian_grads *dg, float *d_xi, void *stream);

/* Left retraction of a pose by a device twist (Sec. 3.5's pose update as the
 * tracker applies it): pose_out (device float[7]) = (q', t') of
 * fl(exp(xi^) T), q' normalised with w >= 0, formed in double precision on
 * the device; xi = (rho, phi) device float[6].  Stream-ordered, no context,
 * no allocation.  GSR_ERR_INVALID_ARG on NULL arguments, GSR_ERR_CUDA if the
 * launch fails. */
GSR_API gsr_status gsr_pose_retract(const gsr_pose *pose, const float *xi, float *pose_out, void *stream);

/* -------------------------------------------------------------- losses */

/* Mapping loss, Eq. (joint_loss) without L_reg (Sec. 3.4):
 *   L = w_color [(1-lambda) mean|I^-I| + lambda (1 - SSIM(I^, I))] + w_depth mean_valid|D^-D|
 * SSIM: 11x11 Gaussian window (sigma 1.5), zero padding, C1 = 0.01^2,
 * C2 = 0.03^2, mean over pixels and channels; valid = target depth > 0.
 * Writes d_rgb [3,H,W], d_depth [H,W] (overwritten, scaled by `scale`) and
 * the scalar loss * scale to loss_dev (device float, overwritten; NULL = skip). */
GSR_API gsr_status gsr_loss_map(gsr_ctx *ctx, int32_t width, int32_t height, const float *rgb,
                        const float *depth, const float *rgb_target, const float *depth_target,
                        float lambda_ssim, float w_color, float w_depth, float scale,
                        float *d_rgb, float *d_depth, float *loss_dev, void *stream);

/* Tracking loss (Sec. 3.5 and supplementary Sec. B):
 *   L = sum_p M_inlier M_alpha (lambda_c sum_ch |I^-I| + (1-lambda_c)|D^-D|)
 * M_alpha = alpha^alpha_pow (no gradient through it), M_inlier = valid &
 * |D^-D| <= k_median * (lower median of |D^-D| over valid pixels), found by an
 * exact radix select.  Writes d_rgb, d_depth (overwritten), loss to loss_dev
 * and the median to median_dev (device floats; NULL = skip). */
GSR_API gsr_status gsr_loss_track(gsr_ctx *ctx, int32_t width, int32_t height, const float *rgb,
                          const float *depth, const float *alpha, const float *rgb_target,
                          const float *depth_target, float lambda_c, float k_median,
                          float alpha_pow, float *d_rgb, float *d_depth, float *loss_dev,
                          float *median_dev, void *stream);

/* Largest image (width * height) gsr_loss_track_noalloc accepts: 1280 x 720. */
#define GSR_NOALLOC_MAX_PIXELS 921600

/* Allocation-free variant of gsr_loss_track (the paper has no counterpart;
 * it is an interface for callers).  Some callers cannot call cudaMalloc: code
 * that runs inside another framework's memory pool with a fixed budget, or a
 * real-time tracking loop that must not meet cudaMalloc's implicit device
 * synchronisation.  They cannot create a gsr_ctx (whose scratch is
 * allocated), so this call needs no context and allocates nothing.  Inputs,
 * outputs, scale and the result are those of gsr_loss_track.
 *
 * Its scratch (about 3.7 MB) is one static device array in libgsr.so, held
 * by every GPU that loads the library until the process exits.  Each call
 * looks up that array's device address in the current CUDA context (no
 * allocation; the first call in a context also loads the library's module
 * there, so the first call on each device should come before any stream
 * capture).  Every call on a device shares the array, which keeps the last
 * call's contents (the call clears what must start at zero): calls that
 * overlap on the GPU (different streams, or host threads) race and must be
 * serialised by the caller.
 *
 * Errors: GSR_ERR_INVALID_ARG for a null pointer or a non-positive size,
 * GSR_ERR_CAPACITY when width * height > GSR_NOALLOC_MAX_PIXELS (nothing is
 * launched), GSR_ERR_CUDA if the address lookup or one of this call's
 * launches fails (an error left pending by earlier work is cleared first, not
 * reported).  The call never synchronises, so unlike gsr_loss_track (whose
 * context latches it for the next synchronising call) it does NOT report a
 * non-finite loss as GSR_ERR_NONFINITE: check the value written to loss_dev,
 * which is then NaN or Inf. */
GSR_API gsr_status gsr_loss_track_noalloc(int32_t width, int32_t height, const float *rgb, const float *depth,
                                          const float *alpha, const float *rgb_target, const float *depth_target,
                                          float lambda_c, float k_median, float alpha_pow, float *d_rgb,
                                          float *d_depth, float *loss_dev, float *median_dev, void *stream);

/* ------------------------------------------------------------ optimiser */

typedef struct {
    float lr_mean, lr_log_scale, lr_quat, lr_opacity, lr_rgb;
    float beta1, beta2, eps;
    float w_reg;  /* weight of the isotropic regulariser L_reg (Sec. 3.4) */
} gsr_adam_opts;

/* Adam moments (device, same SoA layout as the parameters) + step counter. */
typedef struct {
    float *m_mean, *m_log_scale, *m_quat, *m_opacity_logit, *m_rgb;
    float *v_mean, *v_log_scale, *v_quat, *v_opacity_logit, *v_rgb;
    int32_t *step;  /* device int32, incremented on the device by each update */
} gsr_adam_state;

typedef struct {
    float *mean, *log_scale, *quat, *opacity_logit, *rgb;
    int64_t n;
} gsr_gaussians_mut;

/* One bias-corrected Adam step on every Gaussian parameter with gradients
 * `grads`, adding w_reg * dL_reg/dlog_scale of the isotropic regulariser
 * L_reg = (1/n) sum_k |s_k - mean(s_k)|_1 (Sec. 3.4).  If loss_reg_dev is not
 * NULL, w_reg * L_reg is ADDED to it. */
GSR_API gsr_status gsr_adam_step(gsr_ctx *ctx, gsr_gaussians_mut *g, const gsr_gaussian_grads *grads,
                         gsr_adam_state *st, const gsr_adam_opts *opt, float *loss_reg_dev,
                         void *stream);

/* ------------------------------------------------------------- tracking */

typedef struct {
    float lambda_c;     /* colour weight inside L_tracking (0.5) */
    float k_median;     /* inlier threshold factor (50) */
    float alpha_pow;    /* M_alpha = alpha^alpha_pow (3) */
    float lr_rho, lr_phi;
    float beta1, beta2, eps;
    int32_t use_graph;  /* 1: capture one iteration in a CUDA graph and replay it */
} gsr_track_opts;

typedef struct {
    float loss_first, loss_last;  /* L_tracking at the first and the last iteration */
    int32_t iters;
} gsr_track_stats;

/* Frame-to-model tracking (Sec. 3.5): n_iters iterations of render ->
 * L_tracking -> pose-only backward -> Adam on the twist -> left retraction
 * T <- exp(delta^) T, all on the device with the Gaussians frozen.  rgb_in
 * [3,H,W] and depth_in [H,W] are the frame (device).  *pose_inout is the
 * initial pose (e.g. the constant-velocity guess) and receives the result.
 * Synchronising. */
GSR_API gsr_status gsr_track_step(gsr_ctx *ctx, const gsr_gaussians *g, const gsr_camera *cam,
                          const float *rgb_in, const float *depth_in, gsr_pose *pose_inout,
                          int32_t n_iters, const gsr_track_opts *opt, gsr_track_stats *out,
                          void *stream);

/* ------------------------------------------------------------- mapping */

typedef struct {
    gsr_pose pose;
    const float *rgb;    /* [3,H,W] device */
    const float *depth;  /* [H,W] device, 0 = invalid */
} gsr_keyframe;

typedef struct {
    float lambda_ssim, w_color, w_depth;
    gsr_adam_opts adam;
    int32_t use_graph;   /* 1: capture one iteration in a CUDA graph and replay it */
} gsr_map_opts;

typedef struct {
    float loss_last;  /* weighted mapping loss (+ w_reg L_reg) of the last iteration */
    int32_t iters;
} gsr_map_stats;

/* Sub-map optimisation (Sec. 3.2 "Sub-map Optimization", Eq. (joint_loss)):
 * n_iters iterations of: render every keyframe, fused mapping loss weighted
 * by kf_weights[k] (host array, NULL = uniform 1/n_kf), back-propagate all
 * keyframes into one gradient, Adam with L_reg.  The keyframes are rendered
 * and back-propagated by one batched forward and one batched backward launch
 * over (keyframe, tile) work items.  Updates g and st in place.
 * `out` may be NULL; when given, the call synchronises to fill it. */
GSR_API gsr_status gsr_map_step(gsr_ctx *ctx, gsr_gaussians_mut *g, gsr_adam_state *st,
                        const gsr_camera *cam, const gsr_keyframe *kfs, int32_t n_kf,
                        const float *kf_weights, int32_t n_iters, const gsr_map_opts *opt,
                        gsr_map_stats *out, void *stream);

/* Stream-ordered read of the mapping loss of Eq. (joint_loss), Sec. 3.2/3.4
 * (no synchronisation): enqueues on
 * `stream` a copy of the weighted loss (+ w_reg L_reg) of the last iteration
 * of the last gsr_map_step on this context into *loss_dev (caller-owned
 * device float), so a caller can read every step's loss back without
 * stalling the next step.  Call it on the stream of that gsr_map_step
 * (before any map step it copies 0).  GSR_ERR_INVALID_ARG on NULL arguments. */
GSR_API gsr_status gsr_map_loss(gsr_ctx *ctx, float *loss_dev, void *stream);

/* ------------------------------------------------------------ autotune */

typedef struct {
    int32_t tile_w, tile_h, batch, ppt_fwd, ppt_bwd;
    float ms_fwd, ms_bwd;  /* mean time of the forwards / backwards over all given poses */
    float ms;              /* ms_fwd + ms_bwd */
} gsr_tune_result;

/* Launch-configuration autotuner (no counterpart in the paper: tile shape,
 * Gaussians per shared-memory batch and pixels per thread are parameters of
 * this implementation of Sec. 3.1's tile-based rasterisation).
 * Times gsr_render_forward and gsr_render_backward (all gradients, dL/dpixel
 * = 1) of `g` at each of the n_poses poses for every tile shape {16x16, 8x8,
 * 16x8, 32x8} x batch {32, 64, 128, 256}, each with 1 and 2 pixels per thread
 * for the forward and for the backward (`reps` timed repetitions after one
 * warm-up), and keeps the fastest combination on the context (its captured
 * graphs are dropped).  The tile shape
 * changes which Gaussians a tile lists (the rectangle rule is per tile), so a
 * context's results are reproducible for a fixed configuration; batch and
 * pixels per thread do not change results.  *best receives the winner; all
 * (nullable, n_all entries) the timings in the order tried.  Synchronising;
 * the Gaussians are not modified. */
GSR_API gsr_status gsr_autotune(gsr_ctx *ctx, const gsr_gaussians *g, const gsr_camera *cam, const gsr_pose *poses,
                                int32_t n_poses, int32_t reps, gsr_tune_result *best, gsr_tune_result *all,
                                int32_t n_all, void *stream);

/* ------------------------------------------------------------- seeding */

/* Sub-map seeding (Sec. 3.2 densification; Sec. 4 and supplementary Sec. A
 * for the constants).  A keyframe adds Gaussians to the active sub-map:
 *   1. candidate pixels (valid depth > 0 only): on the first keyframe of a
 *      sub-map (first_keyframe = 1) m_u pixels drawn uniformly without
 *      replacement plus the m_c pixels of largest squared luminance gradient;
 *      on later keyframes m_k pixels drawn uniformly among those whose
 *      rendered alpha is below alpha_n.  "Drawn uniformly" = the pixels with
 *      the smallest key (splitmix64(seed + pixel index) >> 32, ties by index);
 *      the gradient is the central difference of Y = (R + G + B) / 3
 *      (0 on the image border), ties by pixel index;
 *   2. back-projection with the keyframe pose: p_c = ((x - cx) z / fx,
 *      (y - cy) z / fy, z) at the pixel centre (x, y) = (j + 0.5, i + 0.5),
 *      p_w = R^T (p_c - t);
 *   3. a candidate is kept when no existing Gaussian mean lies at squared
 *      distance < rho^2 (a hashed grid of cell size rho, 27 cells per query);
 *   4. every kept point becomes a Gaussian appended after the n_existing ones:
 *      mean p_w, opacity logit 0 (opacity 0.5), the pixel's RGB, identity
 *      rotation, all three log-scales = log of its nearest-neighbour distance
 *      among all n_existing + n_added means (exact, by a ring search on a
 *      hashed grid), clamped to [s_min, s_max]. */
typedef struct {
    int32_t first_keyframe; /* 1: m_u uniform + m_c gradient; 0: m_k uniform where alpha < alpha_n */
    int64_t m_u, m_c, m_k;  /* sample sizes (100000, 50000, 100000) */
    float alpha_n;          /* 0.6 */
    float rho;              /* search radius, m (0.01) */
    float s_min, s_max;     /* scale clamp, m (1e-4, 0.1) */
    uint64_t seed;          /* sampling key seed */
} gsr_seed_opts;

typedef struct {
    int64_t n_candidates; /* candidate pixels after sampling */
    int64_t n_added;      /* Gaussians appended */
} gsr_seed_stats;

GSR_API void gsr_default_seed_opts(gsr_seed_opts *o);

/* rgb [3,H,W], depth [H,W] (0 = invalid) and alpha [H,W] (the sub-map's
 * render at this pose; may be NULL when first_keyframe = 1) are device
 * arrays of the keyframe; pose is world-to-camera.  `g` holds the sub-map in
 * arrays of `capacity` Gaussians, the first n_existing in use (g->n is
 * ignored); new Gaussians are written at [n_existing, n_existing + n_added).
 * GSR_ERR_CAPACITY (nothing written) when they do not fit.  Synchronising
 * (the count is read back once). */
GSR_API gsr_status gsr_seed_keyframe(gsr_ctx *ctx, const gsr_camera *cam, const gsr_pose *pose, const float *rgb,
                                     const float *depth, const float *alpha, const gsr_seed_opts *opt,
                                     gsr_gaussians_mut *g, int64_t n_existing, int64_t capacity,
                                     gsr_seed_stats *out, void *stream);

/* The last gsr_seed_keyframe's candidates (ascending pixel index): pixel
 * index, kept flag (1/0) and the squared distance to the nearest existing
 * mean within the 27 searched cells (+inf if none).  Device arrays of
 * `capacity` entries; *n receives the count (nothing is copied when it
 * exceeds capacity: GSR_ERR_CAPACITY).  Synchronising. */
GSR_API gsr_status gsr_seed_candidates_get(gsr_ctx *ctx, int32_t *pix, int32_t *keep, float *d2, int64_t capacity,
                                           int64_t *n, void *stream);

/* Pruning (supplementary Sec. A: Gaussians whose opacity falls below o_thre
 * are removed at the middle and the end of a new keyframe's mapping).  Keeps
 * the Gaussians with sigmoid(opacity_logit) >= min_opacity (tested as
 * logit >= log(t / (1 - t)) in float32), compacting g's arrays -- and st's
 * moments when st is not NULL -- in place, in their original order; entries
 * past the kept count are left unspecified.  g->n is the count in use;
 * *n_kept receives the new count (synchronising). */
GSR_API gsr_status gsr_prune(gsr_ctx *ctx, gsr_gaussians_mut *g, gsr_adam_state *st, float min_opacity,
                             int64_t *n_kept, void *stream);

/* Global map merge (supplementary Sec. A: the saved sub-maps are merged in
 * sequence, each Gaussian added with the seeding rule).  Appends to `global`
 * (arrays of `capacity`, the first n_global in use) the Gaussians of `sub`
 * whose mean has no global mean at squared distance < rho^2, in their
 * order, copying every parameter; other Gaussians of `sub` do not reject each
 * other.  GSR_ERR_CAPACITY (nothing written) when they do not fit.
 * *n_added receives the count (synchronising). */
GSR_API gsr_status gsr_merge_submap(gsr_ctx *ctx, gsr_gaussians_mut *global, int64_t n_global, int64_t capacity,
                                    const gsr_gaussians *sub, float rho, int64_t *n_added, void *stream);

/* Throughput probes (no counterpart in the paper): the measured denominators
 * of the ALU rooflines of the blend kernels.  gsr_probe_fma launches `blocks`
 * blocks of 256 threads; each thread runs `iters` rounds of 8 independent
 * FP32 fused multiply-adds (16 FLOP per round), so one launch performs
 * blocks * 256 * iters * 16 FLOP.  gsr_probe_exp does the same with 8
 * independent base-2 exponentials (ex2.approx) per round: blocks * 256 *
 * iters * 8 exponentials.  out: caller-owned device float[blocks * 256]
 * (a sink so the work cannot be elided; its values are meaningless).
 * iters must be a positive multiple of 32.  Asynchronous on `stream`; time
 * them with events on that stream.  GSR_ERR_INVALID_ARG on bad sizes,
 * GSR_ERR_CUDA if the launch fails. */
GSR_API gsr_status gsr_probe_fma(float *out, int32_t blocks, int32_t iters, void *stream);
GSR_API gsr_status gsr_probe_exp(float *out, int32_t blocks, int32_t iters, void *stream);
/* y[i] = the single-precision exponential the blend kernels use for
 * alpha = o exp(-sigma), at x[i] (device float[n] each), so a test can check
 * its error against the bound the parity margins assume.
 * GSR_ERR_INVALID_ARG on NULL or n <= 0. */
GSR_API gsr_status gsr_probe_expf(const float *x, float *y, int64_t n, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* GSR_H */
