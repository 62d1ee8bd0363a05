// gsr_internal.cuh -- internal declarations of the GB300 (sm_103a) rasterizer.
// Not part of the ABI; the public interface is include/gsr.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/gsr.h"

typedef uint32_t u32;

// ----------------------------------------------------------------- constants
// Blend decisions (the same constants in forward and backward).
#define GSR_ALPHA_MIN (1.0f / 255.0f)
#define GSR_ALPHA_MAX 0.99f
#define GSR_T_STOP 1e-4f
#define GSR_GUARD 1.3f

// Device status word bits.
#define GSR_FLAG_CAPACITY 1u
#define GSR_FLAG_NONFINITE 2u
#define GSR_FLAG_TIMEOUT 4u

// Counters block layout (u32 words in ctx->counters).
enum {
    CNT_VISIBLE = 0,   // V of the current view
    CNT_INSTANCES = 1, // I (before clamping to capacity)
    CNT_SORTN = 2,     // min(I, capacity): instances actually sorted
    CNT_STATUS = 3,    // sticky status bits
    CNT_NVALID = 4,    // valid target depth pixels of the last mapping loss
    CNT_TRACK_N = 5,   // valid pixels of the tracking loss
    CNT_SEL = 6,       // radix-select state: [6] prefix bits, [7] remaining rank
    CNT_WORDS = 16
};

// --------------------------------------------------------------- scratch
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

// Per-view scratch of the projection/binning/blend pipeline.
struct ViewScratch {
    DevBuf rec;         // float4 x3 per Gaussian id: (u,v,ca,cb) (cc,o,z,rect_lo) (r,g,b,rect_hi)
    DevBuf flag;        // u32 per Gaussian id: 1 = visible
    DevBuf compact;     // u32 per Gaussian id: exclusive scan of flag
    DevBuf rank_of_gid; // int32 per Gaussian id: depth rank, -1 = culled
    DevBuf dkeys[2];    // u32 depth keys (ping-pong)
    DevBuf dvals[2];    // u32 Gaussian ids
    DevBuf rec_sorted;  // float4 x3 per depth rank
    DevBuf tcount;      // u32 kept tile instances per depth rank
    DevBuf inst_off;    // u32 exclusive scan of tcount
    DevBuf tkeys[2];    // u32 tile id per instance
    DevBuf tvals[2];    // u32 depth rank per instance
    DevBuf ranges;      // uint2 per tile
    DevBuf order;       // u32 per tile: tile ids by list length, longest first (blend launch order)
    DevBuf order_hist;  // u32 per length bucket and block of the launch-order sort
    DevBuf g2d;         // float x12 per rank: image-space gradients
    DevBuf counters;    // u32[CNT_WORDS]
    DevBuf pose;        // float[8]: q(4), t(3)
    DevBuf scan_tmp;    // block sums of this view's scans
    DevBuf radix_hist;  // digit histograms and look-back of this view's sorts
    DevBuf loss_maps;   // SSIM adjoint maps of this view's mapping loss (batched mapping)
    DevBuf loss_part;   // per-block partial sums of this view's mapping loss
    int64_t cap_n = 0, cap_i = 0, cap_t = 0;
    bool culled = false;  // the lists hold only entries that pass the tile test
    bool g2d_zero = false;  // g2d was zeroed by the last binning and no backward has added to it since
    bool order_valid = false;  // order holds the launch order of the last binning
    // identity of the last forward, to decide whether the saved lists are valid
    uint64_t generation = 0;
};

// Pointers one blend kernel needs for one view.
struct BlendView {
    const uint2 *ranges;
    const u32 *tvals;
    const float4 *rec;
    float *rgb, *depth, *alpha, *final_T;
    int32_t *last_idx, *n_contrib;
    const float *d_rgb, *d_depth, *d_alpha;
    float *g2d;
    const u32 *order;  // the tile of block b is order[b] (nullptr: b)
    int culled;    // 1: every list entry passed the tile test when the lists were built
    int reserved;  // explicit padding (descriptors are compared bytewise)
};
// per-keyframe inputs of the multi-keyframe projection backward
struct ProjView {
    const int32_t *rank_of_gid;
    const float *g2d;
    const float *pose;
};
// Scratch of keyframe seeding (csrc/seed.cu).
struct SeedScratch {
    DevBuf flag, sel, off;     // u32 per pixel: eligible, selected, exclusive scans
    DevBuf keys[2], vals[2];   // u32 sort pairs (pixels, then grid cells)
    DevBuf cnt;                // u32 counters: eligible, candidates, kept
    DevBuf cand_pix, cand_pts; // per candidate: pixel index, world point (float4)
    DevBuf keep, keep_off, d2; // per candidate: kept flag, its scan, squared distance to the sub-map
    DevBuf new_cand;           // per kept point: candidate index
    DevBuf prune_tmp;          // packed rows of the Gaussians kept by gsr_prune
};

struct gsr_ctx {
    gsr_options opt;
    int ppt_fwd = 1, ppt_bwd = 2;  // pixels per thread of the blend kernels
    int device = 0;
    std::string err;
    int64_t launches = 0;
    uint64_t generation = 0;
    ViewScratch view;
    // generic scratch
    DevBuf scan_tmp;     // block sums of device scans
    DevBuf radix_hist;   // per-block digit histograms
    DevBuf pose_part;    // per-block pose partial sums
    DevBuf loss_part;    // per-block loss partial sums
    DevBuf loss_maps;    // SSIM adjoint maps [9,H,W] / tracking residual
    DevBuf img_tmp;      // images of iterative loops
    DevBuf small;        // misc device scalars (losses, Adam state of the pose)
    DevBuf grads;        // gradients of map_step [n,14]
    // forward identity
    const float *fwd_ptrs[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    int64_t fwd_n = -1;
    gsr_camera fwd_cam{};
    gsr_pose fwd_pose{};
    const float *fwd_xi = nullptr;  // device twist of the last forward (nullptr: none)
    // graphs
    cudaGraphExec_t track_graph = nullptr;
    uint64_t track_key = 0;
    cudaGraphExec_t map_graph = nullptr;
    uint64_t map_key = 0, map_sized_key = 0;
    int64_t track_graph_kernels = 0, map_graph_kernels = 0;
    // per-phase CUDA events (profiling mode)
    bool prof = false;
    cudaEvent_t prof_ev[2 * 8] = {};
    u32 *host_pinned = nullptr; // small pinned readback buffer
    // batched multi-keyframe mapping: per-keyframe scratch and frames
    std::vector<ViewScratch> mv;
    DevBuf mv_frames, mv_desc, mv_pview, mv_items, mv_order_hist, mv_counter;
    // side streams of the batched binning (one chain of binning kernels per
    // keyframe runs on each; forked from and joined to the caller's stream)
    static constexpr int N_SIDE = 8;
    cudaStream_t side[N_SIDE] = {};
    cudaEvent_t fork_ev = nullptr, join_ev[N_SIDE] = {};
    std::vector<BlendView> mv_desc_host;
    std::vector<ProjView> mv_pview_host;
    SeedScratch seed;
    int64_t seed_last_candidates = 0;
};

// -------------------------------------------------------------- host helpers
gsr_status gsr_fail(gsr_ctx *ctx, gsr_status s, const std::string &msg);
gsr_status gsr_cuda_check(gsr_ctx *ctx, cudaError_t e, const char *what);
gsr_status ensure_buf(gsr_ctx *ctx, DevBuf &b, size_t bytes);
void free_buf(DevBuf &b);

#define GSR_TRY(expr)                          \
    do {                                       \
        gsr_status _s = (expr);                \
        if (_s != GSR_OK) return _s;           \
    } while (0)
#define GSR_CUDA(ctx, expr) GSR_TRY(gsr_cuda_check((ctx), (expr), #expr))
#define GSR_LAUNCHED(ctx) GSR_TRY(gsr_cuda_check((ctx), cudaGetLastError(), "kernel launch"))

static inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// --------------------------------------------------------- scan / radix sort
// Device-wide exclusive scan of u32.  The element count is min(*d_n, n_cap)
// when d_n is given, else n_cap.  The total is written to *d_total (nullable).
// tmp: the block-sum scratch (nullptr: the context's).
gsr_status scan_exclusive(gsr_ctx *ctx, const u32 *in, u32 *out, int64_t n_cap, const u32 *d_n,
                          u32 *d_total, cudaStream_t s, DevBuf *tmp = nullptr);
// Stable LSD radix sort of (key, value) pairs on key bits [0, bits), 8 bits
// per pass.  The element count is read on the device from *d_n (<= n_cap).
// The sorted pairs end in keys[0]/vals[0].
// hist: the histogram / look-back scratch (nullptr: the context's).
gsr_status radix_sort_pairs(gsr_ctx *ctx, u32 *keys[2], u32 *vals[2], int64_t n_cap, const u32 *d_n,
                            int bits, cudaStream_t s, DevBuf *hist = nullptr);

// Grows the tile-instance capacity of V (and the sort scratch sized from it).
gsr_status grow_instance_capacity(gsr_ctx *ctx, ViewScratch &V, int64_t c);

// ------------------------------------------------------------ device math
struct CamK {
    int W, H, tw, th, tiles_x, tiles_y;
    float fx, fy, cx, cy, z_near, eps2d, limx, limy;
    float inv_tw;  // 1 / tw, exact: tile widths are powers of two
};

CamK make_camk(const gsr_camera &c, int tw, int th);

__device__ __forceinline__ void quat_rot(float qw, float qx, float qy, float qz, float R[9])
{
    R[0] = 1.f - 2.f * (qy * qy + qz * qz);
    R[1] = 2.f * (qx * qy - qw * qz);
    R[2] = 2.f * (qx * qz + qw * qy);
    R[3] = 2.f * (qx * qy + qw * qz);
    R[4] = 1.f - 2.f * (qx * qx + qz * qz);
    R[5] = 2.f * (qy * qz - qw * qx);
    R[6] = 2.f * (qx * qz - qw * qy);
    R[7] = 2.f * (qy * qz + qw * qx);
    R[8] = 1.f - 2.f * (qx * qx + qy * qy);
}

// Device pose record: q(4) t(3) pad(1) R_hi(9) R_lo(9); see project.cu.
#define GSR_POSE_WORDS 32

// Forms R(q/|q|) in double precision from pose[0..3] and stores its float
// hi/lo split in pose[8..25] (one thread).
__device__ __forceinline__ void pose_rotation_split(float *pose)
{
    double w = pose[0], x = pose[1], y = pose[2], z = pose[3];
    double n = sqrt(w * w + x * x + y * y + z * z);
    w /= n;
    x /= n;
    y /= n;
    z /= n;
    double R[9] = {1.0 - 2.0 * (y * y + z * z), 2.0 * (x * y - w * z),       2.0 * (x * z + w * y),
                   2.0 * (x * y + w * z),       1.0 - 2.0 * (x * x + z * z), 2.0 * (y * z - w * x),
                   2.0 * (x * z - w * y),       2.0 * (y * z + w * x),       1.0 - 2.0 * (x * x + y * y)};
    for (int k = 0; k < 9; ++k) {
        float hi = (float)R[k];
        pose[8 + k] = hi;
        pose[17 + k] = (float)(R[k] - (double)hi);
    }
}

// Image-space evaluation of one Gaussian at one pixel.  Every operation is an
// explicitly rounded intrinsic so that the forward and the backward kernels,
// which both call it, take bit-identical skip decisions.
struct Eval {
    float dx, dy, ex, G, alpha;
    bool use;  // composited (before the transmittance test)
};

__device__ __forceinline__ Eval eval_gaussian(float px, float py, float u, float v, float ca, float cb,
                                              float cc, float op)
{
    Eval e;
    e.dx = __fsub_rn(px, u);
    e.dy = __fsub_rn(py, v);
    float q = __fmaf_rn(ca, __fmul_rn(e.dx, e.dx), __fmul_rn(cc, __fmul_rn(e.dy, e.dy)));
    float sigma = __fmaf_rn(cb, __fmul_rn(e.dx, e.dy), __fmul_rn(0.5f, q));
    e.ex = __expf(-sigma);
    e.G = __fmul_rn(op, e.ex);
    e.alpha = fminf(GSR_ALPHA_MAX, e.G);
    e.use = (sigma >= 0.f) && (e.alpha >= GSR_ALPHA_MIN);
    return e;
}

// sigma beyond which alpha = o exp(-sigma) is certainly below 1/255:
// ln(255 o) plus a margin far above the float32 error of __logf/__expf, so a
// reject on it never changes a skip decision of eval_gaussian.
__device__ __forceinline__ float sigma_reject(float op) { return __logf(255.f * op) + 0.02f; }

// ------------------------------------------------------------- Adam
// One bias-corrected Adam update of one parameter (shared by the optimiser
// kernels and the fused projection backward + Adam of the one-keyframe step).
__device__ __forceinline__ void adam_update(float &p, float g, float &m, float &v, float lr, float b1, float b2,
                                            float eps, float bc1, float bc2)
{
    m = b1 * m + (1.f - b1) * g;
    v = b2 * v + (1.f - b2) * g * g;
    p -= lr * (m / bc1) / (sqrtf(v / bc2) + eps);
}

// The same update with the bias corrections passed as reciprocals and a fast
// division (a few ulp; the fused projection backward + Adam).
__device__ __forceinline__ void adam_update_fast(float &p, float g, float &m, float &v, float lr, float b1, float b2,
                                                 float eps, float ib1, float ib2)
{
    m = b1 * m + (1.f - b1) * g;
    v = b2 * v + (1.f - b2) * g * g;
    p -= __fdividef(lr * (m * ib1), sqrtf(v * ib2) + eps);
}

__device__ __forceinline__ float sign_of(float x) { return (x > 0.f) ? 1.f : ((x < 0.f) ? -1.f : 0.f); }

// One Gaussian's three log-scales p (in registers) with gradient g plus the
// gradient of rw * |s - mean(s)|_1 (s = exp(p), Sec. 3.4 L_reg); returns the
// unweighted L_reg term.
// FAST: bc1, bc2 are the reciprocals of the bias corrections and the update
// is adam_update_fast
template <bool FAST = false>
__device__ __forceinline__ float adam_log_scales3(float *p, const float *g, float *m, float *v, float rw, float lr,
                                                  const gsr_adam_opts &o, float bc1, float bc2)
{
    float sc[3], sb = 0.f, lsum = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        sc[k] = expf(p[k]);
        sb += sc[k];
    }
    sb *= (1.f / 3.f);
    float sg[3], ssum = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        lsum += fabsf(sc[k] - sb);
        sg[k] = sign_of(sc[k] - sb);
        ssum += sg[k];
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float gk = g[k] + rw * (sg[k] - ssum * (1.f / 3.f)) * sc[k];
        if (FAST) adam_update_fast(p[k], gk, m[k], v[k], lr, o.beta1, o.beta2, o.eps, bc1, bc2);
        else adam_update(p[k], gk, m[k], v[k], lr, o.beta1, o.beta2, o.eps, bc1, bc2);
    }
    return lsum;
}

// Pixel-centre box of a tile (clipped to the image).
struct TileBox {
    float x0, x1, y0, y1;
};

__device__ __forceinline__ TileBox tile_box(const CamK &ck, int tile, int TW, int TH)
{
    const int tx = tile % ck.tiles_x, ty = tile / ck.tiles_x;
    TileBox b;
    b.x0 = (float)(tx * TW) + 0.5f;
    b.x1 = (float)min(tx * TW + TW, ck.W) - 0.5f;
    b.y0 = (float)(ty * TH) + 0.5f;
    b.y1 = (float)min(ty * TH + TH, ck.H) - 0.5f;
    return b;
}

// min over y in [y0, y1] of 0.5 A x^2 + B x y + 0.5 C y^2 (C > 0, iC ~ 1/C:
// an inexact minimiser only raises the value by a second-order amount)
__device__ __forceinline__ float edge_min(float x, float y0, float y1, float A, float B, float C, float iC)
{
    const float y = fminf(fmaxf(-B * x * iC, y0), y1);
    return 0.5f * A * x * x + B * x * y + 0.5f * C * y * y;
}

// false only if sigma exceeds the skip threshold b.w at every pixel centre
// of the box, as the per-pixel evaluation would compute it.  With kappa the
// conic's condition number, both the per-pixel sigma and the box minimum m
// computed here are within 1e-6 kappa (relative) of the exact values (a few
// float32 roundings on terms whose absolute sum is at most kappa sigma), so
// m (1 - e) > thr (1 + e), e = 1e-6 kappa, implies a skip at every pixel.
__device__ __forceinline__ bool tile_may_hit(const float4 &a, const float4 &b, const TileBox &box)
{
    const float ca = a.z, cb = a.w, cc = b.x, thr = b.w;
    const float det = ca * cc - cb * cb;
    if (!(ca > 0.f && cc > 0.f && det > 0.f)) return true;
    const float hd = 0.5f * (ca - cc);
    const float lmax = 0.5f * (ca + cc) + sqrtf(hd * hd + cb * cb);
    const float e = 1e-6f * __fdividef(lmax * lmax, det);
    if (!(e < 0.25f)) return true;
    const float X0 = box.x0 - a.x, X1 = box.x1 - a.x, Y0 = box.y0 - a.y, Y1 = box.y1 - a.y;
    float m = 0.f;
    if (!(X0 <= 0.f && X1 >= 0.f && Y0 <= 0.f && Y1 >= 0.f)) {
        const float ia = __fdividef(1.f, ca), ic = __fdividef(1.f, cc);
        m = fminf(fminf(edge_min(X0, Y0, Y1, ca, cb, cc, ic), edge_min(X1, Y0, Y1, ca, cb, cc, ic)),
                  fminf(edge_min(Y0, X0, X1, cc, cb, ca, ia), edge_min(Y1, X0, X1, cc, cb, ca, ia)));
    }
    return !(m * (1.f - e) > thr * (1.f + e));
}

// --------------------------------------------------------------- launchers
struct Params {
    const float *mean, *log_scale, *quat, *opacity_logit, *rgb;
    int64_t n;
};

BlendView blend_view(const ViewScratch &V, const gsr_render_out *o, const float *d_rgb, const float *d_depth,
                     const float *d_alpha);
gsr_status zero_g2d(gsr_ctx *ctx, ViewScratch &V, cudaStream_t s);
// persistent blend over items (view << 16 | tile) of several views
gsr_status run_blend_multi(gsr_ctx *ctx, const CamK &ck, bool backward, const BlendView *views, const u32 *items,
                           int n_items, u32 *counter, cudaStream_t s);

gsr_status launch_set_pose(gsr_ctx *ctx, float *d_pose, const gsr_pose &p, cudaStream_t s);
// exp(xi^) applied to the (q, t) of a device pose record (xi: device float[6])
gsr_status launch_perturb_pose(gsr_ctx *ctx, float *d_pose, const float *xi, cudaStream_t s);
// g6 <- J_l(xi)^T g6 (device float[6] each)
gsr_status launch_pose_grad_xi(gsr_ctx *ctx, float *g6, const float *xi, cudaStream_t s);
// Projection + binning into V; returns after enqueueing (no sync unless
// allow_grow, which reads the instance count back once to size V).
// launch_order: also write V.order, the one-view blend launch order (the
// persistent multi-view blend builds its own work list instead)
gsr_status run_binning(gsr_ctx *ctx, ViewScratch &V, const Params &P, const CamK &ck, const float *d_pose,
                       bool allow_grow, cudaStream_t s, bool launch_order = true);
gsr_status run_blend_forward(gsr_ctx *ctx, const Params &P, const CamK &ck, gsr_render_out *out,
                             cudaStream_t s);
gsr_status run_blend_backward(gsr_ctx *ctx, const CamK &ck, const gsr_render_out *saved,
                              const float *d_rgb, const float *d_depth, const float *d_alpha,
                              bool pose_only, cudaStream_t s);
// chain image-space gradients to parameters; accumulate = add w * grad into
// the outputs instead of overwriting them.
gsr_status run_project_backward(gsr_ctx *ctx, ViewScratch &V, const Params &P, const CamK &ck,
                                const float *d_pose, gsr_gaussian_grads *dg, float *d_pose6, bool accumulate,
                                float weight, cudaStream_t s);
// adds the gradients of every keyframe's image-space gradients to dg (one pass)
gsr_status run_project_backward_multi(gsr_ctx *ctx, const Params &P, const CamK &ck, const ProjView *views,
                                      int n_views, gsr_gaussian_grads *dg, cudaStream_t s);
// The mapping loss of one view: run_loss_map = run_loss_map_kernels (SSIM
// forward and backward; the per-pixel adjoints) + run_loss_map_final (the
// scalar).  V (nullable): the view whose loss scratch and counters to use,
// so that several views' kernels may run concurrently on different streams
// (their finals then run in order on one stream).
gsr_status run_loss_map(gsr_ctx *ctx, int W, int H, const float *rgb, const float *depth,
                        const float *rgb_t, const float *depth_t, float lam, float wc, float wd,
                        float scale, float *d_rgb, float *d_depth, float *loss_dev, bool accumulate_loss,
                        cudaStream_t s);
gsr_status run_loss_map_kernels(gsr_ctx *ctx, ViewScratch *V, int W, int H, const float *rgb, const float *depth,
                                const float *rgb_t, const float *depth_t, float lam, float wc, float wd,
                                float scale, float *d_rgb, float *d_depth, cudaStream_t s);
gsr_status run_loss_map_final(gsr_ctx *ctx, ViewScratch *V, int W, int H, float lam, float wc, float wd,
                              float scale, float *loss_dev, bool accumulate_loss, cudaStream_t s);
gsr_status run_loss_track(gsr_ctx *ctx, int W, int H, const float *rgb, const float *depth,
                          const float *alpha, const float *rgb_t, const float *depth_t, float lam_c,
                          float k_med, float apow, float *d_rgb, float *d_depth, float *loss_dev,
                          float *median_dev, cudaStream_t s);
// step counter advance + bias corrections (device float[2], returned in *bc),
// and the final L_reg reduction into *loss_reg_dev (part: nb block partial sums)
gsr_status adam_prep(gsr_ctx *ctx, gsr_adam_state *st, const gsr_adam_opts *o, float **bc, cudaStream_t s);
gsr_status adam_lreg_final(gsr_ctx *ctx, const float *part, int nb, float scale, float *loss_reg_dev, cudaStream_t s);
// as adam_lreg_final, and then advances the Adam step counter (for the fused
// projection backward + Adam, which reads the counter without advancing it)
gsr_status adam_lreg_final_step(gsr_ctx *ctx, const float *part, int nb, float scale, float *loss_reg_dev,
                                int32_t *step, cudaStream_t s);
// one-keyframe step: projection backward of every Gaussian fused with its Adam
// update and L_reg (the gradients never reach memory)
gsr_status run_project_backward_adam(gsr_ctx *ctx, ViewScratch &V, gsr_gaussians_mut *g, gsr_adam_state *st,
                                     const gsr_adam_opts *o, const CamK &ck, const float *d_pose,
                                     float *loss_reg_dev, cudaStream_t s);
// number of per-block L_reg partials run_project_backward_adam writes for n Gaussians
int64_t project_bwd_adam_partials(int64_t n);
gsr_status run_adam(gsr_ctx *ctx, gsr_gaussians_mut *g, const gsr_gaussian_grads *gr,
                    gsr_adam_state *st, const gsr_adam_opts *o, float *loss_reg_dev, cudaStream_t s);
gsr_status run_pose_adam(gsr_ctx *ctx, float *d_pose, const float *d_grad6, float *m6, float *v6,
                         int32_t *step, float lr_rho, float lr_phi, float b1, float b2, float eps,
                         cudaStream_t s);
gsr_status copy_tile_lists(gsr_ctx *ctx, int64_t n, int64_t n_tiles, u32 *ranges_h, int32_t *gids_h,
                           int64_t capacity, u32 *depth_h, int64_t *n_inst, cudaStream_t s);

// profiling phases
enum { PROF_BIN = 0, PROF_FWD = 1, PROF_LOSS = 2, PROF_BWD = 3, PROF_PBWD = 4, PROF_ADAM = 5, PROF_NSLOT = 6 };
// records the start (end = false) or end event of a phase on `s` when profiling
gsr_status prof_mark(gsr_ctx *ctx, int phase, bool end, cudaStream_t s);
// work list of the persistent blend: items (view << 16 | tile) of n_views
// views (descriptors in device memory), longest tile list first by length
// bucket (order within a bucket unspecified)
gsr_status run_make_items(gsr_ctx *ctx, const BlendView *views, int n_views, int tiles, u32 *items, cudaStream_t s);
// launch order of one view's blend kernels: tile ids, longest list first
// (as run_make_items, one view)
gsr_status run_order_tiles(gsr_ctx *ctx, ViewScratch &V, int tiles, cudaStream_t s);
// scratch bytes of the launch-order sort of n items (sized before graph capture)
size_t order_hist_bytes(int64_t n);
