// api.cu -- the C ABI of include/gsr.h: context, scratch, renderer entry
// points, fused losses, Adam, tracking and mapping loops.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>

#include "gsr_internal.cuh"

// layout of ctx->small (floats)
enum {
    SM_BC = 0,        // Adam bias corrections [2]
    SM_POSE = 32,     // tracking pose record (GSR_POSE_WORDS floats)
    SM_G6 = 64,       // pose gradient [6]
    SM_M6 = 72,       // pose Adam moments
    SM_V6 = 80,
    SM_STEP = 88,     // int32 pose Adam step
    SM_LOSS0 = 96,    // tracking loss of the first iteration
    SM_LOSS1 = 97,    // loss of the latest iteration
    SM_MED = 98,
    SM_MAPLOSS = 100, // mapping loss accumulator
    SM_WORDS = 256
};

gsr_status gsr_fail(gsr_ctx *ctx, gsr_status s, const std::string &msg)
{
    if (ctx) ctx->err = msg;
    return s;
}

gsr_status gsr_cuda_check(gsr_ctx *ctx, cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return GSR_OK;
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) return gsr_fail(ctx, GSR_ERR_OOM, m);
    return gsr_fail(ctx, GSR_ERR_CUDA, m);
}

gsr_status ensure_buf(gsr_ctx *ctx, DevBuf &b, size_t bytes)
{
    if (bytes <= b.bytes && b.p) return GSR_OK;
    if (b.p) {
        // buffers may be in use by queued work: wait before releasing
        GSR_CUDA(ctx, cudaDeviceSynchronize());
        cudaFree(b.p);
        b.p = nullptr;
        b.bytes = 0;
        // captured graphs may hold the old address: drop them (the next
        // map / track step runs eagerly and captures again)
        if (ctx->map_graph) cudaGraphExecDestroy(ctx->map_graph);
        if (ctx->track_graph) cudaGraphExecDestroy(ctx->track_graph);
        ctx->map_graph = ctx->track_graph = nullptr;
        ctx->map_key = ctx->map_sized_key = ctx->track_key = 0;
        ctx->generation += 1;
    }
    size_t want = bytes > 0 ? bytes : 16;
    cudaError_t e = cudaMalloc(&b.p, want);
    if (e != cudaSuccess) {
        b.p = nullptr;
        (void)cudaGetLastError();
        return gsr_fail(ctx, GSR_ERR_OOM, "cudaMalloc of " + std::to_string(want) + " bytes failed");
    }
    b.bytes = want;
    return GSR_OK;
}

void free_buf(DevBuf &b)
{
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
}

gsr_status prof_mark(gsr_ctx *ctx, int phase, bool end, cudaStream_t s)
{
    if (!ctx->prof) return GSR_OK;
    cudaEvent_t ev = ctx->prof_ev[2 * phase + (end ? 1 : 0)];
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    GSR_CUDA(ctx, cudaStreamIsCapturing(s, &cs));
    if (cs == cudaStreamCaptureStatusActive) GSR_CUDA(ctx, cudaEventRecordWithFlags(ev, s, cudaEventRecordExternal));
    else GSR_CUDA(ctx, cudaEventRecord(ev, s));
    return GSR_OK;
}

extern "C" {

gsr_status gsr_profile_enable(gsr_ctx *ctx, int32_t on)
{
    if (!ctx) return GSR_ERR_INVALID_ARG;
    if (on && !ctx->prof_ev[0])
        for (int i = 0; i < 2 * PROF_NSLOT; ++i) GSR_CUDA(ctx, cudaEventCreate(&ctx->prof_ev[i]));
    ctx->prof = on != 0;
    return GSR_OK;
}

gsr_status gsr_profile_read(gsr_ctx *ctx, float *ms, int32_t n, void *stream)
{
    if (!ctx || !ms || n < 0) return GSR_ERR_INVALID_ARG;
    if (!ctx->prof_ev[0]) return gsr_fail(ctx, GSR_ERR_STATE, "profiling was never enabled");
    GSR_CUDA(ctx, cudaStreamSynchronize((cudaStream_t)stream));
    for (int i = 0; i < n && i < PROF_NSLOT; ++i) {
        float t = -1.f;
        if (cudaEventElapsedTime(&t, ctx->prof_ev[2 * i], ctx->prof_ev[2 * i + 1]) != cudaSuccess) {
            (void)cudaGetLastError();
            t = -1.f;  // phase not executed since profiling was enabled
        }
        ms[i] = t;
    }
    return GSR_OK;
}

void gsr_default_options(gsr_options *o)
{
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->tile_w = 16;
    o->tile_h = 16;
    o->batch = 256;
}

void gsr_default_camera(gsr_camera *c, int32_t width, int32_t height, float fx, float fy, float cx, float cy)
{
    if (!c) return;
    c->width = width;
    c->height = height;
    c->fx = fx;
    c->fy = fy;
    c->cx = cx;
    c->cy = cy;
    c->z_near = 0.2f;
    c->eps2d = 0.3f;
}

const char *gsr_status_string(gsr_status s)
{
    switch (s) {
    case GSR_OK: return "GSR_OK";
    case GSR_ERR_INVALID_ARG: return "GSR_ERR_INVALID_ARG";
    case GSR_ERR_CUDA: return "GSR_ERR_CUDA";
    case GSR_ERR_OOM: return "GSR_ERR_OOM";
    case GSR_ERR_CAPACITY: return "GSR_ERR_CAPACITY";
    case GSR_ERR_TIMEOUT: return "GSR_ERR_TIMEOUT";
    case GSR_ERR_NONFINITE: return "GSR_ERR_NONFINITE";
    case GSR_ERR_STATE: return "GSR_ERR_STATE";
    }
    return "GSR_ERR_UNKNOWN";
}

static bool valid_tile(int w, int h)
{
    return (w == 16 && h == 16) || (w == 8 && h == 8) || (w == 16 && h == 8) || (w == 32 && h == 8);
}

gsr_status gsr_create(gsr_ctx **out, const gsr_options *opt)
{
    if (!out) return GSR_ERR_INVALID_ARG;
    *out = nullptr;
    gsr_options o;
    gsr_default_options(&o);
    if (opt) o = *opt;
    if (!valid_tile(o.tile_w, o.tile_h)) return GSR_ERR_INVALID_ARG;
    if (o.batch != 32 && o.batch != 64 && o.batch != 128 && o.batch != 256) return GSR_ERR_INVALID_ARG;
    if (o.max_gaussians < 0 || o.max_instances < 0 || o.max_pixels < 0) return GSR_ERR_INVALID_ARG;
    if (o.ppt_fwd < 0 || o.ppt_fwd > 2 || o.ppt_bwd < 0 || o.ppt_bwd > 2) return GSR_ERR_INVALID_ARG;
    if (o.rect_lists != 0 && o.rect_lists != 1) return GSR_ERR_INVALID_ARG;
    gsr_ctx *c = new (std::nothrow) gsr_ctx();
    if (!c) return GSR_ERR_OOM;
    c->opt = o;
    c->ppt_fwd = o.ppt_fwd ? o.ppt_fwd : 1;
    c->ppt_bwd = o.ppt_bwd ? o.ppt_bwd : 2;
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        (void)cudaGetLastError();
        delete c;
        return GSR_ERR_CUDA;
    }
    if (cudaMallocHost((void **)&c->host_pinned, 256) != cudaSuccess) {
        (void)cudaGetLastError();
        delete c;
        return GSR_ERR_CUDA;
    }
    gsr_status s = ensure_buf(c, c->small, SM_WORDS * sizeof(float));
    if (s == GSR_OK) s = ensure_buf(c, c->view.counters, sizeof(u32) * CNT_WORDS);
    if (s == GSR_OK && cudaMemset(c->view.counters.p, 0, sizeof(u32) * CNT_WORDS) != cudaSuccess) s = GSR_ERR_CUDA;
    if (s == GSR_OK && cudaMemset(c->small.p, 0, SM_WORDS * sizeof(float)) != cudaSuccess) s = GSR_ERR_CUDA;
    // pre-size scratch from the hints
    ViewScratch &V = c->view;
    if (s == GSR_OK && o.max_gaussians > 0) {
        int64_t n = o.max_gaussians;
        DevBuf *bufs[] = {&V.flag, &V.compact, &V.rank_of_gid, &V.dkeys[0], &V.dkeys[1], &V.dvals[0], &V.dvals[1],
                          &V.tcount, &V.inst_off};
        for (DevBuf *b : bufs)
            if (s == GSR_OK) s = ensure_buf(c, *b, sizeof(u32) * n);
        if (s == GSR_OK) s = ensure_buf(c, V.rec, sizeof(float4) * 3 * n);
        if (s == GSR_OK) s = ensure_buf(c, V.rec_sorted, sizeof(float4) * 3 * n);
        if (s == GSR_OK) s = ensure_buf(c, V.g2d, sizeof(float) * 12 * n);
        if (s == GSR_OK) V.cap_n = n;
    }
    if (s == GSR_OK && o.max_instances > 0) s = grow_instance_capacity(c, c->view, o.max_instances);
    if (s != GSR_OK) {
        gsr_destroy(c);
        return s;
    }
    *out = c;
    return GSR_OK;
}

void gsr_destroy(gsr_ctx *c)
{
    if (!c) return;
    cudaDeviceSynchronize();
    ViewScratch &V = c->view;
    DevBuf *bufs[] = {&V.rec, &V.flag, &V.compact, &V.rank_of_gid, &V.dkeys[0], &V.dkeys[1], &V.dvals[0], &V.dvals[1],
                      &V.rec_sorted, &V.tcount, &V.inst_off, &V.tkeys[0], &V.tkeys[1], &V.tvals[0], &V.tvals[1],
                      &V.ranges, &V.order, &V.order_hist, &V.g2d, &V.counters, &V.pose, &V.scan_tmp, &V.radix_hist, &V.loss_maps,
                      &V.loss_part, &c->scan_tmp,
                      &c->radix_hist, &c->pose_part,
                      &c->loss_part, &c->loss_maps, &c->img_tmp, &c->small, &c->grads};
    for (DevBuf *b : bufs) free_buf(*b);
    for (ViewScratch &W : c->mv) {
        DevBuf *vb[] = {&W.rec, &W.flag, &W.compact, &W.rank_of_gid, &W.dkeys[0], &W.dkeys[1], &W.dvals[0],
                        &W.dvals[1], &W.rec_sorted, &W.tcount, &W.inst_off, &W.tkeys[0], &W.tkeys[1], &W.tvals[0],
                        &W.tvals[1], &W.ranges, &W.order, &W.order_hist, &W.g2d, &W.counters, &W.pose, &W.scan_tmp, &W.radix_hist,
                        &W.loss_maps, &W.loss_part};
        for (DevBuf *b : vb) free_buf(*b);
    }
    DevBuf *mb[] = {&c->mv_frames, &c->mv_desc, &c->mv_pview, &c->mv_items, &c->mv_order_hist, &c->mv_counter};
    for (DevBuf *b : mb) free_buf(*b);
    SeedScratch &S = c->seed;
    DevBuf *sb[] = {&S.flag, &S.sel, &S.off, &S.keys[0], &S.keys[1], &S.vals[0], &S.vals[1], &S.cnt, &S.cand_pix,
                    &S.cand_pts, &S.keep, &S.keep_off, &S.d2, &S.new_cand, &S.prune_tmp};
    for (DevBuf *b : sb) free_buf(*b);
    if (c->track_graph) cudaGraphExecDestroy(c->track_graph);
    if (c->map_graph) cudaGraphExecDestroy(c->map_graph);
    if (c->host_pinned) cudaFreeHost(c->host_pinned);
    if (c->fork_ev) cudaEventDestroy(c->fork_ev);
    for (int i = 0; i < gsr_ctx::N_SIDE; ++i) {
        if (c->side[i]) cudaStreamDestroy(c->side[i]);
        if (c->join_ev[i]) cudaEventDestroy(c->join_ev[i]);
    }
    for (int i = 0; i < 2 * PROF_NSLOT; ++i)
        if (c->prof_ev[i]) cudaEventDestroy(c->prof_ev[i]);
    delete c;
}

const char *gsr_last_error(const gsr_ctx *c) { return c ? c->err.c_str() : "null context"; }

int64_t gsr_kernel_launches(const gsr_ctx *c) { return c ? c->launches : 0; }

} // extern "C"

// ------------------------------------------------------------------ helpers
static gsr_status check_gaussians(gsr_ctx *ctx, const gsr_gaussians *g)
{
    if (!g || g->n < 0) return gsr_fail(ctx, GSR_ERR_INVALID_ARG, "null Gaussians or negative count");
    if (g->n > 0 && (!g->mean || !g->log_scale || !g->quat || !g->opacity_logit || !g->rgb))
        return gsr_fail(ctx, GSR_ERR_INVALID_ARG, "null Gaussian parameter pointer");
    if (g->n > 0x7fffffffLL) return gsr_fail(ctx, GSR_ERR_INVALID_ARG, "more than 2^31-1 Gaussians");
    return GSR_OK;
}

static gsr_status check_camera(gsr_ctx *ctx, const gsr_camera *c)
{
    if (!c) return gsr_fail(ctx, GSR_ERR_INVALID_ARG, "null camera");
    if (c->width <= 0 || c->height <= 0 || c->width > 32768 || c->height > 32768)
        return gsr_fail(ctx, GSR_ERR_INVALID_ARG, "image size out of range");
    if (!(c->fx > 0.f) || !(c->fy > 0.f) || !(c->z_near > 0.f) || !(c->eps2d >= 0.f))
        return gsr_fail(ctx, GSR_ERR_INVALID_ARG, "invalid camera intrinsics");
    int64_t tiles = ceil_div(c->width, ctx->opt.tile_w) * ceil_div(c->height, ctx->opt.tile_h);
    if (tiles >= 65536) return gsr_fail(ctx, GSR_ERR_INVALID_ARG, "more than 65535 tiles");
    return GSR_OK;
}

static Params to_params(const gsr_gaussians *g)
{
    Params P;
    P.mean = g->mean;
    P.log_scale = g->log_scale;
    P.quat = g->quat;
    P.opacity_logit = g->opacity_logit;
    P.rgb = g->rgb;
    P.n = g->n;
    return P;
}

static gsr_status take_status(gsr_ctx *ctx, cudaStream_t s)
{
    u32 *cnt = (u32 *)ctx->view.counters.p;
    GSR_CUDA(ctx, cudaMemcpyAsync(ctx->host_pinned + 8, cnt + CNT_STATUS, sizeof(u32), cudaMemcpyDeviceToHost, s));
    GSR_CUDA(ctx, cudaStreamSynchronize(s));
    u32 st = ctx->host_pinned[8];
    if (st) GSR_CUDA(ctx, cudaMemsetAsync(cnt + CNT_STATUS, 0, sizeof(u32), s));
    if (st & GSR_FLAG_CAPACITY) return gsr_fail(ctx, GSR_ERR_CAPACITY, "tile-instance capacity exceeded");
    if (st & GSR_FLAG_NONFINITE) return gsr_fail(ctx, GSR_ERR_NONFINITE, "non-finite loss");
    if (st & GSR_FLAG_TIMEOUT) return gsr_fail(ctx, GSR_ERR_TIMEOUT, "a bounded device wait expired");
    return GSR_OK;
}

static bool same_forward(const gsr_ctx *ctx, const gsr_gaussians *g, const gsr_camera *c, const gsr_pose *p,
                         const float *xi)
{
    return ctx->fwd_n == g->n && ctx->fwd_xi == xi && ctx->fwd_ptrs[0] == g->mean && ctx->fwd_ptrs[1] == g->log_scale &&
           ctx->fwd_ptrs[2] == g->quat && ctx->fwd_ptrs[3] == g->opacity_logit && ctx->fwd_ptrs[4] == g->rgb &&
           memcmp(&ctx->fwd_cam, c, sizeof(*c)) == 0 && memcmp(&ctx->fwd_pose, p, sizeof(*p)) == 0;
}

static void remember_forward(gsr_ctx *ctx, const gsr_gaussians *g, const gsr_camera *c, const gsr_pose *p,
                             const float *xi)
{
    ctx->fwd_n = g->n;
    ctx->fwd_xi = xi;
    ctx->fwd_ptrs[0] = g->mean;
    ctx->fwd_ptrs[1] = g->log_scale;
    ctx->fwd_ptrs[2] = g->quat;
    ctx->fwd_ptrs[3] = g->opacity_logit;
    ctx->fwd_ptrs[4] = g->rgb;
    ctx->fwd_cam = *c;
    ctx->fwd_pose = *p;
}

static void forget_forward(gsr_ctx *ctx) { ctx->fwd_n = -1; }

static gsr_status ensure_view_pose(gsr_ctx *ctx)
{
    return ensure_buf(ctx, ctx->view.pose, GSR_POSE_WORDS * sizeof(float));
}

// ---------------------------------------------------------------- renderer
static gsr_status render_forward(gsr_ctx *ctx, const gsr_gaussians *g, const gsr_camera *cam, const gsr_pose *pose,
                                 const float *xi, gsr_render_out *out, void *stream)
{
    if (!ctx) return GSR_ERR_INVALID_ARG;
    GSR_TRY(check_gaussians(ctx, g));
    GSR_TRY(check_camera(ctx, cam));
    if (!pose || !out || !out->rgb || !out->depth || !out->alpha || !out->final_T || !out->last_idx)
        return gsr_fail(ctx, GSR_ERR_INVALID_ARG, "null pose or output pointer");
    cudaStream_t s = (cudaStream_t)stream;
    forget_forward(ctx);
    GSR_TRY(ensure_view_pose(ctx));
    float *d_pose = (float *)ctx->view.pose.p;
    GSR_TRY(launch_set_pose(ctx, d_pose, *pose, s));
    if (xi) GSR_TRY(launch_perturb_pose(ctx, d_pose, xi, s));
    CamK ck = make_camk(*cam, ctx->opt.tile_w, ctx->opt.tile_h);
    Params P = to_params(g);
    GSR_TRY(prof_mark(ctx, PROF_BIN, false, s));
    GSR_TRY(run_binning(ctx, ctx->view, P, ck, d_pose, !ctx->opt.fixed_capacity, s));
    GSR_TRY(prof_mark(ctx, PROF_BIN, true, s));
    GSR_TRY(prof_mark(ctx, PROF_FWD, false, s));
    GSR_TRY(run_blend_forward(ctx, P, ck, out, s));
    GSR_TRY(prof_mark(ctx, PROF_FWD, true, s));
    remember_forward(ctx, g, cam, pose, xi);
    return GSR_OK;
}

extern "C" gsr_status gsr_render_forward(gsr_ctx *ctx, const gsr_gaussians *g, const gsr_camera *cam,
                                         const gsr_pose *pose, gsr_render_out *out, void *stream)
{
    return render_forward(ctx, g, cam, pose, nullptr, out, stream);
}

extern "C" gsr_status gsr_render_forward_xi(gsr_ctx *ctx, const gsr_gaussians *g, const gsr_camera *cam,
                                            const gsr_pose *pose, const float *xi, gsr_render_out *out, void *stream)
{
    if (ctx && !xi) return gsr_fail(ctx, GSR_ERR_INVALID_ARG, "null twist");
    return render_forward(ctx, g, cam, pose, xi, out, stream);
}

extern "C" gsr_status gsr_frame_stats_get(gsr_ctx *ctx, gsr_frame_stats *st, void *stream)
{
    if (!ctx || !st) return GSR_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    u32 *cnt = (u32 *)ctx->view.counters.p;
    GSR_CUDA(ctx, cudaMemcpyAsync(ctx->host_pinned, cnt, sizeof(u32) * 4, cudaMemcpyDeviceToHost, s));
    GSR_CUDA(ctx, cudaStreamSynchronize(s));
    st->n_visible = ctx->host_pinned[CNT_VISIBLE];
    st->n_instances = ctx->host_pinned[CNT_INSTANCES];
    st->n_tiles = ctx->fwd_n >= 0 ? ceil_div(ctx->fwd_cam.width, ctx->opt.tile_w) *
                                        ceil_div(ctx->fwd_cam.height, ctx->opt.tile_h)
                                  : 0;
    st->capacity_instances = ctx->view.cap_i;
    return take_status(ctx, s);  // the counters are filled either way
}

// Defined in sort.cu: one warp runs the radix sort's bounded look-back wait
// on `word`, giving up after `polls` polls with GSR_FLAG_TIMEOUT in *status.
gsr_status lookback_wait_check(gsr_ctx *ctx, const u32 *word, int32_t polls, u32 *status, cudaStream_t s);

extern "C" gsr_status gsr_check_wait_timeout(gsr_ctx *ctx, int32_t polls, void *stream)
{
    if (!ctx) return GSR_ERR_INVALID_ARG;
    if (polls < 1 || polls > 1000000) return gsr_fail(ctx, GSR_ERR_INVALID_ARG, "polls must lie in [1, 1000000]");
    cudaStream_t s = (cudaStream_t)stream;
    GSR_TRY(ensure_buf(ctx, ctx->view.counters, sizeof(u32) * CNT_WORDS));
    u32 *cnt = (u32 *)ctx->view.counters.p;
    // the last word of the counter block is written by no kernel: zero it, then wait on it
    u32 *word = cnt + (CNT_WORDS - 1);
    GSR_CUDA(ctx, cudaMemsetAsync(word, 0, sizeof(u32), s));
    GSR_TRY(lookback_wait_check(ctx, word, polls, cnt + CNT_STATUS, s));
    return take_status(ctx, s);
}

extern "C" gsr_status gsr_tile_lists_get(gsr_ctx *ctx, uint32_t *ranges, int32_t *gids, int64_t capacity,
                                         uint32_t *depth_bits, int64_t *n_instances, void *stream)
{
    if (!ctx || !n_instances || capacity < 0) return GSR_ERR_INVALID_ARG;
    if (ctx->fwd_n < 0) return gsr_fail(ctx, GSR_ERR_STATE, "no forward on this context");
    int64_t tiles = ceil_div(ctx->fwd_cam.width, ctx->opt.tile_w) * ceil_div(ctx->fwd_cam.height, ctx->opt.tile_h);
    return copy_tile_lists(ctx, ctx->fwd_n, tiles, ranges, gids, capacity, depth_bits, n_instances,
                           (cudaStream_t)stream);
}

extern "C" gsr_status gsr_records_get(gsr_ctx *ctx, float *rec, uint32_t *visible, int64_t n, void *stream)
{
    if (!ctx || !rec || !visible || n < 0) return GSR_ERR_INVALID_ARG;
    if (ctx->fwd_n < 0) return gsr_fail(ctx, GSR_ERR_STATE, "no forward on this context");
    if (n != ctx->fwd_n) return gsr_fail(ctx, GSR_ERR_INVALID_ARG, "n differs from the last forward's count");
    if (n == 0) return GSR_OK;
    cudaStream_t s = (cudaStream_t)stream;
    GSR_CUDA(ctx, cudaMemcpyAsync(rec, ctx->view.rec.p, sizeof(float) * 12 * (size_t)n, cudaMemcpyDeviceToHost, s));
    GSR_CUDA(ctx, cudaMemcpyAsync(visible, ctx->view.flag.p, sizeof(uint32_t) * (size_t)n, cudaMemcpyDeviceToHost, s));
    GSR_CUDA(ctx, cudaStreamSynchronize(s));
    return GSR_OK;
}

static gsr_status render_backward(gsr_ctx *ctx, const gsr_gaussians *g, const gsr_camera *cam,
                                  const gsr_pose *pose, const float *xi, const gsr_render_out *saved,
                                  const float *d_rgb, const float *d_depth, const float *d_alpha,
                                  gsr_gaussian_grads *dg, float *d_pose6, void *stream)
{
    if (!ctx) return GSR_ERR_INVALID_ARG;
    GSR_TRY(check_gaussians(ctx, g));
    GSR_TRY(check_camera(ctx, cam));
    if (!pose || !saved || !saved->final_T || !saved->last_idx)
        return gsr_fail(ctx, GSR_ERR_INVALID_ARG, "null pose or saved forward state");
    cudaStream_t s = (cudaStream_t)stream;
    CamK ck = make_camk(*cam, ctx->opt.tile_w, ctx->opt.tile_h);
    Params P = to_params(g);
    GSR_TRY(ensure_view_pose(ctx));
    float *d_pose = (float *)ctx->view.pose.p;
    if (ctx->opt.memory_saving || !same_forward(ctx, g, cam, pose, xi)) {
        // rebuild the (deterministic) tile lists instead of keeping them alive
        GSR_TRY(launch_set_pose(ctx, d_pose, *pose, s));
        if (xi) GSR_TRY(launch_perturb_pose(ctx, d_pose, xi, s));
        GSR_TRY(run_binning(ctx, ctx->view, P, ck, d_pose, !ctx->opt.fixed_capacity, s));
        remember_forward(ctx, g, cam, pose, xi);
    }
    bool want_params = dg && (dg->mean || dg->log_scale || dg->quat || dg->opacity_logit || dg->rgb);
    GSR_TRY(prof_mark(ctx, PROF_BWD, false, s));
    GSR_TRY(run_blend_backward(ctx, ck, saved, d_rgb, d_depth, d_alpha, !want_params, s));
    GSR_TRY(prof_mark(ctx, PROF_BWD, true, s));
    GSR_TRY(prof_mark(ctx, PROF_PBWD, false, s));
    GSR_TRY(run_project_backward(ctx, ctx->view, P, ck, d_pose, want_params ? dg : nullptr, d_pose6, false, 1.f, s));
    if (xi && d_pose6) GSR_TRY(launch_pose_grad_xi(ctx, d_pose6, xi, s));
    GSR_TRY(prof_mark(ctx, PROF_PBWD, true, s));
    return GSR_OK;
}

extern "C" gsr_status gsr_render_backward(gsr_ctx *ctx, const gsr_gaussians *g, const gsr_camera *cam,
                                          const gsr_pose *pose, const gsr_render_out *saved, const float *d_rgb,
                                          const float *d_depth, const float *d_alpha, gsr_gaussian_grads *dg,
                                          float *d_pose6, void *stream)
{
    return render_backward(ctx, g, cam, pose, nullptr, saved, d_rgb, d_depth, d_alpha, dg, d_pose6, stream);
}

extern "C" gsr_status gsr_render_backward_xi(gsr_ctx *ctx, const gsr_gaussians *g, const gsr_camera *cam,
                                             const gsr_pose *pose, const float *xi, const gsr_render_out *saved,
                                             const float *d_rgb, const float *d_depth, const float *d_alpha,
                                             gsr_gaussian_grads *dg, float *d_xi, void *stream)
{
    if (ctx && !xi) return gsr_fail(ctx, GSR_ERR_INVALID_ARG, "null twist");
    return render_backward(ctx, g, cam, pose, xi, saved, d_rgb, d_depth, d_alpha, dg, d_xi, stream);
}

// ------------------------------------------------------------------ losses
extern "C" gsr_status gsr_loss_map(gsr_ctx *ctx, int32_t width, int32_t height, const float *rgb, const float *depth,
                                   const float *rgb_target, const float *depth_target, float lambda_ssim,
                                   float w_color, float w_depth, float scale, float *d_rgb, float *d_depth,
                                   float *loss_dev, void *stream)
{
    if (!ctx) return GSR_ERR_INVALID_ARG;
    if (width <= 0 || height <= 0 || !rgb || !depth || !rgb_target || !depth_target || !d_rgb || !d_depth)
        return gsr_fail(ctx, GSR_ERR_INVALID_ARG, "invalid loss arguments");
    return run_loss_map(ctx, width, height, rgb, depth, rgb_target, depth_target, lambda_ssim, w_color, w_depth,
                        scale, d_rgb, d_depth, loss_dev, false, (cudaStream_t)stream);
}

extern "C" gsr_status gsr_loss_track(gsr_ctx *ctx, int32_t width, int32_t height, const float *rgb,
                                     const float *depth, const float *alpha, const float *rgb_target,
                                     const float *depth_target, float lambda_c, float k_median, float alpha_pow,
                                     float *d_rgb, float *d_depth, float *loss_dev, float *median_dev, void *stream)
{
    if (!ctx) return GSR_ERR_INVALID_ARG;
    if (width <= 0 || height <= 0 || !rgb || !depth || !alpha || !rgb_target || !depth_target || !d_rgb || !d_depth)
        return gsr_fail(ctx, GSR_ERR_INVALID_ARG, "invalid loss arguments");
    return run_loss_track(ctx, width, height, rgb, depth, alpha, rgb_target, depth_target, lambda_c, k_median,
                          alpha_pow, d_rgb, d_depth, loss_dev, median_dev, (cudaStream_t)stream);
}

extern "C" gsr_status gsr_adam_step(gsr_ctx *ctx, gsr_gaussians_mut *g, const gsr_gaussian_grads *grads,
                                    gsr_adam_state *st, const gsr_adam_opts *opt, float *loss_reg_dev, void *stream)
{
    if (!ctx) return GSR_ERR_INVALID_ARG;
    if (!g || !grads || !st || !opt || g->n < 0) return gsr_fail(ctx, GSR_ERR_INVALID_ARG, "null Adam argument");
    if (g->n == 0) return GSR_OK;
    if (!g->mean || !g->log_scale || !g->quat || !g->opacity_logit || !g->rgb || !grads->mean || !grads->log_scale ||
        !grads->quat || !grads->opacity_logit || !grads->rgb || !st->step || !st->m_mean || !st->v_mean ||
        !st->m_log_scale || !st->v_log_scale || !st->m_quat || !st->v_quat || !st->m_opacity_logit ||
        !st->v_opacity_logit || !st->m_rgb || !st->v_rgb)
        return gsr_fail(ctx, GSR_ERR_INVALID_ARG, "null Adam pointer");
    return run_adam(ctx, g, grads, st, opt, loss_reg_dev, (cudaStream_t)stream);
}

// ---------------------------------------------------------------- tracking
struct FrameBufs {
    float *rgb, *depth, *alpha, *T, *d_rgb, *d_depth;
    int32_t *last;
};

static gsr_status frame_bufs(gsr_ctx *ctx, int64_t HW, FrameBufs &f)
{
    GSR_TRY(ensure_buf(ctx, ctx->img_tmp, sizeof(float) * 12 * (size_t)HW));
    float *b = (float *)ctx->img_tmp.p;
    f.rgb = b;
    f.depth = b + 3 * HW;
    f.alpha = b + 4 * HW;
    f.T = b + 5 * HW;
    f.last = (int32_t *)(b + 6 * HW);
    f.d_rgb = b + 7 * HW;
    f.d_depth = b + 10 * HW;
    return GSR_OK;
}

static gsr_status track_iter(gsr_ctx *ctx, const Params &P, const CamK &ck, const FrameBufs &f, const float *rgb_in,
                             const float *depth_in, const gsr_track_opts *o, float *loss_slot, bool grow,
                             cudaStream_t s)
{
    float *sm = (float *)ctx->small.p;
    gsr_render_out ro{f.rgb, f.depth, f.alpha, f.T, f.last, nullptr};
    GSR_TRY(run_binning(ctx, ctx->view, P, ck, sm + SM_POSE, grow, s));
    GSR_TRY(run_blend_forward(ctx, P, ck, &ro, s));
    GSR_TRY(run_loss_track(ctx, ck.W, ck.H, f.rgb, f.depth, f.alpha, rgb_in, depth_in, o->lambda_c, o->k_median,
                           o->alpha_pow, f.d_rgb, f.d_depth, loss_slot, sm + SM_MED, s));
    GSR_TRY(run_blend_backward(ctx, ck, &ro, f.d_rgb, f.d_depth, nullptr, true, s));
    GSR_TRY(run_project_backward(ctx, ctx->view, P, ck, sm + SM_POSE, nullptr, sm + SM_G6, false, 1.f, s));
    GSR_TRY(run_pose_adam(ctx, sm + SM_POSE, sm + SM_G6, sm + SM_M6, sm + SM_V6, (int32_t *)(sm + SM_STEP),
                          o->lr_rho, o->lr_phi, o->beta1, o->beta2, o->eps, s));
    return GSR_OK;
}

extern "C" gsr_status gsr_track_step(gsr_ctx *ctx, const gsr_gaussians *g, const gsr_camera *cam,
                                     const float *rgb_in, const float *depth_in, gsr_pose *pose_inout,
                                     int32_t n_iters, const gsr_track_opts *opt, gsr_track_stats *out, void *stream)
{
    if (!ctx) return GSR_ERR_INVALID_ARG;
    GSR_TRY(check_gaussians(ctx, g));
    GSR_TRY(check_camera(ctx, cam));
    if (!rgb_in || !depth_in || !pose_inout || !opt || n_iters < 0)
        return gsr_fail(ctx, GSR_ERR_INVALID_ARG, "invalid tracking arguments");
    cudaStream_t s = (cudaStream_t)stream;
    forget_forward(ctx);
    CamK ck = make_camk(*cam, ctx->opt.tile_w, ctx->opt.tile_h);
    Params P = to_params(g);
    const int64_t HW = (int64_t)cam->width * cam->height;
    FrameBufs f;
    GSR_TRY(frame_bufs(ctx, HW, f));
    float *sm = (float *)ctx->small.p;
    GSR_TRY(launch_set_pose(ctx, sm + SM_POSE, *pose_inout, s));
    GSR_CUDA(ctx, cudaMemsetAsync(sm + SM_M6, 0, sizeof(float) * (SM_STEP + 1 - SM_M6), s));
    GSR_CUDA(ctx, cudaMemsetAsync(sm + SM_LOSS0, 0, sizeof(float) * 3, s));
    const bool grow = !ctx->opt.fixed_capacity;
    for (int32_t it = 0; it < n_iters; ++it) {
        bool first = it == 0;
        if (!first && opt->use_graph) {
            // capture one iteration on the first pass, replay it afterwards
            // keyed by every pointer, size, camera value and option the graph bakes in
            uint64_t key = 1469598103934665603ull;
            auto mix = [&key](uint64_t v) { key = (key ^ v) * 1099511628211ull; };
            const void *ptrs[] = {g->mean, g->log_scale, g->quat, g->opacity_logit, g->rgb, rgb_in, depth_in};
            for (const void *q : ptrs) mix((uint64_t)(uintptr_t)q);
            mix((uint64_t)g->n);
            mix((uint64_t)ctx->prof);
            const unsigned char *cb = (const unsigned char *)cam;
            for (size_t i = 0; i < sizeof(*cam); ++i) mix(cb[i]);
            const unsigned char *ob = (const unsigned char *)opt;
            for (size_t i = 0; i < sizeof(*opt); ++i) mix(ob[i]);
            if (!ctx->track_graph || ctx->track_key != key) {
                if (ctx->track_graph) cudaGraphExecDestroy(ctx->track_graph);
                ctx->track_graph = nullptr;
                cudaStream_t cs;
                GSR_CUDA(ctx, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
                GSR_CUDA(ctx, cudaStreamSynchronize(s));
                GSR_CUDA(ctx, cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
                const int64_t l0 = ctx->launches;
                gsr_status st = track_iter(ctx, P, ck, f, rgb_in, depth_in, opt, sm + SM_LOSS1, false, cs);
                ctx->track_graph_kernels = ctx->launches - l0;
                ctx->launches = l0;
                cudaGraph_t graph = nullptr;
                cudaError_t e = cudaStreamEndCapture(cs, &graph);
                cudaStreamDestroy(cs);
                if (st != GSR_OK) {
                    if (graph) cudaGraphDestroy(graph);
                    return st;
                }
                GSR_CUDA(ctx, e);
                e = cudaGraphInstantiate(&ctx->track_graph, graph, 0);
                cudaGraphDestroy(graph);
                GSR_CUDA(ctx, e);
                ctx->track_key = key;
            }
            GSR_CUDA(ctx, cudaGraphLaunch(ctx->track_graph, s));
            ctx->launches += ctx->track_graph_kernels;
        } else {
            GSR_TRY(track_iter(ctx, P, ck, f, rgb_in, depth_in, opt, sm + (first ? SM_LOSS0 : SM_LOSS1), grow, s));
            if (first && opt->use_graph && grow) {
                // headroom for the instance count to move while the pose changes
                ViewScratch &V = ctx->view;
                GSR_CUDA(ctx, cudaStreamSynchronize(s));
                int64_t need = (int64_t)ctx->host_pinned[0];
                int64_t c = need + need / 2 + 4096;
                if (c > V.cap_i) {
                    GSR_TRY(grow_instance_capacity(ctx, V, c));
                    if (ctx->track_graph) cudaGraphExecDestroy(ctx->track_graph);
                    ctx->track_graph = nullptr;
                }
            }
        }
    }
    GSR_CUDA(ctx, cudaMemcpyAsync(ctx->host_pinned, sm + SM_POSE, sizeof(float) * 7, cudaMemcpyDeviceToHost, s));
    GSR_CUDA(ctx, cudaMemcpyAsync(ctx->host_pinned + 16, sm + SM_LOSS0, sizeof(float) * 2, cudaMemcpyDeviceToHost, s));
    GSR_TRY(take_status(ctx, s));
    const float *hp = (const float *)ctx->host_pinned;
    for (int k = 0; k < 4; ++k) pose_inout->q[k] = hp[k];
    for (int k = 0; k < 3; ++k) pose_inout->t[k] = hp[4 + k];
    if (out) {
        out->loss_first = hp[16];
        out->loss_last = n_iters > 1 ? hp[17] : hp[16];
        out->iters = n_iters;
    }
    return GSR_OK;
}

// ----------------------------------------------------------------- mapping
static gsr_status map_iter(gsr_ctx *ctx, gsr_gaussians_mut *g, gsr_adam_state *st, const CamK &ck,
                           const gsr_keyframe *kfs, int n_kf, const float *w, const gsr_map_opts *o, bool grow,
                           cudaStream_t s)
{
    const int64_t n = g->n, HW = (int64_t)ck.W * ck.H;
    float *G = (float *)ctx->grads.p;
    gsr_gaussian_grads gr{G, G + 3 * n, G + 6 * n, G + 10 * n, G + 11 * n};
    float *sm = (float *)ctx->small.p;
    FrameBufs f;
    GSR_TRY(frame_bufs(ctx, HW, f));
    // one keyframe: the projection backward writes every gradient (no zeroing,
    // no read-modify-write); several: they accumulate into zeroed arrays
    if (n_kf > 1) GSR_CUDA(ctx, cudaMemsetAsync(G, 0, sizeof(float) * 14 * n, s));
    GSR_CUDA(ctx, cudaMemsetAsync(sm + SM_MAPLOSS, 0, sizeof(float), s));
    Params P{g->mean, g->log_scale, g->quat, g->opacity_logit, g->rgb, n};
    float *d_pose = (float *)ctx->view.pose.p;
    for (int k = 0; k < n_kf; ++k) {
        gsr_render_out ro{f.rgb, f.depth, f.alpha, f.T, f.last, nullptr};
        GSR_TRY(prof_mark(ctx, PROF_BIN, false, s));
        GSR_TRY(launch_set_pose(ctx, d_pose, kfs[k].pose, s));
        GSR_TRY(run_binning(ctx, ctx->view, P, ck, d_pose, grow, s));
        GSR_TRY(prof_mark(ctx, PROF_BIN, true, s));
        GSR_TRY(prof_mark(ctx, PROF_FWD, false, s));
        GSR_TRY(run_blend_forward(ctx, P, ck, &ro, s));
        GSR_TRY(prof_mark(ctx, PROF_FWD, true, s));
        GSR_TRY(prof_mark(ctx, PROF_LOSS, false, s));
        GSR_TRY(run_loss_map(ctx, ck.W, ck.H, f.rgb, f.depth, kfs[k].rgb, kfs[k].depth, o->lambda_ssim, o->w_color,
                             o->w_depth, w[k], f.d_rgb, f.d_depth, sm + SM_MAPLOSS, true, s));
        GSR_TRY(prof_mark(ctx, PROF_LOSS, true, s));
        GSR_TRY(prof_mark(ctx, PROF_BWD, false, s));
        GSR_TRY(run_blend_backward(ctx, ck, &ro, f.d_rgb, f.d_depth, nullptr, false, s));
        GSR_TRY(prof_mark(ctx, PROF_BWD, true, s));
        GSR_TRY(prof_mark(ctx, PROF_PBWD, false, s));
        if (n_kf == 1) {
            // projection backward fused with Adam (the "adam" phase holds only the L_reg sum)
            GSR_TRY(run_project_backward_adam(ctx, ctx->view, g, st, &o->adam, ck, d_pose, nullptr, s));
            GSR_TRY(prof_mark(ctx, PROF_PBWD, true, s));
            GSR_TRY(prof_mark(ctx, PROF_ADAM, false, s));
            const unsigned nb = (unsigned)project_bwd_adam_partials(n);
            GSR_TRY(adam_lreg_final_step(ctx, (const float *)ctx->pose_part.p, (int)nb,
                                         o->adam.w_reg / (float)(n > 0 ? n : 1), sm + SM_MAPLOSS, st->step, s));
            GSR_TRY(prof_mark(ctx, PROF_ADAM, true, s));
            return GSR_OK;
        }
        GSR_TRY(run_project_backward(ctx, ctx->view, P, ck, d_pose, &gr, nullptr, true, 1.f, s));
        GSR_TRY(prof_mark(ctx, PROF_PBWD, true, s));
    }
    GSR_TRY(prof_mark(ctx, PROF_ADAM, false, s));
    GSR_TRY(run_adam(ctx, g, &gr, st, &o->adam, sm + SM_MAPLOSS, s));
    GSR_TRY(prof_mark(ctx, PROF_ADAM, true, s));
    return GSR_OK;
}

// Batched iteration over n_kf >= 2 keyframes: every keyframe is binned into
// its own scratch, then ONE persistent forward launch and ONE persistent
// backward launch cover all (keyframe, tile) items, longest lists first; the
// projection backward chains all keyframes' gradients in one pass.
static gsr_status map_iter_multi(gsr_ctx *ctx, gsr_gaussians_mut *g, gsr_adam_state *st, const CamK &ck,
                                 const gsr_keyframe *kfs, int n_kf, const float *w, const gsr_map_opts *o, bool grow,
                                 cudaStream_t s)
{
    const int64_t n = g->n, HW = (int64_t)ck.W * ck.H;
    const int tiles = ck.tiles_x * ck.tiles_y;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    GSR_CUDA(ctx, cudaStreamIsCapturing(s, &cap));
    const bool capturing = cap == cudaStreamCaptureStatusActive;
    if ((int)ctx->mv.size() < n_kf) {
        if (capturing) return gsr_fail(ctx, GSR_ERR_STATE, "keyframe scratch must exist before capture");
        ctx->mv.resize(n_kf);
    }
    GSR_TRY(ensure_buf(ctx, ctx->mv_frames, sizeof(float) * 12 * (size_t)HW * n_kf));
    GSR_TRY(ensure_buf(ctx, ctx->mv_desc, sizeof(BlendView) * n_kf));
    GSR_TRY(ensure_buf(ctx, ctx->mv_pview, sizeof(ProjView) * n_kf));
    GSR_TRY(ensure_buf(ctx, ctx->mv_items, sizeof(u32) * (size_t)tiles * n_kf));
    GSR_TRY(ensure_buf(ctx, ctx->mv_order_hist, order_hist_bytes((int64_t)tiles * n_kf)));
    GSR_TRY(ensure_buf(ctx, ctx->mv_counter, sizeof(u32)));
    float *G = (float *)ctx->grads.p;
    gsr_gaussian_grads gr{G, G + 3 * n, G + 6 * n, G + 10 * n, G + 11 * n};
    float *sm = (float *)ctx->small.p;
    GSR_CUDA(ctx, cudaMemsetAsync(G, 0, sizeof(float) * 14 * n, s));
    GSR_CUDA(ctx, cudaMemsetAsync(sm + SM_MAPLOSS, 0, sizeof(float), s));
    Params P{g->mean, g->log_scale, g->quat, g->opacity_logit, g->rgb, n};

    // the keyframes' binning chains are independent (each has its own scratch):
    // fork them onto side streams, keyframe k on stream k % N_SIDE, and join
    const int ns = std::min(n_kf, gsr_ctx::N_SIDE);
    if (!ctx->fork_ev) {
        if (capturing) return gsr_fail(ctx, GSR_ERR_STATE, "side streams must exist before capture");
        GSR_CUDA(ctx, cudaEventCreateWithFlags(&ctx->fork_ev, cudaEventDisableTiming));
        for (int i = 0; i < gsr_ctx::N_SIDE; ++i) {
            GSR_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->side[i], cudaStreamNonBlocking));
            GSR_CUDA(ctx, cudaEventCreateWithFlags(&ctx->join_ev[i], cudaEventDisableTiming));
        }
    }
    GSR_TRY(prof_mark(ctx, PROF_BIN, false, s));
    GSR_CUDA(ctx, cudaEventRecord(ctx->fork_ev, s));
    for (int i = 0; i < ns; ++i) GSR_CUDA(ctx, cudaStreamWaitEvent(ctx->side[i], ctx->fork_ev, 0));
    for (int k = 0; k < n_kf; ++k) {
        ViewScratch &V = ctx->mv[k];
        cudaStream_t sk = ctx->side[k % ns];
        GSR_TRY(ensure_buf(ctx, V.pose, GSR_POSE_WORDS * sizeof(float)));
        GSR_TRY(launch_set_pose(ctx, (float *)V.pose.p, kfs[k].pose, sk));
        GSR_TRY(run_binning(ctx, V, P, ck, (float *)V.pose.p, grow, sk, false));
    }
    for (int i = 0; i < ns; ++i) {
        GSR_CUDA(ctx, cudaEventRecord(ctx->join_ev[i], ctx->side[i]));
        GSR_CUDA(ctx, cudaStreamWaitEvent(s, ctx->join_ev[i], 0));
    }
    // per-keyframe descriptors (device pointers only; fixed once sized)
    std::vector<BlendView> bv(n_kf);
    std::vector<ProjView> pv(n_kf);
    float *frames = (float *)ctx->mv_frames.p;
    for (int k = 0; k < n_kf; ++k) {
        float *f = frames + (size_t)k * 12 * HW;
        gsr_render_out ro{f, f + 3 * HW, f + 4 * HW, f + 5 * HW, (int32_t *)(f + 6 * HW), nullptr};
        bv[k] = blend_view(ctx->mv[k], &ro, f + 7 * HW, f + 10 * HW, nullptr);
        pv[k] = ProjView{(const int32_t *)ctx->mv[k].rank_of_gid.p, (const float *)ctx->mv[k].g2d.p,
                         (const float *)ctx->mv[k].pose.p};
    }
    const bool same = ctx->mv_desc_host.size() == bv.size() &&
                      memcmp(ctx->mv_desc_host.data(), bv.data(), sizeof(BlendView) * n_kf) == 0 &&
                      memcmp(ctx->mv_pview_host.data(), pv.data(), sizeof(ProjView) * n_kf) == 0;
    if (!same) {
        if (capturing) return gsr_fail(ctx, GSR_ERR_STATE, "keyframe scratch moved during capture");
        GSR_CUDA(ctx, cudaMemcpyAsync(ctx->mv_desc.p, bv.data(), sizeof(BlendView) * n_kf, cudaMemcpyHostToDevice, s));
        GSR_CUDA(ctx, cudaMemcpyAsync(ctx->mv_pview.p, pv.data(), sizeof(ProjView) * n_kf, cudaMemcpyHostToDevice, s));
        GSR_CUDA(ctx, cudaStreamSynchronize(s));  // the host vectors go out of scope
        ctx->mv_desc_host = bv;
        ctx->mv_pview_host = pv;
    }
    const BlendView *dv = (const BlendView *)ctx->mv_desc.p;
    u32 *items = (u32 *)ctx->mv_items.p;
    GSR_TRY(run_make_items(ctx, dv, n_kf, tiles, items, s));
    GSR_TRY(prof_mark(ctx, PROF_BIN, true, s));

    GSR_TRY(prof_mark(ctx, PROF_FWD, false, s));
    GSR_TRY(run_blend_multi(ctx, ck, false, dv, items, n_kf * tiles, (u32 *)ctx->mv_counter.p, s));
    GSR_TRY(prof_mark(ctx, PROF_FWD, true, s));
    GSR_TRY(prof_mark(ctx, PROF_LOSS, false, s));
    // per-keyframe losses on the side streams (own scratch), the scalar sums in order here
    GSR_CUDA(ctx, cudaEventRecord(ctx->fork_ev, s));
    for (int i = 0; i < ns; ++i) GSR_CUDA(ctx, cudaStreamWaitEvent(ctx->side[i], ctx->fork_ev, 0));
    for (int k = 0; k < n_kf; ++k) {
        float *f = frames + (size_t)k * 12 * HW;
        GSR_TRY(run_loss_map_kernels(ctx, &ctx->mv[k], ck.W, ck.H, f, f + 3 * HW, kfs[k].rgb, kfs[k].depth,
                                     o->lambda_ssim, o->w_color, o->w_depth, w[k], f + 7 * HW, f + 10 * HW,
                                     ctx->side[k % ns]));
    }
    for (int i = 0; i < ns; ++i) {
        GSR_CUDA(ctx, cudaEventRecord(ctx->join_ev[i], ctx->side[i]));
        GSR_CUDA(ctx, cudaStreamWaitEvent(s, ctx->join_ev[i], 0));
    }
    for (int k = 0; k < n_kf; ++k)
        GSR_TRY(run_loss_map_final(ctx, &ctx->mv[k], ck.W, ck.H, o->lambda_ssim, o->w_color, o->w_depth, w[k],
                                   sm + SM_MAPLOSS, true, s));
    GSR_TRY(prof_mark(ctx, PROF_LOSS, true, s));
    GSR_TRY(prof_mark(ctx, PROF_BWD, false, s));
    for (int k = 0; k < n_kf; ++k) GSR_TRY(zero_g2d(ctx, ctx->mv[k], s));
    GSR_TRY(run_blend_multi(ctx, ck, true, dv, items, n_kf * tiles, (u32 *)ctx->mv_counter.p, s));
    GSR_TRY(prof_mark(ctx, PROF_BWD, true, s));
    GSR_TRY(prof_mark(ctx, PROF_PBWD, false, s));
    GSR_TRY(run_project_backward_multi(ctx, P, ck, (const ProjView *)ctx->mv_pview.p, n_kf, &gr, s));
    GSR_TRY(prof_mark(ctx, PROF_PBWD, true, s));
    GSR_TRY(prof_mark(ctx, PROF_ADAM, false, s));
    GSR_TRY(run_adam(ctx, g, &gr, st, &o->adam, sm + SM_MAPLOSS, s));
    GSR_TRY(prof_mark(ctx, PROF_ADAM, true, s));
    return GSR_OK;
}

extern "C" gsr_status gsr_map_loss(gsr_ctx *ctx, float *loss_dev, void *stream)
{
    if (!ctx || !loss_dev) return GSR_ERR_INVALID_ARG;
    GSR_CUDA(ctx, cudaMemcpyAsync(loss_dev, (const float *)ctx->small.p + SM_MAPLOSS, sizeof(float),
                                  cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return GSR_OK;
}

extern "C" gsr_status gsr_map_step(gsr_ctx *ctx, gsr_gaussians_mut *g, gsr_adam_state *st, const gsr_camera *cam,
                                   const gsr_keyframe *kfs, int32_t n_kf, const float *kf_weights, int32_t n_iters,
                                   const gsr_map_opts *opt, gsr_map_stats *out, void *stream)
{
    if (!ctx) return GSR_ERR_INVALID_ARG;
    if (!g || !st || !kfs || n_kf <= 0 || n_kf > 64 || n_iters < 0 || !opt)
        return gsr_fail(ctx, GSR_ERR_INVALID_ARG, "invalid mapping arguments");
    gsr_gaussians gc{g->mean, g->log_scale, g->quat, g->opacity_logit, g->rgb, g->n};
    GSR_TRY(check_gaussians(ctx, &gc));
    GSR_TRY(check_camera(ctx, cam));
    for (int k = 0; k < n_kf; ++k)
        if (!kfs[k].rgb || !kfs[k].depth) return gsr_fail(ctx, GSR_ERR_INVALID_ARG, "null keyframe image");
    cudaStream_t s = (cudaStream_t)stream;
    forget_forward(ctx);
    float w[64];
    for (int k = 0; k < n_kf; ++k) w[k] = kf_weights ? kf_weights[k] : 1.f / (float)n_kf;
    CamK ck = make_camk(*cam, ctx->opt.tile_w, ctx->opt.tile_h);
    GSR_TRY(ensure_buf(ctx, ctx->grads, sizeof(float) * 14 * (size_t)(g->n > 0 ? g->n : 1)));
    GSR_TRY(ensure_view_pose(ctx));
    const bool grow = !ctx->opt.fixed_capacity;
    // the graph is keyed by every pointer, size and option it bakes in
    uint64_t key = 1469598103934665603ull;
    auto mix = [&key](uint64_t v) { key = (key ^ v) * 1099511628211ull; };
    const void *ptrs[] = {g->mean, g->log_scale, g->quat, g->opacity_logit, g->rgb, st->m_mean, st->v_mean, st->step};
    for (const void *q : ptrs) mix((uint64_t)(uintptr_t)q);
    mix((uint64_t)g->n);
    mix((uint64_t)n_kf);
    mix((uint64_t)ctx->prof);
    {
        uint64_t h = 0;
        const unsigned char *b = (const unsigned char *)cam;
        for (size_t i = 0; i < sizeof(*cam); ++i) h = h * 131 + b[i];
        mix(h);
        b = (const unsigned char *)opt;
        for (size_t i = 0; i < sizeof(*opt); ++i) h = h * 131 + b[i];
        mix(h);
    }
    for (int k = 0; k < n_kf; ++k) {
        mix((uint64_t)(uintptr_t)kfs[k].rgb);
        mix((uint64_t)(uintptr_t)kfs[k].depth);
        uint64_t h = 0;
        const unsigned char *b = (const unsigned char *)&kfs[k].pose;
        for (size_t i = 0; i < sizeof(gsr_pose); ++i) h = h * 131 + b[i];
        mix(h);
        uint32_t wb;
        memcpy(&wb, &w[k], 4);
        mix(wb);
    }
    for (int32_t it = 0; it < n_iters; ++it) {
        // the first iteration with a new key runs eagerly (it sizes the scratch);
        // later ones are captured once and replayed
        if (opt->use_graph && ctx->map_sized_key == key) {
            if (!ctx->map_graph || ctx->map_key != key) {
                if (ctx->map_graph) cudaGraphExecDestroy(ctx->map_graph);
                ctx->map_graph = nullptr;
                cudaStream_t cs;
                GSR_CUDA(ctx, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
                GSR_CUDA(ctx, cudaStreamSynchronize(s));
                GSR_CUDA(ctx, cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
                const int64_t l0 = ctx->launches;
                gsr_status stt = n_kf >= 2 ? map_iter_multi(ctx, g, st, ck, kfs, n_kf, w, opt, false, cs)
                                           : map_iter(ctx, g, st, ck, kfs, n_kf, w, opt, false, cs);
                ctx->map_graph_kernels = ctx->launches - l0;
                ctx->launches = l0;
                cudaGraph_t graph = nullptr;
                cudaError_t e = cudaStreamEndCapture(cs, &graph);
                cudaStreamDestroy(cs);
                if (stt != GSR_OK) {
                    if (graph) cudaGraphDestroy(graph);
                    return stt;
                }
                GSR_CUDA(ctx, e);
                e = cudaGraphInstantiate(&ctx->map_graph, graph, 0);
                cudaGraphDestroy(graph);
                GSR_CUDA(ctx, e);
                ctx->map_key = key;
            }
            GSR_CUDA(ctx, cudaGraphLaunch(ctx->map_graph, s));
            ctx->launches += ctx->map_graph_kernels;
        } else {
            if (n_kf >= 2) GSR_TRY(map_iter_multi(ctx, g, st, ck, kfs, n_kf, w, opt, grow, s));
            else GSR_TRY(map_iter(ctx, g, st, ck, kfs, n_kf, w, opt, grow, s));
            ctx->map_sized_key = key;
        }
    }
    if (out) {
        float *sm = (float *)ctx->small.p;
        GSR_CUDA(ctx, cudaMemcpyAsync(ctx->host_pinned + 20, sm + SM_MAPLOSS, sizeof(float), cudaMemcpyDeviceToHost, s));
        GSR_TRY(take_status(ctx, s));
        out->loss_last = ((const float *)ctx->host_pinned)[20];
        out->iters = n_iters;
    }
    return GSR_OK;
}

// --------------------------------------------------------------- autotune
extern "C" gsr_status gsr_autotune(gsr_ctx *ctx, const gsr_gaussians *g, const gsr_camera *cam, const gsr_pose *poses,
                                   int32_t n_poses, int32_t reps, gsr_tune_result *best, gsr_tune_result *all,
                                   int32_t n_all, void *stream)
{
    if (!ctx) return GSR_ERR_INVALID_ARG;
    GSR_TRY(check_gaussians(ctx, g));
    if (!cam || !poses || n_poses <= 0 || reps <= 0 || !best || (n_all > 0 && !all))
        return gsr_fail(ctx, GSR_ERR_INVALID_ARG, "invalid autotune arguments");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t HW = (int64_t)cam->width * cam->height;
    FrameBufs f;
    GSR_TRY(frame_bufs(ctx, HW, f));
    GSR_TRY(ensure_buf(ctx, ctx->grads, sizeof(float) * 14 * (size_t)(g->n > 0 ? g->n : 1)));
    float *G = (float *)ctx->grads.p;
    const int64_t n = g->n;
    gsr_gaussian_grads dg{G, G + 3 * n, G + 6 * n, G + 10 * n, G + 11 * n};
    // dL/dpixel = 1 everywhere (the d_rgb / d_depth planes of the frame buffers)
    {
        std::vector<float> ones((size_t)HW * 4, 1.f);
        GSR_CUDA(ctx, cudaMemcpy(f.d_rgb, ones.data(), sizeof(float) * 4 * HW, cudaMemcpyHostToDevice));
    }
    const int tiles[4][2] = {{16, 16}, {8, 8}, {16, 8}, {32, 8}};
    const int batches[4] = {32, 64, 128, 256};
    const gsr_options saved = ctx->opt;
    const int saved_pf = ctx->ppt_fwd, saved_pb = ctx->ppt_bwd;
    cudaEvent_t ev[3];
    for (int i = 0; i < 3; ++i) GSR_CUDA(ctx, cudaEventCreate(&ev[i]));
    gsr_tune_result win{};
    win.ms = 3.4e38f;
    int idx = 0;
    gsr_status st = GSR_OK;
    gsr_render_out ro{f.rgb, f.depth, f.alpha, f.T, f.last, nullptr};
    for (int ti = 0; ti < 4 && st == GSR_OK; ++ti)
        for (int bi = 0; bi < 4 && st == GSR_OK; ++bi) {
            ctx->opt.tile_w = tiles[ti][0];
            ctx->opt.tile_h = tiles[ti][1];
            ctx->opt.batch = batches[bi];
            if (check_camera(ctx, cam) != GSR_OK) continue;  // too many tiles for this shape
            float tf[3] = {0.f, 0.f, 0.f}, tb[3] = {0.f, 0.f, 0.f};
            for (int ppt = 1; ppt <= 2 && st == GSR_OK; ++ppt) {
                ctx->ppt_fwd = ctx->ppt_bwd = ppt;
                for (int r = 0; r <= reps && st == GSR_OK; ++r)
                    for (int k = 0; k < n_poses && st == GSR_OK; ++k) {
                        st = gsr_cuda_check(ctx, cudaEventRecord(ev[0], s), "event");
                        if (st == GSR_OK) st = gsr_render_forward(ctx, g, cam, &poses[k], &ro, stream);
                        if (st == GSR_OK) st = gsr_cuda_check(ctx, cudaEventRecord(ev[1], s), "event");
                        if (st == GSR_OK)
                            st = gsr_render_backward(ctx, g, cam, &poses[k], &ro, f.d_rgb, f.d_depth, nullptr, &dg,
                                                     nullptr, stream);
                        if (st == GSR_OK) st = gsr_cuda_check(ctx, cudaEventRecord(ev[2], s), "event");
                        if (st == GSR_OK) st = gsr_cuda_check(ctx, cudaEventSynchronize(ev[2]), "event");
                        float a = 0.f, b = 0.f;
                        if (st == GSR_OK) st = gsr_cuda_check(ctx, cudaEventElapsedTime(&a, ev[0], ev[1]), "event");
                        if (st == GSR_OK) st = gsr_cuda_check(ctx, cudaEventElapsedTime(&b, ev[1], ev[2]), "event");
                        if (r > 0) {  // r = 0 warms up (and sizes the scratch)
                            tf[ppt] += a;
                            tb[ppt] += b;
                        }
                    }
            }
            if (st != GSR_OK) break;
            gsr_tune_result res{};
            res.tile_w = tiles[ti][0];
            res.tile_h = tiles[ti][1];
            res.batch = batches[bi];
            res.ppt_fwd = tf[1] <= tf[2] ? 1 : 2;
            res.ppt_bwd = tb[1] <= tb[2] ? 1 : 2;
            res.ms_fwd = tf[res.ppt_fwd] / (float)reps;
            res.ms_bwd = tb[res.ppt_bwd] / (float)reps;
            res.ms = res.ms_fwd + res.ms_bwd;
            if (idx < n_all) all[idx] = res;
            ++idx;
            if (res.ms < win.ms) win = res;
        }
    for (int i = 0; i < 3; ++i) cudaEventDestroy(ev[i]);
    ctx->opt = saved;
    ctx->ppt_fwd = saved_pf;
    ctx->ppt_bwd = saved_pb;
    if (st != GSR_OK) return st;
    ctx->opt.tile_w = win.tile_w;
    ctx->opt.tile_h = win.tile_h;
    ctx->opt.batch = win.batch;
    ctx->opt.ppt_fwd = ctx->ppt_fwd = win.ppt_fwd;
    ctx->opt.ppt_bwd = ctx->ppt_bwd = win.ppt_bwd;
    // graphs baked the old configuration
    if (ctx->map_graph) cudaGraphExecDestroy(ctx->map_graph);
    if (ctx->track_graph) cudaGraphExecDestroy(ctx->track_graph);
    ctx->map_graph = ctx->track_graph = nullptr;
    ctx->map_key = ctx->map_sized_key = ctx->track_key = 0;
    forget_forward(ctx);
    *best = win;
    return GSR_OK;
}
