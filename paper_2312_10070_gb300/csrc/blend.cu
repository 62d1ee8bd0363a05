// blend.cu -- per-tile front-to-back alpha blending (forward, Sec. 3.1
// Eq. (color_blending) and the depth rendering of Sec. 3.4) and its
// back-to-front replay (backward, Sec. 3.4 adjoints).
//
// One CTA per pixel tile, one thread per pixel.  Gaussian records of the
// tile's depth-ordered list are staged cooperatively in shared memory, BATCH
// at a time; a CTA stops loading once every pixel's transmittance fell below
// the stop threshold.  The backward walks the same list from the largest
// last-composited index of the tile down to 0, recovering T_j = T_{j+1} /
// (1 - alpha_j) from the saved final transmittance, and reduces the
// per-pixel contributions of each Gaussian across the warp with shuffles
// before one atomic add per warp and gradient component.
#include "gsr_internal.cuh"

namespace {

template <int TW, int TH, int BATCH>
__global__ void __launch_bounds__(TW *TH) k_blend_fwd(CamK ck, const uint2 *__restrict__ ranges,
                                                      const u32 *__restrict__ tvals,
                                                      const float4 *__restrict__ rec,
                                                      float *__restrict__ out_rgb, float *__restrict__ out_depth,
                                                      float *__restrict__ out_alpha, float *__restrict__ out_T,
                                                      int32_t *__restrict__ out_last, int32_t *__restrict__ out_nc)
{
    constexpr int NT = TW * TH;
    __shared__ float4 sA[BATCH], sB[BATCH], sC[BATCH];
    const int tile = blockIdx.x;
    const int tx = tile % ck.tiles_x, ty = tile / ck.tiles_x;
    const int ix = tx * TW + (int)threadIdx.x % TW, iy = ty * TH + (int)threadIdx.x / TW;
    const bool inside = ix < ck.W && iy < ck.H;
    const float px = (float)ix + 0.5f, py = (float)iy + 0.5f;
    const uint2 rg = ranges[tile];
    const int n = (int)(rg.y - rg.x);
    float T = 1.f, c0 = 0.f, c1 = 0.f, c2 = 0.f, d = 0.f;
    int last = -1, nc = 0;
    bool done = !inside;
    for (int base = 0; base < n; base += BATCH) {
        if (__syncthreads_count(done) == NT) break;
        for (int k = threadIdx.x; k < BATCH; k += NT) {
            const int j = base + k;
            if (j < n) {
                const int64_t r = tvals[rg.x + j];
                sA[k] = rec[3 * r];
                sB[k] = rec[3 * r + 1];
                sC[k] = rec[3 * r + 2];
            }
        }
        __syncthreads();
        const int cnt = min(BATCH, n - base);
        if (!done) {
            for (int k = 0; k < cnt; ++k) {
                const float4 a = sA[k], b = sB[k];
                const Eval e = eval_gaussian(px, py, a.x, a.y, a.z, a.w, b.x, b.y);
                if (!e.use) continue;
                const float Tn = __fmul_rn(T, __fsub_rn(1.f, e.alpha));
                if (Tn < GSR_T_STOP) {
                    done = true;
                    break;
                }
                const float4 c = sC[k];
                const float w = e.alpha * T;
                c0 = fmaf(c.x, w, c0);
                c1 = fmaf(c.y, w, c1);
                c2 = fmaf(c.z, w, c2);
                d = fmaf(b.z, w, d);
                T = Tn;
                last = base + k;
                ++nc;
            }
        }
    }
    if (inside) {
        const int64_t HW = (int64_t)ck.W * ck.H, p = (int64_t)iy * ck.W + ix;
        out_rgb[p] = c0;
        out_rgb[HW + p] = c1;
        out_rgb[2 * HW + p] = c2;
        out_depth[p] = d;
        out_alpha[p] = 1.f - T;
        out_T[p] = T;
        out_last[p] = last;
        if (out_nc) out_nc[p] = nc;
    }
}

template <int NV>
__device__ __forceinline__ void warp_sum_and_add(float (&v)[NV], const int (&slot)[NV], float *dst)
{
#pragma unroll
    for (int i = 0; i < NV; ++i) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
    }
    const int lane = threadIdx.x & 31;
    float mine = 0.f;
    int s = 0;
#pragma unroll
    for (int i = 0; i < NV; ++i)
        if (lane == i) {
            mine = v[i];
            s = slot[i];
        }
    if (lane < NV && mine != 0.f) atomicAdd(dst + s, mine);
}

// POSE_ONLY: the tracker needs only the gradients feeding the pose
// (u, v, conic, depth); colour and opacity gradients are skipped.
template <int TW, int TH, int BATCH, bool POSE_ONLY>
__global__ void __launch_bounds__(TW *TH) k_blend_bwd(CamK ck, const uint2 *__restrict__ ranges,
                                                      const u32 *__restrict__ tvals,
                                                      const float4 *__restrict__ rec,
                                                      const float *__restrict__ fin_T,
                                                      const int32_t *__restrict__ last_idx,
                                                      const float *__restrict__ d_rgb,
                                                      const float *__restrict__ d_depth,
                                                      const float *__restrict__ d_alpha, float *__restrict__ g2d)
{
    constexpr int NT = TW * TH;
    __shared__ float4 sA[BATCH], sB[BATCH], sC[BATCH];
    __shared__ u32 sR[BATCH];
    __shared__ int s_max;
    const int tile = blockIdx.x;
    const int tx = tile % ck.tiles_x, ty = tile / ck.tiles_x;
    const int ix = tx * TW + (int)threadIdx.x % TW, iy = ty * TH + (int)threadIdx.x / TW;
    const bool inside = ix < ck.W && iy < ck.H;
    const float px = (float)ix + 0.5f, py = (float)iy + 0.5f;
    const uint2 rg = ranges[tile];
    const int64_t HW = (int64_t)ck.W * ck.H, p = (int64_t)iy * ck.W + ix;
    int L = -1;
    float Tf = 1.f, g0 = 0.f, g1 = 0.f, g2 = 0.f, gd = 0.f, ga = 0.f;
    if (inside) {
        L = last_idx[p];
        Tf = fin_T[p];
        if (d_rgb) {
            g0 = d_rgb[p];
            g1 = d_rgb[HW + p];
            g2 = d_rgb[2 * HW + p];
        }
        if (d_depth) gd = d_depth[p];
        if (d_alpha) ga = d_alpha[p];
    }
    if (threadIdx.x == 0) s_max = -1;
    __syncthreads();
    const int wmax = __reduce_max_sync(0xffffffffu, L);
    if ((threadIdx.x & 31) == 0) atomicMax(&s_max, wmax);
    __syncthreads();
    const int nend = min(s_max + 1, (int)(rg.y - rg.x));  // saved state never reads past the list
    float T = Tf, S0 = 0.f, S1 = 0.f, S2 = 0.f, Sd = 0.f;
    const float gaT = ga * Tf;
    for (int bend = nend; bend > 0; bend -= BATCH) {
        const int bstart = max(0, bend - BATCH);
        const int cnt = bend - bstart;
        __syncthreads();
        for (int k = threadIdx.x; k < cnt; k += NT) {
            const u32 r = tvals[rg.x + bstart + k];
            sR[k] = r;
            sA[k] = rec[3 * (int64_t)r];
            sB[k] = rec[3 * (int64_t)r + 1];
            sC[k] = rec[3 * (int64_t)r + 2];
        }
        __syncthreads();
        for (int k = cnt - 1; k >= 0; --k) {
            const int j = bstart + k;
            float gu = 0.f, gv = 0.f, gca = 0.f, gcb = 0.f, gcc = 0.f, gop = 0.f, gr = 0.f, gg = 0.f,
                  gb = 0.f, gz = 0.f;
            bool contrib = false;
            if (j <= L) {
                const float4 a = sA[k], b = sB[k];
                const Eval e = eval_gaussian(px, py, a.x, a.y, a.z, a.w, b.x, b.y);
                if (e.use) {
                    contrib = true;
                    const float4 c = sC[k];
                    const float om = 1.f - e.alpha;
                    const float iom = 1.f / om;
                    T = T * iom;  // T_j
                    const float w = e.alpha * T;
                    float dLda = g0 * (c.x * T - S0 * iom) + g1 * (c.y * T - S1 * iom) + g2 * (c.z * T - S2 * iom)
                               + gd * (b.z * T - Sd * iom) + gaT * iom;
                    S0 = fmaf(c.x, w, S0);
                    S1 = fmaf(c.y, w, S1);
                    S2 = fmaf(c.z, w, S2);
                    Sd = fmaf(b.z, w, Sd);
                    gz = gd * w;
                    if (!POSE_ONLY) {
                        gr = g0 * w;
                        gg = g1 * w;
                        gb = g2 * w;
                    }
                    if (e.G <= GSR_ALPHA_MAX) {
                        if (!POSE_ONLY) gop = dLda * e.ex;
                        const float ds = -dLda * e.G;
                        gu = -ds * (a.z * e.dx + a.w * e.dy);
                        gv = -ds * (a.w * e.dx + b.x * e.dy);
                        gca = 0.5f * ds * e.dx * e.dx;
                        gcb = ds * e.dx * e.dy;
                        gcc = 0.5f * ds * e.dy * e.dy;
                    }
                }
            }
            if (__ballot_sync(0xffffffffu, contrib)) {
                float *dst = g2d + 12 * (int64_t)sR[k];
                if (POSE_ONLY) {
                    float v[6] = {gu, gv, gca, gcb, gcc, gz};
                    const int slot[6] = {0, 1, 2, 3, 4, 9};
                    warp_sum_and_add<6>(v, slot, dst);
                } else {
                    float v[10] = {gu, gv, gca, gcb, gcc, gop, gr, gg, gb, gz};
                    const int slot[10] = {0, 1, 2, 3, 4, 5, 6, 7, 8, 9};
                    warp_sum_and_add<10>(v, slot, dst);
                }
            }
        }
    }
}

__global__ void k_zero_g2d(int64_t cap, const u32 *__restrict__ d_v, float4 *__restrict__ g2d)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t n = (int64_t)*d_v * 3;
    if (i < n && i < cap * 3) g2d[i] = make_float4(0.f, 0.f, 0.f, 0.f);
}

template <int TW, int TH, int BATCH>
gsr_status launch_fwd(gsr_ctx *ctx, const CamK &ck, gsr_render_out *o, cudaStream_t s)
{
    ViewScratch &V = ctx->view;
    const unsigned tiles = (unsigned)(ck.tiles_x * ck.tiles_y);
    k_blend_fwd<TW, TH, BATCH><<<tiles, TW * TH, 0, s>>>(ck, (uint2 *)V.ranges.p, (u32 *)V.tvals[0].p,
                                                        (float4 *)V.rec_sorted.p, o->rgb, o->depth, o->alpha,
                                                        o->final_T, o->last_idx, o->n_contrib);
    ctx->launches += 1;
    GSR_LAUNCHED(ctx);
    return GSR_OK;
}

template <int TW, int TH, int BATCH>
gsr_status launch_bwd(gsr_ctx *ctx, const CamK &ck, const gsr_render_out *sv, const float *d_rgb,
                      const float *d_depth, const float *d_alpha, bool pose_only, cudaStream_t s)
{
    ViewScratch &V = ctx->view;
    const unsigned tiles = (unsigned)(ck.tiles_x * ck.tiles_y);
    if (pose_only)
        k_blend_bwd<TW, TH, BATCH, true><<<tiles, TW * TH, 0, s>>>(
            ck, (uint2 *)V.ranges.p, (u32 *)V.tvals[0].p, (float4 *)V.rec_sorted.p, sv->final_T, sv->last_idx,
            d_rgb, d_depth, d_alpha, (float *)V.g2d.p);
    else
        k_blend_bwd<TW, TH, BATCH, false><<<tiles, TW * TH, 0, s>>>(
            ck, (uint2 *)V.ranges.p, (u32 *)V.tvals[0].p, (float4 *)V.rec_sorted.p, sv->final_T, sv->last_idx,
            d_rgb, d_depth, d_alpha, (float *)V.g2d.p);
    ctx->launches += 1;
    GSR_LAUNCHED(ctx);
    return GSR_OK;
}

template <int TW, int TH>
gsr_status dispatch_batch_fwd(gsr_ctx *ctx, const CamK &ck, gsr_render_out *o, cudaStream_t s)
{
    switch (ctx->opt.batch) {
    case 32: return launch_fwd<TW, TH, 32>(ctx, ck, o, s);
    case 64: return launch_fwd<TW, TH, 64>(ctx, ck, o, s);
    case 128: return launch_fwd<TW, TH, 128>(ctx, ck, o, s);
    default: return launch_fwd<TW, TH, 256>(ctx, ck, o, s);
    }
}

template <int TW, int TH>
gsr_status dispatch_batch_bwd(gsr_ctx *ctx, const CamK &ck, const gsr_render_out *sv, const float *a,
                              const float *b, const float *c, bool po, cudaStream_t s)
{
    switch (ctx->opt.batch) {
    case 32: return launch_bwd<TW, TH, 32>(ctx, ck, sv, a, b, c, po, s);
    case 64: return launch_bwd<TW, TH, 64>(ctx, ck, sv, a, b, c, po, s);
    case 128: return launch_bwd<TW, TH, 128>(ctx, ck, sv, a, b, c, po, s);
    default: return launch_bwd<TW, TH, 256>(ctx, ck, sv, a, b, c, po, s);
    }
}

} // namespace

gsr_status run_blend_forward(gsr_ctx *ctx, const Params &, const CamK &ck, gsr_render_out *o, cudaStream_t s)
{
    const int tw = ctx->opt.tile_w, th = ctx->opt.tile_h;
    if (tw == 16 && th == 16) return dispatch_batch_fwd<16, 16>(ctx, ck, o, s);
    if (tw == 8 && th == 8) return dispatch_batch_fwd<8, 8>(ctx, ck, o, s);
    if (tw == 16 && th == 8) return dispatch_batch_fwd<16, 8>(ctx, ck, o, s);
    if (tw == 32 && th == 8) return dispatch_batch_fwd<32, 8>(ctx, ck, o, s);
    return gsr_fail(ctx, GSR_ERR_INVALID_ARG, "unsupported tile size");
}

gsr_status run_blend_backward(gsr_ctx *ctx, const CamK &ck, const gsr_render_out *sv, const float *d_rgb,
                              const float *d_depth, const float *d_alpha, bool pose_only, cudaStream_t s)
{
    ViewScratch &V = ctx->view;
    k_zero_g2d<<<(unsigned)ceil_div(V.cap_n * 3, 256), 256, 0, s>>>(V.cap_n, (u32 *)V.counters.p + CNT_VISIBLE,
                                                                    (float4 *)V.g2d.p);
    ctx->launches += 1;
    GSR_LAUNCHED(ctx);
    const int tw = ctx->opt.tile_w, th = ctx->opt.tile_h;
    if (tw == 16 && th == 16) return dispatch_batch_bwd<16, 16>(ctx, ck, sv, d_rgb, d_depth, d_alpha, pose_only, s);
    if (tw == 8 && th == 8) return dispatch_batch_bwd<8, 8>(ctx, ck, sv, d_rgb, d_depth, d_alpha, pose_only, s);
    if (tw == 16 && th == 8) return dispatch_batch_bwd<16, 8>(ctx, ck, sv, d_rgb, d_depth, d_alpha, pose_only, s);
    if (tw == 32 && th == 8) return dispatch_batch_bwd<32, 8>(ctx, ck, sv, d_rgb, d_depth, d_alpha, pose_only, s);
    return gsr_fail(ctx, GSR_ERR_INVALID_ARG, "unsupported tile size");
}
