// seed.cu -- sub-map seeding (Sec. 3.2 densification; constants of Sec. 4 and
// supplementary Sec. A).  See gsr_seed_keyframe in include/gsr.h for the
// exact rules.
//
// Pipeline (all counts stay on the device until the single read-back that
// checks the sub-map capacity):
//   eligible pixels -> scan -> 32-bit sampling keys (splitmix64) -> stable
//   radix sort -> the first m pixels are selected; on a sub-map's first
//   keyframe also the m_c pixels of largest luminance gradient (sort key =
//   complemented float bits, so larger gradients come first) -> scan of the
//   selection -> back-projected candidates -> hashed grid of the existing
//   means (cell size rho, sorted by cell hash) -> 27-cell radius test ->
//   scan of the kept flags -> new means appended -> hashed grid of all means
//   (cell size 2 rho) -> exact nearest-neighbour ring search -> scales.
// A hash collision only adds points to a cell's run; every candidate
// distance is computed exactly, so collisions never change a result.
#include <math.h>

#include "gsr_internal.cuh"

namespace {

// splitmix64 (Steele, Lea and Flood, OOPSLA 2014) as a counter-based hash
__device__ __forceinline__ uint64_t splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ u32 cell_hash(int cx, int cy, int cz)
{
    const uint64_t k = ((uint64_t)(cx & 0x1FFFFF) << 42) | ((uint64_t)(cy & 0x1FFFFF) << 21) |
                       (uint64_t)(cz & 0x1FFFFF);
    return (u32)(splitmix64(k) >> 32);
}

__device__ __forceinline__ int cell_of(float x, float inv_h) { return (int)floorf(x * inv_h); }

// first index j in [0, n) with keys[j] >= key
__device__ __forceinline__ int64_t lower_bound(const u32 *__restrict__ keys, int64_t n, u32 key)
{
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (keys[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ int64_t dev_count(int64_t cap, const u32 *d_n) { return min(cap, (int64_t)*d_n); }

__global__ void k_seed_eligible(int64_t P, const float *__restrict__ depth, const float *__restrict__ alpha,
                                float alpha_n, u32 *__restrict__ flag)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    bool e = depth[p] > 0.f;
    if (alpha) e = e && alpha[p] < alpha_n;
    flag[p] = e ? 1u : 0u;
}

// sort pairs of the eligible pixels: uniform keys, or gradient keys
__global__ void k_seed_keys(int W, int H, const u32 *__restrict__ flag, const u32 *__restrict__ off,
                            const float *__restrict__ rgb, uint64_t seed, int gradient, u32 *__restrict__ keys,
                            u32 *__restrict__ vals)
{
    const int64_t P = (int64_t)W * H;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P || !flag[p]) return;
    const u32 i = off[p];
    u32 key;
    if (!gradient) {
        key = (u32)(splitmix64(seed + (uint64_t)p) >> 32);
    } else {
        const int r = (int)(p / W), c = (int)(p % W);
        float g2 = 0.f;
        if (r > 0 && r < H - 1 && c > 0 && c < W - 1) {
            auto Y = [&](int64_t q) { return (rgb[q] + rgb[P + q] + rgb[2 * P + q]) / 3.f; };
            const float gx = (Y(p + 1) - Y(p - 1)) * 0.5f, gy = (Y(p + W) - Y(p - W)) * 0.5f;
            g2 = gx * gx + gy * gy;
        }
        key = ~__float_as_uint(g2);  // g2 >= 0: larger gradient, smaller key
    }
    keys[i] = key;
    vals[i] = (u32)p;
}

__global__ void k_seed_mark(int64_t cap, const u32 *__restrict__ d_n, const u32 *__restrict__ sorted_vals, int64_t m,
                            u32 *__restrict__ sel)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= min(m, dev_count(cap, d_n))) return;
    sel[sorted_vals[i]] = 1u;
}

struct SeedPose {
    float R[9], t[3];
};

__global__ void k_seed_backproject(int W, int H, const u32 *__restrict__ sel, const u32 *__restrict__ off,
                                   const float *__restrict__ depth, float fx, float fy, float cx, float cy, SeedPose ps,
                                   u32 *__restrict__ cand_pix, float4 *__restrict__ cand_pts)
{
    const int64_t P = (int64_t)W * H;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P || !sel[p]) return;
    const u32 i = off[p];
    const int r = (int)(p / W), c = (int)(p % W);
    const float z = depth[p];
    const float d0 = ((float)c + 0.5f - cx) * z / fx - ps.t[0];
    const float d1 = ((float)r + 0.5f - cy) * z / fy - ps.t[1];
    const float d2 = z - ps.t[2];
    cand_pix[i] = (u32)p;
    cand_pts[i] = make_float4(ps.R[0] * d0 + ps.R[3] * d1 + ps.R[6] * d2, ps.R[1] * d0 + ps.R[4] * d1 + ps.R[7] * d2,
                              ps.R[2] * d0 + ps.R[5] * d1 + ps.R[8] * d2, 0.f);
}

__global__ void k_cell_keys(int64_t n, const float *__restrict__ means, float inv_h, u32 *__restrict__ keys,
                            u32 *__restrict__ vals)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    keys[i] = cell_hash(cell_of(means[3 * i], inv_h), cell_of(means[3 * i + 1], inv_h), cell_of(means[3 * i + 2], inv_h));
    vals[i] = (u32)i;
}

// smallest squared distance from q to the means listed in cell (cx, cy, cz)
__device__ __forceinline__ float cell_min_d2(float qx, float qy, float qz, int cx, int cy, int cz,
                                             const float *__restrict__ means, const u32 *__restrict__ gk,
                                             const u32 *__restrict__ gv, int64_t n, int64_t skip, float best)
{
    const u32 key = cell_hash(cx, cy, cz);
    for (int64_t j = lower_bound(gk, n, key); j < n && gk[j] == key; ++j) {
        const int64_t m = gv[j];
        if (m == skip) continue;
        const float dx = qx - means[3 * m], dy = qy - means[3 * m + 1], dz = qz - means[3 * m + 2];
        best = fminf(best, dx * dx + dy * dy + dz * dz);
    }
    return best;
}

__global__ void k_seed_reject(int64_t cap, const u32 *__restrict__ d_n, const float4 *__restrict__ pts,
                              const float *__restrict__ means, const u32 *__restrict__ gk, const u32 *__restrict__ gv,
                              int64_t n_grid, float inv_h, float rho2, u32 *__restrict__ keep, float *__restrict__ d2)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= dev_count(cap, d_n)) return;
    const float4 q = pts[i];
    const int cx = cell_of(q.x, inv_h), cy = cell_of(q.y, inv_h), cz = cell_of(q.z, inv_h);
    float best = INFINITY;
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx)
                best = cell_min_d2(q.x, q.y, q.z, cx + dx, cy + dy, cz + dz, means, gk, gv, n_grid, -1, best);
    keep[i] = best < rho2 ? 0u : 1u;
    d2[i] = best;
}

// appended Gaussians (all but the scales)
__global__ void k_seed_write(int64_t cap, const u32 *__restrict__ d_n, const u32 *__restrict__ keep,
                             const u32 *__restrict__ keep_off, const float4 *__restrict__ pts,
                             const u32 *__restrict__ cand_pix, const float *__restrict__ rgb, int64_t P,
                             int64_t n_exist, float *__restrict__ mean, float *__restrict__ quat,
                             float *__restrict__ logit, float *__restrict__ col)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= dev_count(cap, d_n) || !keep[i]) return;
    const int64_t o = n_exist + keep_off[i];
    const float4 q = pts[i];
    const int64_t p = cand_pix[i];
    mean[3 * o] = q.x;
    mean[3 * o + 1] = q.y;
    mean[3 * o + 2] = q.z;
    quat[4 * o] = 1.f;
    quat[4 * o + 1] = 0.f;
    quat[4 * o + 2] = 0.f;
    quat[4 * o + 3] = 0.f;
    logit[o] = 0.f;
    col[3 * o] = rgb[p];
    col[3 * o + 1] = rgb[P + p];
    col[3 * o + 2] = rgb[2 * P + p];
}

// exact nearest neighbour by shells of cells (Chebyshev radius r) around the
// query's cell: after shell r every unvisited mean is farther than r h
// (less a rounding margin), so the search stops once the best is within it
__global__ void k_seed_nn(int64_t n_new, int64_t n_exist, const float *__restrict__ means, const u32 *__restrict__ gk,
                          const u32 *__restrict__ gv, int64_t n_grid, float h, float inv_h, int R, float s_min,
                          float s_max, float *__restrict__ log_scale)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_new) return;
    const int64_t self = n_exist + i;
    const float qx = means[3 * self], qy = means[3 * self + 1], qz = means[3 * self + 2];
    const int cx = cell_of(qx, inv_h), cy = cell_of(qy, inv_h), cz = cell_of(qz, inv_h);
    float best = INFINITY;
    for (int r = 0; r <= R; ++r) {
        for (int dz = -r; dz <= r; ++dz)
            for (int dy = -r; dy <= r; ++dy) {
                const bool face = dz == -r || dz == r || dy == -r || dy == r;
                for (int dx = -r; dx <= r; dx += (face || r == 0) ? 1 : 2 * r)
                    best = cell_min_d2(qx, qy, qz, cx + dx, cy + dy, cz + dz, means, gk, gv, n_grid, self, best);
            }
        const float lim = (float)r * h * (1.f - 1e-4f);
        if (best <= lim * lim) break;
    }
    const float d = fminf(fmaxf(sqrtf(best), s_min), s_max);  // +inf -> s_max
    const float ls = logf(d);
    log_scale[3 * self] = ls;
    log_scale[3 * self + 1] = ls;
    log_scale[3 * self + 2] = ls;
}

unsigned nblk(int64_t n, int t = 256) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

gsr_status sort_cells(gsr_ctx *ctx, SeedScratch &S, const float *means, int64_t n, float inv_h, cudaStream_t s)
{
    if (n <= 0) return GSR_OK;
    u32 *keys[2] = {(u32 *)S.keys[0].p, (u32 *)S.keys[1].p}, *vals[2] = {(u32 *)S.vals[0].p, (u32 *)S.vals[1].p};
    k_cell_keys<<<nblk(n), 256, 0, s>>>(n, means, inv_h, keys[0], vals[0]);
    ctx->launches += 1;
    GSR_LAUNCHED(ctx);
    return radix_sort_pairs(ctx, keys, vals, n, nullptr, 32, s);
}

} // namespace

extern "C" {

void gsr_default_seed_opts(gsr_seed_opts *o)
{
    if (!o) return;
    o->first_keyframe = 1;
    o->m_u = 100000;
    o->m_c = 50000;
    o->m_k = 100000;
    o->alpha_n = 0.6f;
    o->rho = 0.01f;
    o->s_min = 1e-4f;
    o->s_max = 0.1f;
    o->seed = 0;
}

gsr_status gsr_seed_keyframe(gsr_ctx *ctx, const gsr_camera *cam, const gsr_pose *pose, const float *rgb,
                             const float *depth, const float *alpha, const gsr_seed_opts *opt, gsr_gaussians_mut *g,
                             int64_t n_existing, int64_t capacity, gsr_seed_stats *out, void *stream)
{
    if (!ctx || !cam || !pose || !rgb || !depth || !opt || !g) return GSR_ERR_INVALID_ARG;
    if (!g->mean || !g->log_scale || !g->quat || !g->opacity_logit || !g->rgb)
        return gsr_fail(ctx, GSR_ERR_INVALID_ARG, "null Gaussian array");
    if (!opt->first_keyframe && !alpha) return gsr_fail(ctx, GSR_ERR_INVALID_ARG, "alpha is needed after the first keyframe");
    if (cam->width <= 0 || cam->height <= 0 || n_existing < 0 || capacity < n_existing || capacity > 0x7fffffff ||
        opt->m_u < 0 || opt->m_c < 0 || opt->m_k < 0 || !(opt->rho > 0.f) || !(opt->s_min > 0.f) ||
        !(opt->s_max >= opt->s_min))
        return gsr_fail(ctx, GSR_ERR_INVALID_ARG, "invalid seeding argument");
    cudaStream_t s = (cudaStream_t)stream;
    const int W = cam->width, H = cam->height;
    const int64_t P = (int64_t)W * H;
    SeedScratch &S = ctx->seed;
    const int64_t nk = std::max<int64_t>(P, capacity);
    GSR_TRY(ensure_buf(ctx, S.flag, sizeof(u32) * P));
    GSR_TRY(ensure_buf(ctx, S.sel, sizeof(u32) * P));
    GSR_TRY(ensure_buf(ctx, S.off, sizeof(u32) * P));
    for (int k = 0; k < 2; ++k) {
        GSR_TRY(ensure_buf(ctx, S.keys[k], sizeof(u32) * nk));
        GSR_TRY(ensure_buf(ctx, S.vals[k], sizeof(u32) * nk));
    }
    GSR_TRY(ensure_buf(ctx, S.cnt, sizeof(u32) * 4));
    GSR_TRY(ensure_buf(ctx, S.cand_pix, sizeof(u32) * P));
    GSR_TRY(ensure_buf(ctx, S.cand_pts, sizeof(float4) * P));
    GSR_TRY(ensure_buf(ctx, S.keep, sizeof(u32) * P));
    GSR_TRY(ensure_buf(ctx, S.keep_off, sizeof(u32) * P));
    GSR_TRY(ensure_buf(ctx, S.d2, sizeof(float) * P));
    u32 *cnt = (u32 *)S.cnt.p, *flag = (u32 *)S.flag.p, *sel = (u32 *)S.sel.p, *off = (u32 *)S.off.p;
    u32 *keys[2] = {(u32 *)S.keys[0].p, (u32 *)S.keys[1].p}, *vals[2] = {(u32 *)S.vals[0].p, (u32 *)S.vals[1].p};
    GSR_CUDA(ctx, cudaMemsetAsync(cnt, 0, sizeof(u32) * 4, s));
    GSR_CUDA(ctx, cudaMemsetAsync(sel, 0, sizeof(u32) * P, s));
    // 1. candidates
    k_seed_eligible<<<nblk(P), 256, 0, s>>>(P, depth, opt->first_keyframe ? nullptr : alpha, opt->alpha_n, flag);
    ctx->launches += 1;
    GSR_LAUNCHED(ctx);
    GSR_TRY(scan_exclusive(ctx, flag, off, P, nullptr, cnt + 0, s));
    const int64_t m_uni = opt->first_keyframe ? opt->m_u : opt->m_k;
    for (int pass = 0; pass < (opt->first_keyframe ? 2 : 1); ++pass) {
        const int64_t m = pass == 0 ? m_uni : opt->m_c;
        if (m == 0) continue;
        k_seed_keys<<<nblk(P), 256, 0, s>>>(W, H, flag, off, rgb, opt->seed, pass, keys[0], vals[0]);
        ctx->launches += 1;
        GSR_LAUNCHED(ctx);
        GSR_TRY(radix_sort_pairs(ctx, keys, vals, P, cnt + 0, 32, s));
        k_seed_mark<<<nblk(std::min<int64_t>(m, P)), 256, 0, s>>>(P, cnt + 0, vals[0], m, sel);
        ctx->launches += 1;
        GSR_LAUNCHED(ctx);
    }
    GSR_TRY(scan_exclusive(ctx, sel, off, P, nullptr, cnt + 1, s));
    // 2. back-projection (rotation formed in double from the unit quaternion)
    SeedPose ps;
    {
        double q[4] = {pose->q[0], pose->q[1], pose->q[2], pose->q[3]};
        const double nq = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
        if (!(nq > 0.0)) return gsr_fail(ctx, GSR_ERR_INVALID_ARG, "zero quaternion");
        for (double &v : q) v /= nq;
        const double w = q[0], x = q[1], y = q[2], z = q[3];
        const double R[9] = {1 - 2 * (y * y + z * z), 2 * (x * y - w * z),     2 * (x * z + w * y),
                             2 * (x * y + w * z),     1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
                             2 * (x * z - w * y),     2 * (y * z + w * x),     1 - 2 * (x * x + y * y)};
        for (int k = 0; k < 9; ++k) ps.R[k] = (float)R[k];
        for (int k = 0; k < 3; ++k) ps.t[k] = pose->t[k];
    }
    k_seed_backproject<<<nblk(P), 256, 0, s>>>(W, H, sel, off, depth, cam->fx, cam->fy, cam->cx, cam->cy, ps,
                                               (u32 *)S.cand_pix.p, (float4 *)S.cand_pts.p);
    ctx->launches += 1;
    GSR_LAUNCHED(ctx);
    // 3. radius test against the existing means
    const float inv_h = 1.f / (opt->rho * (1.f + 1e-4f));
    GSR_TRY(sort_cells(ctx, S, g->mean, n_existing, inv_h, s));
    k_seed_reject<<<nblk(P), 256, 0, s>>>(P, cnt + 1, (const float4 *)S.cand_pts.p, g->mean, keys[0], vals[0],
                                          n_existing, inv_h, opt->rho * opt->rho, (u32 *)S.keep.p, (float *)S.d2.p);
    ctx->launches += 1;
    GSR_LAUNCHED(ctx);
    GSR_TRY(scan_exclusive(ctx, (const u32 *)S.keep.p, (u32 *)S.keep_off.p, P, cnt + 1, cnt + 2, s));
    GSR_CUDA(ctx, cudaMemcpyAsync(ctx->host_pinned + 40, cnt, sizeof(u32) * 3, cudaMemcpyDeviceToHost, s));
    GSR_CUDA(ctx, cudaStreamSynchronize(s));
    const int64_t n_cand = ctx->host_pinned[41], n_new = ctx->host_pinned[42];
    ctx->seed_last_candidates = n_cand;
    if (n_existing + n_new > capacity)
        return gsr_fail(ctx, GSR_ERR_CAPACITY, "seeding would exceed the sub-map capacity");
    // 4. new Gaussians and their scales
    k_seed_write<<<nblk(P), 256, 0, s>>>(P, cnt + 1, (const u32 *)S.keep.p, (const u32 *)S.keep_off.p,
                                         (const float4 *)S.cand_pts.p, (const u32 *)S.cand_pix.p, rgb, P, n_existing,
                                         g->mean, g->quat, g->opacity_logit, g->rgb);
    ctx->launches += 1;
    GSR_LAUNCHED(ctx);
    if (n_new > 0) {
        const float h2 = 2.f * opt->rho, inv_h2 = 1.f / h2;
        GSR_TRY(sort_cells(ctx, S, g->mean, n_existing + n_new, inv_h2, s));
        const int R = (int)ceilf(opt->s_max / (h2 * (1.f - 1e-4f)));
        k_seed_nn<<<nblk(n_new), 256, 0, s>>>(n_new, n_existing, g->mean, keys[0], vals[0], n_existing + n_new, h2,
                                              inv_h2, R, opt->s_min, opt->s_max, g->log_scale);
        ctx->launches += 1;
        GSR_LAUNCHED(ctx);
    }
    if (out) {
        out->n_candidates = n_cand;
        out->n_added = n_new;
    }
    return GSR_OK;
}

gsr_status gsr_seed_candidates_get(gsr_ctx *ctx, int32_t *pix, int32_t *keep, float *d2, int64_t capacity, int64_t *n,
                                   void *stream)
{
    if (!ctx || !n) return GSR_ERR_INVALID_ARG;
    const int64_t c = ctx->seed_last_candidates;
    *n = c;
    if (c > capacity) return gsr_fail(ctx, GSR_ERR_CAPACITY, "candidate list larger than capacity");
    if (c == 0) return GSR_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if (pix) GSR_CUDA(ctx, cudaMemcpyAsync(pix, ctx->seed.cand_pix.p, sizeof(u32) * c, cudaMemcpyDeviceToDevice, s));
    if (keep) GSR_CUDA(ctx, cudaMemcpyAsync(keep, ctx->seed.keep.p, sizeof(u32) * c, cudaMemcpyDeviceToDevice, s));
    if (d2) GSR_CUDA(ctx, cudaMemcpyAsync(d2, ctx->seed.d2.p, sizeof(float) * c, cudaMemcpyDeviceToDevice, s));
    GSR_CUDA(ctx, cudaStreamSynchronize(s));
    return GSR_OK;
}

} // extern "C"

// ------------------------------------------------------------------ pruning
namespace {

struct PruneArrays {
    float *p[15];  // 5 parameter arrays, then 5 first and 5 second moments (nullable)
    int w[15];     // floats per Gaussian
    int n_arr;
};

__global__ void k_prune_flags(int64_t n, const float *__restrict__ logit, float thr, u32 *__restrict__ keep)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) keep[i] = logit[i] >= thr ? 1u : 0u;
}

// kept rows of every array -> packed scratch rows of `row` floats
__global__ void k_prune_gather(int64_t n, const u32 *__restrict__ keep, const u32 *__restrict__ off, PruneArrays a,
                               int row, float *__restrict__ tmp)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !keep[i]) return;
    float *dst = tmp + (int64_t)off[i] * row;
    int c = 0;
    for (int k = 0; k < a.n_arr; ++k)
        for (int j = 0; j < a.w[k]; ++j) dst[c++] = a.p[k][i * a.w[k] + j];
}

__global__ void k_prune_scatter(const u32 *__restrict__ d_kept, PruneArrays a, int row, const float *__restrict__ tmp)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)*d_kept) return;
    const float *src = tmp + i * row;
    int c = 0;
    for (int k = 0; k < a.n_arr; ++k)
        for (int j = 0; j < a.w[k]; ++j) a.p[k][i * a.w[k] + j] = src[c++];
}

} // namespace

extern "C" gsr_status gsr_prune(gsr_ctx *ctx, gsr_gaussians_mut *g, gsr_adam_state *st, float min_opacity,
                                int64_t *n_kept, void *stream)
{
    if (!ctx || !g || !n_kept) return GSR_ERR_INVALID_ARG;
    if (!g->mean || !g->log_scale || !g->quat || !g->opacity_logit || !g->rgb || g->n < 0 || g->n > 0x7fffffff)
        return gsr_fail(ctx, GSR_ERR_INVALID_ARG, "invalid Gaussian arrays");
    if (!(min_opacity > 0.f && min_opacity < 1.f)) return gsr_fail(ctx, GSR_ERR_INVALID_ARG, "min_opacity not in (0, 1)");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = g->n;
    *n_kept = n;
    if (n == 0) return GSR_OK;
    PruneArrays a{};
    float *pa[5] = {g->mean, g->log_scale, g->quat, g->opacity_logit, g->rgb};
    const int wa[5] = {3, 3, 4, 1, 3};
    for (int k = 0; k < 5; ++k) {
        a.p[a.n_arr] = pa[k];
        a.w[a.n_arr++] = wa[k];
    }
    if (st) {
        float *ma[10] = {st->m_mean, st->m_log_scale, st->m_quat, st->m_opacity_logit, st->m_rgb,
                         st->v_mean, st->v_log_scale, st->v_quat, st->v_opacity_logit, st->v_rgb};
        for (int k = 0; k < 10; ++k) {
            if (!ma[k]) return gsr_fail(ctx, GSR_ERR_INVALID_ARG, "null Adam moment array");
            a.p[a.n_arr] = ma[k];
            a.w[a.n_arr++] = wa[k % 5];
        }
    }
    int row = 0;
    for (int k = 0; k < a.n_arr; ++k) row += a.w[k];
    SeedScratch &S = ctx->seed;
    GSR_TRY(ensure_buf(ctx, S.flag, sizeof(u32) * n));
    GSR_TRY(ensure_buf(ctx, S.off, sizeof(u32) * n));
    GSR_TRY(ensure_buf(ctx, S.cnt, sizeof(u32) * 4));
    GSR_TRY(ensure_buf(ctx, S.prune_tmp, sizeof(float) * n * row));
    u32 *keep = (u32 *)S.flag.p, *off = (u32 *)S.off.p, *cnt = (u32 *)S.cnt.p;
    // sigmoid(x) >= t  <=>  x >= log(t / (1 - t))
    const float thr = (float)log((double)min_opacity / (1.0 - (double)min_opacity));
    k_prune_flags<<<nblk(n), 256, 0, s>>>(n, g->opacity_logit, thr, keep);
    ctx->launches += 1;
    GSR_LAUNCHED(ctx);
    GSR_TRY(scan_exclusive(ctx, keep, off, n, nullptr, cnt + 3, s));
    k_prune_gather<<<nblk(n), 256, 0, s>>>(n, keep, off, a, row, (float *)S.prune_tmp.p);
    k_prune_scatter<<<nblk(n), 256, 0, s>>>(cnt + 3, a, row, (const float *)S.prune_tmp.p);
    ctx->launches += 2;
    GSR_LAUNCHED(ctx);
    GSR_CUDA(ctx, cudaMemcpyAsync(ctx->host_pinned + 44, cnt + 3, sizeof(u32), cudaMemcpyDeviceToHost, s));
    GSR_CUDA(ctx, cudaStreamSynchronize(s));
    *n_kept = ctx->host_pinned[44];
    return GSR_OK;
}

// ------------------------------------------------------------ global merge
namespace {

__global__ void k_merge_reject(int64_t n, const float *__restrict__ q3, const float *__restrict__ means,
                               const u32 *__restrict__ gk, const u32 *__restrict__ gv, int64_t n_grid, float inv_h,
                               float rho2, u32 *__restrict__ keep)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float qx = q3[3 * i], qy = q3[3 * i + 1], qz = q3[3 * i + 2];
    const int cx = cell_of(qx, inv_h), cy = cell_of(qy, inv_h), cz = cell_of(qz, inv_h);
    float best = INFINITY;
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx)
                best = cell_min_d2(qx, qy, qz, cx + dx, cy + dy, cz + dz, means, gk, gv, n_grid, -1, best);
    keep[i] = best < rho2 ? 0u : 1u;
}

__global__ void k_merge_append(int64_t n, const u32 *__restrict__ keep, const u32 *__restrict__ off, gsr_gaussians src,
                               gsr_gaussians_mut dst, int64_t base)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !keep[i]) return;
    const int64_t o = base + off[i];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        dst.mean[3 * o + k] = src.mean[3 * i + k];
        dst.log_scale[3 * o + k] = src.log_scale[3 * i + k];
        dst.rgb[3 * o + k] = src.rgb[3 * i + k];
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) dst.quat[4 * o + k] = src.quat[4 * i + k];
    dst.opacity_logit[o] = src.opacity_logit[i];
}

} // namespace

extern "C" gsr_status gsr_merge_submap(gsr_ctx *ctx, gsr_gaussians_mut *global, int64_t n_global, int64_t capacity,
                                       const gsr_gaussians *sub, float rho, int64_t *n_added, void *stream)
{
    if (!ctx || !global || !sub || !n_added) return GSR_ERR_INVALID_ARG;
    if (!global->mean || !global->log_scale || !global->quat || !global->opacity_logit || !global->rgb ||
        (sub->n > 0 && (!sub->mean || !sub->log_scale || !sub->quat || !sub->opacity_logit || !sub->rgb)))
        return gsr_fail(ctx, GSR_ERR_INVALID_ARG, "null Gaussian array");
    if (n_global < 0 || capacity < n_global || capacity > 0x7fffffff || sub->n < 0 || sub->n > 0x7fffffff ||
        !(rho > 0.f))
        return gsr_fail(ctx, GSR_ERR_INVALID_ARG, "invalid merge argument");
    *n_added = 0;
    const int64_t n = sub->n;
    if (n == 0) return GSR_OK;
    cudaStream_t s = (cudaStream_t)stream;
    SeedScratch &S = ctx->seed;
    const int64_t nk = std::max<int64_t>(n_global, 1);
    for (int k = 0; k < 2; ++k) {
        GSR_TRY(ensure_buf(ctx, S.keys[k], sizeof(u32) * nk));
        GSR_TRY(ensure_buf(ctx, S.vals[k], sizeof(u32) * nk));
    }
    GSR_TRY(ensure_buf(ctx, S.keep, sizeof(u32) * n));
    GSR_TRY(ensure_buf(ctx, S.keep_off, sizeof(u32) * n));
    GSR_TRY(ensure_buf(ctx, S.cnt, sizeof(u32) * 4));
    const float inv_h = 1.f / (rho * (1.f + 1e-4f));
    GSR_TRY(sort_cells(ctx, S, global->mean, n_global, inv_h, s));
    k_merge_reject<<<nblk(n), 256, 0, s>>>(n, sub->mean, global->mean, (const u32 *)S.keys[0].p,
                                           (const u32 *)S.vals[0].p, n_global, inv_h, rho * rho, (u32 *)S.keep.p);
    ctx->launches += 1;
    GSR_LAUNCHED(ctx);
    u32 *cnt = (u32 *)S.cnt.p;
    GSR_TRY(scan_exclusive(ctx, (const u32 *)S.keep.p, (u32 *)S.keep_off.p, n, nullptr, cnt + 3, s));
    GSR_CUDA(ctx, cudaMemcpyAsync(ctx->host_pinned + 44, cnt + 3, sizeof(u32), cudaMemcpyDeviceToHost, s));
    GSR_CUDA(ctx, cudaStreamSynchronize(s));
    const int64_t add = ctx->host_pinned[44];
    if (n_global + add > capacity) return gsr_fail(ctx, GSR_ERR_CAPACITY, "merge would exceed the global capacity");
    k_merge_append<<<nblk(n), 256, 0, s>>>(n, (const u32 *)S.keep.p, (const u32 *)S.keep_off.p, *sub, *global,
                                           n_global);
    ctx->launches += 1;
    GSR_LAUNCHED(ctx);
    *n_added = add;
    return GSR_OK;
}
