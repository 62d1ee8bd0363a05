// blend.cu -- per-tile front-to-back alpha blending (forward, Sec. 3.1
// Eq. (color_blending) and the depth rendering of Sec. 3.4) and its
// back-to-front replay (backward, Sec. 3.4 adjoints).
//
// A CTA renders one pixel tile; each thread owns PPT vertically adjacent
// pixels of one column, so a warp covers a 16 x (2 PPT) block.  Gaussian
// records of the tile's depth-ordered list are staged cooperatively in
// shared memory, BATCH at a time, and every staged record is evaluated for
// all PPT pixels of a thread (one shared-memory read, PPT evaluations).  The
// per-pixel arithmetic does not depend on PPT, so outputs are bit-identical
// for every PPT.  A CTA stops loading once every pixel's transmittance fell
// below the stop threshold.
//
// While staging, each list entry is also tested against the whole tile: if
// the minimum of sigma over the tile's pixel-centre box exceeds the skip
// threshold by more than the float32 error bound of both evaluations, no
// pixel of the tile can composite it and it is not staged.  Kept entries are
// compacted in list order and carry their list position, so every per-pixel
// decision, last_idx and n_contrib are unchanged.
//
// The backward walks the same list from the largest last-composited index of
// the tile down to 0, recovering T_j = T_{j+1} / (1 - alpha_j) from the saved
// final transmittance; each thread first sums its PPT pixels' contributions
// to a Gaussian.  When more than SPARSE_LANES lanes of the warp composite the
// Gaussian, a transposed warp reduction (12 shuffles for 10 components) sums
// the warp and one atomic add per warp and component lands in the
// per-Gaussian accumulator; when at most SPARSE_LANES lanes do, each of them
// adds its own 10 components with three vector atomics (fewer issue slots
// than the reduction, and few enough atomics that the L2 keeps up).
//
// The same tile bodies run in two launch forms: one CTA per tile of one view,
// block b taking tile order[b] (tiles by list length, longest first, written
// by the binning), and a persistent grid over (keyframe, tile) items of
// several views, pulled from a longest-first work list through an atomic
// counter (no waits).
#include <algorithm>

#include "gsr_internal.cuh"

namespace {

// Cheap pre-test: sigma (computed exactly as in eval_gaussian) above the
// staged threshold b.w means alpha < 1/255 for certain, so the entry is
// skipped without the exponential; decisions are unchanged.
__device__ __forceinline__ bool quick_reject(float px, float py, const float4 &a, const float4 &b)
{
    const float dx = __fsub_rn(px, a.x), dy = __fsub_rn(py, a.y);
    const float q = __fmaf_rn(a.z, __fmul_rn(dx, dx), __fmul_rn(b.x, __fmul_rn(dy, dy)));
    const float sigma = __fmaf_rn(a.w, __fmul_rn(dx, dy), __fmul_rn(0.5f, q));
    return sigma > b.w;
}

// One staged list entry: the Gaussian's record with b.w = its skip threshold
// and c.w = its position in the tile list (int bits), so one base address
// serves every field.
struct Staged {
    float4 a, b, c;
};
__device__ __forceinline__ int staged_pos(const Staged &e) { return __float_as_int(e.c.w); }

// Stage list entries [lo, hi) (hi - lo <= BATCH) of a tile: entries that may
// hit the tile are written in list order to sS (b.w = skip threshold, c.w =
// list position) with their Gaussian rank in sR.  Returns the number
// staged (uniform over the CTA).  s_cnt holds NT/32 ints.  The caller
// synchronises before reading the staged entries.
template <int NT>
__device__ __forceinline__ int stage_entries(const BlendView &vp, u32 list_base, int lo, int hi, const TileBox &box,
                                             Staged *sS, u32 *sR, int *s_cnt)
{
    constexpr int NW = NT / 32;
    const int warp = (int)threadIdx.x >> 5, lane = (int)threadIdx.x & 31;
    int total = 0;
    for (int c0 = lo; c0 < hi; c0 += NT) {
        const int j = c0 + (int)threadIdx.x;
        bool keep = false;
        float4 a, b;
        u32 r = 0;
        if (j < hi) {
            r = vp.tvals[list_base + j];
            a = vp.rec[3 * (int64_t)r];
            b = vp.rec[3 * (int64_t)r + 1];
            b.w = sigma_reject(b.y);  // replaces the rectangle bits, unused here
            keep = vp.culled || tile_may_hit(a, b, box);  // culled lists: tested when built
        }
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        int off = total, sum = __popc(bal);
        if (NW > 1) {
            if (lane == 0) s_cnt[warp] = sum;
            __syncthreads();
            sum = 0;
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                const int cw = s_cnt[w];
                off += w < warp ? cw : 0;
                sum += cw;
            }
        }
        if (keep) {
            const int pos = off + __popc(bal & ((1u << lane) - 1u));
            float4 c = vp.rec[3 * (int64_t)r + 2];
            c.w = __int_as_float(j);  // replaces the rectangle bits, unused here
            sS[pos].a = a;
            sS[pos].b = b;
            sS[pos].c = c;
            sR[pos] = r;
        }
        total += sum;
        if (NW > 1) __syncthreads();  // s_cnt is rewritten by the next chunk
    }
    return total;
}

template <int TW, int TH, int BATCH, int PPT>
__device__ __forceinline__ void fwd_tile(const CamK &ck, const BlendView &vp, int tile, Staged *sS,
                                         u32 *sR, int *s_cnt)
{
    constexpr int NT = TW * TH / PPT;
    const int tx = tile % ck.tiles_x, ty = tile / ck.tiles_x;
    const int col = (int)threadIdx.x % TW, row0 = ((int)threadIdx.x / TW) * PPT;
    const int ix = tx * TW + col;
    const float px = (float)ix + 0.5f;
    float py[PPT], T[PPT], c0[PPT], c1[PPT], c2[PPT], d[PPT];
    int last[PPT], nc[PPT];
    bool done[PPT];
    bool tdone = true;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const int iy = ty * TH + row0 + k;
        py[k] = (float)iy + 0.5f;
        done[k] = !(ix < ck.W && iy < ck.H);
        tdone = tdone && done[k];
        T[k] = 1.f;
        c0[k] = c1[k] = c2[k] = d[k] = 0.f;
        last[k] = -1;
        nc[k] = 0;
    }
    const uint2 rg = vp.ranges[tile];
    const int n = (int)(rg.y - rg.x);
    const TileBox box = tile_box(ck, tile, TW, TH);
    for (int base = 0; base < n; base += BATCH) {
        if (__syncthreads_count(tdone) == NT) break;
        const int cnt = stage_entries<NT>(vp, rg.x, base, min(n, base + BATCH), box, sS, sR, s_cnt);
        __syncthreads();
        for (int j = 0; j < cnt && !tdone; ++j) {
            const float4 a = sS[j].a, b = sS[j].b;
            bool all = true;
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
                if (!done[k] && !quick_reject(px, py[k], a, b)) {
                    const Eval e = eval_gaussian(px, py[k], a.x, a.y, a.z, a.w, b.x, b.y);
                    if (e.use) {
                        const float Tn = __fmul_rn(T[k], __fsub_rn(1.f, e.alpha));
                        if (Tn < GSR_T_STOP) {
                            done[k] = true;
                        } else {
                            const float4 c = sS[j].c;
                            const float w = e.alpha * T[k];
                            c0[k] = fmaf(c.x, w, c0[k]);
                            c1[k] = fmaf(c.y, w, c1[k]);
                            c2[k] = fmaf(c.z, w, c2[k]);
                            d[k] = fmaf(b.z, w, d[k]);
                            T[k] = Tn;
                            last[k] = staged_pos(sS[j]);
                            ++nc[k];
                        }
                    }
                }
                all = all && done[k];
            }
            tdone = all;
        }
    }
    const int64_t HW = (int64_t)ck.W * ck.H;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const int iy = ty * TH + row0 + k;
        if (ix < ck.W && iy < ck.H) {
            const int64_t p = (int64_t)iy * ck.W + ix;
            vp.rgb[p] = c0[k];
            vp.rgb[HW + p] = c1[k];
            vp.rgb[2 * HW + p] = c2[k];
            vp.depth[p] = d[k];
            vp.alpha[p] = 1.f - T[k];
            vp.final_T[p] = T[k];
            vp.last_idx[p] = last[k];
            if (vp.n_contrib) vp.n_contrib[p] = nc[k];
        }
    }
}

// Largest number of compositing lanes for which a warp skips the reduction and
// the lanes add their gradients with their own atomics.  Measured on the
// 1200 x 680 / 500k-Gaussian view with 8 x 8 tiles and two pixels per thread,
// with the three vector atomics per lane: 8 lanes 0.283 ms, 12 lanes 0.275 ms,
// 16 lanes 0.266 ms, 20 and 24 lanes 0.265 ms, never reducing 0.330 ms (atomic
// contention); the 8-keyframe step, with more contention, runs 10 % slower at
// 24 lanes than at 16.  (With ten scalar atomics per lane 8 lanes was best.)
constexpr int SPARSE_LANES = 16;

// Transposed warp reductions: every shuffle step halves the number of live
// values per lane, so the 10 image-space gradient components of one Gaussian
// are summed over the warp with 12 shuffles (instead of 5 per component).
// Afterwards the lane pair (l, l^1) holds one component's total; the even
// lane of each pair adds it to the accumulator (g2d slot).
__device__ __forceinline__ float pick(bool hi, float a, float b) { return hi ? b : a; }

__device__ __forceinline__ void warp_reduce_add10(const float (&v)[10], float *dst)
{
    const unsigned F = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const bool h4 = lane & 16, h3 = lane & 8, h2 = lane & 4, h1 = lane & 2;
    float a[6];
#pragma unroll
    for (int i = 0; i < 5; ++i) a[i] = pick(h4, v[i], v[i + 5]) + __shfl_xor_sync(F, pick(h4, v[i + 5], v[i]), 16);
    a[5] = 0.f;
    float b[4];
#pragma unroll
    for (int i = 0; i < 3; ++i) b[i] = pick(h3, a[i], a[i + 3]) + __shfl_xor_sync(F, pick(h3, a[i + 3], a[i]), 8);
    b[3] = 0.f;
    float c[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) c[i] = pick(h2, b[i], b[i + 2]) + __shfl_xor_sync(F, pick(h2, b[i + 2], b[i]), 4);
    float d = pick(h1, c[0], c[1]) + __shfl_xor_sync(F, pick(h1, c[1], c[0]), 2);
    d += __shfl_xor_sync(F, d, 1);
    const int bi = (h2 ? 2 : 0) + (h1 ? 1 : 0);  // index into b (3 = padding)
    const int ai = (h3 ? 3 : 0) + bi;            // index into a (5 = padding)
    if (!(lane & 1) && bi < 3 && ai < 5 && d != 0.f) atomicAdd(dst + (h4 ? 5 : 0) + ai, d);
}

// pose-only variant: (u, v, conic a, b, c, z) -> slots 0..4 and 9; 8 shuffles
__device__ __forceinline__ void warp_reduce_add6(const float (&v)[6], float *dst)
{
    const unsigned F = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const bool h4 = lane & 16, h3 = lane & 8, h2 = lane & 4;
    float a[4];
#pragma unroll
    for (int i = 0; i < 3; ++i) a[i] = pick(h4, v[i], v[i + 3]) + __shfl_xor_sync(F, pick(h4, v[i + 3], v[i]), 16);
    a[3] = 0.f;
    float b[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) b[i] = pick(h3, a[i], a[i + 2]) + __shfl_xor_sync(F, pick(h3, a[i + 2], a[i]), 8);
    float c = pick(h2, b[0], b[1]) + __shfl_xor_sync(F, pick(h2, b[1], b[0]), 4);
    c += __shfl_xor_sync(F, c, 2);
    c += __shfl_xor_sync(F, c, 1);
    const int ai = (h3 ? 2 : 0) + (h2 ? 1 : 0);  // index into a (3 = padding)
    const int comp = (h4 ? 3 : 0) + ai;          // 0..5
    if (!(lane & 3) && ai < 3 && c != 0.f) atomicAdd(dst + (comp == 5 ? 9 : comp), c);
}

// One lane's 10 components of an entry added to its Gaussian's accumulator
// (slots as in warp_reduce_add10) with vector atomics: float4 and float2 adds
// to global memory (sm_90 and later; atomic per element).  A record is 12
// floats (48 bytes) from a 256-byte aligned base, so slots 0 and 4 are
// 16-byte and slot 8 8-byte aligned.
template <bool POSE_ONLY>
__device__ __forceinline__ void lane_add10(float *dst, float gu, float gv, float gca, float gcb, float gcc, float gop,
                                           float gr, float gg, float gb, float gz)
{
    atomicAdd(reinterpret_cast<float4 *>(dst), make_float4(gu, gv, gca, gcb));
    if (!POSE_ONLY) {
        atomicAdd(reinterpret_cast<float4 *>(dst + 4), make_float4(gcc, gop, gr, gg));
        atomicAdd(reinterpret_cast<float2 *>(dst + 8), make_float2(gb, gz));
    } else {
        atomicAdd(dst + 4, gcc);
        atomicAdd(dst + 9, gz);
    }
}

// POSE_ONLY: the tracker needs only the gradients feeding the pose
// (u, v, conic, depth); colour and opacity gradients are skipped.
template <int TW, int TH, int BATCH, int PPT, bool POSE_ONLY>
__device__ __forceinline__ void bwd_tile(const CamK &ck, const BlendView &vp, int tile, Staged *sS,
                                         u32 *sR, int *s_cnt, int *s_max)
{
    constexpr int NT = TW * TH / PPT;
    const int tx = tile % ck.tiles_x, ty = tile / ck.tiles_x;
    const int col = (int)threadIdx.x % TW, row0 = ((int)threadIdx.x / TW) * PPT;
    const int ix = tx * TW + col;
    const float px = (float)ix + 0.5f;
    const uint2 rg = vp.ranges[tile];
    const int64_t HW = (int64_t)ck.W * ck.H;
    // Q = sum over the entries behind the current one of (dL/dC . c_u + dL/dD z_u) alpha_u T_u:
    // the four suffix sums of the colour / depth adjoints folded into one dot product
    float py[PPT], T[PPT], g0[PPT], g1[PPT], g2[PPT], gd[PPT], gaT[PPT], Q[PPT];
    int L[PPT];
    int lmax = -1;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const int iy = ty * TH + row0 + k;
        py[k] = (float)iy + 0.5f;
        L[k] = -1;
        T[k] = 1.f;
        g0[k] = g1[k] = g2[k] = gd[k] = gaT[k] = 0.f;
        Q[k] = 0.f;
        if (ix < ck.W && iy < ck.H) {
            const int64_t p = (int64_t)iy * ck.W + ix;
            L[k] = vp.last_idx[p];
            T[k] = vp.final_T[p];
            if (vp.d_rgb) {
                g0[k] = vp.d_rgb[p];
                g1[k] = vp.d_rgb[HW + p];
                g2[k] = vp.d_rgb[2 * HW + p];
            }
            if (vp.d_depth) gd[k] = vp.d_depth[p];
            if (vp.d_alpha) gaT[k] = vp.d_alpha[p] * T[k];
        }
        lmax = max(lmax, L[k]);
    }
    if (threadIdx.x == 0) *s_max = -1;
    __syncthreads();
    const int wmax = __reduce_max_sync(0xffffffffu, lmax);
    if ((threadIdx.x & 31) == 0) atomicMax(s_max, wmax);
    __syncthreads();
    const int nend = min(*s_max + 1, (int)(rg.y - rg.x));  // saved state never reads past the list
    const TileBox box = tile_box(ck, tile, TW, TH);
    for (int bend = nend; bend > 0; bend -= BATCH) {
        const int bstart = max(0, bend - BATCH);
        __syncthreads();
        const int cnt = stage_entries<NT>(vp, rg.x, bstart, bend, box, sS, sR, s_cnt);
        __syncthreads();
        for (int j = cnt - 1; j >= 0; --j) {
            const int jj = staged_pos(sS[j]);
            float gu = 0.f, gv = 0.f, gca = 0.f, gcb = 0.f, gcc = 0.f, gop = 0.f, gr = 0.f, gg = 0.f, gb = 0.f,
                  gz = 0.f;
            bool contrib = false;
            const float4 a = sS[j].a, b = sS[j].b;
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
                if (jj <= L[k] && !quick_reject(px, py[k], a, b)) {
                    const Eval e = eval_gaussian(px, py[k], a.x, a.y, a.z, a.w, b.x, b.y);
                    if (e.use) {
                        contrib = true;
                        const float4 c = sS[j].c;
                        // gradient-only use (decisions come from eval_gaussian): fast reciprocal
                        const float iom = __fdividef(1.f, 1.f - e.alpha);
                        T[k] = T[k] * iom;  // T_j
                        const float w = e.alpha * T[k];
                        // dL/dalpha_j = sum_c g_c (c_j T_j - S_c / (1 - alpha_j)) + gaT / (1 - alpha_j)
                        //             = T_j P - (Q - gaT) / (1 - alpha_j),  P = g . (c_j, z_j)
                        const float P = fmaf(g0[k], c.x, fmaf(g1[k], c.y, fmaf(g2[k], c.z, gd[k] * b.z)));
                        const float dLda = fmaf(T[k], P, -(Q[k] - gaT[k]) * iom);
                        Q[k] = fmaf(P, w, Q[k]);
                        gz = fmaf(gd[k], w, gz);
                        if (!POSE_ONLY) {
                            gr = fmaf(g0[k], w, gr);
                            gg = fmaf(g1[k], w, gg);
                            gb = fmaf(g2[k], w, gb);
                        }
                        if (e.G <= GSR_ALPHA_MAX) {
                            if (!POSE_ONLY) gop = fmaf(dLda, e.ex, gop);
                            const float ds = -dLda * e.G;
                            gu = fmaf(-ds, a.z * e.dx + a.w * e.dy, gu);
                            gv = fmaf(-ds, a.w * e.dx + b.x * e.dy, gv);
                            gca = fmaf(0.5f * ds, e.dx * e.dx, gca);
                            gcb = fmaf(ds, e.dx * e.dy, gcb);
                            gcc = fmaf(0.5f * ds, e.dy * e.dy, gcc);
                        }
                    }
                }
            }
            const unsigned bal = __ballot_sync(0xffffffffu, contrib);
            if (bal) {
                float *dst = vp.g2d + 12 * (int64_t)sR[j];
                if (__popc(bal) <= SPARSE_LANES) {
                    if (contrib) lane_add10<POSE_ONLY>(dst, gu, gv, gca, gcb, gcc, gop, gr, gg, gb, gz);
                } else if (POSE_ONLY) {
                    const float v[6] = {gu, gv, gca, gcb, gcc, gz};
                    warp_reduce_add6(v, dst);
                } else {
                    const float v[10] = {gu, gv, gca, gcb, gcc, gop, gr, gg, gb, gz};
                    warp_reduce_add10(v, dst);
                }
            }
        }
    }
}

// ---------------------------------------------------- two pixels per thread
// With two pixels per thread (vertically adjacent: same column, so dx is
// shared) the per-pixel arithmetic runs on packed float pairs: add, mul and
// fma.rn.f32x2 round each half exactly like the scalar operation, so every
// sigma, alpha, transmittance and decision is bit-identical to the
// one-pixel-per-thread kernels (eval_gaussian); only the order in which a
// thread sums its two pixels' gradient contributions differs.
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// sigma of one staged Gaussian at the pixel pair (px, py.x) / (px, py.y), in
// eval_gaussian's order of operations; dx shared, dy / dy^2 / dx dy per pixel
struct PairSigma {
    float dx, dxdx;
    float2 dy, dydy, dxdy, sig;
};

__device__ __forceinline__ PairSigma pair_sigma(float px, float2 py, const float4 &a, const float4 &b)
{
    PairSigma r;
    r.dx = __fsub_rn(px, a.x);
    r.dxdx = __fmul_rn(r.dx, r.dx);
    r.dy = add2(py, f2(-a.y));
    r.dydy = mul2(r.dy, r.dy);
    const float2 q = fma2(f2(a.z), f2(r.dxdx), mul2(f2(b.x), r.dydy));
    r.dxdy = mul2(f2(r.dx), r.dy);
    r.sig = fma2(f2(a.w), r.dxdy, mul2(f2(0.5f), q));
    return r;
}

// COUNT: also count each pixel's compositing entries (n_contrib requested)
template <int TW, int TH, int BATCH, bool COUNT>
__device__ __forceinline__ void fwd_tile2(const CamK &ck, const BlendView &vp, int tile, Staged *sS,
                                          u32 *sR, int *s_cnt)
{
    constexpr int NT = TW * TH / 2;
    const int tx = tile % ck.tiles_x, ty = tile / ck.tiles_x;
    const int col = (int)threadIdx.x % TW, row0 = ((int)threadIdx.x / TW) * 2;
    const int ix = tx * TW + col, iy0 = ty * TH + row0;
    const float px = (float)ix + 0.5f;
    const float2 py = make_float2((float)iy0 + 0.5f, (float)(iy0 + 1) + 0.5f);
    float2 T = f2(1.f), c0 = f2(0.f), c1 = f2(0.f), c2 = f2(0.f), d = f2(0.f);
    int last0 = -1, last1 = -1, nc0 = 0, nc1 = 0;
    bool done0 = !(ix < ck.W && iy0 < ck.H), done1 = !(ix < ck.W && iy0 + 1 < ck.H);
    bool tdone = done0 && done1;
    const uint2 rg = vp.ranges[tile];
    const int n = (int)(rg.y - rg.x);
    const TileBox box = tile_box(ck, tile, TW, TH);
    for (int base = 0; base < n; base += BATCH) {
        if (__syncthreads_count(tdone) == NT) break;
        const int cnt = stage_entries<NT>(vp, rg.x, base, min(n, base + BATCH), box, sS, sR, s_cnt);
        __syncthreads();
        for (int j = 0; j < cnt && !tdone; ++j) {
            const float4 a = sS[j].a, b = sS[j].b;
            const PairSigma S = pair_sigma(px, py, a, b);
            const bool r0 = done0 || S.sig.x > b.w, r1 = done1 || S.sig.y > b.w;
            if (r0 && r1) continue;
            const float2 G = mul2(f2(b.y), make_float2(__expf(-S.sig.x), __expf(-S.sig.y)));
            const float al0 = fminf(GSR_ALPHA_MAX, G.x), al1 = fminf(GSR_ALPHA_MAX, G.y);
            const bool u0 = !r0 && S.sig.x >= 0.f && al0 >= GSR_ALPHA_MIN;
            const bool u1 = !r1 && S.sig.y >= 0.f && al1 >= GSR_ALPHA_MIN;
            if (!(u0 || u1)) continue;
            const float2 al = make_float2(al0, al1);
            const float2 Tn = mul2(T, add2(f2(1.f), make_float2(-al0, -al1)));
            const bool s0 = u0 && Tn.x < GSR_T_STOP, s1 = u1 && Tn.y < GSR_T_STOP;
            const bool k0 = u0 && !s0, k1 = u1 && !s1;  // composited
            done0 = done0 || s0;
            done1 = done1 || s1;
            const float4 c = sS[j].c;
            const float2 w = mul2(make_float2(k0 ? al.x : 0.f, k1 ? al.y : 0.f), T);
            c0 = fma2(f2(c.x), w, c0);
            c1 = fma2(f2(c.y), w, c1);
            c2 = fma2(f2(c.z), w, c2);
            d = fma2(f2(b.z), w, d);
            T = make_float2(k0 ? Tn.x : T.x, k1 ? Tn.y : T.y);
            const int jj = staged_pos(sS[j]);
            last0 = k0 ? jj : last0;
            last1 = k1 ? jj : last1;
            if (COUNT) {
                nc0 += k0;
                nc1 += k1;
            }
            tdone = done0 && done1;
        }
    }
    const int64_t HW = (int64_t)ck.W * ck.H;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int iy = iy0 + k;
        if (ix < ck.W && iy < ck.H) {
            const int64_t p = (int64_t)iy * ck.W + ix;
            const float Tk = k ? T.y : T.x;
            vp.rgb[p] = k ? c0.y : c0.x;
            vp.rgb[HW + p] = k ? c1.y : c1.x;
            vp.rgb[2 * HW + p] = k ? c2.y : c2.x;
            vp.depth[p] = k ? d.y : d.x;
            vp.alpha[p] = 1.f - Tk;
            vp.final_T[p] = Tk;
            vp.last_idx[p] = k ? last1 : last0;
            if (COUNT) vp.n_contrib[p] = k ? nc1 : nc0;
        }
    }
}

template <int TW, int TH, int BATCH, bool POSE_ONLY>
__device__ __forceinline__ void bwd_tile2(const CamK &ck, const BlendView &vp, int tile, Staged *sS,
                                          u32 *sR, int *s_cnt, int *s_max)
{
    constexpr int NT = TW * TH / 2;
    const int tx = tile % ck.tiles_x, ty = tile / ck.tiles_x;
    const int col = (int)threadIdx.x % TW, row0 = ((int)threadIdx.x / TW) * 2;
    const int ix = tx * TW + col, iy0 = ty * TH + row0;
    const float px = (float)ix + 0.5f;
    const float2 py = make_float2((float)iy0 + 0.5f, (float)(iy0 + 1) + 0.5f);
    const uint2 rg = vp.ranges[tile];
    const int64_t HW = (int64_t)ck.W * ck.H;
    // per pixel: T recovered back to front, the image gradients, and Q = the
    // folded suffix sum of (dL/dC . c_u + dL/dD z_u) alpha_u T_u
    float2 T = f2(1.f), g0 = f2(0.f), g1 = f2(0.f), g2 = f2(0.f), gd = f2(0.f), gaT = f2(0.f), Q = f2(0.f);
    int L0 = -1, L1 = -1;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int iy = iy0 + k;
        if (ix < ck.W && iy < ck.H) {
            const int64_t p = (int64_t)iy * ck.W + ix;
            const int Lk = vp.last_idx[p];
            const float Tk = vp.final_T[p];
            float a0 = 0.f, a1 = 0.f, a2 = 0.f, ad = 0.f, aa = 0.f;
            if (vp.d_rgb) {
                a0 = vp.d_rgb[p];
                a1 = vp.d_rgb[HW + p];
                a2 = vp.d_rgb[2 * HW + p];
            }
            if (vp.d_depth) ad = vp.d_depth[p];
            if (vp.d_alpha) aa = vp.d_alpha[p] * Tk;
            if (k) {
                L1 = Lk; T.y = Tk; g0.y = a0; g1.y = a1; g2.y = a2; gd.y = ad; gaT.y = aa;
            } else {
                L0 = Lk; T.x = Tk; g0.x = a0; g1.x = a1; g2.x = a2; gd.x = ad; gaT.x = aa;
            }
        }
    }
    const int lmax = max(L0, L1);
    if (threadIdx.x == 0) *s_max = -1;
    __syncthreads();
    const int wmax = __reduce_max_sync(0xffffffffu, lmax);
    if ((threadIdx.x & 31) == 0) atomicMax(s_max, wmax);
    __syncthreads();
    const int nend = min(*s_max + 1, (int)(rg.y - rg.x));  // saved state never reads past the list
    const TileBox box = tile_box(ck, tile, TW, TH);
    for (int bend = nend; bend > 0; bend -= BATCH) {
        const int bstart = max(0, bend - BATCH);
        __syncthreads();
        const int cnt = stage_entries<NT>(vp, rg.x, bstart, bend, box, sS, sR, s_cnt);
        __syncthreads();
        // two entries per trip: the next entry's loads and sigma overlap this one's reduction
#pragma unroll 2
        for (int j = cnt - 1; j >= 0; --j) {
            const int jj = staged_pos(sS[j]);
            const float4 a = sS[j].a, b = sS[j].b;
            float gu = 0.f, gv = 0.f, gca = 0.f, gcb = 0.f, gcc = 0.f, gop = 0.f, gr = 0.f, gg = 0.f, gb = 0.f,
                  gz = 0.f;
            bool contrib = false;
            const bool n0 = jj <= L0, n1 = jj <= L1;
            if (n0 || n1) {
                const PairSigma S = pair_sigma(px, py, a, b);
                const bool r0 = !n0 || S.sig.x > b.w, r1 = !n1 || S.sig.y > b.w;
                if (!(r0 && r1)) {
                    const float ex0 = __expf(-S.sig.x), ex1 = __expf(-S.sig.y);
                    const float2 G = mul2(f2(b.y), make_float2(ex0, ex1));
                    const float al0 = fminf(GSR_ALPHA_MAX, G.x), al1 = fminf(GSR_ALPHA_MAX, G.y);
                    const bool u0 = !r0 && S.sig.x >= 0.f && al0 >= GSR_ALPHA_MIN;
                    const bool u1 = !r1 && S.sig.y >= 0.f && al1 >= GSR_ALPHA_MIN;
                    if (u0 || u1) {
                        contrib = true;
                        const float4 c = sS[j].c;
                        const float2 al = make_float2(u0 ? al0 : 0.f, u1 ? al1 : 0.f);
                        const float2 om = add2(f2(1.f), make_float2(-al.x, -al.y));
                        // gradient-only use (decisions come from the forward's arithmetic): fast reciprocal
                        const float2 iom = make_float2(u0 ? __fdividef(1.f, om.x) : 1.f, u1 ? __fdividef(1.f, om.y) : 1.f);
                        T = mul2(T, iom);  // T_j
                        const float2 w = mul2(al, T);
                        // dL/dalpha_j = T_j P - (Q - gaT) / (1 - alpha_j),  P = g . (c_j, z_j)
                        const float2 P = fma2(g0, f2(c.x), fma2(g1, f2(c.y), fma2(g2, f2(c.z), mul2(gd, f2(b.z)))));
                        const float2 dLda = fma2(T, P, mul2(add2(gaT, make_float2(-Q.x, -Q.y)), iom));
                        Q = fma2(P, w, Q);
                        gz = fmaf(gd.y, w.y, gd.x * w.x);
                        if (!POSE_ONLY) {
                            gr = fmaf(g0.y, w.y, g0.x * w.x);
                            gg = fmaf(g1.y, w.y, g1.x * w.x);
                            gb = fmaf(g2.y, w.y, g2.x * w.x);
                        }
                        // the cap alpha = min(0.99, G) passes no gradient where it is active
                        const bool l0 = u0 && G.x <= GSR_ALPHA_MAX, l1 = u1 && G.y <= GSR_ALPHA_MAX;
                        if (!POSE_ONLY) gop = fmaf(dLda.y, l1 ? ex1 : 0.f, dLda.x * (l0 ? ex0 : 0.f));
                        // nds = -dL/dsigma per pixel; the pixels share dx
                        const float2 nds = mul2(dLda, make_float2(l0 ? G.x : 0.f, l1 ? G.y : 0.f));
                        const float sn = nds.x + nds.y;
                        const float sny = fmaf(nds.y, S.dy.y, nds.x * S.dy.x);
                        gu = fmaf(a.z * S.dx, sn, a.w * sny);
                        gv = fmaf(a.w * S.dx, sn, b.x * sny);
                        gca = -0.5f * S.dxdx * sn;
                        gcb = -S.dx * sny;
                        gcc = -0.5f * fmaf(nds.y, S.dydy.y, nds.x * S.dydy.x);
                    }
                }
            }
            const unsigned bal = __ballot_sync(0xffffffffu, contrib);
            if (bal) {
                float *dst = vp.g2d + 12 * (int64_t)sR[j];
                if (__popc(bal) <= SPARSE_LANES) {
                    if (contrib) lane_add10<POSE_ONLY>(dst, gu, gv, gca, gcb, gcc, gop, gr, gg, gb, gz);
                } else if (POSE_ONLY) {
                    const float v[6] = {gu, gv, gca, gcb, gcc, gz};
                    warp_reduce_add6(v, dst);
                } else {
                    const float v[10] = {gu, gv, gca, gcb, gcc, gop, gr, gg, gb, gz};
                    warp_reduce_add10(v, dst);
                }
            }
        }
    }
}

// the tile this block renders (launch order: longest lists first)
__device__ __forceinline__ int block_tile(const BlendView &vp) { return vp.order ? (int)vp.order[blockIdx.x] : (int)blockIdx.x; }

template <int TW, int TH, int BATCH, int PPT>
__global__ void __launch_bounds__(TW *TH / PPT) k_blend_fwd(CamK ck, BlendView vp)
{
    __shared__ Staged sS[BATCH];
    __shared__ u32 sR[BATCH];
    __shared__ int s_cnt[TW * TH / PPT / 32];
    if constexpr (PPT == 2) {
        if (vp.n_contrib) fwd_tile2<TW, TH, BATCH, true>(ck, vp, block_tile(vp), sS, sR, s_cnt);
        else fwd_tile2<TW, TH, BATCH, false>(ck, vp, block_tile(vp), sS, sR, s_cnt);
    }
    else fwd_tile<TW, TH, BATCH, PPT>(ck, vp, block_tile(vp), sS, sR, s_cnt);
}

template <int TW, int TH, int BATCH, int PPT, bool POSE_ONLY>
__global__ void __launch_bounds__(TW *TH / PPT) k_blend_bwd(CamK ck, BlendView vp)
{
    __shared__ Staged sS[BATCH];
    __shared__ u32 sR[BATCH];
    __shared__ int s_cnt[TW * TH / PPT / 32];
    __shared__ int s_max;
    if constexpr (PPT == 2) bwd_tile2<TW, TH, BATCH, POSE_ONLY>(ck, vp, block_tile(vp), sS, sR, s_cnt, &s_max);
    else bwd_tile<TW, TH, BATCH, PPT, POSE_ONLY>(ck, vp, block_tile(vp), sS, sR, s_cnt, &s_max);
}

// Persistent forms: items[i] = (view << 16) | tile, longest lists first.
__device__ __forceinline__ int next_item(u32 *counter, int *s_item)
{
    __syncthreads();  // everyone has read the previous item
    if (threadIdx.x == 0) *s_item = (int)atomicAdd(counter, 1u);
    __syncthreads();
    return *s_item;
}

template <int TW, int TH, int BATCH, int PPT>
__global__ void __launch_bounds__(TW *TH / PPT) k_blend_fwd_multi(CamK ck, const BlendView *__restrict__ views,
                                                                  const u32 *__restrict__ items, int n_items,
                                                                  u32 *counter)
{
    __shared__ Staged sS[BATCH];
    __shared__ u32 sR[BATCH];
    __shared__ int s_cnt[TW * TH / PPT / 32];
    __shared__ int s_item;
    for (int it = next_item(counter, &s_item); it < n_items; it = next_item(counter, &s_item)) {
        const u32 w = items[it];
        if constexpr (PPT == 2) {
            const BlendView &v = views[w >> 16];
            if (v.n_contrib) fwd_tile2<TW, TH, BATCH, true>(ck, v, (int)(w & 0xffffu), sS, sR, s_cnt);
            else fwd_tile2<TW, TH, BATCH, false>(ck, v, (int)(w & 0xffffu), sS, sR, s_cnt);
        }
        else fwd_tile<TW, TH, BATCH, PPT>(ck, views[w >> 16], (int)(w & 0xffffu), sS, sR, s_cnt);
    }
}

template <int TW, int TH, int BATCH, int PPT>
__global__ void __launch_bounds__(TW *TH / PPT) k_blend_bwd_multi(CamK ck, const BlendView *__restrict__ views,
                                                                  const u32 *__restrict__ items, int n_items,
                                                                  u32 *counter)
{
    __shared__ Staged sS[BATCH];
    __shared__ u32 sR[BATCH];
    __shared__ int s_cnt[TW * TH / PPT / 32];
    __shared__ int s_max, s_item;
    for (int it = next_item(counter, &s_item); it < n_items; it = next_item(counter, &s_item)) {
        const u32 w = items[it];
        if constexpr (PPT == 2)
            bwd_tile2<TW, TH, BATCH, false>(ck, views[w >> 16], (int)(w & 0xffffu), sS, sR, s_cnt, &s_max);
        else
            bwd_tile<TW, TH, BATCH, PPT, false>(ck, views[w >> 16], (int)(w & 0xffffu), sS, sR, s_cnt,
                                                &s_max);
    }
}


// Launch order of the blend kernels: (view, tile) items by list length,
// longest first, so the long tiles start in the first wave instead of ending
// the launch on them.  A counting sort over length buckets on a log scale
// (four per octave; bucket 0 = empty tiles, placed last), in two launches of
// ORDER_ITEMS items per block: k_order_count writes each block's bucket
// counts, k_order_place derives its bucket starts from all blocks' counts
// and places its items.  The order within a bucket follows shared-memory
// atomics: only the schedule depends on it, since every tile's result is
// computed by one block wherever it is placed.  Item i = view * tiles + tile
// is written as (view << 16) | tile.
constexpr int ORDER_BUCKETS = 72, ORDER_THREADS = 256, ORDER_PER_THREAD = 4;
constexpr int ORDER_ITEMS = ORDER_THREADS * ORDER_PER_THREAD;

__device__ __forceinline__ int length_bucket(u32 len)
{
    if (len == 0) return 0;
    const int l = 31 - __clz(len);                                // floor(log2 len)
    const int frac = l >= 2 ? (int)((len >> (l - 2)) & 3u) : 0;  // two bits below the leading one
    return min(1 + 4 * l + frac, ORDER_BUCKETS - 1);
}

// The views' tile ranges: one view's array, or the descriptors of several.
struct ItemLen {
    const uint2 *ranges;       // one view (views == nullptr)
    const BlendView *views;
    int tiles;
    __device__ __forceinline__ u32 operator()(int i) const
    {
        const uint2 rg = views ? views[i / tiles].ranges[i % tiles] : ranges[i];
        return rg.y - rg.x;
    }
};

__global__ void __launch_bounds__(ORDER_THREADS) k_order_count(ItemLen len, int n, u32 *__restrict__ hist)
{
    __shared__ u32 cnt[ORDER_BUCKETS];
    for (int b = threadIdx.x; b < ORDER_BUCKETS; b += ORDER_THREADS) cnt[b] = 0;
    __syncthreads();
    int bk[ORDER_PER_THREAD];
#pragma unroll
    for (int k = 0; k < ORDER_PER_THREAD; ++k) {
        const int i = blockIdx.x * ORDER_ITEMS + k * ORDER_THREADS + (int)threadIdx.x;
        bk[k] = i < n ? length_bucket(len(i)) : -1;
    }
#pragma unroll
    for (int k = 0; k < ORDER_PER_THREAD; ++k)
        if (bk[k] >= 0) atomicAdd(&cnt[bk[k]], 1u);
    __syncthreads();
    for (int b = threadIdx.x; b < ORDER_BUCKETS; b += ORDER_THREADS)
        hist[(int64_t)blockIdx.x * ORDER_BUCKETS + b] = cnt[b];
}

__global__ void __launch_bounds__(ORDER_THREADS) k_order_place(ItemLen len, int n, const u32 *__restrict__ hist,
                                                               u32 *__restrict__ items)
{
    __shared__ u32 total[ORDER_BUCKETS], start[ORDER_BUCKETS];
    int bk[ORDER_PER_THREAD];
#pragma unroll
    for (int k = 0; k < ORDER_PER_THREAD; ++k) {
        const int i = blockIdx.x * ORDER_ITEMS + k * ORDER_THREADS + (int)threadIdx.x;
        bk[k] = i < n ? length_bucket(len(i)) : -1;
    }
    const int b = threadIdx.x;
    u32 before = 0;  // items of bucket b in earlier blocks
    if (b < ORDER_BUCKETS) {
        u32 tot = 0;
        for (int blk = 0; blk < (int)gridDim.x; ++blk) {
            const u32 h = hist[(int64_t)blk * ORDER_BUCKETS + b];
            tot += h;
            before += blk < (int)blockIdx.x ? h : 0u;
        }
        total[b] = tot;
    }
    __syncthreads();
    if (b < ORDER_BUCKETS) {  // longer buckets first
        u32 s = before;
        for (int c = b + 1; c < ORDER_BUCKETS; ++c) s += total[c];
        start[b] = s;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < ORDER_PER_THREAD; ++k) {
        if (bk[k] < 0) continue;
        const int i = blockIdx.x * ORDER_ITEMS + k * ORDER_THREADS + (int)threadIdx.x;
        items[atomicAdd(&start[bk[k]], 1u)] = ((u32)(i / len.tiles) << 16) | (u32)(i % len.tiles);
    }
}

__global__ void k_zero_g2d(int64_t cap, const u32 *__restrict__ d_v, float4 *__restrict__ g2d)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t n = (int64_t)*d_v * 3;
    if (i < n && i < cap * 3) g2d[i] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// ------------------------------------------------------------- dispatch
enum Kind { FWD, BWD, BWD_POSE, FWD_MULTI, BWD_MULTI };

struct Launch {
    Kind kind;
    int ppt;
    const CamK *ck;
    BlendView vp;
    const BlendView *views;
    const u32 *items;
    int n_items;
    u32 *counter;
    unsigned grid;
};

template <int TW, int TH, int BATCH, int PPT>
gsr_status launch_cfg(gsr_ctx *ctx, const Launch &L, cudaStream_t s)
{
    constexpr int NT = TW * TH / PPT;
    switch (L.kind) {
    case FWD: k_blend_fwd<TW, TH, BATCH, PPT><<<L.grid, NT, 0, s>>>(*L.ck, L.vp); break;
    case BWD: k_blend_bwd<TW, TH, BATCH, PPT, false><<<L.grid, NT, 0, s>>>(*L.ck, L.vp); break;
    case BWD_POSE: k_blend_bwd<TW, TH, BATCH, PPT, true><<<L.grid, NT, 0, s>>>(*L.ck, L.vp); break;
    case FWD_MULTI:
        k_blend_fwd_multi<TW, TH, BATCH, PPT><<<L.grid, NT, 0, s>>>(*L.ck, L.views, L.items, L.n_items, L.counter);
        break;
    case BWD_MULTI:
        k_blend_bwd_multi<TW, TH, BATCH, PPT><<<L.grid, NT, 0, s>>>(*L.ck, L.views, L.items, L.n_items, L.counter);
        break;
    }
    ctx->launches += 1;
    GSR_LAUNCHED(ctx);
    return GSR_OK;
}

template <int TW, int TH, int PPT>
gsr_status by_batch(gsr_ctx *ctx, const Launch &L, cudaStream_t s)
{
    switch (ctx->opt.batch) {
    case 32: return launch_cfg<TW, TH, 32, PPT>(ctx, L, s);
    case 64: return launch_cfg<TW, TH, 64, PPT>(ctx, L, s);
    case 128: return launch_cfg<TW, TH, 128, PPT>(ctx, L, s);
    default: return launch_cfg<TW, TH, 256, PPT>(ctx, L, s);
    }
}

template <int TW, int TH>
gsr_status by_ppt(gsr_ctx *ctx, const Launch &L, cudaStream_t s)
{
    if (L.ppt == 1) return by_batch<TW, TH, 1>(ctx, L, s);
    return by_batch<TW, TH, 2>(ctx, L, s);
}

gsr_status dispatch(gsr_ctx *ctx, const Launch &L, cudaStream_t s)
{
    const int tw = ctx->opt.tile_w, th = ctx->opt.tile_h;
    if (tw == 16 && th == 16) return by_ppt<16, 16>(ctx, L, s);
    if (tw == 8 && th == 8) return by_ppt<8, 8>(ctx, L, s);
    if (tw == 16 && th == 8) return by_ppt<16, 8>(ctx, L, s);
    if (tw == 32 && th == 8) return by_ppt<32, 8>(ctx, L, s);
    return gsr_fail(ctx, GSR_ERR_INVALID_ARG, "unsupported tile size");
}

template <int TW, int TH, int BATCH, int PPT>
int occ_cfg(bool fwd)
{
    int nb = 0;
    constexpr int NT = TW * TH / PPT;
    cudaError_t e;
    if (fwd) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_blend_fwd_multi<TW, TH, BATCH, PPT>, NT, 0);
    else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_blend_bwd_multi<TW, TH, BATCH, PPT>, NT, 0);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        nb = 1;
    }
    return nb;
}

template <int TW, int TH, int PPT>
int occ_batch(int batch, bool fwd)
{
    switch (batch) {
    case 32: return occ_cfg<TW, TH, 32, PPT>(fwd);
    case 64: return occ_cfg<TW, TH, 64, PPT>(fwd);
    case 128: return occ_cfg<TW, TH, 128, PPT>(fwd);
    default: return occ_cfg<TW, TH, 256, PPT>(fwd);
    }
}

template <int TW, int TH>
int occ_ppt(int ppt, int batch, bool fwd)
{
    return ppt == 1 ? occ_batch<TW, TH, 1>(batch, fwd) : occ_batch<TW, TH, 2>(batch, fwd);
}

} // namespace

BlendView blend_view(const ViewScratch &V, const gsr_render_out *o, const float *d_rgb, const float *d_depth,
                     const float *d_alpha)
{
    BlendView b{};
    b.ranges = (const uint2 *)V.ranges.p;
    b.tvals = (const u32 *)V.tvals[0].p;
    b.rec = (const float4 *)V.rec_sorted.p;
    b.rgb = o->rgb;
    b.depth = o->depth;
    b.alpha = o->alpha;
    b.final_T = o->final_T;
    b.last_idx = o->last_idx;
    b.n_contrib = o->n_contrib;
    b.d_rgb = d_rgb;
    b.d_depth = d_depth;
    b.d_alpha = d_alpha;
    b.g2d = (float *)V.g2d.p;
    b.order = V.order_valid ? (const u32 *)V.order.p : nullptr;
    b.culled = V.culled ? 1 : 0;
    return b;
}

gsr_status run_blend_forward(gsr_ctx *ctx, const Params &, const CamK &ck, gsr_render_out *o, cudaStream_t s)
{
    Launch L{};
    L.kind = FWD;
    L.ppt = ctx->ppt_fwd;
    L.ck = &ck;
    L.vp = blend_view(ctx->view, o, nullptr, nullptr, nullptr);
    L.grid = (unsigned)(ck.tiles_x * ck.tiles_y);
    return dispatch(ctx, L, s);
}

gsr_status zero_g2d(gsr_ctx *ctx, ViewScratch &V, cudaStream_t s)
{
    // the binning zeroes the accumulators; a second backward on the same lists must start again from zero
    if (V.g2d_zero) {
        V.g2d_zero = false;
        return GSR_OK;
    }
    k_zero_g2d<<<(unsigned)ceil_div(V.cap_n * 3, 256), 256, 0, s>>>(V.cap_n, (u32 *)V.counters.p + CNT_VISIBLE,
                                                                    (float4 *)V.g2d.p);
    ctx->launches += 1;
    GSR_LAUNCHED(ctx);
    return GSR_OK;
}

gsr_status run_blend_backward(gsr_ctx *ctx, const CamK &ck, const gsr_render_out *sv, const float *d_rgb,
                              const float *d_depth, const float *d_alpha, bool pose_only, cudaStream_t s)
{
    GSR_TRY(zero_g2d(ctx, ctx->view, s));
    Launch L{};
    L.kind = pose_only ? BWD_POSE : BWD;
    L.ppt = ctx->ppt_bwd;
    L.ck = &ck;
    L.vp = blend_view(ctx->view, sv, d_rgb, d_depth, d_alpha);
    L.grid = (unsigned)(ck.tiles_x * ck.tiles_y);
    return dispatch(ctx, L, s);
}

gsr_status run_blend_multi(gsr_ctx *ctx, const CamK &ck, bool backward, const BlendView *views, const u32 *items,
                           int n_items, u32 *counter, cudaStream_t s)
{
    int dev_sms = 0;
    GSR_CUDA(ctx, cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, ctx->device));
    const int tw = ctx->opt.tile_w, th = ctx->opt.tile_h, b = ctx->opt.batch;
    const int ppt = backward ? ctx->ppt_bwd : ctx->ppt_fwd;
    int per_sm = 1;
    if (tw == 16 && th == 16) per_sm = occ_ppt<16, 16>(ppt, b, !backward);
    else if (tw == 8 && th == 8) per_sm = occ_ppt<8, 8>(ppt, b, !backward);
    else if (tw == 16 && th == 8) per_sm = occ_ppt<16, 8>(ppt, b, !backward);
    else if (tw == 32 && th == 8) per_sm = occ_ppt<32, 8>(ppt, b, !backward);
    if (per_sm < 1) per_sm = 1;
    Launch L{};
    L.kind = backward ? BWD_MULTI : FWD_MULTI;
    L.ppt = ppt;
    L.ck = &ck;
    L.views = views;
    L.items = items;
    L.n_items = n_items;
    L.counter = counter;
    L.grid = (unsigned)std::min<int64_t>((int64_t)dev_sms * per_sm, n_items > 0 ? n_items : 1);
    GSR_CUDA(ctx, cudaMemsetAsync(counter, 0, sizeof(u32), s));
    return dispatch(ctx, L, s);
}

size_t order_hist_bytes(int64_t n) { return sizeof(u32) * ORDER_BUCKETS * (size_t)ceil_div(n > 0 ? n : 1, ORDER_ITEMS); }

static gsr_status run_order(gsr_ctx *ctx, const ItemLen &len, int n, u32 *items, DevBuf &hist, cudaStream_t s)
{
    const int nb = (int)ceil_div(n > 0 ? n : 1, ORDER_ITEMS);
    GSR_TRY(ensure_buf(ctx, hist, order_hist_bytes(n)));
    k_order_count<<<nb, ORDER_THREADS, 0, s>>>(len, n, (u32 *)hist.p);
    k_order_place<<<nb, ORDER_THREADS, 0, s>>>(len, n, (const u32 *)hist.p, items);
    ctx->launches += 2;
    GSR_LAUNCHED(ctx);
    return GSR_OK;
}

gsr_status run_order_tiles(gsr_ctx *ctx, ViewScratch &V, int tiles, cudaStream_t s)
{
    return run_order(ctx, ItemLen{(const uint2 *)V.ranges.p, nullptr, tiles}, tiles, (u32 *)V.order.p, V.order_hist,
                     s);
}

gsr_status run_make_items(gsr_ctx *ctx, const BlendView *views, int n_views, int tiles, u32 *items, cudaStream_t s)
{
    return run_order(ctx, ItemLen{nullptr, views, tiles}, n_views * tiles, items, ctx->mv_order_hist, s);
}
