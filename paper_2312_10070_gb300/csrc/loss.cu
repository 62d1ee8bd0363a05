// loss.cu -- fused per-pixel losses and their image gradients.
//
// Mapping (Sec. 3.4, Eqs. (depth_loss), (color_loss), (joint_loss)):
//   L = w_c [(1-lam) mean|I^-I| + lam (1 - SSIM)] + w_d mean_valid |D^-D|
// SSIM uses the 11x11 Gaussian window (sigma 1.5) of Wang et al. with zero
// padding, C1 = 0.01^2, C2 = 0.03^2, averaged over pixels and channels.  Two
// kernels: the first forms the five window sums per channel of a 32x48 output
// tile from a 42x58 shared-memory tile (in two groups, so that the grid of a
// 1200x680 frame is resident in one wave), the SSIM value and the adjoint maps
// dS/dmu_x, dS/dE[x^2], dS/dE[xy]; the second blurs the adjoint maps with the
// same (symmetric) window and assembles dL/dI^ and dL/dD^.  Both separable
// passes slide the window in registers: a horizontal task reads 14 inputs
// once and produces 4 outputs, a thread of the vertical pass reads 16 rows
// once and produces 6 outputs.
//
// Tracking (Sec. 3.5, supplementary Sec. B):
//   L = sum M_inlier alpha^3 (lam_c sum_ch |I^-I| + (1-lam_c)|D^-D|)
// with the lower median of |D^-D| over valid pixels found exactly by a
// 4-pass 8-bit radix select on the float bits.
//
// Reductions are deterministic: per-block partials, then one ordered pass.
#include <algorithm>

#include "gsr_internal.cuh"

namespace {

// 4-byte asynchronous global -> shared copy; ok = false writes 0 (src-size 0)
__device__ __forceinline__ void cp_async4(float *dst, const float *src, bool ok)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(ok ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
// 8-byte form (both addresses 8-byte aligned); ok = false writes zeros
__device__ __forceinline__ void cp_async8(float2 *dst, const float2 *src, bool ok)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(ok ? 8 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// wait until at most N of this thread's committed groups are still in flight
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

constexpr int SHALO = 5;                 // window radius
constexpr int TX = 32, TY = 48;          // output tile
constexpr int LW = TX + 2 * SHALO;       // 42 columns loaded
constexpr int LH = TY + 2 * SHALO;       // 58 rows loaded
constexpr int LP = LW + 1;               // padded row of the loaded tile
constexpr int HP = TX + 1;               // padded row of the horizontal sums
constexpr int HSEG = 4;                  // outputs per horizontal task (8 tasks per row)
constexpr int VSEG = TY / 8;             // outputs per thread, vertical pass (8 warps of 32 columns)

__device__ __forceinline__ float sgnf(float x) { return (x > 0.f) ? 1.f : ((x < 0.f) ? -1.f : 0.f); }

// The 11-tap window: w_k = exp(-(k - 5)^2 / (2 * 1.5^2)) normalised to sum 1,
// rounded to float32 (computed in double precision).  As compile-time
// constants the taps are immediate operands of the FMAs.
__host__ __device__ constexpr float wtap(int k)
{
    return k == 0 || k == 10 ? 0.001028380123898387f
         : k == 1 || k == 9  ? 0.0075987582094967365f
         : k == 2 || k == 8  ? 0.036000773310661316f
         : k == 3 || k == 7  ? 0.10936068743467331f
         : k == 4 || k == 6  ? 0.21300554275512695f
                             : 0.26601171493530273f;
}

// block sum of NV values over 256 threads; thread 0 gets the totals
template <int NV>
__device__ __forceinline__ void block_sum256(float (&v)[NV])
{
    __shared__ float red[NV][8];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        float x = v[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) red[i][w] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            float x = 0.f;
            for (int k = 0; k < 8; ++k) x += red[i][k];
            v[i] = x;
        }
    }
}

// Horizontal pass tasks of a thread: segment `warp` (HSEG output columns) of
// the loaded rows lane, lane + 32, ... (conflict-free: odd row pitches).
// HSEG horizontal window sums of f(x_i, y_i) over inputs i = col0 .. col0 + HSEG + 9
template <typename F>
__device__ __forceinline__ void hsum(const float (&xv)[HSEG + 10], const float (&yv)[HSEG + 10], const float (&wk)[11],
                                      F f, float (&out)[HSEG])
{
#pragma unroll
    for (int j = 0; j < HSEG; ++j) out[j] = 0.f;
#pragma unroll
    for (int i = 0; i < HSEG + 10; ++i) {
        const float q = f(xv[i], yv[i]);
#pragma unroll
        for (int j = 0; j < HSEG; ++j)
            if (i - j >= 0 && i - j <= 10) out[j] = fmaf(wk[i - j], q, out[j]);
    }
}

// Vertical window sums of NQ horizontal-sum planes, VSEG outputs per thread
template <int NQ>
__device__ __forceinline__ void vsum(const float (*hq)[LH][HP], int r0, int c, const float (&wk)[11],
                                     float (&out)[NQ][VSEG])
{
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        float col[VSEG + 10];
#pragma unroll
        for (int i = 0; i < VSEG + 10; ++i) col[i] = hq[q][r0 + i][c];
#pragma unroll
        for (int j = 0; j < VSEG; ++j) {
            float a = 0.f;
#pragma unroll
            for (int k = 0; k < 11; ++k) a = fmaf(wk[k], col[j + k], a);
            out[q][j] = a;
        }
    }
}

// Packed forms: two planes summed at once in float pairs (fma.rn.f32x2 rounds
// each half like fmaf, in the same order, so the sums equal the scalar ones).
__device__ __forceinline__ float2 wfma2(float w, float2 q, float2 a) { return __ffma2_rn(make_float2(w, w), q, a); }

template <typename F>
__device__ __forceinline__ void hsum2(const float2 (&v)[HSEG + 10], const float (&wk)[11], F f, float2 (&out)[HSEG])
{
#pragma unroll
    for (int j = 0; j < HSEG; ++j) out[j] = make_float2(0.f, 0.f);
#pragma unroll
    for (int i = 0; i < HSEG + 10; ++i) {
        const float2 q = f(v[i]);
#pragma unroll
        for (int j = 0; j < HSEG; ++j)
            if (i - j >= 0 && i - j <= 10) out[j] = wfma2(wk[i - j], q, out[j]);
    }
}

__device__ __forceinline__ void vsum2(const float2 (*hq)[HP], int r0, int c, const float (&wk)[11], float2 (&out)[VSEG])
{
    float2 col[VSEG + 10];
#pragma unroll
    for (int i = 0; i < VSEG + 10; ++i) col[i] = hq[r0 + i][c];
#pragma unroll
    for (int j = 0; j < VSEG; ++j) {
        float2 a = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < 11; ++k) a = wfma2(wk[k], col[j + k], a);
        out[j] = a;
    }
}

__device__ __forceinline__ void vsum1(const float (*hq)[HP], int r0, int c, const float (&wk)[11], float (&out)[VSEG])
{
    float col[VSEG + 10];
#pragma unroll
    for (int i = 0; i < VSEG + 10; ++i) col[i] = hq[r0 + i][c];
#pragma unroll
    for (int j = 0; j < VSEG; ++j) {
        float a = 0.f;
#pragma unroll
        for (int k = 0; k < 11; ++k) a = fmaf(wk[k], col[j + k], a);
        out[j] = a;
    }
}

// The five window sums are formed in two groups through float-pair planes:
// (mu_x, mu_y) packed plus E[x^2] scalar, then (E[y^2], E[xy]) packed; the
// inputs sit in shared memory as (x, y) pairs.  A block needs 43 KB of shared
// memory and the whole 1200x680 grid (570 blocks) fits in one wave at four
// blocks per SM.  The adjoint maps are written as the pair (dS/dmu_x,
// dS/dE[x^2]) per channel (planes 2 ch, 2 ch + 1, interleaved) and dS/dE[xy]
// (plane 6 + ch).
__global__ void __launch_bounds__(256, 4) k_ssim_fwd(int W, int H, const float *__restrict__ x, const float *__restrict__ y,
                                                  const float *__restrict__ dep, const float *__restrict__ dep_t,
                                                  float gscale, float *__restrict__ P, float *__restrict__ part,
                                                  u32 *__restrict__ nvalid)
{
    __shared__ float2 sxy[LH][LP];
    __shared__ float2 hp[LH][HP];
    __shared__ float hs[LH][HP];
    float wk[11];
#pragma unroll
    for (int k = 0; k < 11; ++k) wk[k] = wtap(k);
    const int ox = blockIdx.x * TX, oy = blockIdx.y * TY;
    const int c = (int)threadIdx.x & 31, r0 = ((int)threadIdx.x >> 5) * VSEG;  // vertical task
    const int gx = ox + c;
    const int64_t HW = (int64_t)W * H;
    const float C1 = 1e-4f, C2 = 9e-4f;
    float acc[3] = {0.f, 0.f, 0.f};  // SSIM sum, |x - y| sum, valid |D^ - D| sum
    const int hc = ((int)threadIdx.x >> 5) * HSEG, hlane = (int)threadIdx.x & 31;
    // channel ch + 1's halo is copied into sxy asynchronously while channel
    // ch's vertical sums and outputs are computed (its planes are read out by then)
    auto load_channel = [&](int ch) {
#pragma unroll 1
        for (int i = threadIdx.x; i < LH * LW; i += 256) {
            const int rr = i / LW, cc = i % LW;
            const int yy = oy - SHALO + rr, xx = ox - SHALO + cc;
            const bool ok = xx >= 0 && xx < W && yy >= 0 && yy < H;
            const int64_t q = ok ? (int64_t)ch * HW + (int64_t)yy * W + xx : 0;
            cp_async4(&sxy[rr][cc].x, x + q, ok);
            cp_async4(&sxy[rr][cc].y, y + q, ok);
        }
    };
    load_channel(0);
    for (int ch = 0; ch < 3; ++ch) {
        cp_async_wait_all();
        __syncthreads();
        for (int hr = hlane; hr < LH; hr += 32) {
            float2 v[HSEG + 10], o[HSEG];
            float xv[HSEG + 10], o1[HSEG];
#pragma unroll
            for (int i = 0; i < HSEG + 10; ++i) {
                v[i] = sxy[hr][hc + i];
                xv[i] = v[i].x;
            }
            hsum2(v, wk, [](float2 a) { return a; }, o);
#pragma unroll
            for (int j = 0; j < HSEG; ++j) hp[hr][hc + j] = o[j];
            hsum(xv, xv, wk, [](float a, float) { return a * a; }, o1);
#pragma unroll
            for (int j = 0; j < HSEG; ++j) hs[hr][hc + j] = o1[j];
        }
        __syncthreads();
        float2 mxy[VSEG];
        float e11[VSEG];
        vsum2(hp, r0, c, wk, mxy);
        vsum1(hs, r0, c, wk, e11);
        __syncthreads();
        for (int hr = hlane; hr < LH; hr += 32) {
            float2 v[HSEG + 10], o[HSEG];
#pragma unroll
            for (int i = 0; i < HSEG + 10; ++i) v[i] = sxy[hr][hc + i];
            // (y^2, x y)
            hsum2(v, wk, [](float2 a) { return __fmul2_rn(make_float2(a.y, a.x), make_float2(a.y, a.y)); }, o);
#pragma unroll
            for (int j = 0; j < HSEG; ++j) hp[hr][hc + j] = o[j];
        }
        float l1 = 0.f;  // this thread's |x - y| of the channel, read before sxy is refilled
#pragma unroll
        for (int j = 0; j < VSEG; ++j)
            if (gx < W && oy + r0 + j < H) {
                const float2 v = sxy[r0 + j + SHALO][c + SHALO];
                l1 += fabsf(v.x - v.y);
            }
        acc[1] += l1;
        __syncthreads();
        if (ch < 2) load_channel(ch + 1);
        float2 m22[VSEG];  // (E[y^2], E[xy])
        vsum2(hp, r0, c, wk, m22);
        float2 *P01 = reinterpret_cast<float2 *>(P) + (int64_t)ch * HW;
        float *P2 = P + (int64_t)(6 + ch) * HW;
#pragma unroll
        for (int j = 0; j < VSEG; ++j) {
            const int gy = oy + r0 + j;
            if (gx < W && gy < H) {
                const float m1 = mxy[j].x, m2 = mxy[j].y, e22 = m22[j].x, e12 = m22[j].y;
                const float A1 = 2.f * m1 * m2 + C1, A2 = 2.f * (e12 - m1 * m2) + C2;
                const float B1 = m1 * m1 + m2 * m2 + C1, B2 = (e11[j] - m1 * m1) + (e22 - m2 * m2) + C2;
                // B1, B2 >= C1, C2 > 0: fast reciprocals (2 ulp) are ample here
                const float iB1 = __fdividef(1.f, B1), iB2 = __fdividef(1.f, B2);
                const float iB = iB1 * iB2;
                const float S = A1 * A2 * iB;
                acc[0] += S;
                const int64_t p = (int64_t)gy * W + gx;
                P01[p] = make_float2(gscale * (2.f * m2 * (A2 - A1) * iB - 2.f * m1 * S * (iB1 - iB2)),
                                     gscale * (-S * iB2));
                P2[p] = gscale * (2.f * A1 * iB);
            }
        }
        __syncthreads();
    }
    u32 nv = 0;
#pragma unroll
    for (int j = 0; j < VSEG; ++j) {
        const int gy = oy + r0 + j;
        if (gx < W && gy < H) {
            const int64_t p = (int64_t)gy * W + gx;
            const float dt = dep_t[p];
            if (dt > 0.f) {
                acc[2] += fabsf(dep[p] - dt);
                ++nv;
            }
        }
    }
    // the block's valid-depth count rides along the float sums (exact: at most
    // TX * TY = 1536 per block) and reaches the counter in one atomic per block
    float sums[4] = {acc[0], acc[1], acc[2], (float)nv};
    block_sum256<4>(sums);
    if (threadIdx.x == 0) {
        const int64_t b = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
        part[3 * b] = sums[0];
        part[3 * b + 1] = sums[1];
        part[3 * b + 2] = sums[2];
        const u32 bn = (u32)sums[3];
        if (bn) atomicAdd(nvalid, bn);
    }
}

// The adjoint maps are blurred per channel in two passes, the pair
// (dS/dmu_x, dS/dE[x^2]) packed, then dS/dE[xy], each through its own loaded
// plane and one shared horizontal-sum plane (45 KB of shared memory per
// block).  The six plane loads are asynchronous copies issued one stage
// ahead: plane k + 2 is copied while planes k and k + 1 are summed.
__global__ void __launch_bounds__(256, 4) k_ssim_bwd(int W, int H, const float *__restrict__ x, const float *__restrict__ y,
                                                  const float *__restrict__ dep, const float *__restrict__ dep_t,
                                                  const float *__restrict__ P, float l1s, float dscale,
                                                  const u32 *__restrict__ nvalid, float *__restrict__ d_rgb,
                                                  float *__restrict__ d_dep)
{
    __shared__ float2 sa[LH][LP];  // (dS/dmu_x, dS/dE[x^2]) of the loaded tile
    __shared__ float sb[LH][LP];   // dS/dE[xy] of the loaded tile
    __shared__ float2 hq2[LH][HP];
    float (*hq)[HP] = reinterpret_cast<float (*)[HP]>(&hq2[0][0]);
    float wk[11];
#pragma unroll
    for (int k = 0; k < 11; ++k) wk[k] = wtap(k);
    const int ox = blockIdx.x * TX, oy = blockIdx.y * TY;
    const int c = (int)threadIdx.x & 31, r0 = ((int)threadIdx.x >> 5) * VSEG;
    const int gx = ox + c;
    const int64_t HW = (int64_t)W * H;
    const int hc = ((int)threadIdx.x >> 5) * HSEG, hlane = (int)threadIdx.x & 31;
    const float2 *P01 = reinterpret_cast<const float2 *>(P);
    const float *P2 = P + 6 * HW;
    auto load01 = [&](int ch) {
#pragma unroll 1
        for (int i = threadIdx.x; i < LH * LW; i += 256) {
            const int rr = i / LW, cc = i % LW;
            const int yy = oy - SHALO + rr, xx = ox - SHALO + cc;
            const bool ok = xx >= 0 && xx < W && yy >= 0 && yy < H;
            cp_async8(&sa[rr][cc], P01 + (ok ? (int64_t)ch * HW + (int64_t)yy * W + xx : 0), ok);
        }
        cp_async_commit();
    };
    auto load2 = [&](int ch) {
#pragma unroll 1
        for (int i = threadIdx.x; i < LH * LW; i += 256) {
            const int rr = i / LW, cc = i % LW;
            const int yy = oy - SHALO + rr, xx = ox - SHALO + cc;
            const bool ok = xx >= 0 && xx < W && yy >= 0 && yy < H;
            cp_async4(&sb[rr][cc], P2 + (ok ? (int64_t)ch * HW + (int64_t)yy * W + xx : 0), ok);
        }
        cp_async_commit();
    };
    load01(0);
    load2(0);
    {  // depth gradient while the first planes arrive
        const u32 nv = *nvalid;
        const float dsn = nv > 0 ? dscale / (float)nv : 0.f;
#pragma unroll
        for (int j = 0; j < VSEG; ++j) {
            const int gy = oy + r0 + j;
            if (gx < W && gy < H) {
                const int64_t p = (int64_t)gy * W + gx;
                const float dt = dep_t[p];
                d_dep[p] = dt > 0.f ? dsn * sgnf(dep[p] - dt) : 0.f;
            }
        }
    }
    for (int ch = 0; ch < 3; ++ch) {
        float xv[VSEG], yv[VSEG];  // this thread's pixels, read while the planes are summed
#pragma unroll
        for (int j = 0; j < VSEG; ++j) {
            const int gy = oy + r0 + j;
            const int64_t p = (gx < W && gy < H) ? ch * HW + (int64_t)gy * W + gx : 0;
            xv[j] = x[p];
            yv[j] = y[p];
        }
        cp_async_wait<1>();  // (dS/dmu_x, dS/dE[x^2]) of channel ch has landed
        __syncthreads();
        for (int hr = hlane; hr < LH; hr += 32) {
            float2 v[HSEG + 10], o[HSEG];
#pragma unroll
            for (int i = 0; i < HSEG + 10; ++i) v[i] = sa[hr][hc + i];
            hsum2(v, wk, [](float2 a) { return a; }, o);
#pragma unroll
            for (int j = 0; j < HSEG; ++j) hq2[hr][hc + j] = o[j];
        }
        __syncthreads();
        if (ch < 2) load01(ch + 1);
        float2 b01[VSEG];
        vsum2(hq2, r0, c, wk, b01);
        if (ch < 2)
            cp_async_wait<1>();  // dS/dE[xy] of channel ch has landed
        else
            cp_async_wait<0>();
        __syncthreads();
        for (int hr = hlane; hr < LH; hr += 32) {
            float v[HSEG + 10], o[HSEG];
#pragma unroll
            for (int i = 0; i < HSEG + 10; ++i) v[i] = sb[hr][hc + i];
            hsum(v, v, wk, [](float a, float) { return a; }, o);
#pragma unroll
            for (int j = 0; j < HSEG; ++j) hq[hr][hc + j] = o[j];
        }
        __syncthreads();
        if (ch < 2) load2(ch + 1);
        float b2[VSEG];
        vsum1(hq, r0, c, wk, b2);
#pragma unroll
        for (int j = 0; j < VSEG; ++j) {
            const int gy = oy + r0 + j;
            if (gx < W && gy < H) {
                const int64_t p = (int64_t)gy * W + gx;
                d_rgb[ch * HW + p] = l1s * sgnf(xv[j] - yv[j]) + b01[j].x + 2.f * xv[j] * b01[j].y + yv[j] * b2[j];
            }
        }
    }
}

__global__ void k_loss_map_final(const float *__restrict__ part, int nb, const u32 *__restrict__ nvalid, float inv3hw,
                                 float lam, float wc, float wd, float scale, float *loss, int accumulate,
                                 u32 *status)
{
    __shared__ float red[3][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;  // 3 warps
    float v = 0.f;
    for (int b = lane; b < nb; b += 32) v += part[3 * b + w];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[w][0] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        float ssim = red[0][0] * inv3hw, l1c = red[1][0] * inv3hw;
        u32 nv = *nvalid;
        float l1d = nv > 0 ? red[2][0] / (float)nv : 0.f;
        float L = scale * (wc * ((1.f - lam) * l1c + lam * (1.f - ssim)) + wd * l1d);
        if (!isfinite(L)) atomicOr(status, GSR_FLAG_NONFINITE);
        if (loss) {
            if (accumulate) *loss += L;
            else *loss = L;
        }
    }
}

// ---------------------------------------------------------------- tracking
__global__ void k_track_resid(int64_t HW, const float *__restrict__ dep, const float *__restrict__ dep_t,
                              u32 *__restrict__ ebits, u32 *__restrict__ nvalid)
{
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool valid = false;
    if (p < HW) {
        float dt = dep_t[p];
        valid = dt > 0.f;
        ebits[p] = valid ? __float_as_uint(fabsf(dep[p] - dt)) : 0xffffffffu;
    }
    // one atomic per block on the shared counter (per warp, the blocks of this
    // short kernel queued on one L2 address)
    const int bn = __syncthreads_count(valid);
    if (threadIdx.x == 0 && bn) atomicAdd(nvalid, (u32)bn);
}

// state: sel[0] = prefix bits, sel[1] = remaining rank
__global__ void k_sel_init(const u32 *__restrict__ nvalid, u32 *__restrict__ sel, u32 *__restrict__ hist)
{
    u32 n = *nvalid;
    if (threadIdx.x == 0) {
        sel[0] = 0u;
        sel[1] = n > 0 ? (n - 1u) / 2u : 0u;
    }
    hist[threadIdx.x] = 0u;
}

// SEL_UNROLL residuals per thread are loaded before their histogram updates;
// the loop's trip count is uniform over the block, and each warp adds one
// shared-memory atomic per distinct bin (the first pass bins the exponent
// byte, which few values share, so per-lane atomics would queue on them)
constexpr int SEL_UNROLL = 4;

__global__ void __launch_bounds__(256) k_sel_hist(int64_t HW, const u32 *__restrict__ ebits, int shift,
                                                  const u32 *__restrict__ sel, u32 *__restrict__ hist)
{
    __shared__ u32 h[256];
    h[threadIdx.x] = 0u;
    __syncthreads();
    const u32 prefix = sel[0];
    const u32 hmask = shift == 24 ? 0u : (0xffffffffu << (shift + 8));
    const int lane = threadIdx.x & 31;
    for (int64_t base = (int64_t)blockIdx.x * 256 * SEL_UNROLL; base < HW;
         base += (int64_t)gridDim.x * 256 * SEL_UNROLL) {
        u32 bv[SEL_UNROLL];
#pragma unroll
        for (int u = 0; u < SEL_UNROLL; ++u) {
            const int64_t p = base + u * 256 + threadIdx.x;
            bv[u] = p < HW ? ebits[p] : 0xffffffffu;
        }
#pragma unroll
        for (int u = 0; u < SEL_UNROLL; ++u) {
            const u32 b = bv[u];
            const int bin = (b != 0xffffffffu && (b & hmask) == (prefix & hmask)) ? (int)((b >> shift) & 255u) : -1;
            const unsigned peers = __match_any_sync(0xffffffffu, bin);
            if (bin >= 0 && lane == __ffs(peers) - 1) atomicAdd(&h[bin], (u32)__popc(peers));
        }
    }
    __syncthreads();
    if (h[threadIdx.x]) atomicAdd(&hist[threadIdx.x], h[threadIdx.x]);
}

__global__ void __launch_bounds__(256) k_sel_pick(int shift, u32 *__restrict__ sel, u32 *__restrict__ hist)
{
    __shared__ u32 s_wt[8];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const u32 v = hist[threadIdx.x];
    // inclusive scan of the 256 bins: shuffles within each warp, then the warp totals
    u32 incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const u32 t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) s_wt[w] = incl;
    __syncthreads();
    for (int k = 0; k < w; ++k) incl += s_wt[k];
    const u32 k = sel[1];
    const u32 excl = incl - v;
    __syncthreads();  // every thread has read sel before the one below writes it
    if (v > 0 && excl <= k && k < incl) {
        sel[0] |= (u32)threadIdx.x << shift;
        sel[1] = k - excl;
    }
    hist[threadIdx.x] = 0u;
}

__global__ void __launch_bounds__(256) k_track_loss(int64_t HW, const float *__restrict__ rgb, const float *__restrict__ dep,
                                                    const float *__restrict__ alpha, const float *__restrict__ rgb_t,
                                                    const float *__restrict__ dep_t, const u32 *__restrict__ sel,
                                                    const u32 *__restrict__ nvalid, float lam_c, float k_med,
                                                    float apow, float *__restrict__ d_rgb, float *__restrict__ d_dep,
                                                    float *__restrict__ part)
{
    int64_t p = (int64_t)blockIdx.x * 256 + threadIdx.x;
    float acc[1] = {0.f};
    if (p < HW) {
        const float med = *nvalid > 0 ? __uint_as_float(sel[0]) : 0.f;
        float dt = dep_t[p], dh = dep[p];
        float e = fabsf(dh - dt);
        bool in = dt > 0.f && e <= k_med * med;
        float a = alpha[p];
        float w = 0.f;
        if (in) w = (apow == 3.f) ? a * a * a : powf(a, apow);
        float lc = 0.f;
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            float diff = rgb[ch * HW + p] - rgb_t[ch * HW + p];
            lc += fabsf(diff);
            d_rgb[ch * HW + p] = w * lam_c * sgnf(diff);
        }
        d_dep[p] = w * (1.f - lam_c) * sgnf(dh - dt);
        acc[0] = w * (lam_c * lc + (1.f - lam_c) * e);
    }
    block_sum256<1>(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = acc[0];
}

__global__ void k_track_final(const float *__restrict__ part, int nb, const u32 *__restrict__ sel,
                              const u32 *__restrict__ nvalid, float *loss, float *median, u32 *status)
{
    __shared__ float red[32];
    float v = 0.f;
    for (int b = threadIdx.x; b < nb; b += 1024) v += part[b];
    // fixed-order block reduction over 1024 threads
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        float L = 0.f;
        for (int k = 0; k < 32; ++k) L += red[k];
        if (!isfinite(L)) atomicOr(status, GSR_FLAG_NONFINITE);
        if (loss) *loss = L;
        if (median) *median = *nvalid > 0 ? __uint_as_float(sel[0]) : 0.f;
    }
}

} // namespace

gsr_status run_loss_map_kernels(gsr_ctx *ctx, ViewScratch *V, int W, int H, const float *rgb, const float *depth,
                                const float *rgb_t, const float *depth_t, float lam, float wc, float wd,
                                float scale, float *d_rgb, float *d_depth, cudaStream_t s)
{
    const int64_t HW = (int64_t)W * H;
    dim3 grid((unsigned)ceil_div(W, TX), (unsigned)ceil_div(H, TY));
    const int nb = (int)(grid.x * grid.y);
    ViewScratch &cv = V ? *V : ctx->view;
    DevBuf &maps = V ? V->loss_maps : ctx->loss_maps, &part = V ? V->loss_part : ctx->loss_part;
    GSR_TRY(ensure_buf(ctx, maps, sizeof(float) * 9 * (size_t)HW));
    GSR_TRY(ensure_buf(ctx, part, sizeof(float) * 3 * (size_t)nb));
    GSR_TRY(ensure_buf(ctx, cv.counters, sizeof(u32) * CNT_WORDS));
    u32 *cnt = (u32 *)cv.counters.p;
    GSR_CUDA(ctx, cudaMemsetAsync(cnt + CNT_NVALID, 0, sizeof(u32), s));
    const float inv3hw = 1.f / (3.f * (float)HW);
    k_ssim_fwd<<<grid, 256, 0, s>>>(W, H, rgb, rgb_t, depth, depth_t, -scale * wc * lam * inv3hw, (float *)maps.p,
                                    (float *)part.p, cnt + CNT_NVALID);
    k_ssim_bwd<<<grid, 256, 0, s>>>(W, H, rgb, rgb_t, depth, depth_t, (float *)maps.p,
                                    scale * wc * (1.f - lam) * inv3hw, scale * wd, cnt + CNT_NVALID, d_rgb, d_depth);
    ctx->launches += 2;
    GSR_LAUNCHED(ctx);
    return GSR_OK;
}

gsr_status run_loss_map_final(gsr_ctx *ctx, ViewScratch *V, int W, int H, float lam, float wc, float wd,
                              float scale, float *loss_dev, bool accumulate_loss, cudaStream_t s)
{
    const int64_t HW = (int64_t)W * H;
    const int nb = (int)(ceil_div(W, TX) * ceil_div(H, TY));
    ViewScratch &cv = V ? *V : ctx->view;
    DevBuf &part = V ? V->loss_part : ctx->loss_part;
    GSR_TRY(ensure_buf(ctx, ctx->view.counters, sizeof(u32) * CNT_WORDS));
    const u32 *cnt = (const u32 *)cv.counters.p;
    u32 *status = (u32 *)ctx->view.counters.p + CNT_STATUS;  // the context's status word
    k_loss_map_final<<<1, 96, 0, s>>>((float *)part.p, nb, cnt + CNT_NVALID, 1.f / (3.f * (float)HW), lam, wc, wd,
                                      scale, loss_dev, accumulate_loss ? 1 : 0, status);
    ctx->launches += 1;
    GSR_LAUNCHED(ctx);
    return GSR_OK;
}

gsr_status run_loss_map(gsr_ctx *ctx, int W, int H, const float *rgb, const float *depth, const float *rgb_t,
                        const float *depth_t, float lam, float wc, float wd, float scale, float *d_rgb,
                        float *d_depth, float *loss_dev, bool accumulate_loss, cudaStream_t s)
{
    GSR_TRY(run_loss_map_kernels(ctx, nullptr, W, H, rgb, depth, rgb_t, depth_t, lam, wc, wd, scale, d_rgb, d_depth,
                                 s));
    return run_loss_map_final(ctx, nullptr, W, H, lam, wc, wd, scale, loss_dev, accumulate_loss, s);
}

gsr_status run_loss_track(gsr_ctx *ctx, int W, int H, const float *rgb, const float *depth, const float *alpha,
                          const float *rgb_t, const float *depth_t, float lam_c, float k_med, float apow,
                          float *d_rgb, float *d_depth, float *loss_dev, float *median_dev, cudaStream_t s)
{
    const int64_t HW = (int64_t)W * H;
    const unsigned nb = (unsigned)ceil_div(HW, 256);
    GSR_TRY(ensure_buf(ctx, ctx->loss_maps, sizeof(u32) * (size_t)HW + sizeof(u32) * 256));
    GSR_TRY(ensure_buf(ctx, ctx->loss_part, sizeof(float) * nb));
    GSR_TRY(ensure_buf(ctx, ctx->view.counters, sizeof(u32) * CNT_WORDS));
    u32 *cnt = (u32 *)ctx->view.counters.p;
    u32 *ebits = (u32 *)ctx->loss_maps.p;
    u32 *hist = ebits + HW;
    GSR_CUDA(ctx, cudaMemsetAsync(cnt + CNT_TRACK_N, 0, sizeof(u32), s));
    k_track_resid<<<nb, 256, 0, s>>>(HW, depth, depth_t, ebits, cnt + CNT_TRACK_N);
    k_sel_init<<<1, 256, 0, s>>>(cnt + CNT_TRACK_N, cnt + CNT_SEL, hist);
    const unsigned hb = (unsigned)std::min<int64_t>(ceil_div(HW, 256 * SEL_UNROLL), 1216);
    for (int shift = 24; shift >= 0; shift -= 8) {
        k_sel_hist<<<hb, 256, 0, s>>>(HW, ebits, shift, cnt + CNT_SEL, hist);
        k_sel_pick<<<1, 256, 0, s>>>(shift, cnt + CNT_SEL, hist);
    }
    k_track_loss<<<nb, 256, 0, s>>>(HW, rgb, depth, alpha, rgb_t, depth_t, cnt + CNT_SEL, cnt + CNT_TRACK_N, lam_c,
                                    k_med, apow, d_rgb, d_depth, (float *)ctx->loss_part.p);
    k_track_final<<<1, 1024, 0, s>>>((float *)ctx->loss_part.p, (int)nb, cnt + CNT_SEL, cnt + CNT_TRACK_N, loss_dev,
                                     median_dev, cnt + CNT_STATUS);
    ctx->launches += 12;
    GSR_LAUNCHED(ctx);
    return GSR_OK;
}

// ----------------------------------------------------- allocation-free variant
// Scratch of gsr_loss_track_noalloc: one static device array, laid out as
// [residual bits: MAXP][select histogram: 256][block partials: MAXB][counters: 16]
// (u32 words).  It belongs to the library, not to a context, so a caller that
// cannot allocate device memory can still run the tracking loss.
namespace {
constexpr int64_t NA_MAXP = GSR_NOALLOC_MAX_PIXELS;
constexpr int64_t NA_MAXB = (NA_MAXP + 255) / 256;
constexpr int64_t NA_HIST = NA_MAXP;
constexpr int64_t NA_PART = NA_HIST + 256;
constexpr int64_t NA_CNT = NA_PART + NA_MAXB;
constexpr int64_t NA_WORDS = NA_CNT + 16;
}  // namespace

static __device__ __align__(256) u32 g_noalloc_scratch[NA_WORDS];

extern "C" gsr_status gsr_loss_track_noalloc(int32_t width, int32_t height, const float *rgb, const float *depth,
                                             const float *alpha, const float *rgb_target, const float *depth_target,
                                             float lambda_c, float k_median, float alpha_pow, float *d_rgb,
                                             float *d_depth, float *loss_dev, float *median_dev, void *stream)
{
    if (width <= 0 || height <= 0 || !rgb || !depth || !alpha || !rgb_target || !depth_target || !d_rgb || !d_depth)
        return GSR_ERR_INVALID_ARG;
    const int64_t HW = (int64_t)width * height;
    if (HW > NA_MAXP) return GSR_ERR_CAPACITY;
    // an error left pending by earlier, unrelated work must not be reported as this call's
    (void)cudaGetLastError();
    // Host code only knows the array's host-side stand-in; the kernels need its
    // device address in the CURRENT context.  The address is looked up on every
    // call (a table lookup once the module is loaded in that context) rather
    // than cached per device ordinal: a cached address would go stale after
    // cudaDeviceReset or under another context of the same device.
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
        (void)cudaGetLastError();
        return GSR_ERR_CUDA;
    }
    u32 *base = (u32 *)p;
    cudaStream_t s = (cudaStream_t)stream;
    u32 *ebits = base, *hist = base + NA_HIST, *cnt = base + NA_CNT;
    float *part = (float *)(base + NA_PART);
    u32 *nvalid = cnt + 0, *sel = cnt + 1, *status = cnt + 4;
    const unsigned nb = (unsigned)ceil_div(HW, 256);
    // the array keeps the previous call's contents: reset what accumulates
    if (cudaMemsetAsync(cnt, 0, 16 * sizeof(u32), s) != cudaSuccess) {
        (void)cudaGetLastError();
        return GSR_ERR_CUDA;
    }
    k_track_resid<<<nb, 256, 0, s>>>(HW, depth, depth_target, ebits, nvalid);
    k_sel_init<<<1, 256, 0, s>>>(nvalid, sel, hist);
    const unsigned hb = (unsigned)std::min<int64_t>(ceil_div(HW, 256 * SEL_UNROLL), 1216);
    for (int shift = 24; shift >= 0; shift -= 8) {
        k_sel_hist<<<hb, 256, 0, s>>>(HW, ebits, shift, sel, hist);
        k_sel_pick<<<1, 256, 0, s>>>(shift, sel, hist);
    }
    k_track_loss<<<nb, 256, 0, s>>>(HW, rgb, depth, alpha, rgb_target, depth_target, sel, nvalid, lambda_c, k_median,
                                    alpha_pow, d_rgb, d_depth, part);
    k_track_final<<<1, 1024, 0, s>>>(part, (int)nb, sel, nvalid, loss_dev, median_dev, status);
    if (cudaGetLastError() != cudaSuccess) return GSR_ERR_CUDA;
    return GSR_OK;
}
