// cnn.cu -- the learned tracking warm-start network on BF16 tensor cores.
//
// Not a step of the paper's method (its tracker starts from the
// constant-velocity extrapolation of Sec. 3.5): a small network that predicts
// the twist correcting that initial pose from the rendered-versus-input RGB-D
// residual.  Sizes and layouts are given in include/gsr_warmstart.h.
//
// Every layer is a GEMM with FP32 accumulation:
//   forward         Z[M,N]   = im2col(X)[M,K] . W[N,K]^T        (+ bias, ReLU, -> BF16)
//   data gradient   dX = the adjoint of the convolution, as one GEMM per parity
//                   class of input pixels (then the previous ReLU's mask)
//   weight gradient dW[N,K]  = dZ^T[N,M] . im2col(X)[M,K]       (split over M, FP32 atomics)
// with M = batch x output pixels, N = output channels, K = 9 x input channels.
// One kernel serves all three (see the GEMM section): the im2col matrix is
// never materialised, its tiles are gathered from the NHWC activations while
// staging.
#include <cuda_bf16.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <random>
#include <string>
#include <vector>

#include "../../include/gsr_warmstart.h"
#include "gsr_internal.cuh"

typedef __nv_bfloat16 bf16;

namespace {

constexpr int NL = 6;
constexpr int CIN[NL] = {8, 32, 64, 128, 128, 256};
constexpr int CINP[NL] = {8, 32, 64, 128, 128, 256};  // stored channels (equal to CIN: powers of two)
constexpr int COUT[NL] = {32, 64, 128, 128, 256, 256};
constexpr int HIN[NL] = {120, 60, 30, 15, 8, 4};
constexpr int WIN[NL] = {160, 80, 40, 20, 10, 5};
constexpr int HOUT[NL] = {60, 30, 15, 8, 4, 2};
constexpr int WOUT[NL] = {80, 40, 20, 10, 5, 3};
constexpr int FLAT = 2 * 3 * 256, HID = 256, NOUT = 6, NOUTP = 8;
constexpr int NSEG = NL + 2;

struct Layout {
    int64_t w_off[NSEG], b_off[NSEG];  // flat FP32 vector
    int64_t wb_off[NSEG + 1];          // BF16 GEMM operands [N][K] (dense 2 padded to 8 rows)
    int64_t n_params;
    int cin[NL], cinp[NL];             // conv input channels: true and stored
};

struct LossW {
    float w[NOUT];
};

// ------------------------------------------------------------------ GEMM
// C[M,N] (op)= sum_k A(m,k) B(n,k) on 128 x 64 output tiles, 8 warps of 32 x 32,
// BF16 mma.sync m16n8k16 with FP32 accumulation.  Operand tiles of 32
// reduction indices are copied global -> shared by cp.async (16 bytes, zero
// fill outside the operand) in a 3-stage ring, in the operand's own memory
// order; fragments come from ldmatrix, transposed (.trans) for operands whose
// row index is the contiguous one.  Operand kinds:
//   OP_KC     element (r, k) at p[r*ld + k]            (reduction index contiguous)
//   OP_RC     element (r, k) at p[k*ld + r]            (row index contiguous)
//   OP_IM_KC  im2col of an NHWC tensor for a 3x3, stride-2, padding-1
//             convolution: r = output position (b, oy, ox), k = (ky, kx, c)
//   OP_IM_RC  the same matrix with roles swapped: r = (ky, kx, c), k = position
//   OP_DT_KC  data gradient of that convolution for one parity class (py, px)
//             of input pixels: r = input pixel (b, iy, ix) with iy = py mod 2,
//             ix = px mod 2; k = (tap t of the class, output channel n);
//             element dZ[b, (iy + 1 - ky) / 2, (ix + 1 - kx) / 2, n] or 0
//   OP_WT_RC  the matching weights: r = input channel c, k = (t, n);
//             element W[n][ky][kx][c]
// A stride-2 3x3 kernel touches an even input row only through ky = 1 and an
// odd one through ky = 0 and 2 (likewise columns), so the four classes have
// 1, 2, 2 and 4 taps and the data gradient needs no column matrix.
// Channel counts are powers of two >= 8, so an 8-element chunk never crosses
// a tap.
constexpr int BM = 128, BN = 64, BKT = 32, NSTAGE = 3;
constexpr int KC_ROW = BKT + 8;                       // shared row (elements), reduction-contiguous tiles
constexpr int A_STAGE = BM * KC_ROW;                  // >= BKT * (BM + 8)
constexpr int B_STAGE = BN * KC_ROW;                  // >= BKT * (BN + 8)
enum { EPI_STORE = 0, EPI_ATOMIC = 1, EPI_BIAS_RELU_BF16 = 2, EPI_BIAS = 3, EPI_MASK_BF16 = 4, EPI_ATOMIC_T = 5 };
enum { OP_KC = 0, OP_RC = 1, OP_IM_KC = 2, OP_IM_RC = 3, OP_DT_KC = 4, OP_WT_RC = 5 };

struct Operand {
    const bf16 *p;
    int ld;                // OP_KC / OP_RC; OP_WT_RC: 9 x input channels
    int rows;              // staging bound on the row index (a multiple of 8 for row-contiguous kinds)
    int H, W, lc, Ho, Wo;  // OP_IM_*: input H x W x 2^lc channels, output Ho x Wo;
                           // OP_DT_KC / OP_WT_RC: lc = log2 of the output channels n
    int py, px, Hc, Wc;    // OP_DT_KC / OP_WT_RC: parity class and its pixel grid
    int cin;               // OP_WT_RC: input channels
    int ones_row;          // OP_IM_RC: row index holding 1 for every position (bias gradient), else -1
};

// taps of parity class (py, px): t -> (ky, kx)
__device__ __forceinline__ void class_tap(int t, int py, int px, int &ky, int &kx)
{
    const int ntx = px ? 2 : 1;
    const int ty = t / ntx, tx = t - ty * ntx;
    ky = py ? (ty ? 2 : 0) : 1;
    kx = px ? (tx ? 2 : 0) : 1;
}

__device__ __forceinline__ void ldsm_x4(const bf16 *p, u32 &r0, u32 &r1, u32 &r2, u32 &r3)
{
    const u32 a = (u32)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(a));
}

__device__ __forceinline__ void ldsm_x4_t(const bf16 *p, u32 &r0, u32 &r1, u32 &r2, u32 &r3)
{
    const u32 a = (u32)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(a));
}

__device__ __forceinline__ void ldsm_x2(const bf16 *p, u32 &r0, u32 &r1)
{
    const u32 a = (u32)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n" : "=r"(r0), "=r"(r1) : "r"(a));
}

__device__ __forceinline__ void ldsm_x2_t(const bf16 *p, u32 &r0, u32 &r1)
{
    const u32 a = (u32)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];\n" : "=r"(r0), "=r"(r1) : "r"(a));
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const u32 (&a)[4], u32 b0, u32 b1)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};\n"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// 16-byte asynchronous copy; a false `valid` writes 16 zero bytes and reads nothing
__device__ __forceinline__ void cp_async16(bf16 *smem, const bf16 *gmem, bool valid)
{
    const u32 sa = (u32)__cvta_generic_to_shared(smem);
    const int n = valid ? 16 : 0;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(n) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Copy rows [r0, r0 + ROWS) x reduction indices [k0, k0 + BKT) of an operand
// into one stage: reduction-contiguous kinds as [ROWS][KC_ROW], row-contiguous
// kinds as [BKT][ROWS + 8].  Elements outside rows x [0, kend) are zero.
// rinfo (OP_IM_KC): per tile row {image offset, 2 oy - 1, 2 ox - 1, row valid}.
template <int ROWS, int MODE>
__device__ __forceinline__ void load_stage(bf16 *sm, const Operand &op, int64_t kend, int r0, int64_t k0,
                                           const int4 *rinfo)
{
    if (MODE == OP_KC || MODE == OP_IM_KC || MODE == OP_DT_KC) {
        constexpr int CH = ROWS * (BKT / 8);
#pragma unroll
        for (int c = threadIdx.x; c < CH; c += 256) {
            const int r = c >> 2, kc = (c & 3) * 8;
            const int64_t gk = k0 + kc;
            const bf16 *src = op.p;
            bool ok = gk < kend;
            if (MODE == OP_KC) {
                ok = ok && r0 + r < op.rows;
                if (ok) src = op.p + (int64_t)(r0 + r) * op.ld + gk;
            } else if (MODE == OP_DT_KC) {
                const int4 ri = rinfo[r];  // {dZ image offset, iy, ix, valid}
                const int t = (int)(gk >> op.lc), n = (int)gk & ((1 << op.lc) - 1);
                int ky, kx;
                class_tap(t, op.py, op.px, ky, kx);
                const int oy = (ri.y + 1 - ky) >> 1, ox = (ri.z + 1 - kx) >> 1;
                ok = ok && ri.w && oy < op.Ho && ox < op.Wo;
                if (ok) src = op.p + ri.x + ((int64_t)(oy * op.Wo + ox) << op.lc) + n;
            } else {
                const int4 ri = rinfo[r];
                const int tap = (int)(gk >> op.lc), ch = (int)gk & ((1 << op.lc) - 1);
                const int ky = tap / 3, kx = tap - 3 * ky;
                const int iy = ri.y + ky, ix = ri.z + kx;
                ok = ok && ri.w && iy >= 0 && iy < op.H && ix >= 0 && ix < op.W;
                if (ok) src = op.p + ri.x + ((int64_t)(iy * op.W + ix) << op.lc) + ch;
            }
            cp_async16(sm + r * KC_ROW + kc, src, ok);
        }
    } else {
        constexpr int RCH = ROWS / 8, CH = BKT * RCH;
#pragma unroll
        for (int c = threadIdx.x; c < CH; c += 256) {
            const int kr = c / RCH, rc = (c % RCH) * 8;
            const int64_t gk = k0 + kr;
            const int gr = r0 + rc;
            const bf16 *src = op.p;
            bool ok = gk < kend && gr < op.rows;
            if (MODE == OP_IM_RC && gr == op.ones_row) {  // (1, 0, ..., 0) for every position
                const uint4 one = make_uint4(ok ? 0x3F80u : 0u, 0u, 0u, 0u);  // BF16 1.0 in the low half
                *reinterpret_cast<uint4 *>(sm + kr * (ROWS + 8) + rc) = one;
                continue;
            }
            if (MODE == OP_RC) {
                if (ok) src = op.p + gk * op.ld + gr;
            } else if (MODE == OP_WT_RC) {
                const int t = (int)(gk >> op.lc), n = (int)gk & ((1 << op.lc) - 1);
                int ky, kx;
                class_tap(t, op.py, op.px, ky, kx);
                if (ok) src = op.p + (int64_t)n * op.ld + (ky * 3 + kx) * op.cin + gr;
            } else {
                const int hw = op.Ho * op.Wo;
                const int m = (int)gk;
                const int b = m / hw, rem = m - b * hw;
                const int oy = rem / op.Wo, ox = rem - oy * op.Wo;
                const int tap = gr >> op.lc, ch = gr & ((1 << op.lc) - 1);
                const int ky = tap / 3, kx = tap - 3 * ky;
                const int iy = 2 * oy - 1 + ky, ix = 2 * ox - 1 + kx;
                ok = ok && iy >= 0 && iy < op.H && ix >= 0 && ix < op.W;
                if (ok) src = op.p + (((int64_t)b * op.H * op.W + iy * op.W + ix) << op.lc) + ch;
            }
            cp_async16(sm + kr * (ROWS + 8) + rc, src, ok);
        }
    }
}

// A fragment (16 x 16 at rows mb, reduction kk) of a stage
template <int MODE>
__device__ __forceinline__ void frag_a(const bf16 *sm, int mb, int kk, u32 (&a)[4])
{
    const int lane = threadIdx.x & 31;
    if (MODE == OP_KC || MODE == OP_IM_KC || MODE == OP_DT_KC) {
        ldsm_x4(sm + (mb + (lane & 15)) * KC_ROW + kk + (lane >> 4) * 8, a[0], a[1], a[2], a[3]);
    } else {
        const int q = lane >> 3, r = lane & 7;  // matrix q: (k + 8 (q >> 1), m + 8 (q & 1))
        ldsm_x4_t(sm + (kk + (q >> 1) * 8 + r) * (BM + 8) + mb + (q & 1) * 8, a[0], a[1], a[2], a[3]);
    }
}

// B fragment (16 reduction x 8 columns at nb, kk) of a stage with TN columns
template <int MODE, int TN>
__device__ __forceinline__ void frag_b(const bf16 *sm, int nb, int kk, u32 &b0, u32 &b1)
{
    const int lane = threadIdx.x & 31;
    if (MODE == OP_KC || MODE == OP_IM_KC || MODE == OP_DT_KC) {
        ldsm_x2(sm + (nb + (lane & 7)) * KC_ROW + kk + ((lane >> 3) & 1) * 8, b0, b1);
    } else {
        ldsm_x2_t(sm + (kk + ((lane >> 3) & 1) * 8 + (lane & 7)) * (TN + 8) + nb, b0, b1);
    }
}

// Output tiles of 128 x TN (TN = 64, or 32 for 32-column products).
// Grid (ceil(N/TN), ceil(M/128), splits): split z reduces over
// [z*kchunk, min(K, (z+1)*kchunk)); EPI_ATOMIC adds into C.
// EPI_MASK_BF16 (with A = OP_DT_KC): C[pixel(row), col] = BF16(mask[...] > 0 ? v : 0).
template <int AMODE, int BMODE, int EPI, int TN>
__global__ void __launch_bounds__(256) k_gemm(int M, int N, int64_t K, int64_t kchunk, Operand A, Operand B, void *C,
                                              int ldc, const float *__restrict__ bias, const bf16 *__restrict__ mask,
                                              float *__restrict__ aux)
{
    __shared__ __align__(128) bf16 sA[NSTAGE][A_STAGE];
    __shared__ __align__(128) bf16 sB[NSTAGE][B_STAGE];
    __shared__ int4 rinfo[AMODE == OP_IM_KC || AMODE == OP_DT_KC ? BM : 1];
    __shared__ int s_pix[AMODE == OP_DT_KC ? BM : 1];
    constexpr int NI = TN / 16;  // n8 fragments per warp (warps: 4 x 2 of 32 x TN/2)
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * TN;
    const int64_t kbeg = (int64_t)blockIdx.z * kchunk, kend = min(K, kbeg + kchunk);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wm = warp & 3, wn = warp >> 2;
    if (AMODE == OP_IM_KC) {
        if (threadIdx.x < BM) {
            const int m = m0 + threadIdx.x;
            const int hw = A.Ho * A.Wo;
            const int b = m / hw, rem = m - b * hw;
            const int oy = rem / A.Wo, ox = rem - oy * A.Wo;
            rinfo[threadIdx.x] = make_int4((b * A.H * A.W) << A.lc, 2 * oy - 1, 2 * ox - 1, m < A.rows ? 1 : 0);
        }
        __syncthreads();
    }
    if (AMODE == OP_DT_KC) {
        if (threadIdx.x < BM) {
            const int m = m0 + threadIdx.x;
            const int hw = A.Hc * A.Wc;
            const int b = m / hw, rem = m - b * hw;
            const int iy = 2 * (rem / A.Wc) + A.py, ix = 2 * (rem % A.Wc) + A.px;
            rinfo[threadIdx.x] = make_int4((b * A.Ho * A.Wo) << A.lc, iy, ix, m < A.rows ? 1 : 0);
            s_pix[threadIdx.x] = ((b * A.H + iy) * A.W + ix) * ldc;
        }
        __syncthreads();
    }
    float acc[2][NI][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < NI; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;
    const int nk = (int)((kend - kbeg + BKT - 1) / BKT);
#pragma unroll
    for (int st = 0; st < NSTAGE - 1; ++st) {
        if (st < nk) {
            load_stage<BM, AMODE>(sA[st], A, kend, m0, kbeg + (int64_t)st * BKT, rinfo);
            load_stage<TN, BMODE>(sB[st], B, kend, n0, kbeg + (int64_t)st * BKT, rinfo);
        }
        cp_async_commit();
    }
    for (int it = 0; it < nk; ++it) {
        cp_async_wait<NSTAGE - 2>();
        __syncthreads();  // stage `it` landed; every warp is done with stage it - 1
        const int nx = it + NSTAGE - 1;
        if (nx < nk) {
            load_stage<BM, AMODE>(sA[nx % NSTAGE], A, kend, m0, kbeg + (int64_t)nx * BKT, rinfo);
            load_stage<TN, BMODE>(sB[nx % NSTAGE], B, kend, n0, kbeg + (int64_t)nx * BKT, rinfo);
        }
        cp_async_commit();
        const bf16 *a_s = sA[it % NSTAGE], *b_s = sB[it % NSTAGE];
#pragma unroll
        for (int kk = 0; kk < BKT; kk += 16) {
            u32 af[2][4], bfr[NI][2];
#pragma unroll
            for (int mi = 0; mi < 2; ++mi) frag_a<AMODE>(a_s, wm * 32 + mi * 16, kk, af[mi]);
#pragma unroll
            for (int ni = 0; ni < NI; ++ni)
                frag_b<BMODE, TN>(b_s, wn * (TN / 2) + ni * 8, kk, bfr[ni][0], bfr[ni][1]);
#pragma unroll
            for (int mi = 0; mi < 2; ++mi)
#pragma unroll
                for (int ni = 0; ni < NI; ++ni) mma_bf16(acc[mi][ni], af[mi], bfr[ni][0], bfr[ni][1]);
        }
    }
    cp_async_wait<0>();
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < NI; ++ni)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int row = m0 + wm * 32 + mi * 16 + g + (q >> 1) * 8;
                const int col = n0 + wn * (TN / 2) + ni * 8 + t * 2 + (q & 1);
                if (row >= M || col >= N) continue;
                const float v = acc[mi][ni][q];
                if (EPI == EPI_MASK_BF16) {
                    const int64_t o = (int64_t)s_pix[row - m0] + col;
                    ((bf16 *)C)[o] = __float2bfloat16(__bfloat162float(mask[o]) > 0.f ? v : 0.f);
                    continue;
                }
                if (EPI == EPI_ATOMIC_T) {  // C[col][row]; the ones row of A sums into aux[col]
                    if (row == A.ones_row) atomicAdd(aux + col, v);
                    else atomicAdd((float *)C + (int64_t)col * ldc + row, v);
                    continue;
                }
                if (EPI == EPI_ATOMIC && col == B.ones_row) {  // the ones row of B sums into aux[row]
                    atomicAdd(aux + row, v);
                    continue;
                }
                const int64_t o = (int64_t)row * ldc + col;
                if (EPI == EPI_STORE) ((float *)C)[o] = v;
                else if (EPI == EPI_ATOMIC) atomicAdd((float *)C + o, v);
                else if (EPI == EPI_BIAS) ((float *)C)[o] = v + bias[col];
                else ((bf16 *)C)[o] = __float2bfloat16(fmaxf(v + bias[col], 0.f));
            }
}

// ------------------------------------------------------- tcgen05 GEMM
// Forward products with both operands stored reduction-contiguous (OP_KC or
// OP_IM_KC for A, OP_KC for B) on the 5th-generation tensor cores: a
// persistent, warp-specialised kernel.  Each CTA (12 warps) walks output tiles
// of 128 x TN (tile = blockIdx.x, += gridDim.x):
//   - warps 1-7 produce: they copy operand tiles of 32 reduction indices by
//     cp.async into a 6-stage ring of shared memory and each signals the
//     stage's "full" mbarrier with cp.async.mbarrier.arrive (it fires when
//     that thread's copies have landed);
//   - one thread of warp 0 issues tcgen05.mma (M = 128, N = TN, K = 16,
//     BF16 x BF16 -> FP32) into one of two accumulators in tensor memory
//     (2 x TN FP32 columns x 128 lanes), commits each stage to its "empty"
//     mbarrier (the producers refill after it) and each finished tile to the
//     accumulator's "ready" mbarrier;
//   - warps 8-11 drain a ready accumulator (tcgen05.ld; warp w reads lane
//     quarter w % 4) through the epilogue and release it ("free" mbarrier),
//     so the epilogue of one tile overlaps the MMAs of the next.
// The ring runs across tiles; no block-wide barrier runs inside the loops.
// Shared-memory tiles use the canonical no-swizzle K-major layout: 8-row x
// 16-byte core matrices, the core matrix (r / 8, k / 8) at byte offset
// ((r / 8) * 4 + k / 8) * 128, so K-adjacent core matrices are 128 bytes apart
// (leading byte offset) and 8-row groups 512 bytes (stride byte offset).
// Every wait is bounded: on expiry a role raises GSR_FLAG_TIMEOUT in *status
// and stops; the CTA drains its copies, frees its tensor memory and returns.
constexpr int TC_BM = 128, TC_BK = 32, TC_STAGES = 6;
constexpr int TC_PRODUCER_WARPS = 7, TC_EPI_WARPS = 4;
constexpr int TC_THREADS = 32 * (1 + TC_PRODUCER_WARPS + TC_EPI_WARPS);  // 384
constexpr int TC_PRODUCERS = 32 * TC_PRODUCER_WARPS;
constexpr int TC_EPI0 = 32 * (1 + TC_PRODUCER_WARPS);                    // first epilogue thread
constexpr int TC_SPIN = 1 << 24;
constexpr int TC_BAR_SLOTS = 16;  // full[6], empty[6], ready[2], free[2]
static_assert(TC_BAR_SLOTS >= 2 * TC_STAGES + 4 && TC_BAR_SLOTS % 2 == 0, "mbarrier slots");
static_assert(TC_EPI0 % 128 == 0, "epilogue warps w % 4 = 0..3 cover the four lane quarters");

__device__ __forceinline__ u32 smem_u32(const void *p) { return (u32)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t tc_desc(const void *smem, u32 lbo, u32 sbo)
{
    return (uint64_t)((smem_u32(smem) >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);  // version 1, no swizzle
}

// kind::f16 instruction descriptor: FP32 accumulator, BF16 A and B, both K-major
__host__ __device__ constexpr u32 tc_idesc(int m, int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((u32)(n >> 3) << 17) | ((u32)(m >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, u32 count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t *bar, u32 parity)
{
    u32 ok;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}\n"
                 : "=r"(ok)
                 : "r"(smem_u32(bar)), "r"(parity)
                 : "memory");
    return ok != 0;
}

// bounded wait for the completion of the phase with the given parity
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, u32 parity)
{
    for (int i = 0; i < TC_SPIN; ++i)
        if (mbar_try(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}\n" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(smem_u32(bar))
                 : "memory");
}

// Producer share of one stage: A rows [m0, m0 + 128) and B rows [n0, n0 + TN)
// x reduction indices [k0, k0 + 32) into the core-matrix layout (zeros
// outside); producer p takes chunks p, p + TC_PRODUCERS, ...
template <int AMODE, int TN>
__device__ __forceinline__ void tc_load_stage(int p, bf16 *sa, bf16 *sb, const Operand &A, const Operand &B,
                                              int64_t K, int m0, int n0, int64_t k0)
{
    constexpr int KC = TC_BK / 8;  // chunks of 8 elements per row
    for (int c = p; c < (TC_BM + TN) * KC; c += TC_PRODUCERS) {
        const bool isa = c < TC_BM * KC;
        const int cc = isa ? c : c - TC_BM * KC;
        const int r = cc / KC, kc = cc % KC;
        const int64_t gk = k0 + kc * 8;
        bf16 *dst = (isa ? sa : sb) + ((r >> 3) * KC + kc) * 64 + (r & 7) * 8;
        const bf16 *src = A.p;
        bool ok = gk < K;
        if (isa) {
            const int m = m0 + r;
            ok = ok && m < A.rows;
            if (AMODE == OP_KC) {
                if (ok) src = A.p + (int64_t)m * A.ld + gk;
            } else if (ok) {
                const int hw = A.Ho * A.Wo;
                const int b = m / hw, rem = m - b * hw;
                const int oy = rem / A.Wo, ox = rem - oy * A.Wo;
                const int tap = (int)(gk >> A.lc), ch = (int)gk & ((1 << A.lc) - 1);
                const int ky = tap / 3, kx = tap - 3 * ky;
                const int iy = 2 * oy - 1 + ky, ix = 2 * ox - 1 + kx;
                ok = iy >= 0 && iy < A.H && ix >= 0 && ix < A.W;
                if (ok) src = A.p + (((int64_t)b * A.H * A.W + iy * A.W + ix) << A.lc) + ch;
            }
        } else {
            ok = ok && n0 + r < B.rows;
            src = B.p;
            if (ok) src = B.p + (int64_t)(n0 + r) * B.ld + gk;
        }
        cp_async16(dst, src, ok);
    }
}

template <int AMODE, int EPI, int TN>
__global__ void __launch_bounds__(TC_THREADS) k_gemm_tc(int M, int N, int64_t K, Operand A, Operand B, void *C, int ldc,
                                                        const float *__restrict__ bias, u32 *status)
{
    constexpr int NCOLS = 2 * TN <= 32 ? 32 : (2 * TN <= 64 ? 64 : (2 * TN <= 128 ? 128 : 256));
    constexpr int A_ELEMS = TC_BM * TC_BK, B_ELEMS = TN * TC_BK;
    extern __shared__ __align__(1024) uint8_t tc_smem[];
    bf16 *sA = reinterpret_cast<bf16 *>(tc_smem);
    bf16 *sB = sA + TC_STAGES * A_ELEMS;
    uint64_t *bar = reinterpret_cast<uint64_t *>(sB + TC_STAGES * B_ELEMS);
    uint64_t *full = bar, *empty = bar + TC_STAGES, *ready = bar + 2 * TC_STAGES, *freeb = ready + 2;
    u32 *tslot = reinterpret_cast<u32 *>(bar + TC_BAR_SLOTS);
    const int warp = (int)threadIdx.x >> 5, lane = (int)threadIdx.x & 31;
    const int tiles_n = (N + TN - 1) / TN, tiles = ((M + TC_BM - 1) / TC_BM) * tiles_n;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tslot)),
                     "r"((u32)NCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (threadIdx.x == 0) {
        for (int i = 0; i < TC_STAGES; ++i) {
            mbar_init(&full[i], TC_PRODUCERS);
            mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&ready[i], 1);
            mbar_init(&freeb[i], 32 * TC_EPI_WARPS);
        }
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const u32 tmem = *tslot;
    const int nk = (int)((K + TC_BK - 1) / TC_BK);
    bool failed = false;
    if (warp >= 1 && warp <= TC_PRODUCER_WARPS) {
        // producers: one stage after another over all tiles of this CTA
        const int p = (int)threadIdx.x - 32;
        int64_t g = 0;  // running stage count
        for (int t = blockIdx.x; t < tiles && !failed; t += gridDim.x) {
            const int m0 = (t / tiles_n) * TC_BM, n0 = (t % tiles_n) * TN;
            for (int k = 0; k < nk; ++k, ++g) {
                const int st = (int)(g % TC_STAGES);
                const int64_t use = g / TC_STAGES;
                if (use > 0 && !mbar_wait(&empty[st], (u32)((use - 1) & 1))) {
                    failed = true;
                    break;
                }
                tc_load_stage<AMODE, TN>(p, sA + st * A_ELEMS, sB + st * B_ELEMS, A, B, K, m0, n0,
                                         (int64_t)k * TC_BK);
                asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];\n" ::"r"(smem_u32(&full[st]))
                             : "memory");
            }
        }
        cp_async_wait<0>();
    } else if (warp == 0) {
        if (lane == 0) {
            // MMA issue: tile i accumulates into buffer i % 2
            constexpr u32 IDESC = tc_idesc(TC_BM, TN);
            int64_t g = 0;
            int i = 0;
            for (int t = blockIdx.x; t < tiles && !failed; t += gridDim.x, ++i) {
                const int ab = i & 1;
                // the epilogue must have drained this accumulator (tile i - 2)
                if (i >= 2 && !mbar_wait(&freeb[ab], (u32)(((i - 2) >> 1) & 1))) {
                    failed = true;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                const u32 dacc = tmem + (u32)(ab * TN);
                for (int k = 0; k < nk; ++k, ++g) {
                    const int st = (int)(g % TC_STAGES);
                    if (!mbar_wait(&full[st], (u32)((g / TC_STAGES) & 1))) {
                        failed = true;
                        break;
                    }
                    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
#pragma unroll
                    for (int kk = 0; kk < TC_BK / 16; ++kk) {
                        // a K step of 16 spans two core matrices along K: 256 bytes
                        const uint64_t da = tc_desc(sA + st * A_ELEMS + kk * 128, 128, (TC_BK / 8) * 128);
                        const uint64_t db = tc_desc(sB + st * B_ELEMS + kk * 128, 128, (TC_BK / 8) * 128);
                        const u32 acc = (k > 0 || kk > 0) ? 1u : 0u;
                        asm volatile("{\n\t.reg .pred p;\n\t"
                                     "setp.ne.b32 p, %4, 0;\n\t"
                                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dacc),
                                     "l"(da), "l"(db), "r"(IDESC), "r"(acc)
                                     : "memory");
                    }
                    tc_commit(&empty[st]);
                }
                tc_commit(&ready[ab]);
            }
        }
    } else {
        // epilogue: warp w drains lane quarter w % 4 of each finished tile
        const int q4 = warp & 3;
        const bool vec = ((uintptr_t)C & 15) == 0 && ((uintptr_t)bias & 15) == 0 &&
                         ldc % (EPI == EPI_BIAS ? 4 : 8) == 0;
        int i = 0;
        for (int t = blockIdx.x; t < tiles && !failed; t += gridDim.x, ++i) {
            const int ab = i & 1;
            if (!mbar_wait(&ready[ab], (u32)((i >> 1) & 1))) {
                failed = true;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const int m0 = (t / tiles_n) * TC_BM, n0 = (t % tiles_n) * TN;
            const int row = m0 + q4 * 32 + lane;
#pragma unroll
            for (int c0 = 0; c0 < TN; c0 += 16) {
                u32 r[16];
                const u32 taddr = tmem + ((u32)(q4 * 32) << 16) + (u32)(ab * TN + c0);
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
                             "%14,%15}, [%16];\n"
                             : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                               "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                               "=r"(r[14]), "=r"(r[15])
                             : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
                const int cb = n0 + c0;
                if (row < M && vec && cb + 16 <= N) {
                    // 16 consecutive outputs of this row: 16-byte stores
                    const int64_t o = (int64_t)row * ldc + cb;
                    if (EPI == EPI_BIAS) {
#pragma unroll
                        for (int q = 0; q < 16; q += 4) {
                            const float4 bq = *reinterpret_cast<const float4 *>(bias + cb + q);
                            *reinterpret_cast<float4 *>((float *)C + o + q) =
                                make_float4(__uint_as_float(r[q]) + bq.x, __uint_as_float(r[q + 1]) + bq.y,
                                            __uint_as_float(r[q + 2]) + bq.z, __uint_as_float(r[q + 3]) + bq.w);
                        }
                    } else {
#pragma unroll
                        for (int q = 0; q < 16; q += 8) {
                            uint4 pk;
                            u32 *pw = reinterpret_cast<u32 *>(&pk);
#pragma unroll
                            for (int e = 0; e < 8; e += 2) {
                                const __nv_bfloat162 h = __floats2bfloat162_rn(
                                    fmaxf(__uint_as_float(r[q + e]) + bias[cb + q + e], 0.f),
                                    fmaxf(__uint_as_float(r[q + e + 1]) + bias[cb + q + e + 1], 0.f));
                                pw[e / 2] = *reinterpret_cast<const u32 *>(&h);
                            }
                            *reinterpret_cast<uint4 *>((bf16 *)C + o + q) = pk;
                        }
                    }
                } else if (row < M) {
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const int col = cb + q;
                        if (col >= N) continue;
                        const float v = __uint_as_float(r[q]);
                        const int64_t o = (int64_t)row * ldc + col;
                        if (EPI == EPI_BIAS) ((float *)C)[o] = v + bias[col];
                        else ((bf16 *)C)[o] = __float2bfloat16(fmaxf(v + bias[col], 0.f));
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
            mbar_arrive(&freeb[ab]);
        }
    }
    failed = __syncthreads_or(failed);
    if (failed && threadIdx.x == 0) atomicOr(status, GSR_FLAG_TIMEOUT);
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"((u32)NCOLS) : "memory");
}

template <int TN>
constexpr size_t tc_smem_bytes()
{
    return (size_t)TC_STAGES * (TC_BM + TN) * TC_BK * sizeof(bf16) + TC_BAR_SLOTS * 8 + 16;
}

// --------------------------------------------------------- data movement
// x f32 [npix, 8] -> bf16 [npix, 8] (16 bytes per pixel)
__global__ void k_input_bf16(int64_t npix, const float *__restrict__ x, bf16 *__restrict__ y)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npix) return;
    const float4 a = reinterpret_cast<const float4 *>(x)[2 * i], b = reinterpret_cast<const float4 *>(x)[2 * i + 1];
    __align__(16) bf16 v[8] = {__float2bfloat16(a.x), __float2bfloat16(a.y), __float2bfloat16(a.z),
                               __float2bfloat16(a.w), __float2bfloat16(b.x), __float2bfloat16(b.y),
                               __float2bfloat16(b.z), __float2bfloat16(b.w)};
    reinterpret_cast<uint4 *>(y)[i] = *reinterpret_cast<const uint4 *>(v);
}

// out[n] += sum over rows of z[row * ld + n] (bias gradients); block 256 = 8 row
// lanes x 32 columns, grid (ceil(N/32), row splits)
__global__ void k_colsum(int64_t M, int N, int ld, const bf16 *__restrict__ z, float *__restrict__ out)
{
    const int n = blockIdx.x * 32 + (threadIdx.x & 31);
    const int64_t per = (M + gridDim.y - 1) / gridDim.y;
    const int64_t r0 = (int64_t)blockIdx.y * per, r1 = min(M, r0 + per);
    float s = 0.f;
    if (n < N)
        for (int64_t r = r0 + (threadIdx.x >> 5); r < r1; r += 8) s += __bfloat162float(z[r * ld + n]);
    __shared__ float red[8][33];
    red[threadIdx.x >> 5][threadIdx.x & 31] = s;
    __syncthreads();
    if (threadIdx.x < 32 && n < N) {
        float t = 0.f;
#pragma unroll
        for (int k = 0; k < 8; ++k) t += red[k][threadIdx.x];
        atomicAdd(&out[n], t);
    }
}

// weighted squared error of the 6 outputs: loss = (1/B) sum w r^2 and the BF16
// upstream gradient dout [B, 8] = 2 w r / B (columns 6, 7 zero)
__global__ void k_twist_loss(int B, const float *__restrict__ out, const float *__restrict__ tgt, LossW w,
                             float *__restrict__ dout, float *__restrict__ loss)
{
    __shared__ float red[256];
    float s = 0.f;
    for (int i = threadIdx.x; i < B * NOUTP; i += 256) {
        const int b = i / NOUTP, c = i % NOUTP;
        float d = 0.f;
        if (c < NOUT) {
            const float r = out[b * NOUTP + c] - tgt[b * NOUT + c];
            s += w.w[c] * r * r;
            d = 2.f * w.w[c] * r / (float)B;
        }
        dout[i] = d;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0 && loss) *loss = red[0] / (float)B;
}

// f32 [B, 6] (row stride ld_in) -> bf16 [B, 8] (columns 6, 7 zero)
__global__ void k_dout_bf16(int B, const float *__restrict__ d, int ld_in, bf16 *__restrict__ o)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * NOUTP) return;
    const int b = i / NOUTP, c = i % NOUTP;
    o[i] = __float2bfloat16(c < NOUT ? d[b * ld_in + c] : 0.f);
}

// dz = d * (h > 0) in BF16
__global__ void k_relu_bwd(int64_t n, const float *__restrict__ d, const bf16 *__restrict__ h, bf16 *__restrict__ dz)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dz[i] = __float2bfloat16(__bfloat162float(h[i]) > 0.f ? d[i] : 0.f);
}

// FP32 masters (flat layout) -> BF16 GEMM operands
__global__ void k_pack(const float *__restrict__ master, bf16 *__restrict__ wb, Layout L)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= L.wb_off[NSEG]) return;
    int s = 0;
    while (s < NSEG - 1 && i >= L.wb_off[s + 1]) ++s;
    const int64_t j = i - L.wb_off[s];
    float v = 0.f;
    if (s < NL) {
        const int cp = L.cinp[s], ci = L.cin[s];
        const int64_t K = 9 * (int64_t)cp;
        const int64_t n = j / K, kk = j % K;
        const int tap = (int)(kk / cp), c = (int)(kk % cp);
        if (c < ci) v = master[L.w_off[s] + (n * 9 + tap) * ci + c];
    } else if (s == NL || j < (int64_t)NOUT * HID) {
        v = master[L.w_off[s] + j];
    }
    wb[i] = __float2bfloat16(v);
}

__global__ void k_adam(int64_t n, float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, float lr, float b1, float b2, float eps, float bc1, float bc2)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
}

// network input from a 160x120 render and a full-resolution frame (box average)
__global__ void k_make_input(int h, int w, const float *__restrict__ rgb_r, const float *__restrict__ d_r,
                             const float *__restrict__ rgb_i, const float *__restrict__ d_i, float inv_scale,
                             float *__restrict__ out)
{
    constexpr int H = GSR_WS_IN_H, W = GSR_WS_IN_W, HW = H * W;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= HW) return;
    const int i = p / W, j = p % W;
    const int y0 = (int)(((int64_t)i * h) / H), y1 = (int)(((int64_t)(i + 1) * h) / H);
    const int x0 = (int)(((int64_t)j * w) / W), x1 = (int)(((int64_t)(j + 1) * w) / W);
    const int64_t hw = (int64_t)h * w;
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, sd = 0.f;
    int nd = 0;
    for (int y = y0; y < y1; ++y)
        for (int x = x0; x < x1; ++x) {
            const int64_t q = (int64_t)y * w + x;
            s0 += rgb_i[q];
            s1 += rgb_i[hw + q];
            s2 += rgb_i[2 * hw + q];
            const float d = d_i[q];
            if (d > 0.f) {
                sd += d;
                ++nd;
            }
        }
    const float inv = 1.f / (float)((y1 - y0) * (x1 - x0));
    const float di = nd ? sd / (float)nd : 0.f, dr = d_r[p];
    const float r0 = rgb_r[p], r1 = rgb_r[HW + p], r2 = rgb_r[2 * HW + p];
    float *o = out + (int64_t)p * 8;
    o[0] = r0;
    o[1] = r1;
    o[2] = r2;
    o[3] = dr * inv_scale;
    o[4] = s0 * inv - r0;
    o[5] = s1 * inv - r1;
    o[6] = s2 * inv - r2;
    o[7] = (dr > 0.f && di > 0.f) ? (di - dr) * inv_scale : 0.f;
}

unsigned blocks(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

void make_layout(Layout &L)
{
    int64_t o = 0, wo = 0;
    for (int l = 0; l < NSEG; ++l) {
        const int64_t nout = l < NL ? COUT[l] : (l == NL ? HID : NOUT);
        const int64_t kin = l < NL ? 9 * (int64_t)CIN[l] : (l == NL ? FLAT : HID);
        const int64_t kst = l < NL ? 9 * (int64_t)CINP[l] : kin;
        const int64_t nst = l == NL + 1 ? NOUTP : nout;
        L.w_off[l] = o;
        o += nout * kin;
        L.b_off[l] = o;
        o += nout;
        L.wb_off[l] = wo;
        wo += nst * kst;
    }
    L.wb_off[NSEG] = wo;
    L.n_params = o;
    for (int l = 0; l < NL; ++l) {
        L.cin[l] = CIN[l];
        L.cinp[l] = CINP[l];
    }
}

} // namespace

// ------------------------------------------------------------------ state
struct gsr_warmstart {
    int max_batch = 0;
    int last_batch = 0;  // batch of the last forward (0 = none)
    int64_t step = 0;
    std::string err;
    Layout L{};
    DevBuf master, m1, m2, grad, wb;
    DevBuf act[NL + 2];  // act[0] input (16 ch), act[l+1] conv l output, act[NL+1] dense-1 output
    DevBuf dz, dz2, dbuf, out, dout32, dout, loss_tmp;  // dz / dz2: ping-pong upstream gradients
    DevBuf status;         // u32 device flags raised by kernels (bounded waits)
    // side streams of the backward: per convolution layer the weight gradient
    // runs on side[0] while the four parity-class data-gradient GEMMs run on
    // the caller's stream and side[1..3] (forked and joined with events)
    cudaStream_t side[4] = {};
    cudaEvent_t ev_fork = nullptr, ev_part[4] = {}, ev_wgrad[NL] = {};
    int tc_min_k = -1;     // forward products with K >= tc_min_k run on tcgen05 (< 0: never; the default,
                           // as the mma.sync kernel measured faster on every layer)
};

namespace {

gsr_status ws_fail(gsr_warmstart *w, gsr_status s, const std::string &m)
{
    if (w) w->err = m;
    return s;
}

gsr_status ws_alloc(gsr_warmstart *w, DevBuf &b, size_t bytes)
{
    if (cudaMalloc(&b.p, bytes ? bytes : 16) != cudaSuccess) {
        (void)cudaGetLastError();
        b.p = nullptr;
        return ws_fail(w, GSR_ERR_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
    }
    b.bytes = bytes;
    return GSR_OK;
}

gsr_status launched(gsr_warmstart *w)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return ws_fail(w, GSR_ERR_CUDA, std::string("launch failed: ") + cudaGetErrorString(e));
    return GSR_OK;
}

#define WS_TRY(e)                    \
    do {                             \
        gsr_status _s = (e);         \
        if (_s != GSR_OK) return _s; \
    } while (0)

// Number of reduction splits for a GEMM with the given output tiles: enough
// CTAs to cover the 152 SMs about twice, each split at least 8 k-tiles long.
int64_t split_count(int M, int N, int64_t K, int tn)
{
    const int64_t tiles = (int64_t)((M + BM - 1) / BM) * ((N + tn - 1) / tn);
    int64_t s = std::max<int64_t>(1, 304 / tiles);
    s = std::min<int64_t>(s, std::max<int64_t>(1, K / (8 * BKT)));
    return std::min<int64_t>(s, 65535);
}

Operand dense(const bf16 *p, int ld, int rows)
{
    Operand o{};
    o.p = p;
    o.ld = ld;
    o.rows = rows;
    o.ones_row = -1;
    return o;
}

int ilog2(int c)
{
    int l = 0;
    while ((1 << l) < c) ++l;
    return l;
}

// im2col operand of conv layer l over the stored activation x (rows = bound on
// the row index: output positions for OP_IM_KC, 9 x channels for OP_IM_RC)
Operand im2col(const bf16 *x, int l, int rows)
{
    Operand o{};
    o.p = x;
    o.rows = rows;
    o.H = HIN[l];
    o.W = WIN[l];
    o.lc = ilog2(CINP[l]);
    o.Ho = HOUT[l];
    o.Wo = WOUT[l];
    o.ones_row = -1;
    return o;
}

template <int AMODE, int BMODE, int EPI>
gsr_status gemm(gsr_warmstart *w, int M, int N, int64_t K, const Operand &A, const Operand &B, void *C, int ldc,
                const float *bias, cudaStream_t s, const bf16 *mask = nullptr, float *aux = nullptr)
{
    auto bad = [](const Operand &o, int mode) {
        if (((uintptr_t)o.p) & 15) return true;
        if ((mode == OP_KC || mode == OP_RC || mode == OP_WT_RC) && (o.ld % 8)) return true;
        if ((mode == OP_RC || mode == OP_IM_RC || mode == OP_WT_RC) && (o.rows % 8)) return true;
        if (mode == OP_WT_RC && (o.cin % 8)) return true;
        return false;
    };
    // reduction-contiguous operands are copied in whole 8-element chunks of k
    const bool kc = AMODE == OP_KC || AMODE == OP_IM_KC || AMODE == OP_DT_KC || BMODE == OP_KC || BMODE == OP_IM_KC;
    if (bad(A, AMODE) || bad(B, BMODE) || (kc && (K % 8)))
        return ws_fail(w, GSR_ERR_INVALID_ARG, "GEMM operand not 16-byte aligned");
    const int tn = N <= 32 ? 32 : 64;
    int64_t splits = 1;
    if (EPI == EPI_ATOMIC || EPI == EPI_ATOMIC_T) splits = split_count(M, N, K, tn);
    int64_t kchunk = (K + splits - 1) / splits;
    kchunk = (kchunk + BKT - 1) / BKT * BKT;
    splits = (K + kchunk - 1) / kchunk;
    dim3 grid((unsigned)((N + tn - 1) / tn), (unsigned)((M + BM - 1) / BM), (unsigned)std::max<int64_t>(1, splits));
    if (tn == 32)
        k_gemm<AMODE, BMODE, EPI, 32><<<grid, 256, 0, s>>>(M, N, K, kchunk, A, B, C, ldc, bias, mask, aux);
    else
        k_gemm<AMODE, BMODE, EPI, 64><<<grid, 256, 0, s>>>(M, N, K, kchunk, A, B, C, ldc, bias, mask, aux);
    return launched(w);
}

template <int AMODE, int EPI, int TN>
gsr_status gemm_tc_n(gsr_warmstart *w, int M, int N, int64_t K, const Operand &A, const Operand &B, void *C, int ldc,
                     const float *bias, cudaStream_t s)
{
    constexpr size_t smem = tc_smem_bytes<TN>();
    static bool attr_set = false;  // per process; the attribute is per function and device-independent here
    if (!attr_set) {
        if (cudaFuncSetAttribute(k_gemm_tc<AMODE, EPI, TN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return ws_fail(w, GSR_ERR_CUDA, "tcgen05 GEMM: shared-memory attribute refused");
        attr_set = true;
    }
    // persistent: as many CTAs as fit at once (shared memory and tensor memory
    // allow two per SM), each walking tiles blockIdx.x, += gridDim.x
    const int64_t tiles = (int64_t)((N + TN - 1) / TN) * ((M + TC_BM - 1) / TC_BM);
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(tiles, 2 * 152));
    k_gemm_tc<AMODE, EPI, TN><<<grid, TC_THREADS, smem, s>>>(M, N, K, A, B, C, ldc, bias, (u32 *)w->status.p);
    return launched(w);
}

// forward product on the tensor cores (N = 256 as two 128-column tiles) when N is one of 32, 64, 128, 256 and
// K a multiple of 8 (else the mma.sync kernel)
template <int AMODE, int EPI>
gsr_status gemm_fwd(gsr_warmstart *w, int M, int N, int64_t K, const Operand &A, const Operand &B, void *C, int ldc,
                    const float *bias, cudaStream_t s)
{
    if (w->tc_min_k >= 0 && K >= w->tc_min_k && (K % 8) == 0 && (((uintptr_t)A.p | (uintptr_t)B.p) & 15) == 0 && (AMODE != OP_KC || A.ld % 8 == 0) &&
        B.ld % 8 == 0) {
        switch (N) {
        case 32: return gemm_tc_n<AMODE, EPI, 32>(w, M, N, K, A, B, C, ldc, bias, s);
        case 64: return gemm_tc_n<AMODE, EPI, 64>(w, M, N, K, A, B, C, ldc, bias, s);
        case 128:
        case 256: return gemm_tc_n<AMODE, EPI, 128>(w, M, N, K, A, B, C, ldc, bias, s);
        default: break;
        }
    }
    return gemm<AMODE, OP_KC, EPI>(w, M, N, K, A, B, C, ldc, bias, s);
}

gsr_status pack(gsr_warmstart *w, cudaStream_t s)
{
    k_pack<<<blocks(w->L.wb_off[NSEG]), 256, 0, s>>>((const float *)w->master.p, (bf16 *)w->wb.p, w->L);
    return launched(w);
}

gsr_status backward_impl(gsr_warmstart *w, const bf16 *dout, int batch, cudaStream_t s)
{
    const int64_t B = batch;
    const Layout &L = w->L;
    const bf16 *wb = (const bf16 *)w->wb.p;
    float *grad = (float *)w->grad.p;
    float *dbuf = (float *)w->dbuf.p;
    bf16 *dz = (bf16 *)w->dz.p;
    if (cudaMemsetAsync(grad, 0, sizeof(float) * L.n_params, s) != cudaSuccess)
        return ws_fail(w, GSR_ERR_CUDA, "memset failed");
    // dense 2: dW = dout^T h1, db = column sums of dout, dh1 = dout W
    WS_TRY((gemm<OP_RC, OP_RC, EPI_ATOMIC>(w, NOUT, HID, B, dense(dout, NOUTP, NOUTP),
                                           dense((const bf16 *)w->act[NL + 1].p, HID, HID), grad + L.w_off[NL + 1],
                                           HID, nullptr, s)));
    k_colsum<<<dim3(1, 4), 256, 0, s>>>(B, NOUT, NOUTP, dout, grad + L.b_off[NL + 1]);
    WS_TRY(launched(w));
    WS_TRY((gemm<OP_KC, OP_RC, EPI_STORE>(w, batch, HID, NOUTP, dense(dout, NOUTP, batch),
                                          dense(wb + L.wb_off[NL + 1], HID, HID), dbuf, HID, nullptr, s)));
    k_relu_bwd<<<blocks(B * HID), 256, 0, s>>>(B * HID, dbuf, (const bf16 *)w->act[NL + 1].p, dz);
    WS_TRY(launched(w));
    // dense 1: dW = dz^T h0, db, dh0 = dz W, then the mask of conv 5's ReLU
    WS_TRY((gemm<OP_RC, OP_RC, EPI_ATOMIC>(w, HID, FLAT, B, dense(dz, HID, HID),
                                           dense((const bf16 *)w->act[NL].p, FLAT, FLAT), grad + L.w_off[NL], FLAT,
                                           nullptr, s)));
    k_colsum<<<dim3(HID / 32, 4), 256, 0, s>>>(B, HID, HID, dz, grad + L.b_off[NL]);
    WS_TRY(launched(w));
    WS_TRY((gemm<OP_KC, OP_RC, EPI_STORE>(w, batch, FLAT, HID, dense(dz, HID, batch), dense(wb + L.wb_off[NL], FLAT, FLAT),
                                          dbuf, FLAT, nullptr, s)));
    k_relu_bwd<<<blocks(B * FLAT), 256, 0, s>>>(B * FLAT, dbuf, (const bf16 *)w->act[NL].p, dz);
    WS_TRY(launched(w));
    auto ev = [&](cudaError_t e) { return e == cudaSuccess ? GSR_OK : ws_fail(w, GSR_ERR_CUDA, "stream event failed"); };
    for (int l = NL - 1; l >= 0; --l) {
        const int64_t M = B * HOUT[l] * WOUT[l];
        const int K = 9 * CINP[l], N = COUT[l];
        // dz of this layer is complete on s: fork
        WS_TRY(ev(cudaEventRecord(w->ev_fork, s)));
        for (int i = 0; i < 4; ++i) WS_TRY(ev(cudaStreamWaitEvent(w->side[i], w->ev_fork, 0)));
        // weight and bias gradients in one GEMM reducing over positions (on
        // side[0]); the im2col operand carries an extra row of ones whose
        // product is the bias gradient.  The larger of (N, K) takes the 128-row
        // side of the tile.
        Operand im = im2col((const bf16 *)w->act[l].p, l, K + 8);
        im.ones_row = K;
        if (K > N) {
            WS_TRY((gemm<OP_IM_RC, OP_RC, EPI_ATOMIC_T>(w, K + 1, N, M, im, dense(dz, N, N), grad + L.w_off[l], K,
                                                        nullptr, w->side[0], nullptr, grad + L.b_off[l])));
        } else {
            WS_TRY((gemm<OP_RC, OP_IM_RC, EPI_ATOMIC>(w, N, K + 1, M, dense(dz, N, N), im, grad + L.w_off[l], K,
                                                      nullptr, w->side[0], nullptr, grad + L.b_off[l])));
        }
        WS_TRY(ev(cudaEventRecord(w->ev_wgrad[l], w->side[0])));
        if (l == 0) break;
        // data gradient straight into the previous layer's output gradient (ReLU
        // mask applied), one GEMM per parity class of input pixels
        bf16 *dz_prev = dz == (bf16 *)w->dz.p ? (bf16 *)w->dz2.p : (bf16 *)w->dz.p;
        // dz_prev is the buffer the weight gradient of layer l + 1 reads
        if (l + 1 < NL)
            for (int i = 0; i < 4; ++i) {
                cudaStream_t sc = i == 0 ? s : w->side[i];
                WS_TRY(ev(cudaStreamWaitEvent(sc, w->ev_wgrad[l + 1], 0)));
            }
        for (int cls = 0; cls < 4; ++cls) {
            cudaStream_t sc = cls == 0 ? s : w->side[cls];
            const int py = cls >> 1, px = cls & 1;
            const int Hc = (HIN[l] - py + 1) >> 1, Wc = (WIN[l] - px + 1) >> 1;
            const int rows = batch * Hc * Wc, ntap = (py ? 2 : 1) * (px ? 2 : 1);
            if (rows == 0) continue;
            Operand a{}, bw{};
            a.p = dz;
            a.rows = rows;
            a.H = HIN[l];
            a.W = WIN[l];
            a.lc = ilog2(N);
            a.Ho = HOUT[l];
            a.Wo = WOUT[l];
            a.py = py;
            a.px = px;
            a.Hc = Hc;
            a.Wc = Wc;
            bw.p = wb + L.wb_off[l];
            bw.ld = K;
            bw.rows = CINP[l];
            bw.lc = ilog2(N);
            bw.py = py;
            bw.px = px;
            bw.cin = CINP[l];
            WS_TRY((gemm<OP_DT_KC, OP_WT_RC, EPI_MASK_BF16>(w, rows, CINP[l], (int64_t)ntap * N, a, bw, dz_prev,
                                                             CINP[l], nullptr, sc, (const bf16 *)w->act[l].p)));
        }
        // join the parity classes: the next layer reads all of dz_prev
        for (int i = 1; i < 4; ++i) {
            WS_TRY(ev(cudaEventRecord(w->ev_part[i], w->side[i])));
            WS_TRY(ev(cudaStreamWaitEvent(s, w->ev_part[i], 0)));
        }
        dz = dz_prev;
    }
    // every weight gradient is in before the caller's stream goes on (Adam)
    for (int l = 0; l < NL; ++l) WS_TRY(ev(cudaStreamWaitEvent(s, w->ev_wgrad[l], 0)));
    return GSR_OK;
}

} // namespace

extern "C" {

int64_t gsr_warmstart_num_params(void)
{
    Layout L;
    make_layout(L);
    return L.n_params;
}

void gsr_warmstart_default_opts(gsr_warmstart_opts *o)
{
    if (!o) return;
    o->lr = 1e-3f;
    o->beta1 = 0.9f;
    o->beta2 = 0.999f;
    o->eps = 1e-8f;
    for (int i = 0; i < 6; ++i) o->w[i] = 1.f;
}

void gsr_warmstart_destroy(gsr_warmstart *w)
{
    if (!w) return;
    cudaDeviceSynchronize();
    DevBuf *bufs[] = {&w->master, &w->m1, &w->m2, &w->grad, &w->wb, &w->dz, &w->dz2, &w->dbuf,
                      &w->out, &w->dout32, &w->dout, &w->loss_tmp, &w->status};
    for (DevBuf *b : bufs)
        if (b->p) cudaFree(b->p);
    for (int l = 0; l < NL + 2; ++l)
        if (w->act[l].p) cudaFree(w->act[l].p);
    for (int i = 0; i < 4; ++i) {
        if (w->side[i]) cudaStreamDestroy(w->side[i]);
        if (w->ev_part[i]) cudaEventDestroy(w->ev_part[i]);
    }
    for (int l = 0; l < NL; ++l)
        if (w->ev_wgrad[l]) cudaEventDestroy(w->ev_wgrad[l]);
    if (w->ev_fork) cudaEventDestroy(w->ev_fork);
    delete w;
}

gsr_status gsr_warmstart_create(gsr_warmstart **out, int32_t max_batch, uint64_t seed)
{
    if (!out || max_batch <= 0 || max_batch > 1024) return GSR_ERR_INVALID_ARG;  // grid.y of the first GEMM
    *out = nullptr;
    gsr_warmstart *w = new (std::nothrow) gsr_warmstart();
    if (!w) return GSR_ERR_OOM;
    w->max_batch = max_batch;
    make_layout(w->L);
    const Layout &L = w->L;
    const int64_t P = L.n_params, B = max_batch;
    int64_t max_dz = B * FLAT, max_dbuf = B * FLAT;
    for (int l = 0; l < NL; ++l) {
        const int64_t M = B * HOUT[l] * WOUT[l];
        max_dz = std::max(max_dz, M * COUT[l]);
        max_dz = std::max(max_dz, B * HIN[l] * WIN[l] * CINP[l]);
    }
    gsr_status st = GSR_OK;
    auto A = [&](DevBuf &b, size_t bytes) {
        if (st == GSR_OK) st = ws_alloc(w, b, bytes);
    };
    A(w->master, sizeof(float) * P);
    A(w->m1, sizeof(float) * P);
    A(w->m2, sizeof(float) * P);
    A(w->grad, sizeof(float) * P);
    A(w->wb, sizeof(bf16) * L.wb_off[NSEG]);
    A(w->act[0], sizeof(bf16) * B * HIN[0] * WIN[0] * CINP[0]);
    for (int l = 0; l < NL; ++l) {
        const int64_t M = B * HOUT[l] * WOUT[l];
        A(w->act[l + 1], sizeof(bf16) * M * COUT[l]);
    }
    A(w->act[NL + 1], sizeof(bf16) * B * HID);
    A(w->dz, sizeof(bf16) * max_dz);
    A(w->dz2, sizeof(bf16) * max_dz);
    A(w->dbuf, sizeof(float) * max_dbuf);
    A(w->out, sizeof(float) * B * NOUTP);
    A(w->dout32, sizeof(float) * B * NOUTP);
    A(w->dout, sizeof(bf16) * B * NOUTP);
    A(w->loss_tmp, sizeof(float) * 4);
    A(w->status, sizeof(u32) * 4);
    for (int i = 0; i < 4 && st == GSR_OK; ++i)
        if (cudaStreamCreateWithFlags(&w->side[i], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&w->ev_part[i], cudaEventDisableTiming) != cudaSuccess)
            st = ws_fail(w, GSR_ERR_CUDA, "stream / event creation failed");
    for (int l = 0; l < NL && st == GSR_OK; ++l)
        if (cudaEventCreateWithFlags(&w->ev_wgrad[l], cudaEventDisableTiming) != cudaSuccess)
            st = ws_fail(w, GSR_ERR_CUDA, "event creation failed");
    if (st == GSR_OK && cudaEventCreateWithFlags(&w->ev_fork, cudaEventDisableTiming) != cudaSuccess)
        st = ws_fail(w, GSR_ERR_CUDA, "event creation failed");
    if (st != GSR_OK) {
        gsr_warmstart_destroy(w);
        return st;
    }
    // He-normal weights from the seed (output layer x 0.01), zero biases
    std::vector<float> h((size_t)P, 0.f);
    std::mt19937_64 rng(seed);
    auto fill = [&](int64_t off, int64_t n, int64_t fan_in, float scale) {
        std::normal_distribution<float> nd(0.f, scale * sqrtf(2.f / (float)fan_in));
        for (int64_t i = 0; i < n; ++i) h[(size_t)(off + i)] = nd(rng);
    };
    for (int l = 0; l < NL; ++l) fill(L.w_off[l], (int64_t)COUT[l] * 9 * CIN[l], 9 * CIN[l], 1.f);
    fill(L.w_off[NL], (int64_t)HID * FLAT, FLAT, 1.f);
    fill(L.w_off[NL + 1], (int64_t)NOUT * HID, HID, 0.01f);
    if (cudaMemset(w->status.p, 0, sizeof(u32) * 4) != cudaSuccess ||
        cudaMemcpy(w->master.p, h.data(), sizeof(float) * P, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(w->m1.p, 0, sizeof(float) * P) != cudaSuccess ||
        cudaMemset(w->m2.p, 0, sizeof(float) * P) != cudaSuccess || pack(w, 0) != GSR_OK ||
        cudaDeviceSynchronize() != cudaSuccess) {
        (void)cudaGetLastError();
        gsr_warmstart_destroy(w);
        return GSR_ERR_CUDA;
    }
    *out = w;
    return GSR_OK;
}

const char *gsr_warmstart_last_error(const gsr_warmstart *w) { return w ? w->err.c_str() : "null network"; }

gsr_status gsr_warmstart_set_params(gsr_warmstart *w, const float *params, void *stream)
{
    if (!w || !params) return GSR_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t bytes = sizeof(float) * w->L.n_params;
    if (cudaMemcpyAsync(w->master.p, params, bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(w->m1.p, 0, bytes, s) != cudaSuccess || cudaMemsetAsync(w->m2.p, 0, bytes, s) != cudaSuccess)
        return ws_fail(w, GSR_ERR_CUDA, "parameter copy failed");
    w->step = 0;
    return pack(w, s);
}

gsr_status gsr_warmstart_get_params(gsr_warmstart *w, float *params, void *stream)
{
    if (!w || !params) return GSR_ERR_INVALID_ARG;
    if (cudaMemcpyAsync(params, w->master.p, sizeof(float) * w->L.n_params, cudaMemcpyDeviceToDevice,
                        (cudaStream_t)stream) != cudaSuccess)
        return ws_fail(w, GSR_ERR_CUDA, "parameter copy failed");
    return GSR_OK;
}

gsr_status gsr_warmstart_forward(gsr_warmstart *w, const float *x, int32_t batch, float *out, void *stream)
{
    if (!w || !x || batch <= 0) return GSR_ERR_INVALID_ARG;
    if (((uintptr_t)x) & 15) return ws_fail(w, GSR_ERR_INVALID_ARG, "x must be 16-byte aligned");
    if (batch > w->max_batch) return ws_fail(w, GSR_ERR_CAPACITY, "batch exceeds the network's max_batch");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t B = batch;
    const Layout &L = w->L;
    const bf16 *wb = (const bf16 *)w->wb.p;
    const float *master = (const float *)w->master.p;
    w->last_batch = 0;
    const int64_t npix = B * HIN[0] * WIN[0];
    k_input_bf16<<<blocks(npix), 256, 0, s>>>(npix, x, (bf16 *)w->act[0].p);
    WS_TRY(launched(w));
    for (int l = 0; l < NL; ++l) {
        const int64_t M = B * HOUT[l] * WOUT[l];
        const int K = 9 * CINP[l];
        WS_TRY((gemm_fwd<OP_IM_KC, EPI_BIAS_RELU_BF16>(w, (int)M, COUT[l], K,
                                                       im2col((const bf16 *)w->act[l].p, l, (int)M),
                                                       dense(wb + L.wb_off[l], K, COUT[l]), w->act[l + 1].p, COUT[l],
                                                       master + L.b_off[l], s)));
    }
    WS_TRY((gemm_fwd<OP_KC, EPI_BIAS_RELU_BF16>(w, batch, HID, FLAT, dense((const bf16 *)w->act[NL].p, FLAT, batch),
                                                dense(wb + L.wb_off[NL], FLAT, HID), w->act[NL + 1].p, HID,
                                                master + L.b_off[NL], s)));
    WS_TRY((gemm<OP_KC, OP_KC, EPI_BIAS>(w, batch, NOUT, HID, dense((const bf16 *)w->act[NL + 1].p, HID, batch),
                                         dense(wb + L.wb_off[NL + 1], HID, NOUTP), w->out.p, NOUTP,
                                         master + L.b_off[NL + 1], s)));
    if (out && cudaMemcpy2DAsync(out, sizeof(float) * NOUT, w->out.p, sizeof(float) * NOUTP, sizeof(float) * NOUT,
                                 (size_t)B, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return ws_fail(w, GSR_ERR_CUDA, "output copy failed");
    w->last_batch = batch;
    return GSR_OK;
}

gsr_status gsr_warmstart_backward(gsr_warmstart *w, const float *d_out, int32_t batch, float *grad, void *stream)
{
    if (!w || !d_out || batch <= 0) return GSR_ERR_INVALID_ARG;
    if (batch != w->last_batch) return ws_fail(w, GSR_ERR_STATE, "backward needs a forward of the same batch");
    cudaStream_t s = (cudaStream_t)stream;
    k_dout_bf16<<<blocks((int64_t)batch * NOUTP), 256, 0, s>>>(batch, d_out, NOUT, (bf16 *)w->dout.p);
    WS_TRY(launched(w));
    WS_TRY(backward_impl(w, (const bf16 *)w->dout.p, batch, s));
    if (grad && cudaMemcpyAsync(grad, w->grad.p, sizeof(float) * w->L.n_params, cudaMemcpyDeviceToDevice, s) !=
                    cudaSuccess)
        return ws_fail(w, GSR_ERR_CUDA, "gradient copy failed");
    return GSR_OK;
}

gsr_status gsr_warmstart_train_step(gsr_warmstart *w, const float *x, const float *target, int32_t batch,
                                    const gsr_warmstart_opts *opts, float *loss, void *stream)
{
    if (!w || !x || !target || batch <= 0) return GSR_ERR_INVALID_ARG;
    gsr_warmstart_opts o;
    gsr_warmstart_default_opts(&o);
    if (opts) o = *opts;
    if (!(o.lr >= 0.f) || !(o.beta1 >= 0.f && o.beta1 < 1.f) || !(o.beta2 >= 0.f && o.beta2 < 1.f) || !(o.eps > 0.f))
        return ws_fail(w, GSR_ERR_INVALID_ARG, "invalid Adam options");
    cudaStream_t s = (cudaStream_t)stream;
    WS_TRY(gsr_warmstart_forward(w, x, batch, nullptr, stream));
    LossW lw;
    for (int i = 0; i < NOUT; ++i) lw.w[i] = o.w[i];
    k_twist_loss<<<1, 256, 0, s>>>(batch, (const float *)w->out.p, target, lw, (float *)w->dout32.p,
                                   loss ? loss : (float *)w->loss_tmp.p);
    WS_TRY(launched(w));
    k_dout_bf16<<<blocks((int64_t)batch * NOUTP), 256, 0, s>>>(batch, (const float *)w->dout32.p, NOUTP,
                                                               (bf16 *)w->dout.p);
    WS_TRY(launched(w));
    WS_TRY(backward_impl(w, (const bf16 *)w->dout.p, batch, s));
    w->step += 1;
    const float bc1 = 1.f - powf(o.beta1, (float)w->step), bc2 = 1.f - powf(o.beta2, (float)w->step);
    k_adam<<<blocks(w->L.n_params), 256, 0, s>>>(w->L.n_params, (float *)w->master.p, (const float *)w->grad.p,
                                                 (float *)w->m1.p, (float *)w->m2.p, o.lr, o.beta1, o.beta2, o.eps,
                                                 bc1, bc2);
    WS_TRY(launched(w));
    return pack(w, s);
}

gsr_status gsr_warmstart_set_kernels(gsr_warmstart *w, int32_t tcgen05_min_k)
{
    if (!w) return GSR_ERR_INVALID_ARG;
    w->tc_min_k = tcgen05_min_k;
    return GSR_OK;
}

gsr_status gsr_warmstart_check(gsr_warmstart *w, void *stream)
{
    if (!w) return GSR_ERR_INVALID_ARG;
    u32 flags = 0;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaStreamSynchronize(s) != cudaSuccess ||
        cudaMemcpy(&flags, w->status.p, sizeof(u32), cudaMemcpyDeviceToHost) != cudaSuccess)
        return ws_fail(w, GSR_ERR_CUDA, "status read failed");
    if (flags & GSR_FLAG_TIMEOUT) {
        cudaMemset(w->status.p, 0, sizeof(u32));
        return ws_fail(w, GSR_ERR_TIMEOUT, "a tensor-core GEMM wait expired");
    }
    return GSR_OK;
}

gsr_status gsr_warmstart_make_input(const float *rgb_r, const float *depth_r, const float *rgb_i,
                                    const float *depth_i, int32_t h, int32_t w, float depth_scale, float *out,
                                    void *stream)
{
    if (!rgb_r || !depth_r || !rgb_i || !depth_i || !out || h < GSR_WS_IN_H || w < GSR_WS_IN_W ||
        !(depth_scale > 0.f))
        return GSR_ERR_INVALID_ARG;
    k_make_input<<<blocks(GSR_WS_IN_H * GSR_WS_IN_W), 256, 0, (cudaStream_t)stream>>>(
        h, w, rgb_r, depth_r, rgb_i, depth_i, 1.f / depth_scale, out);
    return cudaGetLastError() == cudaSuccess ? GSR_OK : GSR_ERR_CUDA;
}

} // extern "C"
