// adam.cu -- optimiser steps.
//
// Gaussians: bias-corrected Adam on the 14 parameters of every Gaussian with
// the gradient of the isotropic regulariser L_reg (Sec. 3.4) fused in:
//   L_reg = (1/n) sum_k |s_k - mean(s_k)|_1,  s = exp(log_scale).
// The step counter lives in device memory so that a captured CUDA graph can
// be replayed: a one-thread kernel advances it and writes the bias
// corrections before the update kernel reads them.
//
// Pose (tracking, Sec. 3.5): Adam on the twist of a left perturbation, then
// the retraction T <- exp(delta^) T with the closed-form SE(3) exponential.
#include <math.h>

#include "gsr_internal.cuh"

namespace {


__global__ void k_adam_prep(int32_t *step, float b1, float b2, float *bc)
{
    int t = *step + 1;
    *step = t;
    bc[0] = 1.f - powf(b1, (float)t);
    bc[1] = 1.f - powf(b2, (float)t);
}

__device__ __forceinline__ void adam1(float &p, float g, float &m, float &v, float lr, float b1, float b2, float eps,
                                      float bc1, float bc2)
{
    adam_update(p, g, m, v, lr, b1, b2, eps, bc1, bc2);
}

// Flat layout: the five parameter arrays are one index space of float4
// chunks (mean, log-scale, quaternion, opacity, colour; 14 n floats); each
// thread updates one float4 of one array (its parameter, gradient and both
// moments: 4 vector loads, 3 vector stores), so every access is a coalesced
// 16-byte vector.  The isotropic regulariser needs a Gaussian's three scales
// together: the log-scale chunks are handled as groups of 4 Gaussians
// (3 float4), one group per thread.  Arrays whose base is not 16-byte aligned,
// and tails, take a scalar path.
struct FlatSeg {
    float *p, *m, *v;
    const float *g;
    float lr;
    int64_t n;  // floats
};

__device__ __forceinline__ void adam_chunk(const FlatSeg &sgm, int64_t c4, const gsr_adam_opts &o, float bc1, float bc2)
{
    const int64_t off = 4 * c4;
    if (off + 4 <= sgm.n) {
        float4 p = reinterpret_cast<float4 *>(sgm.p)[c4], m = reinterpret_cast<float4 *>(sgm.m)[c4];
        float4 v = reinterpret_cast<float4 *>(sgm.v)[c4];
        const float4 g = reinterpret_cast<const float4 *>(sgm.g)[c4];
        adam1(p.x, g.x, m.x, v.x, sgm.lr, o.beta1, o.beta2, o.eps, bc1, bc2);
        adam1(p.y, g.y, m.y, v.y, sgm.lr, o.beta1, o.beta2, o.eps, bc1, bc2);
        adam1(p.z, g.z, m.z, v.z, sgm.lr, o.beta1, o.beta2, o.eps, bc1, bc2);
        adam1(p.w, g.w, m.w, v.w, sgm.lr, o.beta1, o.beta2, o.eps, bc1, bc2);
        reinterpret_cast<float4 *>(sgm.p)[c4] = p;
        reinterpret_cast<float4 *>(sgm.m)[c4] = m;
        reinterpret_cast<float4 *>(sgm.v)[c4] = v;
    } else {
        for (int64_t k = off; k < sgm.n; ++k)
            adam1(sgm.p[k], sgm.g[k], sgm.m[k], sgm.v[k], sgm.lr, o.beta1, o.beta2, o.eps, bc1, bc2);
    }
}

// one Gaussian's three log-scales (in registers) with the L_reg gradient; returns its L_reg term
__device__ __forceinline__ float adam_log_scale3(float *p, const float *g, float *m, float *v, float rw,
                                                 const FlatSeg &sgm, const gsr_adam_opts &o, float bc1, float bc2)
{
    return adam_log_scales3(p, g, m, v, rw, sgm.lr, o, bc1, bc2);
}

// log-scales of Gaussians [i0, i0 + cnt) with the L_reg gradient; returns their L_reg terms.
// A full group of 4 Gaussians is 12 floats = 3 float4 per array, all loaded before any update.
__device__ __forceinline__ float adam_log_scales(const FlatSeg &sgm, int64_t i0, int cnt, float rw,
                                                 const gsr_adam_opts &o, float bc1, float bc2)
{
    float lsum = 0.f;
    if (cnt == 4) {
        const int64_t c4 = 3 * i0 / 4;  // i0 is a multiple of 4
        float P[12], G[12], M[12], Vv[12];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            *reinterpret_cast<float4 *>(P + 4 * k) = reinterpret_cast<const float4 *>(sgm.p)[c4 + k];
            *reinterpret_cast<float4 *>(G + 4 * k) = reinterpret_cast<const float4 *>(sgm.g)[c4 + k];
            *reinterpret_cast<float4 *>(M + 4 * k) = reinterpret_cast<const float4 *>(sgm.m)[c4 + k];
            *reinterpret_cast<float4 *>(Vv + 4 * k) = reinterpret_cast<const float4 *>(sgm.v)[c4 + k];
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
            lsum += adam_log_scale3(P + 3 * q, G + 3 * q, M + 3 * q, Vv + 3 * q, rw, sgm, o, bc1, bc2);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            reinterpret_cast<float4 *>(sgm.p)[c4 + k] = *reinterpret_cast<const float4 *>(P + 4 * k);
            reinterpret_cast<float4 *>(sgm.m)[c4 + k] = *reinterpret_cast<const float4 *>(M + 4 * k);
            reinterpret_cast<float4 *>(sgm.v)[c4 + k] = *reinterpret_cast<const float4 *>(Vv + 4 * k);
        }
        return lsum;
    }
    for (int q = 0; q < cnt; ++q) {
        const int64_t b = 3 * (i0 + q);
        float P[3], G[3], M[3], Vv[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            P[k] = sgm.p[b + k];
            G[k] = sgm.g[b + k];
            M[k] = sgm.m[b + k];
            Vv[k] = sgm.v[b + k];
        }
        lsum += adam_log_scale3(P, G, M, Vv, rw, sgm, o, bc1, bc2);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            sgm.p[b + k] = P[k];
            sgm.m[b + k] = M[k];
            sgm.v[b + k] = Vv[k];
        }
    }
    return lsum;
}

// Log-scales with the L_reg gradient: one group of 4 Gaussians per thread
// (3 float4 per array, all loads issued before any update); per-block L_reg
// partial sums in part[blockIdx.x].  A kernel of its own: its 48 live values
// per thread would halve the occupancy of the flat kernel below.
__global__ void __launch_bounds__(256) k_adam_log_scale(gsr_gaussians_mut g, gsr_gaussian_grads gr,
                                                        gsr_adam_state st, gsr_adam_opts o,
                                                        const float *__restrict__ bc, float *__restrict__ part,
                                                        int64_t nls)
{
    const int64_t t = (int64_t)blockIdx.x * 256 + threadIdx.x;
    float lreg = 0.f;
    if (t < nls) {
        const FlatSeg sg{g.log_scale, st.m_log_scale, st.v_log_scale, gr.log_scale, o.lr_log_scale, 3 * g.n};
        const int64_t i0 = 4 * t;
        const int cnt = (int)min((int64_t)4, g.n - i0);
        lreg = adam_log_scales(sg, i0, cnt, o.w_reg / (float)g.n, o, bc[0], bc[1]);
    }
    if (part) {
        __shared__ float red[8];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) lreg += __shfl_down_sync(0xffffffffu, lreg, off);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = lreg;
        __syncthreads();
        if (threadIdx.x == 0) {
            float tt = 0.f;
            for (int k = 0; k < 8; ++k) tt += red[k];
            part[blockIdx.x] = tt;
        }
    }
}

// the other four arrays: float4 chunks of mean, quaternion, opacity, colour, in order
__global__ void __launch_bounds__(256) k_adam(gsr_gaussians_mut g, gsr_gaussian_grads gr, gsr_adam_state st,
                                              gsr_adam_opts o, const float *__restrict__ bc, int64_t c_mean,
                                              int64_t c_quat, int64_t c_op, int64_t c_rgb)
{
    int64_t c = (int64_t)blockIdx.x * 256 + threadIdx.x;
    const float bc1 = bc[0], bc2 = bc[1];
    if (c < c_mean) {
        adam_chunk(FlatSeg{g.mean, st.m_mean, st.v_mean, gr.mean, o.lr_mean, 3 * g.n}, c, o, bc1, bc2);
    } else if ((c -= c_mean) < c_quat) {
        adam_chunk(FlatSeg{g.quat, st.m_quat, st.v_quat, gr.quat, o.lr_quat, 4 * g.n}, c, o, bc1, bc2);
    } else if ((c -= c_quat) < c_op) {
        adam_chunk(FlatSeg{g.opacity_logit, st.m_opacity_logit, st.v_opacity_logit, gr.opacity_logit, o.lr_opacity,
                            g.n},
                   c, o, bc1, bc2);
    } else if ((c -= c_op) < c_rgb) {
        adam_chunk(FlatSeg{g.rgb, st.m_rgb, st.v_rgb, gr.rgb, o.lr_rgb, 3 * g.n}, c, o, bc1, bc2);
    }
}

// scalar fallback for unaligned arrays: one Gaussian per thread
__global__ void __launch_bounds__(256) k_adam_scalar(gsr_gaussians_mut g, gsr_gaussian_grads gr, gsr_adam_state st,
                                                     gsr_adam_opts o, const float *__restrict__ bc,
                                                     float *__restrict__ part)
{
    const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
    const float bc1 = bc[0], bc2 = bc[1];
    float lreg = 0.f;
    if (i < g.n) {
        lreg = adam_log_scales(FlatSeg{g.log_scale, st.m_log_scale, st.v_log_scale, gr.log_scale, o.lr_log_scale,
                                       3 * g.n},
                               i, 1, o.w_reg / (float)g.n, o, bc1, bc2);
        for (int k = 0; k < 3; ++k) {
            adam1(g.mean[3 * i + k], gr.mean[3 * i + k], st.m_mean[3 * i + k], st.v_mean[3 * i + k], o.lr_mean,
                  o.beta1, o.beta2, o.eps, bc1, bc2);
            adam1(g.rgb[3 * i + k], gr.rgb[3 * i + k], st.m_rgb[3 * i + k], st.v_rgb[3 * i + k], o.lr_rgb, o.beta1,
                  o.beta2, o.eps, bc1, bc2);
        }
        for (int k = 0; k < 4; ++k)
            adam1(g.quat[4 * i + k], gr.quat[4 * i + k], st.m_quat[4 * i + k], st.v_quat[4 * i + k], o.lr_quat,
                  o.beta1, o.beta2, o.eps, bc1, bc2);
        adam1(g.opacity_logit[i], gr.opacity_logit[i], st.m_opacity_logit[i], st.v_opacity_logit[i], o.lr_opacity,
              o.beta1, o.beta2, o.eps, bc1, bc2);
    }
    if (part) {
        __shared__ float red[8];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) lreg += __shfl_down_sync(0xffffffffu, lreg, off);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = lreg;
        __syncthreads();
        if (threadIdx.x == 0) {
            float tt = 0.f;
            for (int k = 0; k < 8; ++k) tt += red[k];
            part[blockIdx.x] = tt;
        }
    }
}

__global__ void k_lreg_final(const float *__restrict__ part, int nb, float scale, float *out, int32_t *step)
{
    __shared__ float red[32];
    float v = 0.f;
    for (int b = threadIdx.x; b < nb; b += 1024) v += part[b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int k = 0; k < 32; ++k) t += red[k];
        if (out) *out += scale * t;
        if (step) *step += 1;
    }
}

// Adam on the 6-vector twist, then T <- exp(delta^) T (q, t stored on device)
__global__ void k_pose_adam(float *pose, const float *__restrict__ g6, float *m6, float *v6, int32_t *step,
                            float lr_rho, float lr_phi, float b1, float b2, float eps)
{
    const int t = *step + 1;
    *step = t;
    const float bc1 = 1.f - powf(b1, (float)t), bc2 = 1.f - powf(b2, (float)t);
    float d[6];
    for (int k = 0; k < 6; ++k) {
        float g = g6[k];
        m6[k] = b1 * m6[k] + (1.f - b1) * g;
        v6[k] = b2 * v6[k] + (1.f - b2) * g * g;
        float lr = k < 3 ? lr_rho : lr_phi;
        d[k] = -lr * (m6[k] / bc1) / (sqrtf(v6[k] / bc2) + eps);
    }
    // SE(3) exponential: rotation quaternion of phi, V = I + B [phi]x + C [phi]x^2
    const float wx = d[3], wy = d[4], wz = d[5];
    const float th2 = wx * wx + wy * wy + wz * wz, th = sqrtf(th2);
    float B, C, qs, qv;
    if (th < 1e-4f) {
        B = 0.5f - th2 / 24.f;
        C = 1.f / 6.f - th2 / 120.f;
        qs = 1.f - th2 / 8.f;
        qv = 0.5f - th2 / 48.f;
    } else {
        B = (1.f - cosf(th)) / th2;
        C = (th - sinf(th)) / (th2 * th);
        qs = cosf(0.5f * th);
        qv = sinf(0.5f * th) / th;
    }
    const float dq[4] = {qs, qv * wx, qv * wy, qv * wz};
    float Rd[9];
    quat_rot(dq[0], dq[1], dq[2], dq[3], Rd);
    const float K[9] = {0.f, -wz, wy, wz, 0.f, -wx, -wy, wx, 0.f};
    float K2[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) K2[3 * r + c] = K[3 * r] * K[c] + K[3 * r + 1] * K[3 + c] + K[3 * r + 2] * K[6 + c];
    float tn[3];
    for (int r = 0; r < 3; ++r) {
        float vr = 0.f;
        for (int c = 0; c < 3; ++c) {
            float Vrc = (r == c ? 1.f : 0.f) + B * K[3 * r + c] + C * K2[3 * r + c];
            vr += Vrc * d[c];
        }
        tn[r] = Rd[3 * r] * pose[4] + Rd[3 * r + 1] * pose[5] + Rd[3 * r + 2] * pose[6] + vr;
    }
    // q <- dq * q (Hamilton product), renormalised
    const float aw = dq[0], ax = dq[1], ay = dq[2], az = dq[3];
    const float bw = pose[0], bx = pose[1], by = pose[2], bz = pose[3];
    float q[4] = {aw * bw - ax * bx - ay * by - az * bz, aw * bx + ax * bw + ay * bz - az * by,
                  aw * by - ax * bz + ay * bw + az * bx, aw * bz + ax * by - ay * bx + az * bw};
    float inv = 1.f / sqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    if (q[0] < 0.f) inv = -inv;
    for (int k = 0; k < 4; ++k) pose[k] = q[k] * inv;
    for (int k = 0; k < 3; ++k) pose[4 + k] = tn[k];
    pose_rotation_split(pose);
}

} // namespace

gsr_status run_adam(gsr_ctx *ctx, gsr_gaussians_mut *g, const gsr_gaussian_grads *gr, gsr_adam_state *st,
                    const gsr_adam_opts *o, float *loss_reg_dev, cudaStream_t s)
{
    // 16-byte vectors need 16-byte aligned bases for every array
    bool vec4 = true;
    const void *ptrs[] = {g->mean, g->log_scale, g->quat, g->opacity_logit, g->rgb, gr->mean, gr->log_scale,
                          gr->quat, gr->opacity_logit, gr->rgb, st->m_mean, st->m_log_scale, st->m_quat,
                          st->m_opacity_logit, st->m_rgb, st->v_mean, st->v_log_scale, st->v_quat,
                          st->v_opacity_logit, st->v_rgb};
    for (const void *q : ptrs) vec4 = vec4 && ((uintptr_t)q % 16 == 0);
    const int64_t n = g->n > 0 ? g->n : 1;
    const int64_t nls = ceil_div(n, 4), c_mean = ceil_div(3 * n, 4), c_quat = n, c_op = ceil_div(n, 4),
                  c_rgb = ceil_div(3 * n, 4);
    // the scalar path: one Gaussian per thread, all arrays; the vector path: log-scale
    // groups (nb blocks, which also write the L_reg partial sums) and flat chunks
    const unsigned nb = (unsigned)ceil_div(vec4 ? nls : n, 256);
    const unsigned nb_flat = (unsigned)ceil_div(c_mean + c_quat + c_op + c_rgb, 256);
    GSR_TRY(ensure_buf(ctx, ctx->small, 256 * sizeof(float)));
    float *bc = (float *)ctx->small.p;  // [0..1] bias corrections
    float *part = nullptr;
    if (loss_reg_dev) {
        GSR_TRY(ensure_buf(ctx, ctx->pose_part, sizeof(float) * 6 * nb));
        part = (float *)ctx->pose_part.p;
    }
    k_adam_prep<<<1, 1, 0, s>>>(st->step, o->beta1, o->beta2, bc);
    if (vec4) {
        k_adam_log_scale<<<nb, 256, 0, s>>>(*g, *gr, *st, *o, bc, part, nls);
        k_adam<<<nb_flat, 256, 0, s>>>(*g, *gr, *st, *o, bc, c_mean, c_quat, c_op, c_rgb);
        ctx->launches += 3;
    } else {
        k_adam_scalar<<<nb, 256, 0, s>>>(*g, *gr, *st, *o, bc, part);
        ctx->launches += 2;
    }
    if (loss_reg_dev) {
        k_lreg_final<<<1, 1024, 0, s>>>(part, (int)nb, o->w_reg / (float)(g->n > 0 ? g->n : 1), loss_reg_dev,
                                        nullptr);
        ctx->launches += 1;
    }
    GSR_LAUNCHED(ctx);
    return GSR_OK;
}

gsr_status adam_prep(gsr_ctx *ctx, gsr_adam_state *st, const gsr_adam_opts *o, float **bc, cudaStream_t s)
{
    GSR_TRY(ensure_buf(ctx, ctx->small, 256 * sizeof(float)));
    *bc = (float *)ctx->small.p;  // [0..1] bias corrections
    k_adam_prep<<<1, 1, 0, s>>>(st->step, o->beta1, o->beta2, *bc);
    ctx->launches += 1;
    GSR_LAUNCHED(ctx);
    return GSR_OK;
}

gsr_status adam_lreg_final(gsr_ctx *ctx, const float *part, int nb, float scale, float *loss_reg_dev, cudaStream_t s)
{
    k_lreg_final<<<1, 1024, 0, s>>>(part, nb, scale, loss_reg_dev, nullptr);
    ctx->launches += 1;
    GSR_LAUNCHED(ctx);
    return GSR_OK;
}

gsr_status adam_lreg_final_step(gsr_ctx *ctx, const float *part, int nb, float scale, float *loss_reg_dev,
                                int32_t *step, cudaStream_t s)
{
    k_lreg_final<<<1, 1024, 0, s>>>(part, nb, scale, loss_reg_dev, step);
    ctx->launches += 1;
    GSR_LAUNCHED(ctx);
    return GSR_OK;
}

gsr_status run_pose_adam(gsr_ctx *ctx, float *d_pose, const float *d_grad6, float *m6, float *v6, int32_t *step,
                         float lr_rho, float lr_phi, float b1, float b2, float eps, cudaStream_t s)
{
    k_pose_adam<<<1, 1, 0, s>>>(d_pose, d_grad6, m6, v6, step, lr_rho, lr_phi, b1, b2, eps);
    ctx->launches += 1;
    GSR_LAUNCHED(ctx);
    return GSR_OK;
}
