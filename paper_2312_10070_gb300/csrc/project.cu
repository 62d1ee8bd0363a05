// project.cu -- per-Gaussian projection (Sec. 3.1), tile binning glue and
// the projection backward with the 6-DoF pose adjoint.
//
// Numerics: the 2D covariance is formed as Sigma' = T T^T + eps I with
// T = J W M (M = R diag(s), W = R_wc), so a and c are sums of squares and
// det(Sigma') = |T_0 x T_1|^2 + eps (|T_0|^2 + |T_1|^2) + eps^2 (Lagrange's
// identity) is a sum of positive terms: no cancellation for thin Gaussians.
#include "gsr_internal.cuh"

CamK make_camk(const gsr_camera &c, int tw, int th)
{
    CamK k;
    k.W = c.width;
    k.H = c.height;
    k.tw = tw;
    k.th = th;
    k.inv_tw = 1.f / (float)tw;
    k.tiles_x = (c.width + tw - 1) / tw;
    k.tiles_y = (c.height + th - 1) / th;
    k.fx = c.fx;
    k.fy = c.fy;
    k.cx = c.cx;
    k.cy = c.cy;
    k.z_near = c.z_near;
    k.eps2d = c.eps2d;
    k.limx = GSR_GUARD * 0.5f * (float)c.width / c.fx;
    k.limy = GSR_GUARD * 0.5f * (float)c.height / c.fy;
    return k;
}

namespace {

// Device pose record (float[GSR_POSE_WORDS]): q (4), t (3), pad, then the
// rotation R(q / |q|) formed in double precision and split into float
// hi + lo parts (9 + 9).  The camera transform p = R mu + t is evaluated as
// a compensated dot product on the FP32 pipe, so p is faithfully rounded:
// the depth keys equal the float rounding of the exact depth except within
// one ulp, and u, v carry no cancellation error from large world coordinates.
struct PoseR {
    float R[9], Rlo[9], t[3];
};

__device__ __forceinline__ PoseR load_pose(const float *__restrict__ pose)
{
    PoseR P;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        P.R[k] = pose[8 + k];
        P.Rlo[k] = pose[17 + k];
    }
    P.t[0] = pose[4];
    P.t[1] = pose[5];
    P.t[2] = pose[6];
    return P;
}

// error-free transformations (Knuth two-sum, FMA two-product)
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// (R_hi + R_lo) . x + t, compensated (Ogita-Rump-Oishi Dot2 with the lo parts)
__device__ __forceinline__ float dot3_comp(const float *Rh, const float *Rl, float x0, float x1, float x2, float t)
{
    float p = __fmul_rn(Rh[0], x0);
    float s = __fmaf_rn(Rh[0], x0, -p);
    float h, r, q;
    h = __fmul_rn(Rh[1], x1);
    r = __fmaf_rn(Rh[1], x1, -h);
    two_sum(p, h, p, q);
    s = __fadd_rn(s, __fadd_rn(q, r));
    h = __fmul_rn(Rh[2], x2);
    r = __fmaf_rn(Rh[2], x2, -h);
    two_sum(p, h, p, q);
    s = __fadd_rn(s, __fadd_rn(q, r));
    two_sum(p, t, p, q);
    s = __fadd_rn(s, q);
    s = __fmaf_rn(Rl[0], x0, s);
    s = __fmaf_rn(Rl[1], x1, s);
    s = __fmaf_rn(Rl[2], x2, s);
    return __fadd_rn(p, s);
}

// Full forward state of one Gaussian, recomputed by the backward.
struct GProj {
    float p[3];       // camera-space mean
    float R[9];       // Gaussian rotation (normalised quaternion)
    float qh[4], qn;  // normalised quaternion and |q|
    float s[3];       // scales
    float A[9];       // W M
    float J[6];
    float T[6];       // J W M (2x3)
    float tx, ty;
    bool clx, cly;
    float a, b, c;    // Sigma' entries (with eps)
    float det;
    float op;
};

// returns false when culled by depth
__device__ __forceinline__ bool project_core(const CamK &ck, const PoseR &P, const float *__restrict__ mean,
                                             const float *__restrict__ ls, const float *__restrict__ quat,
                                             float logit, int64_t i, GProj &g)
{
    float mx = mean[3 * i], my = mean[3 * i + 1], mz = mean[3 * i + 2];
    g.p[0] = dot3_comp(P.R, P.Rlo, mx, my, mz, P.t[0]);
    g.p[1] = dot3_comp(P.R + 3, P.Rlo + 3, mx, my, mz, P.t[1]);
    g.p[2] = dot3_comp(P.R + 6, P.Rlo + 6, mx, my, mz, P.t[2]);
    g.op = 1.f / (1.f + expf(-logit));
    if (!(g.p[2] > ck.z_near)) return false;
    float qw = quat[4 * i], qx = quat[4 * i + 1], qy = quat[4 * i + 2], qz = quat[4 * i + 3];
    g.qn = sqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
    float inv = 1.f / g.qn;
    g.qh[0] = qw * inv;
    g.qh[1] = qx * inv;
    g.qh[2] = qy * inv;
    g.qh[3] = qz * inv;
    quat_rot(g.qh[0], g.qh[1], g.qh[2], g.qh[3], g.R);
#pragma unroll
    for (int k = 0; k < 3; ++k) g.s[k] = expf(ls[3 * i + k]);
    // A = W R diag(s)
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k)
            g.A[3 * r + k] = (P.R[3 * r] * g.R[k] + P.R[3 * r + 1] * g.R[3 + k] + P.R[3 * r + 2] * g.R[6 + k]) * g.s[k];
    float iz = 1.f / g.p[2];
    float tx = g.p[0] * iz, ty = g.p[1] * iz;
    g.clx = fabsf(tx) > ck.limx;
    g.cly = fabsf(ty) > ck.limy;
    g.tx = fminf(fmaxf(tx, -ck.limx), ck.limx);
    g.ty = fminf(fmaxf(ty, -ck.limy), ck.limy);
    g.J[0] = ck.fx * iz;
    g.J[1] = 0.f;
    g.J[2] = -ck.fx * g.tx * iz;
    g.J[3] = 0.f;
    g.J[4] = ck.fy * iz;
    g.J[5] = -ck.fy * g.ty * iz;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        g.T[k] = fmaf(g.J[0], g.A[k], g.J[2] * g.A[6 + k]);
        g.T[3 + k] = fmaf(g.J[4], g.A[3 + k], g.J[5] * g.A[6 + k]);
    }
    float a0 = g.T[0] * g.T[0] + g.T[1] * g.T[1] + g.T[2] * g.T[2];
    float c0 = g.T[3] * g.T[3] + g.T[4] * g.T[4] + g.T[5] * g.T[5];
    g.a = a0 + ck.eps2d;
    g.c = c0 + ck.eps2d;
    g.b = g.T[0] * g.T[3] + g.T[1] * g.T[4] + g.T[2] * g.T[5];
    float x0 = g.T[1] * g.T[5] - g.T[2] * g.T[4];
    float x1 = g.T[2] * g.T[3] - g.T[0] * g.T[5];
    float x2 = g.T[0] * g.T[4] - g.T[1] * g.T[3];
    g.det = (x0 * x0 + x1 * x1 + x2 * x2) + ck.eps2d * (a0 + c0) + ck.eps2d * ck.eps2d;
    return true;
}

__global__ void k_set_pose(float *d, gsr_pose p)
{
    d[0] = p.q[0];
    d[1] = p.q[1];
    d[2] = p.q[2];
    d[3] = p.q[3];
    d[4] = p.t[0];
    d[5] = p.t[1];
    d[6] = p.t[2];
    d[7] = 0.f;
    pose_rotation_split(d);
}

// ------------------------------------------ twist perturbation (Sec. 3.5)
// The tracker optimises a left perturbation T(xi) = exp(xi^) T of the pose,
// xi = (rho, phi).  exp(xi^) = [[R(phi), V(phi) rho], [0, 1]] with K = [phi]x,
// th = |phi|, R = I + A K + B K^2, V = I + B K + C K^2, A = sin th / th,
// B = (1 - cos th) / th^2, C = (th - sin th) / th^3 (series below 1e-3).
__device__ __forceinline__ void so3_coeffs_d(double th, double &A, double &B, double &C)
{
    const double t2 = th * th;
    if (th < 1e-3) {
        A = 1.0 - t2 / 6.0 + t2 * t2 / 120.0;
        B = 0.5 - t2 / 24.0 + t2 * t2 / 720.0;
        C = 1.0 / 6.0 - t2 / 120.0 + t2 * t2 / 5040.0;
    } else {
        A = sin(th) / th;
        B = (1.0 - cos(th)) / t2;
        C = (th - sin(th)) / (t2 * th);
    }
}

__device__ __forceinline__ void skew_d(const double *w, double K[9])
{
    K[0] = 0.0;   K[1] = -w[2]; K[2] = w[1];
    K[3] = w[2];  K[4] = 0.0;   K[5] = -w[0];
    K[6] = -w[1]; K[7] = w[0];  K[8] = 0.0;
}

__device__ __forceinline__ void mat3_mul_d(const double *A, const double *B, double *C)
{
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) C[3 * r + c] = A[3 * r] * B[c] + A[3 * r + 1] * B[3 + c] + A[3 * r + 2] * B[6 + c];
}

// Replaces the (q, t) of a pose record by exp(xi^) (q, t), in double
// precision, then rounds q', t' to float and re-forms the split rotation, so
// the record is that of the float pose fl(exp(xi^) T) like any other pose.
__device__ void perturb_record(float *d, const float *__restrict__ xi)
{
    double x[6];
    for (int k = 0; k < 6; ++k) x[k] = (double)xi[k];
    const double th = sqrt(x[3] * x[3] + x[4] * x[4] + x[5] * x[5]);
    double A, B, C;
    so3_coeffs_d(th, A, B, C);
    double K[9], K2[9];
    skew_d(x + 3, K);
    mat3_mul_d(K, K, K2);
    double Rd[9], V[9];
    for (int i = 0; i < 9; ++i) {
        const double I = (i % 4 == 0) ? 1.0 : 0.0;
        Rd[i] = I + A * K[i] + B * K2[i];
        V[i] = I + B * K[i] + C * K2[i];
    }
    // unit quaternion of the rotation by phi: (cos th/2, sin(th/2)/th phi)
    const double hs = th < 1e-3 ? 0.5 - th * th / 48.0 : sin(0.5 * th) / th;
    const double aw = cos(0.5 * th), ax = hs * x[3], ay = hs * x[4], az = hs * x[5];
    double bw = d[0], bx = d[1], by = d[2], bz = d[3];
    const double bn = sqrt(bw * bw + bx * bx + by * by + bz * bz);
    bw /= bn;
    bx /= bn;
    by /= bn;
    bz /= bn;
    double q[4] = {aw * bw - ax * bx - ay * by - az * bz, aw * bx + ax * bw + ay * bz - az * by,
                   aw * by - ax * bz + ay * bw + az * bx, aw * bz + ax * by - ay * bx + az * bw};
    double qn = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    if (q[0] < 0.0) qn = -qn;
    const double t[3] = {d[4], d[5], d[6]};
    for (int r = 0; r < 3; ++r) {
        const double tr = Rd[3 * r] * t[0] + Rd[3 * r + 1] * t[1] + Rd[3 * r + 2] * t[2] + V[3 * r] * x[0] +
                          V[3 * r + 1] * x[1] + V[3 * r + 2] * x[2];
        d[4 + r] = (float)tr;
    }
    for (int k = 0; k < 4; ++k) d[k] = (float)(q[k] / qn);
    pose_rotation_split(d);
}

__global__ void k_perturb_pose(float *d, const float *__restrict__ xi) { perturb_record(d, xi); }

// (q', t') = fl(exp(xi^) (q, t)) written to out[0..7) (q' with w >= 0)
__global__ void k_pose_retract(gsr_pose p, const float *__restrict__ xi, float *__restrict__ out)
{
    float d[GSR_POSE_WORDS];
    for (int k = 0; k < 4; ++k) d[k] = p.q[k];
    for (int k = 0; k < 3; ++k) d[4 + k] = p.t[k];
    perturb_record(d, xi);
    for (int k = 0; k < 7; ++k) out[k] = d[k];
}

// g6 <- J_l(xi)^T g6: the pose gradient at exp(xi^) T taken with respect to
// xi itself.  exp((xi + e)^) = exp((J_l(xi) e)^) exp(xi^) + O(e^2), with the
// SE(3) left Jacobian J_l = [[V, Q], [0, V]] (rho first) and
//   Q = 1/2 P + c1 (K P + P K + K P K) + c2 (K K P + P K K - 3 K P K)
//       + c3 (K P K K + K K P K),   P = [rho]x,
//   c1 = (th - sin th) / th^3, c2 = (th^2 + 2 cos th - 2) / (2 th^4),
//   c3 = (2 th - 3 sin th + th cos th) / (2 th^5)  (series below 1e-2).
__global__ void k_pose_grad_xi(float *g6, const float *__restrict__ xi)
{
    double x[6], g[6];
    for (int k = 0; k < 6; ++k) {
        x[k] = (double)xi[k];
        g[k] = (double)g6[k];
    }
    const double th = sqrt(x[3] * x[3] + x[4] * x[4] + x[5] * x[5]), t2 = th * th;
    double A, B, C;
    so3_coeffs_d(th, A, B, C);
    double c1, c2, c3;
    if (th < 1e-2) {
        c1 = 1.0 / 6.0 - t2 / 120.0 + t2 * t2 / 5040.0;
        c2 = 1.0 / 24.0 - t2 / 720.0 + t2 * t2 / 40320.0;
        c3 = 1.0 / 120.0 - t2 / 2520.0 + t2 * t2 / 120960.0;
    } else {
        c1 = (th - sin(th)) / (t2 * th);
        c2 = (t2 + 2.0 * cos(th) - 2.0) / (2.0 * t2 * t2);
        c3 = (2.0 * th - 3.0 * sin(th) + th * cos(th)) / (2.0 * t2 * t2 * th);
    }
    double K[9], P[9], KK[9], KP[9], PK[9], KPK[9], KKP[9], PKK[9], KPKK[9], KKPK[9], V[9], Q[9];
    skew_d(x + 3, K);
    skew_d(x, P);
    mat3_mul_d(K, K, KK);
    mat3_mul_d(K, P, KP);
    mat3_mul_d(P, K, PK);
    mat3_mul_d(KP, K, KPK);
    mat3_mul_d(KK, P, KKP);
    mat3_mul_d(P, KK, PKK);
    mat3_mul_d(KPK, K, KPKK);
    mat3_mul_d(K, KPK, KKPK);
    for (int i = 0; i < 9; ++i) {
        const double I = (i % 4 == 0) ? 1.0 : 0.0;
        V[i] = I + B * K[i] + C * KK[i];
        Q[i] = 0.5 * P[i] + c1 * (KP[i] + PK[i] + KPK[i]) + c2 * (KKP[i] + PKK[i] - 3.0 * KPK[i]) +
               c3 * (KPKK[i] + KKPK[i]);
    }
    // [g_rho'; g_phi'] = [[V^T, 0], [Q^T, V^T]] [g_rho; g_phi]
    for (int c = 0; c < 3; ++c) {
        double r = 0.0, p = 0.0;
        for (int k = 0; k < 3; ++k) {
            r += V[3 * k + c] * g[k];
            p += Q[3 * k + c] * g[k] + V[3 * k + c] * g[3 + k];
        }
        g6[c] = (float)r;
        g6[3 + c] = (float)p;
    }
}

// K1: projection, culling, radius, tile rectangle.  rec[gid] holds
// (u, v, conic a, conic b) (conic c, opacity, depth, rect lo) (r, g, b, rect hi).
__global__ void __launch_bounds__(256) k_project(Params P, CamK ck, const float *__restrict__ pose,
                                                 float4 *__restrict__ rec, u32 *__restrict__ flag,
                                                 int32_t *__restrict__ rank_of_gid)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n) return;
    PoseR pr = load_pose(pose);
    GProj g;
    u32 vis = 0;
    rank_of_gid[i] = -1;
    if (project_core(ck, pr, P.mean, P.log_scale, P.quat, P.opacity_logit[i], i, g) && g.det > 0.f) {
        float idet = 1.f / g.det;
        float hm = 0.5f * (g.a + g.c), hd = 0.5f * (g.a - g.c);
        float lmax = hm + sqrtf(hd * hd + g.b * g.b);
        float r = ceilf(3.f * sqrtf(lmax));
        float iz = 1.f / g.p[2];
        float u = fmaf(ck.fx, g.p[0] * iz, ck.cx);
        float v = fmaf(ck.fy, g.p[1] * iz, ck.cy);
        if (!(u + r < 0.f || u - r >= (float)ck.W || v + r < 0.f || v - r >= (float)ck.H)) {
            int x0 = max(0, (int)floorf((u - r) / (float)ck.tw));
            int x1 = min(ck.tiles_x - 1, (int)floorf((u + r) / (float)ck.tw));
            int y0 = max(0, (int)floorf((v - r) / (float)ck.th));
            int y1 = min(ck.tiles_y - 1, (int)floorf((v + r) / (float)ck.th));
            vis = 1;
            rec[3 * i] = make_float4(u, v, g.c * idet, -g.b * idet);
            rec[3 * i + 1] = make_float4(g.a * idet, g.op, g.p[2], __uint_as_float((u32)x0 | ((u32)y0 << 16)));
            rec[3 * i + 2] = make_float4(P.rgb[3 * i], P.rgb[3 * i + 1], P.rgb[3 * i + 2],
                                         __uint_as_float((u32)x1 | ((u32)y1 << 16)));
        }
    }
    flag[i] = vis;
}

// stable compaction of visible Gaussians: depth key + id
__global__ void k_compact(int64_t n, const u32 *__restrict__ flag, const u32 *__restrict__ off,
                          const float4 *__restrict__ rec, u32 *__restrict__ keys, u32 *__restrict__ vals)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !flag[i]) return;
    u32 o = off[i];
    keys[o] = __float_as_uint(rec[3 * i + 1].z);  // positive depth: bit order = value order
    vals[o] = (u32)i;
}

// Tile culling by rows.  A tile of the rectangle is kept when its Gaussian may
// composite at one of its pixel centres: when the minimum of sigma over the
// tile's pixel-centre box is at most the skip threshold T (ln(255 o) + 0.02,
// widened by the float32 error margin of tile_may_hit: T (1 + e) / (1 - e),
// e = 1e-6 kappa).  sigma is convex, so within one tile row (the band
// dy in [Y0, Y1]) the x offsets where min over the band of sigma <= T form one
// interval [L, R]: the x-extent of the ellipse sigma <= T cut by the band.
// The ellipse's extreme points are at dy = -/+ (b / c) x_max, x_max =
// sqrt(2 c T / det), and its boundary at dy is dx = (-b dy +/- sqrt(2 a T -
// det dy^2)) / a, so R (L) is that boundary at the extreme point's dy clamped
// to the band (cut to the ellipse's dy-extent sqrt(2 a T / det)).  The kept
// tiles of the row are one run of columns; [L, R] is widened by 2e-4 px plus
// a relative 2e-6 so that float32 rounding never drops a tile the exact test
// keeps.  The box test of tile_may_hit decides the same tiles up to that
// widening.
struct RowCull {
    float u = 0.f, v = 0.f, a = 1.f, b = 0.f, det = 1.f, ia = 1.f, t2a = 0.f, ymax = 0.f, kx = 0.f;
    int mode = 0;  // 0: by rows, 1: every tile of the rectangle, 2: none
};

// Both the counting and the emitting kernel evaluate these two functions; every
// operation is an explicitly rounded intrinsic, so no contraction can make the
// two kernels decide a tile differently (the emitter writes exactly the counted
// instances).
__device__ __forceinline__ RowCull row_cull_setup(const float4 &A, const float4 &B, float thr0, bool cull)
{
    RowCull q;
    q.mode = 1;
    if (!cull) return q;
    const float a = A.z, b = A.w, c = B.x;
    const float det = __fsub_rn(__fmul_rn(a, c), __fmul_rn(b, b));
    if (!(a > 0.f && c > 0.f && det > 0.f)) return q;
    const float hd = __fmul_rn(0.5f, __fsub_rn(a, c));
    const float lmax = __fadd_rn(__fmul_rn(0.5f, __fadd_rn(a, c)),
                                 __fsqrt_rn(__fadd_rn(__fmul_rn(hd, hd), __fmul_rn(b, b))));
    const float e = __fmul_rn(1e-6f, __fdiv_rn(__fmul_rn(lmax, lmax), det));
    if (!(e < 0.25f)) return q;
    float T = __fmul_rn(thr0, __fdiv_rn(__fadd_rn(1.f, e), __fsub_rn(1.f, e)));
    T = __fadd_rn(T, __fmul_rn(1e-6f, fabsf(T)));
    if (!(T >= 0.f)) {
        q.mode = 2;
        return q;
    }
    q.mode = 0;
    q.u = A.x;
    q.v = A.y;
    q.a = a;
    q.b = b;
    q.det = det;
    q.ia = __frcp_rn(a);
    q.t2a = __fmul_rn(__fmul_rn(2.f, a), T);
    q.ymax = __fsqrt_rn(__fdiv_rn(q.t2a, det));
    q.kx = __fmul_rn(__fdiv_rn(b, c), __fsqrt_rn(__fdiv_rn(__fmul_rn(__fmul_rn(2.f, c), T), det)));
    return q;
}

// kept tile columns [*lo, *hi] of tile row ty (within [rx0, rx1]; *lo > *hi: none)
__device__ __forceinline__ void row_cols(const RowCull &q, const CamK &ck, int ty, int rx0, int rx1, int *lo, int *hi)
{
    *lo = rx0;
    *hi = rx1;
    if (q.mode == 1) return;
    if (q.mode == 2) {
        *hi = rx0 - 1;
        return;
    }
    const float Y0 = __fsub_rn(__fadd_rn((float)(ty * ck.th), 0.5f), q.v);
    const float Y1 = __fsub_rn(__fsub_rn((float)min(ty * ck.th + ck.th, ck.H), 0.5f), q.v);
    float ylo = fmaxf(Y0, -q.ymax), yhi = fminf(Y1, q.ymax);
    if (ylo > __fadd_rn(yhi, 2e-4f)) {
        *hi = rx0 - 1;
        return;
    }
    yhi = fmaxf(yhi, ylo);
    const float dR = fminf(fmaxf(-q.kx, ylo), yhi), dL = fminf(fmaxf(q.kx, ylo), yhi);
    const float sR = __fsqrt_rn(fmaxf(0.f, __fsub_rn(q.t2a, __fmul_rn(q.det, __fmul_rn(dR, dR)))));
    const float sL = __fsqrt_rn(fmaxf(0.f, __fsub_rn(q.t2a, __fmul_rn(q.det, __fmul_rn(dL, dL)))));
    float R = __fmul_rn(__fadd_rn(__fmul_rn(-q.b, dR), sR), q.ia);
    float L = __fmul_rn(__fsub_rn(__fmul_rn(-q.b, dL), sL), q.ia);
    const float d = __fadd_rn(2e-4f, __fmul_rn(2e-6f, __fadd_rn(fabsf(L), fabsf(R))));
    L = __fsub_rn(L, d);
    R = __fadd_rn(R, d);
    // column tx's box spans x offsets [tx tw + 0.5 - u, tx tw + tw - 0.5 - u] (the
    // last column unclipped: conservative); clamp before converting to int
    // x / tw as x * (1 / tw): the same float, since tw is a power of two
    const float itw = ck.inv_tw;
    const float flo = fmaxf(ceilf(__fsub_rn(__fmul_rn(__fadd_rn(__fadd_rn(L, q.u), 0.5f), itw), 1.f)), (float)rx0);
    const float fhi = fminf(floorf(__fmul_rn(__fsub_rn(__fadd_rn(R, q.u), 0.5f), itw)), (float)rx1);
    *lo = (int)flo;
    *hi = fhi < flo ? *lo - 1 : (int)fhi;
}

// records in depth order; kept tile instances per rank
template <bool CULL>
__global__ void k_gather(int64_t cap, const u32 *__restrict__ d_v, const u32 *__restrict__ vals,
                         const float4 *__restrict__ rec, float4 *__restrict__ rec_sorted,
                         int32_t *__restrict__ rank_of_gid, CamK ck, u32 *__restrict__ tcount,
                         float4 *__restrict__ g2d)
{
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= cap || r >= (int64_t)*d_v) return;
    u32 gid = vals[r];
    float4 a = rec[3 * (int64_t)gid], b = rec[3 * (int64_t)gid + 1], c = rec[3 * (int64_t)gid + 2];
    rec_sorted[3 * r] = a;
    rec_sorted[3 * r + 1] = b;
    rec_sorted[3 * r + 2] = c;
    // the rank's image-space gradient accumulator starts at zero for the next backward
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    g2d[3 * r] = z;
    g2d[3 * r + 1] = z;
    g2d[3 * r + 2] = z;
    rank_of_gid[gid] = (int32_t)r;
    const u32 lo = __float_as_uint(b.w), hi = __float_as_uint(c.w);
    const int x0 = (int)(lo & 0xffffu), y0 = (int)(lo >> 16), x1 = (int)(hi & 0xffffu), y1 = (int)(hi >> 16);
    if (!CULL) {
        tcount[r] = (u32)((x1 - x0 + 1) * (y1 - y0 + 1));
        return;
    }
    const RowCull q = row_cull_setup(a, b, sigma_reject(b.y), true);
    u32 n = 0;
    for (int ty = y0; ty <= y1; ++ty) {
        int l, h;
        row_cols(q, ck, ty, x0, x1, &l, &h);
        n += (u32)max(0, h - l + 1);
    }
    tcount[r] = n;
}

// One instance (tile id, depth rank) per kept tile, written from off[rank]
// (the exclusive scan of the counts); the stream is in depth order, so a
// stable sort on the tile id yields depth-ordered lists.  The 32 ranks of a
// warp own one contiguous output range.  Each lane lists its rank's row runs
// (output offset, tile row, first column) in a per-warp table in shared
// memory, in output order; then the lanes write the warp's range position by
// position, each finding its run by binary search, so consecutive lanes store
// to consecutive addresses.  A warp whose rows exceed the table writes
// rank by rank from each lane instead.
constexpr int EMIT_RUNS = 512;  // row runs per warp

template <bool CULL>
__global__ void __launch_bounds__(256) k_emit(int64_t cap_v, const u32 *__restrict__ d_v,
                                              const float4 *__restrict__ rec_sorted, const u32 *__restrict__ tcount,
                                              const u32 *__restrict__ off, CamK ck, int64_t cap_i,
                                              u32 *__restrict__ tkeys, u32 *__restrict__ tvals,
                                              u32 *__restrict__ counters)
{
    __shared__ u32 s_start[8][EMIT_RUNS];  // run's first output offset, relative to the warp's range
    __shared__ u32 s_cell[8][EMIT_RUNS];   // (tile row << 16) | first column
    __shared__ uint8_t s_lane[8][EMIT_RUNS];
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r == 0) {
        u32 total = counters[CNT_INSTANCES];
        counters[CNT_SORTN] = (int64_t)total > cap_i ? (u32)cap_i : total;
        if ((int64_t)total > cap_i) atomicOr(&counters[CNT_STATUS], GSR_FLAG_CAPACITY);
    }
    const unsigned F = 0xffffffffu;
    const int lane = threadIdx.x & 31, w = (int)threadIdx.x >> 5;
    const int64_t V = (int64_t)*d_v, r0 = r - lane;
    if (r0 >= V || r0 >= cap_v) return;  // warp-uniform
    const bool valid = r < V && r < cap_v;
    int x0 = 0, y0 = 0, x1 = -1, y1 = -1;
    u32 cnt = 0, base = 0;
    RowCull q;
    if (valid) {
        const float4 a = rec_sorted[3 * r], b = rec_sorted[3 * r + 1];
        const u32 lo = __float_as_uint(b.w), hi = __float_as_uint(rec_sorted[3 * r + 2].w);
        x0 = (int)(lo & 0xffffu);
        y0 = (int)(lo >> 16);
        x1 = (int)(hi & 0xffffu);
        y1 = (int)(hi >> 16);
        q = row_cull_setup(a, b, sigma_reject(b.y), CULL);
        cnt = tcount[r];
        base = off[r];
    }
    const u32 wbase = __shfl_sync(F, base, 0);  // lane 0's rank is valid (r0 < V)
    const u32 wend = __reduce_max_sync(F, valid ? base + cnt : 0u);
    // table slots: one per row of each rank with instances (empty rows included)
    const u32 nrow = (valid && cnt > 0u) ? (u32)(y1 - y0 + 1) : 0u;
    u32 incl = nrow;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const u32 t = __shfl_up_sync(F, incl, o);
        if (lane >= o) incl += t;
    }
    const u32 nruns = __shfl_sync(F, incl, 31);
    if (nruns <= (u32)EMIT_RUNS) {
        u32 slot = incl - nrow, rel = base - wbase;
        for (u32 k = 0; k < nrow; ++k, ++slot) {
            const int ty = y0 + (int)k;
            int l, h;
            row_cols(q, ck, ty, x0, x1, &l, &h);
            s_start[w][slot] = rel;
            s_cell[w][slot] = ((u32)ty << 16) | (u32)l;
            s_lane[w][slot] = (uint8_t)lane;
            rel += (u32)max(0, h - l + 1);
        }
        __syncwarp();
        const u32 total = wend - wbase;
        for (u32 p = lane; p < total; p += 32) {
            // the last run starting at or before p (empty runs share the next run's start)
            int lo = 0, hi = (int)nruns - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (s_start[w][mid] <= p) lo = mid;
                else hi = mid - 1;
            }
            const u32 cell = s_cell[w][lo];
            const int64_t o = (int64_t)wbase + p;
            if (o < cap_i) {
                tkeys[o] = (cell >> 16) * (u32)ck.tiles_x + (cell & 0xffffu) + (p - s_start[w][lo]);
                tvals[o] = (u32)(r0 + s_lane[w][lo]);
            }
        }
        return;
    }
    // too many rows for the table: each lane writes its own rank
    if (valid && cnt > 0u) {
        const int64_t end = (int64_t)base + cnt;  // never past the counted instances
        int64_t o = base;
        for (int ty = y0; ty <= y1; ++ty) {
            int l, h;
            row_cols(q, ck, ty, x0, x1, &l, &h);
            for (int tx = l; tx <= h && o < end; ++tx, ++o)
                if (o < cap_i) {
                    tkeys[o] = (u32)(ty * ck.tiles_x + tx);
                    tvals[o] = (u32)r;
                }
        }
    }
}

// four sorted keys per thread: a tile's range starts where its key differs
// from the previous one and ends where it differs from the next one
__global__ void k_ranges(int64_t cap_i, const u32 *__restrict__ d_n, const u32 *__restrict__ tkeys,
                         uint2 *__restrict__ ranges)
{
    const int64_t i0 = 4 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
    const int64_t n = min((int64_t)*d_n, cap_i);
    if (i0 >= n) return;
    u32 k[6];
    k[0] = i0 > 0 ? tkeys[i0 - 1] : 0xffffffffu;
#pragma unroll
    for (int q = 1; q <= 5; ++q) k[q] = i0 + q - 1 < n ? tkeys[i0 + q - 1] : 0xffffffffu;
#pragma unroll
    for (int q = 1; q <= 4; ++q) {
        const int64_t i = i0 + q - 1;
        if (i >= n) break;
        if (k[q - 1] != k[q]) ranges[k[q]].x = (u32)i;
        if (k[q + 1] != k[q]) ranges[k[q]].y = (u32)(i + 1);
    }
}


// --------------------------------------------------------------- backward
// Chain of one Gaussian's image-space gradients
//   q0 = (u, v, conic a, conic b), q1 = (conic c, opacity, r, g), q2 = (b, z, -, -)
// back through the projection of Sec. 3.1 to its mean, log-scales, quaternion
// and opacity logit, and (gpose != nullptr) to the left perturbation
// xi = (rho, phi) of the pose.  Colour gradients pass through unchanged.
__device__ __forceinline__ void chain_to_params(const CamK &ck, const PoseR &pr, const GProj &g, float4 q0, float4 q1,
                                                float4 q2, float gm[3], float gls[3], float gq[4], float *glog,
                                                float gpose[6])
{
    const float gu = q0.x, gv = q0.y, gca = q0.z, gcb = q0.w, gcc = q1.x, gop = q1.y, gz = q2.y;
    *glog = gop * g.op * (1.f - g.op);
    // conic Q = S^-1: G_S = -Q G_Q Q with G_Q = [[ga, gb/2], [gb/2, gc]]
    const float idet = 1.f / g.det;
    const float Qa = g.c * idet, Qb = -g.b * idet, Qc = g.a * idet;
    const float hb = 0.5f * gcb;
    const float t00 = Qa * gca + Qb * hb, t01 = Qa * hb + Qb * gcc;
    const float t10 = Qb * gca + Qc * hb, t11 = Qb * hb + Qc * gcc;
    const float S00 = -(t00 * Qa + t01 * Qb), S01 = -(t00 * Qb + t01 * Qc);
    const float S11 = -(t10 * Qb + t11 * Qc);
    // S = T T^T + eps I  ->  G_T = 2 G_S T
    float GT[6];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        GT[k] = 2.f * (S00 * g.T[k] + S01 * g.T[3 + k]);
        GT[3 + k] = 2.f * (S01 * g.T[k] + S11 * g.T[3 + k]);
    }
    // T = J A -> G_J = G_T A^T (only J00, J02, J11, J12 depend on p), G_A = J^T G_T
    const float GJ00 = GT[0] * g.A[0] + GT[1] * g.A[1] + GT[2] * g.A[2];
    const float GJ02 = GT[0] * g.A[6] + GT[1] * g.A[7] + GT[2] * g.A[8];
    const float GJ11 = GT[3] * g.A[3] + GT[4] * g.A[4] + GT[5] * g.A[5];
    const float GJ12 = GT[3] * g.A[6] + GT[4] * g.A[7] + GT[5] * g.A[8];
    float GA[9];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        GA[k] = g.J[0] * GT[k];
        GA[3 + k] = g.J[4] * GT[3 + k];
        GA[6 + k] = g.J[2] * GT[k] + g.J[5] * GT[3 + k];
    }
    const float px = g.p[0], py = g.p[1], pz = g.p[2];
    const float iz = 1.f / pz, iz2 = iz * iz;
    float gp0 = gu * ck.fx * iz;
    float gp1 = gv * ck.fy * iz;
    float gp2 = -(gu * ck.fx * px + gv * ck.fy * py) * iz2 + gz;
    gp2 += GJ00 * (-ck.fx * iz2) + GJ02 * (ck.fx * g.tx * iz2) + GJ11 * (-ck.fy * iz2) + GJ12 * (ck.fy * g.ty * iz2);
    const float gtx = GJ02 * (-ck.fx * iz), gty = GJ12 * (-ck.fy * iz);
    if (!g.clx) {
        gp0 += gtx * iz;
        gp2 -= gtx * px * iz2;
    }
    if (!g.cly) {
        gp1 += gty * iz;
        gp2 -= gty * py * iz2;
    }
    if (gpose) {
        // rho = g_p, phi = p x g_p + vee(G_W W^T), G_W W^T = G_A A^T
        float Y[9];
#pragma unroll
        for (int r2 = 0; r2 < 3; ++r2)
#pragma unroll
            for (int c2 = 0; c2 < 3; ++c2)
                Y[3 * r2 + c2] = GA[3 * r2] * g.A[3 * c2] + GA[3 * r2 + 1] * g.A[3 * c2 + 1]
                               + GA[3 * r2 + 2] * g.A[3 * c2 + 2];
        gpose[0] = gp0;
        gpose[1] = gp1;
        gpose[2] = gp2;
        gpose[3] = py * gp2 - pz * gp1 + (Y[7] - Y[5]);
        gpose[4] = pz * gp0 - px * gp2 + (Y[2] - Y[6]);
        gpose[5] = px * gp1 - py * gp0 + (Y[3] - Y[1]);
    }
    if (gm) {
        // mean: p = W mu + t
#pragma unroll
        for (int k = 0; k < 3; ++k) gm[k] = pr.R[k] * gp0 + pr.R[3 + k] * gp1 + pr.R[6 + k] * gp2;
        // A = W M -> G_M = W^T G_A; M = R diag(s)
        float GM[9];
#pragma unroll
        for (int r2 = 0; r2 < 3; ++r2)
#pragma unroll
            for (int k = 0; k < 3; ++k)
                GM[3 * r2 + k] = pr.R[r2] * GA[k] + pr.R[3 + r2] * GA[3 + k] + pr.R[6 + r2] * GA[6 + k];
        float GR[9];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float gsk = GM[k] * g.R[k] + GM[3 + k] * g.R[3 + k] + GM[6 + k] * g.R[6 + k];
            gls[k] = gsk * g.s[k];
            GR[k] = GM[k] * g.s[k];
            GR[3 + k] = GM[3 + k] * g.s[k];
            GR[6 + k] = GM[6 + k] * g.s[k];
        }
        const float w = g.qh[0], x = g.qh[1], y = g.qh[2], z = g.qh[3];
        const float gw = 2.f * (-z * GR[1] + y * GR[2] + z * GR[3] - x * GR[5] - y * GR[6] + x * GR[7]);
        const float gx = 2.f * (y * GR[1] + z * GR[2] + y * GR[3] - 2.f * x * GR[4] - w * GR[5] + z * GR[6]
                                + w * GR[7] - 2.f * x * GR[8]);
        const float gy = 2.f * (-2.f * y * GR[0] + x * GR[1] + w * GR[2] + x * GR[3] + z * GR[5] - w * GR[6]
                                + z * GR[7] - 2.f * y * GR[8]);
        const float gzq = 2.f * (-2.f * z * GR[0] - w * GR[1] + x * GR[2] + w * GR[3] - 2.f * z * GR[4]
                                 + y * GR[5] + x * GR[6] + y * GR[7]);
        const float dot = gw * w + gx * x + gy * y + gzq * z;
        const float iq = 1.f / g.qn;
        gq[0] = (gw - w * dot) * iq;
        gq[1] = (gx - x * dot) * iq;
        gq[2] = (gy - y * dot) * iq;
        gq[3] = (gzq - z * dot) * iq;
    }
}

// K6: image-space gradients -> parameter gradients and the pose adjoint
// (block partial sums, reduced in a second pass).
template <bool WANT_PARAMS>
__global__ void __launch_bounds__(256, 4) k_project_bwd(Params P, CamK ck, const float *__restrict__ pose,
                                                     const int32_t *__restrict__ rank_of_gid,
                                                     const float *__restrict__ g2d, gsr_gaussian_grads dg,
                                                     int accumulate, float weight,
                                                     float *__restrict__ pose_part)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float gpose[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (i < P.n) {
        // start the parameter loads while the rank (which decides whether they are needed) arrives
        asm volatile("prefetch.global.L2 [%0];" ::"l"(P.mean + 3 * i));
        asm volatile("prefetch.global.L2 [%0];" ::"l"(P.log_scale + 3 * i));
        asm volatile("prefetch.global.L2 [%0];" ::"l"(P.quat + 4 * i));
        asm volatile("prefetch.global.L2 [%0];" ::"l"(P.opacity_logit + i));
        int32_t r = rank_of_gid[i];
        float gm[3] = {0.f, 0.f, 0.f}, gls[3] = {0.f, 0.f, 0.f}, gq[4] = {0.f, 0.f, 0.f, 0.f};
        float glog = 0.f, grgb[3] = {0.f, 0.f, 0.f};
        if (r >= 0) {
            const PoseR pr = load_pose(pose);
            GProj g;
            project_core(ck, pr, P.mean, P.log_scale, P.quat, P.opacity_logit[i], i, g);
            const float4 *G4 = reinterpret_cast<const float4 *>(g2d + 12 * (int64_t)r);
            const float4 q0 = G4[0], q1 = G4[1], q2 = G4[2];
            grgb[0] = q1.z;
            grgb[1] = q1.w;
            grgb[2] = q2.x;
            chain_to_params(ck, pr, g, q0, q1, q2, WANT_PARAMS ? gm : nullptr, gls, gq, &glog,
                            pose_part ? gpose : nullptr);
        }
        if (WANT_PARAMS) {
#define GSR_PUT(ptr, idx, val) \
    if (ptr) { if (accumulate) (ptr)[idx] += weight * (val); else (ptr)[idx] = (val); }
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                GSR_PUT(dg.mean, 3 * i + k, gm[k]);
                GSR_PUT(dg.log_scale, 3 * i + k, gls[k]);
                GSR_PUT(dg.rgb, 3 * i + k, grgb[k]);
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) GSR_PUT(dg.quat, 4 * i + k, gq[k]);
            GSR_PUT(dg.opacity_logit, i, glog);
#undef GSR_PUT
        }
    }
    if (pose_part) {
        // block reduction of the 6 pose components (deterministic order)
        __shared__ float red[6][8];
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            float v = gpose[k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (lane == 0) red[k][w] = v;
        }
        __syncthreads();
        if (threadIdx.x < 6) {
            float v = 0.f;
            for (int ww = 0; ww < 8; ++ww) v += red[threadIdx.x][ww];
            pose_part[6 * (int64_t)blockIdx.x + threadIdx.x] = v;
        }
    }
}

// Asynchronous global -> shared copies (cp.async): 16 bytes (both addresses
// 16-byte aligned) or 4 bytes.
__device__ __forceinline__ void cpa16(float *dst, const float *src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cpa4(float *dst, const float *src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}

// count consecutive floats from global src into shared dst by the whole block
// (V16: src 16-byte aligned, 16-byte copies and 4-byte ones for the last
// count % 4)
template <bool V16>
__device__ __forceinline__ void stage_in(float *dst, const float *src, int count)
{
    int q0 = 0;
    if (V16) {
        const int n4 = count >> 2;
        for (int q = threadIdx.x; q < n4; q += blockDim.x) cpa16(dst + 4 * q, src + 4 * q);
        q0 = 4 * n4;
    }
    for (int q = q0 + (int)threadIdx.x; q < count; q += blockDim.x) cpa4(dst + q, src + q);
}

template <bool V16>
__device__ __forceinline__ void stage_out(float *dst, const float *src, int count)
{
    int q0 = 0;
    if (V16) {
        const int n4 = count >> 2;
        for (int q = threadIdx.x; q < n4; q += blockDim.x)
            reinterpret_cast<float4 *>(dst)[q] = reinterpret_cast<const float4 *>(src)[q];
        q0 = 4 * n4;
    }
    for (int q = q0 + (int)threadIdx.x; q < count; q += blockDim.x) dst[q] = src[q];
}

// One-keyframe mapping step: the projection backward of Gaussian i (as in
// k_project_bwd) followed at once by its Adam update with L_reg, so its 14
// gradients never leave the block: the parameters are read once, the moments
// read and written once, and no gradient array is written or read back.
// Gaussians outside the view have zero gradients and still take their Adam
// step.  Per-block sums of the L_reg terms go to lreg_part.  The kernel reads
// the Adam step counter t - 1 (the bias corrections of step t are formed per
// block); the kernel after it advances the counter.
//
// None of the loads depends on a computed value except the image-gradient
// row (it needs the Gaussian's depth rank), so a block of PBA Gaussians first
// copies its slice of all 15 parameter and moment arrays and its gathered
// image-gradient rows into shared memory with asynchronous copies (27 KB in
// flight per block), then updates them there and writes the slices back with
// coalesced stores.  V16: every array base is 16-byte aligned.
constexpr int PBA = 128;
static_assert(PBA >= GSR_POSE_WORDS, "the pose record is staged by one thread per word");

template <bool V16>
__global__ void __launch_bounds__(PBA, 8) k_project_bwd_adam(gsr_gaussians_mut gw, CamK ck,
                                                             const float *__restrict__ pose,
                                                             const int32_t *__restrict__ rank_of_gid,
                                                             const float *__restrict__ g2d, gsr_adam_state st,
                                                             gsr_adam_opts o, float *__restrict__ lreg_part)
{
    // [params | m | v] x [mean 3 | log_scale 3 | quat 4 | opacity 1 | rgb 3] x PBA, then the image-gradient rows
    constexpr int OM = 0, OL = 3 * PBA, OQ = 6 * PBA, OO = 10 * PBA, OC = 11 * PBA, GROUP = 14 * PBA;
    __shared__ __align__(16) float sh[3 * GROUP + 12 * PBA];
    __shared__ float s_bc[2], s_pose[GSR_POSE_WORDS];
    float *sg = sh + 3 * GROUP;
    const int t = (int)threadIdx.x;
    const int64_t i0 = (int64_t)blockIdx.x * PBA, i = i0 + t;
    const int nloc = (int)min((int64_t)PBA, gw.n - i0);
    const float *arr[3][5] = {{gw.mean, gw.log_scale, gw.quat, gw.opacity_logit, gw.rgb},
                              {st.m_mean, st.m_log_scale, st.m_quat, st.m_opacity_logit, st.m_rgb},
                              {st.v_mean, st.v_log_scale, st.v_quat, st.v_opacity_logit, st.v_rgb}};
    constexpr int width[5] = {3, 3, 4, 1, 3}, off[5] = {OM, OL, OQ, OO, OC};
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int f = 0; f < 5; ++f)
            stage_in<V16>(sh + a * GROUP + off[f], arr[a][f] + width[f] * i0, width[f] * nloc);
    const int32_t r = t < nloc ? rank_of_gid[i] : -1;
    if (r >= 0) {
        const float *row = g2d + 12 * (int64_t)r;
        cpa16(sg + 12 * t, row);
        cpa16(sg + 12 * t + 4, row + 4);
        cpa16(sg + 12 * t + 8, row + 8);
    }
    if (t < GSR_POSE_WORDS) cpa4(s_pose + t, pose + t);
    if (t == 0) {
        const int ts = *st.step + 1;
        s_bc[0] = 1.f / (1.f - powf(o.beta1, (float)ts));
        s_bc[1] = 1.f / (1.f - powf(o.beta2, (float)ts));
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncthreads();
    float lreg = 0.f;
    if (t < nloc) {
        float *sp = sh, *smo = sh + GROUP, *svo = sh + 2 * GROUP;
        float gm[3] = {0.f, 0.f, 0.f}, gls[3] = {0.f, 0.f, 0.f}, gq[4] = {0.f, 0.f, 0.f, 0.f};
        float glog = 0.f, grgb[3] = {0.f, 0.f, 0.f};
        if (r >= 0) {
            const PoseR pr = load_pose(s_pose);
            GProj g;
            project_core(ck, pr, sp + OM, sp + OL, sp + OQ, sp[OO + t], t, g);
            const float4 *G4 = reinterpret_cast<const float4 *>(sg + 12 * t);
            const float4 q0 = G4[0], q1 = G4[1], q2 = G4[2];
            grgb[0] = q1.z;
            grgb[1] = q1.w;
            grgb[2] = q2.x;
            chain_to_params(ck, pr, g, q0, q1, q2, gm, gls, gq, &glog, nullptr);
        }
        const float ib1 = s_bc[0], ib2 = s_bc[1];  // reciprocal bias corrections
        // log-scales with L_reg
        float p[3], m[3], v[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            p[k] = sp[OL + 3 * t + k];
            m[k] = smo[OL + 3 * t + k];
            v[k] = svo[OL + 3 * t + k];
        }
        lreg = adam_log_scales3<true>(p, gls, m, v, o.w_reg / (float)gw.n, o.lr_log_scale, o, ib1, ib2);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            sp[OL + 3 * t + k] = p[k];
            smo[OL + 3 * t + k] = m[k];
            svo[OL + 3 * t + k] = v[k];
        }
        // means, colours, quaternion, opacity
        auto upd = [&](int idx, float gk, float lr) {
            adam_update_fast(sp[idx], gk, smo[idx], svo[idx], lr, o.beta1, o.beta2, o.eps, ib1, ib2);
        };
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            upd(OM + 3 * t + k, gm[k], o.lr_mean);
            upd(OC + 3 * t + k, grgb[k], o.lr_rgb);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) upd(OQ + 4 * t + k, gq[k], o.lr_quat);
        upd(OO + t, glog, o.lr_opacity);
    }
    __syncthreads();
    float *const warr[3][5] = {{gw.mean, gw.log_scale, gw.quat, gw.opacity_logit, gw.rgb},
                               {st.m_mean, st.m_log_scale, st.m_quat, st.m_opacity_logit, st.m_rgb},
                               {st.v_mean, st.v_log_scale, st.v_quat, st.v_opacity_logit, st.v_rgb}};
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int f = 0; f < 5; ++f)
            stage_out<V16>(warr[a][f] + width[f] * i0, sh + a * GROUP + off[f], width[f] * nloc);
    __shared__ float red[PBA / 32];
#pragma unroll
    for (int offs = 16; offs > 0; offs >>= 1) lreg += __shfl_down_sync(0xffffffffu, lreg, offs);
    if ((t & 31) == 0) red[t >> 5] = lreg;
    __syncthreads();
    if (t == 0) {
        float tot = 0.f;
        for (int k = 0; k < PBA / 32; ++k) tot += red[k];
        lreg_part[blockIdx.x] = tot;
    }
}

// Multi-keyframe projection backward: every Gaussian's parameters are read
// once, its image-space gradients of each keyframe in which it is visible
// are chained through that keyframe's pose and summed in registers, and the
// total is added to the gradient arrays (deterministic: no atomics).
__global__ void __launch_bounds__(256) k_project_bwd_multi(Params P, CamK ck, const ProjView *__restrict__ views,
                                                           int n_views, gsr_gaussian_grads dg)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n) return;
    float gm[3] = {0.f, 0.f, 0.f}, gls[3] = {0.f, 0.f, 0.f}, gq[4] = {0.f, 0.f, 0.f, 0.f}, glog = 0.f;
    float grgb[3] = {0.f, 0.f, 0.f};
    for (int k = 0; k < n_views; ++k) {
        const int32_t r = views[k].rank_of_gid[i];
        if (r < 0) continue;
        const PoseR pr = load_pose(views[k].pose);
        GProj g;
        project_core(ck, pr, P.mean, P.log_scale, P.quat, P.opacity_logit[i], i, g);
        const float4 *G4 = reinterpret_cast<const float4 *>(views[k].g2d + 12 * (int64_t)r);
        const float4 q0 = G4[0], q1 = G4[1], q2 = G4[2];
        float pm[3], pls[3], pq[4], plog;
        chain_to_params(ck, pr, g, q0, q1, q2, pm, pls, pq, &plog, nullptr);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            gm[c] += pm[c];
            gls[c] += pls[c];
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) gq[c] += pq[c];
        glog += plog;
        grgb[0] += q1.z;
        grgb[1] += q1.w;
        grgb[2] += q2.x;
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        dg.mean[3 * i + c] += gm[c];
        dg.log_scale[3 * i + c] += gls[c];
        dg.rgb[3 * i + c] += grgb[c];
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) dg.quat[4 * i + c] += gq[c];
    dg.opacity_logit[i] += glog;
}

// list entries as Gaussian ids; per-id depth bits (culled: 0xffffffff)
__global__ void k_lists_to_gid(int64_t cap_i, const u32 *__restrict__ d_n, const u32 *__restrict__ tvals,
                               const u32 *__restrict__ rank2gid, u32 *__restrict__ out)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < cap_i && i < (int64_t)*d_n) out[i] = rank2gid[tvals[i]];
}

__global__ void k_depth_bits(int64_t n, const u32 *__restrict__ flag, const float4 *__restrict__ rec,
                             u32 *__restrict__ out)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = flag[i] ? __float_as_uint(rec[3 * i + 1].z) : 0xffffffffu;
}

__global__ void k_pose_reduce(const float *__restrict__ part, int nb, float *__restrict__ out, int accumulate,
                              float weight)
{
    __shared__ float red[6][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;  // 6 warps? no: 192 threads = 6 warps of 32
    // warp w reduces component w over all blocks
    float v = 0.f;
    for (int b = lane; b < nb; b += 32) v += part[6 * b + w];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[w][0] = v;
    __syncthreads();
    if (threadIdx.x < 6) {
        if (accumulate) out[threadIdx.x] += weight * red[threadIdx.x][0];
        else out[threadIdx.x] = red[threadIdx.x][0];
    }
}

} // namespace

gsr_status launch_set_pose(gsr_ctx *ctx, float *d_pose, const gsr_pose &p, cudaStream_t s)
{
    k_set_pose<<<1, 1, 0, s>>>(d_pose, p);
    ctx->launches += 1;
    GSR_LAUNCHED(ctx);
    return GSR_OK;
}

gsr_status launch_perturb_pose(gsr_ctx *ctx, float *d_pose, const float *xi, cudaStream_t s)
{
    k_perturb_pose<<<1, 1, 0, s>>>(d_pose, xi);
    ctx->launches += 1;
    GSR_LAUNCHED(ctx);
    return GSR_OK;
}

extern "C" gsr_status gsr_pose_retract(const gsr_pose *pose, const float *xi, float *pose_out, void *stream)
{
    if (!pose || !xi || !pose_out) return GSR_ERR_INVALID_ARG;
    (void)cudaGetLastError();  // report only this call's launch
    k_pose_retract<<<1, 1, 0, (cudaStream_t)stream>>>(*pose, xi, pose_out);
    return cudaGetLastError() == cudaSuccess ? GSR_OK : GSR_ERR_CUDA;
}

gsr_status launch_pose_grad_xi(gsr_ctx *ctx, float *g6, const float *xi, cudaStream_t s)
{
    k_pose_grad_xi<<<1, 1, 0, s>>>(g6, xi);
    ctx->launches += 1;
    GSR_LAUNCHED(ctx);
    return GSR_OK;
}

static int bits_for(int64_t v)
{
    int b = 1;
    while (b < 32 && ((int64_t)1 << b) < v) ++b;
    return b;
}

gsr_status run_binning(gsr_ctx *ctx, ViewScratch &V, const Params &P, const CamK &ck, const float *d_pose,
                       bool allow_grow, cudaStream_t s, bool launch_order)
{
    V.order_valid = false;  // until this binning writes the order
    const int64_t n = P.n;
    const int64_t tiles = (int64_t)ck.tiles_x * ck.tiles_y;
    if (n > V.cap_n) {
        int64_t c = n;
        GSR_TRY(ensure_buf(ctx, V.rec, sizeof(float4) * 3 * c));
        GSR_TRY(ensure_buf(ctx, V.flag, sizeof(u32) * c));
        GSR_TRY(ensure_buf(ctx, V.compact, sizeof(u32) * c));
        GSR_TRY(ensure_buf(ctx, V.rank_of_gid, sizeof(int32_t) * c));
        for (int k = 0; k < 2; ++k) {
            GSR_TRY(ensure_buf(ctx, V.dkeys[k], sizeof(u32) * c));
            GSR_TRY(ensure_buf(ctx, V.dvals[k], sizeof(u32) * c));
        }
        GSR_TRY(ensure_buf(ctx, V.rec_sorted, sizeof(float4) * 3 * c));
        GSR_TRY(ensure_buf(ctx, V.tcount, sizeof(u32) * c));
        GSR_TRY(ensure_buf(ctx, V.inst_off, sizeof(u32) * c));
        GSR_TRY(ensure_buf(ctx, V.g2d, sizeof(float) * 12 * c));
        V.cap_n = c;
    }
    if (tiles > V.cap_t) {
        GSR_TRY(ensure_buf(ctx, V.ranges, sizeof(uint2) * tiles));
        GSR_TRY(ensure_buf(ctx, V.order, sizeof(u32) * tiles));
        GSR_TRY(ensure_buf(ctx, V.order_hist, order_hist_bytes(tiles)));
        V.cap_t = tiles;
    }
    GSR_TRY(ensure_buf(ctx, V.counters, sizeof(u32) * CNT_WORDS));
    u32 *cnt = (u32 *)V.counters.p;
    const unsigned nb = (unsigned)ceil_div(n > 0 ? n : 1, 256);

    k_project<<<nb, 256, 0, s>>>(P, ck, d_pose, (float4 *)V.rec.p, (u32 *)V.flag.p, (int32_t *)V.rank_of_gid.p);
    ctx->launches += 1;
    GSR_LAUNCHED(ctx);
    GSR_TRY(scan_exclusive(ctx, (u32 *)V.flag.p, (u32 *)V.compact.p, n, nullptr, cnt + CNT_VISIBLE, s,
                           &V.scan_tmp));
    k_compact<<<nb, 256, 0, s>>>(n, (u32 *)V.flag.p, (u32 *)V.compact.p, (float4 *)V.rec.p, (u32 *)V.dkeys[0].p,
                                 (u32 *)V.dvals[0].p);
    ctx->launches += 1;
    GSR_LAUNCHED(ctx);
    u32 *dk[2] = {(u32 *)V.dkeys[0].p, (u32 *)V.dkeys[1].p};
    u32 *dv[2] = {(u32 *)V.dvals[0].p, (u32 *)V.dvals[1].p};
    GSR_TRY(radix_sort_pairs(ctx, dk, dv, n, cnt + CNT_VISIBLE, 32, s, &V.radix_hist));
    const bool cull = !ctx->opt.rect_lists;
    if (cull)
        k_gather<true><<<nb, 256, 0, s>>>(n, cnt + CNT_VISIBLE, dv[0], (float4 *)V.rec.p, (float4 *)V.rec_sorted.p,
                                          (int32_t *)V.rank_of_gid.p, ck, (u32 *)V.tcount.p, (float4 *)V.g2d.p);
    else
        k_gather<false><<<nb, 256, 0, s>>>(n, cnt + CNT_VISIBLE, dv[0], (float4 *)V.rec.p, (float4 *)V.rec_sorted.p,
                                           (int32_t *)V.rank_of_gid.p, ck, (u32 *)V.tcount.p, (float4 *)V.g2d.p);
    ctx->launches += 1;
    GSR_LAUNCHED(ctx);
    V.g2d_zero = true;
    GSR_TRY(scan_exclusive(ctx, (u32 *)V.tcount.p, (u32 *)V.inst_off.p, n, cnt + CNT_VISIBLE,
                           cnt + CNT_INSTANCES, s, &V.scan_tmp));
    V.culled = cull;
    if (allow_grow) {
        // one 4-byte readback sizes the instance buffers (grow-on-demand mode)
        GSR_CUDA(ctx, cudaMemcpyAsync(ctx->host_pinned, cnt + CNT_INSTANCES, sizeof(u32), cudaMemcpyDeviceToHost, s));
        GSR_CUDA(ctx, cudaStreamSynchronize(s));
        int64_t need = (int64_t)ctx->host_pinned[0];
        if (need > V.cap_i) GSR_TRY(grow_instance_capacity(ctx, V, need + need / 4 + 1024));
    }
    if (V.cap_i <= 0) return gsr_fail(ctx, GSR_ERR_CAPACITY, "instance capacity is zero in fixed-capacity mode");
    if (cull)
        k_emit<true><<<nb, 256, 0, s>>>(n, cnt + CNT_VISIBLE, (float4 *)V.rec_sorted.p, (u32 *)V.tcount.p,
                                        (u32 *)V.inst_off.p, ck, V.cap_i, (u32 *)V.tkeys[0].p, (u32 *)V.tvals[0].p,
                                        cnt);
    else
        k_emit<false><<<nb, 256, 0, s>>>(n, cnt + CNT_VISIBLE, (float4 *)V.rec_sorted.p, (u32 *)V.tcount.p,
                                         (u32 *)V.inst_off.p, ck, V.cap_i, (u32 *)V.tkeys[0].p, (u32 *)V.tvals[0].p,
                                         cnt);
    ctx->launches += 1;
    GSR_LAUNCHED(ctx);
    u32 *tk[2] = {(u32 *)V.tkeys[0].p, (u32 *)V.tkeys[1].p};
    u32 *tv[2] = {(u32 *)V.tvals[0].p, (u32 *)V.tvals[1].p};
    GSR_TRY(radix_sort_pairs(ctx, tk, tv, V.cap_i, cnt + CNT_SORTN, bits_for(tiles), s, &V.radix_hist));
    GSR_CUDA(ctx, cudaMemsetAsync(V.ranges.p, 0, sizeof(uint2) * tiles, s));
    k_ranges<<<(unsigned)ceil_div(ceil_div(V.cap_i, 4), 256), 256, 0, s>>>(V.cap_i, cnt + CNT_SORTN, tk[0],
                                                                          (uint2 *)V.ranges.p);
    ctx->launches += 1;
    GSR_LAUNCHED(ctx);
    V.order_valid = launch_order;
    if (launch_order) GSR_TRY(run_order_tiles(ctx, V, tiles, s));
    return GSR_OK;
}

gsr_status run_project_backward(gsr_ctx *ctx, ViewScratch &V, const Params &P, const CamK &ck, const float *d_pose,
                                gsr_gaussian_grads *dg, float *d_pose6, bool accumulate, float weight,
                                cudaStream_t s)
{
    const int64_t n = P.n;
    const unsigned nb = (unsigned)ceil_div(n > 0 ? n : 1, 256);
    float *part = nullptr;
    if (d_pose6) {
        GSR_TRY(ensure_buf(ctx, ctx->pose_part, sizeof(float) * 6 * nb));
        part = (float *)ctx->pose_part.p;
    }
    gsr_gaussian_grads none{};
    bool want = dg && (dg->mean || dg->log_scale || dg->quat || dg->opacity_logit || dg->rgb);
    if (!want && !d_pose6) return GSR_OK;
    if (want)
        k_project_bwd<true><<<nb, 256, 0, s>>>(P, ck, d_pose, (int32_t *)V.rank_of_gid.p, (float *)V.g2d.p, *dg,
                                               accumulate ? 1 : 0, weight, part);
    else
        k_project_bwd<false><<<nb, 256, 0, s>>>(P, ck, d_pose, (int32_t *)V.rank_of_gid.p, (float *)V.g2d.p, none,
                                                0, weight, part);
    ctx->launches += 1;
    GSR_LAUNCHED(ctx);
    if (d_pose6) {
        k_pose_reduce<<<1, 192, 0, s>>>(part, (int)nb, d_pose6, accumulate ? 1 : 0, weight);
        ctx->launches += 1;
        GSR_LAUNCHED(ctx);
    }
    return GSR_OK;
}

int64_t project_bwd_adam_partials(int64_t n) { return ceil_div(n > 0 ? n : 1, PBA); }

gsr_status run_project_backward_adam(gsr_ctx *ctx, ViewScratch &V, gsr_gaussians_mut *g, gsr_adam_state *st,
                                     const gsr_adam_opts *o, const CamK &ck, const float *d_pose,
                                     float *loss_reg_dev, cudaStream_t s)
{
    const int64_t n = g->n;
    const unsigned nb = (unsigned)project_bwd_adam_partials(n);
    GSR_TRY(ensure_buf(ctx, ctx->pose_part, sizeof(float) * 6 * nb));
    float *part = (float *)ctx->pose_part.p;
    const void *ptrs[15] = {g->mean, g->log_scale, g->quat, g->opacity_logit, g->rgb,
                            st->m_mean, st->m_log_scale, st->m_quat, st->m_opacity_logit, st->m_rgb,
                            st->v_mean, st->v_log_scale, st->v_quat, st->v_opacity_logit, st->v_rgb};
    bool v16 = true;
    for (const void *q : ptrs) v16 = v16 && ((uintptr_t)q & 15u) == 0;
    if (v16)
        k_project_bwd_adam<true><<<nb, PBA, 0, s>>>(*g, ck, d_pose, (const int32_t *)V.rank_of_gid.p,
                                                   (const float *)V.g2d.p, *st, *o, part);
    else
        k_project_bwd_adam<false><<<nb, PBA, 0, s>>>(*g, ck, d_pose, (const int32_t *)V.rank_of_gid.p,
                                                    (const float *)V.g2d.p, *st, *o, part);
    ctx->launches += 1;
    GSR_LAUNCHED(ctx);
    if (loss_reg_dev)
        GSR_TRY(adam_lreg_final_step(ctx, part, (int)nb, o->w_reg / (float)(n > 0 ? n : 1), loss_reg_dev, st->step, s));
    return GSR_OK;
}

gsr_status copy_tile_lists(gsr_ctx *ctx, int64_t n, int64_t n_tiles, u32 *ranges_h, int32_t *gids_h,
                           int64_t capacity, u32 *depth_h, int64_t *n_inst, cudaStream_t s)
{
    ViewScratch &V = ctx->view;
    u32 *cnt = (u32 *)V.counters.p;
    GSR_CUDA(ctx, cudaMemcpyAsync(ctx->host_pinned, cnt, sizeof(u32) * 4, cudaMemcpyDeviceToHost, s));
    GSR_CUDA(ctx, cudaStreamSynchronize(s));
    int64_t ni = ctx->host_pinned[CNT_SORTN];
    *n_inst = ctx->host_pinned[CNT_INSTANCES];
    if (ranges_h) GSR_CUDA(ctx, cudaMemcpy(ranges_h, V.ranges.p, sizeof(uint2) * n_tiles, cudaMemcpyDeviceToHost));
    if (depth_h && n > 0) {
        // the depth-sort ping buffer 1 is free once the sort finished
        k_depth_bits<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(n, (u32 *)V.flag.p, (float4 *)V.rec.p,
                                                                (u32 *)V.dkeys[1].p);
        GSR_LAUNCHED(ctx);
        GSR_CUDA(ctx, cudaMemcpyAsync(depth_h, V.dkeys[1].p, sizeof(u32) * n, cudaMemcpyDeviceToHost, s));
        GSR_CUDA(ctx, cudaStreamSynchronize(s));
    }
    if (*n_inst > capacity || *n_inst > ni) return gsr_fail(ctx, GSR_ERR_CAPACITY, "tile list capacity");
    if (gids_h && ni > 0) {
        k_lists_to_gid<<<(unsigned)ceil_div(ni, 256), 256, 0, s>>>(V.cap_i, cnt + CNT_SORTN, (u32 *)V.tvals[0].p,
                                                                   (u32 *)V.dvals[0].p, (u32 *)V.tkeys[1].p);
        GSR_LAUNCHED(ctx);
        GSR_CUDA(ctx, cudaMemcpyAsync(gids_h, V.tkeys[1].p, sizeof(u32) * ni, cudaMemcpyDeviceToHost, s));
        GSR_CUDA(ctx, cudaStreamSynchronize(s));
    }
    return GSR_OK;
}

gsr_status run_project_backward_multi(gsr_ctx *ctx, const Params &P, const CamK &ck, const ProjView *views,
                                      int n_views, gsr_gaussian_grads *dg, cudaStream_t s)
{
    const unsigned nb = (unsigned)ceil_div(P.n > 0 ? P.n : 1, 256);
    k_project_bwd_multi<<<nb, 256, 0, s>>>(P, ck, views, n_views, *dg);
    ctx->launches += 1;
    GSR_LAUNCHED(ctx);
    return GSR_OK;
}
