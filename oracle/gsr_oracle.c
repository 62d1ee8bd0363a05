/*
 * gsr_oracle.c -- plain FP64 CPU oracle of the differentiable 3D-Gaussian
 * rasterizer used by Gaussian-SLAM (arXiv 2312.10070).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline leg of bench.py may load this library.  It shares no code,
 * header, table or helper with the CUDA path.
 *
 * Every step is written in the paper's order and notation, slow and direct:
 *   projection of the mean            Sec. 3.1, equation for mu^I
 *   EWA 2D covariance J R Sigma R^T J^T Sec. 3.1, equation for Sigma^I
 *   Sigma = R S S^T R^T                Sec. 3.1 (quaternion + scale)
 *   alpha_j = o_j exp(-sigma_j)       Sec. 3.1, equation for alpha_j
 *   colour blending C = sum c a T     Sec. 3.1, Eq. (color_blending)
 *   depth D = sum mu^z a T            Sec. 3.4, depth rendering equation
 *   dD/dalpha_j                       Sec. 3.4, depth adjoint equation
 *   L_depth, L_color (L1 + SSIM)      Sec. 3.4, Eqs. (depth_loss), (color_loss)
 *   L_reg, joint loss                 Sec. 3.4, Eq. (joint_loss)
 *   L_tracking with alpha^3 and 50x-median inlier masks
 *                                     Sec. 3.5 + supplementary Sec. B
 * Points the paper leaves open (pixel centres, dilation, thresholds, the
 * tile inclusion rule, sort tie-break, SSIM window) are fixed parameters
 * documented in the project's design notes; they are passed in through
 * orc_camera where they vary.
 *
 * Floating point: every quantity is double.  Inputs are float values the
 * caller promoted exactly to double (or arbitrary doubles for finite
 * differences).  The only float rounding is the sort key: tile lists are
 * ordered by (float(depth), index), the definition of the key order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int32_t width, height, tile_w, tile_h;
    double fx, fy, cx, cy;
    double z_near;   /* cull p_z <= z_near */
    double eps2d;    /* low-pass dilation added to the 2D covariance (px^2) */
    double guard;    /* guard band of the J linearisation, x half-FOV tangent */
    double amb_rel;  /* relative margin under which a blend decision is flagged */
    double guard_y;  /* guard band in y when > 0 (else `guard`); lets a crop keep
                        the full image's linearisation limits */
} orc_camera;

#define ALPHA_MIN (1.0 / 255.0)
#define ALPHA_MAX 0.99
#define T_STOP 1e-4

/* Rounding-error bounds of the float32 implementation, in units of the unit
 * roundoff U32 = 2^-24 (used only to flag decisions as ambiguous). */
#define U32 (1.0 / 16777216.0)
#define ERR_DF 1e-13        /* compensated p = R mu + t, relative to sum |terms| */
#define ERR_RATIO 5.0       /* u, v: on fx p_x / p_z (4 roundings) */
#define ERR_ROUND 1.25      /* u, v: the final rounding */
#define ERR_CONIC 32.0      /* conic as a quadratic form, x sqrt(kappa) */
#define ERR_OPAC 4.0        /* sigmoid in float */
#define ERR_SIGMA 6.0       /* sigma from the float conic and offsets, x sum |terms| */
#define ERR_EXP 5e-7        /* relative error of the single-precision exponential for sigma in [0, 6] */

/* per-Gaussian projection state (Sec. 3.1) */
typedef struct {
    int visible, radius, x0, y0, x1, y1;
    int amb;          /* bit0: a discrete projection decision is near its threshold
                         bit1: a gradient clamp is near its threshold */
    int vis_amb;      /* the cull decision itself is near its threshold */
    int ox0, oy0, ox1, oy1, ix0, iy0, ix1, iy1; /* outer / inner possible tile rectangles */
    double err_z, err_u, err_v; /* bounds of the float32 rounding error of p_z, u, v */
    int key_unc;      /* the float depth key may differ from the float rounding of p_z */
    double e_q;       /* relative error bound of the float conic as a quadratic form */
    int clamp_x, clamp_y;
    double u, v, depth, opacity;
    double cov[3];    /* Sigma^I + eps I:   a b c */
    double conic[3];  /* (Sigma^I + eps I)^-1 */
    double tx, ty;    /* (clamped) p_x/p_z, p_y/p_z */
    double p[3];      /* camera-space mean */
    double R[9];      /* rotation of the Gaussian */
    double s[3];      /* activated scales */
    double Sc[9];     /* camera-space covariance R_wc Sigma R_wc^T */
    double J[6];
    double qhat[4], qnorm;
} oproj;

static int imin(int a, int b) { return a < b ? a : b; }
static int imax(int a, int b) { return a > b ? a : b; }

/* unit quaternion (w, x, y, z) -> rotation matrix, row major */
static void quat_to_R(const double q[4], double R[9], double qhat[4], double *norm)
{
    double n = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    double w = q[0] / n, x = q[1] / n, y = q[2] / n, z = q[3] / n;
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
    if (qhat) { qhat[0] = w; qhat[1] = x; qhat[2] = y; qhat[3] = z; }
    if (norm) *norm = n;
}

static void matmul3(const double A[9], const double B[9], double C[9])
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0;
            for (int k = 0; k < 3; ++k) s += A[3 * i + k] * B[3 * k + j];
            C[3 * i + j] = s;
        }
}
static void transpose3(const double A[9], double B[9])
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) B[3 * j + i] = A[3 * i + j];
}

static double near_int_dist(double x) { return fabs(x - nearbyint(x)); }

static void project_one(const orc_camera *c, const double Rcw[9], const double tcw[3],
                        const double *mean, const double *log_scale, const double *quat,
                        double logit, oproj *o)
{
    memset(o, 0, sizeof(*o));
    /* activations: s = exp(log s), unit quaternion, o = sigmoid(logit) */
    for (int i = 0; i < 3; ++i) o->s[i] = exp(log_scale[i]);
    quat_to_R(quat, o->R, o->qhat, &o->qnorm);
    o->opacity = 1.0 / (1.0 + exp(-logit));

    /* Sigma = R S S^T R^T */
    double M[9], Mt[9], Sig[9];
    for (int r = 0; r < 3; ++r)
        for (int k = 0; k < 3; ++k) M[3 * r + k] = o->R[3 * r + k] * o->s[k];
    transpose3(M, Mt);
    matmul3(M, Mt, Sig);

    /* camera-space mean p = R_wc mu + t_wc (world-to-camera) */
    for (int i = 0; i < 3; ++i)
        o->p[i] = Rcw[3 * i] * mean[0] + Rcw[3 * i + 1] * mean[1] + Rcw[3 * i + 2] * mean[2] + tcw[i];
    double px = o->p[0], py = o->p[1], pz = o->p[2];
    o->depth = pz;
    /* Error model of the float32 implementation (each a bound; a decision
     * closer to its threshold than its bound is flagged as ambiguous and not
     * compared).  p = R mu + t is evaluated in compensated (double-float)
     * arithmetic, so before its final rounding p_z is within
     * ERR_DF (sum_j |R_zj mu_j| + |t_z|) of the exact value: the float depth
     * key is the correctly rounded p_z unless p_z lies within that distance
     * of a rounding midpoint (key_unc). */
    {
        double sabs = fabs(Rcw[6] * mean[0]) + fabs(Rcw[7] * mean[1]) + fabs(Rcw[8] * mean[2]) + fabs(tcw[2]);
        o->err_z = ERR_DF * sabs + 1e-300;
        float f = (float)pz;
        double up = nextafterf(f, INFINITY), dn = nextafterf(f, -INFINITY);
        double d1 = fabs(pz - 0.5 * ((double)f + up)), d2 = fabs(pz - 0.5 * ((double)f + dn));
        o->key_unc = fmin(d1, d2) <= o->err_z;
    }
    /* the near-plane test compares the float key with the float z_near */
    int z_amb = fabs(pz - c->z_near) <= o->err_z + 1.2e-7 * c->z_near;
    if (z_amb) { o->amb |= 1; o->vis_amb = 1; } /* its tiles (computed below) are marked */
    if (pz <= c->z_near && !z_amb) return;

    /* Sigma_cam = R_wc Sigma R_wc^T */
    double T1[9], Rt[9];
    matmul3(Rcw, Sig, T1);
    transpose3(Rcw, Rt);
    matmul3(T1, Rt, o->Sc);

    /* J: affine approximation of the perspective projection at p */
    double limx = c->guard * 0.5 * c->width / c->fx;
    double limy = (c->guard_y > 0 ? c->guard_y : c->guard) * 0.5 * c->height / c->fy;
    double tx = px / pz, ty = py / pz;
    if (fabs(fabs(tx) - limx) <= 1e-6 * limx || fabs(fabs(ty) - limy) <= 1e-6 * limy) o->amb |= 2;
    if (tx > limx) { tx = limx; o->clamp_x = 1; }
    if (tx < -limx) { tx = -limx; o->clamp_x = 1; }
    if (ty > limy) { ty = limy; o->clamp_y = 1; }
    if (ty < -limy) { ty = -limy; o->clamp_y = 1; }
    o->tx = tx; o->ty = ty;
    double *J = o->J;
    J[0] = c->fx / pz; J[1] = 0; J[2] = -c->fx * tx / pz;
    J[3] = 0; J[4] = c->fy / pz; J[5] = -c->fy * ty / pz;

    /* Sigma^I = J Sigma_cam J^T (+ eps I) */
    double JS[6];
    for (int r = 0; r < 2; ++r)
        for (int k = 0; k < 3; ++k)
            JS[3 * r + k] = J[3 * r] * o->Sc[k] + J[3 * r + 1] * o->Sc[3 + k] + J[3 * r + 2] * o->Sc[6 + k];
    double a = JS[0] * J[0] + JS[1] * J[1] + JS[2] * J[2] + c->eps2d;
    double b = JS[0] * J[3] + JS[1] * J[4] + JS[2] * J[5];
    double cc = JS[3] * J[3] + JS[4] * J[4] + JS[5] * J[5] + c->eps2d;
    o->cov[0] = a; o->cov[1] = b; o->cov[2] = cc;
    double det = a * cc - b * b;
    if (fabs(det) <= 1e-5 * fabs(a * cc)) { o->amb |= 1; o->vis_amb = 2; }
    if (det <= 0) return;
    o->conic[0] = cc / det; o->conic[1] = -b / det; o->conic[2] = a / det;
    {
        /* the float conic (inverse of Sigma^I = T T^T + eps I, T = J W R S
         * formed from float inputs) errs as a quadratic form by at most
         * ERR_CONIC u sqrt(kappa), kappa = the condition number of Sigma^I:
         * first-order propagation of the entry errors of T through T T^T
         * and the inverse scales with sqrt(kappa) */
        double hm = 0.5 * (a + cc), hd = sqrt(0.25 * (a - cc) * (a - cc) + b * b);
        double kappa = (hm + hd) / fmax(hm - hd, 1e-300);
        o->e_q = ERR_CONIC * U32 * sqrt(kappa);
    }

    /* screen radius: 3 sqrt(largest eigenvalue), rounded up */
    double lmax = 0.5 * (a + cc) + sqrt(0.25 * (a - cc) * (a - cc) + b * b);
    double r3 = 3.0 * sqrt(lmax);
    int rad = (int)ceil(r3);
    int rad_lo = rad, rad_hi = rad;
    if (near_int_dist(r3) <= 2e-6 * fmax(1.0, r3)) {
        o->amb |= 1;
        if (r3 - floor(r3) < 0.5) rad_lo = rad - 1; else rad_hi = rad + 1;
        if (rad_lo < 0) rad_lo = 0;
    }
    o->radius = rad;

    /* pinhole projection; pixel (i, j) has its centre at (i + 0.5, j + 0.5) */
    o->u = c->fx * px / pz + c->cx;
    o->v = c->fy * py / pz + c->cy;
    /* u = fx (p_x / p_z) + c_x in float from the rounded p_x, p_z: the ratio
     * carries four roundings (p_x, p_z, the reciprocal, the product), the
     * fused multiply-add one more on u */
    o->err_u = ERR_RATIO * U32 * c->fx * fabs(px / pz) + ERR_ROUND * U32 * fabs(o->u) + 1e-9;
    o->err_v = ERR_RATIO * U32 * c->fy * fabs(py / pz) + ERR_ROUND * U32 * fabs(o->v) + 1e-9;

    /* tile rectangle, inclusive, clamped to the tile grid */
    int tiles_x = (c->width + c->tile_w - 1) / c->tile_w;
    int tiles_y = (c->height + c->tile_h - 1) / c->tile_h;
    double ex[4] = {o->u - rad, o->u + rad, o->v - rad, o->v + rad};
    const double mu_ = o->err_u, mv_ = o->err_v; /* pixel margins of the rectangle edges */
    int empty = ex[1] < 0 || ex[0] >= c->width || ex[3] < 0 || ex[2] >= c->height;
    if (fabs(o->u + rad_lo) <= mu_ || fabs(o->u + rad_hi) <= mu_ || fabs(o->u - rad_lo - c->width) <= mu_
        || fabs(o->u - rad_hi - c->width) <= mu_ || fabs(o->v + rad_lo) <= mv_ || fabs(o->v + rad_hi) <= mv_
        || fabs(o->v - rad_lo - c->height) <= mv_ || fabs(o->v - rad_hi - c->height) <= mv_
        || (rad_lo != rad_hi && ((o->u + rad_lo < 0) != (o->u + rad_hi < 0)
                                 || (o->u - rad_lo >= c->width) != (o->u - rad_hi >= c->width)
                                 || (o->v + rad_lo < 0) != (o->v + rad_hi < 0)
                                 || (o->v - rad_lo >= c->height) != (o->v - rad_hi >= c->height)))) {
        o->amb |= 1;
        o->vis_amb = 1;
    }
    /* possible edge tiles under the margins */
    o->ox0 = imax(0, (int)floor((o->u - rad_hi - mu_) / c->tile_w));
    o->ix0 = imax(0, (int)floor((o->u - rad_lo + mu_) / c->tile_w));
    o->ix1 = imin(tiles_x - 1, (int)floor((o->u + rad_lo - mu_) / c->tile_w));
    o->ox1 = imin(tiles_x - 1, (int)floor((o->u + rad_hi + mu_) / c->tile_w));
    o->oy0 = imax(0, (int)floor((o->v - rad_hi - mv_) / c->tile_h));
    o->iy0 = imax(0, (int)floor((o->v - rad_lo + mv_) / c->tile_h));
    o->iy1 = imin(tiles_y - 1, (int)floor((o->v + rad_lo - mv_) / c->tile_h));
    o->oy1 = imin(tiles_y - 1, (int)floor((o->v + rad_hi + mv_) / c->tile_h));
    if (o->ox0 != o->ix0 || o->ox1 != o->ix1 || o->oy0 != o->iy0 || o->oy1 != o->iy1) o->amb |= 1;
    if (empty || pz <= c->z_near) return;
    o->x0 = imax(0, (int)floor(ex[0] / c->tile_w));
    o->x1 = imin(tiles_x - 1, (int)floor(ex[1] / c->tile_w));
    o->y0 = imax(0, (int)floor(ex[2] / c->tile_h));
    o->y1 = imin(tiles_y - 1, (int)floor(ex[3] / c->tile_h));
    o->visible = 1;
}

static void pose_R(const double *pose_q, double Rcw[9])
{
    quat_to_R(pose_q, Rcw, NULL, NULL);
}

static oproj *project_all(int64_t n, const double *mean, const double *log_scale, const double *quat,
                          const double *logit, const double *pose_q, const double *pose_t,
                          const orc_camera *cam)
{
    double Rcw[9];
    pose_R(pose_q, Rcw);
    oproj *P = (oproj *)malloc(sizeof(oproj) * (size_t)(n > 0 ? n : 1));
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i)
        project_one(cam, Rcw, pose_t, mean + 3 * i, log_scale + 3 * i, quat + 4 * i, logit[i], &P[i]);
    return P;
}

/* ---------------------------------------------------------------- binning */

typedef struct {
    int64_t n_tiles;
    int64_t total;
    int64_t *start;  /* n_tiles + 1 */
    int32_t *gid;    /* total, per tile ordered by (float depth, index) */
} olists;

static const oproj *g_sort_proj;
static int cmp_depth_gid(const void *pa, const void *pb)
{
    int32_t a = *(const int32_t *)pa, b = *(const int32_t *)pb;
    float da = (float)g_sort_proj[a].depth, db = (float)g_sort_proj[b].depth;
    if (da < db) return -1;
    if (da > db) return 1;
    return (a > b) - (a < b);
}

static void build_lists(int64_t n, const oproj *P, const orc_camera *cam, olists *L)
{
    int tiles_x = (cam->width + cam->tile_w - 1) / cam->tile_w;
    int tiles_y = (cam->height + cam->tile_h - 1) / cam->tile_h;
    L->n_tiles = (int64_t)tiles_x * tiles_y;
    L->start = (int64_t *)calloc((size_t)L->n_tiles + 1, sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) {
        if (!P[i].visible) continue;
        for (int ty = P[i].y0; ty <= P[i].y1; ++ty)
            for (int tx = P[i].x0; tx <= P[i].x1; ++tx) L->start[(int64_t)ty * tiles_x + tx + 1]++;
    }
    for (int64_t t = 0; t < L->n_tiles; ++t) L->start[t + 1] += L->start[t];
    L->total = L->start[L->n_tiles];
    L->gid = (int32_t *)malloc(sizeof(int32_t) * (size_t)(L->total > 0 ? L->total : 1));
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)L->n_tiles);
    memcpy(fill, L->start, sizeof(int64_t) * (size_t)L->n_tiles);
    for (int64_t i = 0; i < n; ++i) {
        if (!P[i].visible) continue;
        for (int ty = P[i].y0; ty <= P[i].y1; ++ty)
            for (int tx = P[i].x0; tx <= P[i].x1; ++tx) L->gid[fill[(int64_t)ty * tiles_x + tx]++] = (int32_t)i;
    }
    free(fill);
    g_sort_proj = P;
    for (int64_t t = 0; t < L->n_tiles; ++t)
        qsort(L->gid + L->start[t], (size_t)(L->start[t + 1] - L->start[t]), sizeof(int32_t), cmp_depth_gid);
}

static void free_lists(olists *L)
{
    free(L->start);
    free(L->gid);
}

/* two Gaussians whose float depth keys a float32 implementation may order
 * differently from the oracle: the keys are the correctly rounded depths
 * (ties broken by index on both sides) unless one of them is uncertain, and
 * then only neighbouring keys can swap */
static int depth_near_tie(const oproj *a, const oproj *b)
{
    return (a->key_unc || b->key_unc) && fabs(a->depth - b->depth) <= 2.5e-7 * fmax(fabs(a->depth), fabs(b->depth));
}

/* Gaussians whose list membership in a tile may differ because a projection
 * decision is within its margin, per tile (CSR): the tiles between the outer
 * and inner possible rectangles, all of the outer rectangle when the cull
 * decision itself is marginal.  `global` is set when a Gaussian with a
 * marginal determinant has no rectangle at all (its membership may differ
 * anywhere).  A pixel of such a tile is ambiguous only if the Gaussian could
 * composite there (tile_pixel_ambiguous). */
typedef struct { int64_t *start; int32_t *gid; int global; } oamb;

static int amb_marks(const oproj *g, int tx, int ty)
{
    if (g->vis_amb == 2) return 0;  /* handled as global */
    int outer = tx >= g->ox0 && tx <= g->ox1 && ty >= g->oy0 && ty <= g->oy1;
    int inner = tx >= g->ix0 && tx <= g->ix1 && ty >= g->iy0 && ty <= g->iy1;
    return outer && (g->vis_amb || !inner);
}

static void ambiguous_tiles(int64_t n, const oproj *P, const orc_camera *cam, oamb *A)
{
    int tiles_x = (cam->width + cam->tile_w - 1) / cam->tile_w;
    int tiles_y = (cam->height + cam->tile_h - 1) / cam->tile_h;
    int64_t nt = (int64_t)tiles_x * tiles_y;
    A->start = (int64_t *)calloc((size_t)nt + 1, sizeof(int64_t));
    A->global = 0;
    for (int pass = 0; pass < 2; ++pass) {
        int64_t *fill = pass ? (int64_t *)calloc((size_t)nt, sizeof(int64_t)) : NULL;
        for (int64_t i = 0; i < n; ++i) {
            const oproj *g = &P[i];
            if (!(g->amb & 1)) continue;
            if (g->vis_amb == 2) { A->global = 1; continue; }
            for (int ty = imax(0, g->oy0); ty <= imin(tiles_y - 1, g->oy1); ++ty)
                for (int tx = imax(0, g->ox0); tx <= imin(tiles_x - 1, g->ox1); ++tx) {
                    if (!amb_marks(g, tx, ty)) continue;
                    int64_t t = (int64_t)ty * tiles_x + tx;
                    if (pass == 0) A->start[t + 1]++;
                    else A->gid[A->start[t] + fill[t]++] = (int32_t)i;
                }
        }
        if (pass == 0) {
            for (int64_t t = 0; t < nt; ++t) A->start[t + 1] += A->start[t];
            A->gid = (int32_t *)malloc(sizeof(int32_t) * (size_t)(A->start[nt] > 0 ? A->start[nt] : 1));
        }
        free(fill);
    }
}

static void free_amb(oamb *A) { free(A->start); free(A->gid); }

/* 1 when a Gaussian whose membership in the pixel's tile is marginal could
 * composite at the pixel (alpha >= 1/255 up to a relative 1e-3): its presence
 * or absence then may change the pixel; otherwise it cannot. */
static int tile_pixel_ambiguous(const oamb *A, const oproj *P, int64_t t, int ix, int iy)
{
    if (A->global) return 1;
    const double xc = ix + 0.5, yc = iy + 0.5;  /* the pixel's centre */
    for (int64_t k = A->start[t]; k < A->start[t + 1]; ++k) {
        const oproj *g = &P[A->gid[k]];
        if (!(g->conic[0] > 0 && g->conic[2] > 0)) return 1;
        double dx = xc - g->u, dy = yc - g->v;
        double sigma = 0.5 * (g->conic[0] * dx * dx + g->conic[2] * dy * dy) + g->conic[1] * dx * dy;
        if (g->opacity * exp(-sigma) >= ALPHA_MIN * (1.0 - 1e-3)) return 1;
    }
    return 0;
}

/* ------------------------------------------------------------ public API */

/* Projection of every Gaussian.  Any output pointer may be NULL.
 * Returns the number of tile instances (sum of rectangle areas). */
int64_t orc_project(int64_t n, const double *mean, const double *log_scale, const double *quat,
                    const double *logit, const double *pose_q, const double *pose_t,
                    const orc_camera *cam, int32_t *visible, double *uv, double *depth,
                    double *cov2d, double *conic, double *opacity, int32_t *radius,
                    int32_t *rect, int32_t *amb)
{
    oproj *P = project_all(n, mean, log_scale, quat, logit, pose_q, pose_t, cam);
    int64_t total = 0;
    for (int64_t i = 0; i < n; ++i) {
        const oproj *o = &P[i];
        if (visible) visible[i] = o->visible;
        if (uv) { uv[2 * i] = o->u; uv[2 * i + 1] = o->v; }
        if (depth) depth[i] = o->depth;
        if (cov2d) for (int k = 0; k < 3; ++k) cov2d[3 * i + k] = o->cov[k];
        if (conic) for (int k = 0; k < 3; ++k) conic[3 * i + k] = o->conic[k];
        if (opacity) opacity[i] = o->opacity;
        if (radius) radius[i] = o->radius;
        if (rect) { rect[4 * i] = o->x0; rect[4 * i + 1] = o->y0; rect[4 * i + 2] = o->x1; rect[4 * i + 3] = o->y1; }
        if (amb) amb[i] = o->amb;
        if (o->visible) total += (int64_t)(o->x1 - o->x0 + 1) * (o->y1 - o->y0 + 1);
    }
    free(P);
    return total;
}

/* Per-tile ordered Gaussian lists.  tile_start has n_tiles+1 entries,
 * tile_gid and near_tie have capacity entries (near_tie may be NULL).
 * Returns the instance count, or -1 when capacity is too small. */
int64_t orc_bin(int64_t n, const double *mean, const double *log_scale, const double *quat,
                const double *logit, const double *pose_q, const double *pose_t,
                const orc_camera *cam, int64_t capacity, int64_t *tile_start, int32_t *tile_gid,
                int32_t *near_tie)
{
    oproj *P = project_all(n, mean, log_scale, quat, logit, pose_q, pose_t, cam);
    olists L;
    build_lists(n, P, cam, &L);
    int64_t total = L.total;
    if (total <= capacity) {
        memcpy(tile_start, L.start, sizeof(int64_t) * (size_t)(L.n_tiles + 1));
        memcpy(tile_gid, L.gid, sizeof(int32_t) * (size_t)total);
        if (near_tie)
            for (int64_t t = 0; t < L.n_tiles; ++t)
                for (int64_t k = L.start[t]; k < L.start[t + 1]; ++k)
                    near_tie[k] = (k > L.start[t]) && depth_near_tie(&P[L.gid[k]], &P[L.gid[k - 1]]);
    } else {
        total = -1;
    }
    free_lists(&L);
    free(P);
    return total;
}

/* ------------------------------------------------------------- blending */

/* one composited entry of a pixel's walk */
typedef struct { int32_t gid; double alpha, G, T, dx, dy, ex; int clamped; } ocontrib;

/* One pixel's front-to-back walk over its tile list (Eq. color_blending and
 * the depth equation of Sec. 3.4).  Entries are skipped when alpha < 1/255;
 * the walk stops, before compositing, at the first entry that would push the
 * transmittance below 1e-4.  `trace`, when non-NULL, receives the composited
 * entries in order. */
static void blend_pixel(const orc_camera *cam, const oproj *P, const double *rgb,
                        const int32_t *list, int64_t len, int ix, int iy,
                        double C[3], double *D, double *T_out, int32_t *last, int32_t *ncontrib,
                        int64_t *neval, int *amb, ocontrib *trace, unsigned flip, int *n_enum)
{
    /* flip: bit k takes the other branch of the k-th marginal skip (alpha vs
     * 1/255) or stop (T (1 - alpha) vs 1e-4) decision met on this walk, both
     * branches being results a float32 implementation may produce; n_enum
     * receives the number of such decisions met.  amb bit 0: some decision was
     * marginal; bit 1: a marginal alpha cap (gradient only); bit 3: a marginal
     * decision other than those two kinds (sigma sign, depth order). */
    int ne_k = 0;
    double px = ix + 0.5, py = iy + 0.5;
    double T = 1.0;
    int32_t lastpos = -1, nc = 0;
    int64_t ne = 0;
    int a = 0;
    const oproj *prev = NULL;
    /* relative error bound of the float transmittance so far (each composited
     * entry adds its alpha error amplified by alpha / (1 - alpha), plus one
     * rounding of the product), and an extra relative margin (amb_rel) */
    double eT = 0.0, eps = cam->amb_rel;
    C[0] = C[1] = C[2] = 0;
    *D = 0;
    for (int64_t k = 0; k < len; ++k) {
        int32_t gi = list[k];
        const oproj *g = &P[gi];
        ++ne;
        double dx = px - g->u, dy = py - g->v;
        /* sigma = 1/2 Delta^T (Sigma^I)^-1 Delta */
        double sigma = 0.5 * (g->conic[0] * dx * dx + g->conic[2] * dy * dy) + g->conic[1] * dx * dy;
        if (fabs(sigma) <= 1e-9) a |= 1 | 8;
        if (sigma < 0) continue;
        double ex = exp(-sigma);
        double G = g->opacity * ex; /* alpha_j = o_j exp(-sigma_j) */
        /* relative error bound of the float G: the float (u, v) moves sigma by
         * es, the float conic by e_q sigma, the float evaluation of sigma by
         * ERR_SIGMA u (sum of the magnitudes of its terms); the exponential,
         * the sigmoid and the product add their own */
        double es = fabs(g->conic[0] * dx + g->conic[1] * dy) * g->err_u
                  + fabs(g->conic[1] * dx + g->conic[2] * dy) * g->err_v;
        double sabs = 0.5 * (fabs(g->conic[0]) * dx * dx + fabs(g->conic[2]) * dy * dy) + fabs(g->conic[1] * dx * dy);
        double mg = eps + es + g->e_q * sigma + ERR_SIGMA * U32 * sabs + ERR_EXP + ERR_OPAC * U32 + U32;
        if (fabs(G - ALPHA_MAX) <= mg * ALPHA_MAX) a |= 2;
        int clamped = G > ALPHA_MAX;
        double alpha = clamped ? ALPHA_MAX : G;
        int skip = alpha < ALPHA_MIN;
        if (fabs(G - ALPHA_MIN) <= mg * ALPHA_MIN) {
            a |= 1;
            if ((flip >> ne_k) & 1u) skip = !skip;
            ++ne_k;
        }
        if (skip) continue;
        double ea = clamped ? 2e-8 : mg; /* the cap is 0.99 in float */
        double Tn = T * (1.0 - alpha);
        double eTn = eT + ea * alpha / (1.0 - alpha) + 2 * U32;
        int stop = Tn < T_STOP;
        if (fabs(Tn - T_STOP) <= (eps + eTn) * T_STOP) {
            a |= 1;
            if ((flip >> ne_k) & 1u) stop = !stop;
            ++ne_k;
        }
        if (stop) break;
        a |= g->amb & 2;
        if (prev && depth_near_tie(prev, g)) a |= 1 | 8;
        prev = g;
        eT = eTn;
        if (trace) {
            ocontrib *t = &trace[nc];
            t->gid = gi; t->alpha = alpha; t->G = G; t->T = T; t->dx = dx; t->dy = dy; t->ex = ex;
            t->clamped = clamped;
        }
        double w = alpha * T;
        for (int ch = 0; ch < 3; ++ch) C[ch] += rgb[3 * gi + ch] * w;
        *D += g->depth * w; /* D = sum mu^z alpha T, camera-space z */
        T = Tn;
        lastpos = (int32_t)k;
        ++nc;
    }
    *T_out = T;
    *last = lastpos;
    *ncontrib = nc;
    *neval = ne;
    *amb = a;
    if (n_enum) *n_enum = ne_k;
}

/* Render colour [3,H,W], depth [H,W], alpha = 1 - T_final [H,W], T_final,
 * last_idx (position in the tile list of the last composited entry, -1 if
 * none), n_contrib, pixel ambiguity flags, and the evaluation count E
 * (list entries visited over all pixels).  Any output may be NULL.  flips
 * [H,W] (NULL = none) selects, per pixel, the branches of its marginal skip
 * / stop decisions (as orc_render_alternatives). */
int orc_render(int64_t n, const double *mean, const double *log_scale, const double *quat,
               const double *logit, const double *rgb, const double *pose_q, const double *pose_t,
               const orc_camera *cam, double *out_rgb, double *out_depth, double *out_alpha,
               double *out_T, int32_t *out_last, int32_t *out_ncontrib, int32_t *out_amb,
               int64_t *out_neval, const uint32_t *flips)
{
    oproj *P = project_all(n, mean, log_scale, quat, logit, pose_q, pose_t, cam);
    olists L;
    build_lists(n, P, cam, &L);
    oamb A;
    ambiguous_tiles(n, P, cam, &A);
    int W = cam->width, H = cam->height;
    int tiles_x = (W + cam->tile_w - 1) / cam->tile_w;
    int64_t HW = (int64_t)W * H, etotal = 0;
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : etotal)
    for (int iy = 0; iy < H; ++iy) {
        for (int ix = 0; ix < W; ++ix) {
            int64_t t = (int64_t)(iy / cam->tile_h) * tiles_x + ix / cam->tile_w;
            double C[3], D, T;
            int32_t last, nc;
            int64_t ne;
            int a;
            blend_pixel(cam, P, rgb, L.gid + L.start[t], L.start[t + 1] - L.start[t], ix, iy, C, &D, &T,
                        &last, &nc, &ne, &a, NULL, flips ? flips[(int64_t)iy * W + ix] : 0u, NULL);
            int64_t p = (int64_t)iy * W + ix;
            if (out_rgb) for (int ch = 0; ch < 3; ++ch) out_rgb[ch * HW + p] = C[ch];
            if (out_depth) out_depth[p] = D;
            if (out_alpha) out_alpha[p] = 1.0 - T;
            if (out_T) out_T[p] = T;
            if (out_last) out_last[p] = last;
            if (out_ncontrib) out_ncontrib[p] = nc;
            if (out_amb) out_amb[p] = a | (tile_pixel_ambiguous(&A, P, t, ix, iy) ? 1 | 8 : 0);
            etotal += ne;
        }
    }
    if (out_neval) *out_neval = etotal;
    free_amb(&A);
    free_lists(&L);
    free(P);
    return 0;
}

/* Every result a float32 implementation may produce at the given pixels:
 * per pixel, the walks that take either branch of each marginal skip / stop
 * decision (bit k of a flip mask = the k-th such decision met, as
 * blend_pixel), up to 2^max_bits of them and at most kmax.  Outputs, [npix,
 * kmax] (colour [npix, kmax, 3]): colour, depth, final T, the Gaussian index
 * of the last composited entry (-1 if none), n_contrib and the flip mask of
 * each alternative; count [npix] the number of alternatives (1 where no
 * decision is marginal); amb [npix] the pixel's ambiguity flags. */
int orc_render_alternatives(int64_t n, const double *mean, const double *log_scale, const double *quat,
                            const double *logit, const double *rgb, const double *pose_q, const double *pose_t,
                            const orc_camera *cam, const int64_t *pix, int64_t npix, int max_bits, int kmax,
                            double *out_rgb, double *out_depth, double *out_T, int32_t *out_lastgid,
                            int32_t *out_nc, uint32_t *out_flip, int32_t *out_count, int32_t *out_amb)
{
    oproj *P = project_all(n, mean, log_scale, quat, logit, pose_q, pose_t, cam);
    olists L;
    build_lists(n, P, cam, &L);
    oamb A;
    ambiguous_tiles(n, P, cam, &A);
    int W = cam->width;
    int tiles_x = (W + cam->tile_w - 1) / cam->tile_w;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < npix; ++i) {
        int ix = (int)(pix[i] % W), iy = (int)(pix[i] / W);
        int64_t t = (int64_t)(iy / cam->tile_h) * tiles_x + ix / cam->tile_w;
        const int32_t *list = L.gid + L.start[t];
        int64_t len = L.start[t + 1] - L.start[t];
        double C[3], D, T;
        int32_t last, nc;
        int64_t ne;
        int a, nen = 0;
        blend_pixel(cam, P, rgb, list, len, ix, iy, C, &D, &T, &last, &nc, &ne, &a, NULL, 0u, &nen);
        out_amb[i] = a | (tile_pixel_ambiguous(&A, P, t, ix, iy) ? 1 | 8 : 0);
        int bits = nen < max_bits ? nen : max_bits;
        int cnt = 1 << bits;
        if (cnt > kmax) cnt = kmax;
        for (int m = 0; m < cnt; ++m) {
            if (m > 0) blend_pixel(cam, P, rgb, list, len, ix, iy, C, &D, &T, &last, &nc, &ne, &a, NULL, (unsigned)m, NULL);
            int64_t o = i * kmax + m;
            for (int ch = 0; ch < 3; ++ch) out_rgb[3 * o + ch] = C[ch];
            out_depth[o] = D;
            out_T[o] = T;
            out_lastgid[o] = last >= 0 ? list[last] : -1;
            out_nc[o] = nc;
            out_flip[o] = (uint32_t)m;
        }
        out_count[i] = cnt;
    }
    free_amb(&A);
    free_lists(&L);
    free(P);
    return 0;
}

/* ------------------------------------------------------------- backward */

/* d(R(qhat))/d(qhat_k) contracted with G_R */
static void rot_grad_quat(const double qh[4], const double GR[9], double gq[4])
{
    double w = qh[0], x = qh[1], y = qh[2], z = qh[3];
    double dw[9] = {0, -2 * z, 2 * y, 2 * z, 0, -2 * x, -2 * y, 2 * x, 0};
    double dx[9] = {0, 2 * y, 2 * z, 2 * y, -4 * x, -2 * w, 2 * z, 2 * w, -4 * x};
    double dy[9] = {-4 * y, 2 * x, 2 * w, 2 * x, 0, 2 * z, -2 * w, 2 * z, -4 * y};
    double dz[9] = {-4 * z, -2 * w, 2 * x, 2 * w, -4 * z, 2 * y, 2 * x, 2 * y, 0};
    gq[0] = gq[1] = gq[2] = gq[3] = 0;
    for (int i = 0; i < 9; ++i) {
        gq[0] += GR[i] * dw[i];
        gq[1] += GR[i] * dx[i];
        gq[2] += GR[i] * dy[i];
        gq[3] += GR[i] * dz[i];
    }
}

/* Chain of one Gaussian's image-space gradient
 *   g2 = [d_u, d_v, d_conic_a, d_conic_b, d_conic_c, d_opacity, d_r, d_g, d_b, d_depth]
 * back through Sec. 3.1's projection to its parameters and to the left
 * perturbation xi = (rho, phi) of the world-to-camera pose. */
static void project_backward_one(const orc_camera *cam, const double Rcw[9], const oproj *o,
                                 const double g2[10], double g_mean[3], double g_ls[3],
                                 double g_quat[4], double *g_logit, double g_rgb[3], double g_pose[6])
{
    double fx = cam->fx, fy = cam->fy;
    double px = o->p[0], py = o->p[1], pz = o->p[2];
    *g_logit = g2[5] * o->opacity * (1.0 - o->opacity);
    for (int k = 0; k < 3; ++k) g_rgb[k] = g2[6 + k];

    /* conic Q = S^-1, G_S = -Q G_Q Q, G_Q = [[ga, gb/2], [gb/2, gc]] */
    double Q[4] = {o->conic[0], o->conic[1], o->conic[1], o->conic[2]};
    double GQ[4] = {g2[2], 0.5 * g2[3], 0.5 * g2[3], g2[4]};
    double T2[4], GS[4];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) T2[2 * i + j] = Q[2 * i] * GQ[j] + Q[2 * i + 1] * GQ[2 + j];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) GS[2 * i + j] = -(T2[2 * i] * Q[j] + T2[2 * i + 1] * Q[2 + j]);

    /* S = J Sc J^T + eps I  ->  G_Sc = J^T G_S J,  G_J = 2 G_S J Sc */
    const double *J = o->J, *Sc = o->Sc;
    double GSc[9], GJ[6], JSc[6];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0;
            for (int a = 0; a < 2; ++a)
                for (int b = 0; b < 2; ++b) s += J[3 * a + i] * GS[2 * a + b] * J[3 * b + j];
            GSc[3 * i + j] = s;
        }
    for (int r = 0; r < 2; ++r)
        for (int k = 0; k < 3; ++k) JSc[3 * r + k] = J[3 * r] * Sc[k] + J[3 * r + 1] * Sc[3 + k] + J[3 * r + 2] * Sc[6 + k];
    for (int r = 0; r < 2; ++r)
        for (int k = 0; k < 3; ++k) GJ[3 * r + k] = 2.0 * (GS[2 * r] * JSc[k] + GS[2 * r + 1] * JSc[3 + k]);

    double gp[3] = {0, 0, 0};
    /* u = fx px/pz + cx,  v = fy py/pz + cy */
    gp[0] += g2[0] * fx / pz;
    gp[2] += -g2[0] * fx * px / (pz * pz);
    gp[1] += g2[1] * fy / pz;
    gp[2] += -g2[1] * fy * py / (pz * pz);
    /* depth route of D = sum z alpha T */
    gp[2] += g2[9];
    /* J entries: J00 = fx/pz, J02 = -fx tx/pz, J11 = fy/pz, J12 = -fy ty/pz */
    gp[2] += GJ[0] * (-fx / (pz * pz)) + GJ[2] * (fx * o->tx / (pz * pz))
           + GJ[4] * (-fy / (pz * pz)) + GJ[5] * (fy * o->ty / (pz * pz));
    double gtx = GJ[2] * (-fx / pz), gty = GJ[5] * (-fy / pz);
    if (!o->clamp_x) { gp[0] += gtx / pz; gp[2] += -gtx * px / (pz * pz); }
    if (!o->clamp_y) { gp[1] += gty / pz; gp[2] += -gty * py / (pz * pz); }

    /* p = R_wc mu + t */
    for (int k = 0; k < 3; ++k) g_mean[k] = Rcw[k] * gp[0] + Rcw[3 + k] * gp[1] + Rcw[6 + k] * gp[2];

    /* Sc = R_wc Sigma R_wc^T -> G_Sigma = R_wc^T G_Sc R_wc */
    double Rt[9], T3[9], GSig[9];
    transpose3(Rcw, Rt);
    matmul3(Rt, GSc, T3);
    matmul3(T3, Rcw, GSig);

    /* Sigma = M M^T, M = R diag(s) -> G_M = 2 G_Sigma M */
    double M[9], GM[9], GR[9];
    for (int r = 0; r < 3; ++r)
        for (int k = 0; k < 3; ++k) M[3 * r + k] = o->R[3 * r + k] * o->s[k];
    matmul3(GSig, M, GM);
    for (int i = 0; i < 9; ++i) GM[i] *= 2.0;
    for (int k = 0; k < 3; ++k) {
        double gs = 0;
        for (int r = 0; r < 3; ++r) gs += GM[3 * r + k] * o->R[3 * r + k];
        g_ls[k] = gs * o->s[k];
    }
    for (int r = 0; r < 3; ++r)
        for (int k = 0; k < 3; ++k) GR[3 * r + k] = GM[3 * r + k] * o->s[k];
    double gqh[4];
    rot_grad_quat(o->qhat, GR, gqh);
    double dot = gqh[0] * o->qhat[0] + gqh[1] * o->qhat[1] + gqh[2] * o->qhat[2] + gqh[3] * o->qhat[3];
    for (int k = 0; k < 4; ++k) g_quat[k] = (gqh[k] - o->qhat[k] * dot) / o->qnorm;

    /* pose, left perturbation exp(xi^) T_wc:  dp = drho + dphi x p,
     * dSc = [dphi]x Sc + Sc [dphi]x^T */
    g_pose[0] = gp[0]; g_pose[1] = gp[1]; g_pose[2] = gp[2];
    g_pose[3] = py * gp[2] - pz * gp[1];
    g_pose[4] = pz * gp[0] - px * gp[2];
    g_pose[5] = px * gp[1] - py * gp[0];
    double Y[9];
    matmul3(GSc, Sc, Y);
    g_pose[3] += 2.0 * (Y[7] - Y[5]);
    g_pose[4] += 2.0 * (Y[2] - Y[6]);
    g_pose[5] += 2.0 * (Y[3] - Y[1]);
}

/* Backward of the renderer.  Inputs dL/dC [3,H,W], dL/dD [H,W], dL/dA [H,W]
 * (any may be NULL = zero); flips [H,W] (NULL = none) selects, per pixel,
 * the branches of its marginal decisions (as orc_render_alternatives).  Outputs (NULL = not wanted): per-Gaussian
 * gradients of mean [n,3], log_scale [n,3], quat [n,4], opacity logit [n],
 * rgb [n,3], pose [6] (rho, phi), and the image-space gradients g2 [n,10]. */
int orc_render_backward(int64_t n, const double *mean, const double *log_scale, const double *quat,
                        const double *logit, const double *rgb, const double *pose_q,
                        const double *pose_t, const orc_camera *cam, const double *dL_drgb,
                        const double *dL_ddepth, const double *dL_dalpha, double *g_mean,
                        double *g_log_scale, double *g_quat, double *g_logit, double *g_rgb,
                        double *g_pose, double *g2d_out, const uint32_t *flips)
{
    oproj *P = project_all(n, mean, log_scale, quat, logit, pose_q, pose_t, cam);
    olists L;
    build_lists(n, P, cam, &L);
    int W = cam->width, H = cam->height;
    int tiles_x = (W + cam->tile_w - 1) / cam->tile_w;
    int64_t HW = (int64_t)W * H;
    double *g2 = (double *)calloc((size_t)(n > 0 ? n : 1) * 10, sizeof(double));
    int64_t maxlen = 1;
    for (int64_t t = 0; t < L.n_tiles; ++t)
        if (L.start[t + 1] - L.start[t] > maxlen) maxlen = L.start[t + 1] - L.start[t];

#pragma omp parallel
    {
        ocontrib *tr = (ocontrib *)malloc(sizeof(ocontrib) * (size_t)maxlen);
#pragma omp for schedule(dynamic, 4)
        for (int iy = 0; iy < H; ++iy) {
            for (int ix = 0; ix < W; ++ix) {
                int64_t t = (int64_t)(iy / cam->tile_h) * tiles_x + ix / cam->tile_w;
                int64_t p = (int64_t)iy * W + ix;
                double C[3], D, Tf;
                int32_t last, nc;
                int64_t ne;
                int a;
                blend_pixel(cam, P, rgb, L.gid + L.start[t], L.start[t + 1] - L.start[t], ix, iy, C, &D,
                            &Tf, &last, &nc, &ne, &a, tr, flips ? flips[p] : 0u, NULL);
                double dC[3], dD, dA;
                for (int ch = 0; ch < 3; ++ch) dC[ch] = dL_drgb ? dL_drgb[ch * HW + p] : 0.0;
                dD = dL_ddepth ? dL_ddepth[p] : 0.0;
                dA = dL_dalpha ? dL_dalpha[p] : 0.0;
                /* back to front; S = sum over later entries u > j of x_u alpha_u T_u */
                double Sc[3] = {0, 0, 0}, Sd = 0;
                for (int j = nc - 1; j >= 0; --j) {
                    const ocontrib *e = &tr[j];
                    const oproj *g = &P[e->gid];
                    double w = e->alpha * e->T, om = 1.0 - e->alpha;
                    double *gg = g2 + 10 * (int64_t)e->gid;
                    double cj[3] = {rgb[3 * e->gid], rgb[3 * e->gid + 1], rgb[3 * e->gid + 2]};
                    /* dC/dalpha_j = c_j T_j - S_c/(1 - alpha_j); same form for depth
                     * (Sec. 3.4's depth adjoint); dA/dalpha_j = T_final/(1 - alpha_j) */
                    double dLda = 0;
                    for (int ch = 0; ch < 3; ++ch) dLda += dC[ch] * (cj[ch] * e->T - Sc[ch] / om);
                    dLda += dD * (g->depth * e->T - Sd / om);
                    dLda += dA * (Tf / om);
                    double du = 0, dv = 0, da = 0, db = 0, dc = 0, dop = 0;
                    if (!e->clamped) {
                        dop = dLda * e->ex;
                        double dsig = -dLda * e->G;
                        du = dsig * -(g->conic[0] * e->dx + g->conic[1] * e->dy);
                        dv = dsig * -(g->conic[1] * e->dx + g->conic[2] * e->dy);
                        da = dsig * 0.5 * e->dx * e->dx;
                        db = dsig * e->dx * e->dy;
                        dc = dsig * 0.5 * e->dy * e->dy;
                    }
                    double add[10] = {du, dv, da, db, dc, dop, dC[0] * w, dC[1] * w, dC[2] * w, dD * w};
                    for (int k = 0; k < 10; ++k) {
#pragma omp atomic
                        gg[k] += add[k];
                    }
                    for (int ch = 0; ch < 3; ++ch) Sc[ch] += cj[ch] * w;
                    Sd += g->depth * w;
                }
            }
        }
        free(tr);
    }

    double Rcw[9];
    pose_R(pose_q, Rcw);
    double gpose[6] = {0, 0, 0, 0, 0, 0};
    for (int64_t i = 0; i < n; ++i) {
        double gm[3] = {0, 0, 0}, gl[3] = {0, 0, 0}, gq[4] = {0, 0, 0, 0}, go = 0, gc[3] = {0, 0, 0};
        double gpo[6] = {0, 0, 0, 0, 0, 0};
        if (P[i].visible) {
            project_backward_one(cam, Rcw, &P[i], g2 + 10 * i, gm, gl, gq, &go, gc, gpo);
            for (int k = 0; k < 6; ++k) gpose[k] += gpo[k];
        }
        if (g_mean) for (int k = 0; k < 3; ++k) g_mean[3 * i + k] = gm[k];
        if (g_log_scale) for (int k = 0; k < 3; ++k) g_log_scale[3 * i + k] = gl[k];
        if (g_quat) for (int k = 0; k < 4; ++k) g_quat[4 * i + k] = gq[k];
        if (g_logit) g_logit[i] = go;
        if (g_rgb) for (int k = 0; k < 3; ++k) g_rgb[3 * i + k] = gc[k];
    }
    if (g_pose) for (int k = 0; k < 6; ++k) g_pose[k] = gpose[k];
    if (g2d_out) memcpy(g2d_out, g2, sizeof(double) * (size_t)n * 10);
    free(g2);
    free_lists(&L);
    free(P);
    return 0;
}

/* Backward of the projection alone, from given image-space gradients g2d
 * [n,10] (layout as orc_render_backward's g2d_out). */
int orc_project_backward(int64_t n, const double *mean, const double *log_scale, const double *quat,
                         const double *logit, const double *pose_q, const double *pose_t,
                         const orc_camera *cam, const double *g2d, double *g_mean, double *g_log_scale,
                         double *g_quat, double *g_logit, double *g_rgb, double *g_pose)
{
    oproj *P = project_all(n, mean, log_scale, quat, logit, pose_q, pose_t, cam);
    double Rcw[9];
    pose_R(pose_q, Rcw);
    double gpose[6] = {0, 0, 0, 0, 0, 0};
    for (int64_t i = 0; i < n; ++i) {
        double gm[3] = {0, 0, 0}, gl[3] = {0, 0, 0}, gq[4] = {0, 0, 0, 0}, go = 0, gc[3] = {0, 0, 0};
        double gpo[6] = {0, 0, 0, 0, 0, 0};
        if (P[i].visible) {
            project_backward_one(cam, Rcw, &P[i], g2d + 10 * i, gm, gl, gq, &go, gc, gpo);
            for (int k = 0; k < 6; ++k) gpose[k] += gpo[k];
        }
        if (g_mean) for (int k = 0; k < 3; ++k) g_mean[3 * i + k] = gm[k];
        if (g_log_scale) for (int k = 0; k < 3; ++k) g_log_scale[3 * i + k] = gl[k];
        if (g_quat) for (int k = 0; k < 4; ++k) g_quat[4 * i + k] = gq[k];
        if (g_logit) g_logit[i] = go;
        if (g_rgb) for (int k = 0; k < 3; ++k) g_rgb[3 * i + k] = gc[k];
    }
    if (g_pose) for (int k = 0; k < 6; ++k) g_pose[k] = gpose[k];
    free(P);
    return 0;
}

/* --------------------------------------------------------------- losses */

static double sgn(double x) { return (x > 0) - (x < 0); }

/* 11x11 Gaussian window, sigma 1.5, normalised to sum 1 (Wang et al. SSIM) */
static void ssim_window(double w[11][11])
{
    double g[11], s = 0;
    for (int k = 0; k < 11; ++k) { g[k] = exp(-((k - 5) * (k - 5)) / (2.0 * 1.5 * 1.5)); s += g[k]; }
    for (int i = 0; i < 11; ++i)
        for (int j = 0; j < 11; ++j) w[i][j] = (g[i] / s) * (g[j] / s);
}

/* windowed sum with zero padding: out(p) = sum_k w(k) f(p + k - 5) */
static void window_sum(int H, int W, const double w[11][11], const double *f, double *out)
{
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            double s = 0;
            for (int i = 0; i < 11; ++i) {
                int yy = y + i - 5;
                if (yy < 0 || yy >= H) continue;
                for (int j = 0; j < 11; ++j) {
                    int xx = x + j - 5;
                    if (xx < 0 || xx >= W) continue;
                    s += w[i][j] * f[(int64_t)yy * W + xx];
                }
            }
            out[(int64_t)y * W + x] = s;
        }
}

/* Mean SSIM over pixels and the 3 channels; optional per-pixel map [3,H,W]
 * and gradient d(mean SSIM)/dx accumulated with weight `gscale` into dx. */
static double ssim_mean(int H, int W, const double *x, const double *y, double *map, double *dx,
                        double gscale)
{
    const double C1 = 0.01 * 0.01, C2 = 0.03 * 0.03;
    double w[11][11];
    ssim_window(w);
    int64_t HW = (int64_t)H * W;
    double *buf = (double *)malloc(sizeof(double) * (size_t)HW * 11);
    double *mx = buf, *my = buf + HW, *exx = buf + 2 * HW, *eyy = buf + 3 * HW, *exy = buf + 4 * HW;
    double *t = buf + 5 * HW, *P1 = buf + 6 * HW, *P2 = buf + 7 * HW, *P3 = buf + 8 * HW;
    double *B1w = buf + 9 * HW, *B2w = buf + 10 * HW;
    double total = 0;
    for (int ch = 0; ch < 3; ++ch) {
        const double *xc = x + ch * HW, *yc = y + ch * HW;
        window_sum(H, W, w, xc, mx);
        window_sum(H, W, w, yc, my);
        for (int64_t p = 0; p < HW; ++p) t[p] = xc[p] * xc[p];
        window_sum(H, W, w, t, exx);
        for (int64_t p = 0; p < HW; ++p) t[p] = yc[p] * yc[p];
        window_sum(H, W, w, t, eyy);
        for (int64_t p = 0; p < HW; ++p) t[p] = xc[p] * yc[p];
        window_sum(H, W, w, t, exy);
        for (int64_t p = 0; p < HW; ++p) {
            double m1 = mx[p], m2 = my[p];
            double sx = exx[p] - m1 * m1, sy = eyy[p] - m2 * m2, sxy = exy[p] - m1 * m2;
            double A1 = 2 * m1 * m2 + C1, A2 = 2 * sxy + C2;
            double B1 = m1 * m1 + m2 * m2 + C1, B2 = sx + sy + C2;
            double S = (A1 * A2) / (B1 * B2);
            total += S;
            if (map) map[ch * HW + p] = S;
            /* dS/dmu_x, dS/dE[x^2], dS/dE[xy] */
            P1[p] = gscale * (2 * m2 * (A2 - A1) / (B1 * B2) - 2 * m1 * S * (1.0 / B1 - 1.0 / B2));
            P2[p] = gscale * (-S / B2);
            P3[p] = gscale * (2 * A1 / (B1 * B2));
        }
        if (dx) {
            /* the window is symmetric: the adjoint of the windowed sum is itself */
            window_sum(H, W, w, P1, B1w);
            window_sum(H, W, w, P2, B2w);
            window_sum(H, W, w, P3, t);
            for (int64_t p = 0; p < HW; ++p) dx[ch * HW + p] += B1w[p] + 2 * xc[p] * B2w[p] + yc[p] * t[p];
        }
    }
    free(buf);
    return total / (3.0 * HW);
}

/* Mapping loss, Eq. (joint_loss) without L_reg:
 *   L = w_color [(1 - lam) mean|I^ - I| + lam (1 - SSIM(I^, I))] + w_depth mean_valid|D^ - D|
 * valid = target depth > 0.  Writes dL/dI^ [3,H,W] and dL/dD^ [H,W] (NULL = skip)
 * and the SSIM map (NULL = skip).  Returns L. */
double orc_loss_map(int H, int W, const double *rgb, const double *depth, const double *rgb_t,
                    const double *depth_t, double lam, double w_color, double w_depth,
                    double *d_rgb, double *d_depth, double *ssim_map, double *parts)
{
    int64_t HW = (int64_t)H * W, nvalid = 0;
    double l1c = 0, l1d = 0;
    for (int64_t i = 0; i < 3 * HW; ++i) l1c += fabs(rgb[i] - rgb_t[i]);
    l1c /= (3.0 * HW);
    for (int64_t p = 0; p < HW; ++p)
        if (depth_t[p] > 0) { ++nvalid; l1d += fabs(depth[p] - depth_t[p]); }
    if (nvalid > 0) l1d /= (double)nvalid;
    if (d_rgb) for (int64_t i = 0; i < 3 * HW; ++i) d_rgb[i] = w_color * (1 - lam) * sgn(rgb[i] - rgb_t[i]) / (3.0 * HW);
    double ssim = ssim_mean(H, W, rgb, rgb_t, ssim_map, d_rgb, -w_color * lam / (3.0 * HW));
    if (d_depth)
        for (int64_t p = 0; p < HW; ++p)
            d_depth[p] = (depth_t[p] > 0 && nvalid > 0) ? w_depth * sgn(depth[p] - depth_t[p]) / (double)nvalid : 0.0;
    if (parts) { parts[0] = l1c; parts[1] = ssim; parts[2] = l1d; parts[3] = (double)nvalid; }
    return w_color * ((1 - lam) * l1c + lam * (1 - ssim)) + w_depth * l1d;
}

static int cmp_double(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

/* Tracking loss (Sec. 3.5, supplementary Sec. B):
 *   L = sum_p M_inlier M_alpha (lam_c sum_ch |I^ - I| + (1 - lam_c)|D^ - D|)
 * M_alpha = alpha^apow (detached), M_inlier = valid & |D^ - D| <= k * lower median
 * of |D^ - D| over valid pixels.  Writes dL/dI^, dL/dD^, the inlier mask and
 * the median (NULL = skip).  Returns L. */
double orc_loss_track(int H, int W, const double *rgb, const double *depth, const double *alpha,
                      const double *rgb_t, const double *depth_t, double lam_c, double k_med,
                      double apow, double *d_rgb, double *d_depth, int32_t *inlier, double *median)
{
    int64_t HW = (int64_t)H * W, nv = 0;
    double *e = (double *)malloc(sizeof(double) * (size_t)(HW > 0 ? HW : 1));
    for (int64_t p = 0; p < HW; ++p)
        if (depth_t[p] > 0) e[nv++] = fabs(depth[p] - depth_t[p]);
    double med = 0;
    if (nv > 0) {
        qsort(e, (size_t)nv, sizeof(double), cmp_double);
        med = e[(nv - 1) / 2];
    }
    free(e);
    if (median) *median = med;
    double L = 0;
    for (int64_t p = 0; p < HW; ++p) {
        int valid = depth_t[p] > 0;
        double ed = fabs(depth[p] - depth_t[p]);
        int in = valid && ed <= k_med * med;
        double w = in ? pow(alpha[p], apow) : 0.0;
        double lc = 0;
        for (int ch = 0; ch < 3; ++ch) lc += fabs(rgb[ch * HW + p] - rgb_t[ch * HW + p]);
        L += w * (lam_c * lc + (1 - lam_c) * ed);
        if (d_rgb) for (int ch = 0; ch < 3; ++ch) d_rgb[ch * HW + p] = w * lam_c * sgn(rgb[ch * HW + p] - rgb_t[ch * HW + p]);
        if (d_depth) d_depth[p] = w * (1 - lam_c) * sgn(depth[p] - depth_t[p]);
        if (inlier) inlier[p] = in;
    }
    return L;
}

/* Isotropic regulariser L_reg = (1/|K|) sum_k |s_k - sbar_k|_1 with s = exp(log_scale)
 * and sbar_k the mean of Gaussian k's three scales.  Adds w * dL_reg/dlog_scale
 * into g_log_scale (NULL = skip).  Returns L_reg. */
double orc_lreg(int64_t n, const double *log_scale, double w, double *g_log_scale)
{
    if (n <= 0) return 0;
    double L = 0;
    for (int64_t k = 0; k < n; ++k) {
        double s[3], sb = 0;
        for (int a = 0; a < 3; ++a) { s[a] = exp(log_scale[3 * k + a]); sb += s[a]; }
        sb /= 3.0;
        double sg[3], ssum = 0;
        for (int a = 0; a < 3; ++a) { L += fabs(s[a] - sb); sg[a] = sgn(s[a] - sb); ssum += sg[a]; }
        if (g_log_scale)
            for (int a = 0; a < 3; ++a) g_log_scale[3 * k + a] += w * (sg[a] - ssum / 3.0) * s[a] / (double)n;
    }
    return L / (double)n;
}

/* Adam (bias corrected) on m elements; `step` is the 1-based step count. */
void orc_adam(int64_t m, double *param, const double *grad, double *m1, double *m2, int64_t step,
              double lr, double b1, double b2, double eps)
{
    double bc1 = 1.0 - pow(b1, (double)step), bc2 = 1.0 - pow(b2, (double)step);
    for (int64_t i = 0; i < m; ++i) {
        m1[i] = b1 * m1[i] + (1 - b1) * grad[i];
        m2[i] = b2 * m2[i] + (1 - b2) * grad[i] * grad[i];
        double mh = m1[i] / bc1, vh = m2[i] / bc2;
        param[i] -= lr * mh / (sqrt(vh) + eps);
    }
}

/* Left retraction of a world-to-camera pose: T <- exp(xi^) T with
 * xi = (rho, phi), the SE(3) exponential in closed form (Rodrigues + V). */
void orc_pose_retract(const double *q_in, const double *t_in, const double *xi, double *q_out,
                      double *t_out)
{
    const double *rho = xi, *phi = xi + 3;
    double th = sqrt(phi[0] * phi[0] + phi[1] * phi[1] + phi[2] * phi[2]);
    double K[9] = {0, -phi[2], phi[1], phi[2], 0, -phi[0], -phi[1], phi[0], 0};
    double K2[9];
    matmul3(K, K, K2);
    double A, B, Cc;
    if (th < 1e-8) { A = 1.0; B = 0.5; Cc = 1.0 / 6.0; }
    else { A = sin(th) / th; B = (1 - cos(th)) / (th * th); Cc = (th - sin(th)) / (th * th * th); }
    double Rd[9], V[9];
    for (int i = 0; i < 9; ++i) {
        double I = (i % 4 == 0) ? 1.0 : 0.0;
        Rd[i] = I + A * K[i] + B * K2[i];
        V[i] = I + B * K[i] + Cc * K2[i];
    }
    double R0[9], R1[9];
    quat_to_R(q_in, R0, NULL, NULL);
    matmul3(Rd, R0, R1);
    for (int i = 0; i < 3; ++i)
        t_out[i] = Rd[3 * i] * t_in[0] + Rd[3 * i + 1] * t_in[1] + Rd[3 * i + 2] * t_in[2]
                 + V[3 * i] * rho[0] + V[3 * i + 1] * rho[1] + V[3 * i + 2] * rho[2];
    /* rotation matrix -> unit quaternion (w >= 0) */
    double tr = R1[0] + R1[4] + R1[8], w, x, y, z;
    if (tr > 0) {
        double s = sqrt(tr + 1.0) * 2;
        w = 0.25 * s; x = (R1[7] - R1[5]) / s; y = (R1[2] - R1[6]) / s; z = (R1[3] - R1[1]) / s;
    } else if (R1[0] > R1[4] && R1[0] > R1[8]) {
        double s = sqrt(1.0 + R1[0] - R1[4] - R1[8]) * 2;
        w = (R1[7] - R1[5]) / s; x = 0.25 * s; y = (R1[1] + R1[3]) / s; z = (R1[2] + R1[6]) / s;
    } else if (R1[4] > R1[8]) {
        double s = sqrt(1.0 + R1[4] - R1[0] - R1[8]) * 2;
        w = (R1[2] - R1[6]) / s; x = (R1[1] + R1[3]) / s; y = 0.25 * s; z = (R1[5] + R1[7]) / s;
    } else {
        double s = sqrt(1.0 + R1[8] - R1[0] - R1[4]) * 2;
        w = (R1[3] - R1[1]) / s; x = (R1[2] + R1[6]) / s; y = (R1[5] + R1[7]) / s; z = 0.25 * s;
    }
    if (w < 0) { w = -w; x = -x; y = -y; z = -z; }
    q_out[0] = w; q_out[1] = x; q_out[2] = y; q_out[3] = z;
}

/* SE(3) left Jacobian J_l(xi), xi = (rho, phi), row major 6x6: to first
 * order exp((xi + e)^) = exp((J_l e)^) exp(xi^).  With K = [phi]x,
 * P = [rho]x and th = |phi| it is [[V, Q], [0, V]], V = I + B K + C K^2 the
 * SO(3) left Jacobian (B, C of orc_pose_retract) and
 *   Q = P/2 + c1 (K P + P K + K P K) + c2 (K K P + P K K - 3 K P K)
 *         + c3 (K P K K + K K P K),
 *   c1 = (th - sin th)/th^3, c2 = (th^2 + 2 cos th - 2)/(2 th^4),
 *   c3 = (2 th - 3 sin th + th cos th)/(2 th^5)
 * (their Taylor series near th = 0).  The gradient of a loss with respect to
 * the twist of T(xi) = exp(xi^) T is J_l(xi)^T times its left-perturbation
 * gradient at T(xi). */
void orc_se3_left_jacobian(const double *xi, double *J)
{
    const double *rho = xi, *phi = xi + 3;
    double th = sqrt(phi[0] * phi[0] + phi[1] * phi[1] + phi[2] * phi[2]), t2 = th * th;
    double B, Cc, c1, c2, c3;
    if (th < 1e-2) {
        B = 0.5 - t2 / 24.0 + t2 * t2 / 720.0;
        Cc = 1.0 / 6.0 - t2 / 120.0 + t2 * t2 / 5040.0;
        c1 = Cc;
        c2 = 1.0 / 24.0 - t2 / 720.0 + t2 * t2 / 40320.0;
        c3 = 1.0 / 120.0 - t2 / 2520.0 + t2 * t2 / 120960.0;
    } else {
        B = (1 - cos(th)) / t2;
        Cc = (th - sin(th)) / (t2 * th);
        c1 = Cc;
        c2 = (t2 + 2 * cos(th) - 2) / (2 * t2 * t2);
        c3 = (2 * th - 3 * sin(th) + th * cos(th)) / (2 * t2 * t2 * th);
    }
    double K[9] = {0, -phi[2], phi[1], phi[2], 0, -phi[0], -phi[1], phi[0], 0};
    double P[9] = {0, -rho[2], rho[1], rho[2], 0, -rho[0], -rho[1], rho[0], 0};
    double KK[9], KP[9], PK[9], KPK[9], KKP[9], PKK[9], KPKK[9], KKPK[9];
    matmul3(K, K, KK);
    matmul3(K, P, KP);
    matmul3(P, K, PK);
    matmul3(KP, K, KPK);
    matmul3(KK, P, KKP);
    matmul3(P, KK, PKK);
    matmul3(KPK, K, KPKK);
    matmul3(K, KPK, KKPK);
    memset(J, 0, sizeof(double) * 36);
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            int i = 3 * r + c;
            double V = (r == c ? 1.0 : 0.0) + B * K[i] + Cc * KK[i];
            double Q = 0.5 * P[i] + c1 * (KP[i] + PK[i] + KPK[i]) + c2 * (KKP[i] + PKK[i] - 3 * KPK[i])
                     + c3 * (KPKK[i] + KKPK[i]);
            J[6 * r + c] = V;
            J[6 * (r + 3) + (c + 3)] = V;
            J[6 * r + (c + 3)] = Q;
        }
}

/* The float32 error model behind the ambiguity flags, for the tests that
 * check an implementation against it: U32, ERR_DF, ERR_RATIO, ERR_ROUND,
 * ERR_CONIC, ERR_OPAC, ERR_SIGMA, ERR_EXP (in that order). */
void orc_error_model(double *c)
{
    c[0] = U32; c[1] = ERR_DF; c[2] = ERR_RATIO; c[3] = ERR_ROUND;
    c[4] = ERR_CONIC; c[5] = ERR_OPAC; c[6] = ERR_SIGMA; c[7] = ERR_EXP;
}

/* number of OpenMP threads the oracle uses (1 without OpenMP) */
int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Thread count of the OpenMP loops (timing runs: 1 for the single-thread
 * baseline); n <= 0 leaves it unchanged. */
void orc_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
