/*
 * FP64 CPU oracle of the differentiable 3DGS mapping step (RMGS-SLAM, §III-C).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or load this file;
 * it exists so the tests, the smoke check and the bench's CPU baseline can compare the
 * CUDA path against a plain, slow, obviously correct restatement of what the step
 * computes.  It shares no source with the CUDA library.
 *
 * What the step computes (each function below cites its passage):
 *   or_project           per-Gaussian EWA projection and SH colour ("standard differentiable
 *                        Gaussian splatting", §III-C; tile-based rasterizer of §II-A)
 *   or_render            brute-force front-to-back compositing of colour and of depth with
 *                        the same weights (§III-C, depth equation D = sum z_i T_i alpha_i);
 *                        no tiles: every visible Gaussian is tested at every pixel
 *   or_l1_loss           the photometric and depth L1 terms (§III-C, loss equations)
 *   or_render_backward   adjoint of or_render, reverse sweep over stored per-fragment state
 *   or_project_backward  chain rule from screen-space gradients to the Gaussian parameters
 *                        and to a left-multiplied SE(3) twist of the camera pose
 *   or_adam              masked ("visible and unfrozen", §III-C) Adam step
 *   or_bin_view / or_sort_pairs / or_tile_ranges
 *                        (tile, depth) keys, stable sort and per-tile ranges
 *
 * Readings where the paper is silent (the same defaults as the library):
 *   alpha = min(alpha_max, o * exp(-q/2)); fragments with alpha < alpha_min are skipped;
 *   if T*(1-alpha) < T_min the fragment is not added and the pixel stops.  Pixel (x, y) is
 *   sampled at (x+0.5, y+0.5).  The 2-D covariance gets `dilation` on its diagonal.  x/z and
 *   y/z inside the Jacobian are clamped to +-clamp_fov * (W/2)/fx (resp. H, fy).  A
 *   Gaussian is culled when z <= near_z, det <= 0 or o < alpha_min.  Its screen box has
 *   half-extents ceil(sqrt(tau Sigma'_xx)), ceil(sqrt(tau Sigma'_yy)), tau = 2 ln(o/alpha_min):
 *   the bounding box of the ellipse outside which alpha < alpha_min.
 *   rgb = max(0, sum_k sh_k Y_k(dir) + 0.5) with dir = normalize(mu - camera centre).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int32_t width, height;
    double fx, fy, cx, cy;
    double R[9]; /* world -> camera rotation, row-major */
    double t[3];
} or_camera;

typedef struct {
    double near_z, dilation, alpha_min, alpha_max, T_min, clamp_fov;
    double bg[3];
} or_opts;

/* Per-Gaussian projection results for one view (arrays of length n). */
typedef struct {
    int32_t *visible;  /* 1 if not culled (radius > 0) */
    double *u, *v, *z; /* pixel-space centre and camera depth */
    double *cov2d;     /* [3n] (a, b, c) of the dilated 2x2 covariance */
    double *conic;     /* [3n] inverse of cov2d, (A, B, C) */
    double *opacity;   /* sigmoid(logit) */
    double *rgb;       /* [3n] */
    int32_t *rx, *ry;  /* half-extents (px) of the alpha >= alpha_min box, 0 if culled */
    int32_t *fragile;  /* 1 if a cull decision lies within a relative 1e-5 of its threshold */
    float *zkey;       /* FP32 depth key that orders the compositing (see depth_key) */
} or_proj;

/* ------------------------------------------------------------------------------------ */
/* Real spherical harmonics up to degree 3 (orthonormal on the unit sphere, with the     */
/* Condon-Shortley phase).  The constants are the normalisations of the real SH          */
/* polynomials, computed here from their closed forms.                                   */
/* ------------------------------------------------------------------------------------ */
static void sh_consts(double c[10]) {
    const double pi = 3.14159265358979323846;
    c[0] = 0.5 * sqrt(1.0 / pi);          /* Y00 */
    c[1] = sqrt(3.0 / (4.0 * pi));        /* degree 1 */
    c[2] = 0.5 * sqrt(15.0 / pi);         /* xy, yz, xz */
    c[3] = 0.25 * sqrt(5.0 / pi);         /* 3z^2 - 1 */
    c[4] = 0.25 * sqrt(15.0 / pi);        /* x^2 - y^2 */
    c[5] = 0.25 * sqrt(35.0 / (2 * pi));  /* y(3x^2-y^2), x(x^2-3y^2) */
    c[6] = 0.5 * sqrt(105.0 / pi);        /* xyz */
    c[7] = 0.25 * sqrt(21.0 / (2 * pi));  /* y(5z^2-1), x(5z^2-1) */
    c[8] = 0.25 * sqrt(7.0 / pi);         /* z(5z^2-3) */
    c[9] = 0.25 * sqrt(105.0 / pi);       /* z(x^2-y^2) */
}

/* Y_k(d) for k < (deg+1)^2 and, if grad != NULL, dY_k/dd (as polynomials in x, y, z,
 * i.e. before any normalisation of d). */
void or_sh_basis(int deg, const double d[3], double *Y, double *grad) {
    double c[10];
    sh_consts(c);
    const double x = d[0], y = d[1], z = d[2];
    double g[16][3];
    memset(g, 0, sizeof(g));
    Y[0] = c[0];
    if (deg >= 1) {
        Y[1] = -c[1] * y;  g[1][1] = -c[1];
        Y[2] = c[1] * z;   g[2][2] = c[1];
        Y[3] = -c[1] * x;  g[3][0] = -c[1];
    }
    if (deg >= 2) {
        Y[4] = c[2] * x * y;                    g[4][0] = c[2] * y; g[4][1] = c[2] * x;
        Y[5] = -c[2] * y * z;                   g[5][1] = -c[2] * z; g[5][2] = -c[2] * y;
        Y[6] = c[3] * (2 * z * z - x * x - y * y);
        g[6][0] = -2 * c[3] * x; g[6][1] = -2 * c[3] * y; g[6][2] = 4 * c[3] * z;
        Y[7] = -c[2] * x * z;                   g[7][0] = -c[2] * z; g[7][2] = -c[2] * x;
        Y[8] = c[4] * (x * x - y * y);          g[8][0] = 2 * c[4] * x; g[8][1] = -2 * c[4] * y;
    }
    if (deg >= 3) {
        Y[9] = -c[5] * y * (3 * x * x - y * y);
        g[9][0] = -6 * c[5] * x * y; g[9][1] = -c[5] * (3 * x * x - 3 * y * y);
        Y[10] = c[6] * x * y * z;
        g[10][0] = c[6] * y * z; g[10][1] = c[6] * x * z; g[10][2] = c[6] * x * y;
        Y[11] = -c[7] * y * (4 * z * z - x * x - y * y);
        g[11][0] = 2 * c[7] * x * y; g[11][1] = -c[7] * (4 * z * z - x * x - 3 * y * y);
        g[11][2] = -8 * c[7] * y * z;
        Y[12] = c[8] * z * (2 * z * z - 3 * x * x - 3 * y * y);
        g[12][0] = -6 * c[8] * x * z; g[12][1] = -6 * c[8] * y * z;
        g[12][2] = c[8] * (6 * z * z - 3 * x * x - 3 * y * y);
        Y[13] = -c[7] * x * (4 * z * z - x * x - y * y);
        g[13][0] = -c[7] * (4 * z * z - 3 * x * x - y * y); g[13][1] = 2 * c[7] * x * y;
        g[13][2] = -8 * c[7] * x * z;
        Y[14] = c[9] * z * (x * x - y * y);
        g[14][0] = 2 * c[9] * x * z; g[14][1] = -2 * c[9] * y * z; g[14][2] = c[9] * (x * x - y * y);
        Y[15] = -c[5] * x * (x * x - 3 * y * y);
        g[15][0] = -c[5] * (3 * x * x - 3 * y * y); g[15][1] = 6 * c[5] * x * y;
    }
    if (grad) {
        int K = (deg + 1) * (deg + 1);
        for (int k = 0; k < K; k++)
            for (int j = 0; j < 3; j++) grad[3 * k + j] = g[k][j];
    }
}

/* ------------------------------------------------------------------------------------ */
/* Small dense helpers (row-major).                                                       */
/* ------------------------------------------------------------------------------------ */
static void matmul(const double *A, const double *B, double *C, int m, int k, int n) {
    for (int i = 0; i < m; i++)
        for (int j = 0; j < n; j++) {
            double s = 0;
            for (int l = 0; l < k; l++) s += A[i * k + l] * B[l * n + j];
            C[i * n + j] = s;
        }
}
static void transpose(const double *A, double *At, int m, int n) {
    for (int i = 0; i < m; i++)
        for (int j = 0; j < n; j++) At[j * m + i] = A[i * n + j];
}

/* Rotation matrix of a unit quaternion (w, x, y, z). */
static void quat_to_rot(const double q[4], double R[9]) {
    const double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

/* dR_ij/dq_k for the formula above, dR[k][9]. */
static void quat_to_rot_grad(const double q[4], double dR[4][9]) {
    const double w = q[0], x = q[1], y = q[2], z = q[3];
    double d[4][9] = {
        /* d/dw */ {0, -2 * z, 2 * y, 2 * z, 0, -2 * x, -2 * y, 2 * x, 0},
        /* d/dx */ {0, 2 * y, 2 * z, 2 * y, -4 * x, -2 * w, 2 * z, 2 * w, -4 * x},
        /* d/dy */ {-4 * y, 2 * x, 2 * w, 2 * x, 0, 2 * z, -2 * w, 2 * z, -4 * y},
        /* d/dz */ {-4 * z, -2 * w, 2 * x, 2 * w, -4 * z, 2 * y, 2 * x, 2 * y, 0}};
    memcpy(dR, d, sizeof(d));
}

/* Everything the forward projection of one Gaussian in one view computes. */
typedef struct {
    int culled;
    int fragile;
    double qn[4], qnorm;   /* normalised quaternion and the raw norm */
    double Rq[9], s[3];    /* rotation and scales */
    double M[9];           /* Rq * diag(s) */
    double Sigma[9];       /* world covariance */
    double pc[3];          /* camera-frame centre */
    float zkey;            /* FP32 depth key (depth_key) */
    double tx, ty;         /* clamped x/z, y/z */
    int clx, cly;          /* 1 if clamped */
    double J[6];           /* 2x3 */
    double Tm[6];          /* J * W */
    double cov[4];         /* 2x2 dilated covariance */
    double det;
    double conic[3];
    double o;
    double u, v;
    double dirraw[3], dnorm, dir[3];
    double Y[16], rgb_pre[3], rgb[3];
    int rgb_clamped[3];
    double tau;            /* 2 ln(o / alpha_min): alpha >= alpha_min  <=>  d^T conic d <= tau */
    int32_t rx, ry;
} proj1;

/* The front-to-back order of the compositing (§III-C; ties and precision are not stated by
 * the paper).  Reading: Gaussians are ordered by the IEEE single-precision camera depth
 *   z32 = fma(R22, mu_z, fma(R21, mu_y, R20 * mu_x)) + t_z
 * with every operation rounded to FP32 (fmaf rounds once), taken on the FP32 values of the
 * pose (third row of R_cw, t_cw) and of the mean, and equal keys in ascending Gaussian index.  The order is an integer decision made from floating point, so
 * it is fixed in the precision of the FP32 step, exactly, with this operation order; the
 * continuous quantities (the depth D, the weights) stay in double. */
static float depth_key(const double *W, const double *t, const double *mu) {
    const float r20 = (float)W[6], r21 = (float)W[7], r22 = (float)W[8], tz = (float)t[2];
    const float m0 = (float)mu[0], m1 = (float)mu[1], m2 = (float)mu[2];
    const float p = r20 * m0;                 /* rounded product (no contraction: -ffp-contract=off) */
    const float s = fmaf(r22, m2, fmaf(r21, m1, p));
    return s + tz;
}

static void project_one(const double *mu, const double *ls, const double *q, double logit,
                        const double *shc /* [K][3] */, int deg, const or_camera *cam,
                        const or_opts *opt, proj1 *P) {
    memset(P, 0, sizeof(*P));
    const double *W = cam->R;
    /* camera centre c_w = -R^T t */
    double cw[3];
    for (int i = 0; i < 3; i++) cw[i] = -(W[0 * 3 + i] * cam->t[0] + W[1 * 3 + i] * cam->t[1] + W[2 * 3 + i] * cam->t[2]);
    /* camera-frame centre */
    for (int i = 0; i < 3; i++) P->pc[i] = W[i * 3 + 0] * mu[0] + W[i * 3 + 1] * mu[1] + W[i * 3 + 2] * mu[2] + cam->t[i];
    P->zkey = depth_key(W, cam->t, mu);
    const double x = P->pc[0], y = P->pc[1], z = P->pc[2];
    if (fabs(z - opt->near_z) <= 1e-5 * fabs(opt->near_z) + 1e-12) P->fragile = 1;
    if (!(z > opt->near_z)) { P->culled = 1; return; }
    /* rotation and scale */
    P->qnorm = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    for (int i = 0; i < 4; i++) P->qn[i] = q[i] / P->qnorm;
    quat_to_rot(P->qn, P->Rq);
    for (int i = 0; i < 3; i++) P->s[i] = exp(ls[i]);
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) P->M[i * 3 + j] = P->Rq[i * 3 + j] * P->s[j];
    double Mt[9];
    transpose(P->M, Mt, 3, 3);
    matmul(P->M, Mt, P->Sigma, 3, 3, 3);
    /* Jacobian of the perspective map with clamped x/z, y/z */
    const double limx = opt->clamp_fov * (0.5 * cam->width) / cam->fx;
    const double limy = opt->clamp_fov * (0.5 * cam->height) / cam->fy;
    double rx = x / z, ry = y / z;
    P->tx = rx; P->ty = ry;
    if (rx < -limx) { P->tx = -limx; P->clx = 1; }
    if (rx > limx) { P->tx = limx; P->clx = 1; }
    if (ry < -limy) { P->ty = -limy; P->cly = 1; }
    if (ry > limy) { P->ty = limy; P->cly = 1; }
    P->J[0] = cam->fx / z; P->J[1] = 0; P->J[2] = -cam->fx * P->tx / z;
    P->J[3] = 0; P->J[4] = cam->fy / z; P->J[5] = -cam->fy * P->ty / z;
    matmul(P->J, W, P->Tm, 2, 3, 3);
    double TS[6], Tt[6], cov[4];
    matmul(P->Tm, P->Sigma, TS, 2, 3, 3);
    transpose(P->Tm, Tt, 2, 3);
    matmul(TS, Tt, cov, 2, 3, 2);
    cov[0] += opt->dilation;
    cov[3] += opt->dilation;
    cov[1] = cov[2] = 0.5 * (cov[1] + cov[2]);
    memcpy(P->cov, cov, sizeof(cov));
    P->det = cov[0] * cov[3] - cov[1] * cov[1];
    if (!(P->det > 0)) { P->culled = 1; return; }
    P->conic[0] = cov[3] / P->det;
    P->conic[1] = -cov[1] / P->det;
    P->conic[2] = cov[0] / P->det;
    /* opacity */
    P->o = 1.0 / (1.0 + exp(-logit));
    if (fabs(P->o - opt->alpha_min) <= 1e-5 * opt->alpha_min) P->fragile = 1;
    if (P->o < opt->alpha_min) { P->culled = 1; return; }
    /* alpha >= alpha_min only inside the ellipse d^T conic d <= tau; its bounding box has
     * half-extents sqrt(tau * cov_xx) and sqrt(tau * cov_yy) (support function of an ellipse) */
    P->tau = 2.0 * log(P->o / opt->alpha_min);
    P->rx = (int32_t)ceil(sqrt(P->tau * cov[0]));
    P->ry = (int32_t)ceil(sqrt(P->tau * cov[3]));
    if (P->rx <= 0 || P->ry <= 0) { P->culled = 1; return; }
    P->u = cam->fx * x / z + cam->cx;
    P->v = cam->fy * y / z + cam->cy;
    /* SH colour along the viewing direction */
    for (int i = 0; i < 3; i++) P->dirraw[i] = mu[i] - cw[i];
    P->dnorm = sqrt(P->dirraw[0] * P->dirraw[0] + P->dirraw[1] * P->dirraw[1] + P->dirraw[2] * P->dirraw[2]);
    for (int i = 0; i < 3; i++) P->dir[i] = P->dirraw[i] / P->dnorm;
    or_sh_basis(deg, P->dir, P->Y, NULL);
    const int K = (deg + 1) * (deg + 1);
    for (int c = 0; c < 3; c++) {
        double s = 0;
        for (int k = 0; k < K; k++) s += shc[k * 3 + c] * P->Y[k];
        P->rgb_pre[c] = s + 0.5;
        P->rgb_clamped[c] = P->rgb_pre[c] < 0;
        P->rgb[c] = P->rgb_clamped[c] ? 0.0 : P->rgb_pre[c];
    }
}

/* Gather one Gaussian's parameters from the SoA planes. */
static void gather(int64_t i, int64_t n, int deg, const double *means, const double *ls,
                   const double *quats, const double *logits, const double *sh, double mu[3],
                   double s[3], double q[4], double *lg, double shc[48]) {
    for (int k = 0; k < 3; k++) { mu[k] = means[k * n + i]; s[k] = ls[k * n + i]; }
    for (int k = 0; k < 4; k++) q[k] = quats[k * n + i];
    *lg = logits[i];
    const int K = (deg + 1) * (deg + 1);
    for (int k = 0; k < 3 * K; k++) shc[k] = sh[k * n + i];
}

/* Forward projection of all n Gaussians into one view. */
void or_project(int64_t n, int deg, const double *means, const double *log_scales,
                const double *quats, const double *logits, const double *sh,
                const or_camera *cam, const or_opts *opt, or_proj *out) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        double mu[3], s[3], q[4], lg, shc[48];
        gather(i, n, deg, means, log_scales, quats, logits, sh, mu, s, q, &lg, shc);
        proj1 P;
        project_one(mu, s, q, lg, shc, deg, cam, opt, &P);
        out->fragile[i] = P.fragile;
        out->visible[i] = !P.culled;
        out->rx[i] = P.culled ? 0 : P.rx;
        out->ry[i] = P.culled ? 0 : P.ry;
        out->u[i] = P.u; out->v[i] = P.v; out->z[i] = P.pc[2];
        out->zkey[i] = P.zkey;
        out->opacity[i] = P.o;
        for (int k = 0; k < 3; k++) {
            out->conic[3 * i + k] = P.culled ? 0 : P.conic[k];
            out->rgb[3 * i + k] = P.rgb[k];
        }
        out->cov2d[3 * i + 0] = P.cov[0];
        out->cov2d[3 * i + 1] = P.cov[1];
        out->cov2d[3 * i + 2] = P.cov[3];
    }
}

/* ------------------------------------------------------------------------------------ */
/* Brute-force compositing.                                                              */
/* ------------------------------------------------------------------------------------ */
typedef struct { float z; int64_t id; } zid;
static int cmp_zid(const void *a, const void *b) {
    const zid *x = (const zid *)a, *y = (const zid *)b;
    if (x->z < y->z) return -1;
    if (x->z > y->z) return 1;
    return (x->id > y->id) - (x->id < y->id);
}

/* Visible Gaussians in front-to-back order: ascending FP32 depth key (depth_key), equal keys
 * by ascending index. */
static int64_t depth_order(int64_t n, const or_proj *pr, int64_t *order) {
    zid *tmp = (zid *)malloc(sizeof(zid) * (size_t)(n > 0 ? n : 1));
    int64_t m = 0;
    for (int64_t i = 0; i < n; i++)
        if (pr->visible[i]) { tmp[m].z = pr->zkey[i]; tmp[m].id = i; m++; }
    qsort(tmp, (size_t)m, sizeof(zid), cmp_zid);
    for (int64_t k = 0; k < m; k++) order[k] = tmp[k].id;
    free(tmp);
    return m;
}

static double frag_alpha(const or_proj *pr, int64_t g, double px, double py, const or_opts *opt,
                         double *G_out, double *dx_out, double *dy_out, double *a0_out) {
    const double dx = px - pr->u[g], dy = py - pr->v[g];
    const double A = pr->conic[3 * g], B = pr->conic[3 * g + 1], C = pr->conic[3 * g + 2];
    const double q = A * dx * dx + 2.0 * B * dx * dy + C * dy * dy;
    const double G = exp(-0.5 * q);
    const double a0 = pr->opacity[g] * G;
    if (G_out) *G_out = G;
    if (dx_out) *dx_out = dx;
    if (dy_out) *dy_out = dy;
    if (a0_out) *a0_out = a0;
    return a0 < opt->alpha_max ? a0 : opt->alpha_max;
}

/* Per pixel: C = sum_i c_i alpha_i T_i + T_final bg, D = sum_i z_i alpha_i T_i,
 * T_final, the number of added fragments, and a fragility flag: 1 if a decision taken at
 * this pixel (alpha vs alpha_min, T(1-alpha) vs T_min, alpha vs the alpha_max clamp, a cull
 * decision of an added Gaussian) lies within a relative `margin` of its threshold, so that a
 * correct FP32 implementation may take the other branch.  The depth order is no such
 * decision: it is defined exactly on the FP32 key (depth_key).  Gaussians whose screen box (half-extents rx, ry) does not contain the pixel
 * centre are skipped: outside the box alpha < alpha_min by construction (tested). */
void or_render(int64_t n, const or_proj *pr, const or_camera *cam, const or_opts *opt,
               double margin, int use_square, double *C, double *D, double *T_out,
               int32_t *n_frag, int32_t *fragile_px) {
    const int W = cam->width, H = cam->height;
    int64_t *order = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    const int64_t m = depth_order(n, pr, order);
#pragma omp parallel for schedule(dynamic, 1)
    for (int py = 0; py < H; py++) {
        for (int px = 0; px < W; px++) {
            const double cx = px + 0.5, cy = py + 0.5;
            double T = 1.0, c[3] = {0, 0, 0}, d = 0;
            int cnt = 0, fr = 0;
            for (int64_t k = 0; k < m; k++) {
                const int64_t g = order[k];
                if (use_square) {
                    if (fabs(cx - pr->u[g]) > pr->rx[g] + 1e-9 || fabs(cy - pr->v[g]) > pr->ry[g] + 1e-9) continue;
                }
                double a0;
                const double a = frag_alpha(pr, g, cx, cy, opt, NULL, NULL, NULL, &a0);
                if (fabs(a - opt->alpha_min) <= margin * opt->alpha_min) fr = 1;
                if (fabs(a0 - opt->alpha_max) <= margin * opt->alpha_max) fr = 1;
                if (a < opt->alpha_min) continue;
                const double test_T = T * (1.0 - a);
                if (fabs(test_T - opt->T_min) <= margin * opt->T_min) fr = 1;
                if (test_T < opt->T_min) break;
                if (pr->fragile[g]) fr = 1;
                const double w = a * T;
                for (int ch = 0; ch < 3; ch++) c[ch] += w * pr->rgb[3 * g + ch];
                d += w * pr->z[g];
                T = test_T;
                cnt++;
            }
            const int64_t p = (int64_t)py * W + px;
            for (int ch = 0; ch < 3; ch++) C[(int64_t)ch * W * H + p] = c[ch] + T * opt->bg[ch];
            D[p] = d;
            T_out[p] = T;
            n_frag[p] = cnt;
            fragile_px[p] = fr;
        }
    }
    free(order);
}

/* L1 photometric + depth loss of one view (§III-C):
 *   L = lambda_rgb / |M| * sum_{x in M} sum_ch |C - C~| + lambda_depth / |M_D| * sum_{x in M_D} |D - D~|
 * with M the caller's mask and M_D = M intersected with {D~ > 0} (pixels with a depth
 * reference).  Everything is multiplied by `scale` (1/V when views are averaged).  The
 * sub-gradient uses sign(0) = 0.  Returns the loss; fills dL/dC and dL/dD. */
double or_l1_loss(int W, int H, const double *C, const double *D, const double *tC,
                  const double *tD, const uint8_t *mask, double lambda_rgb, double lambda_depth,
                  double scale, double *gC, double *gD) {
    const int64_t P = (int64_t)W * H;
    int64_t nm = 0, nd = 0;
    for (int64_t p = 0; p < P; p++) {
        if (mask[p]) { nm++; if (tD[p] > 0) nd++; }
    }
    double srgb = 0, sd = 0;
    const double krgb = nm ? lambda_rgb * scale / (double)nm : 0.0;
    const double kd = nd ? lambda_depth * scale / (double)nd : 0.0;
    for (int64_t p = 0; p < P; p++) {
        for (int ch = 0; ch < 3; ch++) {
            const double r = C[ch * P + p] - tC[ch * P + p];
            const double sg = mask[p] ? (double)((r > 0) - (r < 0)) : 0.0;
            if (mask[p]) srgb += fabs(r);
            gC[ch * P + p] = krgb * sg;
        }
        const double r = D[p] - tD[p];
        const int in = mask[p] && tD[p] > 0;
        if (in) sd += fabs(r);
        gD[p] = in ? kd * (double)((r > 0) - (r < 0)) : 0.0;
    }
    return srgb * krgb + sd * kd;
}

/* ------------------------------------------------------------------------------------ */
/* Backward of compositing: stored-state reverse sweep.                                  */
/* Output per Gaussian g (g2d[10*g + ...]):                                              */
/*   0,1 dL/du, dL/dv   2,3,4 dL/dA, dL/dB, dL/dC of the conic (B = stored off-diagonal, */
/*   appearing twice in the quadratic form)   5 dL/do   6,7,8 dL/drgb   9 dL/dz          */
/* ------------------------------------------------------------------------------------ */
typedef struct { int64_t g; double a, a0, G, T, dx, dy; } frag;

void or_render_backward(int64_t n, const or_proj *pr, const or_camera *cam, const or_opts *opt,
                        int use_square, const double *gC, const double *gD, double *g2d) {
    const int W = cam->width, H = cam->height;
    const int64_t P = (int64_t)W * H;
    int64_t *order = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    const int64_t m = depth_order(n, pr, order);
    memset(g2d, 0, sizeof(double) * 10 * (size_t)n);
    int nthreads = 1;
#ifdef _OPENMP
    nthreads = omp_get_max_threads();
#endif
    /* per-thread accumulators, summed at the end */
    double *acc = (double *)calloc((size_t)nthreads * 10 * (size_t)n, sizeof(double));
#pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *my = acc + (size_t)tid * 10 * (size_t)n;
        frag *list = (frag *)malloc(sizeof(frag) * (size_t)(m > 0 ? m : 1));
#pragma omp for schedule(dynamic, 1)
        for (int py = 0; py < H; py++) {
            for (int px = 0; px < W; px++) {
                const int64_t p = (int64_t)py * W + px;
                const double gc[3] = {gC[p], gC[P + p], gC[2 * P + p]}, gd = gD[p];
                if (gc[0] == 0 && gc[1] == 0 && gc[2] == 0 && gd == 0) continue;
                const double cx = px + 0.5, cy = py + 0.5;
                /* forward again, storing every added fragment */
                double T = 1.0;
                int64_t cnt = 0;
                for (int64_t k = 0; k < m; k++) {
                    const int64_t g = order[k];
                    if (use_square) {
                        if (fabs(cx - pr->u[g]) > pr->rx[g] + 1e-9 || fabs(cy - pr->v[g]) > pr->ry[g] + 1e-9) continue;
                    }
                    double G, dx, dy, a0;
                    const double a = frag_alpha(pr, g, cx, cy, opt, &G, &dx, &dy, &a0);
                    if (a < opt->alpha_min) continue;
                    const double test_T = T * (1.0 - a);
                    if (test_T < opt->T_min) break;
                    list[cnt].g = g; list[cnt].a = a; list[cnt].a0 = a0; list[cnt].G = G;
                    list[cnt].T = T; list[cnt].dx = dx; list[cnt].dy = dy;
                    cnt++;
                    T = test_T;
                }
                /* reverse sweep: S = sum over later fragments of c_j w_j, plus T_final bg */
                double S[3] = {T * opt->bg[0], T * opt->bg[1], T * opt->bg[2]}, SD = 0;
                for (int64_t k = cnt - 1; k >= 0; k--) {
                    const frag *f = &list[k];
                    const int64_t g = f->g;
                    const double w = f->a * f->T;
                    const double *c = &pr->rgb[3 * g];
                    const double zg = pr->z[g];
                    double dLda = 0;
                    for (int ch = 0; ch < 3; ch++) {
                        my[10 * g + 6 + ch] += gc[ch] * w;
                        dLda += gc[ch] * (c[ch] * f->T - S[ch] / (1.0 - f->a));
                    }
                    my[10 * g + 9] += gd * w;
                    dLda += gd * (zg * f->T - SD / (1.0 - f->a));
                    for (int ch = 0; ch < 3; ch++) S[ch] += c[ch] * w;
                    SD += zg * w;
                    if (f->a0 < opt->alpha_max) {
                        const double o = pr->opacity[g];
                        my[10 * g + 5] += dLda * f->G;
                        const double dLdG = dLda * o;
                        const double dLdq = -0.5 * f->G * dLdG;
                        const double A = pr->conic[3 * g], B = pr->conic[3 * g + 1], Cc = pr->conic[3 * g + 2];
                        my[10 * g + 2] += dLdq * f->dx * f->dx;
                        my[10 * g + 3] += dLdq * 2.0 * f->dx * f->dy;
                        my[10 * g + 4] += dLdq * f->dy * f->dy;
                        /* q depends on the centre through d = pixel - centre */
                        my[10 * g + 0] += dLdq * (-2.0) * (A * f->dx + B * f->dy);
                        my[10 * g + 1] += dLdq * (-2.0) * (B * f->dx + Cc * f->dy);
                    }
                }
            }
        }
        free(list);
    }
    for (int t = 0; t < nthreads; t++)
        for (int64_t k = 0; k < 10 * n; k++) g2d[k] += acc[(size_t)t * 10 * (size_t)n + k];
    free(acc);
    free(order);
}

/* ------------------------------------------------------------------------------------ */
/* Backward of the projection.  Parameter-gradient planes follow the parameter layout:  */
/* 0..2 means, 3..5 log-scales, 6..9 quats, 10 opacity logit, 11.. SH (k*3 + c).        */
/* Pose twist xi = (rho, phi) perturbs the camera as T_cw <- Exp(xi) T_cw.              */
/* ------------------------------------------------------------------------------------ */
static void cross3(const double a[3], const double b[3], double c[3]) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

void or_project_backward(int64_t n, int deg, const double *means, const double *log_scales,
                         const double *quats, const double *logits, const double *sh,
                         const or_camera *cam, const or_opts *opt, const double *g2d,
                         double *grads, double *twist) {
    const int K = (deg + 1) * (deg + 1);
    const double *W = cam->R;
    double tw[6] = {0, 0, 0, 0, 0, 0};
#pragma omp parallel
    {
        double twl[6] = {0, 0, 0, 0, 0, 0};
#pragma omp for schedule(static)
        for (int64_t i = 0; i < n; i++) {
            double mu[3], s[3], q[4], lg, shc[48];
            gather(i, n, deg, means, log_scales, quats, logits, sh, mu, s, q, &lg, shc);
            proj1 P;
            project_one(mu, s, q, lg, shc, deg, cam, opt, &P);
            if (P.culled) continue;
            const double *gg = &g2d[10 * i];
            const double gu = gg[0], gv = gg[1], gA = gg[2], gB = gg[3], gC = gg[4];
            const double go = gg[5], grgb[3] = {gg[6], gg[7], gg[8]}, gzd = gg[9];
            double g_mu[3] = {0, 0, 0}, g_pc[3] = {0, 0, 0};
            /* conic = inverse(cov): cov = [[a, b], [b, c]], conic = [c, -b, a] / det */
            const double a = P.cov[0], b = P.cov[1], c = P.cov[3], det = P.det, d2 = det * det;
            const double ga = (-c * c * gA + b * c * gB - b * b * gC) / d2;
            const double gb = (2 * b * c * gA - (a * c + b * b) * gB + 2 * a * b * gC) / d2;
            const double gc = (-b * b * gA + a * b * gB - a * a * gC) / d2;
            /* symmetric gradient of cov (= T Sigma T^T + dil I) */
            const double Gc[4] = {ga, 0.5 * gb, 0.5 * gb, gc};
            /* g_T = 2 Gc T Sigma ; g_Sigma = T^T Gc T */
            double TS[6], gT[6], GcT[6], Tt[6], gSig[9];
            matmul(P.Tm, P.Sigma, TS, 2, 3, 3);
            matmul(Gc, TS, gT, 2, 2, 3);
            for (int k = 0; k < 6; k++) gT[k] *= 2.0;
            matmul(Gc, P.Tm, GcT, 2, 2, 3);
            transpose(P.Tm, Tt, 2, 3);
            matmul(Tt, GcT, gSig, 3, 2, 3);
            /* T = J W : g_J = g_T W^T, g_W = J^T g_T */
            double Wt[9], gJ[6], Jt[6], gW[9];
            transpose(W, Wt, 3, 3);
            matmul(gT, Wt, gJ, 2, 3, 3);
            transpose(P.J, Jt, 2, 3);
            matmul(Jt, gT, gW, 3, 2, 3);
            /* J(x, y, z) */
            const double x = P.pc[0], y = P.pc[1], z = P.pc[2];
            const double fx = cam->fx, fy = cam->fy;
            const double dtx_dx = P.clx ? 0 : 1.0 / z, dtx_dz = P.clx ? 0 : -x / (z * z);
            const double dty_dy = P.cly ? 0 : 1.0 / z, dty_dz = P.cly ? 0 : -y / (z * z);
            g_pc[2] += gJ[0] * (-fx / (z * z)) + gJ[4] * (-fy / (z * z));
            g_pc[2] += gJ[2] * (fx * P.tx / (z * z) - fx / z * dtx_dz);
            g_pc[0] += gJ[2] * (-fx / z * dtx_dx);
            g_pc[2] += gJ[5] * (fy * P.ty / (z * z) - fy / z * dty_dz);
            g_pc[1] += gJ[5] * (-fy / z * dty_dy);
            /* pixel centre */
            g_pc[0] += gu * fx / z;
            g_pc[1] += gv * fy / z;
            g_pc[2] += -gu * fx * x / (z * z) - gv * fy * y / (z * z);
            /* compositing depth */
            g_pc[2] += gzd;
            /* p_c = W mu + t */
            for (int k = 0; k < 3; k++) g_mu[k] += W[0 * 3 + k] * g_pc[0] + W[1 * 3 + k] * g_pc[1] + W[2 * 3 + k] * g_pc[2];
            /* pose: p_c(xi) = Exp(phi) p_c + rho ; W(phi) = Exp(phi) W */
            double cr[3];
            cross3(P.pc, g_pc, cr);
            for (int k = 0; k < 3; k++) { twl[k] += g_pc[k]; twl[3 + k] += cr[k]; }
            double Am[9];
            matmul(gW, Wt, Am, 3, 3, 3);
            twl[3] += Am[7] - Am[5];
            twl[4] += Am[2] - Am[6];
            twl[5] += Am[3] - Am[1];
            /* Sigma = M M^T, M = Rq diag(s) */
            double gM[9], gRq[9];
            matmul(gSig, P.M, gM, 3, 3, 3);
            for (int k = 0; k < 9; k++) gM[k] *= 2.0;
            for (int r = 0; r < 3; r++)
                for (int cc = 0; cc < 3; cc++) gRq[r * 3 + cc] = gM[r * 3 + cc] * P.s[cc];
            double gls[3];
            for (int k = 0; k < 3; k++) {
                double sdot = 0;
                for (int r = 0; r < 3; r++) sdot += P.Rq[r * 3 + k] * gM[r * 3 + k];
                gls[k] = sdot * P.s[k];
            }
            double dR[4][9], gqn[4], gq[4];
            quat_to_rot_grad(P.qn, dR);
            for (int k = 0; k < 4; k++) {
                gqn[k] = 0;
                for (int e = 0; e < 9; e++) gqn[k] += gRq[e] * dR[k][e];
            }
            double dotq = 0;
            for (int k = 0; k < 4; k++) dotq += P.qn[k] * gqn[k];
            for (int k = 0; k < 4; k++) gq[k] = (gqn[k] - P.qn[k] * dotq) / P.qnorm;
            /* opacity */
            const double glogit = go * P.o * (1.0 - P.o);
            /* SH colour */
            double Ygrad[48];
            double Y[16];
            or_sh_basis(deg, P.dir, Y, Ygrad);
            double gdir[3] = {0, 0, 0};
            double gsh[48];
            memset(gsh, 0, sizeof(gsh));
            for (int ch = 0; ch < 3; ch++) {
                if (P.rgb_clamped[ch]) continue;
                for (int k = 0; k < K; k++) {
                    gsh[k * 3 + ch] += grgb[ch] * Y[k];
                    for (int j = 0; j < 3; j++) gdir[j] += grgb[ch] * shc[k * 3 + ch] * Ygrad[3 * k + j];
                }
            }
            double ddot = gdir[0] * P.dir[0] + gdir[1] * P.dir[1] + gdir[2] * P.dir[2];
            double gd[3];
            for (int j = 0; j < 3; j++) gd[j] = (gdir[j] - P.dir[j] * ddot) / P.dnorm;
            for (int j = 0; j < 3; j++) g_mu[j] += gd[j];
            /* the camera centre moves by -R^T rho: g_rho += R * gd */
            for (int r = 0; r < 3; r++) twl[r] += W[r * 3 + 0] * gd[0] + W[r * 3 + 1] * gd[1] + W[r * 3 + 2] * gd[2];
            /* accumulate into the planes */
            for (int k = 0; k < 3; k++) grads[(int64_t)k * n + i] += g_mu[k];
            for (int k = 0; k < 3; k++) grads[(int64_t)(3 + k) * n + i] += gls[k];
            for (int k = 0; k < 4; k++) grads[(int64_t)(6 + k) * n + i] += gq[k];
            grads[(int64_t)10 * n + i] += glogit;
            for (int k = 0; k < 3 * K; k++) grads[(int64_t)(11 + k) * n + i] += gsh[k];
        }
#pragma omp critical
        for (int k = 0; k < 6; k++) tw[k] += twl[k];
    }
    for (int k = 0; k < 6; k++) twist[k] += tw[k];
}

/* ------------------------------------------------------------------------------------ */
/* Masked Adam (§III-C: visible and unfrozen Gaussians are updated by a sparse           */
/* gradient-based optimizer).  Rows with update[i] == 0 keep p, m, v unchanged.          */
/* Plane k uses lr[group(k)], groups: means, log-scales, quats, opacity, SH DC, SH rest. */
/* ------------------------------------------------------------------------------------ */
void or_adam(int64_t n, int n_planes, double *p, const double *g, double *m, double *v,
             const uint8_t *update, const double lr[6], double b1, double b2, double eps,
             int64_t step) {
    const double bc1 = 1.0 - pow(b1, (double)step), bc2 = 1.0 - pow(b2, (double)step);
    for (int k = 0; k < n_planes; k++) {
        const int grp = k < 3 ? 0 : k < 6 ? 1 : k < 10 ? 2 : k < 11 ? 3 : k < 14 ? 4 : 5;
        for (int64_t i = 0; i < n; i++) {
            if (update && !update[i]) continue;
            const int64_t e = (int64_t)k * n + i;
            m[e] = b1 * m[e] + (1 - b1) * g[e];
            v[e] = b2 * v[e] + (1 - b2) * g[e] * g[e];
            const double mh = m[e] / bc1, vh = v[e] / bc2;
            p[e] -= lr[grp] * mh / (sqrt(vh) + eps);
        }
    }
}

/* ------------------------------------------------------------------------------------ */
/* Binning: (tile, depth) keys.  Inputs are the FP32 screen-space records; every         */
/* decision is taken in FP32 exactly as defined here, so the keys are unique bits.       */
/*   covered tiles: x in [floor((u - rx)/T), floor((u + rx)/T)] clamped to the grid,     */
/*   y likewise with ry; key = ((tile_offset + ty*tiles_x + tx) << 32) | bits(z);        */
/*   value = idx_offset + i.  Emission order is i ascending, tiles row-major.            */
/* ------------------------------------------------------------------------------------ */
static int tile_span(float c, int32_t r, int tile, int ntiles, int *lo, int *hi) {
    const float rf = (float)r;
    const float a = (c - rf) / (float)tile;
    const float b = (c + rf) / (float)tile;
    float fa = floorf(a), fb = floorf(b);
    if (!(fb >= 0.0f) || !(fa <= (float)(ntiles - 1))) return 0;
    if (fa < 0.0f) fa = 0.0f;
    if (fb > (float)(ntiles - 1)) fb = (float)(ntiles - 1);
    *lo = (int)fa;
    *hi = (int)fb;
    return *hi >= *lo;
}

int64_t or_bin_view(int64_t n, const float *u, const float *v, const float *z, const int32_t *rx,
                    const int32_t *ry, int W, int H, int tile, int64_t tile_offset, int64_t idx_offset,
                    uint64_t *keys, uint32_t *vals, uint32_t *touched) {
    const int tx_n = (W + tile - 1) / tile, ty_n = (H + tile - 1) / tile;
    int64_t P = 0;
    for (int64_t i = 0; i < n; i++) {
        int x0, x1, y0, y1;
        uint32_t cnt = 0;
        if (rx[i] > 0 && ry[i] > 0 && tile_span(u[i], rx[i], tile, tx_n, &x0, &x1) &&
            tile_span(v[i], ry[i], tile, ty_n, &y0, &y1)) {
            uint32_t zb;
            memcpy(&zb, &z[i], 4);
            for (int ty = y0; ty <= y1; ty++)
                for (int tx = x0; tx <= x1; tx++) {
                    if (keys) {
                        keys[P] = ((uint64_t)(tile_offset + (int64_t)ty * tx_n + tx) << 32) | zb;
                        vals[P] = (uint32_t)(idx_offset + i);
                    }
                    P++;
                    cnt++;
                }
        }
        if (touched) touched[i] = cnt;
    }
    return P;
}

typedef struct { uint64_t k; uint32_t v; int64_t pos; } kv;
static int cmp_kv(const void *a, const void *b) {
    const kv *x = (const kv *)a, *y = (const kv *)b;
    if (x->k != y->k) return x->k < y->k ? -1 : 1;
    return (x->pos > y->pos) - (x->pos < y->pos);
}

/* Stable sort of the pairs by key (ties keep emission order). */
void or_sort_pairs(int64_t P, uint64_t *keys, uint32_t *vals) {
    kv *t = (kv *)malloc(sizeof(kv) * (size_t)(P > 0 ? P : 1));
    for (int64_t i = 0; i < P; i++) { t[i].k = keys[i]; t[i].v = vals[i]; t[i].pos = i; }
    qsort(t, (size_t)P, sizeof(kv), cmp_kv);
    for (int64_t i = 0; i < P; i++) { keys[i] = t[i].k; vals[i] = t[i].v; }
    free(t);
}

/* ranges[2t], ranges[2t+1] = [first, last+1) of tile t in the sorted keys (0, 0 if empty). */
void or_tile_ranges(int64_t P, const uint64_t *keys, int64_t n_tiles, uint32_t *ranges) {
    memset(ranges, 0, sizeof(uint32_t) * 2 * (size_t)n_tiles);
    for (int64_t i = 0; i < P; i++) {
        const int64_t t = (int64_t)(keys[i] >> 32);
        if (i == 0 || (keys[i - 1] >> 32) != (uint64_t)t) ranges[2 * t] = (uint32_t)i;
        if (i == P - 1 || (keys[i + 1] >> 32) != (uint64_t)t) ranges[2 * t + 1] = (uint32_t)(i + 1);
    }
}
