/*
 * FP64 CPU oracle of the voxel-PCA geometric fitting (RMGS-SLAM §III-A) -- TEST
 * INFRASTRUCTURE ONLY (see gs_oracle.c).
 *
 * Points are grouped into cubic voxels of side s: the voxel of p is (floor(p_x/s),
 * floor(p_y/s), floor(p_z/s)), evaluated in FP32 on the FP32 input coordinates (the integer
 * decision is taken in the precision the GPU uses).  For every voxel with at least min_pts
 * points, in double precision:
 *   mean mu, covariance C = 1/N sum (p - mu)(p - mu)^T,
 *   eigen-decomposition by cyclic Jacobi rotations, eigenvalues sorted ascending
 *   (l_min <= l_mid <= l_max) with eigenvectors V = [v_min v_mid v_max]; each eigenvector is
 *   signed so that its largest-magnitude component is positive, then v_max = v_min x v_mid,
 *   classification (the order of §III-A): planar if l_min < tau_p (normal v_min), else linear
 *   if l_max / l_min > tau_l (direction v_max), else unreliable,
 *   descriptor covariance Sigma_g = sum_i J_i Sigma_i J_i^T with J_i = [V F_i ; I/N] and rows
 *   f_i^(m) = (p_i - mu)^T (v_m v_k^T + v_k v_m^T) / (N (l_k - l_m)) for m != k, 0 for m = k
 *   (k = min for planar, max for linear), Sigma_i = sigma^2 I (synthetic point noise),
 *   reliable iff classified, the eigenvalue gaps are not degenerate (relative gap > 1e-6) and
 *   trace(Sigma_g[0:3, 0:3]) < tau_trace.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Eigen-decomposition of a symmetric 3x3 matrix (row-major A) by cyclic Jacobi rotations.
 * On return lam[0..2] are the eigenvalues and the columns of V the eigenvectors (unsorted). */
void or_jacobi3(const double *A_in, double *lam, double *V) {
    double A[9];
    memcpy(A, A_in, sizeof(A));
    for (int i = 0; i < 9; i++) V[i] = (i % 4 == 0) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 50; sweep++) {
        const double off = A[1] * A[1] + A[2] * A[2] + A[5] * A[5];
        const double diag = A[0] * A[0] + A[4] * A[4] + A[8] * A[8];
        if (off <= 1e-30 * (diag > 0 ? diag : 1.0)) break;
        for (int p = 0; p < 2; p++) {
            for (int q = p + 1; q < 3; q++) {
                const double apq = A[p * 3 + q];
                if (apq == 0.0) continue;
                const double app = A[p * 3 + p], aqq = A[q * 3 + q];
                /* rotation angle that zeroes A[p][q] */
                const double theta = 0.5 * (aqq - app) / apq;
                const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                /* A <- J^T A J with J the rotation in the (p, q) plane */
                for (int k = 0; k < 3; k++) {
                    const double akp = A[k * 3 + p], akq = A[k * 3 + q];
                    A[k * 3 + p] = c * akp - s * akq;
                    A[k * 3 + q] = s * akp + c * akq;
                }
                for (int k = 0; k < 3; k++) {
                    const double apk = A[p * 3 + k], aqk = A[q * 3 + k];
                    A[p * 3 + k] = c * apk - s * aqk;
                    A[q * 3 + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < 3; k++) {
                    const double vkp = V[k * 3 + p], vkq = V[k * 3 + q];
                    V[k * 3 + p] = c * vkp - s * vkq;
                    V[k * 3 + q] = s * vkp + c * vkq;
                }
            }
        }
    }
    lam[0] = A[0];
    lam[1] = A[4];
    lam[2] = A[8];
}

/* Sorted, sign-canonical, right-handed eigen-decomposition (see the header comment). */
void or_eig_sorted(const double *C, double *lam, double *V) {
    double l[3], W[9];
    or_jacobi3(C, l, W);
    int idx[3] = {0, 1, 2};
    for (int i = 0; i < 3; i++)
        for (int j = i + 1; j < 3; j++)
            if (l[idx[j]] < l[idx[i]]) { int t = idx[i]; idx[i] = idx[j]; idx[j] = t; }
    for (int c = 0; c < 3; c++) {
        lam[c] = l[idx[c]];
        for (int r = 0; r < 3; r++) V[r * 3 + c] = W[r * 3 + idx[c]];
    }
    for (int c = 0; c < 2; c++) {
        int big = 0;
        for (int r = 1; r < 3; r++)
            if (fabs(V[r * 3 + c]) > fabs(V[big * 3 + c])) big = r;
        if (V[big * 3 + c] < 0)
            for (int r = 0; r < 3; r++) V[r * 3 + c] = -V[r * 3 + c];
    }
    /* v_max = v_min x v_mid */
    V[0 * 3 + 2] = V[1 * 3 + 0] * V[2 * 3 + 1] - V[2 * 3 + 0] * V[1 * 3 + 1];
    V[1 * 3 + 2] = V[2 * 3 + 0] * V[0 * 3 + 1] - V[0 * 3 + 0] * V[2 * 3 + 1];
    V[2 * 3 + 2] = V[0 * 3 + 0] * V[1 * 3 + 1] - V[1 * 3 + 0] * V[0 * 3 + 1];
}

typedef struct { int64_t key; int64_t idx; } kidx;
static int cmp_kidx(const void *a, const void *b) {
    const kidx *x = (const kidx *)a, *y = (const kidx *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return (x->idx > y->idx) - (x->idx < y->idx);
}

/* Descriptor Jacobians and covariance of one voxel (§III-A): for its N points P[N][3] with
 * mean mu, sorted eigen-system (l, V) and selected eigenvector k (0 = v_min, 2 = v_max):
 *   J_i = [V F_i ; I/N] (6x3),  F_i row m = (p_i - mu)^T (v_m v_k^T + v_k v_m^T) / (N (l_k - l_m))
 *   for m != k and 0 for m = k;  Sigma_g = sum_i J_i (sigma^2 I) J_i^T (6x6, row-major).
 * J (optional) receives the N Jacobians, each 6x3 row-major. */
void or_descriptor_cov(int64_t N, const double *P, const double *mu, const double *l, const double *V, int k,
                       double sigma, double *Sg, double *J) {
    memset(Sg, 0, sizeof(double) * 36);
    for (int64_t i = 0; i < N; i++) {
        double d[3], F[9], Ji[18];
        for (int q = 0; q < 3; q++) d[q] = P[3 * i + q] - mu[q];
        for (int m = 0; m < 3; m++) {
            for (int c = 0; c < 3; c++) F[m * 3 + c] = 0.0;
            if (m == k) continue;
            const double den = (double)N * (l[k] - l[m]);
            /* (p - mu)^T (v_m v_k^T + v_k v_m^T) = (d.v_m) v_k^T + (d.v_k) v_m^T */
            double dm = 0, dk = 0;
            for (int q = 0; q < 3; q++) { dm += d[q] * V[q * 3 + m]; dk += d[q] * V[q * 3 + k]; }
            for (int c = 0; c < 3; c++) F[m * 3 + c] = (dm * V[c * 3 + k] + dk * V[c * 3 + m]) / den;
        }
        /* rows 0..2: V F_i; rows 3..5: I / N */
        for (int r = 0; r < 3; r++)
            for (int c = 0; c < 3; c++) {
                double acc = 0;
                for (int q = 0; q < 3; q++) acc += V[r * 3 + q] * F[q * 3 + c];
                Ji[r * 3 + c] = acc;
                Ji[(3 + r) * 3 + c] = (r == c) ? 1.0 / (double)N : 0.0;
            }
        for (int r = 0; r < 6; r++)
            for (int c = 0; c < 6; c++) {
                double acc = 0;
                for (int q = 0; q < 3; q++) acc += Ji[r * 3 + q] * Ji[c * 3 + q];
                Sg[r * 6 + c] += sigma * sigma * acc;
            }
        if (J) memcpy(J + 18 * i, Ji, sizeof(Ji));
    }
}

/* Voxel key of an FP32 point: 21 bits per axis, offset by 2^20. */
int64_t or_voxel_key(const float *p, float s) {
    int64_t k = 0;
    for (int a = 0; a < 3; a++) {
        float q = floorf(p[a] / s);
        if (q < -1048576.0f) q = -1048576.0f;
        if (q > 1048575.0f) q = 1048575.0f;
        k = (k << 21) | (int64_t)((int32_t)q + 1048576);
    }
    return k;
}

/* Per point outputs (arrays of n):
 *   vox [n]      voxel index (dense, in ascending key order); npts [n] points in it
 *   lam [3n]     eigenvalues ascending, V [9n] row-major eigenvector matrix, mu [3n]
 *   cls [n]      0 unreliable, 1 planar, 2 linear; reliable [n]; trace [n] of Sigma_g[0:3,0:3]
 * Voxels with fewer than min_pts points get npts < min_pts and zero features. */
int64_t or_voxel_pca(int64_t n, const float *pts /* [3][n] */, float s, int min_pts, double tau_p, double tau_l,
                     double sigma, double tau_trace, int64_t *vox, int32_t *npts, double *lam, double *V,
                     double *mu, int32_t *cls, int32_t *reliable, double *trace) {
    kidx *t = (kidx *)malloc(sizeof(kidx) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; i++) {
        const float p[3] = {pts[i], pts[n + i], pts[2 * n + i]};
        t[i].key = or_voxel_key(p, s);
        t[i].idx = i;
    }
    qsort(t, (size_t)n, sizeof(kidx), cmp_kidx);
    int64_t nv = 0;
    for (int64_t a = 0; a < n;) {
        int64_t b = a;
        while (b < n && t[b].key == t[a].key) b++;
        const int64_t N = b - a;
        double m[3] = {0, 0, 0}, C[9] = {0}, l[3] = {0, 0, 0}, W[9] = {0};
        int c = 0, rel = 0;
        double tr = 0;
        if (N >= min_pts) {
            for (int64_t j = a; j < b; j++)
                for (int k = 0; k < 3; k++) m[k] += pts[(int64_t)k * n + t[j].idx];
            for (int k = 0; k < 3; k++) m[k] /= (double)N;
            for (int64_t j = a; j < b; j++) {
                double d[3];
                for (int k = 0; k < 3; k++) d[k] = pts[(int64_t)k * n + t[j].idx] - m[k];
                for (int r = 0; r < 3; r++)
                    for (int q = 0; q < 3; q++) C[r * 3 + q] += d[r] * d[q];
            }
            for (int k = 0; k < 9; k++) C[k] /= (double)N;
            or_eig_sorted(C, l, W);
            if (l[0] < tau_p) c = 1;
            else if (l[2] > tau_l * l[0]) c = 2;
            const double g1 = (l[1] - l[0]) / fmax(l[2], 1e-300), g2 = (l[2] - l[1]) / fmax(l[2], 1e-300);
            if (c != 0 && g1 > 1e-6 && g2 > 1e-6) {
                double *P = (double *)malloc(sizeof(double) * 3 * (size_t)N);
                for (int64_t j = a; j < b; j++)
                    for (int q = 0; q < 3; q++) P[3 * (j - a) + q] = pts[(int64_t)q * n + t[j].idx];
                double Sg[36];
                or_descriptor_cov(N, P, m, l, W, c == 1 ? 0 : 2, sigma, Sg, NULL);
                free(P);
                tr = Sg[0] + Sg[7] + Sg[14];
                rel = tr < tau_trace;
            }
        }
        for (int64_t j = a; j < b; j++) {
            const int64_t i = t[j].idx;
            vox[i] = nv;
            npts[i] = (int32_t)N;
            for (int k = 0; k < 3; k++) { lam[3 * i + k] = l[k]; mu[3 * i + k] = m[k]; }
            for (int k = 0; k < 9; k++) V[9 * i + k] = W[k];
            cls[i] = c;
            reliable[i] = rel;
            trace[i] = tr;
        }
        nv++;
        a = b;
    }
    free(t);
    return nv;
}
