"""FP64/NumPy oracle of the Gaussian-GICP loop registration -- TEST INFRASTRUCTURE ONLY
(imported by the tests, never by the product path).

RMGS-SLAM §III-D: the target set is the map Gaussians that project inside the image of at least
one query view around the historical loopframe, lie within d_max of that view's position and do
not belong to the source set (target-set equation); every covariance is regularised to the
planar form with eigenvalues (1, 1, 1e-3); the loop pose minimises the sum over correspondences
of r^T (Sigma~_n + R Sigma~_m R^T)^-1 r with r = mu_n - T mu_m (residual, covariance and
objective equations).

Readings where the paper is silent:
  * in the image: z > near_z (0.2 m), 0 <= u < W and 0 <= v < H for u = fx x / z + cx,
    v = fy y / z + cy, all in FP32 with the kernel's operation order; the distance to the view's
    position (its camera centre) is compared squared, in FP32; d_max = 20 m;
  * planar form: with R from the normalised quaternion, the axis of the smallest log-scale (the
    lower index on ties) gets 1e-3 and the other two get 1: Sigma~ = R diag(l) R^T;
  * correspondences: each source mean, moved by the current T (in FP32), takes the nearest
    target mean (FP32 squared distance, the lower index on ties) if it lies within d_corr (1 m);
  * Gauss-Newton with the weights Omega = (Sigma~_n + R Sigma~_m R^T)^-1 held fixed within an
    iteration, left perturbation T <- Exp(xi) T with xi = (rho, phi); it stops when |xi| < eps
    (1e-7) or after max_iters (30); the cost is the sum of r^T Omega r at the last
    correspondences.
"""
from __future__ import annotations

import numpy as np


def quat_to_R(q):
    w, x, y, z = np.asarray(q, dtype=np.float64) / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def planar_covariance(quat, log_scale):
    """Sigma~ = R diag(l) R^T, l = 1e-3 on the smallest-scale axis, 1 on the others."""
    R = quat_to_R(quat)
    ls = np.asarray(log_scale, dtype=np.float32)
    a = int(np.argmin(ls))          # first minimum on ties
    lam = np.ones(3)
    lam[a] = 1e-3
    return R @ np.diag(lam) @ R.T


def target_set(means, cams, near_z=0.2, d_max=20.0, source_flag=None):
    """uint8 [n]: in the image of some view, within d_max of its centre, not a source row."""
    M = np.asarray(means, dtype=np.float32)
    n = M.shape[1]
    flag = np.zeros(n, bool)
    f32 = np.float32
    dmax2 = f32(d_max) * f32(d_max)
    for cam in cams:
        R = np.asarray(cam["R"], dtype=np.float32).reshape(3, 3)
        t = np.asarray(cam["t"], dtype=np.float32)
        # p_c = R mu + t, each row summed left to right in FP32
        pc = [((R[r, 0] * M[0] + R[r, 1] * M[1]).astype(f32) + (R[r, 2] * M[2]).astype(f32)).astype(f32) + t[r]
              for r in range(3)]
        pc = [p.astype(f32) for p in pc]
        z = pc[2]
        with np.errstate(divide="ignore", invalid="ignore"):
            u = (f32(cam["fx"]) * pc[0] / z).astype(f32) + f32(cam["cx"])
            v = (f32(cam["fy"]) * pc[1] / z).astype(f32) + f32(cam["cy"])
        inside = (z > f32(near_z)) & (u >= 0) & (u < f32(cam["width"])) & (v >= 0) & (v < f32(cam["height"]))
        # camera centre c = -R^T t from the FP32 pose (as the camera record holds it), in FP64,
        # rounded to FP32 once
        R64 = np.asarray(cam["R"], dtype=np.float32).reshape(3, 3).astype(np.float64)
        t64 = np.asarray(cam["t"], dtype=np.float32).astype(np.float64)
        c = (-(R64.T @ t64)).astype(f32)
        d = [(M[k] - c[k]).astype(f32) for k in range(3)]
        d2 = ((d[0] * d[0]).astype(f32) + (d[1] * d[1]).astype(f32)).astype(f32) + (d[2] * d[2]).astype(f32)
        flag |= inside & (d2.astype(f32) < dmax2)
    if source_flag is not None:
        flag &= np.asarray(source_flag) == 0
    return flag.astype(np.uint8)


def _hat(v):
    return np.array([[0, -v[2], v[1]], [v[2], 0, -v[0]], [-v[1], v[0], 0]])


def se3_exp(xi):
    """Exp of (rho, phi) as a 4 x 4 matrix."""
    rho, phi = np.asarray(xi[:3], float), np.asarray(xi[3:], float)
    th = np.linalg.norm(phi)
    K = _hat(phi)
    if th < 1e-12:
        R = np.eye(3) + K
        V = np.eye(3) + 0.5 * K
    else:
        A = np.sin(th) / th
        B = (1 - np.cos(th)) / th ** 2
        C = (1 - A) / th ** 2
        R = np.eye(3) + A * K + B * K @ K
        V = np.eye(3) + B * K + C * K @ K
    T = np.eye(4)
    T[:3, :3] = R
    T[:3, 3] = V @ rho
    return T


def correspondences(src, tar, T, d_corr):
    """For each source mean (FP32, moved by T rounded to FP32) the nearest target within d_corr
    (FP32 squared distance summed in x, y, z order; lower index on ties), else -1."""
    f32 = np.float32
    R = T[:3, :3].astype(f32)
    t = T[:3, 3].astype(f32)
    S = np.asarray(src, dtype=f32)
    q = [(((R[r, 0] * S[0]).astype(f32) + (R[r, 1] * S[1]).astype(f32)).astype(f32) +
          (R[r, 2] * S[2]).astype(f32)).astype(f32) + t[r] for r in range(3)]
    q = np.stack([a.astype(f32) for a in q])
    Tm = np.asarray(tar, dtype=f32)
    r2 = f32(d_corr) * f32(d_corr)
    out = np.full(S.shape[1], -1, np.int64)
    for j0 in range(0, S.shape[1], 512):
        qq = q[:, j0:j0 + 512]
        dx = (qq[0][:, None] - Tm[0][None, :]).astype(f32)
        dy = (qq[1][:, None] - Tm[1][None, :]).astype(f32)
        dz = (qq[2][:, None] - Tm[2][None, :]).astype(f32)
        d2 = ((dx * dx).astype(f32) + (dy * dy).astype(f32)).astype(f32) + (dz * dz).astype(f32)
        best = np.argmin(d2, axis=1)              # first minimum on ties
        ok = d2[np.arange(d2.shape[0]), best] < r2
        out[j0:j0 + 512] = np.where(ok, best, -1)
    return out


def normal_equations(src, src_cov, tar, tar_cov, T, corr):
    """H (6 x 6), g (6), cost and count of the linearised objective at T."""
    R, t = T[:3, :3], T[:3, 3]
    H = np.zeros((6, 6)); g = np.zeros(6); cost = 0.0; cnt = 0
    S = np.asarray(src, np.float64); Tm = np.asarray(tar, np.float64)
    for m in np.nonzero(corr >= 0)[0]:
        n = corr[m]
        q = R @ S[:, m] + t
        r = Tm[:, n] - q
        Om = np.linalg.inv(tar_cov[n] + R @ src_cov[m] @ R.T)
        J = np.hstack([-np.eye(3), _hat(q)])      # dr/dxi for T <- Exp(xi) T
        H += J.T @ Om @ J
        g += J.T @ Om @ r
        cost += r @ Om @ r
        cnt += 1
    return H, g, cost, cnt


def register(src, src_cov, tar, tar_cov, T0, d_corr=1.0, max_iters=30, eps=1e-7):
    """Gauss-Newton; returns (T, cost, correspondences, iterations, converged)."""
    T = np.array(T0, dtype=np.float64)
    converged = False
    it = 0
    for it in range(1, max_iters + 1):
        corr = correspondences(src, tar, T, d_corr)
        H, g, cost, cnt = normal_equations(src, src_cov, tar, tar_cov, T, corr)
        if cnt < 6:
            break
        xi = -np.linalg.solve(H, g)
        T = se3_exp(xi) @ T
        if np.linalg.norm(xi) < eps:
            converged = True
            break
    corr = correspondences(src, tar, T, d_corr)
    H, g, cost, cnt = normal_equations(src, src_cov, tar, tar_cov, T, corr)
    return T, cost, cnt, it, converged
