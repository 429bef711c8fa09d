"""Pins of the GICP oracle (CPU): the planar covariance against an eigen-decomposition, the
SE(3) exponential against the matrix exponential, the residual Jacobian against finite
differences, a hand-made target-set case, and recovery of a known loop transform."""
import numpy as np
import pytest

from oracle import gicp

linalg = pytest.importorskip("scipy.linalg")


def _rand_quat(rng):
    q = rng.normal(size=4)
    return q / np.linalg.norm(q)


def test_planar_covariance_matches_eigendecomposition():
    rng = np.random.default_rng(0)
    for _ in range(20):
        q = _rand_quat(rng)
        ls = rng.normal(-2, 0.5, 3).astype(np.float32)
        R = gicp.quat_to_R(q)
        Sig = R @ np.diag(np.exp(2.0 * ls.astype(np.float64))) @ R.T
        w, V = np.linalg.eigh(Sig)          # ascending: the first is the normal direction
        ref = V @ np.diag([1e-3, 1.0, 1.0]) @ V.T
        np.testing.assert_allclose(gicp.planar_covariance(q, ls), ref, atol=1e-9)


def test_se3_exp_matches_matrix_exponential():
    rng = np.random.default_rng(1)
    for scale in (1e-9, 1e-3, 0.5, 2.0):
        xi = rng.normal(size=6) * scale
        X = np.zeros((4, 4))
        X[:3, :3] = gicp._hat(xi[3:])
        X[:3, 3] = xi[:3]
        np.testing.assert_allclose(gicp.se3_exp(xi), linalg.expm(X), atol=1e-12)


def test_normal_equations_match_finite_differences():
    rng = np.random.default_rng(2)
    ns = 40
    src = rng.uniform(-1, 1, (3, ns))
    T = gicp.se3_exp(rng.normal(size=6) * 0.1)
    tar = (T[:3, :3] @ src + T[:3, 3:]) + rng.normal(0, 0.02, (3, ns))
    covs = [gicp.planar_covariance(_rand_quat(rng), rng.normal(-2, 0.5, 3)) for _ in range(ns)]
    covt = [gicp.planar_covariance(_rand_quat(rng), rng.normal(-2, 0.5, 3)) for _ in range(ns)]
    corr = np.arange(ns)
    H, g, cost, cnt = gicp.normal_equations(src, covs, tar, covt, T, corr)
    assert cnt == ns

    def f(xi):   # the cost with the weights frozen at T
        Tx = gicp.se3_exp(xi) @ T
        R0 = T[:3, :3]
        s = 0.0
        for m in range(ns):
            Om = np.linalg.inv(covt[m] + R0 @ covs[m] @ R0.T)
            r = tar[:, m] - (Tx[:3, :3] @ src[:, m] + Tx[:3, 3])
            s += r @ Om @ r
        return s
    h = 1e-6
    num = np.array([(f(h * e) - f(-h * e)) / (2 * h) for e in np.eye(6)])
    np.testing.assert_allclose(2 * g, num, rtol=1e-5, atol=1e-6)   # d cost / d xi = 2 g
    assert abs(cost - f(np.zeros(6))) < 1e-9 * max(1.0, cost)


def test_target_set_hand_case():
    cam = dict(width=100, height=80, fx=50.0, fy=50.0, cx=50.0, cy=40.0,
               R=np.eye(3), t=np.zeros(3))
    pts = np.array([[0.0, 0.0, 5.0],     # centre of the image
                    [0.0, 0.0, 0.1],     # in front of the near plane
                    [0.0, 0.0, -5.0],    # behind
                    [20.0, 0.0, 5.0],    # u = 250: right of the image
                    [0.0, 0.0, 25.0],    # beyond d_max = 20
                    [0.9, 0.7, 1.0]]).T  # u = 95, v = 75: inside, near the corner
    np.testing.assert_array_equal(gicp.target_set(pts, [cam]), [1, 0, 0, 0, 0, 1])
    src = np.array([0, 0, 0, 0, 0, 1], np.uint8)
    np.testing.assert_array_equal(gicp.target_set(pts, [cam], source_flag=src), [1, 0, 0, 0, 0, 0])


def test_register_recovers_known_transform():
    rng = np.random.default_rng(3)
    nt = 3000
    # a few planes (walls and floor) sampled densely, like LiDAR-shaped Gaussians
    pts = []
    for k in range(6):
        n = rng.normal(size=3); n /= np.linalg.norm(n)
        a = np.cross(n, [1, 0, 0] if abs(n[0]) < 0.9 else [0, 1, 0]); a /= np.linalg.norm(a)
        b = np.cross(n, a)
        uv = rng.uniform(-3, 3, (2, nt // 6))
        pts.append(rng.normal(size=3)[:, None] * 2 + a[:, None] * uv[0] + b[:, None] * uv[1])
    tar = np.concatenate(pts, axis=1)
    quats = [_rand_quat(rng) for _ in range(nt)]
    covt = [gicp.planar_covariance(q, rng.normal(-2, 0.3, 3)) for q in quats]
    sel = rng.choice(nt, 800, replace=False)
    T_gt = gicp.se3_exp(np.array([0.15, -0.1, 0.05, 0.02, -0.03, 0.04]))
    Tinv = np.linalg.inv(T_gt)
    src = Tinv[:3, :3] @ tar[:, sel] + Tinv[:3, 3:]
    covs = [Tinv[:3, :3] @ covt[i] @ Tinv[:3, :3].T for i in sel]
    T, cost, cnt, it, conv = gicp.register(src, covs, tar, covt, np.eye(4), d_corr=1.0)
    assert conv and cnt == 800
    np.testing.assert_allclose(T, T_gt, atol=1e-5)
