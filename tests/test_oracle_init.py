"""Pins of the voxel-PCA and learned-initialiser oracle (no GPU)."""
import math

import numpy as np
import pytest

import oracle
from oracle import init_model as im


def test_jacobi_matches_textbook_eigh():
    rng = np.random.default_rng(0)
    for _ in range(30):
        A = rng.normal(size=(3, 3))
        C = A @ A.T + 1e-3 * np.eye(3)
        lam, V = oracle.eig_sorted(C)
        w, U = np.linalg.eigh(C)
        np.testing.assert_allclose(lam, w, rtol=1e-12, atol=1e-14)
        for c in range(3):
            assert abs(abs(V[:, c] @ U[:, c]) - 1) < 1e-10
        np.testing.assert_allclose(V.T @ V, np.eye(3), atol=1e-12)
        assert np.linalg.det(V) == pytest.approx(1.0, abs=1e-12)
        np.testing.assert_allclose(V @ np.diag(lam) @ V.T, C, atol=1e-12)


def _cloud(rng, n, spread, centre=(0.25, 0.25, 0.25)):
    """Points uniform in a box of half-widths `spread` around a voxel centre (inside one voxel)."""
    return (np.asarray(centre)[:, None] + rng.uniform(-1, 1, (3, n)) * np.asarray(spread)[:, None]).astype(np.float32)


def test_plane_and_line_classification():
    rng = np.random.default_rng(1)
    plane = _cloud(rng, 40, (0.2, 0.15, 0.004))
    out = oracle.voxel_pca(plane)
    assert out["n_voxels"] == 1 and out["cls"][0] == 1
    np.testing.assert_allclose(out["V"][0].reshape(3, 3)[:, 0], [0, 0, 1], atol=0.05)
    line = _cloud(rng, 40, (0.2, 0.03, 0.03))
    out = oracle.voxel_pca(line)
    # lambda_min ~ 4e-4 < tau_p would call it planar: raise tau_p to reach the linear test
    out = oracle.voxel_pca(line, tau_p=1e-5)
    assert out["cls"][0] == 2
    np.testing.assert_allclose(np.abs(out["V"][0].reshape(3, 3)[:, 2]), [1, 0, 0], atol=0.05)
    blob = _cloud(rng, 40, (0.2, 0.2, 0.2))
    assert oracle.voxel_pca(blob)["cls"][0] == 0
    few = _cloud(rng, 4, (0.2, 0.2, 0.004))
    o = oracle.voxel_pca(few)
    assert not o["has_feature"].any() and o["cls"][0] == 0


def test_descriptor_jacobian_matches_finite_differences():
    """Rows 0..2 of J_i are dv_k/dp_i and rows 3..5 are dmu/dp_i (§III-A Jacobian)."""
    rng = np.random.default_rng(2)
    P = (rng.normal(size=(25, 3)) * np.array([0.12, 0.07, 0.02])).astype(np.float64)
    for k in (0, 2):
        Sg, J, lam, V = oracle.descriptor_cov(P, k)
        h = 1e-7
        for i in (0, 7, 19):
            for j in range(3):
                Pp, Pm = P.copy(), P.copy()
                Pp[i, j] += h
                Pm[i, j] -= h
                _, _, _, Vp = oracle.descriptor_cov(Pp, k)
                _, _, _, Vm = oracle.descriptor_cov(Pm, k)
                vp, vm = Vp[:, k], Vm[:, k]
                vm = vm if vm @ vp > 0 else -vm
                fd = (vp - vm) / (2 * h)
                np.testing.assert_allclose(J[i, 0:3, j], fd, rtol=2e-5, atol=1e-7)
                e = np.zeros(3); e[j] = 1.0 / P.shape[0]
                np.testing.assert_allclose(J[i, 3:6, j], e, atol=1e-15)
        # Sigma_g = sum_i J_i sigma^2 J_i^T
        np.testing.assert_allclose(Sg, 0.02 ** 2 * np.einsum("nac,nbc->ab", J, J), rtol=1e-12,
                                   atol=1e-14 * np.abs(Sg).max())


def test_voxel_keys_follow_fp32_floor():
    pts = np.array([[0.0, 0.49999997, 0.5, -0.0000001, 1.0], [0.25] * 5, [0.25] * 5], np.float32)
    out = oracle.voxel_pca(pts, min_pts=1)
    # x voxels: 0, 0, 1, -1, 2 -> 4 distinct voxels, ascending key order
    assert out["n_voxels"] == 4
    assert out["vox"][0] == out["vox"][1] and out["vox"][3] < out["vox"][0] < out["vox"][2] < out["vox"][4]


def test_bf16_rounding_known_values():
    vals = np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, 1 + 2 ** -7, -2.5, 1e-3], np.float64)
    r = im.bf16(vals)
    assert r[0] == 1.0
    assert r[1] == 1.0                      # tie to even
    assert r[2] == 1 + 2 * 2 ** -7          # tie to even (odd neighbour below)
    assert r[3] == 1 + 2 ** -7
    assert r[4] == -2.5
    assert abs(r[5] - 1e-3) / 1e-3 < 2 ** -8


def test_mlp_backward_matches_finite_differences():
    Ws, bs = im.init_weights(3)
    rng = np.random.default_rng(4)
    x = rng.normal(size=(7, im.D_IN))
    t = rng.normal(size=(7, im.D_OUT))
    y, cache = im.mlp_forward(x, Ws, bs, round_bf16=False)
    gW, gb = im.mlp_backward(y, t, cache, Ws, round_bf16=False)
    h = 1e-6
    for l in range(4):
        for (o, i) in ((0, 0), (3, 5), (9, 2)):
            Wp = [w.copy() for w in Ws]; Wm = [w.copy() for w in Ws]
            Wp[l][o, i] += h; Wm[l][o, i] -= h
            fd = (im.mse_loss(im.mlp_forward(x, Wp, bs, False)[0], t) -
                  im.mse_loss(im.mlp_forward(x, Wm, bs, False)[0], t)) / (2 * h)
            assert abs(fd - gW[l][o, i]) < 1e-6 * max(1.0, abs(fd))
        bp = [b.copy() for b in bs]; bm = [b.copy() for b in bs]
        bp[l][1] += h; bm[l][1] -= h
        fd = (im.mse_loss(im.mlp_forward(x, Ws, bp, False)[0], t) -
              im.mse_loss(im.mlp_forward(x, Ws, bm, False)[0], t)) / (2 * h)
        assert abs(fd - gb[l][1]) < 1e-6 * max(1.0, abs(fd))


def test_gelu_closed_forms():
    assert im.gelu(np.array([0.0]))[0] == 0.0
    np.testing.assert_allclose(im.gelu(np.array([10.0])), [10.0], rtol=1e-12)
    np.testing.assert_allclose(im.gelu(np.array([1.0])), [0.8413447460685429], rtol=1e-12)
    z = np.linspace(-3, 3, 13)
    fd = (im.gelu(z + 1e-6) - im.gelu(z - 1e-6)) / 2e-6
    np.testing.assert_allclose(im.gelu_grad(z), fd, atol=1e-8)


def _rot_from_quat(q):
    w, x, y, z = q / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def test_quaternion_from_matrix_round_trip():
    rng = np.random.default_rng(5)
    for _ in range(50):
        q = rng.normal(size=4)
        q /= np.linalg.norm(q)
        q = q if q[0] >= 0 else -q
        np.testing.assert_allclose(im.quat_from_matrix(_rot_from_quat(q)), q, atol=1e-12)


def test_cascade_branches_and_beta():
    rng = np.random.default_rng(6)
    n = 6
    pts = rng.normal(size=(3, n)) + np.array([[0], [0], [5.0]])
    cols = rng.uniform(0, 1, (3, n))
    pca = dict(has_feature=np.array([1, 1, 1, 0, 1, 0], bool), reliable=np.array([1, 1, 0, 0, 1, 0]),
               lam=np.tile([1e-3, 4e-3, 9e-3], (n, 1)), V=np.tile(np.eye(3).reshape(9), (n, 1)))
    depth = np.full(n, 5.0)
    inside = np.array([1, 0, 1, 1, 1, 1], bool)
    y = np.zeros((n, 16)); y[:, 0] = 0.5; y[4, 1] = 4.0     # point 4: |residual| >= 3 -> invalid
    out = im.cascade(pts, cols, pca, depth, inside, 100.0, y)
    # valid model: has feature, inside, small residual -> points 0 and 2
    np.testing.assert_array_equal(out["branch"], [2, 1, 2, 0, 1, 0])
    assert out["beta"] == pytest.approx(max(0.25, 2 / 6))
    np.testing.assert_allclose(out["log_scales"][:, 3], [math.log(0.05)] * 3)     # heuristic log(d/f)
    np.testing.assert_allclose(out["log_scales"][0, 0], 0.5 * math.log(1e-3) + 0.5)  # pca + residual
    np.testing.assert_allclose(out["log_scales"][:, 1], 0.5 * np.log([1e-3, 4e-3, 9e-3]) + math.log(out["beta"]))
    np.testing.assert_allclose(out["quats"][:, 3], [1, 0, 0, 0])
    np.testing.assert_allclose(out["opacity_logits"][1], math.log(0.1 / 0.9))


def test_residual_pairs_hand_case():
    """Training targets of the initialiser on three hand-made rows.
    Row 0: the optimised quaternion is the initial one scaled by -2.5 (the same rotation), so
    its rotation residual is exactly 0; scales, logit and colour move by known amounts.
    Row 1: the initial quaternion is stored as (-1, 0, 0, 0), whose w >= 0 form is the
    identity; the optimised one is a rotation by 60 degrees about z, unnormalised (x 3): the
    residual is (cos 30 - 1, 0, 0, sin 30).
    Row 2: no voxel feature, dropped (and row order kept for the others)."""
    n, K = 3, 4                     # SH degree 1: 11 + 12 planes
    init = np.zeros((11 + 3 * K, n))
    init[6:10, :] = [[1.0, -1.0, 1.0], [0, 0, 0], [0, 0, 0], [0, 0, 0]]   # row 1 stored as -identity
    opt = init.copy()
    q0 = np.array([0.3, -0.5, 0.2, 0.7])
    init[6:10, 0] = q0
    opt[6:10, 0] = -2.5 * q0
    c, s = math.cos(math.pi / 6), math.sin(math.pi / 6)
    opt[6:10, 1] = 3.0 * np.array([c, 0, 0, s])
    init[3:6, 0] = [-3.0, -2.5, -4.0]
    opt[3:6, 0] = [-2.75, -2.5, -4.5]
    init[10, 0], opt[10, 0] = -2.0, 0.5
    init[11:14, 0] = [0.1, 0.2, 0.3]
    opt[11:14, 0] = [0.1 + 1.0 / im.Y00, 0.2, 0.3 - 0.5 / im.Y00]   # colour +1 and -0.5 after * Y00
    opt[14:, 0] = 7.0               # higher SH: not a target
    x = np.arange(3 * 16, dtype=float).reshape(3, 16)
    xs, y = im.residual_pairs(init, opt, x, has_feature=np.array([1, 1, 0]), inside=np.array([1, 1, 1]))
    assert xs.shape == (2, 16) and np.array_equal(xs, x[:2])
    np.testing.assert_allclose(y[0, 0:3], [0.25, 0.0, -0.5], atol=1e-15)
    np.testing.assert_allclose(y[0, 3:7], 0.0, atol=1e-15)
    assert y[0, 7] == 2.5
    np.testing.assert_allclose(y[0, 8:11], [1.0, 0.0, -0.5], atol=1e-14)
    np.testing.assert_allclose(y[1, 3:7], [c - 1.0, 0.0, 0.0, s], atol=1e-15)
    assert np.all(y[:, 11:] == 0)
    # without the flags every row is kept
    assert im.residual_pairs(init, opt, x)[1].shape == (3, 16)
