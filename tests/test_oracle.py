"""Pins of the FP64 oracle against what the mathematics fixes (no GPU).

Each test checks the oracle against something other than itself: a closed form, an
invariant, an independent numeric derivative, a textbook routine, or brute force.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from oracle import Opts

pytestmark = pytest.mark.filterwarnings("ignore")


# ----------------------------------------------------------------------------------------
# Spherical harmonics
# ----------------------------------------------------------------------------------------

def _sphere_quadrature(n_theta=12, n_phi=24):
    """Gauss-Legendre in cos(theta) x uniform phi: exact for polynomials of degree < 2*n."""
    x, w = np.polynomial.legendre.leggauss(n_theta)
    phi = np.arange(n_phi) * 2 * np.pi / n_phi
    pts, wts = [], []
    for ct, wt in zip(x, w):
        st = math.sqrt(1 - ct * ct)
        for p in phi:
            pts.append((st * math.cos(p), st * math.sin(p), ct))
            wts.append(wt * 2 * np.pi / n_phi)
    return np.array(pts), np.array(wts)


def test_sh_basis_is_orthonormal_on_the_sphere():
    pts, wts = _sphere_quadrature()
    Y = np.stack([oracle.sh_basis(3, p)[0] for p in pts])   # [Q, 16]
    gram = (Y * wts[:, None]).T @ Y
    np.testing.assert_allclose(gram, np.eye(16), atol=1e-12)


def test_sh_basis_matches_textbook_low_orders():
    # Y00 = 1/(2 sqrt(pi)); degree 1 is sqrt(3/(4 pi)) * (-y, z, -x) (Condon-Shortley phase)
    d = np.array([0.3, -0.5, 0.81])
    d /= np.linalg.norm(d)
    Y, _ = oracle.sh_basis(1, d)
    c1 = math.sqrt(3 / (4 * math.pi))
    np.testing.assert_allclose(Y, [0.5 / math.sqrt(math.pi), -c1 * d[1], c1 * d[2], -c1 * d[0]],
                               rtol=1e-14)


def test_sh_gradient_matches_central_differences():
    rng = np.random.default_rng(0)
    for _ in range(5):
        d = rng.normal(size=3)
        _, G = oracle.sh_basis(3, d)
        h = 1e-6
        for j in range(3):
            e = np.zeros(3); e[j] = h
            fd = (oracle.sh_basis(3, d + e)[0] - oracle.sh_basis(3, d - e)[0]) / (2 * h)
            np.testing.assert_allclose(G[:, j], fd, atol=1e-8)


# ----------------------------------------------------------------------------------------
# Projection
# ----------------------------------------------------------------------------------------

def _one_gaussian(mu, log_scale, quat=(1, 0, 0, 0), logit=2.0, colour=(0.2, 0.6, 0.9), deg=0):
    K = (deg + 1) ** 2
    sh = np.zeros((3 * K, 1), np.float64)
    sh[0:3, 0] = (np.asarray(colour) - 0.5) * 2 * math.sqrt(math.pi)
    return synth.Scene(np.asarray(mu, np.float64).reshape(3, 1),
                       np.full((3, 1), log_scale, np.float64) if np.isscalar(log_scale)
                       else np.asarray(log_scale, np.float64).reshape(3, 1),
                       np.asarray(quat, np.float64).reshape(4, 1), np.array([logit], np.float64), sh, deg)


def test_projection_on_axis_isotropic_closed_form():
    f, z, s = 300.0, 4.0, 0.05
    cam = synth.camera(320, 240, f)
    sc = _one_gaussian((0, 0, z), math.log(s), quat=(0.3, -0.2, 0.5, 0.1))
    pr = oracle.project(sc, cam)
    var = (f * s / z) ** 2 + 0.3
    np.testing.assert_allclose(pr["cov2d"][0], [var, 0, var], rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(pr["conic"][0], [1 / var, 0, 1 / var], rtol=1e-13, atol=1e-13)
    assert pr["u"][0] == pytest.approx(160.0) and pr["v"][0] == pytest.approx(120.0)
    o = 1 / (1 + math.exp(-2.0))
    r = math.ceil(math.sqrt(2 * math.log(255 * o) * var))
    assert pr["rx"][0] == r and pr["ry"][0] == r
    np.testing.assert_allclose(pr["rgb"][0], [0.2, 0.6, 0.9], rtol=1e-13)


def _rot(axis, ang):
    axis = np.asarray(axis, float) / np.linalg.norm(axis)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * K @ K


def test_projection_matches_numeric_jacobian_off_axis():
    """cov2d - dilation*I equals J_num (W Sigma W^T) J_num^T with J_num a central-difference
    Jacobian of the pinhole map at the camera-frame centre, and Sigma built from an
    independently written rotation (Rodrigues form of the quaternion's axis-angle)."""
    R = _rot([0.2, 1.0, -0.3], 0.4)
    cam = synth.camera(640, 480, 500.0, fy=450.0, cx=310.0, cy=250.0, R=R, t=[0.3, -0.1, 0.5])
    mu = np.array([0.7, -0.4, 3.0])
    ang, axis = 0.9, np.array([1.0, 2.0, -0.5])
    axis /= np.linalg.norm(axis)
    q = np.concatenate([[math.cos(ang / 2)], math.sin(ang / 2) * axis]) * 1.7  # unnormalised
    ls = np.log([0.08, 0.03, 0.2])
    sc = _one_gaussian(mu, ls, quat=q)
    pr = oracle.project(sc, cam)
    Rq = _rot(axis, ang)
    Sigma = Rq @ np.diag(np.exp(2 * ls)) @ Rq.T
    pc = R @ mu + np.asarray(cam["t"])

    def pi(p):
        return np.array([cam["fx"] * p[0] / p[2] + cam["cx"], cam["fy"] * p[1] / p[2] + cam["cy"]])
    Jn = np.zeros((2, 3))
    for j in range(3):
        e = np.zeros(3); e[j] = 1e-6
        Jn[:, j] = (pi(pc + e) - pi(pc - e)) / 2e-6
    cov = Jn @ (R @ Sigma @ R.T) @ Jn.T
    a, b, c = pr["cov2d"][0]
    np.testing.assert_allclose([a - 0.3, b, c - 0.3], [cov[0, 0], cov[0, 1], cov[1, 1]], rtol=1e-7)
    np.testing.assert_allclose([pr["u"][0], pr["v"][0]], pi(pc), rtol=1e-14)
    assert pr["z"][0] == pytest.approx(pc[2], rel=1e-14)


def test_projection_culls_near_and_transparent():
    cam = synth.camera(64, 48, 60.0)
    assert oracle.project(_one_gaussian((0, 0, 0.1), -3.0), cam)["visible"][0] == 0
    assert oracle.project(_one_gaussian((0, 0, 3.0), -3.0, logit=-7.0), cam)["visible"][0] == 0
    assert oracle.project(_one_gaussian((0, 0, 3.0), -3.0), cam)["visible"][0] == 1


# ----------------------------------------------------------------------------------------
# Compositing
# ----------------------------------------------------------------------------------------

def test_single_gaussian_image_closed_form():
    f, z, s = 60.0, 3.0, 0.15
    cam = synth.camera(64, 48, f)
    colour = np.array([0.2, 0.6, 0.9])
    bg = (0.1, 0.3, 0.5)
    logit = 1.2
    sc = _one_gaussian((0.1, -0.05, z), math.log(s), logit=logit, colour=colour)
    op = Opts(bg=bg)
    pr = oracle.project(sc, cam, op)
    img = oracle.render(pr, cam, op)
    # isotropic Sigma = s^2 I, so the image covariance is s^2 J J^T + 0.3 I with J the
    # pinhole Jacobian at (x, y, z) = (0.1, -0.05, z)
    x, y = 0.1, -0.05
    Jm = np.array([[f / z, 0, -f * x / z ** 2], [0, f / z, -f * y / z ** 2]])
    cov = s * s * Jm @ Jm.T + 0.3 * np.eye(2)
    Ci = np.linalg.inv(cov)
    o = 1 / (1 + math.exp(-logit))
    u0, v0 = f * x / z + 32, f * y / z + 24
    ys, xs = np.mgrid[0:48, 0:64] + 0.5
    dx, dy = xs - u0, ys - v0
    q = Ci[0, 0] * dx * dx + 2 * Ci[0, 1] * dx * dy + Ci[1, 1] * dy * dy
    a = np.minimum(0.99, o * np.exp(-0.5 * q))
    keep = a >= 1 / 255
    a = np.where(keep, a, 0.0)
    expect = np.asarray(bg)[:, None, None] * (1 - a) + colour[:, None, None] * a
    np.testing.assert_allclose(img["C"], expect, atol=1e-12)
    np.testing.assert_allclose(img["D"], a * z, atol=1e-12)
    np.testing.assert_allclose(img["T"], 1 - a, atol=1e-12)


def _white_scene(seed, n):
    sc = synth.uniform_box_scene(seed, n, sh_degree=0)
    sc.sh[:] = 0.5 * 2 * math.sqrt(math.pi)      # colour exactly 1 in every channel
    return sc


def test_transmittance_invariant():
    """With unit colour and black background, C = sum_i w_i, and sum_i w_i + T_final = 1."""
    sc = _white_scene(3, 300)
    cam = synth.camera(64, 48, 60.0)
    pr = oracle.project(sc, cam)
    img = oracle.render(pr, cam)
    assert img["n_frag"].max() > 3
    for ch in range(3):
        np.testing.assert_allclose(img["C"][ch] + img["T"], 1.0, atol=1e-12)
    assert img["T"].min() >= 1e-4


def test_depth_order_swaps_contributions():
    cam = synth.camera(16, 16, 20.0)
    c1, c2 = np.array([1.0, 0, 0]), np.array([0, 0, 1.0])

    def two(z1, z2):
        a = _one_gaussian((0, 0, z1), math.log(0.3), logit=0.5, colour=c1)
        b = _one_gaussian((0, 0, z2), math.log(0.3), logit=0.5, colour=c2)
        sc = synth.Scene(np.concatenate([a.means, b.means], 1), np.concatenate([a.log_scales, b.log_scales], 1),
                         np.concatenate([a.quats, b.quats], 1), np.concatenate([a.opacity_logits, b.opacity_logits]),
                         np.concatenate([a.sh, b.sh], 1), 0)
        pr = oracle.project(sc, cam)
        return pr, oracle.render(pr, cam)
    prA, A = two(2.0, 3.0)
    prB, B = two(3.0, 2.0)
    px = (8, 8)

    def alpha(pr, g):
        d = np.array([px[1] + 0.5 - pr["u"][g], px[0] + 0.5 - pr["v"][g]])
        Aq, Bq, Cq = pr["conic"][g]
        return min(0.99, pr["opacity"][g] * math.exp(-0.5 * (Aq * d[0] ** 2 + 2 * Bq * d[0] * d[1] + Cq * d[1] ** 2)))
    a1, a2 = alpha(prA, 0), alpha(prA, 1)
    np.testing.assert_allclose(A["C"][:, px[0], px[1]], c1 * a1 + c2 * a2 * (1 - a1), atol=1e-12)
    b1, b2 = alpha(prB, 0), alpha(prB, 1)
    np.testing.assert_allclose(B["C"][:, px[0], px[1]], c2 * b2 + c1 * b1 * (1 - b2), atol=1e-12)


def _two_gaussians(a, b):
    return synth.Scene(np.concatenate([a.means, b.means], 1), np.concatenate([a.log_scales, b.log_scales], 1),
                       np.concatenate([a.quats, b.quats], 1), np.concatenate([a.opacity_logits, b.opacity_logits]),
                       np.concatenate([a.sh, b.sh], 1), a.sh_degree)


def test_equal_fp32_depth_keys_composite_in_index_order():
    """Two Gaussians whose depths differ below FP32 resolution: the front-to-back order is that
    of their FP32 depth keys, and equal keys go in index order -- even where the FP64 depths
    order them the other way.  Camera turned about y by theta = 2^-20 rad: Gaussian 0 at
    (-2^-5, 0, 3) has depth 3 cos(theta) + 2^-5 sin(theta), Gaussian 1 at (0, 0, 3) depth
    3 cos(theta), so Gaussian 1 is nearer by ~3e-8 m in FP64; in FP32 sin(theta) = 2^-20,
    cos(theta) = 1 and 3 + 2^-25 rounds to 3 (one ulp at 3 is 2^-22): equal keys."""
    th = 2.0 ** -20
    R = np.array([[math.cos(th), 0, math.sin(th)], [0, 1, 0], [-math.sin(th), 0, math.cos(th)]])
    cam = synth.camera(16, 16, 20.0, R=R)
    ca, cb = np.array([1.0, 0, 0]), np.array([0, 0, 1.0])
    a = _one_gaussian((-2.0 ** -5, 0, 3.0), math.log(0.3), logit=0.5, colour=ca)
    b = _one_gaussian((0, 0, 3.0), math.log(0.3), logit=0.5, colour=cb)
    sc = _two_gaussians(a, b)
    pr = oracle.project(sc, cam)
    assert pr["z"][0] > pr["z"][1]                      # FP64: Gaussian 1 is in front
    assert pr["zkey"][0] == pr["zkey"][1] == np.float32(3.0)
    img = oracle.render(pr, cam)
    # each Gaussian's alpha at the centre pixel from its own single-Gaussian image (C = alpha c)
    py = px = 8
    al = [oracle.render(oracle.project(s, cam), cam)["C"][ch, py, px]
          for s, ch in ((a, 0), (b, 2))]
    got = img["C"][:, py, px]
    np.testing.assert_allclose(got, ca * al[0] + cb * al[1] * (1 - al[0]), atol=1e-12)   # index order
    assert np.abs(got - (cb * al[1] + ca * al[0] * (1 - al[1]))).max() > 1e-2             # not FP64 order


def test_depth_key_is_the_fp32_depth():
    """The key is the camera depth rounded through FP32 arithmetic: within a few FP32 ulps of
    the FP64 depth (so no term, sign or row of the pose is lost), ascending with it wherever
    the FP64 depths differ by more than that, and exactly the FP32 value when every product
    and sum is exact (dyadic inputs)."""
    R = _rot([0.3, -1.0, 0.4], 0.7)
    cam = synth.camera(320, 240, 300.0, R=R, t=[0.4, -0.3, 7.5])
    sc = synth.uniform_box_scene(5, 3000, sh_degree=0)
    pr = oracle.project(sc, cam)
    z32 = pr["zkey"].astype(np.float64)
    z = pr["z"]
    bound = 4 * 2.0 ** -24 * (np.abs(R[2]) @ np.abs(sc.means) + 7.5)
    assert np.all(np.abs(z32 - z) <= bound)
    o = np.argsort(z)
    dz = np.diff(z[o])
    far = dz > bound[o][1:] + bound[o][:-1]
    assert np.all(np.diff(z32[o])[far] > 0)
    # dyadic rotation rows and means: every operation exact, key == the exact depth
    Rd = np.array([[0.6, 0.0, -0.8], [0.0, 1.0, 0.0], [0.8, 0.0, 0.6]])
    Rd[2] = [0.75, 0.0, 0.5]                              # only the third row enters the key
    camd = synth.camera(64, 48, 60.0, R=Rd, t=[0, 0, 0.25])
    s = _one_gaussian((1.5, 0.25, 2.125), -3.0)
    assert oracle.project(s, camd)["zkey"][0] == np.float32(0.75 * 1.5 + 0.5 * 2.125 + 0.25)


def test_screen_box_bounds_every_kept_fragment():
    """Outside a Gaussian's screen box (half-extents rx, ry) alpha < alpha_min, so
    restricting each pixel to the Gaussians whose box contains it changes nothing (the tiled
    GPU path relies on this): brute force over all Gaussians equals the restricted form
    exactly, and alpha just outside each box edge is below alpha_min."""
    sc = synth.uniform_box_scene(4, 400, sh_degree=1)
    cam = synth.camera(80, 60, 70.0)
    pr = oracle.project(sc, cam)
    a = oracle.render(pr, cam, use_square=True)
    b = oracle.render(pr, cam, use_square=False)
    for k in ("C", "D", "T"):
        np.testing.assert_array_equal(a[k], b[k])
    # and directly: alpha at pixel centres just outside the square
    for g in np.nonzero(pr["visible"])[0][:200]:
        rx, ry = pr["rx"][g], pr["ry"][g]
        A, B, Cq = pr["conic"][g]
        # the largest alpha on the lines x = +-(rx + eps), y = +-(ry + eps) (closed-form minimum
        # of the quadratic form along each line) stays below alpha_min
        for dx in (rx + 0.01, -rx - 0.01):
            q = dx * dx * (A - B * B / Cq)
            assert pr["opacity"][g] * math.exp(-0.5 * q) < 1 / 255
        for dy in (ry + 0.01, -ry - 0.01):
            q = dy * dy * (Cq - B * B / A)
            assert pr["opacity"][g] * math.exp(-0.5 * q) < 1 / 255


# ----------------------------------------------------------------------------------------
# Backward: central finite differences
# ----------------------------------------------------------------------------------------

def _perturb_param(sc, k, i, delta):
    s = synth.Scene(*(np.asarray(a, np.float64).copy() for a in
                      (sc.means, sc.log_scales, sc.quats, sc.opacity_logits, sc.sh)), sc.sh_degree)
    if k < 3:
        s.means[k, i] += delta
    elif k < 6:
        s.log_scales[k - 3, i] += delta
    elif k < 10:
        s.quats[k - 6, i] += delta
    elif k < 11:
        s.opacity_logits[i] += delta
    else:
        s.sh[k - 11, i] += delta
    return s


def _exp_se3(xi):
    rho, phi = xi[:3], xi[3:]
    th = np.linalg.norm(phi)
    K = np.array([[0, -phi[2], phi[1]], [phi[2], 0, -phi[0]], [-phi[1], phi[0], 0]])
    if th < 1e-12:
        return np.eye(3) + K, np.eye(3) + 0.5 * K
    R = np.eye(3) + math.sin(th) / th * K + (1 - math.cos(th)) / th ** 2 * K @ K
    V = np.eye(3) + (1 - math.cos(th)) / th ** 2 * K + (th - math.sin(th)) / th ** 3 * K @ K
    return R, V


def _cam_pert(cam, xi):
    R, V = _exp_se3(xi)
    c = dict(cam)
    c["R"] = R @ np.asarray(cam["R"])
    c["t"] = R @ np.asarray(cam["t"]) + V @ xi[:3]
    return c


def _linear_loss(sc, cam, up, op):
    pr, im = oracle.forward(sc, [cam], op)[0]
    return (up["gC"] * im["C"]).sum() + (up["gD"] * im["D"]).sum(), im


def _fd_case(op, n, h, seed, n_checks, tol, state_check):
    sc = synth.uniform_box_scene(seed, n, sh_degree=3, box=((-1.5, 1.5), (-1, 1), (2, 5)),
                                 logscale_mu=-2.5)
    cam = synth.camera(64, 48, 60.0, R=_rot([0.3, -1, 0.2], 0.12), t=[0.1, -0.2, 0.3])
    up = synth.random_upstream(seed + 1, [cam])[0]
    fwd = oracle.forward(sc, [cam], op)
    grads, tw = oracle.backward(sc, [cam], fwd, [up], op)
    rng = np.random.default_rng(seed + 2)
    checked = 0
    worst = 0.0
    planes = grads.shape[0]
    vis = np.nonzero(fwd[0][0]["visible"])[0]
    trials = 0
    while checked < n_checks and trials < 20 * n_checks:
        trials += 1
        k, i = int(rng.integers(planes)), int(rng.choice(vis))
        lp, ip = _linear_loss(_perturb_param(sc, k, i, h), cam, up, op)
        lm, im = _linear_loss(_perturb_param(sc, k, i, -h), cam, up, op)
        if state_check and not np.array_equal(ip["n_frag"], im["n_frag"]):
            continue
        fd = (lp - lm) / (2 * h)
        an = grads[k, i]
        scale = max(abs(fd), abs(an), 1e-3)
        worst = max(worst, abs(fd - an) / scale)
        checked += 1
    assert checked >= n_checks // 2
    for j in range(6):
        xi = np.zeros(6); xi[j] = h
        lp, ip = _linear_loss(sc, _cam_pert(cam, xi), up, op)
        lm, im = _linear_loss(sc, _cam_pert(cam, -xi), up, op)
        if state_check and not np.array_equal(ip["n_frag"], im["n_frag"]):
            continue
        fd = (lp - lm) / (2 * h)
        worst = max(worst, abs(fd - tw[0, j]) / max(abs(fd), 1e-3))
    assert worst < tol, worst


def test_backward_matches_finite_differences_smooth():
    """Thresholds moved out of the way (alpha_min 1e-9, no early stop) so the loss is smooth:
    every parameter plane (means, log-scales, quats, opacity, SH degree 3) and the SE(3)
    twist agree with central differences."""
    _fd_case(Opts(alpha_min=1e-9, T_min=0.0), n=60, h=1e-5, seed=11, n_checks=60, tol=1e-5,
             state_check=False)


def test_backward_matches_finite_differences_default_thresholds():
    """Default compositing constants on a 200-Gaussian 64x48 scene; coordinates whose +-h
    perturbation changes the set of added fragments are skipped."""
    _fd_case(Opts(), n=200, h=1e-6, seed=21, n_checks=40, tol=1e-4, state_check=True)


# ----------------------------------------------------------------------------------------
# Loss, optimizer, binning
# ----------------------------------------------------------------------------------------

def test_l1_loss_small_hand_case():
    img = dict(C=np.array([[[0.5, 0.2]], [[0.1, 0.9]], [[0.0, 0.3]]]), D=np.array([[2.0, 5.0]]))
    tgt = dict(rgb=np.array([[[0.25, 0.2]], [[0.3, 0.4]], [[0.0, 0.1]]]), depth=np.array([[3.0, 0.0]]),
               mask=np.array([[1, 1]], np.uint8))
    loss, gC, gD = oracle.l1_loss(img, tgt, Opts(lambda_rgb=1.0, lambda_depth=0.5), scale=1.0)
    # rgb: (0.25 + 0.2 + 0) + (0 + 0.5 + 0.2) over |M| = 2 ; depth: |2-3| over 1 pixel with D~>0
    assert loss == pytest.approx((0.45 + 0.7) / 2 + 0.5 * 1.0)
    np.testing.assert_array_equal(gC[:, 0, 0], [0.5, -0.5, 0.0])
    np.testing.assert_array_equal(gC[:, 0, 1], [0.0, 0.5, 0.5])
    np.testing.assert_array_equal(gD, [[-0.5, 0.0]])


def test_adam_constant_gradient_moves_by_lr_times_sign():
    """With bias correction, a constant gradient g gives m_hat = g and v_hat = g^2 at every
    step, so each step moves p by lr * g / (|g| + eps)."""
    p = np.zeros((14, 5)); g = np.linspace(-2, 2, 70).reshape(14, 5) + 0.01
    m = np.zeros_like(p); v = np.zeros_like(p)
    lr = (0.1, 0.2, 0.3, 0.4, 0.5, 0.6)
    for step in (1, 2, 3):
        p, m, v = oracle.adam(p, g, m, v, None, lr=lr, step=step)
    grp = np.array([0] * 3 + [1] * 3 + [2] * 4 + [3] + [4] * 3)
    expect = -3 * np.asarray(lr)[grp][:, None] * g / (np.abs(g) + 1e-15)
    np.testing.assert_allclose(p, expect, rtol=1e-12)


def test_adam_zero_betas_is_sign_descent_and_mask_is_exact():
    """With beta1 = beta2 = 0 Adam reduces to sign descent, p -= lr * g / (|g| + eps), for
    any gradient sequence; rows outside the update mask keep p, m and v bit for bit."""
    rng = np.random.default_rng(3)
    n = 9
    p0 = rng.normal(size=(12, n)); p = p0.copy()
    m = rng.normal(size=(12, n)); v = rng.uniform(0.1, 1, (12, n))
    m0, v0 = m.copy(), v.copy()
    upd = np.ones(n, np.uint8); upd[[2, 7]] = 0
    expect = p0.copy()
    for step in (1, 2, 3):
        g = rng.normal(size=(12, n))
        p, m, v = oracle.adam(p, g, m, v, upd, lr=(1e-2,) * 6, b1=0.0, b2=0.0, step=step)
        expect[:, upd == 1] -= 1e-2 * g[:, upd == 1] / (np.abs(g[:, upd == 1]) + 1e-15)
    np.testing.assert_allclose(p, expect, rtol=1e-13)
    np.testing.assert_array_equal(p[:, [2, 7]], p0[:, [2, 7]])
    np.testing.assert_array_equal(m[:, [2, 7]], m0[:, [2, 7]])
    np.testing.assert_array_equal(v[:, [2, 7]], v0[:, [2, 7]])


def test_binning_sort_and_ranges():
    cams = [synth.camera(100, 70, 80.0), synth.camera(48, 64, 40.0)]
    items = synth.random_projected_items(7, cams, 3000)
    for tile in (8, 16):
        b = oracle.bin_views(items, cams, tile)
        assert b["keys"].shape[0] == int(b["touched"].sum())
        # the stable order is what a textbook stable sort (NumPy's) gives
        order = np.argsort(b["keys"], kind="stable")
        np.testing.assert_array_equal(b["sorted_keys"], b["keys"][order])
        np.testing.assert_array_equal(b["sorted_vals"], b["vals"][order])
        # ranges cover each tile's run exactly
        tiles = (b["sorted_keys"] >> np.uint64(32)).astype(np.int64)
        counts = np.bincount(tiles, minlength=b["n_tiles"])
        np.testing.assert_array_equal(b["ranges"][:, 1] - b["ranges"][:, 0], counts)
        # conservative coverage: every pixel centre within the box of an item lies in an
        # emitted tile of that item (brute force over pixels)
        off = 0
        toff = 0
        for it, cam in zip(items, cams):
            W, H = cam["width"], cam["height"]
            tx = (W + tile - 1) // tile
            sel = np.nonzero(it["rx"] > 0)[0][:200]
            for i in sel:
                emitted = set((b["keys"][b["vals"] == off + i] >> np.uint64(32)).astype(np.int64) - toff)
                xs = np.arange(W) + 0.5; ys = np.arange(H) + 0.5
                X = xs[np.abs(xs - it["u"][i]) <= it["rx"][i]]; Y = ys[np.abs(ys - it["v"][i]) <= it["ry"][i]]
                need = {int(y // tile) * tx + int(x // tile) for y in Y for x in X}
                assert need <= emitted
            off += it["u"].shape[0]
            toff += tx * ((H + tile - 1) // tile)


def test_sh_colour_uses_plane_k3_plus_c_and_view_direction():
    """Degree-1 colour: only coefficient k=2 (the z term) of the green channel is set, so
    green = 0.5 + sh * sqrt(3/(4 pi)) * dir_z with dir the unit vector from the camera
    centre to the mean, clamped at 0; red and blue stay 0.5."""
    R = _rot([0, 1, 0], 0.3)
    t = np.array([0.2, 0.1, -0.4])
    cam = synth.camera(64, 48, 60.0, R=R, t=t)
    mu = np.array([0.5, 0.2, 3.0])
    for val in (0.7, -3.0):
        sc = _one_gaussian(mu, -3.0, colour=(0.5, 0.5, 0.5), deg=1)
        sc.sh[2 * 3 + 1, 0] = val
        pr = oracle.project(sc, cam)
        cw = -R.T @ t
        d = (mu - cw) / np.linalg.norm(mu - cw)
        g = max(0.0, 0.5 + val * math.sqrt(3 / (4 * math.pi)) * d[2])
        np.testing.assert_allclose(pr["rgb"][0], [0.5, g, 0.5], rtol=1e-13)
