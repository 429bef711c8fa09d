"""FP64 oracle of the learned Gaussian initialiser -- TEST INFRASTRUCTURE ONLY.

RMGS-SLAM §III-A/B initialises one Gaussian per LiDAR point by a cascade: a learned
model's prediction where it is valid, else the voxel-PCA prior where it is geometrically
reliable, else an isotropic depth heuristic.  The paper's model branch is a pretrained
feed-forward network that is not available; here it is a small MLP over the voxel-PCA
features (16 -> 128 -> 128 -> 128 -> 16, GELU, BF16 weights and activations, FP32
accumulation on the GPU).  This module restates, in double precision:

  features()     per-point input x = [ln lambda (3), V (9, row-major), rgb (3), ln(d/f)]
  mlp_forward()  the network with BF16-rounded weights, input and hidden activations
  mlp_backward() mean-squared-error gradients of every weight and bias
  adam()         Adam on FP32 master weights
  cascade()      the three-way choice and the initial parameters (§III-B equations)
  residual_pairs() the model's training targets: optimised minus initial parameters of the
                 rows with a feature inside the loopframe, in the model's output units

Readings (the paper is silent): lambda is floored at (0.01 m)^2 before the logarithm;
the model output is a residual added to the PCA initialisation (log-scale, quaternion
components, opacity logit, colour); a prediction is valid where the point's voxel has a
feature (>= 5 points), the point projects inside the loopframe at positive depth, the output
is finite and every |log-scale residual| < 3; beta = clamp(#(reliable and not valid)/#points,
0.25, 1); constant initial opacity 0.1; higher SH zero; quaternion (w, x, y, z) with w >= 0.
"""
from __future__ import annotations

import math

import numpy as np

D_IN, D_HID, D_OUT, N_OUT_USED = 16, 128, 16, 11
LAMBDA_FLOOR = 1e-4
OPACITY_INIT = 0.1
Y00 = 0.5 / math.sqrt(math.pi)


def bf16(x):
    """Round to bfloat16 (round to nearest, ties to even) and return as float64."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def gelu(z):
    from scipy.special import erf
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    from scipy.special import erf
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def init_weights(seed):
    """He-style initialisation: W_l ~ N(0, 2/fan_in), b = 0; layer shapes (out, in)."""
    rng = np.random.default_rng(seed)
    dims = [(D_HID, D_IN), (D_HID, D_HID), (D_HID, D_HID), (D_OUT, D_HID)]
    Ws = [rng.normal(0, math.sqrt(2.0 / i), (o, i)) for o, i in dims]
    Ws[-1] *= 0.1                      # small initial residuals
    bs = [np.zeros(o) for o, _ in dims]
    return Ws, bs


def mlp_forward(x, Ws, bs, round_bf16=True):
    """Returns (y [n, 16], cache).  With round_bf16 the input, the weights and every hidden
    activation are rounded to BF16 (the GPU keeps them in BF16); sums are exact here."""
    r = bf16 if round_bf16 else (lambda v: np.asarray(v, np.float64))
    a = r(x)
    cache = {"a": [a], "z": []}
    for l, (W, b) in enumerate(zip(Ws, bs)):
        z = a @ r(W).T + b
        cache["z"].append(z)
        if l < len(Ws) - 1:
            a = r(gelu(z))
            cache["a"].append(a)
        else:
            a = z
    return a, cache


def mse_loss(y, t):
    d = y[:, :N_OUT_USED] - t[:, :N_OUT_USED]
    return float((d * d).sum() / (y.shape[0] * N_OUT_USED))


def mlp_backward(y, t, cache, Ws, round_bf16=True):
    """Gradients of mse_loss w.r.t. every W (out, in) and b."""
    r = bf16 if round_bf16 else (lambda v: np.asarray(v, np.float64))
    n = y.shape[0]
    g = np.zeros_like(y)
    g[:, :N_OUT_USED] = 2.0 * (y[:, :N_OUT_USED] - t[:, :N_OUT_USED]) / (n * N_OUT_USED)
    gW = [None] * len(Ws)
    gb = [None] * len(Ws)
    for l in reversed(range(len(Ws))):
        a_prev = cache["a"][l]
        gW[l] = g.T @ a_prev
        gb[l] = g.sum(0)
        if l > 0:
            ga = g @ r(Ws[l])
            g = ga * gelu_grad(cache["z"][l - 1])
    return gW, gb


def adam(params, grads, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    out = []
    for p, g, mm, vv in zip(params, grads, m, v):
        mm[:] = b1 * mm + (1 - b1) * g
        vv[:] = b2 * vv + (1 - b2) * g * g
        mh = mm / (1 - b1 ** step)
        vh = vv / (1 - b2 ** step)
        out.append(p - lr * mh / (np.sqrt(vh) + eps))
    return out


def quat_from_matrix(R):
    """Unit quaternion (w, x, y, z), w >= 0, of a rotation matrix (Shepperd's method)."""
    R = np.asarray(R, np.float64)
    tr = R[0, 0] + R[1, 1] + R[2, 2]
    cands = [1 + tr, 1 + R[0, 0] - R[1, 1] - R[2, 2], 1 - R[0, 0] + R[1, 1] - R[2, 2], 1 - R[0, 0] - R[1, 1] + R[2, 2]]
    k = int(np.argmax(cands))
    s = 2.0 * math.sqrt(max(cands[k], 1e-300))
    if k == 0:
        q = [0.25 * s, (R[2, 1] - R[1, 2]) / s, (R[0, 2] - R[2, 0]) / s, (R[1, 0] - R[0, 1]) / s]
    elif k == 1:
        q = [(R[2, 1] - R[1, 2]) / s, 0.25 * s, (R[0, 1] + R[1, 0]) / s, (R[0, 2] + R[2, 0]) / s]
    elif k == 2:
        q = [(R[0, 2] - R[2, 0]) / s, (R[0, 1] + R[1, 0]) / s, 0.25 * s, (R[1, 2] + R[2, 1]) / s]
    else:
        q = [(R[1, 0] - R[0, 1]) / s, (R[0, 2] + R[2, 0]) / s, (R[1, 2] + R[2, 1]) / s, 0.25 * s]
    q = np.asarray(q)
    q /= np.linalg.norm(q)
    return q if q[0] >= 0 else -q


def point_depth(points, cams):
    """Per point ([3, n] world): the camera-frame depth in the closest of `cams` (a camera or a
    list: the segment's loopframes / keyframes) whose image it projects into at positive
    depth -- the closer view of §III-B -- and whether there is one; if none, the depth in the
    first camera."""
    cams = [cams] if isinstance(cams, dict) else list(cams)
    n = np.asarray(points).shape[1]
    best = np.full(n, np.inf)
    first = None
    for cam in cams:
        R, t = np.asarray(cam["R"], np.float64), np.asarray(cam["t"], np.float64)
        pc = R @ np.asarray(points, np.float64) + t[:, None]
        z = pc[2]
        if first is None:
            first = z
        with np.errstate(divide="ignore", invalid="ignore"):
            u = cam["fx"] * pc[0] / z + cam["cx"]
            v = cam["fy"] * pc[1] / z + cam["cy"]
        ins = (z > 0) & (u >= 0) & (u < cam["width"]) & (v >= 0) & (v < cam["height"])
        best = np.where(ins & (z < best), z, best)
    inside = np.isfinite(best)
    return np.where(inside, best, first), inside


def features(pca, colours, depth, fx):
    """x [n, 16] from the voxel-PCA outputs (oracle.voxel_pca dict), point colours [3, n] and
    loopframe depths; rows without a voxel feature are zero."""
    n = colours.shape[1]
    x = np.zeros((n, D_IN))
    has = pca["has_feature"]
    lam = np.maximum(pca["lam"], LAMBDA_FLOOR)
    x[:, 0:3] = np.log(lam)
    x[:, 3:12] = pca["V"]
    x[:, 12:15] = np.asarray(colours, np.float64).T
    x[:, 15] = np.log(np.maximum(depth, 1e-6) / fx)
    x[~has] = 0.0
    return x


def cascade(points, colours, pca, depth, inside, fx, y=None):
    """Initial Gaussian parameters by the three-way cascade (§III-B equations):
    model where the prediction y [n, 16] is valid, else PCA (s_pca + log beta, R_pca) where
    reliable, else heuristic (log(d/f) isotropic, identity rotation).  Returns a dict with
    log_scales [3, n], quats [4, n], opacity_logits [n], dc [3, n] (SH DC coefficients), the
    branch per point (2 model, 1 pca, 0 heuristic) and beta."""
    n = colours.shape[1]
    has = pca["has_feature"]
    rel = pca["reliable"].astype(bool)
    lam = np.maximum(pca["lam"], LAMBDA_FLOOR)
    s_pca = 0.5 * np.log(lam)                                      # log sqrt(lambda), [n, 3]
    q_pca = np.stack([quat_from_matrix(pca["V"][i].reshape(3, 3)) if has[i] else np.array([1.0, 0, 0, 0])
                      for i in range(n)])
    s_heur = np.log(np.maximum(depth, 1e-6) / fx)
    valid = np.zeros(n, bool)
    if y is not None:
        finite = np.all(np.isfinite(y[:, :N_OUT_USED]), axis=1)
        small = np.all(np.abs(np.nan_to_num(y[:, 0:3], nan=1e9)) < 3.0, axis=1)
        valid = has & inside & finite & small
    beta = float(np.clip(np.sum(rel & ~valid) / max(n, 1), 0.25, 1.0))
    logit0 = math.log(OPACITY_INIT / (1 - OPACITY_INIT))
    ls = np.zeros((n, 3)); q = np.zeros((n, 4)); lo = np.full(n, logit0)
    col = np.asarray(colours, np.float64).T.copy()
    branch = np.zeros(n, np.int32)
    for i in range(n):
        if valid[i]:
            ls[i] = s_pca[i] + y[i, 0:3]
            qq = q_pca[i] + y[i, 3:7]
            q[i] = qq / np.linalg.norm(qq)
            lo[i] = logit0 + y[i, 7]
            col[i] = col[i] + y[i, 8:11]
            branch[i] = 2
        elif rel[i]:
            ls[i] = s_pca[i] + math.log(beta)
            q[i] = q_pca[i]
            branch[i] = 1
        else:
            ls[i] = s_heur[i]
            q[i] = [1.0, 0, 0, 0]
    return dict(log_scales=ls.T, quats=q.T, opacity_logits=lo, dc=((col - 0.5) / Y00).T, branch=branch,
                beta=beta, valid=valid)


def _unit_w_nonneg(q):
    """Quaternions [4, n] (w, x, y, z) normalised, then negated where w < 0 (q and -q are the
    same rotation; the w >= 0 form makes the residual between two of them well defined)."""
    q = np.asarray(q, np.float64)
    u = q / np.linalg.norm(q, axis=0, keepdims=True)
    return np.where(u[0:1] < 0, -u, u)


def residual_pairs(init, opt, x, has_feature=None, inside=None):
    """Training pairs of the initialiser from one run of the plain loop: for the rows with a
    voxel feature that lie inside the loopframe, in row order, the features x and the target
    y [k, 16] = (log-scale_opt - log-scale_init (3), unit_w>=0(q_opt) - unit_w>=0(q_init) (4),
    logit_opt - logit_init, (SH DC_opt - SH DC_init) * Y00 (3, colour units), 0 (5)).
    init, opt: parameter planes [11 + 3K, n] (means, log-scales, quaternion, logit, SH)."""
    init = np.asarray(init, np.float64)
    opt = np.asarray(opt, np.float64)
    n = init.shape[1]
    keep = np.ones(n, bool)
    if has_feature is not None:
        keep &= np.asarray(has_feature) != 0
    if inside is not None:
        keep &= np.asarray(inside) != 0
    y = np.zeros((n, 16))
    y[:, 0:3] = (opt[3:6] - init[3:6]).T
    y[:, 3:7] = (_unit_w_nonneg(opt[6:10]) - _unit_w_nonneg(init[6:10])).T
    y[:, 7] = opt[10] - init[10]
    y[:, 8:11] = ((opt[11:14] - init[11:14]) * Y00).T
    return np.asarray(x, np.float64)[keep], y[keep]
