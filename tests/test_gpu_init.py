"""Learned-initialiser kernels (voxel-PCA, MLP inference / training, cascade) against the
FP64 oracle on the same seeded inputs."""
import math

import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import init_model as im
from paper_2604_12942_gb300 import learned

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def scene():
    sc = synth.lidar_scene(seed=7, n=40_000, sh_degree=0, kind="line", n_boxes=8)
    cams = synth.trajectory_cameras(sc, [(320, 240)] * 3, [60, 100, 140])
    colours = np.clip(sc.sh[0:3] * im.Y00 + 0.5, 0, 1).astype(np.float32)
    return sc.means.astype(np.float32), colours, cams


def test_voxel_pca_matches_oracle(scene):
    pts, cols, cams = scene
    cam = cams[0]
    g = learned.voxel_pca(torch.as_tensor(pts).cuda(), torch.as_tensor(cols).cuda(), cams)
    ref = oracle.voxel_pca(pts)
    depth, inside = im.point_depth(pts, cams)
    has = g["has_feature"].cpu().numpy().astype(bool)
    np.testing.assert_array_equal(has, ref["has_feature"])
    assert has.sum() > 0.5 * len(has)
    # FP32 p_c = R p + t with coordinates of 50-100 m: absolute depth error up to a few 1e-4 m
    np.testing.assert_allclose(g["depth"].cpu().numpy(), depth, rtol=0, atol=1e-3)
    # visibility decided in FP32 on the GPU: only points within rounding of an image edge differ
    assert np.mean(g["inside"].cpu().numpy().astype(bool) != inside) < 1e-3
    x = g["x"].cpu().numpy()
    lam = ref["lam"]
    lmax = lam[:, 2:3]
    # eigenvalues (through the features' ln max(lambda, 1e-4)) where the floor is not active
    xl = np.log(np.maximum(lam, 1e-4))
    ok = has[:, None] & (lam > 2e-4)
    assert np.max(np.abs(x[:, 0:3] - xl)[ok]) < 2e-3
    # eigenvectors where the eigen-gaps are clear and the sign choice is not a near tie
    gaps = np.minimum(lam[:, 1] - lam[:, 0], lam[:, 2] - lam[:, 1]) / np.maximum(lmax[:, 0], 1e-30)
    V = ref["V"].reshape(-1, 3, 3)
    Vg = x[:, 3:12].reshape(-1, 3, 3)
    srt = np.sort(np.abs(V), axis=1)
    clear_sign = (srt[:, 2, :] - srt[:, 1, :]) > 1e-2
    sel = has & (gaps > 1e-2) & clear_sign[:, 0] & clear_sign[:, 1]
    assert sel.sum() > 0.3 * has.sum()
    assert np.max(np.abs(Vg[sel] - V[sel])) < 5e-3
    np.testing.assert_array_equal(x[has, 12:15], cols.T[has])
    # ln(d / f) where the depth is not itself lost to FP32 cancellation (|d| >> 1e-3 m)
    far = has & (depth > 0.5)
    np.testing.assert_allclose(x[far, 15], np.log(depth / cam["fx"])[far], atol=2e-4)
    # classification / reliability, away from their thresholds
    o = oracle.VOXEL_DEFAULTS
    ratio = lam[:, 2] / np.maximum(lam[:, 0], 1e-30)
    near = (np.abs(lam[:, 0] / o["tau_p"] - 1) < 1e-2) | (np.abs(ratio / o["tau_l"] - 1) < 1e-2) | \
           (np.abs(ref["trace"] / o["tau_trace"] - 1) < 1e-2) | (gaps < 1e-4)
    rel_g = g["reliable"].cpu().numpy().astype(bool)
    rel_o = ref["reliable"].astype(bool)
    m = has & ~near
    np.testing.assert_array_equal(rel_g[m], rel_o[m])
    assert rel_o[m].sum() > 100
    # quaternion of V where V is compared
    qg = g["q_pca"].cpu().numpy()
    for i in np.nonzero(sel)[0][:300]:
        np.testing.assert_allclose(qg[i], im.quat_from_matrix(V[i]), atol=1e-2)


def _weights(seed):
    Ws, bs = im.init_weights(seed)
    rng = np.random.default_rng(seed + 1)
    bs = [rng.normal(0, 0.1, b.shape) for b in bs]
    return Ws, bs


def test_mlp_infer_matches_oracle():
    Ws, bs = _weights(11)
    w, b = learned.pack_params(Ws, bs)
    mlp = learned.MLP(w, b)
    rng = np.random.default_rng(12)
    x = rng.normal(size=(1000, 16)).astype(np.float32)        # 1000 rows: several CTAs and a ragged tail
    # same BF16-rounded weights on both sides
    Wq = [im.bf16(W) for W in Ws]
    y_ref, _ = im.mlp_forward(x, Wq, [np.float32(b_) for b_ in bs], round_bf16=True)
    y = mlp.infer(torch.as_tensor(x).cuda()).cpu().numpy()
    err = np.abs(y - y_ref).max() / np.abs(y_ref).max()
    # hidden activations are rounded to BF16 on both sides; FP32 vs FP64 sums can move a
    # rounding decision by one BF16 ulp (2^-8 relative)
    assert err < 1e-2, err
    assert np.corrcoef(y.ravel(), y_ref.ravel())[0, 1] > 0.9999


def test_mlp_train_step_gradients_match_oracle():
    """With lr = eps = 1e6 the first Adam step moves every parameter by -g / (1 + |g|/1e6),
    i.e. by -g: the parameter change reads out the GPU gradient."""
    Ws, bs = _weights(21)
    w, b = learned.pack_params(Ws, bs)
    mlp = learned.MLP(w, b)
    rng = np.random.default_rng(22)
    x = rng.normal(size=(700, 16)).astype(np.float32)
    t = rng.normal(size=(700, 16)).astype(np.float32)
    w0, b0 = mlp.w.clone(), mlp.b.clone()
    loss = mlp.train_step(torch.as_tensor(x).cuda(), torch.as_tensor(t).cuda(), lr=1e6, eps=1e6)
    torch.cuda.synchronize()
    gw = -(mlp.w - w0).cpu().numpy().astype(np.float64)
    gb = -(mlp.b - b0).cpu().numpy().astype(np.float64)
    Wq = [im.bf16(W) for W in Ws]
    bq = [np.float32(b_) for b_ in bs]
    y, cache = im.mlp_forward(x, Wq, bq, round_bf16=True)
    gW_ref, gb_ref = im.mlp_backward(y, t, cache, Wq, round_bf16=True)
    assert abs(float(loss) - im.mse_loss(y, t)) < 1e-2 * im.mse_loss(y, t)
    off = 0
    for l, (o, i) in enumerate(learned.LAYERS):
        g = gw[off:off + o * i].reshape(o, i)
        off += o * i
        e = np.linalg.norm(g - gW_ref[l]) / np.linalg.norm(gW_ref[l])
        # BF16 operands of the backward GEMMs: relative L2 of the gradient within 2e-2
        assert e < 2e-2, (l, e)
    offb = 0
    for l, (o, _) in enumerate(learned.LAYERS):
        e = np.linalg.norm(gb[offb:offb + o] - gb_ref[l]) / np.linalg.norm(gb_ref[l])
        offb += o
        assert e < 2e-2, ("bias", l, e)


def test_mlp_training_fits_a_target_network():
    Wt, bt = _weights(31)
    rng = np.random.default_rng(32)
    x = rng.normal(size=(4096, 16)).astype(np.float32)
    t, _ = im.mlp_forward(x, Wt, bt, round_bf16=False)
    mlp = learned.MLP.init(33)
    xd, td = torch.as_tensor(x).cuda(), torch.as_tensor(t.astype(np.float32)).cuda()
    losses = [float(mlp.train_step(xd, td, lr=2e-3)) for _ in range(150)]
    assert losses[-1] < 0.2 * losses[0], (losses[0], losses[-1])


def test_cascade_matches_oracle():
    rng = np.random.default_rng(41)
    n = 3000
    pts = (rng.normal(size=(3, n)) * [[3], [1], [2]] + [[0], [0], [6]]).astype(np.float32)
    cols = rng.uniform(0, 1, (3, n)).astype(np.float32)
    lam = np.sort(rng.uniform(1e-5, 1e-2, (n, 3)), axis=1)
    Vs = []
    for _ in range(n):
        Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        Q[:, 2] = np.cross(Q[:, 0], Q[:, 1])
        Vs.append(Q)
    V = np.stack(Vs)
    has = rng.uniform(size=n) < 0.8
    rel = (rng.uniform(size=n) < 0.6) & has
    depth = rng.uniform(1, 20, n)
    inside = rng.uniform(size=n) < 0.85
    y = rng.normal(0, 0.3, (n, 16))
    y[rng.uniform(size=n) < 0.05, 0] = 5.0           # invalid: |log-scale residual| >= 3
    y[rng.uniform(size=n) < 0.02, 4] = np.nan        # invalid: non-finite
    pca = dict(has_feature=has, reliable=rel.astype(np.int32), lam=lam, V=V.reshape(n, 9))
    ref = im.cascade(pts, cols, pca, depth, inside, 300.0, y)
    # GPU inputs: the same synthetic PCA outputs in the library's per-point form
    s_pca = 0.5 * np.log(np.maximum(lam, im.LAMBDA_FLOOR))
    q_pca = np.stack([im.quat_from_matrix(V[i]) if has[i] else np.array([1.0, 0, 0, 0]) for i in range(n)])
    dev = lambda a, dt=torch.float32: torch.as_tensor(np.ascontiguousarray(a)).to(dt).cuda()
    gp = dict(has_feature=dev(has, torch.uint8), reliable=dev(rel, torch.uint8), s_pca=dev(s_pca), q_pca=dev(q_pca),
              depth=dev(depth), inside=dev(inside, torch.uint8))
    planes, branch, beta = learned.cascade(dev(pts), dev(cols), gp, 300.0, dev(y), sh_degree=1)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(branch.cpu().numpy(), ref["branch"])
    assert float(beta) == pytest.approx(ref["beta"], rel=1e-6)
    P = planes.cpu().numpy()
    np.testing.assert_array_equal(P[0:3], pts)
    np.testing.assert_allclose(P[3:6], ref["log_scales"], atol=2e-5)
    np.testing.assert_allclose(P[6:10], ref["quats"], atol=2e-5)
    np.testing.assert_allclose(P[10], ref["opacity_logits"], atol=2e-5)
    np.testing.assert_allclose(P[11:14], ref["dc"], atol=2e-5)
    assert np.all(P[14:] == 0)


@pytest.mark.parametrize("n,deg", [(5003, 1), (70_001, 3), (1, 0), (0, 1)])
def test_residual_pairs_match_oracle(n, deg):
    """gs_init_residuals (training pairs of the initialiser) against the oracle: the kept rows
    (feature and inside flags) in row order bit-exactly, the residuals within FP32 rounding;
    quaternions with either sign of w, ragged sizes, a single row and none."""
    rng = np.random.default_rng(n + deg)
    P = 11 + 3 * (deg + 1) ** 2
    init = rng.normal(size=(P, n)).astype(np.float32)
    opt = (init + 0.3 * rng.normal(size=(P, n))).astype(np.float32)
    flip = rng.uniform(size=n) < 0.5
    opt[6:10, flip] *= -1.7                                  # same rotation, other sign and norm
    x = rng.normal(size=(n, 16)).astype(np.float32)
    has = (rng.uniform(size=n) < 0.8).astype(np.uint8)
    ins = (rng.uniform(size=n) < 0.7).astype(np.uint8)
    pca = {"x": torch.as_tensor(x).cuda(), "has_feature": torch.as_tensor(has).cuda(),
           "inside": torch.as_tensor(ins).cuda()}
    xg, yg = learned.residual_pairs(torch.as_tensor(init).cuda(), torch.as_tensor(opt).cuda(), deg, pca)
    xr, yr = im.residual_pairs(init, opt, x, has, ins)
    assert xg.shape[0] == xr.shape[0] == int(((has != 0) & (ins != 0)).sum())
    np.testing.assert_array_equal(xg.cpu().numpy(), xr.astype(np.float32))
    if n:
        np.testing.assert_allclose(yg.cpu().numpy(), yr, rtol=0, atol=2e-6)
