"""Learned initialisation pipeline and its evaluation (host orchestration of the kernels).

RMGS-SLAM §III-B initialises each new segment's Gaussians by a cascade whose first branch
is a learned model.  Here the model is the MLP of include/gs.h, trained on pairs that the
plain mapping loop itself produces:

  features  voxel-PCA features x of each point (gs_voxel_pca)
  init      the cascade without the model (PCA where reliable, else the depth heuristic)
  optimise  the plain loop (gs_step) from that init for a number of iterations
  pairs     (x, residual) with residual = optimised - init in the model's output units:
            log-scale (3), quaternion (4, both with w >= 0), opacity logit (1), colour (3),
            formed by gs_init_residuals

The evaluation compares wall seconds to a held-out PSNR for plain init + one view per step
against learned init + a batch of views per step (§III-C samples several views per
iteration), on scenes not used for training.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass

import numpy as np
import torch

from . import learned
from .core import LR_DEFAULT, MappingStep, Workspace, default_opts, pack_plane, pack_rgb, pixel_offsets

Y00 = 0.28209479177387814
KF_SIZE = (320, 240)


@dataclass
class SceneData:
    gt: torch.Tensor            # ground-truth planes [11 + 3K, n]
    points: torch.Tensor        # [3, n] LiDAR points (noisy copies of the means)
    colours: torch.Tensor       # [3, n]
    train_cams: list
    test_cams: list
    loopframe: dict
    sh_degree: int


def make_scene(seed, n, sh_degree=1, n_kf=32, kind="line", device="cuda"):
    """A LiDAR-shaped scene (synth.lidar_scene) with keyframes along its trajectory: every
    8th keyframe is held out for evaluation."""
    import synth
    sc = synth.lidar_scene(seed=seed, n=n, sh_degree=sh_degree, kind=kind, n_boxes=12)
    n_pose = len(sc.meta["traj_pos"])
    idx = np.linspace(0, n_pose - 1, n_kf).astype(int)
    cams = synth.trajectory_cameras(sc, [KF_SIZE] * n_kf, idx, fx_per_width=0.7)
    test = cams[3::8]
    train = [c for k, c in enumerate(cams) if k % 8 != 3]
    rng = np.random.default_rng(seed + 99)
    pts = sc.means + rng.normal(0, 0.01, sc.means.shape).astype(np.float32)
    cols = np.clip(sc.sh[0:3] * Y00 + 0.5, 0, 1).astype(np.float32)
    gt = torch.as_tensor(sc.planes(), device=device)
    return SceneData(gt, torch.as_tensor(pts, device=device), torch.as_tensor(cols, device=device), train, test,
                     train[len(train) // 2], sh_degree)


def render(planes, sh_degree, cams, tile=16, chunk=64):
    """Colour and depth of `cams` (packed per view) rendered from `planes`."""
    n = planes.shape[1]
    ws = Workspace(n, cams, default_opts(tile=tile, chunk=chunk), max(1 << 20, 64 * n * len(cams)), planes.device)
    P = ws.layout.total_pixels
    rgb = torch.empty(3 * P, device=planes.device)
    dep = torch.empty(P, device=planes.device)
    ws.project(planes, sh_degree)
    ws.bin_sort()
    ws.render_fwd(rgb, dep)
    c = ws.counters()
    if c.status != 0:
        raise RuntimeError(f"render: device status {c.status}")
    return rgb, dep


def psnr(planes, sh_degree, cams, target_rgb):
    rgb, _ = render(planes, sh_degree, cams)
    mse = torch.mean((rgb.clamp(0, 1) - target_rgb) ** 2).item()
    return 10.0 * math.log10(1.0 / max(mse, 1e-12))


def initial_map(sd: SceneData, mlp: learned.MLP | None = None):
    """Cascaded initial map from the scene's points; also returns the PCA outputs."""
    pca = learned.voxel_pca(sd.points, sd.colours, [sd.loopframe] + [c for c in sd.train_cams if c is not sd.loopframe][:31])
    y = mlp.infer(pca["x"]) if mlp is not None else None
    planes, branch, beta = learned.cascade(sd.points, sd.colours, pca, float(sd.loopframe["fx"]), y,
                                           sh_degree=sd.sh_degree)
    return planes, pca, branch


class Optimizer:
    """The mapping loop over a scene's training keyframes, `views` keyframes per step drawn
    at random (the same image size, so one workspace serves every batch)."""

    def __init__(self, planes, sd: SceneData, views, lr=LR_DEFAULT, seed=0, tile=16, chunk=64):
        self.sd = sd
        self.views = views
        self.rng = np.random.default_rng(seed)
        self.targets_rgb, self.targets_dep = render(sd.gt, sd.sh_degree, sd.train_cams)
        self.off = pixel_offsets(sd.train_cams)
        self.px = KF_SIZE[0] * KF_SIZE[1]
        first = list(range(views))
        self.step = MappingStep(planes, sd.sh_degree, [sd.train_cams[i] for i in first],
                                default_opts(tile=tile, chunk=chunk), max_pairs=max(1 << 20, 96 * planes.shape[1] * views),
                                lr=lr)
        self.trgb = torch.empty(3 * self.px * views, device=planes.device)
        self.tdep = torch.empty(self.px * views, device=planes.device)

    def run(self, iters):
        for _ in range(iters):
            sel = self.rng.choice(len(self.sd.train_cams), self.views, replace=False)
            for k, i in enumerate(sel):
                o = self.off[i]
                self.trgb[3 * self.px * k:3 * self.px * (k + 1)] = self.targets_rgb[3 * o:3 * o + 3 * self.px]
                self.tdep[self.px * k:self.px * (k + 1)] = self.targets_dep[o:o + self.px]
            self.step.set_cameras([self.sd.train_cams[i] for i in sel])
            self.step(self.trgb, self.tdep)
        return self.step.planes


def training_pairs(seeds, n, iters=200, views=8, sh_degree=1):
    """(x, y) pairs from the plain loop on the scenes `seeds`."""
    xs, ys = [], []
    for s in seeds:
        sd = make_scene(s, n, sh_degree)
        init, pca, branch = initial_map(sd, None)
        opt = Optimizer(init.clone(), sd, views, seed=s).run(iters)
        x, y = learned.residual_pairs(init, opt, sh_degree, pca)
        xs.append(x)
        ys.append(y)
    return torch.cat(xs), torch.cat(ys)


def train_mlp(x, y, epochs=30, batch=16384, lr=1e-3, seed=0):
    mlp = learned.MLP.init(seed, device=x.device)
    g = torch.Generator(device="cpu").manual_seed(seed)
    losses = []
    for _ in range(epochs):
        perm = torch.randperm(x.shape[0], generator=g).to(x.device)
        for b0 in range(0, x.shape[0], batch):
            idx = perm[b0:b0 + batch]
            mlp.train_step(x[idx], y[idx], lr=lr)
        losses.append(float(mlp.loss))
    return mlp, losses


def seconds_to_psnr(planes, sd: SceneData, views, target_psnr, max_iters, eval_every=25, seed=0):
    """Wall seconds (CUDA-synchronised, evaluation excluded) and iterations until the held-out
    PSNR reaches target_psnr; (inf, max_iters) if it never does."""
    test_rgb, _ = render(sd.gt, sd.sh_degree, sd.test_cams)
    opt = Optimizer(planes, sd, views, seed=seed)
    spent = 0.0
    it = 0
    curve = []
    while it < max_iters:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        opt.run(eval_every)
        torch.cuda.synchronize()
        spent += time.perf_counter() - t0
        it += eval_every
        p = psnr(opt.step.planes, sd.sh_degree, sd.test_cams, test_rgb)
        curve.append((it, spent, p))
        if p >= target_psnr:
            return spent, it, curve
    return math.inf, max_iters, curve


class HeldOutLoss:
    """The mapping objective (L1 colour + depth, gs_render_fwd's fused loss) of a map on the
    scene's held-out keyframes, with one workspace kept across evaluations."""

    def __init__(self, sd: SceneData, n):
        self.target_rgb, self.target_dep = render(sd.gt, sd.sh_degree, sd.test_cams)
        self.ws = Workspace(n, sd.test_cams, default_opts(tile=16, chunk=64), max(1 << 20, 64 * n * len(sd.test_cams)),
                            sd.gt.device)
        P = self.ws.layout.total_pixels
        dev = sd.gt.device
        self.rgb, self.dep = torch.empty(3 * P, device=dev), torch.empty(P, device=dev)
        self.dl, self.dld = torch.empty(3 * P, device=dev), torch.empty(P, device=dev)
        self.loss = torch.empty(len(sd.test_cams) + 1, device=dev)
        self.sh_degree = sd.sh_degree

    def __call__(self, planes) -> float:
        self.ws.project(planes, self.sh_degree)
        self.ws.bin_sort()
        self.ws.render_fwd(self.rgb, self.dep, None, self.target_rgb, self.target_dep, None, self.dl, self.dld,
                           self.loss)
        if self.ws.counters().status != 0:
            raise RuntimeError("held-out render failed")
        return float(self.loss[-1])


def iterations_to_loss(planes, sd: SceneData, views, target_loss, max_iters, eval_every=25, seed=0):
    """Iterations of the plain optimiser (`views` keyframes per step) until the held-out loss
    falls to target_loss (None if it does not within max_iters), and the loss curve."""
    ev = HeldOutLoss(sd, planes.shape[1])
    opt = Optimizer(planes, sd, views, seed=seed)
    curve = []
    it = 0
    while it < max_iters:
        opt.run(eval_every)
        it += eval_every
        lval = ev(opt.step.planes)
        curve.append((it, lval))
        if lval <= target_loss:
            return it, curve
    return None, curve


def final_psnr(planes, sd: SceneData, views, iters, seed=0):
    test_rgb, _ = render(sd.gt, sd.sh_degree, sd.test_cams)
    opt = Optimizer(planes, sd, views, seed=seed)
    opt.run(iters)
    return psnr(opt.step.planes, sd.sh_degree, sd.test_cams, test_rgb)
