"""Binding of the learned Gaussian initialiser (include/gs.h a10-a12): voxel-PCA features,
the BF16 MLP (inference and training) and the cascaded initialisation of §III-B, over
PyTorch device memory.  Marshalling only; every step runs in libgs.so's kernels."""
from __future__ import annotations

import ctypes as C
import math

import numpy as np
import torch

from . import _native as N
from .core import _ptr, _stream, camera_array, gaussians_struct, n_planes

N_W, N_B = 36864, 400
LAYERS = [(128, 16), (128, 128), (128, 128), (16, 128)]


def pca_opts(voxel=0.5, min_pts=5, tau_p=2.5e-3, tau_l=10.0, sigma=0.02, tau_trace=1e-2) -> N.PcaOpts:
    return N.PcaOpts(voxel, min_pts, tau_p, tau_l, sigma, tau_trace)


def voxel_pca(points: torch.Tensor, colours: torch.Tensor, frames, opts: N.PcaOpts | None = None):
    """points, colours: [3, n] float32 CUDA; frames: one camera dict or a list (<= 32, the
    segment's loopframes / keyframes).  Returns a dict of per-point device tensors."""
    frames = [frames] if isinstance(frames, dict) else list(frames)
    opts = opts or pca_opts()
    n = points.shape[1]
    dev = points.device
    ws = torch.empty(int(N.lib().gs_pca_workspace_size(n)), dtype=torch.uint8, device=dev)
    out = dict(x=torch.empty(n, 16, device=dev), has_feature=torch.empty(n, dtype=torch.uint8, device=dev),
               reliable=torch.empty(n, dtype=torch.uint8, device=dev), s_pca=torch.empty(n, 3, device=dev),
               q_pca=torch.empty(n, 4, device=dev), depth=torch.empty(n, device=dev),
               inside=torch.empty(n, dtype=torch.uint8, device=dev))
    cam = camera_array(frames)
    N.check(N.lib().gs_voxel_pca(_ptr(points.contiguous()), _ptr(colours.contiguous()), n, cam, len(frames),
                                 C.byref(opts), _ptr(ws),
                                 ws.numel(), *[_ptr(out[k]) for k in ("x", "has_feature", "reliable", "s_pca", "q_pca",
                                                                      "depth", "inside")], _stream()), "gs_voxel_pca")
    return out


def pack_params(Ws, bs, device="cuda"):
    """Oracle-format lists (W_l [out, in], b_l) -> FP32 master weights [36864], biases [400]."""
    w = torch.cat([torch.as_tensor(np.asarray(W), dtype=torch.float32).reshape(-1) for W in Ws]).to(device)
    b = torch.cat([torch.as_tensor(np.asarray(x), dtype=torch.float32).reshape(-1) for x in bs]).to(device)
    assert w.numel() == N_W and b.numel() == N_B
    return w, b


class MLP:
    """The initialiser network: FP32 master weights, their BF16 copy, biases, Adam state."""

    def __init__(self, w_master: torch.Tensor, bias: torch.Tensor):
        self.w = w_master.contiguous().clone()
        self.b = bias.contiguous().clone()
        self.wq = self.w.to(torch.bfloat16)
        dev = self.w.device
        self.gw = torch.zeros(N_W, device=dev)
        self.gb = torch.zeros(N_B, device=dev)
        self.m = torch.zeros(N_W + N_B, device=dev)
        self.v = torch.zeros(N_W + N_B, device=dev)
        self.t = 0
        self._scratch = None
        self.loss = torch.zeros(1, device=dev)

    @staticmethod
    def init(seed=0, device="cuda"):
        rng = np.random.default_rng(seed)
        Ws = [rng.normal(0, math.sqrt(2.0 / i), (o, i)) for o, i in LAYERS]
        Ws[-1] *= 0.1
        bs = [np.zeros(o) for o, _ in LAYERS]
        return MLP(*pack_params(Ws, bs, device))

    def infer(self, x: torch.Tensor) -> torch.Tensor:
        n = x.shape[0]
        y = torch.empty(n, 16, device=x.device)
        N.check(N.lib().gs_mlp_infer(_ptr(self.wq), _ptr(self.b), _ptr(x.contiguous()), n, _ptr(y), _stream()),
                "gs_mlp_infer")
        return y

    def train_step(self, x, y_target, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        n = x.shape[0]
        need = int(N.lib().gs_mlp_train_scratch_size(n))
        if self._scratch is None or self._scratch.numel() < need:
            self._scratch = torch.empty(need, dtype=torch.uint8, device=x.device)
        self.t += 1
        N.check(N.lib().gs_mlp_train_step(_ptr(self.w), _ptr(self.wq), _ptr(self.b), _ptr(self.gw), _ptr(self.gb),
                                          _ptr(self.m), _ptr(self.v), _ptr(x.contiguous()), _ptr(y_target.contiguous()),
                                          n, lr, b1, b2, eps, self.t, _ptr(self._scratch), self._scratch.numel(),
                                          _ptr(self.loss), _stream()), "gs_mlp_train_step")
        return self.loss


def residual_pairs(init: torch.Tensor, opt: torch.Tensor, sh_degree: int, pca):
    """Training pairs (x [k, 16], y [k, 16]) of the initialiser: the features and the
    optimised-minus-initial residuals of the rows with a voxel feature inside the loopframe
    (gs_init_residuals)."""
    n = init.shape[1]
    dev = init.device
    gi, go = gaussians_struct(init.contiguous(), sh_degree), gaussians_struct(opt.contiguous(), sh_degree)
    x_out = torch.empty(max(n, 1), 16, device=dev)
    y_out = torch.empty(max(n, 1), 16, device=dev)
    scratch = torch.empty(int(N.lib().gs_init_residuals_scratch_bytes(n)), dtype=torch.uint8, device=dev)
    k = C.c_int64()
    N.check(N.lib().gs_init_residuals(C.byref(gi), C.byref(go), _ptr(pca["x"].contiguous()), _ptr(pca["has_feature"]),
                                      _ptr(pca["inside"]), _ptr(x_out), _ptr(y_out), C.byref(k), _ptr(scratch),
                                      scratch.numel(), _stream()), "gs_init_residuals")
    return x_out[:k.value], y_out[:k.value]


def cascade(points, colours, pca, fx, y=None, sh_degree=3, opacity_init=0.1):
    """Initial Gaussian map [11 + 3K, n] by the cascade; returns (planes, branch, beta)."""
    n = points.shape[1]
    dev = points.device
    planes = torch.zeros(n_planes(sh_degree), n, device=dev)
    g = gaussians_struct(planes, sh_degree)
    branch = torch.empty(n, dtype=torch.int32, device=dev)
    tmp = torch.zeros(1, dtype=torch.int32, device=dev)
    beta = torch.zeros(1, device=dev)
    N.check(N.lib().gs_init_cascade(_ptr(points.contiguous()), _ptr(colours.contiguous()), n,
                                    _ptr(y.contiguous()) if y is not None else None, _ptr(pca["has_feature"]),
                                    _ptr(pca["reliable"]), _ptr(pca["s_pca"].contiguous()),
                                    _ptr(pca["q_pca"].contiguous()), _ptr(pca["depth"]), _ptr(pca["inside"]), fx,
                                    opacity_init, C.byref(g), _ptr(branch), _ptr(tmp), _ptr(beta), _stream()),
            "gs_init_cascade")
    return planes, branch, beta
