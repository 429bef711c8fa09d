"""The view-parallel form of the mapping step: the keyframes of one batch rendered on several
GPUs, one process per GPU.

RMGS-SLAM's optimisation (§III-C) renders a batch of keyframes per iteration and updates the
visible, unfrozen Gaussians.  The batch shards naturally by view: every rank holds a replica
of the map, renders its share of the views forward and backward with the library (gs_step
without the optimiser, so the gradients, the pose twists and the per-Gaussian visibility stay
on the device), and the only exchange is

    gradient planes  summed over the ranks      (one all-reduce of [11 + 3K, n] float32)
    pose twists      summed ([V, 6]; each view's row is non-zero on its own rank only)
    visibility       the union over the ranks   (one all-reduce MAX of n bytes)

after which every rank applies the identical masked Adam update (gs_adam_step) to its replica,
so the replicas stay equal.  The loss weights of a rank holding V_r of the V views are
scaled by V_r / V, so that its gradient is exactly its views' share of the batch gradient
(the step averages its loss over its own views) and the sum over the ranks equals the
gradient of the whole batch.

The collectives are torch.distributed calls on the caller's process group (NCCL between
GPUs); no kernel of the library communicates.
"""
from __future__ import annotations

import ctypes as C

import torch

from . import _native as N
from .core import LR_DEFAULT, MappingStep, _ptr, _stream, default_opts, gaussians_struct


def partition_views(sizes, world: int) -> list[list[int]]:
    """Views of a batch assigned to `world` ranks, balanced by pixel count: views in
    descending size (ties by index) each go to the rank with the fewest pixels so far (ties
    by rank); every rank's list is returned in ascending view order.  sizes: [(W, H), ...]."""
    if world < 1:
        raise ValueError("world must be >= 1")
    if len(sizes) < world:
        raise ValueError(f"{len(sizes)} views cannot be shared by {world} ranks (every rank needs one)")
    load = [0] * world
    parts = [[] for _ in range(world)]
    for v in sorted(range(len(sizes)), key=lambda i: (-sizes[i][0] * sizes[i][1], i)):
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(v)
        load[r] += sizes[v][0] * sizes[v][1]
    return [sorted(p) for p in parts]


def allreduce_step_state(grads: torch.Tensor, twist: torch.Tensor, visible: torch.Tensor, group=None):
    """Sums the gradient planes and the twists and takes the union of the visibility flags
    over the ranks of `group`, in place."""
    import torch.distributed as dist
    dist.all_reduce(grads, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(twist, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(visible, op=dist.ReduceOp.MAX, group=group)


class ViewParallelStep:
    """One mapping step of a V-view batch sharded over the ranks of `group` (see the module
    docstring).  Every rank constructs it with the same replica `planes` [11 + 3K, n], the
    same V cameras and the same options; it renders views partition_views(...)[rank].

    __call__(target_rgb, target_depth, mask, update_mask): this rank's packed targets (its
    views, in ascending view order) -> the rank's loss share [V_r + 1] on the device (the last
    entry summed over the ranks is the batch loss); the replica and the Adam moments are
    updated in place and `twist` [V, 6] holds the batch's pose gradients."""

    def __init__(self, planes: torch.Tensor, sh_degree: int, cams, opts: N.RenderOpts | None = None,
                 max_pairs: int | None = None, lr=LR_DEFAULT, b1=0.9, b2=0.999, eps=1e-15, group=None):
        import torch.distributed as dist
        self.group = group
        self.world = dist.get_world_size(group) if dist.is_initialized() else 1
        self.rank = dist.get_rank(group) if dist.is_initialized() else 0
        self.V = len(cams)
        self.views = partition_views([(c["width"], c["height"]) for c in cams], self.world)[self.rank]
        base = opts or default_opts()
        o = default_opts()
        C.memmove(C.byref(o), C.byref(base), C.sizeof(o))
        share = len(self.views) / self.V
        o.lambda_rgb = base.lambda_rgb * share
        o.lambda_depth = base.lambda_depth * share
        self.step = MappingStep(planes, sh_degree, [cams[i] for i in self.views], o, max_pairs, lr, b1, b2, eps)
        self.sh_degree = sh_degree
        self.lr, self.b1, self.b2, self.eps = tuple(lr), b1, b2, eps
        self.twist = torch.zeros(self.V, 6, device=planes.device)
        self.adam_t = 0

    @property
    def planes(self):
        return self.step.planes

    def set_cameras(self, cams):
        """New poses for the batch (same image sizes); the rank keeps its views."""
        self.step.set_cameras([cams[i] for i in self.views])

    def __call__(self, target_rgb, target_depth=None, mask=None, update_mask=None):
        s = self.step
        r = s(target_rgb, target_depth, mask, update_mask=None, optimize=False, with_twist=True)
        self.twist.zero_()
        self.twist[self.views] = s.twist
        visible = s.ws.visible().clone()
        if self.world > 1:
            allreduce_step_state(s.grads, self.twist, visible, self.group)
        self.adam_t += 1
        gp, gg, gm, gv = (gaussians_struct(t, self.sh_degree) for t in (s.planes, s.grads, s.m, s.v))
        lrs = (C.c_float * 6)(*self.lr)
        N.check(N.lib().gs_adam_step(C.byref(gp), C.byref(gg), C.byref(gm), C.byref(gv), _ptr(update_mask),
                                     _ptr(visible), lrs, self.b1, self.b2, self.eps, self.adam_t, _stream()),
                "gs_adam_step")
        return r.loss
