"""GB300-native (sm_103a) differentiable 3D Gaussian splatting mapping step of RMGS-SLAM
(arXiv 2604.12942, §III-C): EWA projection with SH colour, (tile, depth) radix sort,
front-to-back compositing of colour and depth, L1 photometric + depth loss, analytic
backward including keyframe SE(3) pose twists, and a masked Adam step -- hand-written CUDA
behind the C ABI of include/gs.h, driven from PyTorch device memory and streams.
"""
from .core import (LR_DEFAULT, MappingStep, RenderFn, Renderer, StepResult, Workspace, adam_step, camera_array, default_opts,
                   dedup_plan, gaussians_struct, gicp_register, gicp_scratch, gicp_target_set, map_update, map_update_scratch, n_planes, pack_plane, pack_rgb,
                   pixel_offsets, prune_plan, unpack_plane, unpack_rgb)

__all__ = ["LR_DEFAULT", "MappingStep", "RenderFn", "Renderer", "StepResult", "Workspace", "adam_step", "camera_array", "default_opts",
           "dedup_plan", "gaussians_struct", "gicp_register", "gicp_scratch", "gicp_target_set", "map_update", "map_update_scratch", "n_planes", "pack_plane", "pack_rgb",
           "pixel_offsets", "prune_plan", "unpack_plane", "unpack_rgb"]
from .viewshard import ViewParallelStep, allreduce_step_state, partition_views  # noqa: E402

__all__ += ["ViewParallelStep", "allreduce_step_state", "partition_views"]
