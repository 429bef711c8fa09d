"""ctypes view of include/gs.h: the structures and the entry points of libgs.so.

Argument marshalling only -- every step of the mapping step runs in the CUDA kernels of
libgs.so.  Loading fails loudly if the library has not been built; there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libgs.so")

MAX_VIEWS = 32
STATUS = {0: "GS_OK", 1: "GS_ERR_INVALID_ARG", 2: "GS_ERR_CUDA", 3: "GS_ERR_CAPACITY", 4: "GS_ERR_TIMEOUT",
          5: "GS_ERR_NONFINITE", 6: "GS_ERR_UNSUPPORTED"}


class Camera(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("R_cw", C.c_float * 9), ("t_cw", C.c_float * 3)]


class Gaussians(C.Structure):
    _fields_ = [("n", C.c_int64), ("sh_degree", C.c_int32), ("means", C.c_void_p), ("log_scales", C.c_void_p),
                ("quats", C.c_void_p), ("opacity_logits", C.c_void_p), ("sh", C.c_void_p)]


class RenderOpts(C.Structure):
    _fields_ = [("near_z", C.c_float), ("dilation", C.c_float), ("alpha_min", C.c_float), ("alpha_max", C.c_float),
                ("T_min", C.c_float), ("clamp_fov", C.c_float), ("bg", C.c_float * 3), ("lambda_rgb", C.c_float),
                ("lambda_depth", C.c_float), ("tile", C.c_int32), ("chunk", C.c_int32),
                ("count_fragments", C.c_int32), ("lambda_ssim", C.c_float), ("mask_opacity", C.c_float),
                ("mask_erode", C.c_int32), ("persistent", C.c_int32), ("sync_spin_limit", C.c_int32),
                ("sync_skip_block", C.c_int32)]


class GicpResult(C.Structure):
    _fields_ = [("T", C.c_double * 12), ("cost", C.c_double), ("n_corr", C.c_int64), ("iters", C.c_int32),
                ("converged", C.c_int32)]


class WsLayout(C.Structure):
    _fields_ = [(k, C.c_size_t) for k in ("views", "counters", "loss_acc", "proj", "vis_bits", "scan_tmp",
                                          "ekeys0", "ekeys1", "evals0", "evals1", "keys0", "keys1", "vals0", "vals1", "pair_mask", "emit_tmp", "sort_tmp", "ranges", "T_final",
                                          "n_contrib", "grad2d", "geo2d", "dirgrad", "visible", "entries", "erect", "tile_order", "render_mask",
                                          "ssim_tmp", "total")] + \
               [("has_ssim", C.c_int32), ("sorted_buf", C.c_int32), ("total_tiles", C.c_int32), ("total_pixels", C.c_int64),
                ("max_pairs", C.c_int64), ("n", C.c_int64), ("n_views", C.c_int32), ("tile", C.c_int32)]


class Counters(C.Structure):
    _fields_ = [("status", C.c_uint32), ("n_entries", C.c_uint32), ("n_pairs", C.c_uint64), ("adam_step", C.c_uint64),
                ("frag_fwd_eval", C.c_uint64), ("frag_fwd_add", C.c_uint64), ("frag_bwd_eval", C.c_uint64),
                ("frag_bwd_add", C.c_uint64), ("visits_fwd", C.c_uint32), ("visits_bwd", C.c_uint32)]


class StepIO(C.Structure):
    _fields_ = [("target_rgb", C.c_void_p), ("target_depth", C.c_void_p), ("mask", C.c_void_p),
                ("out_rgb", C.c_void_p), ("out_depth", C.c_void_p), ("dl_drgb", C.c_void_p), ("dl_ddepth", C.c_void_p),
                ("loss_out", C.c_void_p), ("grad_twist", C.c_void_p), ("update_mask", C.c_void_p),
                ("lr", C.c_float * 6), ("b1", C.c_float), ("b2", C.c_float), ("eps", C.c_float),
                ("optimize", C.c_int32), ("host_target_rgb", C.c_void_p), ("host_target_depth", C.c_void_p),
                ("host_mask", C.c_void_p), ("host_loss_out", C.c_void_p)]


class PcaOpts(C.Structure):
    _fields_ = [("voxel", C.c_float), ("min_pts", C.c_int32), ("tau_p", C.c_float), ("tau_l", C.c_float),
                ("sigma", C.c_float), ("tau_trace", C.c_float)]


class GsError(RuntimeError):
    pass


_lock = threading.Lock()
_lib = None

# name -> (argtypes, restype)
_SIGS = {
    "gs_default_opts": ([C.POINTER(RenderOpts)], None),
    "gs_last_error": ([], C.c_char_p),
    "gs_version": ([], C.c_char_p),
    "gs_workspace_size": ([C.c_int64, C.c_int32, C.POINTER(Camera), C.POINTER(RenderOpts), C.c_int64], C.c_size_t),
    "gs_workspace_layout": ([C.c_int64, C.c_int32, C.POINTER(Camera), C.POINTER(RenderOpts), C.c_int64,
                             C.POINTER(WsLayout)], C.c_int),
    "gs_read_counters": ([C.POINTER(WsLayout), C.c_void_p, C.POINTER(Counters), C.c_void_p], C.c_int),
    "gs_workspace_init": ([C.POINTER(WsLayout), C.c_void_p, C.c_void_p], C.c_int),
    "gs_step": ([C.POINTER(Gaussians)] * 4 + [C.POINTER(Camera), C.POINTER(RenderOpts), C.POINTER(WsLayout),
                                              C.c_void_p, C.POINTER(StepIO), C.c_void_p], C.c_int),
    "gs_graph_create": ([C.POINTER(C.c_void_p)] + [C.POINTER(Gaussians)] * 4 +
                        [C.POINTER(Camera), C.POINTER(RenderOpts), C.POINTER(WsLayout), C.c_void_p, C.POINTER(StepIO),
                         C.c_void_p], C.c_int),
    "gs_graph_launch": ([C.c_void_p, C.c_void_p], C.c_int),
    "gs_graph_set_cameras": ([C.c_void_p, C.POINTER(Camera)], C.c_int),
    "gs_graph_destroy": ([C.c_void_p], C.c_int),
    "gs_project": ([C.POINTER(Gaussians), C.POINTER(Camera), C.POINTER(RenderOpts), C.POINTER(WsLayout), C.c_void_p,
                    C.c_void_p], C.c_int),
    "gs_bin_sort": ([C.POINTER(Camera), C.POINTER(RenderOpts), C.POINTER(WsLayout), C.c_void_p, C.c_void_p], C.c_int),
    "gs_render_fwd": ([C.POINTER(Camera), C.POINTER(RenderOpts), C.POINTER(WsLayout), C.c_void_p] + [C.c_void_p] * 3 +
                      [C.c_void_p] * 3 + [C.c_void_p] * 3 + [C.c_void_p], C.c_int),
    "gs_render_mask": ([C.POINTER(Camera), C.POINTER(RenderOpts), C.POINTER(WsLayout), C.c_void_p, C.c_void_p,
                        C.c_void_p, C.c_void_p], C.c_int),
    "gs_objective": ([C.POINTER(Camera), C.POINTER(RenderOpts), C.POINTER(WsLayout), C.c_void_p] + [C.c_void_p] * 9,
                     C.c_int),
    "gs_map_update_scratch_bytes": ([C.c_int64, C.c_int64], C.c_size_t),
    "gs_prune_plan": ([C.POINTER(Gaussians), C.c_float, C.c_double, C.c_void_p, C.c_void_p, C.c_size_t,
                       C.POINTER(C.c_int64), C.c_void_p], C.c_int),
    "gs_dedup_plan": ([C.POINTER(Gaussians), C.c_void_p, C.c_int64, C.c_float, C.c_void_p, C.c_void_p, C.c_size_t,
                       C.POINTER(C.c_int64), C.c_void_p], C.c_int),
    "gs_map_update": ([C.POINTER(Gaussians)] * 3 + [C.c_void_p, C.POINTER(Gaussians), C.c_void_p, C.c_void_p, C.c_void_p] +
                      [C.POINTER(Gaussians)] * 3 + [C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p], C.c_int),
    "gs_gicp_scratch_bytes": ([C.c_int64], C.c_size_t),
    "gs_gicp_target_set": ([C.POINTER(Gaussians), C.POINTER(Camera), C.c_int32, C.c_float, C.c_float, C.c_void_p,
                            C.c_void_p, C.c_void_p, C.c_size_t, C.POINTER(C.c_int64), C.c_void_p], C.c_int),
    "gs_gicp_register": ([C.POINTER(Gaussians), C.c_void_p, C.POINTER(Gaussians), C.c_void_p, C.POINTER(C.c_double),
                          C.c_float, C.c_int32, C.c_double, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p], C.c_int),
    "gs_render_bwd": ([C.POINTER(Gaussians), C.POINTER(Camera), C.POINTER(RenderOpts), C.POINTER(WsLayout), C.c_void_p,
                       C.c_void_p, C.c_void_p, C.POINTER(Gaussians), C.c_void_p, C.c_void_p], C.c_int),
    "gs_composite_bwd": ([C.POINTER(Camera), C.POINTER(RenderOpts), C.POINTER(WsLayout), C.c_void_p, C.c_void_p,
                          C.c_void_p, C.c_void_p], C.c_int),
    "gs_project_bwd": ([C.POINTER(Gaussians), C.POINTER(Camera), C.POINTER(RenderOpts), C.POINTER(WsLayout),
                        C.c_void_p, C.POINTER(Gaussians), C.c_void_p, C.c_void_p], C.c_int),
    "gs_project_bwd_adam": ([C.POINTER(Gaussians), C.POINTER(Camera), C.POINTER(RenderOpts), C.POINTER(WsLayout),
                             C.c_void_p, C.POINTER(Gaussians), C.POINTER(Gaussians), C.c_void_p,
                             C.POINTER(C.c_float), C.c_float, C.c_float, C.c_float, C.c_int64, C.c_void_p,
                             C.c_void_p], C.c_int),
    "gs_init_residuals_scratch_bytes": ([C.c_int64], C.c_size_t),
    "gs_init_residuals": ([C.POINTER(Gaussians), C.POINTER(Gaussians)] + [C.c_void_p] * 5 +
                          [C.POINTER(C.c_int64), C.c_void_p, C.c_size_t, C.c_void_p], C.c_int),
    "gs_twist_cameras": ([C.POINTER(Camera), C.c_void_p, C.c_int32, C.POINTER(Camera)], C.c_int),
    "gs_twist_grad": ([C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p], C.c_int),
    "gs_sort_pairs_noalloc": ([C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p],
                              C.c_int),
    "gs_pca_workspace_size": ([C.c_int64], C.c_size_t),
    "gs_voxel_pca": ([C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(Camera), C.c_int32, C.POINTER(PcaOpts), C.c_void_p,
                      C.c_size_t]
                     + [C.c_void_p] * 7 + [C.c_void_p], C.c_int),
    "gs_mlp_infer": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p], C.c_int),
    "gs_mlp_train_scratch_size": ([C.c_int64], C.c_size_t),
    "gs_mlp_train_step": ([C.c_void_p] * 9 + [C.c_int64, C.c_float, C.c_float, C.c_float, C.c_float, C.c_int64,
                                               C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p], C.c_int),
    "gs_init_cascade": ([C.c_void_p] * 2 + [C.c_int64] + [C.c_void_p] * 7 + [C.c_float, C.c_float, C.POINTER(Gaussians),
                                                                          C.c_void_p, C.c_void_p, C.c_void_p,
                                                                          C.c_void_p], C.c_int),
    "gs_adam_step": ([C.POINTER(Gaussians)] * 4 + [C.c_void_p, C.c_void_p, C.POINTER(C.c_float), C.c_float, C.c_float,
                                                   C.c_float, C.c_int64, C.c_void_p], C.c_int),
}


def exported_names():
    return list(_SIGS)


def lib(path: str | None = None):
    """The loaded libgs.so.  Raises if it is missing (build it with __graft_entry__.build())."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise GsError(f"libgs.so not built ({p}); run __graft_entry__.build() -- there is no CPU fallback")
            L = C.CDLL(p)
            for name, (args, res) in _SIGS.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
            _lib = L
    return _lib


def check(status: int, what: str = ""):
    if status != 0:
        msg = lib().gs_last_error().decode(errors="replace")
        raise GsError(f"{what}: {STATUS.get(status, status)}: {msg}")
