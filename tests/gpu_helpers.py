"""Shared helpers of the GPU parity tests: move seeded synthetic inputs to the device and
compare with the oracle."""
import numpy as np
import torch

import paper_2604_12942_gb300 as gs


def planes_of(scene, device="cuda"):
    return torch.as_tensor(scene.planes(), device=device).contiguous()


def rel_l2(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


GROUPS = {"means": slice(0, 3), "log_scales": slice(3, 6), "quats": slice(6, 10), "opacity": slice(10, 11),
          "sh_dc": slice(11, 14), "sh_rest": slice(14, None)}


def gpu_forward(scene, cams, opts=None, max_pairs=None):
    opts = opts or gs.default_opts()
    planes = planes_of(scene)
    n = scene.n
    ws = gs.Workspace(n, cams, opts, max_pairs or max(1 << 16, 256 * n * len(cams)))
    P = ws.layout.total_pixels
    rgb = torch.zeros(3 * P, device="cuda")
    depth = torch.zeros(P, device="cuda")
    T = torch.zeros(P, device="cuda")
    ws.project(planes, scene.sh_degree)
    ws.bin_sort()
    ws.render_fwd(rgb, depth, T)
    torch.cuda.synchronize()
    return ws, planes, rgb, depth, T
