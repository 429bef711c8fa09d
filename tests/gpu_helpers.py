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


def pack_vis_bits(seen):
    """[V, n] booleans -> the workspace's visibility words: per view, bit i % 32 of word i / 32,
    the view padded to whole words."""
    seen = np.asarray(seen, bool)
    V, n = seen.shape
    nw = (n + 31) // 32
    pad = np.zeros((V, nw * 32), bool)
    pad[:, :n] = seen
    w = np.packbits(pad.reshape(V, nw, 4, 8), axis=-1, bitorder="little").reshape(V, nw, 4)
    return w.reshape(V, nw * 4).view("<u4").reshape(V, nw)


def unpack_vis_bits(words, V, n):
    """The inverse of pack_vis_bits: [V, n] booleans."""
    w = np.ascontiguousarray(np.asarray(words).astype("<u4").reshape(V, -1))
    bits = np.unpackbits(w.view(np.uint8), bitorder="little").reshape(V, -1)
    return bits[:, :n].astype(bool)


def set_vis_bits(ws, seen):
    """Write [V, n] visibility into the workspace (the input gs_bin_sort reads)."""
    w = pack_vis_bits(seen)
    ws.region("vis_bits", torch.int32, w.size).copy_(torch.as_tensor(w.reshape(-1).view(np.int32)))


def get_vis_bits(ws, V, n):
    nw = (n + 31) // 32
    w = ws.region("vis_bits", torch.int32, V * nw).cpu().numpy().view(np.uint32)
    return unpack_vis_bits(w, V, n)


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
