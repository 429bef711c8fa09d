"""Parity at the benchmark's full size: the 2M-Gaussian SH-3 LiDAR loop scene with its 8 views of
uneven size, in the launch configuration bench.py times (8x8 tiles, chunks of 64), checked on
samples the FP64 oracle can compute: every pixel of one crop per image-size class (brute force
over all 2M Gaussians), and every parameter gradient and pose twist when the upstream gradient
is restricted to those crops.

A crop is the view's camera with the principal point moved by the crop offset; the Jacobian
clamp limit clamp_fov (W/2)/fx is kept equal to the full view's by scaling clamp_fov with
W / w, which holds for x and y alike because each crop has its view's aspect ratio."""
import numpy as np
import pytest
import torch

import oracle
import paper_2604_12942_gb300 as gs
import synth
from tests.gpu_helpers import GROUPS, rel_l2

pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-3
# view -> crop size (one view of each size class; the crop keeps the view's aspect ratio)
CROPS = {0: (64, 48), 2: (64, 36), 4: (64, 36), 6: (80, 64)}


def _crop(cam, w, h):
    """Centred w x h crop of `cam` and its oracle options (clamp limit of the full view)."""
    x0, y0 = (cam["width"] - w) // 2, (cam["height"] - h) // 2
    c = dict(cam)
    c["cx"] = cam["cx"] - x0
    c["cy"] = cam["cy"] - y0
    c["width"], c["height"] = w, h
    assert cam["width"] * h == cam["height"] * w
    return c, oracle.Opts(clamp_fov=1.3 * cam["width"] / w), x0, y0


@pytest.fixture(scope="module")
def full():
    import bench
    sc, _, cams = bench.make_workload(2_000_000, 0)
    opts = gs.default_opts(tile=8, chunk=64)
    ws = gs.Workspace(sc.n, cams, opts, 64_000_000)
    planes = torch.as_tensor(sc.planes(), device="cuda").contiguous()
    P = ws.layout.total_pixels
    rgb = torch.zeros(3 * P, device="cuda")
    depth = torch.zeros(P, device="cuda")
    ws.project(planes, 3)
    ws.bin_sort()
    ws.render_fwd(rgb, depth)
    torch.cuda.synchronize()
    c = ws.counters()
    assert c.status == 0 and c.n_pairs > 20_000_000
    crops = {}
    for v, (w, h) in CROPS.items():
        cam, o_opts, x0, y0 = _crop(cams[v], w, h)
        pr = oracle.project(sc, cam, o_opts)
        img = oracle.render(pr, cam, o_opts)
        crops[v] = (cam, o_opts, x0, y0, pr, img)
    return sc, cams, ws, planes, rgb, depth, crops


def test_fullsize_forward_crops_match_oracle(full):
    sc, cams, ws, planes, rgb, depth, crops = full
    C = gs.unpack_rgb(rgb, cams)
    D = gs.unpack_plane(depth, cams)
    for v, (cam, o_opts, x0, y0, pr, img) in crops.items():
        w, h = cam["width"], cam["height"]
        Cg = C[v][:, y0:y0 + h, x0:x0 + w].cpu().numpy()
        Dg = D[v][y0:y0 + h, x0:x0 + w].cpu().numpy()
        # At this density most pixels are "fragile": two of their added fragments lie at depths
        # within 1e-5 (relative) of each other -- Gaussians on one facade -- and FP32 depths may
        # order them either way.  Those pixels are checked for validity, the others exactly.
        ok = ~img["fragile"]
        assert ok.sum() > 200, (v, ok.mean())
        assert np.abs(Cg - img["C"])[:, ok].max() < 1e-4, v
        assert (np.abs(Dg - img["D"]) / np.maximum(1.0, np.abs(img["D"])))[ok].max() < 1e-4, v
        assert np.isfinite(Cg).all() and (Cg >= -1e-6).all()
        err = np.abs(Cg - img["C"]).max(axis=0)
        assert np.mean(err < 0.02) > 0.95 and np.median(err) < 1e-3, (v, np.mean(err < 0.02), np.median(err))


def test_fullsize_backward_crops_match_oracle(full):
    sc, cams, ws, planes, rgb, depth, crops = full
    P = ws.layout.total_pixels
    off = gs.pixel_offsets(cams)
    dl_rgb = torch.zeros(3 * P, device="cuda")
    dl_d = torch.zeros(P, device="cuda")
    ups = synth.random_upstream(21, [crops[v][0] for v in CROPS])
    grads_ref = None
    tw_ref = np.zeros((len(cams), 6))
    for (v, (cam, o_opts, x0, y0, pr, img)), up in zip(crops.items(), ups):
        # the crop's upstream gradient, zero at pixels whose FP32 branches may differ
        up["gC"][:, img["fragile"]] = 0.0
        up["gD"][img["fragile"]] = 0.0
        W, H = cams[v]["width"], cams[v]["height"]
        full_c = np.zeros((3, H, W), np.float32)
        full_d = np.zeros((H, W), np.float32)
        full_c[:, y0:y0 + cam["height"], x0:x0 + cam["width"]] = up["gC"]
        full_d[y0:y0 + cam["height"], x0:x0 + cam["width"]] = up["gD"]
        o, px = off[v], W * H
        dl_rgb[3 * o:3 * o + 3 * px] = torch.as_tensor(full_c.reshape(-1), device="cuda")
        dl_d[o:o + px] = torch.as_tensor(full_d.reshape(-1), device="cuda")
        g2d = oracle.render_backward(pr, cam, up["gC"], up["gD"], o_opts)
        g, tw = oracle.project_backward(sc, cam, g2d, o_opts)
        grads_ref = g if grads_ref is None else grads_ref + g
        tw_ref[v] = tw
    grads = torch.zeros_like(planes)
    twist = torch.zeros(len(cams), 6, device="cuda")
    ws.render_bwd(planes, 3, grads, dl_rgb, dl_d, twist)
    torch.cuda.synchronize()
    g = grads.cpu().numpy()
    assert np.count_nonzero(np.abs(grads_ref).sum(0)) > 1000   # the crops see many Gaussians
    for name, sl in GROUPS.items():
        e = rel_l2(g[sl], grads_ref[sl])
        assert e < GRAD_TOL, (name, e)
    for v in CROPS:
        e = rel_l2(twist[v].cpu().numpy(), tw_ref[v])
        assert e < GRAD_TOL, ("twist", v, e)
    others = [v for v in range(len(cams)) if v not in CROPS]
    assert float(twist[others].abs().max()) == 0.0
