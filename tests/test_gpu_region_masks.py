"""The forward's warp-region masks (the byte it stores per sorted pair, which also steers the
backward): a region whose pixel centres include one with alpha >= alpha_min must keep its bit
(checked in FP64 on the projected records, for 16 x 16 tiles -- eight 8 x 4 regions -- and 8 x 8
tiles -- two), bits beyond the tile's regions stay clear, and the exact ellipse test does drop
part of what the alpha box admits.  Only list positions below a tile's largest contribution
count are checked: the forward may stop a tile's list early once all its pixels are saturated,
and the backward never reads past that count."""
import numpy as np
import pytest
import torch

import paper_2604_12942_gb300 as gs
import synth
from tests.gpu_helpers import gpu_forward

pytestmark = pytest.mark.gpu


def _cams():
    # ragged sizes (not multiples of 16), one translated view
    cams = [synth.camera(320, 240, 300.0), synth.camera(203, 157, 180.0), synth.camera(96, 131, 120.0)]
    cams[1]["t"] = np.array([0.3, -0.1, 0.4])
    return cams


@pytest.mark.parametrize("tile,chunk", [(16, 256), (8, 64)])
def test_region_masks_are_conservative(tile, chunk):
    scene = synth.uniform_box_scene(5, 8000, sh_degree=0)
    cams = _cams()
    opts = gs.default_opts(tile=tile, chunk=chunk)
    ws, *_ = gpu_forward(scene, cams, opts)
    c = ws.counters()
    assert c.status == 0 and c.n_pairs > 10_000
    P = int(c.n_pairs)
    L = ws.layout
    n, V = scene.n, len(cams)
    kname, vname = ("keys1", "vals1") if L.sorted_buf else ("keys0", "vals0")
    tiles = ws.region(kname, torch.int32, P).cpu().numpy().view(np.uint32).astype(np.int64)
    vals = ws.region(vname, torch.int32, P).cpu().numpy().view(np.uint32).astype(np.int64)
    mask = ws.region("pair_mask", torch.uint8, P).cpu().numpy().astype(np.int64)
    ranges = ws.region("ranges", torch.int32, 2 * L.total_tiles).view(-1, 2).cpu().numpy().view(np.uint32)
    rec = ws.region("proj", torch.float32, 12 * V * n).view(V * n, 12).cpu().numpy().astype(np.float64)
    n_contrib = ws.region("n_contrib", torch.int32, L.total_pixels).cpu().numpy()

    # per view: tile grid, first global tile, first pixel
    wx, rh = tile // 8, 4   # forward regions: 8 x 4 pixels, wx per tile row
    nr = tile // rh
    tile_off, pix_off, geo = [], [], []
    t0 = p0 = 0
    for cam in cams:
        W, H = int(cam["width"]), int(cam["height"])
        tx, ty = -(-W // tile), -(-H // tile)
        tile_off.append(t0)
        pix_off.append(p0)
        geo.append((W, H, tx, ty))
        t0 += tx * ty
        p0 += W * H
    assert t0 == L.total_tiles

    # the largest contribution count of each tile's pixels
    tile_cmax = np.zeros(L.total_tiles, np.int64)
    for v, (W, H, tx, ty) in enumerate(geo):
        nc = n_contrib[pix_off[v]:pix_off[v] + W * H].reshape(H, W).astype(np.int64)
        pad = np.zeros((ty * tile, tx * tile), np.int64)
        pad[:H, :W] = nc
        tile_cmax[tile_off[v]:tile_off[v] + tx * ty] = pad.reshape(ty, tile, tx, tile).max(axis=(1, 3)).reshape(-1)

    pos = np.arange(P, dtype=np.int64) - ranges[tiles, 0].astype(np.int64)
    sel = pos < tile_cmax[tiles]
    assert sel.sum() > 1000
    t_sel, v_sel, m_sel = tiles[sel], vals[sel], mask[sel]
    # bits beyond the tile's regions are clear
    assert np.all((m_sel >> (wx * nr)) == 0)

    view = np.searchsorted(np.array(tile_off), t_sel, side="right") - 1
    W_v = np.array([g[0] for g in geo])[view]
    H_v = np.array([g[1] for g in geo])[view]
    tx_v = np.array([g[2] for g in geo])[view]
    lt = t_sel - np.array(tile_off)[view]
    X0 = (lt % tx_v) * tile
    Y0 = (lt // tx_v) * tile
    r = rec[v_sel]
    u, vv, o = r[:, 0], r[:, 1], r[:, 3]
    a, b, cc = r[:, 4], r[:, 5], r[:, 6]   # conic scaled by -log2(e) / 2: alpha = o 2^e
    amin = float(opts.alpha_min)

    missing = 0
    box_regions = kept = 0
    # the alpha box test in FP32, as the kernel computes it
    f32 = np.float32
    rx = np.ascontiguousarray(r[:, 7].astype(f32)).view(np.int32).astype(f32)
    ry = np.ascontiguousarray(r[:, 11].astype(f32)).view(np.int32).astype(f32)
    u32, v32 = u.astype(f32), vv.astype(f32)
    for row in range(nr):
        for col in range(wx):
            bit = 1 << (row * wx + col)
            xs = X0[:, None] + col * 8 + np.arange(8)[None, :] + 0.5            # [n, 8]
            ys = Y0[:, None] + row * rh + np.arange(rh)[None, :] + 0.5          # [n, 4]
            dx = xs[:, None, :] - u[:, None, None]
            dy = ys[:, :, None] - vv[:, None, None]
            e = a[:, None, None] * dx * dx + 2 * b[:, None, None] * dx * dy + cc[:, None, None] * dy * dy
            alpha = np.minimum(o[:, None, None] * np.exp2(e), 0.99)
            inside = (xs[:, None, :] < W_v[:, None, None]) & (ys[:, :, None] < H_v[:, None, None])
            need = ((alpha >= amin * (1 + 1e-5)) & inside).any(axis=(1, 2))
            has = (m_sel & bit) != 0
            missing += int(np.sum(need & ~has))
            # regions the alpha box admits (the forward's first test) and the ones kept of those
            x0 = (X0 + col * 8).astype(f32)
            y0 = (Y0 + row * rh).astype(f32)
            inbox = ((u32 - rx <= x0 + f32(7.5)) & (u32 + rx >= x0 + f32(0.5)) &
                     (v32 - ry <= y0 + f32(rh - 0.5)) & (v32 + ry >= y0 + f32(0.5)))
            box_regions += int(inbox.sum())
            kept += int((has & inbox).sum())
            assert np.all(~has | inbox)   # a kept region is inside the alpha box
    assert missing == 0, missing
    # the exact test drops part of what the box admits
    assert kept < 0.95 * box_regions, (kept, box_regions)
