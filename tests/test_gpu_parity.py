"""CUDA path (through the C ABI) against the FP64 oracle on the same seeded inputs.

Tolerances (stated by the target of the build): images max-abs 1e-4, gradients relative
L2 1e-3, keys / values / ranges bit-exact.  Pixels where the oracle reports a decision
within a relative 1e-4 of its threshold (alpha vs 1/255, T vs 1e-4, alpha vs the 0.99 clamp,
a depth near-tie, a cull) are compared only for validity: an FP32 implementation may take
the other branch there.  Their number is bounded.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_2604_12942_gb300 as gs
import synth
from tests.gpu_helpers import GROUPS, get_vis_bits, gpu_forward, planes_of, rel_l2, set_vis_bits

pytestmark = pytest.mark.gpu

IMG_TOL = 1e-4
GRAD_TOL = 1e-3


def _rot(axis, ang):
    axis = np.asarray(axis, float) / np.linalg.norm(axis)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * K @ K


def _scene_c1(n=10_000, deg=0, seed=1):
    return synth.uniform_box_scene(seed, n, sh_degree=deg)


def _cams_small():
    # uneven, ragged sizes (not multiples of 16 or 8), rotated / translated poses
    return [synth.camera(320, 240, 300.0),
            synth.camera(203, 157, 180.0, R=_rot([0.2, 1, 0], 0.15), t=[0.3, -0.1, 0.4]),
            synth.camera(96, 131, 120.0, cx=40.0, cy=70.0, R=_rot([1, 0, 0.3], -0.1), t=[-0.2, 0.2, 0.0])]


@pytest.fixture(scope="module")
def lidar_small():
    sc = synth.lidar_scene(seed=5, n=30_000, sh_degree=3, kind="line", n_boxes=8)
    cams = synth.trajectory_cameras(sc, [(256, 192), (200, 136)], [60, 130], fx_per_width=0.7)
    return sc, cams


# ----------------------------------------------------------------------------------------
# a1 projection
# ----------------------------------------------------------------------------------------

@pytest.mark.parametrize("deg", [0, 3])
def test_project_matches_oracle(deg):
    sc = _scene_c1(4000, deg, seed=2)
    cams = _cams_small()
    ws, planes, *_ = gpu_forward(sc, cams)
    n = sc.n
    rec = ws.region("proj", torch.float32, 12 * len(cams) * n).view(len(cams), n, 12).cpu().numpy()
    seen = get_vis_bits(ws, len(cams), n)
    for v, cam in enumerate(cams):
        pr = oracle.project(sc, cam)
        t = seen[v]
        ok = pr["visible"].astype(bool) & ~pr["fragile"].astype(bool)
        # every GPU-kept Gaussian is visible for the oracle (up to fragile cull decisions)
        assert np.all(pr["visible"][t] | pr["fragile"][t])
        sel = t & ok
        assert sel.sum() > 100
        r = rec[v][sel]
        np.testing.assert_allclose(r[:, 0], pr["u"][sel], atol=2e-3, rtol=0)
        np.testing.assert_allclose(r[:, 1], pr["v"][sel], atol=2e-3, rtol=0)
        np.testing.assert_allclose(r[:, 2], pr["z"][sel], rtol=2e-6)
        np.testing.assert_allclose(r[:, 3], pr["opacity"][sel], rtol=2e-6)
        # conic from the scaled record: (a, b, c) = -log2(e)/2 (A, B, C)
        k = -0.5 / math.log(2.0)
        conic = r[:, 4:7] / k
        scale = np.abs(pr["conic"][sel]).max(1, keepdims=True)
        assert np.max(np.abs(conic - pr["conic"][sel]) / scale) < 2e-4
        np.testing.assert_allclose(r[:, 8:11], pr["rgb"][sel], atol=2e-5)
        for col, key in ((7, "rx"), (11, "ry")):
            rad = np.ascontiguousarray(r[:, col]).view(np.int32)
            assert np.all(np.abs(rad - pr[key][sel]) <= 1)
            assert np.mean(rad == pr[key][sel]) > 0.99


# ----------------------------------------------------------------------------------------
# a2-a4 binning, sort, ranges: bit-exact on synthetic FP32 screen-space records
# ----------------------------------------------------------------------------------------

def _bin_case(cams, n, tile, seed, radius_max=48):
    items = synth.random_projected_items(seed, cams, n, radius_max=radius_max)
    ref = oracle.bin_views(items, cams, tile)
    opts = gs.default_opts(tile=tile)
    P = int(ref["keys"].shape[0])
    ws = gs.Workspace(n, cams, opts, max(P, 1))
    V = len(cams)
    rec = np.zeros((V, n, 12), np.float32)
    for v, it in enumerate(items):
        rec[v, :, 0] = it["u"]; rec[v, :, 1] = it["v"]; rec[v, :, 2] = it["z"]; rec[v, :, 3] = 0.5
        rec[v, :, 7] = it["rx"].view(np.float32)
        rec[v, :, 11] = it["ry"].view(np.float32)
    ws.region("proj", torch.float32, 12 * V * n).copy_(torch.as_tensor(rec.reshape(-1)))
    set_vis_bits(ws, ref["touched"].reshape(V, n) > 0)
    ws.region("counters", torch.int32, 8).zero_()
    ws.bin_sort()
    c = ws.counters()
    assert c.status == 0
    assert c.n_pairs == P
    # the visible entries in depth order: a stable sort of (view, index) order by bits(z)
    vis_ids = np.nonzero(ref["touched"].reshape(-1) > 0)[0]
    assert c.n_entries == len(vis_ids)
    zb = rec.reshape(-1, 12)[vis_ids, 2].view(np.uint32)
    np.testing.assert_array_equal(ws.sorted_entries(len(vis_ids)).cpu().numpy().view(np.uint32),
                                  vis_ids[np.argsort(zb, kind="stable")].astype(np.uint32))
    k, vals = ws.sorted_pairs(P)
    np.testing.assert_array_equal(k.cpu().numpy().view(np.uint64), ref["sorted_keys"])
    np.testing.assert_array_equal(vals.cpu().numpy().view(np.uint32), ref["sorted_vals"])
    rg = ws.region("ranges", torch.int32, 2 * ref["n_tiles"]).view(-1, 2).cpu().numpy().view(np.uint32)
    np.testing.assert_array_equal(rg, ref["ranges"])
    return P


@pytest.mark.parametrize("tile", [8, 16])
def test_bin_sort_bit_exact_small(tile):
    _bin_case(_cams_small(), 3000, tile, seed=3)


def test_bin_sort_bit_exact_multichunk():
    """More than 2.5M pairs: every block of the sort grid owns several chunks, ragged tail."""
    cams = [synth.camera(1280, 720, 900.0), synth.camera(640, 480, 500.0)]
    P = _bin_case(cams, 300_000, 8, seed=4, radius_max=64)
    assert P > 2_500_000


def test_bin_sort_bit_exact_nine_bit_digits():
    """81,920 tiles (17 tile bits): the tile sort takes two 9-bit passes instead of three."""
    cams = [synth.camera(1280, 1024, 900.0) for _ in range(4)]
    P = _bin_case(cams, 100_000, 8, seed=6, radius_max=40)
    assert P > 1_000_000


def test_bin_sort_tiny_ragged():
    # 2 x 37 (view, Gaussian) slots: the visibility bit words straddle the views and the last
    # one is partial
    _bin_case(_cams_small()[:2], 37, 16, seed=7, radius_max=60)


def test_bin_sort_single_tile():
    """One tile per view set: no tile-sort pass, the pairs stay in depth order."""
    _bin_case([synth.camera(16, 16, 20.0)], 2000, 16, seed=5, radius_max=12)


def test_bin_sort_empty():
    cams = [synth.camera(64, 48, 60.0)]
    ws = gs.Workspace(10, cams, gs.default_opts(), 128)
    set_vis_bits(ws, np.zeros((1, 10), bool))
    ws.region("counters", torch.int32, 8).zero_()
    ws.bin_sort()
    c = ws.counters()
    assert c.status == 0 and c.n_pairs == 0
    assert int(ws.region("ranges", torch.int32, 2 * ws.layout.total_tiles).abs().sum()) == 0


# ----------------------------------------------------------------------------------------
# a5 forward compositing
# ----------------------------------------------------------------------------------------

def _compare_images(sc, cams, rgb, depth, T, tile):
    Cs = gs.unpack_rgb(rgb, cams)
    Ds = gs.unpack_plane(depth, cams)
    Ts = gs.unpack_plane(T, cams)
    fragile_total = 0
    px_total = 0
    fr_maps = []
    for v, cam in enumerate(cams):
        pr = oracle.project(sc, cam)
        im = oracle.render(pr, cam)
        ok = ~im["fragile"]
        fr_maps.append(im["fragile"])
        fragile_total += int(im["fragile"].sum())
        px_total += ok.size
        C = Cs[v].cpu().numpy(); D = Ds[v].cpu().numpy(); Tt = Ts[v].cpu().numpy()
        assert np.all(np.isfinite(C)) and np.all(np.isfinite(D))
        err_c = np.abs(C - im["C"])[:, ok].max()
        err_t = np.abs(Tt - im["T"])[ok].max()
        # depth scales with z (up to ~60 m); compare relative to the depth scale
        err_d = (np.abs(D - im["D"]) / np.maximum(1.0, np.abs(im["D"])))[ok].max()
        assert err_c < IMG_TOL, (v, tile, err_c)
        assert err_t < IMG_TOL, (v, tile, err_t)
        assert err_d < IMG_TOL, (v, tile, err_d)
        # validity where FP32 may decide differently: values stay in range, and one flipped
        # alpha_min / T_min decision moves a pixel by at most ~alpha_min + T_min/(1-alpha_max)
        assert np.all(C[:, ~ok] >= -1e-6) and np.all(Tt[~ok] >= 0.0) and np.all(Tt[~ok] <= 1.0)
        if (~ok).any():
            assert np.quantile(np.abs(C - im["C"])[:, ~ok], 0.99) < 0.02
    # The alpha_min margin (1e-4 relative, the FP32 error of alpha for conics of condition
    # number up to ~16) flags a few percent of the pixels of dense LiDAR-shaped scenes.
    assert fragile_total <= 0.05 * px_total, (fragile_total, px_total)
    return fr_maps


@pytest.mark.parametrize("tile,chunk", [(16, 64), (8, 32), (16, 256)])
def test_render_forward_c1_matches_oracle(tile, chunk):
    sc = _scene_c1()
    cams = [synth.camera(320, 240, 300.0)]
    opts = gs.default_opts(tile=tile, chunk=chunk)
    ws, planes, rgb, depth, T = gpu_forward(sc, cams, opts)
    assert ws.counters().status == 0
    _compare_images(sc, cams, rgb, depth, T, tile)


def test_render_forward_multiview_ragged_deg3(lidar_small):
    sc, cams = lidar_small
    cams = cams + [synth.camera(77, 53, 60.0, R=_rot([0, 0, 1], 0.3) @ np.asarray(cams[0]["R"]), t=cams[0]["t"])]
    ws, planes, rgb, depth, T = gpu_forward(sc, cams, gs.default_opts(tile=16, chunk=128))
    _compare_images(sc, cams, rgb, depth, T, 16)


def test_render_forward_background_and_transmittance():
    """Non-black background: C = sum c w + T bg, and for unit colours C + T (1 - bg) = 1."""
    sc = _scene_c1(3000, 0, seed=9)
    sc.sh[:] = 0.5 * 2 * math.sqrt(math.pi)
    cams = [synth.camera(160, 120, 150.0)]
    bg = (0.25, 0.5, 0.75)
    ws, planes, rgb, depth, T = gpu_forward(sc, cams, gs.default_opts(bg=bg))
    C = gs.unpack_rgb(rgb, cams)[0].cpu().numpy()
    Tt = gs.unpack_plane(T, cams)[0].cpu().numpy()
    for ch in range(3):
        np.testing.assert_allclose(C[ch] + Tt * (1 - bg[ch]), 1.0, atol=2e-5)


def test_fragment_counters_optional_and_consistent():
    """The fragment counters are filled only with count_fragments = 1, which changes no output;
    the forward's added fragments equal the oracle's count (each pixel the oracle flags as
    fragile may differ by one or two) and the backward re-adds exactly the same fragments."""
    sc = _scene_c1(10_000, 0, seed=3)
    cams = [synth.camera(320, 240, 300.0)]
    ws0, planes, rgb0, depth0, T0 = gpu_forward(sc, cams, gs.default_opts())
    ws1, _, rgb1, depth1, T1 = gpu_forward(sc, cams, gs.default_opts(count_fragments=1))
    c0, c1 = ws0.counters(), ws1.counters()
    assert (c0.frag_fwd_eval, c0.frag_fwd_add, c0.visits_fwd) == (0, 0, 0)
    assert torch.equal(rgb0, rgb1) and torch.equal(depth0, depth1) and torch.equal(T0, T1)
    im = oracle.render(oracle.project(sc, cams[0]), cams[0])
    n_ref, n_fragile = int(im["n_frag"].sum()), int(im["fragile"].sum())
    assert n_ref > 100_000
    assert abs(int(c1.frag_fwd_add) - n_ref) <= 2 * n_fragile, (c1.frag_fwd_add, n_ref, n_fragile)
    assert c1.frag_fwd_eval >= c1.frag_fwd_add and c1.visits_fwd > 0
    P = ws0.layout.total_pixels
    up = torch.linspace(-1.0, 1.0, 3 * P, device="cuda")
    upd = torch.linspace(0.5, -0.5, P, device="cuda")
    for ws in (ws0, ws1):
        grads = torch.zeros_like(planes)
        ws.render_bwd(planes, 0, grads, up, upd, None)
    torch.cuda.synchronize()
    c0, c1 = ws0.counters(), ws1.counters()
    assert (c0.frag_bwd_eval, c0.frag_bwd_add, c0.visits_bwd) == (0, 0, 0)
    assert c1.frag_bwd_add == c1.frag_fwd_add and c1.frag_bwd_eval >= c1.frag_bwd_add and c1.visits_bwd > 0


# ----------------------------------------------------------------------------------------
# a6-a7 backward
# ----------------------------------------------------------------------------------------

def _backward_case(sc, cams, opts, seed):
    ws, planes, rgb, depth, T = gpu_forward(sc, cams, opts)
    ups = synth.random_upstream(seed, cams)
    fwd = oracle.forward(sc, cams)
    for up, (pr, im) in zip(ups, fwd):
        up["gC"][:, im["fragile"]] = 0.0
        up["gD"][im["fragile"]] = 0.0
    grads_ref, tw_ref = oracle.backward(sc, cams, fwd, ups)
    grads = torch.zeros_like(planes)
    twist = torch.zeros(len(cams), 6, device="cuda")
    dl_drgb = gs.pack_rgb([u["gC"] for u in ups])
    dl_dd = gs.pack_plane([u["gD"] for u in ups])
    ws.render_bwd(planes, sc.sh_degree, grads, dl_drgb, dl_dd, twist)
    torch.cuda.synchronize()
    g = grads.cpu().numpy()
    for name, sl in GROUPS.items():
        if sl.start >= g.shape[0]:
            continue
        e = rel_l2(g[sl], grads_ref[sl])
        assert e < GRAD_TOL, (name, e)
    for v in range(len(cams)):
        e = rel_l2(twist[v].cpu().numpy(), tw_ref[v])
        assert e < GRAD_TOL, ("twist", v, e)


def test_render_backward_c1_matches_oracle():
    _backward_case(_scene_c1(10_000, 0), [synth.camera(320, 240, 300.0)], gs.default_opts(), seed=11)


@pytest.mark.parametrize("tile,chunk", [(16, 64), (8, 128)])
def test_render_backward_multiview_deg3(lidar_small, tile, chunk):
    sc, cams = lidar_small
    _backward_case(sc, cams, gs.default_opts(tile=tile, chunk=chunk), seed=12)


def test_render_backward_rotated_ragged_deg3():
    sc = _scene_c1(5000, 3, seed=13)
    _backward_case(sc, _cams_small(), gs.default_opts(tile=16, chunk=32), seed=14)


# ----------------------------------------------------------------------------------------
# fused loss
# ----------------------------------------------------------------------------------------

def test_fused_l1_loss_matches_oracle():
    sc = _scene_c1(6000, 0, seed=15)
    cams = [synth.camera(160, 120, 150.0), synth.camera(97, 61, 80.0)]
    tg = synth.random_targets(16, cams, depth_hole_frac=0.3)
    tg[1]["mask"][:10] = 0
    opts = gs.default_opts()
    ws, planes, rgb, depth, T = gpu_forward(sc, cams, opts)
    P = ws.layout.total_pixels
    dl_rgb = torch.zeros(3 * P, device="cuda"); dl_d = torch.zeros(P, device="cuda")
    loss = torch.zeros(len(cams) + 1, device="cuda")
    trgb = gs.pack_rgb([t["rgb"] for t in tg]); td = gs.pack_plane([t["depth"] for t in tg])
    mask = gs.pack_plane([t["mask"] for t in tg], dtype=torch.uint8)
    ws.render_fwd(rgb, depth, T, trgb, td, mask, dl_rgb, dl_d, loss)
    ref = oracle.loss_and_grads(sc, cams, tg)
    torch.cuda.synchronize()
    assert abs(loss[-1].item() - ref["loss"]) < 1e-5 * max(1.0, abs(ref["loss"])) + 1e-6
    for v, (up, (pr, im)) in enumerate(zip(ref["upstream"], ref["fwd"])):
        g = gs.unpack_rgb(dl_rgb, cams)[v].cpu().numpy()
        C = gs.unpack_rgb(rgb, cams)[v].cpu().numpy()
        clear = (np.abs(im["C"] - tg[v]["rgb"]) > 1e-4) & ~im["fragile"][None]
        np.testing.assert_allclose(g[clear], up["gC"][clear], rtol=1e-6, atol=1e-12)
        gd = gs.unpack_plane(dl_d, cams)[v].cpu().numpy()
        cleard = (np.abs(im["D"] - tg[v]["depth"]) > 1e-3) & ~im["fragile"]
        np.testing.assert_allclose(gd[cleard], up["gD"][cleard], rtol=1e-6, atol=1e-12)


# ----------------------------------------------------------------------------------------
# a8 Adam
# ----------------------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1000, 1003])
def test_adam_matches_oracle(n):
    rng = np.random.default_rng(17)
    deg = 3
    Pn = gs.n_planes(deg)
    p = rng.normal(size=(Pn, n)).astype(np.float32)
    g = rng.normal(size=(Pn, n)).astype(np.float32)
    m = rng.normal(size=(Pn, n)).astype(np.float32) * 0.1
    v = rng.uniform(0, 0.1, (Pn, n)).astype(np.float32)
    upd = (rng.uniform(size=n) < 0.7).astype(np.uint8)
    vis = (rng.uniform(size=n) < 0.8).astype(np.uint8)
    lr = (1e-3, 2e-3, 3e-3, 4e-3, 5e-3, 6e-3)
    T = [torch.as_tensor(a).cuda().contiguous() for a in (p, g, m, v)]
    gs.adam_step(*T, deg, step=3, lr=lr, update_mask=torch.as_tensor(upd).cuda(), visible=torch.as_tensor(vis).cuda(),
                 eps=1e-8)
    torch.cuda.synchronize()
    # both sides use the same (FP32-rounded) hyper-parameters
    f = lambda x: float(np.float32(x))
    rp, rm, rv = oracle.adam(p, g, m, v, upd & vis, lr=[f(x) for x in lr], b1=f(0.9), b2=f(0.999), eps=f(1e-8),
                             step=3)
    np.testing.assert_allclose(T[0].cpu().numpy(), rp, rtol=2e-6, atol=2e-7)
    np.testing.assert_allclose(T[2].cpu().numpy(), rm, rtol=2e-6, atol=1e-7)
    np.testing.assert_allclose(T[3].cpu().numpy(), rv, rtol=2e-6, atol=1e-9)
    off = (upd & vis) == 0
    np.testing.assert_array_equal(T[0].cpu().numpy()[:, off], p[:, off])
    np.testing.assert_array_equal(T[2].cpu().numpy()[:, off], m[:, off])
    # gradients consumed on visible rows; rows outside `visible` are neither read nor written
    G = T[1].cpu().numpy()
    assert float(np.abs(G[:, vis == 1]).sum()) == 0.0
    np.testing.assert_array_equal(G[:, vis == 0], g[:, vis == 0])


# ----------------------------------------------------------------------------------------
# failure handling on the device: capacity overflow
# ----------------------------------------------------------------------------------------

def test_capacity_overflow_reports_and_skips():
    sc = _scene_c1(3000, 0)
    cams = [synth.camera(160, 120, 150.0)]
    ws, planes, rgb, depth, T = gpu_forward(sc, cams, max_pairs=100)
    c = ws.counters()
    assert c.status == 3 and c.n_pairs > 100
    # a large enough workspace succeeds and reports the same count
    ws2, *_ = gpu_forward(sc, cams, max_pairs=int(c.n_pairs))
    c2 = ws2.counters()
    assert c2.status == 0 and c2.n_pairs == c.n_pairs


def _failed_step_changes_nothing(step, trgb, status):
    before = [t.clone() for t in (step.planes, step.m, step.v)]
    step(trgb)
    torch.cuda.synchronize()
    c = step.ws.counters()
    assert c.status == status and c.adam_step == 0
    for a, b in zip(before, (step.planes, step.m, step.v)):
        assert torch.equal(a.view(torch.int32), b.view(torch.int32))   # bit for bit (a planted NaN included)


def test_capacity_overflow_skips_the_whole_step():
    """Pair capacity exceeded inside an optimising step: no gradient, no Adam update."""
    sc = _scene_c1(3000, 0)
    cams = [synth.camera(160, 120, 150.0)]
    tg = synth.random_targets(5, cams)
    step = gs.MappingStep(planes_of(sc), 0, cams, max_pairs=100)
    _failed_step_changes_nothing(step, gs.pack_rgb([tg[0]["rgb"]]), 3)


@pytest.mark.parametrize("plane,what", [(0, "nan"), (5, "inf"), (8, "nan"), (12, "nan")])
def test_nonfinite_parameter_sets_status_and_skips_the_step(plane, what):
    """A NaN or infinite mean, log-scale, quaternion or SH coefficient of a row some view sees
    makes the projection set GS_ERR_NONFINITE; the step then changes nothing."""
    sc = _scene_c1(3000, 1)
    cams = [synth.camera(160, 120, 150.0)]
    tg = synth.random_targets(6, cams)
    planes = planes_of(sc)
    ws, *_ = gpu_forward(sc, cams)
    row = int(torch.nonzero(ws.visible())[0])
    planes[plane, row] = float("nan") if what == "nan" else float("inf")
    step = gs.MappingStep(planes, 1, cams)
    _failed_step_changes_nothing(step, gs.pack_rgb([tg[0]["rgb"]]), 5)
    # a finite map on the same workspace steps normally again
    step.planes.copy_(planes_of(sc))
    step(gs.pack_rgb([tg[0]["rgb"]]))
    torch.cuda.synchronize()
    assert step.ws.counters().status == 0 and step.ws.counters().adam_step == 1


def test_mapping_step_reduces_loss():
    sc = _scene_c1(5000, 0, seed=21)
    gt = synth.perturbed(sc, 22)
    cams = [synth.camera(160, 120, 150.0)]
    # target = oracle render of the perturbed copy
    pr = oracle.project(gt, cams[0])
    im = oracle.render(pr, cams[0])
    trgb = gs.pack_rgb([im["C"].astype(np.float32)])
    td = gs.pack_plane([im["D"].astype(np.float32)])
    step = gs.MappingStep(planes_of(sc), 0, cams, lr=(1e-3, 1e-2, 1e-2, 5e-2, 1e-2, 1e-3))
    losses = []
    for _ in range(30):
        r = step(trgb, td)
        losses.append(float(r.loss[-1]))
    assert losses[-1] < 0.8 * losses[0], losses
