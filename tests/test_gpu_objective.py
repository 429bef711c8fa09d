"""The render-derived interior mask and the full objective with SSIM (CUDA, through the C ABI)
against the FP64 oracle (oracle/objective.py) on the same inputs.

Bars: the mask is an integer decision taken on the same FP32 transmittance -> bit-exact; losses
within 1e-4 (relative), gradients within 1e-3 relative L2.  Pixels whose rendering the oracle
flags as fragile (an FP32 decision within 1e-4 of its threshold) are kept out of the caller's
mask, so the objective never reads them."""
import numpy as np
import pytest
import torch

import oracle
import paper_2604_12942_gb300 as gs
import synth
from tests.gpu_helpers import GROUPS, gpu_forward, planes_of, rel_l2

pytestmark = pytest.mark.gpu

LOSS_RTOL = 1e-4
GRAD_TOL = 1e-3


def _cams():
    # uneven sizes, not multiples of the 32 x 16 objective tile
    return [synth.camera(203, 157, 180.0), synth.camera(96, 131, 120.0, cx=40.0, cy=70.0, t=[-0.2, 0.2, 0.0])]


def _render(seed=21, n=8000, opts=None):
    sc = synth.uniform_box_scene(seed, n, sh_degree=0)
    cams = _cams()
    ws, planes, rgb, depth, T = gpu_forward(sc, cams, opts or gs.default_opts())
    return sc, cams, ws, planes, rgb, depth, T


@pytest.mark.parametrize("r_erode,tau", [(2, 0.5), (0, 0.3), (4, 0.8)])
def test_render_mask_matches_oracle(r_erode, tau):
    opts = gs.default_opts(mask_erode=r_erode, mask_opacity=tau)
    sc, cams, ws, planes, rgb, depth, T = _render(opts=opts)
    P = ws.layout.total_pixels
    rng = np.random.default_rng(1)
    callers = [(rng.random((c["height"], c["width"])) < 0.9).astype(np.uint8) for c in cams]
    caller = gs.pack_plane(callers, dtype=torch.uint8)
    out = torch.zeros(P, dtype=torch.uint8, device="cuda")
    ws.render_mask(out, caller)
    torch.cuda.synchronize()
    Ts = gs.unpack_plane(T, cams)
    Ms = gs.unpack_plane(out, cams)
    inside = 0
    for v in range(len(cams)):
        ref = oracle.render_mask(Ts[v].cpu().numpy(), tau, r_erode, callers[v])
        np.testing.assert_array_equal(Ms[v].cpu().numpy(), ref)
        inside += int(ref.sum())
    assert 0 < inside < P   # a real mask: neither empty nor everything


def _objective_case(lambda_ssim, with_depth=True, empty_view=False):
    opts = gs.default_opts(lambda_ssim=lambda_ssim)
    sc, cams, ws, planes, rgb, depth, T = _render(opts=opts)
    V, P = len(cams), ws.layout.total_pixels
    tg = synth.random_targets(5, cams)
    trgb = gs.pack_rgb([t["rgb"] for t in tg])
    tdep = gs.pack_plane([t["depth"] for t in tg]) if with_depth else None
    rng = np.random.default_rng(2)
    masks = [(rng.random((c["height"], c["width"])) < 0.85).astype(np.uint8) for c in cams]
    if empty_view:
        masks[1][:] = 0
    mask = gs.pack_plane(masks, dtype=torch.uint8)
    dl = torch.zeros(3 * P, device="cuda")
    dld = torch.zeros(P, device="cuda")
    loss = torch.zeros(V + 1, device="cuda")
    ws.objective(rgb, depth, trgb, tdep, mask, dl, dld if with_depth else None, loss)
    torch.cuda.synchronize()
    Cs, Ds = gs.unpack_rgb(rgb, cams), gs.unpack_plane(depth, cams)
    gCs, gDs = gs.unpack_rgb(dl, cams), gs.unpack_plane(dld, cams)
    total = 0.0
    for v in range(V):
        tD = tg[v]["depth"] if with_depth else np.zeros((cams[v]["height"], cams[v]["width"]))
        l, gC, gD = oracle.masked_objective(Cs[v].cpu().numpy(), Ds[v].cpu().numpy(), tg[v]["rgb"], tD, masks[v],
                                            1.0, lambda_ssim, 0.1 if with_depth else 0.0, 1.0 / V)
        total += l
        assert abs(float(loss[v]) / V - l) <= LOSS_RTOL * max(1e-3, abs(l)), (v, float(loss[v]) / V, l)
        if np.abs(gC).sum() > 0:
            assert rel_l2(gCs[v].cpu().numpy(), gC) < GRAD_TOL, v
        else:
            assert float(gCs[v].abs().max()) == 0.0
        if with_depth and np.abs(gD).sum() > 0:
            assert rel_l2(gDs[v].cpu().numpy(), gD) < GRAD_TOL, v
    assert abs(float(loss[V]) - total) <= LOSS_RTOL * abs(total)


def test_objective_with_ssim_matches_oracle():
    _objective_case(0.2)


def test_objective_ssim_only_rgb_and_empty_view():
    _objective_case(0.5, with_depth=False, empty_view=True)


def test_objective_without_ssim_equals_fused_epilogue():
    """With lambda_ssim = 0 the separate loss kernels repeat the forward's fused L1 epilogue
    exactly (same arithmetic in the same order per pixel)."""
    sc, cams, ws, planes, rgb, depth, T = _render()
    V, P = len(cams), ws.layout.total_pixels
    tg = synth.random_targets(6, cams)
    trgb = gs.pack_rgb([t["rgb"] for t in tg])
    tdep = gs.pack_plane([t["depth"] for t in tg])
    rng = np.random.default_rng(3)
    mask = gs.pack_plane([(rng.random((c["height"], c["width"])) < 0.7).astype(np.uint8) for c in cams],
                         dtype=torch.uint8)
    bufs = [torch.zeros(3 * P, device="cuda"), torch.zeros(P, device="cuda"), torch.zeros(V + 1, device="cuda")]
    rgb2, dep2 = torch.zeros_like(rgb), torch.zeros_like(depth)
    ws.render_fwd(rgb2, dep2, None, trgb, tdep, mask, *bufs)
    sep = [torch.zeros(3 * P, device="cuda"), torch.zeros(P, device="cuda"), torch.zeros(V + 1, device="cuda")]
    ws.objective(rgb2, dep2, trgb, tdep, mask, *sep)
    torch.cuda.synchronize()
    assert torch.equal(bufs[0], sep[0]) and torch.equal(bufs[1], sep[1])
    assert torch.allclose(bufs[2], sep[2], rtol=1e-6)


def test_step_with_ssim_and_render_mask_matches_oracle():
    """gs_step with the SSIM term and the interior mask of its own rendering: the step's mask
    is the oracle's mask of the step's transmittance, and the parameter gradients and pose
    twists follow from the oracle's objective on that mask through the oracle's backward."""
    sc = synth.uniform_box_scene(31, 6000, sh_degree=3)
    cams = _cams()
    V = len(cams)
    tg = synth.random_targets(8, cams)
    opts = gs.default_opts(lambda_ssim=0.2, mask_erode=2, mask_opacity=0.5)
    fwd = oracle.forward(sc, cams)
    # fragile pixels (and nothing else) are kept out by the caller's mask
    callers = [(~img["fragile"]).astype(np.uint8) for _, img in fwd]
    step = gs.MappingStep(planes_of(sc), 3, cams, opts)
    trgb = gs.pack_rgb([t["rgb"] for t in tg])
    tdep = gs.pack_plane([t["depth"] for t in tg])
    caller = gs.pack_plane(callers, dtype=torch.uint8)
    step(trgb, tdep, mask=caller, optimize=False, with_twist=True)
    torch.cuda.synchronize()
    assert step.ws.counters().status == 0
    P = step.ws.layout.total_pixels
    T = step.ws.region("T_final", torch.float32, P)
    Ms = gs.unpack_plane(step.ws.region("render_mask", torch.uint8, P), cams)
    Ts = gs.unpack_plane(T, cams)
    ups, total = [], 0.0
    for v, ((pr, img), t) in enumerate(zip(fwd, tg)):
        M = Ms[v].cpu().numpy()
        np.testing.assert_array_equal(M, oracle.render_mask(Ts[v].cpu().numpy(), 0.5, 2, callers[v]))
        assert M.sum() > 100
        l, gC, gD = oracle.masked_objective(img["C"], img["D"], t["rgb"], t["depth"], M, 1.0, 0.2, 0.1, 1.0 / V)
        total += l
        ups.append(dict(gC=gC, gD=gD))
    assert abs(float(step.loss[V]) - total) <= LOSS_RTOL * abs(total), (float(step.loss[V]), total)
    grads_ref, tw_ref = oracle.backward(sc, cams, fwd, ups)
    g = step.grads.cpu().numpy()
    for name, sl in GROUPS.items():
        if np.abs(grads_ref[sl]).sum() == 0:
            continue
        assert rel_l2(g[sl], grads_ref[sl]) < GRAD_TOL, name
    for v in range(V):
        assert rel_l2(step.twist[v].cpu().numpy(), tw_ref[v]) < GRAD_TOL, ("twist", v)
