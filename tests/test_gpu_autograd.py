"""The autograd form of the renderer (Renderer / RenderFn) against the FP64 oracle.

A linear functional of the rendered images, L = <w_C, C> + <w_D, D> with seeded random
weights, is differentiated by torch.autograd through RenderFn: its gradients w.r.t. the
Gaussian planes and the pose twists must equal the oracle's adjoint for the upstream gradient
(w_C, w_D), with the cameras moved by Exp(xi) and the twist gradient mapped through the SE(3)
left Jacobian (oracle.se3).  The weights are zero at pixels the oracle flags as fragile (an
FP32 branch within 1e-4 of its threshold), as in the other parity tests."""
import numpy as np
import pytest
import torch

import oracle
import paper_2604_12942_gb300 as gs
import synth
from oracle import se3
from tests.gpu_helpers import GROUPS, rel_l2

pytestmark = pytest.mark.gpu

TWISTS = {
    "zero": np.zeros((2, 6)),
    "moved": np.array([[0.03, -0.02, 0.05, 0.02, -0.015, 0.01], [-0.04, 0.01, -0.02, -0.01, 0.03, 0.02]]),
}


def _scene_and_cams():
    sc = synth.uniform_box_scene(7, 3000, sh_degree=3)
    R = se3.exp(np.array([0, 0, 0, 0.05, -0.08, 0.03]))[:3, :3]
    cams = [synth.camera(96, 72, 90.0), synth.camera(80, 64, 75.0, R=R, t=[0.2, -0.1, 0.3])]
    return sc, cams


def _oracle(sc, cams, xi, seed=11):
    ocams = [se3.move_camera(c, xi[v]) for v, c in enumerate(cams)]
    fwd = oracle.forward(sc, ocams)
    rng = np.random.default_rng(seed)
    ups = []
    for (pr, img), c in zip(fwd, ocams):
        H, W = c["height"], c["width"]
        ok = ~img["fragile"]
        ups.append(dict(gC=rng.normal(size=(3, H, W)) * ok, gD=rng.normal(size=(H, W)) * 0.1 * ok))
    grads, tw_left = oracle.backward(sc, ocams, fwd, ups)
    tw = np.stack([se3.twist_grad(xi[v], tw_left[v]) for v in range(len(cams))])
    return fwd, ups, grads, tw


@pytest.mark.parametrize("kind,twist_device", [("zero", "cuda"), ("moved", "cpu"), ("moved", "cuda")])
def test_autograd_of_a_linear_functional_matches_oracle(kind, twist_device):
    sc, cams = _scene_and_cams()
    xi = TWISTS[kind]
    fwd, ups, grads_ref, tw_ref = _oracle(sc, cams, xi)
    planes = torch.as_tensor(sc.planes(), device="cuda").contiguous().requires_grad_(True)
    twist = torch.tensor(xi, dtype=torch.float32, device=twist_device, requires_grad=True)
    r = gs.Renderer(sc.n, cams, 3)
    rgb, depth, T = r(planes, twist)
    assert not T.requires_grad
    wC = gs.pack_rgb([u["gC"] for u in ups])
    wD = gs.pack_plane([u["gD"] for u in ups])
    L = (rgb * wC).sum() + (depth * wD).sum()
    g_planes, g_twist = torch.autograd.grad(L, [planes, twist])
    assert g_twist.device.type == twist_device
    # forward images at the moved poses
    for v, (C_, D_, T_) in enumerate(zip(gs.unpack_rgb(rgb.detach(), cams), gs.unpack_plane(depth.detach(), cams),
                                         gs.unpack_plane(T, cams))):
        img = fwd[v][1]
        ok = ~img["fragile"]
        assert ok.mean() > 0.95
        assert np.abs(C_.cpu().numpy() - img["C"])[:, ok].max() < 1e-4
        assert np.abs(T_.cpu().numpy() - img["T"])[ok].max() < 1e-4
        assert (np.abs(D_.cpu().numpy() - img["D"]) / np.maximum(1, img["D"]))[ok].max() < 1e-4
    g = g_planes.cpu().numpy()
    for name, sl in GROUPS.items():
        assert rel_l2(g[sl], grads_ref[sl]) < 1e-3, (name, rel_l2(g[sl], grads_ref[sl]))
    for v in range(len(cams)):
        e = rel_l2(g_twist[v].cpu().numpy(), tw_ref[v])
        assert e < 1e-3, (v, e)


def test_backward_accumulates_into_leaves_and_without_twist():
    sc, cams = _scene_and_cams()
    fwd, ups, grads_ref, _ = _oracle(sc, cams, TWISTS["zero"])
    planes = torch.as_tensor(sc.planes(), device="cuda").contiguous().requires_grad_(True)
    r = gs.Renderer(sc.n, cams, 3)
    rgb, depth, _ = r(planes)                       # no pose increment: no twist gradient
    L = (rgb * gs.pack_rgb([u["gC"] for u in ups])).sum() + (depth * gs.pack_plane([u["gD"] for u in ups])).sum()
    L.backward()
    assert rel_l2(planes.grad.cpu().numpy(), grads_ref) < 1e-3
    # colour only: a functional of rgb alone gets the same colour part (depth upstream absent)
    planes.grad = None
    rgb, depth, _ = r(planes)
    (rgb * gs.pack_rgb([u["gC"] for u in ups])).sum().backward()
    ref_c, _ = oracle.backward(sc, cams, fwd, [dict(gC=u["gC"], gD=np.zeros_like(u["gD"])) for u in ups])
    assert rel_l2(planes.grad.cpu().numpy(), ref_c) < 1e-3


def test_second_forward_before_backward_is_refused():
    sc, cams = _scene_and_cams()
    planes = torch.as_tensor(sc.planes(), device="cuda").contiguous().requires_grad_(True)
    r = gs.Renderer(sc.n, cams, 3)
    rgb1, _, _ = r(planes)
    rgb2, _, _ = r(planes)
    with pytest.raises(RuntimeError, match="later forward"):
        rgb1.sum().backward()
    rgb2.sum().backward()                             # the latest forward still differentiates
    assert torch.isfinite(planes.grad).all() and planes.grad.abs().sum() > 0
