"""The batched step (gs_step) and its CUDA graph against the staged calls."""
import numpy as np
import pytest
import torch

import paper_2604_12942_gb300 as gs
import synth
from tests.gpu_helpers import planes_of

pytestmark = pytest.mark.gpu


def _setup(seed=41, n=6000):
    sc = synth.uniform_box_scene(seed, n, sh_degree=3)
    cams = [synth.camera(160, 120, 150.0), synth.camera(97, 61, 80.0, t=[0.1, 0.0, 0.2])]
    tg = synth.random_targets(seed + 1, cams)
    trgb = gs.pack_rgb([t["rgb"] for t in tg])
    td = gs.pack_plane([t["depth"] for t in tg])
    return sc, cams, trgb, td


def test_step_equals_staged_calls():
    sc, cams, trgb, td = _setup()
    step = gs.MappingStep(planes_of(sc), 3, cams)
    step(trgb, td, optimize=False, with_twist=True)
    ws = gs.Workspace(sc.n, cams, gs.default_opts(), step.ws.layout.max_pairs)
    P = ws.layout.total_pixels
    planes = planes_of(sc)
    rgb = torch.zeros(3 * P, device="cuda"); dep = torch.zeros(P, device="cuda")
    dl = torch.zeros(3 * P, device="cuda"); dld = torch.zeros(P, device="cuda")
    loss = torch.zeros(len(cams) + 1, device="cuda")
    grads = torch.zeros_like(planes); tw = torch.zeros(len(cams), 6, device="cuda")
    ws.project(planes, 3)
    ws.bin_sort()
    ws.render_fwd(rgb, dep, None, trgb, td, None, dl, dld, loss)
    ws.render_bwd(planes, 3, grads, dl, dld, tw)
    torch.cuda.synchronize()
    assert torch.equal(rgb, step.rgb) and torch.equal(dep, step.depth) and torch.equal(dl, step.dl_drgb)
    assert torch.allclose(loss, step.loss, rtol=1e-6)
    # gradients are sums of float atomics: equal up to the summation order
    assert torch.allclose(grads, step.grads, rtol=1e-5, atol=1e-7 * float(grads.abs().max()))
    assert torch.allclose(tw, step.twist, rtol=1e-4, atol=1e-6 * float(tw.abs().max()))


def test_graph_replay_equals_eager_and_counts_adam_steps():
    sc, cams, trgb, td = _setup(43)
    eager = gs.MappingStep(planes_of(sc), 3, cams, lr=(1e-3, 1e-2, 1e-2, 5e-2, 1e-2, 1e-3))
    graph = gs.MappingStep(planes_of(sc), 3, cams, lr=(1e-3, 1e-2, 1e-2, 5e-2, 1e-2, 1e-3))
    losses_e, losses_g = [], []
    for _ in range(4):
        eager(trgb, td)
        losses_e.append(float(eager.loss[-1]))
    graph.capture(trgb, td)
    for _ in range(4):
        graph.replay()
        losses_g.append(float(graph.loss[-1]))
    torch.cuda.synchronize()
    np.testing.assert_allclose(losses_g, losses_e, rtol=1e-4)
    scale = float(eager.planes.abs().max())
    assert torch.allclose(graph.planes, eager.planes, rtol=1e-4, atol=1e-5 * scale)
    assert eager.ws.counters().adam_step == 4 and graph.ws.counters().adam_step == 4
    assert losses_e[-1] < losses_e[0]
    graph.release()


def test_graph_set_cameras_matches_eager_with_new_poses():
    sc, cams, trgb, td = _setup(45)
    step = gs.MappingStep(planes_of(sc), 3, cams)
    step.capture(trgb, td, optimize=False)
    moved = [dict(c) for c in cams]
    for c in moved:
        c["t"] = np.asarray(c["t"], float) + np.array([0.05, -0.03, 0.1])
    step.set_cameras(moved)
    step.replay()
    torch.cuda.synchronize()
    ref = gs.MappingStep(planes_of(sc), 3, moved)
    ref(trgb, td, optimize=False)
    torch.cuda.synchronize()
    assert torch.equal(step.rgb, ref.rgb) and torch.equal(step.depth, ref.depth)
    step.release()


def test_fused_project_bwd_adam_equals_project_bwd_then_adam():
    """On the same screen-space sums the fused kernel is bit-identical to the two calls."""
    sc, cams, trgb, td = _setup(47)
    lr = (1e-3, 1e-2, 1e-2, 5e-2, 1e-2, 1e-3)
    ws = gs.Workspace(sc.n, cams, gs.default_opts(), 1 << 20)
    P = ws.layout.total_pixels
    planes = planes_of(sc)
    rgb = torch.zeros(3 * P, device="cuda"); dep = torch.zeros(P, device="cuda")
    dl = torch.zeros(3 * P, device="cuda"); dld = torch.zeros(P, device="cuda")
    loss = torch.zeros(len(cams) + 1, device="cuda")
    ws.project(planes, 3)
    ws.bin_sort()
    ws.render_fwd(rgb, dep, None, trgb, td, None, dl, dld, loss)
    ws.composite_bwd(dl, dld)
    rng = np.random.default_rng(5)
    m0 = torch.as_tensor(rng.normal(0, 1e-3, tuple(planes.shape)).astype(np.float32), device="cuda")
    v0 = torch.as_tensor(rng.uniform(0, 1e-6, tuple(planes.shape)).astype(np.float32), device="cuda")
    upd = torch.as_tensor((rng.uniform(size=sc.n) < 0.8).astype(np.uint8), device="cuda")
    # two calls
    pa, ma, va = planes.clone(), m0.clone(), v0.clone()
    grads = torch.zeros_like(planes)
    twa = torch.zeros(len(cams), 6, device="cuda")
    ws.project_bwd(pa, 3, grads, twa)
    gs.adam_step(pa, grads, ma, va, 3, 3, lr, upd, ws.visible())
    # fused
    pb, mb, vb = planes.clone(), m0.clone(), v0.clone()
    twb = torch.zeros(len(cams), 6, device="cuda")
    ws.project_bwd_adam(pb, 3, mb, vb, 3, lr, upd, grad_twist=twb)
    torch.cuda.synchronize()
    assert torch.equal(pa, pb) and torch.equal(ma, mb) and torch.equal(va, vb)
    assert not torch.equal(pa, planes)
    assert torch.allclose(twa, twb, rtol=1e-5, atol=1e-7 * float(twa.abs().max()))
    assert float(grads.abs().sum()) == 0.0   # consumed by the Adam step


def test_optimizing_step_equals_staged_step():
    """gs_step with the optimiser (fused path) against project / bin / fwd / bwd / Adam calls;
    the screen-space sums are float atomics, so results agree up to summation order."""
    sc, cams, trgb, td = _setup(49)
    lr = (1e-3, 1e-2, 1e-2, 5e-2, 1e-2, 1e-3)
    step = gs.MappingStep(planes_of(sc), 3, cams, lr=lr)
    step(trgb, td)
    ws = gs.Workspace(sc.n, cams, gs.default_opts(), step.ws.layout.max_pairs)
    P = ws.layout.total_pixels
    planes = planes_of(sc)
    m = torch.zeros_like(planes); v = torch.zeros_like(planes); grads = torch.zeros_like(planes)
    rgb = torch.zeros(3 * P, device="cuda"); dep = torch.zeros(P, device="cuda")
    dl = torch.zeros(3 * P, device="cuda"); dld = torch.zeros(P, device="cuda")
    loss = torch.zeros(len(cams) + 1, device="cuda")
    ws.project(planes, 3)
    ws.bin_sort()
    ws.render_fwd(rgb, dep, None, trgb, td, None, dl, dld, loss)
    ws.render_bwd(planes, 3, grads, dl, dld)
    gs.adam_step(planes, grads, m, v, 3, 1, lr, None, ws.visible())
    torch.cuda.synchronize()
    assert torch.allclose(m, step.m, rtol=1e-4, atol=1e-6 * float(m.abs().max()))
    assert torch.allclose(v, step.v, rtol=1e-4, atol=1e-6 * float(v.abs().max()))
    # first Adam step moves each parameter by about lr * sign(g): a sign decided by rounding
    # (|g| at the level of the summation error) may differ
    d = (planes - step.planes).abs()
    assert float(d.max()) <= 2.05 * max(lr)
    assert float((d > 1e-6 * float(planes.abs().max())).float().mean()) < 1e-3
    assert float(step.grads.abs().sum()) == 0.0   # the fused step does not touch the gradients


@pytest.mark.parametrize("graph", [False, True])
def test_step_fed_from_host_buffers(graph):
    """The step with its targets in pinned host memory (copied in by the step itself, in a graph
    on a branch overlapped with the projection and binning) and its loss copied back to host
    memory: the same results as the step on device targets."""
    sc, cams, trgb, td = _setup(seed=43)
    dev = gs.MappingStep(planes_of(sc), 3, cams)
    host = gs.MappingStep(planes_of(sc), 3, cams)
    h_rgb, h_dep = trgb.cpu().pin_memory(), td.cpu().pin_memory()
    h_loss = torch.zeros(len(cams) + 1).pin_memory()
    # the host step's device target buffers start as garbage: everything must come from the host
    d_rgb, d_dep = torch.full_like(trgb, 7.0), torch.full_like(td, -3.0)
    if graph:
        dev.capture(trgb, td)
        host.capture(d_rgb, d_dep, host=(h_rgb, h_dep, None, h_loss))
    for k in range(3):
        if graph:
            dev.replay()
            host.replay()
        else:
            dev(trgb, td)
            host(d_rgb, d_dep, host=(h_rgb, h_dep, None, h_loss))
        torch.cuda.synchronize()
        np.testing.assert_allclose(h_loss.numpy(), dev.loss.cpu().numpy(), rtol=1e-6)
    assert torch.equal(d_rgb, trgb) and torch.equal(d_dep, td)
    assert float(((host.planes - dev.planes).abs() > 1e-6).float().mean()) < 1e-3
    assert host.ws.counters().adam_step == 3


def test_step_with_nothing_visible():
    """Every Gaussian behind the camera: the image is the background, the loss is the L1 of the
    black image against the targets (oracle), no row is updated, and the step reports no error."""
    import oracle
    sc = synth.uniform_box_scene(45, 500, sh_degree=3, box=((-3, 3), (-3, 3), (-9, -2)))
    cams = [synth.camera(64, 48, 60.0), synth.camera(40, 30, 40.0)]
    tg = synth.random_targets(46, cams)
    planes = planes_of(sc)
    step = gs.MappingStep(planes.clone(), 3, cams)
    r = step(gs.pack_rgb([t["rgb"] for t in tg]), gs.pack_plane([t["depth"] for t in tg]))
    torch.cuda.synchronize()
    c = step.ws.counters()
    assert c.status == 0 and c.n_pairs == 0 and c.n_entries == 0
    assert float(r.rgb.abs().max()) == 0.0 and float(r.depth.abs().max()) == 0.0
    ref = oracle.loss_and_grads(sc, cams, tg)
    assert abs(float(r.loss[-1]) - ref["loss"]) < 1e-5 * ref["loss"]
    assert torch.equal(step.planes, planes) and float(step.m.abs().max()) == 0.0


def test_single_gaussian_and_the_maximum_view_count():
    """One Gaussian seen by GS_MAX_VIEWS = 32 small views of different poses and sizes: images,
    parameter gradients and all 32 twists against the oracle."""
    import oracle
    from tests.gpu_helpers import rel_l2
    rng = np.random.default_rng(47)
    sc = synth.uniform_box_scene(48, 1, sh_degree=3, box=((-0.2, 0.2), (-0.2, 0.2), (3, 4)))
    sc.log_scales[:] = -1.0
    cams = []
    for v in range(32):
        w, h = int(rng.integers(9, 40)), int(rng.integers(7, 30))
        cams.append(synth.camera(w, h, 0.8 * w, t=rng.uniform(-0.15, 0.15, 3)))
    tg = synth.random_targets(49, cams)
    step = gs.MappingStep(planes_of(sc), 3, cams)
    r = step(gs.pack_rgb([t["rgb"] for t in tg]), gs.pack_plane([t["depth"] for t in tg]), optimize=False,
             with_twist=True)
    torch.cuda.synchronize()
    assert step.ws.counters().status == 0
    ref = oracle.loss_and_grads(sc, cams, tg)
    for v, C_ in enumerate(gs.unpack_rgb(r.rgb, cams)):
        img = ref["fwd"][v][1]
        ok = ~img["fragile"]
        assert np.abs(C_.cpu().numpy() - img["C"])[:, ok].max() < 1e-4, v
    assert abs(float(r.loss[-1]) - ref["loss"]) < 1e-4 * max(1.0, ref["loss"])
    assert rel_l2(step.grads.cpu().numpy(), ref["grads"]) < 1e-3
    assert rel_l2(step.twist.cpu().numpy(), ref["twists"]) < 1e-3
