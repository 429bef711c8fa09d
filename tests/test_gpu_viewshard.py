"""The invariant the view-parallel step rests on, on one GPU: the gradients of a batch's view
subsets, each rendered with its share of the loss weights, sum to the gradient of the whole
batch (planes, pose twists, visibility union) -- and the view-parallel step on one rank is
the ordinary batched step with the optimiser."""
import numpy as np
import pytest
import torch

import paper_2604_12942_gb300 as gs
import synth
from paper_2604_12942_gb300.viewshard import ViewParallelStep, partition_views
from tests.gpu_helpers import rel_l2

pytestmark = pytest.mark.gpu

SIZES = [(96, 72), (80, 60), (96, 72), (80, 60)]


def _problem():
    sc = synth.uniform_box_scene(13, 20_000, sh_degree=3)
    cams = [synth.camera(w, h, 0.9 * w) for w, h in SIZES]
    for k, c in enumerate(cams):
        c["t"] = np.array([0.2 * k - 0.3, 0.05 * k, 0.1 * k])
    tg = synth.random_targets(14, cams)
    return sc, cams, tg


def _targets(tg, views):
    return gs.pack_rgb([tg[v]["rgb"] for v in views]), gs.pack_plane([tg[v]["depth"] for v in views])


def test_view_subsets_sum_to_the_batch_gradient():
    sc, cams, tg = _problem()
    V = len(cams)
    planes = torch.as_tensor(sc.planes(), device="cuda").contiguous()
    full = gs.MappingStep(planes.clone(), 3, cams)
    lf = full(*_targets(tg, range(V)), optimize=False, with_twist=True).loss.clone()
    torch.cuda.synchronize()
    parts = partition_views(SIZES, 2)
    assert [len(p) for p in parts] == [2, 2]
    g_sum = torch.zeros_like(planes)
    tw = torch.zeros(V, 6, device="cuda")
    vis = torch.zeros(sc.n, dtype=torch.uint8, device="cuda")
    loss = 0.0
    for part in parts:
        share = len(part) / V
        o = gs.default_opts(lambda_rgb=share, lambda_depth=0.1 * share)
        st = gs.MappingStep(planes.clone(), 3, [cams[v] for v in part], o)
        r = st(*_targets(tg, part), optimize=False, with_twist=True)
        torch.cuda.synchronize()
        assert st.ws.counters().status == 0
        g_sum += st.grads
        tw[part] = st.twist
        vis = torch.maximum(vis, st.ws.visible())
        loss += float(r.loss[-1])
    assert abs(loss - float(lf[-1])) < 1e-6 * abs(float(lf[-1]))
    assert rel_l2(g_sum.cpu().numpy(), full.grads.cpu().numpy()) < 1e-6
    for v in range(V):
        assert rel_l2(tw[v].cpu().numpy(), full.twist[v].cpu().numpy()) < 1e-6, v
    assert torch.equal(vis, full.ws.visible())
    assert float(full.grads.abs().sum()) > 0


def test_view_parallel_step_on_one_rank_is_the_batched_step():
    sc, cams, tg = _problem()
    planes = torch.as_tensor(sc.planes(), device="cuda").contiguous()
    vp = ViewParallelStep(planes.clone(), 3, cams)
    ms = gs.MappingStep(planes.clone(), 3, cams)
    trgb, tdep = _targets(tg, range(len(cams)))
    for _ in range(3):
        lv = vp(trgb, tdep)
        lm = ms(trgb, tdep).loss
    torch.cuda.synchronize()
    assert abs(float(lv[-1]) - float(lm[-1])) < 1e-5 * abs(float(lm[-1]))
    # identical updates except where FP32 atomics' order flips the sign of a tiny gradient
    d = (vp.planes - ms.planes).abs()
    assert float((d > 1e-6).float().mean()) < 1e-3
    assert float(vp.step.grads.abs().max()) == 0.0          # Adam cleared the gradient rows
    assert float((vp.planes - planes).abs().max()) > 0
