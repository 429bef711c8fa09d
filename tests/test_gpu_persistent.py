"""The persistent form of the step (one cooperative kernel for the forward compositing, the
backward compositing, the projection backward and Adam, phases separated by bounded grid
barriers) against the stage-per-kernel step, and its bounded wait: a barrier that a block
never reaches times out, sets GS_ERR_TIMEOUT, changes nothing, and leaves the GPU usable."""
import numpy as np
import pytest
import torch

import paper_2604_12942_gb300 as gs
import synth

pytestmark = pytest.mark.gpu


def _problem(n=20_000):
    sc = synth.uniform_box_scene(31, n, sh_degree=3)
    cams = [synth.camera(160, 120, 150.0), synth.camera(96, 72, 90.0)]
    cams[1]["t"] = np.array([0.3, -0.1, 0.2])
    tg = synth.random_targets(32, cams)
    planes = torch.as_tensor(sc.planes(), device="cuda").contiguous()
    return planes, cams, gs.pack_rgb([t["rgb"] for t in tg]), gs.pack_plane([t["depth"] for t in tg])


def _close(a, b):
    """Equal updates up to the order of FP32 atomics (which can flip the sign of a tiny
    gradient and so of a first Adam step)."""
    return float(((a - b).abs() > 1e-6).float().mean()) < 1e-3


def test_persistent_step_matches_the_staged_step():
    planes, cams, trgb, tdep = _problem()
    staged = gs.MappingStep(planes.clone(), 3, cams, gs.default_opts(tile=16, chunk=256))
    pers = gs.MappingStep(planes.clone(), 3, cams, gs.default_opts(tile=16, chunk=256, persistent=1))
    for _ in range(3):
        ls = staged(trgb, tdep, with_twist=True).loss.clone()
        lp = pers(trgb, tdep, with_twist=True).loss.clone()
    torch.cuda.synchronize()
    cp = pers.ws.counters()
    assert cp.status == 0 and cp.adam_step == 3
    np.testing.assert_allclose(lp.cpu().numpy(), ls.cpu().numpy(), rtol=1e-5)
    assert _close(pers.planes, staged.planes) and _close(pers.m, staged.m)
    np.testing.assert_allclose(pers.twist.cpu().numpy(), staged.twist.cpu().numpy(), rtol=1e-3, atol=1e-6)
    np.testing.assert_allclose(pers.rgb.cpu().numpy(), staged.rgb.cpu().numpy(), atol=1e-4)
    # captured as a CUDA graph and replayed
    pers.capture(trgb, tdep)
    staged.capture(trgb, tdep)
    for _ in range(3):
        pers.replay()
        staged.replay()
    torch.cuda.synchronize()
    assert pers.ws.counters().status == 0 and pers.ws.counters().adam_step == 6
    assert _close(pers.planes, staged.planes)
    np.testing.assert_allclose(pers.loss.cpu().numpy(), staged.loss.cpu().numpy(), rtol=1e-5)


def test_persistent_barrier_times_out_and_reports():
    planes, cams, trgb, tdep = _problem(5_000)
    o = gs.default_opts(tile=16, chunk=256, persistent=1, sync_skip_block=0, sync_spin_limit=2000)
    step = gs.MappingStep(planes.clone(), 3, cams, o)
    before = [t.clone() for t in (step.planes, step.m, step.v)]
    step(trgb, tdep)
    torch.cuda.synchronize()
    c = step.ws.counters()
    assert c.status == 4 and c.adam_step == 0           # GS_ERR_TIMEOUT, no Adam step taken
    for a, b in zip(before, (step.planes, step.m, step.v)):
        assert torch.equal(a, b)
    # the context is intact: the same workspace steps normally once nothing skips the barrier
    step.opts.sync_skip_block = -1
    step.opts.sync_spin_limit = 0
    step(trgb, tdep)
    torch.cuda.synchronize()
    c = step.ws.counters()
    assert c.status == 0 and c.adam_step == 1
    assert float((step.planes - before[0]).abs().max()) > 0


def test_persistent_requires_its_shape():
    planes, cams, trgb, tdep = _problem(2_000)
    step = gs.MappingStep(planes, 3, cams, gs.default_opts(tile=8, chunk=64, persistent=1))
    with pytest.raises(gs.core.N.GsError, match="UNSUPPORTED"):
        step(trgb, tdep)
