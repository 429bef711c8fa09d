"""The view-parallel step's host logic without a GPU: the view partition, and -- with two gloo
ranks on the CPU -- the exchange (gradient and twist sums, visibility union) followed by the
identical masked Adam.  Each rank's gradients of its views come from the FP64 oracle (the
library's kernels need a GPU); the reduced gradient must equal the oracle's gradient of the
whole batch, and both replicas must end equal to a single process's update of the batch."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import synth
from paper_2604_12942_gb300.viewshard import allreduce_step_state, partition_views

BENCH_SIZES = [(640, 480), (640, 480), (960, 540), (960, 540), (1280, 720), (1280, 720), (1280, 1024), (1280, 1024)]


@pytest.mark.parametrize("world", [1, 2, 3, 4, 8])
def test_partition_covers_every_view_once_and_balances_pixels(world):
    parts = partition_views(BENCH_SIZES, world)
    assert len(parts) == world and all(parts)
    assert sorted(v for p in parts for v in p) == list(range(len(BENCH_SIZES)))
    assert all(p == sorted(p) for p in parts)
    load = [sum(BENCH_SIZES[v][0] * BENCH_SIZES[v][1] for v in p) for p in parts]
    assert max(load) - min(load) <= max(w * h for w, h in BENCH_SIZES)
    assert partition_views(BENCH_SIZES, world) == parts        # deterministic


def test_partition_rejects_more_ranks_than_views():
    with pytest.raises(ValueError):
        partition_views(BENCH_SIZES[:2], 3)


SIZES = [(40, 30), (32, 24), (48, 36), (40, 30)]


def _problem():
    sc = synth.uniform_box_scene(11, 400, sh_degree=1)
    sc.opacity_logits[::7] = -8.0            # transparent: culled in every view, never updated
    cams = [synth.camera(w, h, 0.9 * w) for w, h in SIZES]
    cams[1]["t"] = np.array([0.3, 0.0, 0.0])
    cams[2]["t"] = np.array([-0.2, 0.1, 0.2])
    tg = synth.random_targets(12, cams)
    return sc, cams, tg


def _grads(sc, cams, tg, views, V):
    """Oracle gradients of the views' share of the V-view batch loss, their twists in a [V, 6]
    array, and the union of their visibility."""
    K = (sc.sh_degree + 1) ** 2
    g = np.zeros((11 + 3 * K, sc.n))
    tw = np.zeros((V, 6))
    vis = np.zeros(sc.n, np.uint8)
    for v in views:
        pr = oracle.project(sc, cams[v])
        img = oracle.render(pr, cams[v])
        _, gC, gD = oracle.l1_loss(img, tg[v], scale=1.0 / V)
        gp, t = oracle.backward(sc, [cams[v]], [(pr, img)], [dict(gC=gC, gD=gD)])
        g += gp
        tw[v] = t[0]
        vis |= (pr["visible"] != 0).astype(np.uint8)
    return g, tw, vis


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sc, cams, tg = _problem()
        views = partition_views(SIZES, world)[rank]
        g, tw, vis = _grads(sc, cams, tg, views, len(cams))
        gt, twt, vt = torch.as_tensor(g), torch.as_tensor(tw), torch.as_tensor(vis)
        allreduce_step_state(gt, twt, vt)
        p, m, v = oracle.adam(sc.planes(), gt.numpy(), np.zeros_like(g), np.zeros_like(g), vt.numpy(), step=1)
        out[rank] = (views, gt.numpy(), twt.numpy(), vt.numpy(), p)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_to_the_batch_gradient_and_stay_equal():
    world = 2
    port = _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    sc, cams, tg = _problem()
    g_all, tw_all, vis_all = _grads(sc, cams, tg, range(len(cams)), len(cams))
    p_all, _, _ = oracle.adam(sc.planes(), g_all, np.zeros_like(g_all), np.zeros_like(g_all), vis_all, step=1)
    assert sorted(res[0][0] + res[1][0]) == list(range(len(cams))) and res[0][0] and res[1][0]
    for r in range(world):
        views, g, tw, vis, p = res[r]
        np.testing.assert_allclose(g, g_all, rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(tw, tw_all, rtol=1e-12, atol=1e-15)
        np.testing.assert_array_equal(vis, vis_all)
        np.testing.assert_allclose(p, p_all, rtol=1e-12, atol=1e-15)
    np.testing.assert_array_equal(res[0][4], res[1][4])          # the replicas are identical
    assert np.abs(g_all).sum() > 0 and (vis_all == 0).any() and vis_all.any()
