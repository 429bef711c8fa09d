"""Map-size updates (bounded pruning, proximity dedup, compaction) through the C ABI against
the oracle (oracle/mapupdate.py).  Keep / accept flags are integer decisions taken on the same
FP32 values on both sides: bit-exact.  The compaction copies: exact."""
import numpy as np
import pytest
import torch

import oracle
import paper_2604_12942_gb300 as gs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("max_ratio", [0.01, 0.3, 1.0, 0.0])
def test_prune_plan_matches_oracle(max_ratio):
    rng = np.random.default_rng(int(max_ratio * 100) + 1)
    n = 120_000
    planes = np.zeros((gs.n_planes(0), n), np.float32)
    lg = rng.normal(-3.0, 2.5, n).astype(np.float32)
    lg[rng.integers(0, n, 3000)] = np.float32(-7.25)      # many equal logits below the threshold
    lg[:5] = np.float32(-np.inf)
    planes[10] = lg
    t = torch.as_tensor(planes, device="cuda")
    keep, nk = gs.prune_plan(t, 0, 0.005, max_ratio)
    ref, nk_ref = oracle.prune_plan(lg, 0.005, max_ratio)
    assert nk == nk_ref
    np.testing.assert_array_equal(keep.cpu().numpy(), ref)
    if max_ratio == 0.01:
        assert n - nk == int(np.floor(0.01 * n))     # the bound is what limits here


@pytest.mark.parametrize("offset", [0.0, -150.0])
def test_dedup_plan_matches_oracle(offset):
    rng = np.random.default_rng(7)
    n, nq, r = 20_000, 6_000, 0.05
    M = (rng.uniform(0, 6, (3, n)) + offset).astype(np.float32)
    near = M[:, rng.integers(0, n, nq // 2)] + rng.normal(0, 0.03, (3, nq // 2)).astype(np.float32)
    far = (rng.uniform(0, 6, (3, nq - nq // 2)) + offset).astype(np.float32)
    Q = np.concatenate([near, far], axis=1).astype(np.float32)
    planes = np.zeros((gs.n_planes(0), n), np.float32)
    planes[0:3] = M
    t = torch.as_tensor(planes, device="cuda")
    acc, na = gs.dedup_plan(t, 0, torch.as_tensor(Q, device="cuda"), r)
    ref, na_ref = oracle.dedup_plan(M, Q, r)
    np.testing.assert_array_equal(acc.cpu().numpy(), ref)
    assert na == na_ref and 0 < na < nq


def test_dedup_against_empty_map_accepts_all():
    planes = torch.zeros(gs.n_planes(0), 0, device="cuda")
    Q = torch.rand(3, 100, device="cuda")
    acc, na = gs.dedup_plan(planes, 0, Q, 0.05)
    assert na == 100 and int(acc.sum()) == 100


def test_map_update_matches_oracle():
    rng = np.random.default_rng(3)
    deg, n, nn = 3, 10_000, 3_000
    P = gs.n_planes(deg)
    planes = rng.normal(0, 1, (P, n)).astype(np.float32)
    planes[10] = rng.normal(-4.0, 2.0, n).astype(np.float32)
    m, v = rng.normal(0, 1, (P, n)).astype(np.float32), rng.random((P, n)).astype(np.float32)
    new = rng.normal(0, 1, (P, nn)).astype(np.float32)
    tags = rng.integers(0, 50, n).astype(np.uint32)
    ntags = rng.integers(50, 60, nn).astype(np.uint32)
    T = lambda a: torch.as_tensor(a, device="cuda")
    keep, nk = gs.prune_plan(T(planes), deg, 0.005, 0.2)
    acc = T((rng.random(nn) < 0.6).astype(np.uint8))
    out, mo, vo, to = gs.map_update(T(planes), T(m), T(v), deg, keep, T(new), acc,
                                    T(tags.view(np.int32)), T(ntags.view(np.int32)))
    torch.cuda.synchronize()
    ref = oracle.apply_update(planes, m, v, keep.cpu().numpy(), new, acc.cpu().numpy(), tags, ntags)
    assert out.shape[1] == nk + int(acc.sum())
    np.testing.assert_array_equal(out.cpu().numpy(), ref[0])
    np.testing.assert_array_equal(mo.cpu().numpy(), ref[1])
    np.testing.assert_array_equal(vo.cpu().numpy(), ref[2])
    np.testing.assert_array_equal(to.cpu().numpy().view(np.uint32), ref[3])


def test_map_update_prune_only_and_everything_pruned():
    rng = np.random.default_rng(4)
    P = gs.n_planes(1)
    planes = rng.normal(0, 1, (P, 500)).astype(np.float32)
    planes[10] = -20.0                                   # every row is a candidate
    T = lambda a: torch.as_tensor(a, device="cuda")
    keep, nk = gs.prune_plan(T(planes), 1, 0.005, 1.0)
    assert nk == 0
    out, mo, vo = gs.map_update(T(planes), T(planes), T(planes), 1, keep)
    assert out.shape == (P, 0)
    keep, nk = gs.prune_plan(T(planes), 1, 0.005, 0.1)
    out, mo, vo = gs.map_update(T(planes), T(planes), T(planes), 1, keep)
    ref = oracle.apply_update(planes, planes, planes, keep.cpu().numpy())
    assert nk == 450
    np.testing.assert_array_equal(out.cpu().numpy(), ref[0])
