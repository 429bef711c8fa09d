"""Pins of the oracle's map updates (CPU): brute-force selection for the bounded pruning, a
k-d tree for the proximity test, and plain boolean indexing for the compaction."""
import numpy as np
import pytest

import oracle

spatial = pytest.importorskip("scipy.spatial")


def test_prune_unbounded_is_the_threshold():
    rng = np.random.default_rng(0)
    lg = rng.normal(-3.0, 3.0, 5000).astype(np.float32)
    keep, nk = oracle.prune_plan(lg, 0.005, 1.0)
    np.testing.assert_array_equal(keep, (lg >= oracle.logit_threshold(0.005)).astype(np.uint8))
    assert nk == int(keep.sum())
    # the FP32 threshold is the logit of 0.005
    assert abs(float(oracle.logit_threshold(0.005)) - np.log(0.005 / 0.995)) < 1e-6


def test_prune_bounded_removes_smallest_logit_then_index():
    rng = np.random.default_rng(1)
    lg = rng.choice(np.float32([-9.0, -8.0, -7.5, 0.0, 1.0]), 400).astype(np.float32)   # many ties
    thr = float(oracle.logit_threshold(0.005))
    k = int(np.floor(0.1 * lg.size))
    cands = sorted((float(x), i) for i, x in enumerate(lg) if x < thr)
    removed = {i for _, i in cands[:k]}
    keep, nk = oracle.prune_plan(lg, 0.005, 0.1)
    assert nk == lg.size - min(k, len(cands))
    assert {i for i in range(lg.size) if keep[i] == 0} == removed


def test_dedup_matches_kdtree():
    rng = np.random.default_rng(2)
    M = rng.uniform(0, 4, (3, 3000)).astype(np.float32)
    Q = rng.uniform(0, 4, (3, 1500)).astype(np.float32)
    r = 0.05
    tree = spatial.cKDTree(M.T.astype(np.float64))
    d, _ = tree.query(Q.T.astype(np.float64), k=1)
    clear = np.abs(d - r) > 1e-5          # leave out the queries whose nearest map mean sits on r
    acc, _ = oracle.dedup_plan(M, Q, r)
    np.testing.assert_array_equal(acc[clear], (d[clear] >= r).astype(np.uint8))
    assert (acc == 0).sum() > 10 and (acc == 1).sum() > 10


def test_apply_update_order_and_zero_moments():
    P, n, nn = 5, 7, 4
    planes = np.arange(P * n, dtype=np.float32).reshape(P, n)
    m, v = planes + 100, planes + 200
    keep = np.array([1, 0, 1, 1, 0, 1, 1], np.uint8)
    new = -np.arange(P * nn, dtype=np.float32).reshape(P, nn) - 1
    acc = np.array([0, 1, 1, 0], np.uint8)
    tags = np.arange(n, dtype=np.uint32); ntags = np.arange(nn, dtype=np.uint32) + 50
    p2, m2, v2, t2 = oracle.apply_update(planes, m, v, keep, new, acc, tags, ntags)
    np.testing.assert_array_equal(p2, np.concatenate([planes[:, [0, 2, 3, 5, 6]], new[:, [1, 2]]], axis=1))
    np.testing.assert_array_equal(m2[:, 5:], 0) and np.testing.assert_array_equal(v2[:, :5], v[:, [0, 2, 3, 5, 6]])
    np.testing.assert_array_equal(t2, [0, 2, 3, 5, 6, 51, 52])
