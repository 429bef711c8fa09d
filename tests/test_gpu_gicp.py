"""Gaussian-GICP loop registration through the C ABI against the oracle (oracle/gicp.py): the
frustum target set bit-exact (FP32 decisions taken the same way), and the registered transform
equal to the oracle's and to the known loop transform."""
import numpy as np
import pytest
import torch

import paper_2604_12942_gb300 as gs
import synth
from oracle import gicp

pytestmark = pytest.mark.gpu

Rotation = pytest.importorskip("scipy.spatial.transform").Rotation


def _scene_planes(seed, n, sh_degree=0):
    sc = synth.uniform_box_scene(seed, n, sh_degree=sh_degree, box=((-8, 8), (-8, 8), (-2, 30)))
    return sc, torch.as_tensor(sc.planes(), device="cuda").contiguous()


def test_target_set_matches_oracle():
    sc, planes = _scene_planes(3, 60_000)
    rot = Rotation.from_euler("xyz", [0.1, -0.2, 0.05]).as_matrix()
    cams = [synth.camera(320, 240, 250.0), synth.camera(200, 150, 120.0, R=rot, t=[0.5, -0.3, 1.0]),
            synth.camera(160, 120, 90.0, R=rot.T, t=[-1.0, 0.2, -4.0])]
    rng = np.random.default_rng(1)
    src = (rng.random(sc.n) < 0.1).astype(np.uint8)
    flag, cnt = gs.gicp_target_set(planes, 0, cams, 0.2, 20.0, torch.as_tensor(src, device="cuda"))
    ref = gicp.target_set(sc.planes()[0:3], cams, 0.2, 20.0, src)
    np.testing.assert_array_equal(flag.cpu().numpy(), ref)
    assert cnt == int(ref.sum()) and 0 < cnt < sc.n


def _planar_map(rng, n):
    """Means on a few planes (walls and floor, like LiDAR-shaped maps), flat Gaussians."""
    pts = []
    for k in range(6):
        nrm = rng.normal(size=3); nrm /= np.linalg.norm(nrm)
        a = np.cross(nrm, [1, 0, 0] if abs(nrm[0]) < 0.9 else [0, 1, 0]); a /= np.linalg.norm(a)
        b = np.cross(nrm, a)
        uv = rng.uniform(-3, 3, (2, n // 6))
        pts.append(rng.normal(size=3)[:, None] * 2 + a[:, None] * uv[0] + b[:, None] * uv[1])
    means = np.concatenate(pts, axis=1)
    quats = rng.normal(size=(4, means.shape[1])); quats /= np.linalg.norm(quats, axis=0)
    ls = rng.normal(-2, 0.3, (3, means.shape[1]))
    return means, quats, ls


def _planes_of(means, quats, ls):
    n = means.shape[1]
    P = np.zeros((gs.n_planes(0), n), np.float32)
    P[0:3], P[3:6], P[6:10] = means, ls, quats
    return P


def test_register_matches_oracle_and_known_transform():
    rng = np.random.default_rng(5)
    means, quats, ls = _planar_map(rng, 6000)
    tar = _planes_of(means, quats, ls)
    sel = rng.choice(tar.shape[1], 1500, replace=False)
    T_gt = gicp.se3_exp(np.array([0.2, -0.1, 0.08, 0.03, -0.02, 0.05]))
    Ti = np.linalg.inv(T_gt)
    # the source rows: the selected Gaussians seen from the other side of the loop
    src_means = Ti[:3, :3] @ tar[0:3, sel].astype(np.float64) + Ti[:3, 3:]
    src_R = Ti[:3, :3] @ np.stack([gicp.quat_to_R(q) for q in tar[6:10, sel].T])
    q_xyzw = Rotation.from_matrix(src_R).as_quat()
    src = _planes_of(src_means, np.stack([q_xyzw[:, 3], q_xyzw[:, 0], q_xyzw[:, 1], q_xyzw[:, 2]]), tar[3:6, sel])
    T_dev = torch.as_tensor(tar, device="cuda")
    S_dev = torch.as_tensor(src, device="cuda")
    T, res = gs.gicp_register(S_dev, None, T_dev, None, 0, np.eye(4), d_corr=1.0, max_iters=30, eps=1e-7)
    covs = [gicp.planar_covariance(src[6:10, m], src[3:6, m]) for m in range(src.shape[1])]
    covt = [gicp.planar_covariance(tar[6:10, m], tar[3:6, m]) for m in range(tar.shape[1])]
    T_ref, cost, cnt, it, conv = gicp.register(src[0:3], covs, tar[0:3], covt, np.eye(4), 1.0, 30, 1e-7)
    assert res.converged == 1 and conv
    assert res.n_corr == cnt and res.iters == it
    np.testing.assert_allclose(T, T_ref, atol=1e-6)
    np.testing.assert_allclose(T, T_gt, atol=1e-4)
    assert abs(res.cost - cost) <= 1e-5 * max(1.0, cost)


def test_register_with_flags_uses_only_flagged_rows():
    rng = np.random.default_rng(6)
    means, quats, ls = _planar_map(rng, 3000)
    P = _planes_of(means, quats, ls)
    n = P.shape[1]
    src_flag = (rng.random(n) < 0.3).astype(np.uint8)
    tar_flag = (1 - src_flag).astype(np.uint8)
    dev = torch.as_tensor(P, device="cuda")
    T, res = gs.gicp_register(dev, torch.as_tensor(src_flag, device="cuda"), dev,
                              torch.as_tensor(tar_flag, device="cuda"), 0, np.eye(4), d_corr=0.5, max_iters=10)
    s_idx, t_idx = np.nonzero(src_flag)[0], np.nonzero(tar_flag)[0]
    covs = [gicp.planar_covariance(P[6:10, m], P[3:6, m]) for m in s_idx]
    covt = [gicp.planar_covariance(P[6:10, m], P[3:6, m]) for m in t_idx]
    T_ref, cost, cnt, it, conv = gicp.register(P[0:3, s_idx], covs, P[0:3, t_idx], covt, np.eye(4), 0.5, 10, 1e-7)
    assert res.n_corr == cnt and res.iters == it
    np.testing.assert_allclose(T, T_ref, atol=1e-6)


def test_register_source_map_larger_than_target_hash():
    """A source map of 5000 rows against 600 target rows (hash of 2048 cells): the flagged
    source rows are listed and summed in three segments of the source map; the result is the
    oracle's on the flagged rows alone."""
    rng = np.random.default_rng(9)
    means, quats, ls = _planar_map(rng, 600)
    tar = _planes_of(means, quats, ls)
    T_gt = gicp.se3_exp(np.array([0.1, 0.05, -0.06, -0.02, 0.03, 0.01]))
    Ti = np.linalg.inv(T_gt)
    n_src, sel = 5000, rng.choice(tar.shape[1], 400, replace=False)
    rows = np.sort(rng.choice(n_src, 400, replace=False))        # spread over every segment
    src = _planes_of(rng.uniform(500, 600, (3, n_src)), np.tile([[1.0], [0], [0], [0]], (1, n_src)),
                     np.full((3, n_src), -2.0))                   # unflagged rows far away
    src[0:3, rows] = Ti[:3, :3] @ tar[0:3, sel].astype(np.float64) + Ti[:3, 3:]
    src_R = Ti[:3, :3] @ np.stack([gicp.quat_to_R(q) for q in tar[6:10, sel].T])
    q_xyzw = Rotation.from_matrix(src_R).as_quat()
    src[6:10, rows] = np.stack([q_xyzw[:, 3], q_xyzw[:, 0], q_xyzw[:, 1], q_xyzw[:, 2]])
    src[3:6, rows] = tar[3:6, sel]
    flag = np.zeros(n_src, np.uint8)
    flag[rows] = 1
    T, res = gs.gicp_register(torch.as_tensor(src, device="cuda"), torch.as_tensor(flag, device="cuda"),
                              torch.as_tensor(tar, device="cuda"), None, 0, np.eye(4), d_corr=1.0, max_iters=30,
                              eps=1e-7)
    s = src[:, rows]
    covs = [gicp.planar_covariance(s[6:10, m], s[3:6, m]) for m in range(s.shape[1])]
    covt = [gicp.planar_covariance(tar[6:10, m], tar[3:6, m]) for m in range(tar.shape[1])]
    T_ref, cost, cnt, it, conv = gicp.register(s[0:3], covs, tar[0:3], covt, np.eye(4), 1.0, 30, 1e-7)
    assert res.n_corr == cnt and res.iters == it and res.converged == int(conv)
    np.testing.assert_allclose(T, T_ref, atol=1e-6)
    np.testing.assert_allclose(T, T_gt, atol=1e-4)
    assert abs(res.cost - cost) <= 1e-5 * max(1.0, cost)
