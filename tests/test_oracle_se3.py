"""Pins of the SE(3) pose-increment oracle (no GPU), and the library's host-side twist helpers
(gs_twist_cameras, gs_twist_grad: plain host code, no kernel) against it.

Exp is checked against the Rodrigues closed form written out here; the left Jacobian against
its own defining property by central differences through the matrix logarithm, against the
textbook closed form of its rotation block, and against J(xi) xi = xi."""
import ctypes as C
import math

import numpy as np
import pytest
import scipy.linalg

import synth
from oracle import se3

XIS = [np.zeros(6), np.array([0.3, -0.2, 0.5, 0.1, -0.4, 0.25]), np.array([1.5, 0.0, -2.0, 0.0, 0.0, 2.9]),
       np.array([-0.01, 0.02, 0.005, 1e-4, -2e-4, 3e-4])]


def _skew(w):
    return np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]])


@pytest.mark.parametrize("k", range(len(XIS)))
def test_exp_is_the_rodrigues_closed_form(k):
    xi = XIS[k]
    rho, phi = xi[:3], xi[3:]
    th = np.linalg.norm(phi)
    K = _skew(phi)
    if th < 1e-9:
        R, V = np.eye(3) + K, np.eye(3) + 0.5 * K
    else:
        R = np.eye(3) + math.sin(th) / th * K + (1 - math.cos(th)) / th ** 2 * K @ K
        V = np.eye(3) + (1 - math.cos(th)) / th ** 2 * K + (th - math.sin(th)) / th ** 3 * K @ K
    T = se3.exp(xi)
    np.testing.assert_allclose(T[:3, :3], R, atol=1e-13)
    np.testing.assert_allclose(T[:3, 3], V @ rho, atol=1e-13)
    np.testing.assert_allclose(T[3], [0, 0, 0, 1], atol=0)


@pytest.mark.parametrize("k", range(len(XIS)))
def test_left_jacobian_by_its_definition_and_closed_form(k):
    xi = XIS[k]
    J = se3.left_jacobian(xi)
    # J(xi) xi = xi (ad_xi xi = 0)
    np.testing.assert_allclose(J @ xi, xi, atol=1e-13)
    # block upper-triangular with the SO(3) left Jacobian on the diagonal
    phi = xi[3:]
    th = np.linalg.norm(phi)
    K = _skew(phi)
    Jr = np.eye(3) if th < 1e-9 else (np.eye(3) + (1 - math.cos(th)) / th ** 2 * K
                                      + (th - math.sin(th)) / th ** 3 * K @ K)
    np.testing.assert_allclose(J[:3, :3], Jr, atol=1e-12)
    np.testing.assert_allclose(J[3:, 3:], Jr, atol=1e-12)
    np.testing.assert_allclose(J[3:, :3], 0, atol=1e-14)
    # Exp(xi + h e_k) Exp(xi)^-1 = Exp(h J e_k + O(h^2)): central differences through logm
    Einv = np.linalg.inv(se3.exp(xi))
    h = 1e-6
    for c in range(6):
        e = np.zeros(6)
        e[c] = h
        Lp = np.real(scipy.linalg.logm(se3.exp(xi + e) @ Einv))
        Lm = np.real(scipy.linalg.logm(se3.exp(xi - e) @ Einv))
        np.testing.assert_allclose(se3.vee(Lp - Lm) / (2 * h), J[:, c], atol=1e-7)


def test_twist_grad_is_the_chain_rule_of_a_pose_function():
    """f(T) = sum of a fixed weight matrix times (T p) over a few points: the gradient of
    f(Exp(xi) T0) w.r.t. xi by central differences equals J^T times the left-increment
    gradient at Exp(xi) T0 (itself by central differences)."""
    rng = np.random.default_rng(3)
    P = rng.normal(size=(4, 5))
    P[3] = 1.0
    W = rng.normal(size=(4, 5))
    T0 = se3.exp(np.array([0.2, 0.1, -0.3, 0.4, 0.3, -0.2]))

    def f(T):
        return float(np.sum(W * (T @ P)))
    xi = XIS[1]
    h = 1e-6
    g_xi = np.zeros(6)
    g_left = np.zeros(6)
    for c in range(6):
        e = np.zeros(6)
        e[c] = h
        g_xi[c] = (f(se3.exp(xi + e) @ T0) - f(se3.exp(xi - e) @ T0)) / (2 * h)
        g_left[c] = (f(se3.exp(e) @ se3.exp(xi) @ T0) - f(se3.exp(-e) @ se3.exp(xi) @ T0)) / (2 * h)
    np.testing.assert_allclose(se3.twist_grad(xi, g_left), g_xi, rtol=1e-7, atol=1e-7)


@pytest.fixture(scope="module")
def native():
    from paper_2604_12942_gb300 import build
    build.build()
    from paper_2604_12942_gb300 import _native
    return _native


def test_library_twist_helpers_match_the_oracle(native):
    import paper_2604_12942_gb300 as gs
    lib = native.lib()
    R = se3.exp(np.array([0, 0, 0, 0.3, -0.5, 0.2]))[:3, :3]
    cams = [synth.camera(64, 48, 60.0, R=R, t=[0.5, -1.0, 2.0]), synth.camera(32, 24, 30.0)]
    xi = np.stack([XIS[1], XIS[3]]).astype(np.float32)
    arr = gs.camera_array(cams)
    out = (native.Camera * 2)()
    assert lib.gs_twist_cameras(arr, xi.ctypes.data_as(C.c_void_p), 2, out) == 0
    for v in range(2):
        ref = se3.move_camera(cams[v], xi[v].astype(np.float64))
        np.testing.assert_allclose(np.array(out[v].R_cw).reshape(3, 3), ref["R"], atol=2e-7)
        np.testing.assert_allclose(np.array(out[v].t_cw), ref["t"], atol=1e-6)
        assert out[v].width == cams[v]["width"] and out[v].fx == cams[v]["fx"]
    g = np.random.default_rng(1).normal(size=(2, 6)).astype(np.float32)
    gx = np.zeros((2, 6), np.float32)
    assert lib.gs_twist_grad(xi.ctypes.data_as(C.c_void_p), g.ctypes.data_as(C.c_void_p), 2,
                             gx.ctypes.data_as(C.c_void_p)) == 0
    for v in range(2):
        np.testing.assert_allclose(gx[v], se3.twist_grad(xi[v].astype(np.float64), g[v].astype(np.float64)),
                                   rtol=1e-6, atol=1e-6)
    bad = xi.copy()
    bad[0, 2] = np.nan
    assert lib.gs_twist_cameras(arr, bad.ctypes.data_as(C.c_void_p), 2, out) == 5
    assert lib.gs_twist_grad(bad.ctypes.data_as(C.c_void_p), g.ctypes.data_as(C.c_void_p), 2,
                             gx.ctypes.data_as(C.c_void_p)) == 5
    assert lib.gs_twist_grad(None, g.ctypes.data_as(C.c_void_p), 2, gx.ctypes.data_as(C.c_void_p)) == 1
