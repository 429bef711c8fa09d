"""Pins of the oracle's masks and SSIM objective (CPU): library routines for the erosion and
the windowed sums, closed forms for SSIM, central finite differences for its gradient, and the
C oracle's L1 terms for the lambda_ssim = 0 case."""
import numpy as np
import pytest

import oracle

scipy_ndimage = pytest.importorskip("scipy.ndimage")
scipy_signal = pytest.importorskip("scipy.signal")


def _disk(r):
    y, x = np.mgrid[-r:r + 1, -r:r + 1]
    return (x * x + y * y) <= r * r


@pytest.mark.parametrize("r", [0, 1, 2, 3])
def test_erosion_matches_library(r):
    rng = np.random.default_rng(r)
    m = rng.random((23, 31)) < 0.8
    ref = scipy_ndimage.binary_erosion(m, structure=_disk(r), border_value=0)
    np.testing.assert_array_equal(oracle.erode(m, r), ref)


def test_render_mask_threshold_and_caller_mask():
    T = np.full((9, 9), 0.4, np.float32)
    T[0, 0] = 0.5                       # 1 - 0.5 >= 0.5: inside
    T[8, 8] = np.nextafter(np.float32(0.5), np.float32(1))   # just above: outside
    m = oracle.render_mask(T, tau=0.5, r_erode=0)
    assert m[0, 0] == 1 and m[8, 8] == 0 and m[4, 4] == 1
    caller = np.ones((9, 9), np.uint8); caller[4, 4] = 0
    m = oracle.render_mask(T, tau=0.5, r_erode=1, caller_mask=caller)
    assert m[4, 4] == 0 and m[0, :].sum() == 0 and m[3, 3] == 1


def test_window_and_windowed_sum_match_library():
    w = oracle.gaussian_window()
    assert w.shape == (11, 11) and abs(w.sum() - 1.0) < 1e-14
    g1 = np.exp(-np.arange(-5, 6) ** 2 / (2 * 1.5 ** 2)); g1 /= g1.sum()
    np.testing.assert_allclose(w, np.outer(g1, g1), rtol=0, atol=1e-16)
    img = np.random.default_rng(1).random((17, 20))
    ref = scipy_signal.convolve2d(img, w, mode="same", boundary="fill", fillvalue=0.0)
    np.testing.assert_allclose(oracle.objective.conv_same(img, w), ref, rtol=0, atol=1e-13)


def test_ssim_identical_images_and_constant_closed_form():
    rng = np.random.default_rng(2)
    C = rng.random((3, 20, 24))
    M = np.ones((20, 24), np.uint8)
    loss, g = oracle.ssim_loss(C, C, M)
    assert abs(loss) < 1e-12 and np.abs(g).max() < 1e-12
    a, b = 0.3, 0.7
    t = oracle.objective.ssim_terms(np.full((20, 24), a), np.full((20, 24), b), oracle.gaussian_window())
    ref = (2 * a * b + oracle.objective.SSIM_C1) / (a * a + b * b + oracle.objective.SSIM_C1)
    np.testing.assert_allclose(t["S"][5:-5, 5:-5], ref, rtol=1e-12)


def test_ssim_gradient_matches_finite_differences():
    rng = np.random.default_rng(3)
    H, W = 9, 12
    C = rng.random((3, H, W)); tC = rng.random((3, H, W))
    M = (rng.random((H, W)) < 0.7).astype(np.uint8)
    _, g = oracle.ssim_loss(C, tC, M)
    h = 1e-6
    num = np.zeros_like(C)
    for idx in np.ndindex(C.shape):
        Cp = C.copy(); Cp[idx] += h
        Cm = C.copy(); Cm[idx] -= h
        num[idx] = (oracle.ssim_loss(Cp, tC, M)[0] - oracle.ssim_loss(Cm, tC, M)[0]) / (2 * h)
    np.testing.assert_allclose(g, num, rtol=1e-5, atol=1e-8)
    assert np.all(g[:, M == 0] == 0)


def test_objective_without_ssim_matches_c_oracle_l1():
    rng = np.random.default_rng(4)
    H, W = 14, 17
    C = rng.random((3, H, W)); tC = rng.random((3, H, W))
    D = rng.random((H, W)) * 5; tD = np.where(rng.random((H, W)) < 0.6, rng.random((H, W)) * 5, 0.0)
    M = (rng.random((H, W)) < 0.8).astype(np.uint8)
    l, gC, gD = oracle.masked_objective(C, D, tC, tD, M, 1.0, 0.0, 0.1, 0.5)
    img = dict(C=C, D=D)
    tgt = dict(rgb=tC, depth=tD, mask=M)
    l_ref, gC_ref, gD_ref = oracle.l1_loss(img, tgt, oracle.Opts(lambda_rgb=1.0, lambda_depth=0.1), 0.5)
    assert abs(l - l_ref) < 1e-12
    np.testing.assert_allclose(gC, gC_ref, atol=1e-15)
    np.testing.assert_allclose(gD, gD_ref, atol=1e-15)
