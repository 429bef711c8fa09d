"""FP64 oracle of the full mapping objective with SSIM and the render-derived masks -- TEST
INFRASTRUCTURE ONLY (imported by the tests, never by the product path).

RMGS-SLAM §III-C, "Optimization": the supervision is restricted to an interior mask obtained by
eroding a geometric support mask taken from the accumulated opacity of the current rendering,
and the objective is lambda_rgb L_rgb + lambda_ssim L_ssim + lambda_depth L_depth over that mask.

Readings of what the paper leaves open:
  * M_geo(x) = [1 - T_final(x) >= tau], tau = 0.5, decided on the FP32 T_final in FP32.
  * Erode(M, r): binary erosion with a disk of radius r (offsets with dx^2 + dy^2 <= r^2);
    pixels outside the image count as outside M, so a band of width r at the border erodes.
  * A caller-supplied mask, when given, is intersected with M_int.
  * SSIM(C|_M, C~|_M): x = C * M and y = C~ * M per channel, 11 x 11 Gaussian window with
    sigma 1.5 (normalised), zero padding outside the image, C1 = 0.01^2, C2 = 0.03^2; the SSIM
    map is averaged over the pixels of M and the 3 channels (an empty mask gives L_ssim = 0).
  * The masks are constants of the step: no gradient flows through them.
Everything here is plain NumPy over whole images, written from the definitions.
"""
from __future__ import annotations

import numpy as np

SSIM_C1 = 0.01 ** 2
SSIM_C2 = 0.03 ** 2


def render_mask(T_final, tau=0.5, r_erode=2, caller_mask=None):
    """M_int = Erode(M_geo, r) (and the caller's mask); T_final is the FP32 transmittance."""
    T32 = np.asarray(T_final, dtype=np.float32)
    geo = (np.float32(1.0) - T32) >= np.float32(tau)   # FP32 decision, as the kernel takes it
    m = erode(geo, r_erode)
    if caller_mask is not None:
        m &= np.asarray(caller_mask) != 0
    return m.astype(np.uint8)


def erode(mask, r):
    """Binary erosion with the radius-r disk; outside the image is outside the mask."""
    mask = np.asarray(mask, dtype=bool)
    H, W = mask.shape
    out = mask.copy()
    for dy in range(-r, r + 1):
        for dx in range(-r, r + 1):
            if dx * dx + dy * dy > r * r:
                continue
            shifted = np.zeros_like(mask)
            ys0, ys1 = max(0, dy), min(H, H + dy)      # source rows y + dy inside the image
            xs0, xs1 = max(0, dx), min(W, W + dx)
            shifted[ys0 - dy:ys1 - dy, xs0 - dx:xs1 - dx] = mask[ys0:ys1, xs0:xs1]
            out &= shifted
    return out


def gaussian_window(size=11, sigma=1.5):
    """Normalised 2-D Gaussian window (outer product of the 1-D one)."""
    k = np.arange(size, dtype=np.float64) - (size - 1) / 2.0
    g = np.exp(-(k * k) / (2.0 * sigma * sigma))
    g /= g.sum()
    return np.outer(g, g)


def conv_same(img, w):
    """sum_{a,b} w[a, b] img[y + a - h, x + b - h] with zeros outside (w symmetric, so this
    correlation is also the convolution)."""
    H, W = img.shape
    h = w.shape[0] // 2
    pad = np.zeros((H + 2 * h, W + 2 * h))
    pad[h:h + H, h:h + W] = img
    out = np.zeros((H, W))
    for a in range(w.shape[0]):
        for b in range(w.shape[1]):
            out += w[a, b] * pad[a:a + H, b:b + W]
    return out


def ssim_terms(x, y, w):
    """Local statistics and the SSIM map of one channel."""
    mx, my = conv_same(x, w), conv_same(y, w)
    exx, eyy, exy = conv_same(x * x, w), conv_same(y * y, w), conv_same(x * y, w)
    sxx, syy, sxy = exx - mx * mx, eyy - my * my, exy - mx * my
    A1, A2 = 2 * mx * my + SSIM_C1, 2 * sxy + SSIM_C2
    B1, B2 = mx * mx + my * my + SSIM_C1, sxx + syy + SSIM_C2
    S = A1 * A2 / (B1 * B2)
    return dict(mx=mx, my=my, A1=A1, A2=A2, B1=B1, B2=B2, S=S)


def ssim_loss(C, tC, M, w=None):
    """L_ssim = 1 - mean over M and channels of SSIM(C*M, C~*M), and dL_ssim/dC [3, H, W]."""
    w = gaussian_window() if w is None else w
    M = np.asarray(M, dtype=np.float64)
    nm = M.sum()
    gC = np.zeros(C.shape)
    if nm == 0:
        return 0.0, gC
    total = 0.0
    for c in range(3):
        x, y = C[c] * M, tC[c] * M
        t = ssim_terms(x, y, w)
        total += float((t["S"] * M).sum())
        # dS/dmu_x, dS/dE[x^2], dS/dE[xy] at every window centre q (sigma_x^2 = E[x^2] - mu_x^2,
        # sigma_xy = E[xy] - mu_x mu_y), weighted by the mean's coefficient -M(q) / (3 |M|)
        S, A1, A2, B1, B2, mx, my = t["S"], t["A1"], t["A2"], t["B1"], t["B2"], t["mx"], t["my"]
        d_mu = 2 * my * (A2 - A1) / (B1 * B2) - 2 * mx * S * (1.0 / B1 - 1.0 / B2)
        d_exx = -S / B2
        d_exy = 2 * A1 / (B1 * B2)
        k = -M / (3.0 * nm)
        # x(p) enters mu_x(q), E[x^2](q), E[xy](q) with weight w(q - p): sum over q is a
        # convolution of the weighted partials; then x = C * M
        gx = conv_same(k * d_mu, w) + 2 * x * conv_same(k * d_exx, w) + y * conv_same(k * d_exy, w)
        gC[c] = gx * M
    return 1.0 - total / (3.0 * nm), gC


def masked_objective(C, D, tC, tD, M, lambda_rgb=1.0, lambda_ssim=0.2, lambda_depth=0.1, scale=1.0):
    """One view's lambda_rgb L_rgb + lambda_ssim L_ssim + lambda_depth L_depth over M, with
    dL/dC and dL/dD, all multiplied by `scale` (1 / views for the step's mean over views).
    L_rgb sums the 3 channels' |residuals| over M / |M|; L_depth counts M with D~ > 0."""
    C, D, tC, tD = (np.asarray(a, dtype=np.float64) for a in (C, D, tC, tD))
    M = np.asarray(M) != 0
    nm = int(M.sum())
    Md = M & (tD > 0)
    nd = int(Md.sum())
    gC = np.zeros(C.shape)
    gD = np.zeros(D.shape)
    loss = 0.0
    if nm > 0:
        r = C - tC
        loss += lambda_rgb * float(np.abs(r)[:, M].sum()) / nm
        gC += lambda_rgb * np.sign(r) * M / nm
        ls, gs = ssim_loss(C, tC, M)
        loss += lambda_ssim * ls
        gC += lambda_ssim * gs
    if nd > 0:
        rd = D - tD
        loss += lambda_depth * float(np.abs(rd)[Md].sum()) / nd
        gD += lambda_depth * np.sign(rd) * Md / nd
    return loss * scale, gC * scale, gD * scale
