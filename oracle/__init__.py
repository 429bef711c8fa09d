"""FP64 CPU oracle of the differentiable 3DGS mapping step -- TEST INFRASTRUCTURE ONLY.

Only the tests, `__graft_entry__.smoke()` and the bench's `cpu_baseline` leg may import this
package.  The CUDA product path never routes through it.  The arithmetic lives in
`gs_oracle.c` (plain C, double precision, OpenMP over pixels / Gaussians); this module
builds it with gcc, loads it with ctypes and converts NumPy arrays.

Functions follow the paper's §III-C (rendering, depth by the same weights, L1 losses,
masked sparse optimizer) under the readings listed at the top of gs_oracle.c.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gs_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "voxel_pca.c")]
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libgs_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile gs_oracle.c into oracle/_build/libgs_oracle.so (gcc, -O2, OpenMP, no FP
    contraction so FP32 decisions are taken exactly as written)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or any(os.path.getmtime(_LIB_PATH) < os.path.getmtime(f)
                                                     for f in _SRCS):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp] + _SRCS + ["-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Cam(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("fx", C.c_double), ("fy", C.c_double),
                ("cx", C.c_double), ("cy", C.c_double), ("R", C.c_double * 9), ("t", C.c_double * 3)]


class _Opts(C.Structure):
    _fields_ = [("near_z", C.c_double), ("dilation", C.c_double), ("alpha_min", C.c_double),
                ("alpha_max", C.c_double), ("T_min", C.c_double), ("clamp_fov", C.c_double),
                ("bg", C.c_double * 3)]


class _Proj(C.Structure):
    _fields_ = [("visible", C.c_void_p), ("u", C.c_void_p), ("v", C.c_void_p), ("z", C.c_void_p),
                ("cov2d", C.c_void_p), ("conic", C.c_void_p), ("opacity", C.c_void_p),
                ("rgb", C.c_void_p), ("rx", C.c_void_p), ("ry", C.c_void_p), ("fragile", C.c_void_p),
                ("zkey", C.c_void_p)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            vp, i64, i32, dbl = C.c_void_p, C.c_int64, C.c_int, C.c_double
            L.or_sh_basis.argtypes = [i32, vp, vp, vp]
            L.or_project.argtypes = [i64, i32, vp, vp, vp, vp, vp, C.POINTER(_Cam), C.POINTER(_Opts),
                                     C.POINTER(_Proj)]
            L.or_render.argtypes = [i64, C.POINTER(_Proj), C.POINTER(_Cam), C.POINTER(_Opts), dbl, i32,
                                    vp, vp, vp, vp, vp]
            L.or_l1_loss.argtypes = [i32, i32, vp, vp, vp, vp, vp, dbl, dbl, dbl, vp, vp]
            L.or_l1_loss.restype = dbl
            L.or_render_backward.argtypes = [i64, C.POINTER(_Proj), C.POINTER(_Cam), C.POINTER(_Opts),
                                             i32, vp, vp, vp]
            L.or_project_backward.argtypes = [i64, i32, vp, vp, vp, vp, vp, C.POINTER(_Cam),
                                              C.POINTER(_Opts), vp, vp, vp]
            L.or_adam.argtypes = [i64, i32, vp, vp, vp, vp, vp, vp, dbl, dbl, dbl, i64]
            L.or_bin_view.argtypes = [i64, vp, vp, vp, vp, vp, i32, i32, i32, i64, i64, vp, vp, vp]
            L.or_bin_view.restype = i64
            L.or_sort_pairs.argtypes = [i64, vp, vp]
            L.or_tile_ranges.argtypes = [i64, vp, i64, vp]
            L.or_jacobi3.argtypes = [vp, vp, vp]
            L.or_eig_sorted.argtypes = [vp, vp, vp]
            L.or_descriptor_cov.argtypes = [i64, vp, vp, vp, vp, i32, dbl, vp, vp]
            L.or_voxel_key.argtypes = [vp, C.c_float]
            L.or_voxel_key.restype = i64
            L.or_voxel_pca.argtypes = [i64, vp, C.c_float, i32, dbl, dbl, dbl, dbl, vp, vp, vp, vp, vp, vp, vp, vp]
            L.or_voxel_pca.restype = i64
            _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


@dataclass
class Opts:
    """Compositing constants (readings of the paper's "standard" splatting, §III-C)."""
    near_z: float = 0.2
    dilation: float = 0.3
    alpha_min: float = 1.0 / 255.0
    alpha_max: float = 0.99
    T_min: float = 1e-4
    clamp_fov: float = 1.3
    bg: tuple = (0.0, 0.0, 0.0)
    lambda_rgb: float = 1.0
    lambda_depth: float = 0.1

    def c(self):
        return _Opts(self.near_z, self.dilation, self.alpha_min, self.alpha_max, self.T_min,
                     self.clamp_fov, (C.c_double * 3)(*self.bg))


def _cam(cam) -> _Cam:
    return _Cam(cam["width"], cam["height"], cam["fx"], cam["fy"], cam["cx"], cam["cy"],
                (C.c_double * 9)(*np.asarray(cam["R"], dtype=np.float64).reshape(-1)),
                (C.c_double * 3)(*np.asarray(cam["t"], dtype=np.float64).reshape(-1)))


def sh_basis(deg, d):
    """Real SH Y_k(d) for k < (deg+1)^2 and their gradients dY_k/dd, shape (16,), (16, 3)."""
    d = _f64(d)
    Y = np.zeros(16)
    G = np.zeros(48)
    lib().or_sh_basis(deg, _p(d), _p(Y), _p(G))
    K = (deg + 1) ** 2
    return Y[:K], G.reshape(16, 3)[:K]


def _params(scene):
    return (_f64(scene.means), _f64(scene.log_scales), _f64(scene.quats),
            _f64(scene.opacity_logits), _f64(scene.sh))


_PROJ_FIELDS = ("visible", "u", "v", "z", "cov2d", "conic", "opacity", "rgb", "rx", "ry", "fragile", "zkey")


def project(scene, cam, opts: Opts = Opts()):
    """Per-Gaussian projection into one view.  Returns a dict of arrays; `zkey` is the FP32
    depth key that orders the compositing (front to back, equal keys by index)."""
    n = scene.n
    out = dict(visible=np.zeros(n, np.int32), u=np.zeros(n), v=np.zeros(n), z=np.zeros(n),
               cov2d=np.zeros(3 * n), conic=np.zeros(3 * n), opacity=np.zeros(n),
               rgb=np.zeros(3 * n), rx=np.zeros(n, np.int32), ry=np.zeros(n, np.int32),
               fragile=np.zeros(n, np.int32), zkey=np.zeros(n, np.float32))
    pr = _Proj(*[_p(out[k]).value for k in _PROJ_FIELDS])
    ps = _params(scene)
    lib().or_project(n, scene.sh_degree, *[_p(a) for a in ps], C.byref(_cam(cam)), C.byref(opts.c()),
                     C.byref(pr))
    out["cov2d"] = out["cov2d"].reshape(n, 3)
    out["conic"] = out["conic"].reshape(n, 3)
    out["rgb"] = out["rgb"].reshape(n, 3)
    out["_keep"] = pr
    return out


def _proj_struct(pr):
    for k in ("cov2d", "conic", "rgb"):
        assert pr[k].flags.c_contiguous
    assert pr["zkey"].dtype == np.float32
    return _Proj(*[_p(pr[k]).value for k in _PROJ_FIELDS])


def render(pr, cam, opts: Opts = Opts(), margin=1e-4, use_square=True):
    """Brute-force compositing of one view: C [3,H,W], D, T_final, number of added fragments
    and the per-pixel fragility flag (see gs_oracle.c)."""
    H, W = cam["height"], cam["width"]
    n = pr["u"].shape[0]
    Cimg = np.zeros((3, H, W)); D = np.zeros((H, W)); T = np.zeros((H, W))
    nf = np.zeros((H, W), np.int32); fr = np.zeros((H, W), np.int32)
    lib().or_render(n, C.byref(_proj_struct(pr)), C.byref(_cam(cam)), C.byref(opts.c()), margin,
                    int(use_square), _p(Cimg), _p(D), _p(T), _p(nf), _p(fr))
    return dict(C=Cimg, D=D, T=T, n_frag=nf, fragile=fr.astype(bool))


def l1_loss(img, tgt, opts: Opts = Opts(), scale=1.0):
    """Photometric + depth L1 of one view; returns (loss, dL/dC, dL/dD)."""
    H, W = img["D"].shape
    gC = np.zeros((3, H, W)); gD = np.zeros((H, W))
    Cimg, D = _f64(img["C"]), _f64(img["D"])
    tC, tD = _f64(tgt["rgb"]), _f64(tgt["depth"])
    mask = np.ascontiguousarray(tgt["mask"], dtype=np.uint8)
    loss = lib().or_l1_loss(W, H, _p(Cimg), _p(D), _p(tC), _p(tD), _p(mask), opts.lambda_rgb,
                            opts.lambda_depth, scale, _p(gC), _p(gD))
    return loss, gC, gD


def render_backward(pr, cam, gC, gD, opts: Opts = Opts(), use_square=True):
    """Adjoint of `render`: per-Gaussian [n, 10] gradients w.r.t. (u, v, conic A, B, C,
    opacity, r, g, b, z) for upstream per-pixel dL/dC [3,H,W], dL/dD [H,W]."""
    n = pr["u"].shape[0]
    g2d = np.zeros((n, 10))
    gC, gD = _f64(gC), _f64(gD)
    lib().or_render_backward(n, C.byref(_proj_struct(pr)), C.byref(_cam(cam)), C.byref(opts.c()),
                             int(use_square), _p(gC), _p(gD), _p(g2d))
    return g2d


def project_backward(scene, cam, g2d, opts: Opts = Opts()):
    """Chain rule to the parameter planes [11 + 3K, n] and the pose twist (rho, phi)."""
    n = scene.n
    K = (scene.sh_degree + 1) ** 2
    grads = np.zeros((11 + 3 * K, n))
    twist = np.zeros(6)
    ps = _params(scene)
    g2d = _f64(g2d)
    lib().or_project_backward(n, scene.sh_degree, *[_p(a) for a in ps], C.byref(_cam(cam)),
                              C.byref(opts.c()), _p(g2d), _p(grads), _p(twist))
    return grads, twist


def forward(scene, cams, opts: Opts = Opts(), margin=1e-4):
    """Project and render every view."""
    outs = []
    for cam in cams:
        pr = project(scene, cam, opts)
        img = render(pr, cam, opts, margin)
        outs.append((pr, img))
    return outs


def backward(scene, cams, fwd, upstream, opts: Opts = Opts()):
    """Parameter gradients summed over views and per-view twists, for per-view upstream
    gradients [{gC, gD}]."""
    K = (scene.sh_degree + 1) ** 2
    grads = np.zeros((11 + 3 * K, scene.n))
    twists = np.zeros((len(cams), 6))
    for v, (cam, (pr, img), up) in enumerate(zip(cams, fwd, upstream)):
        g2d = render_backward(pr, cam, up["gC"], up["gD"], opts)
        g, tw = project_backward(scene, cam, g2d, opts)
        grads += g
        twists[v] = tw
    return grads, twists


def loss_and_grads(scene, cams, targets, opts: Opts = Opts(), margin=1e-4):
    """The full mapping-step objective averaged over views, its per-pixel upstream
    gradients, the parameter gradients and the per-view twist gradients."""
    fwd = forward(scene, cams, opts, margin)
    V = len(cams)
    total = 0.0
    ups = []
    for (pr, img), tgt in zip(fwd, targets):
        l, gC, gD = l1_loss(img, tgt, opts, 1.0 / V)
        total += l
        ups.append(dict(gC=gC, gD=gD))
    grads, twists = backward(scene, cams, fwd, ups, opts)
    return dict(loss=total, fwd=fwd, upstream=ups, grads=grads, twists=twists)


LR_DEFAULT = (1.6e-4, 5e-3, 1e-3, 5e-2, 2.5e-3, 1.25e-4)


def adam(p, g, m, v, update, lr=LR_DEFAULT, b1=0.9, b2=0.999, eps=1e-15, step=1):
    """Masked Adam on [P, n] planes in place (float64 copies returned)."""
    p, g, m, v = (_f64(a).copy() for a in (p, g, m, v))
    n_planes, n = p.shape
    upd = None if update is None else np.ascontiguousarray(update, dtype=np.uint8)
    lrs = np.asarray(lr, dtype=np.float64)
    lib().or_adam(n, n_planes, _p(p), _p(g), _p(m), _p(v), None if upd is None else _p(upd), _p(lrs),
                  b1, b2, eps, step)
    return p, m, v


def bin_views(items, cams, tile):
    """Keys/values of every view's records (emission order), then stably sorted, and
    per-tile ranges.  `items` as made by synth.random_projected_items."""
    keys_l, vals_l, touched_l = [], [], []
    tile_off = 0
    idx_off = 0
    tiles_per_view = []
    for it, cam in zip(items, cams):
        W, H = cam["width"], cam["height"]
        n = it["u"].shape[0]
        u = np.ascontiguousarray(it["u"], np.float32); v = np.ascontiguousarray(it["v"], np.float32)
        z = np.ascontiguousarray(it["z"], np.float32)
        rx = np.ascontiguousarray(it["rx"], np.int32); ry = np.ascontiguousarray(it["ry"], np.int32)
        touched = np.zeros(n, np.uint32)
        P = lib().or_bin_view(n, _p(u), _p(v), _p(z), _p(rx), _p(ry), W, H, tile, tile_off, idx_off, None,
                              None, _p(touched))
        keys = np.zeros(P, np.uint64); vals = np.zeros(P, np.uint32)
        lib().or_bin_view(n, _p(u), _p(v), _p(z), _p(rx), _p(ry), W, H, tile, tile_off, idx_off, _p(keys),
                          _p(vals), None)
        keys_l.append(keys); vals_l.append(vals); touched_l.append(touched)
        nt = ((W + tile - 1) // tile) * ((H + tile - 1) // tile)
        tiles_per_view.append(nt)
        tile_off += nt
        idx_off += n
    keys = np.concatenate(keys_l); vals = np.concatenate(vals_l)
    skeys, svals = keys.copy(), vals.copy()
    lib().or_sort_pairs(skeys.shape[0], _p(skeys), _p(svals))
    ranges = np.zeros((tile_off, 2), np.uint32)
    lib().or_tile_ranges(skeys.shape[0], _p(skeys), tile_off, _p(ranges))
    return dict(keys=keys, vals=vals, touched=np.concatenate(touched_l), sorted_keys=skeys,
                sorted_vals=svals, ranges=ranges, n_tiles=tile_off)


# ----------------------------------------------------------------------------------------
# Voxel-PCA geometric fitting (§III-A)
# ----------------------------------------------------------------------------------------

VOXEL_DEFAULTS = dict(voxel=0.5, min_pts=5, tau_p=2.5e-3, tau_l=10.0, sigma=0.02, tau_trace=1e-2)


def voxel_pca(points, voxel=0.5, min_pts=5, tau_p=2.5e-3, tau_l=10.0, sigma=0.02, tau_trace=1e-2):
    """Per-point voxel features of FP32 points [3, n] (see voxel_pca.c): lam [n, 3] ascending,
    V [n, 9] row-major with columns v_min, v_mid, v_max, mu [n, 3], cls, reliable, npts,
    has_feature (npts >= min_pts), vox (dense voxel index), trace, n_voxels."""
    pts = np.ascontiguousarray(points, dtype=np.float32)
    n = pts.shape[1]
    out = dict(vox=np.zeros(n, np.int64), npts=np.zeros(n, np.int32), lam=np.zeros((n, 3)), V=np.zeros((n, 9)),
               mu=np.zeros((n, 3)), cls=np.zeros(n, np.int32), reliable=np.zeros(n, np.int32), trace=np.zeros(n))
    nv = lib().or_voxel_pca(n, _p(pts), voxel, min_pts, tau_p, tau_l, sigma, tau_trace, _p(out["vox"]),
                            _p(out["npts"]), _p(out["lam"]), _p(out["V"]), _p(out["mu"]), _p(out["cls"]),
                            _p(out["reliable"]), _p(out["trace"]))
    out["n_voxels"] = int(nv)
    out["has_feature"] = out["npts"] >= min_pts
    return out


def eig_sorted(C):
    C = _f64(C).reshape(9)
    lam = np.zeros(3); V = np.zeros(9)
    lib().or_eig_sorted(_p(C), _p(lam), _p(V))
    return lam, V.reshape(3, 3)


def descriptor_cov(P, k, sigma=0.02):
    """Sigma_g (6x6) and the per-point Jacobians J_i (N, 6, 3) of one voxel's points P [N, 3]."""
    P = _f64(P)
    N = P.shape[0]
    mu = P.mean(0)
    d = P - mu
    C = d.T @ d / N
    lam, V = eig_sorted(C)
    Sg = np.zeros(36); J = np.zeros(18 * N)
    lib().or_descriptor_cov(N, _p(np.ascontiguousarray(P)), _p(np.ascontiguousarray(mu)), _p(lam),
                            _p(np.ascontiguousarray(V)), k, sigma, _p(Sg), _p(J))
    return Sg.reshape(6, 6), J.reshape(N, 6, 3), lam, V


# The render-derived masks and the SSIM term of the objective (plain NumPy, FP64).
from .objective import (erode, gaussian_window, masked_objective, render_mask,  # noqa: E402,F401
                        ssim_loss)
# Map-size updates between mapping iterations: pruning plan, proximity dedup, compaction.
from .mapupdate import apply_update, dedup_plan, logit_threshold, prune_plan  # noqa: E402,F401
# Gaussian-GICP loop registration (target set, planar covariances, Gauss-Newton on SE(3)).
from . import gicp  # noqa: E402,F401
# SE(3) pose increments (Exp, left Jacobian) of the differentiable rendering's pose gradient.
from . import se3  # noqa: E402,F401
