"""Seeded synthetic inputs shared by the oracle tests, the GPU parity tests and the bench.

This module only draws numbers: it holds none of the mapping step's arithmetic (no
projection, no compositing, no loss, no optimizer).  Every array it returns is a plain
NumPy array; the callers move them to wherever they need them.

Layouts (structure-of-arrays planes, float32):
  means          [3, n]      world-frame centres
  log_scales     [3, n]      per-axis log standard deviation
  quats          [4, n]      unnormalised rotation quaternion, (w, x, y, z)
  opacity_logits [n]         opacity before the sigmoid
  sh             [3*K, n]    spherical-harmonic coefficients, plane (k*3 + c) holds
                             coefficient k (K = (degree+1)^2) of colour channel c

Cameras are dicts {width, height, fx, fy, cx, cy, R (3x3 world->camera), t (3)} with the
camera looking along +z, +x right and +y down.

Workload recipes (the paper's datasets are not available; these stand in for them):
  uniform_box_scene   Gaussians uniform in a box before one pinhole camera.
  lidar_scene         points from a simulated 32-beam spinning LiDAR driven along a
                      trajectory over a ground plane with box facades, coloured by a
                      procedural texture.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Degree-0 colour: a DC coefficient d gives colour d * Y00 + 0.5 with Y00 = 1 / (2 sqrt(pi)),
# so drawing d uniformly in [-sqrt(pi), sqrt(pi)] gives colours uniform in [0, 1].
_DC_HALF_RANGE = math.sqrt(math.pi)
_DC_PER_UNIT_COLOUR = 2.0 * math.sqrt(math.pi)


def sh_count(degree: int) -> int:
    return (degree + 1) ** 2


@dataclass
class Scene:
    means: np.ndarray
    log_scales: np.ndarray
    quats: np.ndarray
    opacity_logits: np.ndarray
    sh: np.ndarray
    sh_degree: int
    segment_id: np.ndarray | None = None
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.means.shape[1])

    def copy(self) -> "Scene":
        return Scene(self.means.copy(), self.log_scales.copy(), self.quats.copy(),
                     self.opacity_logits.copy(), self.sh.copy(), self.sh_degree,
                     None if self.segment_id is None else self.segment_id.copy(),
                     dict(self.meta))

    def subset(self, idx) -> "Scene":
        idx = np.asarray(idx)
        return Scene(self.means[:, idx].copy(), self.log_scales[:, idx].copy(),
                     self.quats[:, idx].copy(), self.opacity_logits[idx].copy(),
                     self.sh[:, idx].copy(), self.sh_degree,
                     None if self.segment_id is None else self.segment_id[idx].copy(),
                     dict(self.meta))

    def planes(self) -> np.ndarray:
        """All parameters as one [11 + 3K, n] float32 array (means, log-scales, quats,
        opacity logit, SH) -- the packed layout the library also accepts."""
        return np.concatenate([self.means, self.log_scales, self.quats,
                               self.opacity_logits[None, :], self.sh], axis=0).astype(np.float32)


def camera(width, height, fx, fy=None, cx=None, cy=None, R=None, t=None) -> dict:
    fy = fx if fy is None else fy
    return dict(width=int(width), height=int(height), fx=float(fx), fy=float(fy),
                cx=float(width) / 2 if cx is None else float(cx),
                cy=float(height) / 2 if cy is None else float(cy),
                R=np.eye(3) if R is None else np.asarray(R, dtype=np.float64),
                t=np.zeros(3) if t is None else np.asarray(t, dtype=np.float64))


def look_camera(width, height, fx, position, heading, pitch=0.0) -> dict:
    """Camera at `position` (world, z up) looking horizontally along `heading` (radians in
    the xy-plane), tilted down by `pitch` radians."""
    f = np.array([math.cos(heading) * math.cos(pitch), math.sin(heading) * math.cos(pitch),
                  -math.sin(pitch)])
    up = np.array([0.0, 0.0, 1.0])
    r = np.cross(f, up)
    r /= np.linalg.norm(r)
    d = np.cross(f, r)          # camera +y (down) completes a right-handed frame
    R = np.stack([r, d, f], axis=0)
    t = -R @ np.asarray(position, dtype=np.float64)
    return camera(width, height, fx, fx, R=R, t=t)


def random_unit_quats(rng, n) -> np.ndarray:
    q = rng.standard_normal((4, n))
    q /= np.linalg.norm(q, axis=0, keepdims=True)
    return q.astype(np.float32)


def uniform_box_scene(seed=1, n=10_000, sh_degree=0, box=((-3, 3), (-3, 3), (2, 10)),
                      logscale_mu=-3.0, logscale_sigma=0.5, sh_rest_sigma=0.1) -> Scene:
    """Gaussians uniform in an axis-aligned box in front of a camera at the origin.

    log-scale ~ N(logscale_mu, logscale_sigma), random unit quaternions, opacity
    sigmoid(N(0, 1)), degree-0 colour uniform in [0, 1], higher SH ~ N(0, sh_rest_sigma)."""
    rng = np.random.default_rng(seed)
    means = np.stack([rng.uniform(lo, hi, n) for lo, hi in box]).astype(np.float32)
    log_scales = rng.normal(logscale_mu, logscale_sigma, (3, n)).astype(np.float32)
    quats = random_unit_quats(rng, n)
    logits = rng.standard_normal(n).astype(np.float32)
    K = sh_count(sh_degree)
    sh = np.zeros((3 * K, n), dtype=np.float32)
    sh[0:3] = rng.uniform(-_DC_HALF_RANGE, _DC_HALF_RANGE, (3, n))
    if K > 1:
        sh[3:] = rng.normal(0.0, sh_rest_sigma, (3 * (K - 1), n))
    return Scene(means, log_scales, quats, logits, sh, sh_degree,
                 np.zeros(n, dtype=np.int32), {"recipe": "uniform_box", "seed": seed})


def random_targets(seed, cams, depth_range=(2.0, 10.0), depth_hole_frac=0.0):
    """Per view: rgb [3, H, W] ~ U[0, 1], depth [H, W] ~ U[depth_range] (with an optional
    fraction of zero 'no LiDAR return' pixels), mask [H, W] of ones."""
    rng = np.random.default_rng(seed)
    out = []
    for c in cams:
        H, W = c["height"], c["width"]
        rgb = rng.uniform(0, 1, (3, H, W)).astype(np.float32)
        d = rng.uniform(*depth_range, (H, W)).astype(np.float32)
        if depth_hole_frac > 0:
            d[rng.uniform(0, 1, (H, W)) < depth_hole_frac] = 0.0
        out.append(dict(rgb=rgb, depth=d, mask=np.ones((H, W), dtype=np.uint8)))
    return out


def random_upstream(seed, cams, scale=1.0):
    """Per view: seeded upstream gradients dL/dC [3, H, W] and dL/dD [H, W] ~ N(0, scale)."""
    rng = np.random.default_rng(seed)
    return [dict(gC=rng.normal(0, scale, (3, c["height"], c["width"])).astype(np.float32),
                 gD=rng.normal(0, scale, (c["height"], c["width"])).astype(np.float32))
            for c in cams]


# ----------------------------------------------------------------------------------------
# LiDAR-camera-shaped scenes
# ----------------------------------------------------------------------------------------

def _boxes(rng, n_boxes, centre_path, max_dist=60.0):
    """Axis-aligned boxes (facades) with sides 2..20 m placed near points of the path but
    never on it."""
    boxes = []
    while len(boxes) < n_boxes:
        p = centre_path[rng.integers(len(centre_path))]
        size = rng.uniform(2.0, 20.0, 3)
        size[2] = rng.uniform(3.0, 20.0)
        ang = rng.uniform(0, 2 * math.pi)
        dist = rng.uniform(6.0, max_dist * 0.6)
        c = np.array([p[0] + dist * math.cos(ang), p[1] + dist * math.sin(ang)])
        lo = np.array([c[0] - size[0] / 2, c[1] - size[1] / 2, 0.0])
        hi = np.array([c[0] + size[0] / 2, c[1] + size[1] / 2, size[2]])
        # keep a 3 m corridor around the whole path free
        dmin = np.min(np.maximum(np.maximum(lo[None, :2] - centre_path, centre_path - hi[None, :2]),
                                 0.0).max(axis=1))
        if dmin > 3.0:
            boxes.append((lo, hi))
    return boxes


def _cast(origin, dirs, boxes, rmin, rmax):
    """Nearest hit of rays (origin + s*dirs) with the ground plane z=0 and the boxes.
    Returns (hit_points [m,3], normal_axis [m] in {0,1,2})."""
    m = dirs.shape[0]
    best = np.full(m, np.inf)
    axis = np.full(m, 2, dtype=np.int64)
    with np.errstate(divide="ignore", invalid="ignore"):
        s = -origin[2] / dirs[:, 2]
    ok = (dirs[:, 2] < 0) & (s > 0)
    best = np.where(ok, s, best)
    for lo, hi in boxes:
        with np.errstate(divide="ignore", invalid="ignore"):
            t1 = (lo[None, :] - origin[None, :]) / dirs
            t2 = (hi[None, :] - origin[None, :]) / dirs
        tmin = np.minimum(t1, t2)
        tmax = np.maximum(t1, t2)
        tmin = np.nan_to_num(tmin, nan=-np.inf)
        tmax = np.nan_to_num(tmax, nan=np.inf)
        enter = tmin.max(axis=1)
        leave = tmax.min(axis=1)
        hit = (enter <= leave) & (enter > 0) & (enter < best)
        ax = tmin.argmax(axis=1)
        best = np.where(hit, enter, best)
        axis = np.where(hit, ax, axis)
    keep = np.isfinite(best) & (best >= rmin) & (best <= rmax)
    pts = origin[None, :] + best[keep, None] * dirs[keep]
    return pts, axis[keep], best[keep]


def _texture(p, rng_seed):
    """Procedural colour: a 1 m checker mixed with smooth value noise, in [0, 1]^3."""
    rng = np.random.default_rng(rng_seed)
    chk = ((np.floor(p[:, 0]) + np.floor(p[:, 1]) + np.floor(p[:, 2] * 2)) % 2)[:, None]
    freq = rng.uniform(0.2, 1.5, (3, 3))
    phase = rng.uniform(0, 2 * math.pi, (3, 3))
    noise = np.zeros((p.shape[0], 3))
    for c in range(3):
        for j in range(3):
            noise[:, c] += np.sin(p[:, j] * freq[c, j] * 2.0 + phase[c, j])
    base = rng.uniform(0.2, 0.8, 3)
    col = 0.55 * base[None, :] + 0.25 * chk + 0.07 * noise
    return np.clip(col, 0.0, 1.0)


def trajectory(kind, n_poses):
    """Sensor positions (z = 1.8 m) and headings.  'line': 40 m straight along +x; 'loop':
    a 200 m closed rounded rectangle (straight sides 60 m and 100 - 60 - 8*pi m, corner
    radius 8 m), driven counter-clockwise."""
    if kind == "line":
        s = np.linspace(0, 40.0, n_poses)
        pos = np.stack([s, np.zeros_like(s), np.full_like(s, 1.8)], 1)
        return pos, np.zeros(n_poses)
    r, a = 8.0, 60.0
    b = 100.0 - a - math.pi * r
    # (length, kind, start point or arc centre, heading or start angle)
    segs = [(a, "s", (-a / 2, -b / 2 - r), 0.0),
            (math.pi * r / 2, "c", (a / 2, -b / 2), -math.pi / 2),
            (b, "s", (a / 2 + r, -b / 2), math.pi / 2),
            (math.pi * r / 2, "c", (a / 2, b / 2), 0.0),
            (a, "s", (a / 2, b / 2 + r), math.pi),
            (math.pi * r / 2, "c", (-a / 2, b / 2), math.pi / 2),
            (b, "s", (-a / 2 - r, b / 2), -math.pi / 2),
            (math.pi * r / 2, "c", (-a / 2, -b / 2), math.pi)]
    total = sum(sg[0] for sg in segs)
    pos = np.zeros((n_poses, 3))
    head = np.zeros(n_poses)
    for k, sk in enumerate(np.linspace(0, total, n_poses, endpoint=False)):
        for length, kind_j, anchor, ang in segs:
            if sk <= length:
                break
            sk -= length
        if kind_j == "s":
            xy = np.array(anchor) + sk * np.array([math.cos(ang), math.sin(ang)])
            h = ang
        else:
            th = ang + sk / r
            xy = np.array(anchor) + r * np.array([math.cos(th), math.sin(th)])
            h = th + math.pi / 2
        pos[k] = [xy[0], xy[1], 1.8]
        head[k] = h
    return pos, head


def lidar_scene(seed=2, n=500_000, sh_degree=3, kind="line", n_boxes=20, sh_rest_sigma=0.1,
                segments=8):
    """Points of a simulated 32-beam spinning LiDAR (elevations -16..+15 deg, 0.2 deg
    azimuth, returns kept at 0.1..60 m, sensor 1.8 m above the ground) taken along a
    trajectory over a ground plane with `n_boxes` axis-aligned box facades, until `n`
    points are collected.  One Gaussian per point: the smallest axis along the surface
    normal, tangential scale from the beam footprint (range x angular step), opacity
    sigmoid(N(0, 1)), DC colour from a procedural texture, higher SH ~ N(0, sh_rest_sigma).
    Segment ids split the trajectory into `segments` equal parts."""
    rng = np.random.default_rng(seed)
    n_scan_poses = 400 if kind == "loop" else 200
    pos, head = trajectory(kind, n_scan_poses)
    boxes = _boxes(rng, n_boxes, pos[:, :2])
    elev = np.deg2rad(np.linspace(-16.0, 15.0, 32))
    az = np.deg2rad(np.arange(0.0, 360.0, 0.2))
    E, A = np.meshgrid(elev, az, indexing="ij")
    dirs = np.stack([np.cos(E) * np.cos(A), np.cos(E) * np.sin(A), np.sin(E)], -1).reshape(-1, 3)
    pts, axes, ranges, segs = [], [], [], []
    total = 0
    order = rng.permutation(n_scan_poses)
    k = 0
    while total < n:
        pi = order[k % n_scan_poses]
        k += 1
        # small per-scan jitter of the azimuth start so repeated poses add new points
        rot = rng.uniform(0, np.deg2rad(0.2))
        ca, sa = math.cos(rot), math.sin(rot)
        d = dirs @ np.array([[ca, sa, 0], [-sa, ca, 0], [0, 0, 1.0]])
        p, ax, rr = _cast(pos[pi], d, boxes, 0.1, 60.0)
        sub = rng.uniform(0, 1, p.shape[0]) < 0.5       # thin each scan
        pts.append(p[sub]); axes.append(ax[sub]); ranges.append(rr[sub])
        segs.append(np.full(int(sub.sum()), int(pi * segments // n_scan_poses), dtype=np.int32))
        total += int(sub.sum())
    P = np.concatenate(pts)[:n]
    AX = np.concatenate(axes)[:n]
    RR = np.concatenate(ranges)[:n]
    SG = np.concatenate(segs)[:n]
    n = P.shape[0]
    P = P + rng.normal(0, 0.01, P.shape)                 # range noise
    tang = np.log(np.maximum(RR * np.deg2rad(0.4), 0.01))
    normal = np.log(np.full(n, 0.01)) + rng.normal(0, 0.2, n)
    log_scales = np.stack([tang + rng.normal(0, 0.2, n), tang + rng.normal(0, 0.2, n), normal])
    # quaternion taking local z to the face normal axis, plus a little noise
    q = np.zeros((4, n))
    q[0] = 1.0
    s2 = math.sqrt(0.5)
    m0 = AX == 0                      # normal along x: rotate +90 deg about y
    q[:, m0] = np.array([[s2], [0], [s2], [0]])
    m1 = AX == 1                      # normal along y: rotate -90 deg about x
    q[:, m1] = np.array([[s2], [-s2], [0], [0]])
    q += rng.normal(0, 0.05, q.shape)
    q /= np.linalg.norm(q, axis=0, keepdims=True)
    col = _texture(P, seed + 1000)
    K = sh_count(sh_degree)
    sh = np.zeros((3 * K, n), dtype=np.float32)
    sh[0:3] = ((col - 0.5) * _DC_PER_UNIT_COLOUR).T
    if K > 1:
        sh[3:] = rng.normal(0, sh_rest_sigma, (3 * (K - 1), n))
    scene = Scene(P.T.astype(np.float32), log_scales.astype(np.float32), q.astype(np.float32),
                  rng.standard_normal(n).astype(np.float32), sh, sh_degree, SG,
                  {"recipe": f"lidar_{kind}", "seed": seed, "traj_pos": pos, "traj_head": head})
    return scene


def perturbed(scene: Scene, seed, mean_sigma=0.02, scale_sigma=0.1, logit_sigma=0.3,
              sh_sigma=0.05) -> Scene:
    """A perturbed copy (mu + N(0, .02 m), log-scale + N(0, .1), logit + N(0, .3),
    SH + N(0, .05)), used as the ground truth whose render is the target."""
    rng = np.random.default_rng(seed)
    s = scene.copy()
    s.means += rng.normal(0, mean_sigma, s.means.shape).astype(np.float32)
    s.log_scales += rng.normal(0, scale_sigma, s.log_scales.shape).astype(np.float32)
    s.opacity_logits += rng.normal(0, logit_sigma, s.opacity_logits.shape).astype(np.float32)
    s.sh += rng.normal(0, sh_sigma, s.sh.shape).astype(np.float32)
    return s


def trajectory_cameras(scene: Scene, sizes, idx, fx_per_width=0.7, pitch_deg=5.0):
    """Cameras at trajectory poses `idx` of a LiDAR scene with image sizes `sizes`
    [(W, H), ...], fx = fy = fx_per_width * W, tilted slightly down."""
    pos, head = scene.meta["traj_pos"], scene.meta["traj_head"]
    return [look_camera(W, H, fx_per_width * W, pos[i], head[i], math.radians(pitch_deg))
            for (W, H), i in zip(sizes, idx)]


def random_projected_items(seed, cams, n, radius_max=48, zero_frac=0.2, tie_frac=0.3,
                           margin=60.0):
    """Synthetic per-(view, Gaussian) screen-space records for binning tests: float32 centre
    (u, v) uniform over the image +- margin, integer half-extents rx, ry (both 0 for a
    fraction), float32 depth with deliberate exact ties.  Returns a list (one per view) of
    dicts."""
    rng = np.random.default_rng(seed)
    out = []
    for c in cams:
        W, H = c["width"], c["height"]
        u = rng.uniform(-margin, W + margin, n).astype(np.float32)
        v = rng.uniform(-margin, H + margin, n).astype(np.float32)
        rx = np.minimum(rng.geometric(0.12, n), radius_max).astype(np.int32)
        ry = np.minimum(rng.geometric(0.12, n), radius_max).astype(np.int32)
        zero = rng.uniform(0, 1, n) < zero_frac
        rx[zero] = 0
        ry[zero] = 0
        z = rng.uniform(0.2, 80.0, n).astype(np.float32)
        tie = rng.uniform(0, 1, n) < tie_frac
        z[tie] = np.float32(np.round(rng.uniform(0.5, 5.0, int(tie.sum())), 1))
        out.append(dict(u=u, v=v, z=z, rx=rx, ry=ry))
    return out
