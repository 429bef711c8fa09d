"""FP64/NumPy oracle of the map-size updates between mapping iterations -- TEST INFRASTRUCTURE
ONLY (imported by the tests, never by the product path).

RMGS-SLAM §III-C: new Gaussians pass a 3-D Euclidean proximity test before insertion (redundant
ones in revisited regions are filtered out), and low-opacity Gaussians are pruned under a
bounded removal ratio.

Readings (the paper gives neither constant nor rule beyond this):
  * prune candidates: opacity sigmoid(logit) < opacity_min, decided on the FP32 logit against
    the FP32 logit of opacity_min (the sigmoid is monotone), opacity_min = 0.005;
  * bounded ratio: at most floor(max_ratio * n) rows go per call (max_ratio = 0.01); when more
    rows are candidates, those with the smallest (logit, row index) go;
  * proximity: a new Gaussian is redundant if some Gaussian already in the map has its mean
    strictly within `radius` (0.05 m), the squared distance summed in FP32 in x, y, z order;
    new Gaussians are not tested against each other;
  * the update keeps the surviving rows in order, appends the accepted new rows in order,
    and gives the new rows zero Adam moments.
"""
from __future__ import annotations

import numpy as np


def logit_threshold(opacity_min):
    """FP32 logit of opacity_min (rows with logit below it are prune candidates)."""
    p = float(opacity_min)
    return np.float32(np.log(p / (1.0 - p)))


def prune_plan(logits, opacity_min=0.005, max_ratio=0.01):
    """keep[i] (uint8) and the number kept."""
    lg = np.asarray(logits, dtype=np.float32)
    n = lg.shape[0]
    cand = np.nonzero(lg < logit_threshold(opacity_min))[0]
    k = min(cand.shape[0], int(np.floor(max_ratio * n)))
    keep = np.ones(n, np.uint8)
    if k > 0:
        order = np.lexsort((cand, lg[cand]))      # by logit, then by index
        keep[cand[order[:k]]] = 0
    return keep, int(keep.sum())


def dedup_plan(map_means, new_means, radius=0.05):
    """accept[j] (uint8) = no map mean within `radius` of new mean j; map_means [3, n]."""
    M = np.asarray(map_means, dtype=np.float32)
    Q = np.asarray(new_means, dtype=np.float32)
    r2 = np.float32(radius) * np.float32(radius)
    accept = np.ones(Q.shape[1], np.uint8)
    step = 256
    for j0 in range(0, Q.shape[1], step):
        q = Q[:, j0:j0 + step]
        dx = (q[0][:, None] - M[0][None, :]).astype(np.float32)
        dy = (q[1][:, None] - M[1][None, :]).astype(np.float32)
        dz = (q[2][:, None] - M[2][None, :]).astype(np.float32)
        d2 = (dx * dx + dy * dy).astype(np.float32) + (dz * dz).astype(np.float32)
        accept[j0:j0 + step] = ~np.any(d2.astype(np.float32) < r2, axis=1)
    return accept, int(accept.sum())


def apply_update(planes, m, v, keep, new_planes=None, accept=None, tags=None, new_tags=None):
    """The updated map: rows with keep != 0 in order, then the new rows with accept != 0.
    planes, m, v: [P, n]; new_planes: [P, n_new]; tags: optional per-row uint32."""
    keep = np.asarray(keep) != 0
    parts_p, parts_m, parts_v = [planes[:, keep]], [m[:, keep]], [v[:, keep]]
    out_tags = [tags[keep]] if tags is not None else None
    if new_planes is not None:
        acc = np.ones(new_planes.shape[1], bool) if accept is None else np.asarray(accept) != 0
        nw = new_planes[:, acc]
        parts_p.append(nw)
        parts_m.append(np.zeros_like(nw))
        parts_v.append(np.zeros_like(nw))
        if out_tags is not None:
            out_tags.append(new_tags[acc])
    res = (np.concatenate(parts_p, axis=1), np.concatenate(parts_m, axis=1), np.concatenate(parts_v, axis=1))
    if out_tags is not None:
        return res + (np.concatenate(out_tags),)
    return res
