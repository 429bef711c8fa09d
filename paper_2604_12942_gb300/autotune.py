"""Autotuner of the batched mapping step's kernel shape.

Picks the tile size (8x8 or 16x16 pixels) and the per-CTA Gaussian chunk staged in shared
memory (32, 64, 128 or 256) by timing whole steps on the device with CUDA events, and
caches the choice in a JSON file keyed by (GPU name, Gaussian-count bucket, image-size
set, SH degree).  Host logic only; the timed work is the library's kernels.
"""
from __future__ import annotations

import json
import math
import os
import threading
from dataclasses import dataclass

TILES = (8, 16)
CHUNKS = (32, 64, 128, 256)
_lock = threading.Lock()


def cache_path() -> str:
    base = os.environ.get("GS_GB300_CACHE") or os.path.join(os.path.expanduser("~"), ".cache", "gs_gb300")
    return os.path.join(base, "autotune.json")


def n_bucket(n: int) -> int:
    """Gaussian counts are bucketed by powers of two (the kernel shape optimum moves slowly)."""
    return 1 << max(0, math.ceil(math.log2(max(1, n))))


def cache_key(gpu_name: str, n: int, sizes, sh_degree: int) -> str:
    res = ",".join(f"{w}x{h}" for w, h in sorted(sizes))
    return f"{gpu_name}|n<={n_bucket(n)}|{res}|sh{sh_degree}"


def load_cache(path: str | None = None) -> dict:
    path = path or cache_path()
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(d: dict, path: str | None = None) -> None:
    path = path or cache_path()
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + f".{os.getpid()}.tmp"
        with open(tmp, "w") as f:
            json.dump(d, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass


@dataclass
class Choice:
    tile: int
    chunk: int
    ms: float
    table: dict


def pick(timings: dict) -> tuple:
    """The (tile, chunk) with the smallest time; ties go to the larger tile, then the smaller
    chunk (fewer CTAs, less shared memory)."""
    return min(timings, key=lambda k: (timings[k], -k[0], k[1]))


def tune(time_config, key: str, candidates=None, path: str | None = None, force: bool = False) -> Choice:
    """Return the cached choice for `key`, or time every candidate with
    `time_config(tile, chunk) -> ms per step` (float('inf') if it cannot run), cache the
    best and return it."""
    with _lock:
        cache = load_cache(path)
        if not force and key in cache:
            c = cache[key]
            return Choice(int(c["tile"]), int(c["chunk"]), float(c["ms"]), c.get("table", {}))
    cands = candidates or [(t, c) for t in TILES for c in CHUNKS]
    timings = {}
    for tile, chunk in cands:
        try:
            timings[(tile, chunk)] = float(time_config(tile, chunk))
        except Exception:  # a configuration that cannot run is simply not chosen
            timings[(tile, chunk)] = float("inf")
    best = pick(timings)
    if not math.isfinite(timings[best]):
        raise RuntimeError("autotune: no candidate configuration ran")
    table = {f"{t}x{c}": round(v, 4) for (t, c), v in timings.items()}
    with _lock:
        cache = load_cache(path)
        cache[key] = {"tile": best[0], "chunk": best[1], "ms": timings[best], "table": table}
        save_cache(cache, path)
    return Choice(best[0], best[1], timings[best], table)


def time_mapping_step(planes, sh_degree, cams, targets, tile, chunk, max_pairs, steps=3, warmup=1):
    """ms per step of the full mapping step (no parameter update, so every candidate sees
    the same map) for one (tile, chunk) configuration."""
    import torch

    from .core import MappingStep, default_opts
    p = planes.clone()
    st = MappingStep(p, sh_degree, cams, default_opts(tile=tile, chunk=chunk), max_pairs=max_pairs)
    trgb, tdep = targets
    for _ in range(warmup):
        st(trgb, tdep, optimize=False)
    torch.cuda.synchronize()
    if st.ws.counters().status != 0:
        return float("inf")
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        st(trgb, tdep, optimize=False)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    del st, p
    return ms
