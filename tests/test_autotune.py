"""Host logic of the autotuner (no GPU): candidate timing, choice, JSON cache."""
import math

import pytest

from paper_2604_12942_gb300 import autotune


def test_key_buckets_and_orders_sizes():
    k1 = autotune.cache_key("GB300", 1_900_000, [(1280, 720), (640, 480)], 3)
    k2 = autotune.cache_key("GB300", 2_000_000, [(640, 480), (1280, 720)], 3)
    assert k1 == k2 == "GB300|n<=2097152|640x480,1280x720|sh3"
    assert autotune.cache_key("GB300", 3_000_000, [(640, 480)], 3) != k1


def test_tune_picks_fastest_and_caches(tmp_path):
    calls = []

    def fake(tile, chunk):
        calls.append((tile, chunk))
        return {8: 5.0, 16: 3.0}[tile] + chunk / 1000.0

    path = str(tmp_path / "at.json")
    c = autotune.tune(fake, "k", path=path)
    assert (c.tile, c.chunk) == (16, 32)
    assert len(calls) == 8 and len(c.table) == 8
    # cached: no more timing
    c2 = autotune.tune(fake, "k", path=path)
    assert len(calls) == 8 and (c2.tile, c2.chunk) == (16, 32)
    # forced: times again
    autotune.tune(fake, "k", path=path, force=True)
    assert len(calls) == 16


def test_tune_skips_failing_candidates(tmp_path):
    def fake(tile, chunk):
        if chunk == 32:
            raise RuntimeError("does not fit")
        return math.inf if tile == 8 else float(chunk)

    c = autotune.tune(fake, "k2", path=str(tmp_path / "a.json"))
    assert (c.tile, c.chunk) == (16, 64)
    with pytest.raises(RuntimeError):
        autotune.tune(lambda t, c: math.inf, "k3", path=str(tmp_path / "b.json"))


def test_ties_prefer_larger_tile_then_smaller_chunk():
    assert autotune.pick({(8, 64): 1.0, (16, 128): 1.0, (16, 64): 1.0}) == (16, 64)
