"""The allocation-free pair sort (gs_sort_pairs_noalloc) against the regular binning sort
and the oracle.

Some callers cannot allocate device memory (a no-allocation policy in a real-time loop, a
host callback, a plug-in whose application owns every allocation).  For them the library
offers a sort whose scratch is a fixed array inside the library.  These tests call it
through the C ABI and check, on two calls in a row, that it returns exactly the pairs of the
oracle's stable sort and of gs_bin_sort on the same records (the sort is bit-exact, so the
tolerance is equality); then odd pass counts, where the first pass writes the output
directly, and full 64-bit keys with many duplicates against a stable NumPy sort.  The file
is named so that pytest collects it last.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import oracle
import paper_2604_12942_gb300 as gs
import synth
from paper_2604_12942_gb300 import _native as N
from tests.gpu_helpers import set_vis_bits

pytestmark = pytest.mark.gpu

LIMIT = 1 << 20


def _regular_sort(items, cams, tile):
    """gs_bin_sort on synthetic FP32 screen-space records: the sorted pairs it leaves in
    the workspace, and the unsorted pairs in emission order (from the oracle's binning,
    which matches the library's emission bit for bit)."""
    ref = oracle.bin_views(items, cams, tile)
    n = items[0]["u"].shape[0]
    V = len(cams)
    P = int(ref["keys"].shape[0])
    ws = gs.Workspace(n, cams, gs.default_opts(tile=tile), max(P, 1))
    rec = np.zeros((V, n, 12), np.float32)
    for v, it in enumerate(items):
        rec[v, :, 0] = it["u"]; rec[v, :, 1] = it["v"]; rec[v, :, 2] = it["z"]
        rec[v, :, 7] = it["rx"].view(np.float32)
        rec[v, :, 11] = it["ry"].view(np.float32)
    ws.region("proj", torch.float32, 12 * V * n).copy_(torch.as_tensor(rec.reshape(-1)))
    set_vis_bits(ws, ref["touched"].reshape(V, n) > 0)
    ws.region("counters", torch.int32, 8).zero_()
    ws.bin_sort()
    c = ws.counters()
    assert c.status == 0 and c.n_pairs == P
    k, v = ws.sorted_pairs(P)
    tiles = ws.layout.total_tiles
    key_bits = 32 + max(1, int(np.ceil(np.log2(max(tiles, 2)))))
    return ref, k.clone(), v.clone(), key_bits


def _noalloc(keys_np, vals_np, key_bits):
    n = keys_np.shape[0]
    kin = torch.as_tensor(keys_np.view(np.int64)).cuda()
    vin = torch.as_tensor(vals_np.view(np.int32)).cuda()
    kout = torch.full_like(kin, -1)
    vout = torch.full_like(vin, -1)
    st = N.lib().gs_sort_pairs_noalloc(C.c_void_p(kin.data_ptr()), C.c_void_p(vin.data_ptr()), n, key_bits,
                                       C.c_void_p(kout.data_ptr()), C.c_void_p(vout.data_ptr()),
                                       C.c_void_p(torch.cuda.current_stream().cuda_stream))
    N.check(st, "gs_sort_pairs_noalloc")
    torch.cuda.synchronize()
    # the input is left untouched
    assert torch.equal(kin.cpu(), torch.as_tensor(keys_np.view(np.int64)))
    return kout, vout


def _equal(k, v, keys_np, vals_np):
    return (np.array_equal(k.cpu().numpy().view(np.uint64), keys_np) and
            np.array_equal(v.cpu().numpy().view(np.uint32), vals_np))


def test_noalloc_sort_matches_oracle_and_bin_sort_on_two_calls():
    cams = [synth.camera(1280, 720, 900.0), synth.camera(333, 250, 300.0)]
    # first call: a large case (several chunks per block of the sort grid)
    items = synth.random_projected_items(31, cams, 60_000, radius_max=32)
    ref, k_ref, v_ref, bits = _regular_sort(items, cams, 16)
    assert 200_000 < ref["keys"].shape[0] <= LIMIT
    k, v = _noalloc(ref["keys"], ref["vals"], bits)
    assert _equal(k, v, ref["sorted_keys"], ref["sorted_vals"])
    assert torch.equal(k, k_ref) and torch.equal(v, v_ref)
    # second call right after: a smaller case with another tile size; nothing of the first
    # call's scratch contents may leak into it
    items2 = synth.random_projected_items(32, cams[1:], 4_000, radius_max=20)
    ref2, k_ref2, v_ref2, bits2 = _regular_sort(items2, cams[1:], 8)
    assert ref2["keys"].shape[0] < ref["keys"].shape[0]
    k2, v2 = _noalloc(ref2["keys"], ref2["vals"], bits2)
    assert _equal(k2, v2, ref2["sorted_keys"], ref2["sorted_vals"])
    assert torch.equal(k2, k_ref2) and torch.equal(v2, v_ref2)


@pytest.mark.parametrize("key_bits,n", [(40, 300_000), (8, 70_001), (64, LIMIT), (17, 1), (33, 5_000)])
def test_noalloc_sort_odd_passes_and_full_64_bit_keys(key_bits, n):
    """Stable sort by the low key_bits bits against NumPy's stable argsort: 5 and 1 passes
    (odd: the first pass writes the caller's output, the scratch holds the intermediate), all
    8 passes on random 64-bit keys drawn from a small pool (many duplicates), a single pair,
    and a ragged count."""
    rng = np.random.default_rng(key_bits * 1000 + n)
    pool = rng.integers(0, np.iinfo(np.uint64).max, size=max(2, n // 50), dtype=np.uint64, endpoint=True)
    keys = pool[rng.integers(0, pool.shape[0], n)]
    vals = rng.permutation(n).astype(np.uint32)
    mask = np.uint64((1 << key_bits) - 1) if key_bits < 64 else np.uint64(np.iinfo(np.uint64).max)
    order = np.argsort(keys & mask, kind="stable")
    k, v = _noalloc(keys, vals, key_bits)
    assert _equal(k, v, keys[order], vals[order])


def test_noalloc_sort_rejects_oversize_and_overlap():
    lib = N.lib()
    buf = torch.zeros(64, dtype=torch.int64, device="cuda")
    base = buf.data_ptr()

    def P(off):
        return C.c_void_p(base + off)
    # 8 pairs: keys 64 B, values 32 B.  Inputs at [0, 64) and [64, 96).
    assert lib.gs_sort_pairs_noalloc(P(0), P(64), LIMIT + 1, 40, P(128), P(192), None) == 1
    assert b"1048576" in lib.gs_last_error()
    assert lib.gs_sort_pairs_noalloc(P(0), P(64), 8, 0, P(128), P(192), None) == 1         # key_bits
    assert lib.gs_sort_pairs_noalloc(P(0), P(64), 8, 40, P(0), P(192), None) == 1          # keys_out == keys_in
    assert lib.gs_sort_pairs_noalloc(P(0), P(64), 8, 40, P(8), P(192), None) == 1          # keys_out inside keys_in
    assert lib.gs_sort_pairs_noalloc(P(0), P(64), 8, 40, P(128), P(40), None) == 1         # vals_out over keys_in
    assert lib.gs_sort_pairs_noalloc(P(0), P(64), 8, 40, P(32), P(192), None) == 1         # keys_out over vals_in
    assert lib.gs_sort_pairs_noalloc(P(0), P(64), 8, 40, P(128), P(160), None) == 1        # outputs overlap
    assert b"overlap" in lib.gs_last_error()
    assert lib.gs_sort_pairs_noalloc(P(0), P(64), 0, 40, P(0), P(0), None) == 0            # n = 0: nothing to do
    # adjacent but disjoint ranges are accepted (and sort)
    assert lib.gs_sort_pairs_noalloc(P(0), P(64), 8, 40, P(96), P(160), None) == 0
    torch.cuda.synchronize()
