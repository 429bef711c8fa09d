"""The allocation-free pair sort (gs_sort_pairs_noalloc) against the regular binning sort.

Some callers cannot allocate device memory (a no-allocation policy in a real-time loop, a
host callback, a plug-in whose application owns every allocation).  For them the library
offers a sort whose scratch is a fixed array inside the library.  These tests call it
through the C ABI and check, on two calls in a row, that it returns exactly the pairs that
gs_bin_sort produces from the same records (the sort is bit-exact, so the tolerance is
equality).  The file is named so that pytest collects it last.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import oracle
import paper_2604_12942_gb300 as gs
import synth
from paper_2604_12942_gb300 import _native as N

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
    ws.region("touched", torch.int32, V * n).copy_(torch.as_tensor(ref["touched"].astype(np.int32)))
    ws.region("counters", torch.int32, 8).zero_()
    ws.bin_sort()
    c = ws.counters()
    assert c.status == 0 and c.n_pairs == P
    k, v = ws.sorted_pairs(P)
    tiles = ws.layout.total_tiles
    key_bits = 32 + max(1, int(np.ceil(np.log2(max(tiles, 2)))))
    return ref["keys"], ref["vals"], k.clone(), v.clone(), key_bits


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


def test_noalloc_sort_matches_bin_sort_on_two_calls():
    cams = [synth.camera(1280, 720, 900.0), synth.camera(333, 250, 300.0)]
    # first call: a large case (several chunks per block of the sort grid)
    items = synth.random_projected_items(31, cams, 60_000, radius_max=32)
    keys, vals, k_ref, v_ref, bits = _regular_sort(items, cams, 16)
    assert 200_000 < keys.shape[0] <= LIMIT
    k, v = _noalloc(keys, vals, bits)
    assert torch.equal(k, k_ref) and torch.equal(v, v_ref)
    # second call right after: a smaller case with another tile size; nothing of the first
    # call's scratch contents may leak into it
    items2 = synth.random_projected_items(32, cams[1:], 4_000, radius_max=20)
    keys2, vals2, k_ref2, v_ref2, bits2 = _regular_sort(items2, cams[1:], 8)
    assert keys2.shape[0] < keys.shape[0]
    k2, v2 = _noalloc(keys2, vals2, bits2)
    assert torch.equal(k2, k_ref2) and torch.equal(v2, v_ref2)


def test_noalloc_sort_rejects_oversize_and_aliasing():
    lib = N.lib()
    buf = torch.zeros(16, dtype=torch.int64, device="cuda")
    p = C.c_void_p(buf.data_ptr())
    assert lib.gs_sort_pairs_noalloc(p, p, LIMIT + 1, 40, p, p, None) == 1
    assert b"1048576" in lib.gs_last_error()
    assert lib.gs_sort_pairs_noalloc(p, p, 8, 40, p, C.c_void_p(buf.data_ptr() + 64), None) == 1
    assert lib.gs_sort_pairs_noalloc(p, p, 8, 0, C.c_void_p(buf.data_ptr() + 64), C.c_void_p(buf.data_ptr() + 96),
                                     None) == 1
    assert lib.gs_sort_pairs_noalloc(p, p, 0, 40, p, p, None) == 0
