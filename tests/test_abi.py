"""The C ABI without a GPU: the library builds, loads, exports every function include/gs.h
declares, and rejects invalid arguments on the host (no kernel is launched)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def native():
    from paper_2604_12942_gb300 import build
    build.build()
    from paper_2604_12942_gb300 import _native
    return _native


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(gs_[a-z0-9_]+)\s*\(", src))
    return names


def test_exports_every_declared_symbol(native):
    lib = native.lib()
    decl = _declared()
    assert {"gs_project", "gs_bin_sort", "gs_render_fwd", "gs_render_bwd", "gs_adam_step"} <= decl
    for name in decl:
        assert hasattr(lib, name), name
    assert set(native.exported_names()) <= decl


def test_layout_is_aligned_and_consistent(native):
    import paper_2604_12942_gb300 as gs
    cams = [synth.camera(640, 480, 500.0), synth.camera(1280, 720, 900.0)]
    for tile in (8, 16):
        o = gs.default_opts(tile=tile)
        L = native.WsLayout()
        assert native.lib().gs_workspace_layout(1000, 2, gs.camera_array(cams), C.byref(o), 5000, C.byref(L)) == 0
        offs = [getattr(L, f) for f, _ in native.WsLayout._fields_[:18]]
        assert all(x % 256 == 0 for x in offs)
        assert offs == sorted(offs) and L.total >= offs[-1]
        tiles = sum(((c["width"] + tile - 1) // tile) * ((c["height"] + tile - 1) // tile) for c in cams)
        assert L.total_tiles == tiles and L.total_pixels == 640 * 480 + 1280 * 720
        assert native.lib().gs_workspace_size(1000, 2, gs.camera_array(cams), C.byref(o), 5000) == L.total


@pytest.mark.parametrize("field,value", [("tile", 12), ("chunk", 48), ("alpha_min", 0.0), ("alpha_max", 0.001)])
def test_invalid_opts_rejected(native, field, value):
    import paper_2604_12942_gb300 as gs
    o = gs.default_opts(**{field: value})
    L = native.WsLayout()
    st = native.lib().gs_workspace_layout(10, 1, gs.camera_array([synth.camera(64, 48, 60.0)]), C.byref(o), 100,
                                          C.byref(L))
    assert st == 1
    assert native.lib().gs_last_error()


def test_invalid_views_and_sizes_rejected(native):
    import paper_2604_12942_gb300 as gs
    o = gs.default_opts()
    L = native.WsLayout()
    lib = native.lib()
    cams = gs.camera_array([synth.camera(64, 48, 60.0)] * 33)
    assert lib.gs_workspace_layout(10, 33, cams, C.byref(o), 100, C.byref(L)) == 1
    assert lib.gs_workspace_layout(10, 0, cams, C.byref(o), 100, C.byref(L)) == 1
    bad = gs.camera_array([synth.camera(0, 48, 60.0)])
    assert lib.gs_workspace_layout(10, 1, bad, C.byref(o), 100, C.byref(L)) == 1
    assert lib.gs_workspace_layout(-1, 1, gs.camera_array([synth.camera(64, 48, 60.0)]), C.byref(o), 100,
                                   C.byref(L)) == 1
    assert lib.gs_workspace_size(10, 1, None, C.byref(o), 100) == 0


def test_stage_calls_reject_bad_arguments_without_launching(native):
    import paper_2604_12942_gb300 as gs
    lib = native.lib()
    o = gs.default_opts()
    cams = gs.camera_array([synth.camera(64, 48, 60.0)])
    L = native.WsLayout()
    assert lib.gs_workspace_layout(10, 1, cams, C.byref(o), 100, C.byref(L)) == 0
    g = native.Gaussians(10, 0, None, None, None, None, None)
    # NULL planes, NULL workspace, mismatched n: all rejected on the host
    assert lib.gs_project(C.byref(g), cams, C.byref(o), C.byref(L), None, None) == 1
    g2 = native.Gaussians(11, 0, 256, 256, 256, 256, 256)
    assert lib.gs_project(C.byref(g2), cams, C.byref(o), C.byref(L), C.c_void_p(256), None) == 1
    assert lib.gs_bin_sort(cams, C.byref(o), C.byref(L), None, None) == 1
    # cameras that do not match the layout's image sizes
    other = gs.camera_array([synth.camera(80, 48, 60.0)])
    assert lib.gs_bin_sort(other, C.byref(o), C.byref(L), C.c_void_p(256), None) == 1
    assert lib.gs_render_fwd(cams, C.byref(o), C.byref(L), C.c_void_p(256), None, None, None, None, None, None, None,
                             None, None, None) == 1
    lr = (C.c_float * 6)(*[1e-3] * 6)
    assert lib.gs_adam_step(C.byref(g2), C.byref(g2), C.byref(g2), C.byref(g2), None, None, lr, 0.9, 0.999, 1e-15, 0,
                            None) == 1
    assert lib.gs_adam_step(C.byref(g2), C.byref(g2), C.byref(g2), C.byref(g2), None, None, lr, 1.5, 0.999, 1e-15, 1,
                            None) == 1


def test_nonfinite_camera_rejected_on_the_host(native):
    import paper_2604_12942_gb300 as gs
    o = gs.default_opts()
    L = native.WsLayout()
    cam = synth.camera(64, 48, 60.0)
    for key, idx in (("t", 1), ("R", 4)):
        bad = dict(cam)
        arr = np.array(bad[key], dtype=np.float64).copy()
        arr.flat[idx] = np.nan
        bad[key] = arr
        assert native.lib().gs_workspace_layout(10, 1, gs.camera_array([bad]), C.byref(o), 100, C.byref(L)) == 5
        assert b"not finite" in native.lib().gs_last_error()
