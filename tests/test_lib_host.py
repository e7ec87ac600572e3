"""Host-only checks of the C ABI library: it builds, loads without a GPU,
exports every entry point include/powerfoam.h declares, and its plan calls
validate arguments (no compute call is made here)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2604_24994_gb300 import build as pfbuild
from paper_2604_24994_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(pf_[a-z_0-9]+)\s*\(", src, flags=re.M))
    return names


@pytest.fixture(scope="module")
def lib():
    pfbuild.build()
    from paper_2604_24994_gb300 import _lib
    return _lib.lib()


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_plan_without_hit_records(lib):
    from paper_2604_24994_gb300 import _lib
    cams = [inputs.look_at((3, 0, 0), 100, 75), inputs.look_at((0, 3, 0), 64, 64)]
    arr = _lib.camera_array(cams)
    h = C.c_void_p()
    assert lib.pf_plan_create(1000, 16, arr, 2, 5000, C.byref(h)) == 0
    full, small = C.c_uint64(), C.c_uint64()
    lib.pf_plan_workspace_bytes(h, C.byref(full))
    assert lib.pf_plan_set_record_hits(h, 0) == 0 and lib.pf_plan_set_record_hits(h, 1) == 0
    assert lib.pf_plan_omit_hit_records(h) == 0
    lib.pf_plan_workspace_bytes(h, C.byref(small))
    # 8 warps x (capacity/32 + tiles + 1) batch slots x 32 pixels x 4 B of masks, then per pixel
    # 256 x 2 B of constraint records and a 4 B hit count (each region 256-byte aligned)
    tiles = 7 * 5 + 4 * 4
    px = 100 * 75 + 64 * 64
    rec = 8 * (5000 // 32 + tiles + 1) * 32 * 4 + px * 256 * 2 + px * 4
    assert rec <= full.value - small.value <= rec + 3 * 256
    assert lib.pf_plan_set_record_hits(h, 1) == _lib.PF_ERR_INVALID_ARG
    assert lib.pf_plan_set_record_hits(h, 0) == 0
    lib.pf_plan_destroy(h)


def test_status_strings(lib):
    from paper_2604_24994_gb300 import _lib
    for s in range(7):
        assert lib.pf_status_string(s)
    assert lib.pf_status_string(_lib.PF_ERR_CAPACITY) == b"instance capacity exceeded"


def test_plan_layout_and_validation(lib):
    from paper_2604_24994_gb300 import _lib
    cams = [inputs.look_at((3, 0, 0), 100, 75), inputs.look_at((0, 3, 0), 64, 64)]
    arr = _lib.camera_array(cams)
    h = C.c_void_p()
    assert lib.pf_plan_create(1000, 16, arr, 2, 5000, C.byref(h)) == 0
    b = C.c_uint64()
    px = C.c_uint64()
    assert lib.pf_plan_workspace_bytes(h, C.byref(b)) == 0
    assert lib.pf_plan_pixels(h, C.byref(px)) == 0
    assert px.value == 100 * 75 + 64 * 64
    # 7 x 5 + 4 x 4 tiles; workspace grows with capacity
    assert b.value > 1000 * (128 + 16 * 24)
    h2 = C.c_void_p()
    assert lib.pf_plan_create(1000, 16, arr, 2, 50000, C.byref(h2)) == 0
    b2 = C.c_uint64()
    lib.pf_plan_workspace_bytes(h2, C.byref(b2))
    assert b2.value - b.value >= 45000 * 28 - 5 * 256  # 28 B per instance, 256-byte aligned regions
    # camera resolution cannot change under a plan
    bad = _lib.camera_array([inputs.look_at((3, 0, 0), 101, 75), cams[1]])
    assert lib.pf_plan_set_cameras(h, bad, 2) == _lib.PF_ERR_INVALID_ARG
    assert b"resolution" in lib.pf_last_error_message()
    assert lib.pf_plan_set_cameras(h, _lib.camera_array(cams[::-1][::-1]), 2) == 0
    lib.pf_plan_destroy(h)
    lib.pf_plan_destroy(h2)
    lib.pf_plan_destroy(None)


@pytest.mark.parametrize("mut", ["width0", "fx0", "nan", "k65", "nviews0"])
def test_plan_rejects_bad_arguments(lib, mut):
    from paper_2604_24994_gb300 import _lib
    cam = inputs.look_at((3, 0, 0), 32, 32)
    k, nv = 8, 1
    if mut == "width0":
        cam.width = 0
    elif mut == "fx0":
        cam.fx = 0.0
    elif mut == "nan":
        cam.origin = np.array([np.nan, 0, 0])
    elif mut == "k65":
        k = 65
    elif mut == "nviews0":
        nv = 0
    h = C.c_void_p()
    assert lib.pf_plan_create(10, k, _lib.camera_array([cam]), nv, 100, C.byref(h)) == _lib.PF_ERR_INVALID_ARG


def test_calls_reject_null_workspace(lib):
    from paper_2604_24994_gb300 import _lib
    h = C.c_void_p()
    assert lib.pf_plan_create(10, 4, _lib.camera_array([inputs.look_at((3, 0, 0), 32, 32)]), 1, 100,
                              C.byref(h)) == 0
    s = _lib.Scene()
    s.n_cells, s.k_nbr = 10, 4
    assert lib.pf_prepare(C.byref(s), h, None, None) == _lib.PF_ERR_INVALID_ARG
    assert lib.pf_bin_sort(h, None, None, None) == _lib.PF_ERR_INVALID_ARG
    # scene size must match the plan
    s.n_cells = 11
    assert lib.pf_project(C.byref(s), h, C.c_void_p(256), None) == _lib.PF_ERR_INVALID_ARG
    lib.pf_plan_destroy(h)


def test_product_path_refuses_to_run_without_library(monkeypatch, tmp_path):
    from paper_2604_24994_gb300 import _lib
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(RuntimeError, match="CUDA library missing"):
        _lib.lib()


def test_neighbour_build_validates_arguments(lib):
    """pf_build_neighbours refuses bad sizes, null pointers and a small
    workspace before any device work; the workspace is ~116 bytes per cell."""
    from paper_2604_24994_gb300 import _lib
    assert lib.pf_neighbours_workspace_bytes(-1) == 0
    b = lib.pf_neighbours_workspace_bytes(1_000_000)
    assert 100e6 < b < 140e6
    fake = C.c_void_p(4096)
    args = lambda n, k, nbr=fake, ws_bytes=b: (fake, fake, fake, n, k, nbr, fake, None, None, fake, ws_bytes, None)
    assert lib.pf_build_neighbours(*args(1_000_000, 65)) == _lib.PF_ERR_INVALID_ARG
    assert lib.pf_build_neighbours(*args(-1, 8)) == _lib.PF_ERR_INVALID_ARG
    assert lib.pf_build_neighbours(*args(100, 8, nbr=None)) == _lib.PF_ERR_INVALID_ARG
    assert lib.pf_build_neighbours(*args(1_000_000, 32, ws_bytes=b - 1)) == _lib.PF_ERR_CAPACITY
    assert b"workspace" in lib.pf_last_error_message()


def test_camera_models(lib):
    from paper_2604_24994_gb300 import _lib
    h = C.c_void_p()
    fe = inputs.fisheye_look_at((3, 0, 0), 64, 48, fov_deg=190.0)
    assert lib.pf_plan_create(10, 4, _lib.camera_array([fe]), 1, 100, C.byref(h)) == 0
    lib.pf_plan_destroy(h)
    bad = _lib.camera_array([fe])
    bad[0].model = 2
    assert lib.pf_plan_create(10, 4, bad, 1, 100, C.byref(h)) == _lib.PF_ERR_INVALID_ARG


def test_extended_face_model_checks(lib):
    """Displacement, learned sites, view-dependent colours and the site
    count: misaligned arrays, a stats pass, a site count other than 4 or 8,
    a contribution adjoint without its weights and a backward without the
    matching gradient arrays are refused on the host."""
    from paper_2604_24994_gb300 import _lib
    h = C.c_void_p()
    assert lib.pf_plan_create(10, 4, _lib.camera_array([inputs.look_at((3, 0, 0), 32, 32)]), 1, 100,
                              C.byref(h)) == 0
    fake = 1 << 20                                       # never dereferenced: every call returns first
    s = _lib.Scene()
    for k in ("pos", "w", "R", "sigma", "rgb", "normal", "offset", "tex", "nbr"):
        setattr(s, k, fake)
    s.n_cells, s.k_nbr = 10, 4
    out = C.c_void_p(fake)
    s.disp = fake + 8                                    # not 16-byte aligned
    assert lib.pf_render_fwd(C.byref(s), h, out, out, out, out, None) == _lib.PF_ERR_INVALID_ARG
    assert b"aligned" in lib.pf_last_error_message()
    s.disp = fake
    assert lib.pf_plan_enable_stats(h, 1) == 0
    assert lib.pf_render_fwd(C.byref(s), h, out, out, out, out, None) == _lib.PF_ERR_INVALID_ARG
    assert lib.pf_plan_enable_stats(h, 0) == 0
    s.disp = None
    s.n_sites = 5
    assert lib.pf_render_fwd(C.byref(s), h, out, out, out, out, None) == _lib.PF_ERR_INVALID_ARG
    assert b"n_sites" in lib.pf_last_error_message()
    s.n_sites = 8
    assert lib.pf_plan_enable_stats(h, 1) == 0          # eight sites: no stats pass either
    assert lib.pf_render_fwd(C.byref(s), h, out, out, out, out, None) == _lib.PF_ERR_INVALID_ARG
    assert lib.pf_plan_enable_stats(h, 0) == 0
    s.n_sites = 0
    g = _lib.SceneGrad()
    for k in ("pos", "w", "R", "sigma", "rgb", "normal", "offset", "tex"):
        setattr(g, k, fake)
    assert lib.pf_render_bwd_contrib(C.byref(s), h, out, out, out, out, out, None, None, C.byref(g),
                                     None) == _lib.PF_ERR_INVALID_ARG
    assert b"contribution weights" in lib.pf_last_error_message()
    for k in ("disp", "sites", "sv"):
        s.disp = s.sites = s.sv = None
        setattr(s, k, fake)
        assert lib.pf_render_bwd(C.byref(s), h, out, out, out, out, out, C.byref(g), None) == _lib.PF_ERR_INVALID_ARG
        assert k.encode() in lib.pf_last_error_message()
    lib.pf_plan_destroy(h)
