"""pf_render_fwd_static: the forward render for callers that cannot allocate
device memory (its scratch is a static __device__ array inside the library).

The test calls the entry point through the C ABI twice in a row, on two
different scenes and cameras, and checks each result against the
workspace-based path (pf_prepare, pf_project, pf_bin_sort, pf_render_fwd)
within the parity tolerances of the other GPU tests.  The second call
shows that the contents the first call left in the shared array do not
leak into the next result.  This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2604_24994_gb300 import inputs
from tests.gpu_util import RGB_TOL, T_TOL
from tests.oracle_util import cluster_scene, f32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2604_24994_gb300 import _lib, build
    build.build()
    l = _lib.lib()
    l.pf_render_fwd_static.argtypes = [C.POINTER(_lib.Scene), C.POINTER(_lib.Camera), C.c_void_p, C.c_void_p,
                                       C.c_void_p, C.c_void_p]
    l.pf_render_fwd_static.restype = C.c_int
    return l


def static_render(lib, ds, cam):
    import torch
    from paper_2604_24994_gb300 import _lib
    n = cam.width * cam.height
    rgb = torch.full((n, 3), float("nan"), device="cuda")
    T = torch.full((n,), float("nan"), device="cuda")
    last = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    c = _lib.camera_struct(cam)
    st = lib.pf_render_fwd_static(C.byref(ds.struct()), C.byref(c), rgb.data_ptr(), T.data_ptr(),
                                  last.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return st, rgb.cpu().numpy(), T.cpu().numpy(), last.cpu().numpy()


def workspace_render(ds, cam):
    import torch
    from paper_2604_24994_gb300 import Renderer
    r = Renderer(ds.n, ds.k, [cam])
    rgb, T, last = r.forward(ds)
    torch.cuda.synchronize()
    return rgb.cpu().numpy(), T.cpu().numpy(), last.cpu().numpy()


def test_static_entry_matches_workspace_path_twice(lib):
    from paper_2604_24994_gb300 import DeviceScene
    a = inputs.tiny_scene()
    cam_a = inputs.tiny_camera()
    b = f32(cluster_scene(np.random.default_rng(3), n=32, spread=0.25, r=(0.05, 0.15), tex_std=0.2))
    cam_b = inputs.look_at((1.1, -0.4, 0.3), 97, 61)
    for sc, cam in ((a, cam_a), (b, cam_b)):
        ds = DeviceScene.from_numpy(sc, "cuda")
        st, rgb, T, last = static_render(lib, ds, cam)
        assert st == 0, lib.pf_last_error_message()
        rgb0, T0, last0 = workspace_render(ds, cam)
        assert np.abs(rgb - rgb0).max() < RGB_TOL
        assert np.abs(T - T0).max() < T_TOL
        assert np.array_equal(last, last0)
        assert (last > 0).any()


def test_static_entry_rejects_sizes_beyond_its_limits(lib):
    from paper_2604_24994_gb300 import DeviceScene
    sc = inputs.uniform_scene(4097, seed=1, K=4)
    ds = DeviceScene.from_numpy(sc, "cuda")
    st, *_ = static_render(lib, ds, inputs.look_at((3, 0, 0), 64, 64))
    assert st == 1 and b"4097 cells" in lib.pf_last_error_message()
    sc = inputs.uniform_scene(100, seed=1, K=4)
    ds = DeviceScene.from_numpy(sc, "cuda")
    st, *_ = static_render(lib, ds, inputs.look_at((3, 0, 0), 257, 64))
    assert st == 1 and b"256x256" in lib.pf_last_error_message()
