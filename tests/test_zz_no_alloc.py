"""pf_render_fwd_static: the forward render for callers that cannot allocate
device memory (its scratch is a static __device__ array inside the library).

Callers without an allocator of their own (a host that has given the whole
device budget to another allocator, a real-time loop that must not allocate)
use this entry point.  The test calls it through the C ABI twice in a row, on
two different scenes and cameras, and checks each result against the
workspace-based path (pf_prepare, pf_project, pf_bin_sort, pf_render_fwd)
within the parity tolerances of the other GPU tests.  The second call shows
that what the first call left in the shared array does not leak into the
next result; around it, the device's free memory and the caching allocator's
allocation count must not change.  A scene with displaced faces and learned
detail sites goes through the same comparison.  This file is collected last
on purpose.
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


def outputs(cam):
    import torch
    n = cam.width * cam.height
    return (torch.full((n, 3), float("nan"), device="cuda"), torch.full((n,), float("nan"), device="cuda"),
            torch.full((n,), -1, dtype=torch.int32, device="cuda"))


def static_call(lib, ds, cam, out, stream=None):
    import torch
    from paper_2604_24994_gb300 import _lib
    rgb, T, last = out
    c = _lib.camera_struct(cam)
    st = stream if stream is not None else torch.cuda.current_stream()
    return lib.pf_render_fwd_static(C.byref(ds.struct()), C.byref(c), rgb.data_ptr(), T.data_ptr(),
                                    last.data_ptr(), st.cuda_stream)


def static_render(lib, ds, cam):
    import torch
    out = outputs(cam)
    st = static_call(lib, ds, cam, out)
    torch.cuda.synchronize()
    return (st,) + tuple(x.cpu().numpy() for x in out)


def workspace_render(ds, cam):
    import torch
    from paper_2604_24994_gb300 import Renderer
    r = Renderer(ds.n, ds.k, [cam])
    rgb, T, last = r.forward(ds)
    torch.cuda.synchronize()
    return rgb.cpu().numpy(), T.cpu().numpy(), last.cpu().numpy()


def check_same(lib, ds, cam, got):
    st, rgb, T, last = got
    assert st == 0, lib.pf_last_error_message()
    rgb0, T0, last0 = workspace_render(ds, cam)
    assert np.abs(rgb - rgb0).max() < RGB_TOL
    assert np.abs(T - T0).max() < T_TOL
    assert np.array_equal(last, last0)
    assert (last > 0).any()


def test_static_entry_matches_workspace_path_twice_without_allocating(lib):
    import torch
    from paper_2604_24994_gb300 import DeviceScene
    a = inputs.tiny_scene()
    cam_a = inputs.tiny_camera()
    b = f32(cluster_scene(np.random.default_rng(3), n=32, spread=0.25, r=(0.05, 0.15), tex_std=0.2))
    cam_b = inputs.look_at((1.1, -0.4, 0.3), 97, 61)
    ds_a = DeviceScene.from_numpy(a, "cuda")
    ds_b = DeviceScene.from_numpy(b, "cuda")
    check_same(lib, ds_a, cam_a, static_render(lib, ds_a, cam_a))
    # the second call, with its outputs allocated first: nothing may be
    # allocated on the device while it runs
    out = outputs(cam_b)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    n_alloc0 = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
    st = static_call(lib, ds_b, cam_b, out)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    n_alloc1 = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
    assert free1 == free0, (free0, free1)
    assert n_alloc1 == n_alloc0
    check_same(lib, ds_b, cam_b, (st,) + tuple(x.cpu().numpy() for x in out))


def test_static_entry_extended_face_model(lib):
    """Displaced faces and learned detail sites (Eq. svdisp): the same
    result as the workspace path."""
    from paper_2604_24994_gb300 import DeviceScene
    rng = np.random.default_rng(11)
    sc = f32(cluster_scene(rng, n=30, spread=0.3, r=(0.06, 0.15), tex_std=0.2))   # all-pairs lists: K = 29
    disp = (rng.uniform(-0.2, 0.2, (sc.n, 4)) * sc.R[:, None]).astype(np.float32)
    sites = rng.uniform(-0.5, 0.5, (sc.n, 4, 2)).astype(np.float32)
    ds = DeviceScene.from_numpy(sc, "cuda", disp=disp, sites=sites)
    cam = inputs.look_at((1.2, 0.5, -0.3), 80, 70)
    check_same(lib, ds, cam, static_render(lib, ds, cam))


def test_static_entry_refuses_a_capturing_stream(lib):
    """The call synchronises its stream once, so it refuses to run while that
    stream is being captured into a graph, and enqueues nothing."""
    import torch
    from paper_2604_24994_gb300 import DeviceScene, _lib
    sc = inputs.tiny_scene()
    cam = inputs.tiny_camera()
    ds = DeviceScene.from_numpy(sc, "cuda")
    out = outputs(cam)
    x = torch.zeros(16, device="cuda")
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        g.capture_begin()
        x.add_(1.0)
        st = static_call(lib, ds, cam, out, stream=s)
        g.capture_end()
    assert st == _lib.PF_ERR_INVALID_ARG
    assert b"captured" in lib.pf_last_error_message()
    torch.cuda.synchronize()
    assert torch.isnan(out[1]).all()   # nothing was enqueued


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
