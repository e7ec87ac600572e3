"""Face displacement (Eq. svdisp, one-step plane shift) in the GPU forward
against the FP64 oracle, and the calls that refuse a displaced scene."""
import numpy as np
import pytest

import oracle
from paper_2604_24994_gb300 import inputs
from tests.gpu_util import assert_close_image
from tests.oracle_util import cluster_scene, f32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2604_24994_gb300 import build
    build.build()


def gpu_render(sc, cams, disp):
    import torch
    from paper_2604_24994_gb300 import DeviceScene, Renderer
    ds = DeviceScene.from_numpy(sc, "cuda", disp=disp)
    r = Renderer(ds.n, ds.k, cams)
    rgb, T, last = r.forward(ds)
    torch.cuda.synchronize()
    return rgb.cpu().numpy().astype(np.float64), T.cpu().numpy().astype(np.float64), last.cpu().numpy()


def random_disp(sc, scale, seed):
    rng = np.random.default_rng(seed)
    return (rng.uniform(-scale, scale, (sc.n, 4)) * sc.R[:, None]).astype(np.float32)


def test_displaced_forward_tiny(tiny):
    sc, cam = tiny
    disp = random_disp(sc, 0.3, 1)
    rgb, T, last = gpu_render(sc, [cam], disp)
    rgb_o, T_o = oracle.Oracle(sc, disp=disp).render(cam)
    assert_close_image(rgb, T, rgb_o, T_o, "displaced tiny")
    # the displacement changes the image
    rgb0, T0 = oracle.Oracle(sc).render(cam)
    assert np.abs(T_o - T0).max() > 1e-2


def test_displaced_forward_cluster_inside_and_fisheye():
    rng = np.random.default_rng(8)
    sc = f32(cluster_scene(rng, n=50, spread=0.3, r=(0.08, 0.2), tex_std=0.15))
    disp = random_disp(sc, 0.4, 2)
    cams = [inputs.look_at((1.2, 0.4, 0.3), 80, 64),
            inputs.look_at((0.03, 0.02, 0.01), 41, 37, target=(1.0, 0.2, 0.1)),
            inputs.fisheye_look_at((0.9, -0.6, 0.2), 60, 60, fov_deg=150.0)]
    rgb, T, last = gpu_render(sc, cams, disp)
    orc = oracle.Oracle(sc, disp=disp)
    o = 0
    for cam in cams:
        n = cam.n_pixels
        rgb_o, T_o = orc.render(cam)
        assert_close_image(rgb[o:o + n], T[o:o + n], rgb_o, T_o, f"displaced {cam.width}x{cam.height}")
        o += n


def test_zero_displacement_matches_the_plain_forward(tiny):
    sc, cam = tiny
    rgb0, T0, last0 = gpu_render(sc, [cam], None)
    rgb1, T1, last1 = gpu_render(sc, [cam], np.zeros((sc.n, 4), np.float32))
    assert np.abs(rgb0 - rgb1).max() < 1e-6 and np.abs(T0 - T1).max() < 1e-6


def test_displaced_scene_refuses_backward_and_contributions(tiny):
    import torch
    from paper_2604_24994_gb300 import DeviceScene, Renderer, _lib
    sc, cam = tiny
    ds = DeviceScene.from_numpy(sc, "cuda", disp=random_disp(sc, 0.2, 3))
    r = Renderer(ds.n, ds.k, [cam])
    rgb, T, last = r.forward(ds)
    g = torch.zeros_like(rgb)
    with pytest.raises(_lib.PFError) as e:
        r.backward(ds, g, None, T, last)
    assert e.value.status == _lib.PF_ERR_INVALID_ARG
    with pytest.raises(_lib.PFError):
        r.render_fwd(ds, contrib=(torch.zeros(ds.n, device="cuda"), torch.zeros(ds.n, device="cuda")))
