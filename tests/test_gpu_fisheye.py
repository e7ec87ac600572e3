"""Equidistant fisheye views (the paper's non-pinhole rasterization,
appendix D) through the same kernels: forward and backward parity with the
FP64 oracle on the same rays, pixels without a ray, and binning that covers
every (tile, cell) pair whose bounding sphere some pixel ray of the tile
meets."""
import numpy as np
import pytest

import oracle
from paper_2604_24994_gb300 import inputs
from tests.gpu_util import assert_close_image, gpu_forward
from tests.oracle_util import cluster_scene, f32
from tests.test_gpu_backward import check_grads, gpu_grads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2604_24994_gb300 import build
    build.build()


def test_fisheye_forward_tiny(tiny):
    sc, _ = tiny
    cams = [inputs.fisheye_look_at((2.2, 0.4, 0.3), 128, 112, fov_deg=120.0),
            inputs.fisheye_look_at((0.1, -0.05, 0.02), 90, 77, fov_deg=200.0, target=(1.0, 0.3, 0.0))]
    rgb, T, last = gpu_forward(sc, cams)
    orc = oracle.Oracle(sc)
    o = 0
    for cam in cams:
        rgb_o, T_o = orc.render(cam)
        n = cam.n_pixels
        assert_close_image(rgb[o:o + n], T[o:o + n], rgb_o, T_o, f"fisheye {cam.width}x{cam.height}")
        assert (last[o:o + n] > 0).sum() > n // 4
        o += n


def test_fisheye_pixels_without_a_ray():
    # 330 degrees across the inscribed circle: the image corners lie beyond
    # theta = pi and must stay empty; the camera sits inside the cluster
    rng = np.random.default_rng(3)
    sc = f32(cluster_scene(rng, n=60, spread=0.5, r=(0.08, 0.2), tex_std=0.15))
    cam = inputs.fisheye_look_at((0.05, 0.0, 0.02), 72, 40, fov_deg=330.0, target=(1.0, 0.0, 0.0))
    rgb, T, last = gpu_forward(sc, [cam])
    rgb_o, T_o = oracle.Oracle(sc).render(cam)
    assert_close_image(rgb, T, rgb_o, T_o, "fisheye 330")
    uu, vv = np.meshgrid(np.arange(cam.width) + 0.5, np.arange(cam.height) + 0.5)
    th = np.hypot((uu - cam.cx) / cam.fx, (vv - cam.cy) / cam.fy).reshape(-1)
    none = th > np.pi
    assert none.sum() > 100
    assert np.all(T[none] == 1.0) and np.all(rgb[none] == 0.0) and np.all(last[none] == 0)
    assert (T[~none] < 1.0).mean() > 0.5


def test_fisheye_backward_cluster():
    rng = np.random.default_rng(12)
    sc = f32(cluster_scene(rng, n=40, spread=0.15, r=(0.06, 0.12), tex_std=0.2))
    cams = [inputs.fisheye_look_at((0.6, 0.2, 0.1), 48, 40, fov_deg=100.0),
            inputs.fisheye_look_at((0.02, 0.01, 0.0), 33, 29, fov_deg=250.0, target=(1.0, 0.2, 0.1))]
    npx = sum(c.n_pixels for c in cams)
    gC = rng.normal(size=(npx, 3))
    gT = rng.normal(size=npx)
    G = gpu_grads(sc, cams, gC, gT)
    orc = oracle.Oracle(sc)
    Go = None
    o = 0
    for cam in cams:
        g = orc.render_grad(cam, gC[o:o + cam.n_pixels], gT[o:o + cam.n_pixels])
        Go = g if Go is None else {k: Go[k] + g[k] for k in g}
        o += cam.n_pixels
    check_grads(G, Go)


def test_fisheye_binning_covers_every_hit(tiny):
    """Several correct binnings exist (the rectangle is conservative); what is
    unique is the set of (tile, cell) pairs some ray of the tile meets: every
    one must be listed, in painter order, and the lists stay tight."""
    sc, _ = tiny
    cam = inputs.fisheye_look_at((1.6, -0.9, 0.5), 96, 80, fov_deg=170.0)
    (rgb, T, last), r, ds = gpu_forward(sc, [cam], stats=True)
    ts, cells, keys, rects = r.read_bins()
    orc = oracle.Oracle(sc)
    _, key_o = orc.bin(cam)
    assert np.array_equal(keys[:sc.n], key_o)      # painter keys do not depend on the model
    need = 0
    for ty in range(cam.tiles_y):
        for tx in range(cam.tiles_x):
            t = ty * cam.tiles_x + tx
            lst = cells[ts[t]:ts[t + 1]].astype(np.int64)
            k = key_o[lst]
            assert np.all(k[1:] >= k[:-1])
            us = np.arange(tx * 16, min(tx * 16 + 16, cam.width))
            vs = np.arange(ty * 16, min(ty * 16 + 16, cam.height))
            pix = np.stack(np.meshgrid(us, vs), -1).reshape(-1, 2).astype(np.int32)
            hit = np.nonzero(orc.hit_cells(cam, pix))[0]
            need += len(hit)
            missing = np.setdiff1d(hit, lst)
            assert len(missing) == 0, f"tile {t}: {missing[:5]}"
    assert r.n_instances <= 3 * need
