"""GPU forward parity: the CUDA path through the C ABI against the FP64 oracle
(1e-4 max abs per RGB channel, 1e-5 in T) and against the CPU binning
(bit-exact rectangles, keys and per-tile lists)."""
import numpy as np
import pytest

import oracle
from paper_2604_24994_gb300 import inputs
from tests.gpu_util import assert_close_image, gpu_forward, pixel_index, sample_pixels
from tests.oracle_util import cluster_scene, f32, make_scene

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2604_24994_gb300 import build
    build.build()


def test_binning_bit_exact_tiny(tiny):
    sc, cam = tiny
    (rgb, T, last), r, ds = gpu_forward(sc, [cam], stats=True)
    ts, cells, keys, rects = r.read_bins()
    orc = oracle.Oracle(sc)
    rect_o, key_o = orc.bin(cam)
    assert np.array_equal(keys[:sc.n], key_o)
    ro = rect_o.copy()
    empty = (ro[:, 0] > ro[:, 2]) | (ro[:, 1] > ro[:, 3])
    rg = rects[:sc.n].astype(np.int64)
    gempty = (rg[:, 0] > rg[:, 2]) | (rg[:, 1] > rg[:, 3])
    assert np.array_equal(empty, gempty)
    assert np.array_equal(rg[~empty], ro[~empty])
    st_o, cells_o = oracle.tile_lists(rect_o, key_o, cam.tiles_x, cam.tiles_y)
    assert np.array_equal(ts.astype(np.int64), st_o)
    assert np.array_equal(cells[:st_o[-1]].astype(np.int64), cells_o)
    assert r.n_instances == st_o[-1] > 0


@pytest.mark.parametrize("dist,fov,seed", [(3.0, 90.0, 11), (60.0, 4.0, 12)])
def test_binning_bit_exact_float_box_at_tile_borders(dist, fov, seed):
    """The tile boxes of spheres whose box edges sit within 2e-3 px of tile
    borders (the float box of the tile rule, Z > 2R), plus spheres near and
    across the camera plane (the FP64 box and the frustum test): rectangles
    and keys bit for bit against the CPU binning (the per-tile lists follow
    from them; the other binning tests compare those)."""
    import torch
    from paper_2604_24994_gb300 import DeviceScene, Renderer
    from tests.oracle_util import border_box_scene
    sc, cam = border_box_scene(dist, fov, seed, 60_000)
    rng = np.random.default_rng(seed + 100)
    # 4,000 more: camera depth between -R and 2R (near / across the camera plane)
    m = 4000
    Mr = np.asarray(cam.rot, np.float64)
    o = np.asarray(cam.origin, np.float64)
    R2 = dist * rng.uniform(0.002, 0.05, m)
    Z2 = R2 * rng.uniform(-1.0, 2.0, m)
    xy2 = rng.normal(0, 1, (m, 2)) * dist * 0.05
    pos2 = (o + np.stack([xy2[:, 0], xy2[:, 1], Z2], 1) @ Mr).astype(np.float32).astype(np.float64)
    R2 = R2.astype(np.float32).astype(np.float64)
    sc = make_scene(np.concatenate([sc.pos, pos2]), np.concatenate([sc.w, R2 * R2]), np.concatenate([sc.R, R2]))
    for k in sc.PARAMS:    # float32 parameters, no neighbour lists (only the bins are compared)
        setattr(sc, k, np.ascontiguousarray(np.asarray(getattr(sc, k)), np.float32))
    ds = DeviceScene.from_numpy(sc, "cuda")
    r = Renderer(ds.n, ds.k, [cam])
    r.bin(ds)
    torch.cuda.synchronize()
    ts, cells, keys, rects = r.read_bins()
    orc = oracle.Oracle(sc)
    rect_o, key_o = orc.bin(cam)
    assert np.array_equal(keys[:sc.n], key_o)
    empty = (rect_o[:, 0] > rect_o[:, 2]) | (rect_o[:, 1] > rect_o[:, 3])
    rg = rects[:sc.n].astype(np.int64)
    assert np.array_equal(empty, (rg[:, 0] > rg[:, 2]) | (rg[:, 1] > rg[:, 3]))
    assert np.array_equal(rg[~empty], rect_o[~empty])
    assert (~empty[-m:]).sum() > m // 8      # many of the near spheres reach the image


def test_forward_tiny_full_frame(tiny):
    sc, cam = tiny
    rgb, T, last = gpu_forward(sc, [cam])
    rgb_o, T_o = oracle.Oracle(sc).render(cam)
    assert_close_image(rgb, T, rgb_o, T_o, "tiny 128x128")
    assert np.all(T[last == 0] == 1.0)     # no contributing cell: nothing composited
    assert (last > 0).sum() > 1000 and (T < 1).sum() > 1000


def test_forward_ragged_inside_multiview():
    """Ragged image sizes, several views of different size in one plan, and
    cameras inside cells (t >= 0 clip, whole-image rectangles)."""
    rng = np.random.default_rng(5)
    sc = f32(cluster_scene(rng, n=60, spread=0.4, r=(0.08, 0.25), tex_std=0.15))
    cams = [inputs.look_at((1.4, 0.3, 0.2), 100, 75),
            inputs.look_at((0.05, 0.02, 0.0), 37, 29, target=(1.0, 0.5, 0.1)),  # inside the cluster
            inputs.look_at((-0.9, -0.9, 0.6), 16, 17)]
    rgb, T, last = gpu_forward(sc, cams)
    orc = oracle.Oracle(sc)
    for v, cam in enumerate(cams):
        rgb_o, T_o = orc.render(cam)
        base = sum(c.width * c.height for c in cams[:v])
        n = cam.width * cam.height
        assert_close_image(rgb[base:base + n], T[base:base + n], rgb_o, T_o, f"view {v}")


def test_forward_dense_clipping_cluster():
    rng = np.random.default_rng(8)
    sc = cluster_scene(rng, n=40, spread=0.15, r=(0.06, 0.12), tex_std=0.2)
    sc.sigma = sc.sigma * 20.0  # near-opaque: early termination paths
    sc = f32(sc)
    cam = inputs.look_at((0.7, 0.2, 0.1), 64, 48, fov_y_deg=40)
    rgb, T, last = gpu_forward(sc, [cam])
    rgb_o, T_o = oracle.Oracle(sc).render(cam)
    assert_close_image(rgb, T, rgb_o, T_o, "cluster")


def test_spurious_neighbours_do_not_change_the_image(tiny):
    """Sec. 3.2 / Fig. cech_equivalence: extra listed neighbours whose planes
    miss the cell leave the render bit-identical."""
    sc, cam = tiny
    rgb0, T0, _ = gpu_forward(sc, [cam])
    rng = np.random.default_rng(1)
    extra = rng.integers(0, sc.n, (sc.n, 16)).astype(np.int32)
    sc2 = sc.copy()
    sc2.nbr = np.concatenate([sc.nbr, extra], 1)
    rgb1, T1, _ = gpu_forward(sc2, [cam])
    assert np.array_equal(rgb0, rgb1) and np.array_equal(T0, T1)


def test_empty_and_invisible_scenes():
    cam = inputs.look_at((3.0, 0, 0), 40, 24)
    sc = f32(make_scene(np.zeros((0, 3)), np.zeros(0), np.zeros(0)))
    rgb, T, last = gpu_forward(sc, [cam])
    assert np.all(rgb == 0) and np.all(T == 1) and np.all(last == 0)
    # everything behind the camera
    sc = f32(make_scene([[5.0, 0, 0], [4.0, 0.1, 0]], [0.01, 0.01], [0.2, 0.2]))
    rgb, T, last = gpu_forward(sc, [cam])
    assert np.all(rgb == 0) and np.all(T == 1)


def test_capacity_overflow_replans(tiny):
    sc, cam = tiny
    (rgb, T, last), r, _ = gpu_forward(sc, [cam], capacity=64, stats=True)
    assert r.plan.capacity >= r.n_instances > 64
    rgb_o, T_o = oracle.Oracle(sc).render(cam)
    assert_close_image(rgb, T, rgb_o, T_o, "after replan")


def test_train_workload_sampled_pixels():
    """100k cells, eight 800x800 views on a ring: sampled pixels of every
    view against the oracle (exact prune)."""
    sc = inputs.train_scene()
    cams = inputs.train_cameras()
    rgb, T, last = gpu_forward(sc, cams)
    orc = oracle.Oracle(sc)
    for v in (0, 3, 6):
        pix = sample_pixels(cams[v], 150, seed=v)
        orc.prune_for(cams[v], pix)
        rgb_o, T_o = orc.render(cams[v], pix)
        idx = pixel_index(cams, v, pix)
        assert_close_image(rgb[idx], T[idx], rgb_o, T_o, f"train view {v}")
