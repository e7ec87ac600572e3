"""Bit-exact binning where the tile lists are long: every per-tile sort path
of pf_bin_sort (lists of at most 2048 entries sorted in 24 KB of shared
memory, 2049-16384 in 192 KB by the persistent kernel, longer lists in
global memory) against the CPU binning (oracle.bin + oracle.tile_lists),
plus the render of those tiles against the FP64 oracle.

The scene puts, for every pixel of two chosen tiles, a column of cells
along the pixel's ray.  Each sphere projects to about 0.3 px around its
pixel centre, so each cell lands in exactly one tile, and one tile lists
20,480 cells, the other 6,144.  Weights are tied to the bound radii
(w = R^2) and the balls are disjoint, so no radical plane cuts any ball
(Sec. 3.2: with tied weights a plane cuts a ball only where the balls
overlap) and empty neighbour lists are complete: the oracle, which clips
against every site, renders the same cells."""
import numpy as np
import pytest

import oracle
from paper_2604_24994_gb300 import inputs
from tests.gpu_util import assert_close_image, pixel_index
from tests.oracle_util import f32, make_scene, random_dirs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2604_24994_gb300 import build
    build.build()


def column_scene(cam, tiles, per_column, seed=0):
    rng = np.random.default_rng(seed)
    ray = oracle.Oracle(make_scene(np.zeros((1, 3)), [0.0], [0.0])).ray
    pos, R = [], []
    for (tx, ty), m in zip(tiles, per_column):
        for v in range(ty * 16, ty * 16 + 16):
            for u in range(tx * 16, tx * 16 + 16):
                o, d = ray(cam, u, v)
                t = 2.0 * (1.0 + rng.uniform(0.0, 0.05))
                for _ in range(m):
                    r = 0.3 * t / cam.fy            # about 0.3 px at this distance
                    pos.append(o + t * d)
                    R.append(r)
                    t += 2.2 * r                     # the next ball starts past this one
    pos = np.array(pos)
    R = np.array(R)
    n = len(R)
    sigma = np.exp(rng.normal(0.0, 1.0, n))
    rgb = rng.uniform(0, 1, (n, 3))
    nrm = random_dirs(rng, n)
    off = rng.uniform(-1, 1, n) * R
    tex = rng.normal(0, 0.1, (n, 12))
    sc = make_scene(pos, R * R, R, sigma, rgb, nrm, off, tex)
    s = sc.copy()
    for k in s.PARAMS:
        setattr(s, k, np.ascontiguousarray(np.asarray(getattr(s, k)), np.float32))
    # tied weights (from the float32 radii) and no neighbour lists
    s.w = (s.R.astype(np.float64) ** 2).astype(np.float32)
    s.nbr = np.zeros((n, 0), np.int32)
    return s


def compare_bins(r, sc, cam):
    ts, cells, keys, rects = r.read_bins()
    orc = oracle.Oracle(sc)
    rect_o, key_o = orc.bin(cam)
    assert np.array_equal(keys[:sc.n], key_o)
    empty_o = (rect_o[:, 0] > rect_o[:, 2]) | (rect_o[:, 1] > rect_o[:, 3])
    rg = rects[:sc.n].astype(np.int64)
    empty_g = (rg[:, 0] > rg[:, 2]) | (rg[:, 1] > rg[:, 3])
    assert np.array_equal(empty_o, empty_g)
    assert np.array_equal(rg[~empty_o], rect_o[~empty_o])
    st_o, cells_o = oracle.tile_lists(rect_o, key_o, cam.tiles_x, cam.tiles_y)
    assert np.array_equal(ts.astype(np.int64), st_o)
    assert np.array_equal(cells[:st_o[-1]].astype(np.int64), cells_o)
    return np.diff(st_o)


def test_long_tile_lists_bit_exact_and_rendered():
    import torch
    from paper_2604_24994_gb300 import DeviceScene, Renderer
    cam = inputs.look_at((3.0, 0.0, 0.0), 640, 360)
    tiles = [(19, 10), (23, 6)]
    sc = column_scene(cam, tiles, [80, 24])
    ds = DeviceScene.from_numpy(sc, "cuda")
    r = Renderer(ds.n, ds.k, [cam])
    rgb, T, last = r.forward(ds)
    torch.cuda.synchronize()
    lens = compare_bins(r, sc, cam)
    assert lens.max() == 256 * 80 > 16384            # the global-memory sort
    assert ((lens > 2048) & (lens <= 16384)).sum() == 1   # the 192 KB shared-memory sort
    # the rendered tiles against the oracle (every pixel of both tiles, and some empty ones)
    pix = np.array([(u, v) for tx, ty in tiles for v in range(ty * 16, ty * 16 + 16)
                    for u in range(tx * 16, tx * 16 + 16)] + [(0, 0), (639, 359), (300, 10)], np.int32)
    orc = oracle.Oracle(sc)
    orc.prune_for(cam, pix)
    rgb_o, T_o, nseg = orc.render(cam, pix, return_nseg=True)
    idx = pixel_index([cam], 0, pix)
    rgb = rgb.cpu().numpy().astype(np.float64)
    T = T.cpu().numpy().astype(np.float64)
    assert_close_image(rgb[idx], T[idx], rgb_o, T_o, "long lists")
    # every ray crosses its whole column; the dense halves keep about three quarters of the chords
    assert nseg[:256].mean() > 40 and nseg[256:512].mean() > 12


def test_long_tile_lists_across_views_and_capacity_growth():
    """The same columns seen by two views of one plan, starting from a
    capacity far too small (the plan grows and re-bins)."""
    import torch
    from paper_2604_24994_gb300 import DeviceScene, Renderer
    cam = inputs.look_at((3.0, 0.0, 0.0), 640, 360)
    sc = column_scene(cam, [(10, 12)], [70], seed=1)
    cam2 = inputs.look_at((3.0, 0.2, -0.1), 320, 200, target=(0.0, 0.2, -0.1))
    ds = DeviceScene.from_numpy(sc, "cuda")
    r = Renderer(ds.n, ds.k, [cam, cam2], capacity=1024)
    r.forward(ds)
    torch.cuda.synchronize()
    ts, cells, keys, rects = r.read_bins()
    orc = oracle.Oracle(sc)
    base = 0
    for v, c in enumerate((cam, cam2)):
        rect_o, key_o = orc.bin(c)
        st_o, cells_o = oracle.tile_lists(rect_o, key_o, c.tiles_x, c.tiles_y)
        nt = c.tiles_x * c.tiles_y
        st_g = ts[base:base + nt + 1].astype(np.int64) - int(ts[base])
        assert np.array_equal(st_g, st_o)
        assert np.array_equal(cells[int(ts[base]):int(ts[base + nt])].astype(np.int64), cells_o)
        assert np.array_equal(keys[v * sc.n:(v + 1) * sc.n], key_o)
        base += nt
    assert np.diff(oracle.tile_lists(*orc.bin(cam), cam.tiles_x, cam.tiles_y)[0]).max() == 256 * 70


def test_equal_keys_in_every_sort_path_bit_exact():
    """Cells duplicated (same site, weight and radius, so the same key) in
    lists that take each radix sort: 488 and 1,944 entries (256 threads,
    32 KB of shared memory; there the bitonic network orders (key, cell)),
    11,674 entries with thousands of equal keys (512 threads, 208 KB: sorted
    again with the cell index's digits first) and 2,570 entries with ten
    (the insertion fix-up).  Equal keys must come out in cell-index order,
    as in the CPU binning, whatever order the atomic bucket fill left them
    in."""
    import torch
    from paper_2604_24994_gb300 import DeviceScene, Renderer
    cam = inputs.look_at((3.0, 0.0, 0.0), 640, 360)
    tiles = [(5, 5), (30, 15), (14, 9), (35, 3)]
    per = [1, 4, 24, 10]
    base = column_scene(cam, tiles, per, seed=2)
    n3 = 256 * (1 + 4 + 24)          # cells of the first three tiles
    rng = np.random.default_rng(5)
    # the first three tiles: every other cell once more, every fifth twice more;
    # the fourth: ten of its cells once more; all appended in a shuffled order
    extra = np.concatenate([np.arange(0, n3, 2), np.arange(0, n3, 5), np.arange(0, n3, 5),
                            n3 + rng.choice(256 * 10, 10, replace=False)])
    extra = extra[rng.permutation(extra.size)]
    src = np.concatenate([np.arange(base.n), extra])
    sc = base.copy()
    for k in sc.PARAMS:
        setattr(sc, k, np.ascontiguousarray(np.asarray(getattr(base, k))[src]))
    sc.nbr = np.zeros((src.size, 0), np.int32)
    ds = DeviceScene.from_numpy(sc, "cuda")
    r = Renderer(ds.n, ds.k, [cam])
    r.forward(ds)
    torch.cuda.synchronize()
    lens = compare_bins(r, sc, cam)
    # each cell lies in one tile: its column's
    tile_of = np.repeat(np.arange(4), [256 * p for p in per])[src]
    want = np.bincount(tile_of)
    assert sorted(lens[lens > 0].tolist()) == sorted(want.tolist())
    assert 256 < want[0] <= 2048 and 256 < want[1] <= 2048 and 2048 < want[2] <= 16384
    assert want[3] == 2570


def test_lists_above_shared_memory_split_bit_exact():
    """Lists longer than the 16,384 entries a CTA sorts in shared memory are
    split by their leading key bits first.  Two such lists: 20,480 distinct
    keys with every third cell duplicated (27,307 entries: equal keys inside
    the shared-memory runs), and 6,144 keys plus one cell repeated 17,000
    times (23,144 entries: a bucket of 17,001 equal keys that no split can
    shorten, ordered by cell index alone).  Bit-exact against the CPU
    binning."""
    import torch
    from paper_2604_24994_gb300 import DeviceScene, Renderer
    cam = inputs.look_at((3.0, 0.0, 0.0), 640, 360)
    tiles = [(19, 10), (23, 6)]
    per = [80, 24]
    base = column_scene(cam, tiles, per, seed=3)
    na = 256 * per[0]
    rng = np.random.default_rng(7)
    extra = np.concatenate([np.arange(0, na, 3), np.full(17000, na + 1000)])
    extra = extra[rng.permutation(extra.size)]
    src = np.concatenate([np.arange(base.n), extra])
    sc = base.copy()
    for k in sc.PARAMS:
        setattr(sc, k, np.ascontiguousarray(np.asarray(getattr(base, k))[src]))
    sc.nbr = np.zeros((src.size, 0), np.int32)
    ds = DeviceScene.from_numpy(sc, "cuda")
    r = Renderer(ds.n, ds.k, [cam])
    r.forward(ds)
    torch.cuda.synchronize()
    lens = compare_bins(r, sc, cam)
    tile_of = np.repeat(np.arange(2), [256 * p for p in per])[src]
    want = np.bincount(tile_of)
    assert sorted(lens[lens > 0].tolist()) == sorted(want.tolist())
    assert want.tolist() == [27307, 23144]
