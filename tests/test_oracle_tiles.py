"""Pins for the oracle's tile-list renderer (the full-frame FP64 CPU
renderer over per-tile lists and K-neighbour candidate lists, Sec. 3.4).

It is checked against the brute-force oracle render: with the neighbour
lists of the input generator (each cell's bound radius clipped so that no
site left out of its list has a plane inside its ball) and the tile lists
of the CPU binning in painter order, every pixel must come out the same."""
import numpy as np

import oracle


def lists_for(orc, cam):
    rect, key = orc.bin(cam)
    ntx = (cam.width + 15) // 16
    nty = (cam.height + 15) // 16
    return oracle.tile_lists(rect, key, ntx, nty)


def brute(sc, cam):
    orc = oracle.Oracle(sc)
    orc.prune_for(cam)
    return orc.render(cam, return_nseg=True)


def test_tile_list_render_equals_brute_force(tiny):
    sc, cam = tiny
    rgb0, T0, n0 = brute(sc, cam)
    orc = oracle.Oracle(sc)
    start, cells = lists_for(orc, cam)
    orc.set_neighbour_lists(sc.nbr)
    rgb, T, n = orc.render_tiles(cam, start, cells, return_nseg=True)
    assert (n0 > 0).mean() > 0.5
    np.testing.assert_allclose(rgb, rgb0, rtol=0, atol=1e-13)
    np.testing.assert_allclose(T, T0, rtol=0, atol=1e-13)
    assert np.array_equal(n, n0)
    # the order matters: the same lists composited back to front differ
    rev = np.concatenate([cells[start[t]:start[t + 1]][::-1] for t in range(len(start) - 1)])
    rgb_r, _ = orc.render_tiles(cam, start, rev)
    assert np.abs(rgb_r - rgb0).max() > 1e-3


def test_tile_list_render_of_a_dense_scene_and_its_stop(tiny):
    """sigma x 50 (most rays end nearly opaque): equal to brute force with
    no stop; with a stop at T < t the colour differs by at most t times the
    brightest colour, and a stopped ray's T is below t."""
    from paper_2604_24994_gb300 import inputs
    sc = inputs.tiny_scene(seed=4)
    sc.sigma = sc.sigma * 50
    cam = inputs.look_at((2.5, 0.8, 0.3), 80, 72)
    rgb0, T0, _ = brute(sc, cam)
    orc = oracle.Oracle(sc)
    start, cells = lists_for(orc, cam)
    orc.set_neighbour_lists(sc.nbr)
    rgb, T = orc.render_tiles(cam, start, cells)
    np.testing.assert_allclose(rgb, rgb0, rtol=0, atol=1e-13)
    assert (T0 < 1e-3).mean() > 0.2
    t = 1e-3
    rgb_s, T_s = orc.render_tiles(cam, start, cells, t_stop=t)
    cmax = 2.0    # rgb + the texture's soft-Voronoi sum stays below this here
    assert np.abs(rgb_s - rgb0).max() <= t * cmax
    stopped = T_s != T0
    assert stopped.any() and np.all(T_s[stopped] < t)


def test_tile_subset_writes_only_its_pixels(tiny):
    sc, cam = tiny
    orc = oracle.Oracle(sc)
    start, cells = lists_for(orc, cam)
    orc.set_neighbour_lists(sc.nbr)
    full, Tf = orc.render_tiles(cam, start, cells)
    sel = np.array([0, 5, 17, 63], np.int32)
    part, Tp = orc.render_tiles(cam, start, cells, tiles=sel)
    ntx = (cam.width + 15) // 16
    u = np.arange(cam.width * cam.height) % cam.width
    v = np.arange(cam.width * cam.height) // cam.width
    inside = np.isin((v // 16) * ntx + u // 16, sel)
    assert np.array_equal(part[inside], full[inside]) and np.array_equal(Tp[inside], Tf[inside])
    assert np.isnan(Tp[~inside]).all()
