"""Parity at the benchmark's full sizes, in the benchmark's launch
configuration: sampled outputs the oracle computes one by one.

- capture workload: 1M cells, 1920x1080 (forward): sampled pixels against
  the brute-force oracle, then every pixel of the frame against the
  oracle's FP64 tile-list renderer (pinned to the brute-force oracle on the
  CPU), and the bins bit for bit;
- training workload: 100k cells on a ring of eight views; its gradients
  for an L2 loss against a target rendered from a perturbed copy, at
  64x64, against the oracle's adjoint (1e-3 relative L2 per tensor) and
  against FP64 central differences of the oracle on 64 sampled parameters.
"""
import numpy as np
import pytest

import oracle
from paper_2604_24994_gb300 import inputs
from tests.gpu_util import GRAD_TOL, assert_close_image, pixel_index, rel_l2

pytestmark = pytest.mark.gpu

PARAMS = ("pos", "w", "R", "sigma", "rgb", "normal", "offset", "tex")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2604_24994_gb300 import build
    build.build()


def stratified_pixels(cam, per_axis=16, extra=64, seed=0):
    """One pixel in each cell of a per_axis x per_axis grid plus random ones."""
    rng = np.random.default_rng(seed)
    xs = (np.arange(per_axis) + rng.uniform(0, 1, per_axis)) * cam.width / per_axis
    ys = (np.arange(per_axis) + rng.uniform(0, 1, per_axis)) * cam.height / per_axis
    g = np.stack(np.meshgrid(xs, ys), -1).reshape(-1, 2).astype(np.int32)
    r = np.stack([rng.integers(0, cam.width, extra), rng.integers(0, cam.height, extra)], 1).astype(np.int32)
    return np.concatenate([g, r])


def test_capture_workload_1080p_sampled_pixels():
    import torch
    from paper_2604_24994_gb300 import DeviceScene, Renderer
    sc = inputs.capture_scene(1_000_000, seed=0, K=32)
    cam = inputs.capture_camera()
    ds = DeviceScene.from_numpy(sc, "cuda")
    r = Renderer(ds.n, ds.k, [cam])
    rgb, T, last = r.forward(ds)          # the benchmark's plan and kernels
    torch.cuda.synchronize()
    rgb = rgb.cpu().numpy().astype(np.float64)
    T = T.cpu().numpy().astype(np.float64)
    pix = stratified_pixels(cam, 16, 64)
    orc = oracle.Oracle(sc)
    orc.prune_for(cam, pix)
    rgb_o, T_o, nseg = orc.render(cam, pix, return_nseg=True)
    idx = pixel_index([cam], 0, pix)
    assert_close_image(rgb[idx], T[idx], rgb_o, T_o, "capture 1080p")
    assert nseg.mean() > 20        # the sampled rays really cross many cells
    # the benchmark plan's bins, bit for bit against the CPU binning: every
    # rectangle, key and per-tile list of the 3.2M (cell, tile) instances
    ts, cells, keys, rects = r.read_bins()
    rect_o, key_o = orc.bin(cam)
    assert np.array_equal(keys[:sc.n], key_o)
    empty_o = (rect_o[:, 0] > rect_o[:, 2]) | (rect_o[:, 1] > rect_o[:, 3])
    rg = rects[:sc.n].astype(np.int64)
    assert np.array_equal(empty_o, (rg[:, 0] > rg[:, 2]) | (rg[:, 1] > rg[:, 3]))
    assert np.array_equal(rg[~empty_o], rect_o[~empty_o])
    st_o, cells_o = oracle.tile_lists(rect_o, key_o, cam.tiles_x, cam.tiles_y)
    assert np.array_equal(ts.astype(np.int64), st_o)
    assert np.array_equal(cells[:st_o[-1]].astype(np.int64), cells_o)
    assert st_o[-1] > 3_000_000 and np.diff(st_o).max() > 2048   # the large-list sort ran too
    # every pixel of the frame: the oracle's FP64 renderer over the same tile
    # lists and neighbour lists, stopping where the kernel stops (T < 1e-6)
    orc.clear_candidates()
    orc.set_neighbour_lists(sc.nbr)
    rgb_f, T_f = orc.render_tiles(cam, st_o, cells_o, t_stop=1e-6)
    assert_close_image(rgb, T, rgb_f, T_f, "capture 1080p, full frame")
    np.testing.assert_allclose(rgb_f[idx], rgb_o, rtol=0, atol=1e-5)


@pytest.fixture(scope="module")
def train_setup():
    """Scene, its perturbed copy, 64x64 ring views and the oracle's L2
    upstream gradient 2 (C - C*) shared by the GPU and the oracle."""
    sc = inputs.train_scene()
    tgt = inputs.perturbed_sites(sc, 0.002, seed=1)
    cams = inputs.train_cameras(64, 64)
    orc = oracle.Oracle(sc)
    orc_t = oracle.Oracle(tgt)
    gC, gT, C = [], [], []
    for cam in cams:
        orc.prune_for(cam)
        c, t = orc.render(cam)
        orc_t.prune_for(cam)
        ct, _ = orc_t.render(cam)
        gC.append(2 * (c - ct))
        gT.append(np.zeros(cam.n_pixels))
        C.append(c)
    return sc, tgt, cams, orc, gC, gT


def gpu_grads(sc, cams, gC, gT):
    import torch
    from paper_2604_24994_gb300 import DeviceScene, Renderer
    ds = DeviceScene.from_numpy(sc, "cuda")
    r = Renderer(ds.n, ds.k, cams)
    rgb, T, last = r.forward(ds)
    g = r.backward(ds, torch.from_numpy(np.concatenate(gC)).float().cuda(),
                   torch.from_numpy(np.concatenate(gT)).float().cuda(), T, last)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy().astype(np.float64) for k, v in g.items()}


def oracle_grads(orc, cams, gC, gT):
    G = None
    for cam, c, t in zip(cams, gC, gT):
        orc.prune_for(cam)
        g = orc.render_grad(cam, c, t)
        G = g if G is None else {k: G[k] + g[k] for k in PARAMS}
    return G


def test_train_workload_gradients_match_oracle(train_setup):
    sc, tgt, cams, orc, gC, gT = train_setup
    G = gpu_grads(sc, cams, gC, gT)
    Go = oracle_grads(orc, cams, gC, gT)
    errs = {k: rel_l2(G[k], Go[k]) for k in PARAMS}
    assert all(e < GRAD_TOL for e in errs.values()), errs


def rays_near(cam, point, radius):
    """Pixels (u, v) whose pixel-centre rays pass within `radius` of `point`
    (selection only: a superset of the pixels a parameter can affect)."""
    u, v = np.meshgrid(np.arange(cam.width), np.arange(cam.height))
    dc = np.stack([(u + 0.5 - cam.cx) / cam.fx, (v + 0.5 - cam.cy) / cam.fy, np.ones_like(u, float)], -1)
    d = dc.reshape(-1, 3) @ np.asarray(cam.rot)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    m = np.asarray(point, np.float64) - np.asarray(cam.origin)
    t = np.maximum(d @ m, 0.0)
    dist = np.linalg.norm(m[None, :] - t[:, None] * d, axis=1)
    sel = dist < radius
    return np.stack([u.reshape(-1)[sel], v.reshape(-1)[sel]], 1).astype(np.int32), np.nonzero(sel)[0]


def test_train_workload_gradients_match_finite_differences(train_setup):
    """64 parameters, eight per group, among those with a non-zero oracle
    gradient; FP64 central differences of the oracle's loss sum gC . C,
    restricted to the pixels whose rays pass near the cell (a parameter of
    cell i changes only cells whose balls its radical planes can reach:
    |p_j - p_i| < R_j + sqrt(R_j^2 - w_j + w_i), well inside 0.15 here)."""
    sc, tgt, cams, orc, gC, gT = train_setup
    G = gpu_grads(sc, cams, gC, gT)
    Go = oracle_grads(orc, cams, gC, gT)
    orc.clear_candidates()
    rng = np.random.default_rng(7)
    P = orc.params
    Rmax = float(np.max(P["R"]))
    checked = 0
    for key in PARAMS:
        flat_go = np.asarray(Go[key]).reshape(-1)
        width = flat_go.size // sc.n
        nz = np.nonzero(np.abs(flat_go) > 1e-3 * np.abs(flat_go).max())[0]
        if key == "normal":  # away from the face-frame seam (n_z ~ 0)
            nz = nz[np.abs(P["normal"][nz // 3, 2]) > 1e-2]
        done = 0
        for j in rng.permutation(nz):
            if done == 8:
                break
            cell = int(j // width)
            scale = {"pos": float(P["R"][cell]), "R": float(P["R"][cell]), "offset": float(P["R"][cell]),
                     "w": float(P["w"][cell]), "sigma": float(P["sigma"][cell])}.get(key, 1.0)
            # central differences at h and h/2, Richardson-extrapolated: at h = 1e-4 scale the
            # h^2 term cancels and the loss's rounding stays far below 1e-6 of the derivative
            # (at 1e-6 scale the cancellation alone reaches ~5e-6 relative)
            h = 1e-4 * scale
            views = []
            for v, cam in enumerate(cams):
                pix, flat = rays_near(cam, P["pos"][cell], 4 * Rmax + float(P["R"][cell]))
                if len(pix):
                    sub = oracle.Oracle(sc)
                    sub.prune_for(cam, pix)
                    views.append((sub, cam, pix, gC[v][flat]))

            def loss(value):
                tot = 0.0
                for sub, cam, pix, g in views:
                    sub.params[key].reshape(-1)[j] = value
                    c, _ = sub.render(cam, pix)
                    tot += float(np.sum(c * g))
                return tot
            old = float(P[key].reshape(-1)[j])
            l0, lp, lm = loss(old), loss(old + h), loss(old - h)
            right, left = (lp - l0) / h, (l0 - lm) / h
            tol = 1e-3 * max(abs(right), 1e-2 * np.abs(flat_go).max())
            if abs(right - left) > tol:
                continue          # an active-constraint switch within h: a kink, not a derivative
            fd1 = (lp - lm) / (2 * h)
            fd2 = (loss(old + 0.5 * h) - loss(old - 0.5 * h)) / h
            fd = (4.0 * fd2 - fd1) / 3.0
            g = G[key].reshape(-1)[j]
            assert abs(fd - flat_go[j]) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(flat_go).max()), \
                ("oracle adjoint vs FD", key, j, flat_go[j], fd)
            assert abs(g - fd) <= 1e-3 * max(abs(fd), 1e-2 * np.abs(flat_go).max()), ("gpu vs FD", key, j, g, fd)
            checked += 1
            done += 1
    assert checked == 64
