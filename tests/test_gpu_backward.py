"""GPU backward parity: pf_render_bwd (back-to-front replay from the (T, last)
checkpoint) against the FP64 oracle's adjoint (1e-3 relative L2 per
parameter tensor) and against FP64 central differences of the oracle."""
import numpy as np
import pytest

import oracle
from paper_2604_24994_gb300 import inputs
from tests.gpu_util import GRAD_TOL, rel_l2
from tests.oracle_util import cluster_scene, f32

pytestmark = pytest.mark.gpu

PARAMS = ("pos", "w", "R", "sigma", "rgb", "normal", "offset", "tex")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2604_24994_gb300 import build
    build.build()


def gpu_grads(sc, cams, gC, gT):
    import torch
    from paper_2604_24994_gb300 import DeviceScene, Renderer
    ds = DeviceScene.from_numpy(sc, "cuda")
    r = Renderer(ds.n, ds.k, cams)
    rgb, T, last = r.forward(ds)
    g = r.backward(ds, torch.from_numpy(gC).float().cuda(), torch.from_numpy(gT).float().cuda(), T, last)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy().astype(np.float64) for k, v in g.items()}


def check_grads(G, Go, tol=GRAD_TOL):
    errs = {}
    for k in PARAMS:
        a, b = G[k], np.asarray(Go[k])
        if np.linalg.norm(b) == 0:
            assert np.linalg.norm(a) < 1e-6, k
            continue
        errs[k] = rel_l2(a, b)
    bad = {k: e for k, e in errs.items() if e > tol}
    assert not bad, f"relative L2 above {tol}: {bad}; all: {errs}"
    return errs


def test_backward_tiny_full_frame(tiny):
    sc, cam = tiny
    rng = np.random.default_rng(0)
    n = cam.n_pixels
    gC = rng.normal(size=(n, 3))
    gT = rng.normal(size=n)
    G = gpu_grads(sc, [cam], gC, gT)
    Go = oracle.Oracle(sc).render_grad(cam, gC, gT)
    check_grads(G, Go)


def test_backward_dense_cluster_multiview():
    rng = np.random.default_rng(12)
    sc = f32(cluster_scene(rng, n=40, spread=0.15, r=(0.06, 0.12), tex_std=0.2))
    cams = [inputs.look_at((0.7, 0.2, 0.1), 48, 40, fov_y_deg=40),
            inputs.look_at((-0.5, 0.5, 0.3), 33, 21, fov_y_deg=50)]
    npx = sum(c.n_pixels for c in cams)
    gC = rng.normal(size=(npx, 3))
    gT = rng.normal(size=npx)
    G = gpu_grads(sc, cams, gC, gT)
    orc = oracle.Oracle(sc)
    Go = None
    o = 0
    for cam in cams:
        g = orc.render_grad(cam, gC[o:o + cam.n_pixels], gT[o:o + cam.n_pixels])
        Go = g if Go is None else {k: Go[k] + g[k] for k in PARAMS}
        o += cam.n_pixels
    check_grads(G, Go)


def test_autograd_function_matches_direct_backward(tiny):
    import torch
    from paper_2604_24994_gb300 import DeviceScene, Renderer, render
    sc, cam = tiny
    ds = DeviceScene.from_numpy(sc, "cuda", requires_grad=True)
    r = Renderer(ds.n, ds.k, [cam])
    rgb, T = render(r, ds)
    target = torch.rand_like(rgb)
    loss = ((rgb - target) ** 2).sum() + T.sum()
    loss.backward()
    gC = (2 * (rgb - target)).detach().cpu().numpy().astype(np.float64)
    gT = np.ones(cam.n_pixels)
    Go = oracle.Oracle(sc).render_grad(cam, gC, gT)
    G = {k: ds.params[k].grad.cpu().numpy().astype(np.float64) for k in PARAMS}
    check_grads(G, Go)


def test_hit_mask_replay_matches_full_retest():
    """The backward replays only the (cell, lane) pairs the forward recorded
    as hits; once the bins are rebuilt (the recorded masks are dropped) it
    re-tests every listed cell instead.  Both replays give the same
    gradients up to the order of the atomic sums, and both match the oracle."""
    import torch
    from paper_2604_24994_gb300 import DeviceScene, Renderer
    sc = inputs.capture_scene(20_000, seed=5, K=32)
    cam = inputs.look_at((2.2, 0.4, 0.3), 96, 72)
    ds = DeviceScene.from_numpy(sc, "cuda")
    r = Renderer(ds.n, ds.k, [cam])
    rgb, T, last = r.forward(ds)
    rng = np.random.default_rng(3)
    gC = torch.from_numpy(rng.normal(size=(cam.n_pixels, 3))).float().cuda()
    gT = torch.from_numpy(rng.normal(size=cam.n_pixels)).float().cuda()
    g_mask = r.backward(ds, gC, gT, T, last)
    r.bin(ds)  # same scene and view: identical bins, but no recorded hits
    g_full = r.backward(ds, gC, gT, T, last)
    r.record_hits(False)  # a forward that records nothing: the backward re-tests
    rgb2, T2, last2 = r.render_fwd(ds)
    g_off = r.backward(ds, gC, gT, T2, last2)
    torch.cuda.synchronize()
    assert torch.equal(rgb, rgb2) and torch.equal(T, T2) and torch.equal(last, last2)
    for k in PARAMS:
        a = g_mask[k].double().cpu().numpy()
        for other in (g_full, g_off):
            b = other[k].double().cpu().numpy()
            assert rel_l2(a, b) < 1e-5, (k, rel_l2(a, b))
    # the oracle's adjoint of the same image (sampled pixels would not do:
    # the gradients are sums over every pixel)
    orc = oracle.Oracle(sc)
    orc.prune_for(cam)
    Go = orc.render_grad(cam, gC.cpu().numpy().astype(np.float64), gT.cpu().numpy().astype(np.float64))
    check_grads({k: v.double().cpu().numpy() for k, v in g_mask.items()}, Go)


def test_replay_beyond_the_recorded_hits_per_pixel():
    """A chain of 300 faint cells along the view axis gives every ray more
    hits than the forward records per pixel (HIT_CAP = 256); the backward
    re-clips the later ones.  Same gradients as a backward with no recorded
    hits at all, and as the oracle."""
    import torch
    from paper_2604_24994_gb300 import DeviceScene, Renderer
    n = 300
    x = np.linspace(-3.0, 3.0, n)
    pos = np.stack([x, 0.001 * np.sin(7 * x), 0.001 * np.cos(5 * x)], 1)
    spacing = 6.0 / (n - 1)
    r = np.full(n, 0.6 * spacing)
    w = r ** 2
    R = np.full(n, 40 * spacing)            # balls much wider than the slabs
    nbr, R, _ = inputs.build_neighbours(pos, w, R, 16)
    rng = np.random.default_rng(4)
    normal = rng.normal(size=(n, 3))
    sc = inputs.Scene(pos=pos.astype(np.float32), w=w.astype(np.float32), R=R.astype(np.float32),
                      sigma=np.full(n, 0.1, np.float32), rgb=rng.uniform(size=(n, 3)).astype(np.float32),
                      normal=normal.astype(np.float32), offset=np.full(n, 0.5 * spacing, np.float32),
                      tex=rng.normal(0, 0.1, size=(n, 12)).astype(np.float32), nbr=nbr)
    cam = inputs.look_at((4.0, 0.0, 0.0), 24, 16, fov_y_deg=0.1)
    ds = DeviceScene.from_numpy(sc, "cuda")
    rd = Renderer(ds.n, ds.k, [cam])
    rd.enable_stats(True)
    rgb, T, last = rd.forward(ds)
    st = rd.stats()
    rd.enable_stats(False)
    assert st["hits"] / cam.n_pixels > 280          # well past the recorded 256 per pixel
    rgb, T, last = rd.forward(ds)                  # a forward that records hits
    gC = torch.from_numpy(rng.normal(size=(cam.n_pixels, 3))).float().cuda()
    gT = torch.from_numpy(rng.normal(size=cam.n_pixels)).float().cuda()
    g_rec = rd.backward(ds, gC, gT, T, last)
    rd.record_hits(False)
    rgb2, T2, last2 = rd.render_fwd(ds)
    g_off = rd.backward(ds, gC, gT, T2, last2)
    torch.cuda.synchronize()
    for k in PARAMS:
        a, b = g_rec[k].double().cpu().numpy(), g_off[k].double().cpu().numpy()
        assert rel_l2(a, b) < 1e-5, (k, rel_l2(a, b))
    Go = oracle.Oracle(sc).render_grad(cam, gC.cpu().numpy().astype(np.float64), gT.cpu().numpy().astype(np.float64))
    check_grads({k: v.double().cpu().numpy() for k, v in g_rec.items()}, Go)


@pytest.mark.parametrize("cap", [1000, 3])
def test_stored_segments_backward(cap):
    """pf_plan_store_segments: the forward stores every hit's segment (or
    only each pixel's first 3, the rest replayed), the backward reads them
    instead of recomputing; the gradients agree with the replaying backward
    and with the FP64 adjoint."""
    import torch
    from paper_2604_24994_gb300 import DeviceScene, Renderer
    rng = np.random.default_rng(17)
    sc = f32(cluster_scene(rng, n=40, spread=0.15, r=(0.06, 0.12), tex_std=0.2))
    cams = [inputs.look_at((0.7, 0.2, 0.1), 48, 40, fov_y_deg=40),
            inputs.look_at((-0.5, 0.5, 0.3), 33, 21, fov_y_deg=50)]
    npx = sum(c.n_pixels for c in cams)
    gC = torch.from_numpy(rng.normal(size=(npx, 3))).float().cuda()
    gT = torch.from_numpy(rng.normal(size=npx)).float().cuda()
    ds = DeviceScene.from_numpy(sc, "cuda")
    out = {}
    for name, kw in (("replay", {}), ("stored", {"store_segments": cap})):
        r = Renderer(ds.n, ds.k, cams, **kw)
        rgb, T, last = r.forward(ds)
        if name == "stored":
            counts = r.hit_counts()
            assert counts.max() > 3 and (cap > counts.max() or cap == 3)
        g = r.backward(ds, gC, gT, T, last)
        torch.cuda.synchronize()
        out[name] = {k: v.cpu().numpy().astype(np.float64) for k, v in g.items()}
    for k in PARAMS:
        if np.linalg.norm(out["replay"][k]) > 0:
            assert rel_l2(out["stored"][k], out["replay"][k]) < 1e-4, k
    orc = oracle.Oracle(sc)
    Go = None
    o = 0
    for cam in cams:
        g = orc.render_grad(cam, gC[o:o + cam.n_pixels].cpu().numpy(), gT[o:o + cam.n_pixels].cpu().numpy())
        Go = g if Go is None else {k: Go[k] + g[k] for k in PARAMS}
        o += cam.n_pixels
    check_grads(out["stored"], Go)
