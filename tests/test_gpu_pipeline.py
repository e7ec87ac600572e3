"""The pipelined forward (the plain face model, with or without hit
recording: the benchmark's forward and forward+backward steps, the server
and the static entry point) against the batch-staged forward (the variant
that counts work, and the one that stores every segment), which the other
parity tests pin to the FP64 oracle: the same per-pixel arithmetic in the
same list order, so rgb, T and last must agree bit for bit, and both
recording forwards must count the same hits per pixel.  The scenes cover
early termination (near-opaque cells), batches cut short by the stage's
plane budget (cells with up to 39 kept planes), several views of different
sizes in one plan, a camera inside the cells, long tile lists, and the
capture workload at 720p.  Every run must leave the pipeline's wait-error
word at zero."""
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


def both(sc, cams, **ext):
    """Render with every variant; `ext`: the extended face model's arrays
    (disp, sites, sv) for DeviceScene.from_numpy.  The work-counting run is
    refused for the extended model, so those scenes compare with the
    segment-storing one only."""
    import torch
    from paper_2604_24994_gb300 import DeviceScene, Renderer
    ds = DeviceScene.from_numpy(sc, "cuda", **ext)
    extended = any(v is not None for v in ext.values()) or np.asarray(sc.tex).shape[1] == 24
    out = {}
    runs = (("staged", dict(hit_records=False), True),            # counts work: batch-staged
            ("staged_rec", dict(hit_records=True, store_segments=1), False),  # stores segments: batch-staged
            ("pipe_rec", dict(hit_records=True), False),
            ("pipe", dict(hit_records=False), False))
    for name, kw, stats in runs:
        if stats and extended:
            continue
        r = Renderer(ds.n, ds.k, cams, **kw)
        if stats:
            r.enable_stats(True)
        rgb, T, last = r.forward(ds)
        torch.cuda.synchronize()
        assert r.stats()["wait_errors"] == 0
        hc = r.hit_counts() if kw["hit_records"] else None
        out[name] = (rgb.cpu().numpy(), T.cpu().numpy(), last.cpu().numpy(), hc)
    ref = out["staged_rec"] if extended else out["staged"]
    for name in ("staged_rec", "pipe_rec", "pipe"):
        for x, y, what in zip(out[name][:3], ref[:3], ("rgb", "T", "last")):
            assert np.array_equal(x, y), (name, what)
    assert np.array_equal(out["pipe_rec"][3], out["staged_rec"][3]), "hit counts"
    return out["pipe"][:3]


def test_tiny_and_multiview(tiny):
    sc, cam = tiny
    rgb, T, last = both(sc, [cam])
    rgb_o, T_o = oracle.Oracle(sc).render(cam)
    assert_close_image(rgb.astype(np.float64), T.astype(np.float64), rgb_o, T_o, "tiny, pipelined")
    rng = np.random.default_rng(5)
    sc = f32(cluster_scene(rng, n=60, spread=0.4, r=(0.08, 0.25), tex_std=0.15))
    both(sc, [inputs.look_at((1.4, 0.3, 0.2), 100, 75),
              inputs.look_at((0.05, 0.02, 0.0), 37, 29, target=(1.0, 0.5, 0.1)),
              inputs.fisheye_look_at((-0.9, -0.9, 0.6), 40, 33, fov_deg=160.0)])


def test_plane_budget_cuts_batches_and_early_termination():
    """A dense cluster with all-pairs lists: cells keep many planes, so the
    stage's plane budget cuts batches short; near-opaque densities end most
    pixels early."""
    rng = np.random.default_rng(8)
    sc = cluster_scene(rng, n=40, spread=0.1, r=(0.08, 0.14), tex_std=0.2)
    sc.sigma = sc.sigma * 20.0
    sc = f32(sc)
    cam = inputs.look_at((0.7, 0.2, 0.1), 64, 48, fov_y_deg=40)
    rgb, T, last = both(sc, [cam])
    rgb_o, T_o = oracle.Oracle(sc).render(cam)
    assert_close_image(rgb.astype(np.float64), T.astype(np.float64), rgb_o, T_o, "opaque cluster, pipelined")
    assert (T < 1e-6).sum() > 100


def test_long_lists_and_capture_720p():
    from tests.test_gpu_binning import column_scene
    cam = inputs.look_at((3.0, 0.0, 0.0), 640, 360)
    both(column_scene(cam, [(19, 10), (23, 6)], [80, 24]), [cam])
    sc = inputs.capture_scene(400_000, seed=0, K=32)
    both(sc, [inputs.capture_camera(1280, 720)])


def test_early_termination_across_random_views():
    """Near-opaque cells seen from inside the capture recipe's shell by
    random cameras of mixed sizes, one plan per view and one multi-view plan
    (as the server batches them): most tiles end early, where the warps of a
    tile finish at different batches; the pipeline must neither hang (its
    bounded waits report in wait_errors) nor change a pixel."""
    sc = inputs.capture_scene(200_000, seed=4, K=32)
    sc.sigma = (sc.sigma * 30.0).astype(np.float32)
    rng = np.random.default_rng(12)
    sizes = [(160, 90), (320, 180), (200, 200), (97, 61)]
    cams = inputs.random_sphere_cameras(rng, 8, 1.6, 3.0, sizes, [0.25] * 4)
    for cam in cams[:4]:
        rgb, T, last = both(sc, [cam])
        assert (T < 1e-6).mean() > 0.05
    both(sc, cams)


def test_extended_face_models():
    """Displaced faces with learned site positions, and view-dependent site
    colours: the pipelined kernel's stages carry each cell's extended rows,
    and the image equals the batch-staged kernel's bit for bit (and the
    oracle's within tolerance).  Eight detail sites take the batch-staged
    kernel in every variant; the same comparisons hold."""
    rng = np.random.default_rng(21)
    sc = f32(cluster_scene(rng, n=50, spread=0.3, r=(0.08, 0.2), tex_std=0.15))
    disp = (rng.uniform(-0.3, 0.3, (sc.n, 4)) * sc.R[:, None]).astype(np.float32)
    base = np.array([[-1, -1], [1, -1], [-1, 1], [1, 1]], np.float64) / 3.0
    sites = (base[None] + rng.uniform(-0.2, 0.2, (sc.n, 4, 2))).astype(np.float32)
    sv = np.concatenate([rng.normal(size=(sc.n, 4, 8, 3)), rng.uniform(0, 1, (sc.n, 4, 8, 3))], -1).astype(np.float32)
    cams = [inputs.look_at((1.2, 0.4, 0.3), 80, 64),
            inputs.fisheye_look_at((-0.9, 0.6, 0.2), 60, 60, fov_deg=150.0)]
    rgb, T, _ = both(sc, cams, disp=disp, sites=sites)
    orc = oracle.Oracle(sc, disp=disp, sites=sites)
    n0 = cams[0].n_pixels
    rgb_o, T_o = orc.render(cams[0])
    assert_close_image(rgb[:n0].astype(np.float64), T[:n0].astype(np.float64), rgb_o, T_o, "displaced, pipelined")
    both(sc, cams, sv=sv)
    both(sc, cams, disp=disp, sites=sites, sv=sv)
    # eight sites: texture [N,24], displacement [N,8], positions [N,8,2], colours [N,8,8,6]
    sc8 = sc.copy()
    sc8.tex = rng.normal(0, 0.2, (sc.n, 24)).astype(np.float32)
    disp8 = (rng.uniform(-0.3, 0.3, (sc.n, 8)) * sc.R[:, None]).astype(np.float32)
    grid = np.array([[-1, -1], [0, -1], [1, -1], [-1, 0], [1, 0], [-1, 1], [0, 1], [1, 1]], np.float64) / 3.0
    sites8 = (grid[None] + rng.uniform(-0.15, 0.15, (sc.n, 8, 2))).astype(np.float32)
    sv8 = np.concatenate([rng.normal(size=(sc.n, 8, 8, 3)), rng.uniform(0, 1, (sc.n, 8, 8, 3))], -1).astype(np.float32)
    rgb, T, _ = both(sc8, cams, disp=disp8, sites=sites8)
    rgb_o, T_o = oracle.Oracle(sc8, disp=disp8, sites=sites8).render(cams[0])
    assert_close_image(rgb[:n0].astype(np.float64), T[:n0].astype(np.float64), rgb_o, T_o, "eight sites, pipelined")
    both(sc8, cams)
    both(sc8, cams, disp=disp8, sites=sites8, sv=sv8)


def test_contributions_pipelined_and_staged(tiny):
    """Per-cell contributions (sum of T alpha, and of T alpha max(n.d, 0)^2)
    from the pipelined forward equal the batch-staged forward's (the one that
    stores segments), up to the order of the float atomics, and the images
    are equal bit for bit; with displaced faces too."""
    import torch
    from paper_2604_24994_gb300 import DeviceScene, Renderer
    sc, cam = tiny
    rng = np.random.default_rng(4)
    for ext in ({}, {"disp": (rng.uniform(-0.2, 0.2, (sc.n, 4)) * sc.R[:, None]).astype(np.float32)}):
        ds = DeviceScene.from_numpy(sc, "cuda", **ext)
        res = []
        for kw in (dict(hit_records=True, store_segments=1), dict(hit_records=True), dict(hit_records=False)):
            r = Renderer(ds.n, ds.k, [cam], **kw)
            r.bin(ds)
            cs = torch.zeros(ds.n, device="cuda")
            cn = torch.zeros(ds.n, device="cuda")
            rgb, T, last = r.render_fwd(ds, contrib=(cs, cn))
            torch.cuda.synchronize()
            assert r.stats()["wait_errors"] == 0
            res.append((rgb.cpu().numpy(), T.cpu().numpy(), cs.cpu().numpy(), cn.cpu().numpy()))
        for got in res[1:]:
            assert np.array_equal(got[0], res[0][0]) and np.array_equal(got[1], res[0][1])
            np.testing.assert_allclose(got[2], res[0][2], rtol=1e-5, atol=1e-6)
            np.testing.assert_allclose(got[3], res[0][3], rtol=1e-5, atol=1e-6)
        assert res[0][2].sum() > 1.0
