"""Face displacement (Eq. svdisp, one-step plane shift), learned detail-site
positions, spherical-Voronoi site colours and eight detail sites per face
(Sec. 3.4) on the GPU: forward and backward against the FP64 oracle, and
the call that refuses such a scene (a counting pass)."""
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


def gpu_render(sc, cams, disp, sites=None):
    import torch
    from paper_2604_24994_gb300 import DeviceScene, Renderer
    ds = DeviceScene.from_numpy(sc, "cuda", disp=disp, sites=sites)
    r = Renderer(ds.n, ds.k, cams)
    rgb, T, last = r.forward(ds)
    torch.cuda.synchronize()
    return rgb.cpu().numpy().astype(np.float64), T.cpu().numpy().astype(np.float64), last.cpu().numpy()


def random_disp(sc, scale, seed):
    rng = np.random.default_rng(seed)
    return (rng.uniform(-scale, scale, (sc.n, 4)) * sc.R[:, None]).astype(np.float32)


def random_sites(sc, spread, seed):
    rng = np.random.default_rng(seed)
    base = np.array([[-1, -1], [1, -1], [-1, 1], [1, 1]], np.float64) / 3.0
    return (base[None] + rng.uniform(-spread, spread, (sc.n, 4, 2))).astype(np.float32)


@pytest.mark.parametrize("with_disp", [True, False])
def test_learned_sites_forward_tiny(tiny, with_disp):
    sc, cam = tiny
    disp = random_disp(sc, 0.3, 5) if with_disp else None
    sites = random_sites(sc, 0.2, 6)
    rgb, T, last = gpu_render(sc, [cam], disp, sites)
    rgb_o, T_o = oracle.Oracle(sc, disp=disp, sites=sites).render(cam)
    assert_close_image(rgb, T, rgb_o, T_o, f"learned sites, displaced={with_disp}")


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


@pytest.mark.parametrize("with_masks,with_disp,with_sites", [(True, True, False), (False, True, False),
                                                             (True, True, True), (False, False, True)])
def test_displaced_backward_matches_the_oracle(with_masks, with_disp, with_sites):
    """pf_render_bwd on a displaced scene and / or learned sites: every
    parameter's gradient, the displacements' and the sites' included, within
    1e-3 relative L2 of the FP64 adjoint (replaying the forward's recorded
    hits, or re-clipping)."""
    import torch
    from paper_2604_24994_gb300 import DeviceScene, Renderer
    from tests.test_gpu_backward import check_grads
    rng = np.random.default_rng(31)
    sc = f32(cluster_scene(rng, n=40, spread=0.15, r=(0.06, 0.12), tex_std=0.2))
    disp = random_disp(sc, 0.35, 4) if with_disp else None
    sites = random_sites(sc, 0.2, 7) if with_sites else None
    cams = [inputs.look_at((0.7, 0.2, 0.1), 48, 40, fov_y_deg=40),
            inputs.fisheye_look_at((-0.5, 0.5, 0.3), 33, 29, fov_deg=70.0)]
    npx = sum(c.n_pixels for c in cams)
    gC = rng.normal(size=(npx, 3))
    gT = rng.normal(size=npx)
    ds = DeviceScene.from_numpy(sc, "cuda", disp=disp, sites=sites)
    r = Renderer(ds.n, ds.k, cams, hit_records=with_masks)
    rgb, T, last = r.forward(ds)
    g = r.backward(ds, torch.from_numpy(gC).float().cuda(), torch.from_numpy(gT).float().cuda(), T, last)
    torch.cuda.synchronize()
    G = {k: v.cpu().numpy().astype(np.float64) for k, v in g.items()}
    orc = oracle.Oracle(sc, disp=disp, sites=sites)
    Go = None
    o = 0
    for cam in cams:
        gg = orc.render_grad(cam, gC[o:o + cam.n_pixels], gT[o:o + cam.n_pixels])
        Go = gg if Go is None else {k: Go[k] + gg[k] for k in gg}
        o += cam.n_pixels
    check_grads(G, Go)
    from tests.gpu_util import rel_l2
    for k in ("disp", "sites"):
        if k in Go:
            assert np.linalg.norm(Go[k]) > 0
            assert rel_l2(G[k].reshape(-1), Go[k].reshape(-1)) < 1e-3, k


def test_displaced_scene_refuses_a_stats_pass(tiny):
    """The work counters cover the plain face model only: a counting forward
    of a displaced scene is refused on the host (contributions are not:
    tests/test_gpu_contrib.py checks them for every face model)."""
    from paper_2604_24994_gb300 import DeviceScene, Renderer, _lib
    sc, cam = tiny
    ds = DeviceScene.from_numpy(sc, "cuda", disp=random_disp(sc, 0.2, 3))
    r = Renderer(ds.n, ds.k, [cam])
    r.bin(ds)
    r.enable_stats(True)
    with pytest.raises(_lib.PFError) as e:
        r.render_fwd(ds)
    assert e.value.status == _lib.PF_ERR_INVALID_ARG


def random_sv(sc, seed):
    rng = np.random.default_rng(seed)
    axes = rng.normal(size=(sc.n, 4, 8, 3))
    cols = rng.uniform(0, 1, (sc.n, 4, 8, 3))
    return np.concatenate([axes, cols], -1).astype(np.float32)


@pytest.mark.parametrize("with_disp,with_sites", [(False, False), (True, True)])
def test_view_dependent_site_colours_forward(with_disp, with_sites):
    """Spherical-Voronoi site colours (eight axes per site) in the forward,
    alone and with displacement and learned sites, pinhole and fisheye
    views, against the FP64 oracle."""
    import torch
    from paper_2604_24994_gb300 import DeviceScene, Renderer
    rng = np.random.default_rng(9)
    sc = f32(cluster_scene(rng, n=50, spread=0.3, r=(0.08, 0.2), tex_std=0.15))
    disp = random_disp(sc, 0.3, 8) if with_disp else None
    sites = random_sites(sc, 0.2, 9) if with_sites else None
    sv = random_sv(sc, 10)
    cams = [inputs.look_at((1.2, 0.4, 0.3), 80, 64),
            inputs.fisheye_look_at((-0.9, 0.6, 0.2), 60, 60, fov_deg=150.0)]
    ds = DeviceScene.from_numpy(sc, "cuda", disp=disp, sites=sites, sv=sv)
    r = Renderer(ds.n, ds.k, cams)
    rgb, T, last = r.forward(ds)
    torch.cuda.synchronize()
    rgb = rgb.cpu().numpy().astype(np.float64)
    T = T.cpu().numpy().astype(np.float64)
    orc = oracle.Oracle(sc, disp=disp, sites=sites, sv=sv)
    o = 0
    for cam in cams:
        n = cam.n_pixels
        rgb_o, T_o = orc.render(cam)
        assert_close_image(rgb[o:o + n], T[o:o + n], rgb_o, T_o, f"sv {cam.width}x{cam.height}")
        o += n
    # the colours are view dependent: the constant-colour image differs
    rgb_c, _ = oracle.Oracle(sc, disp=disp, sites=sites).render(cams[0])
    assert np.abs(rgb_c - rgb[:cams[0].n_pixels]).max() > 1e-2


@pytest.mark.parametrize("with_masks,with_disp", [(True, False), (False, True)])
def test_view_dependent_site_colours_backward(with_masks, with_disp):
    """The backward with spherical-Voronoi site colours: every parameter's
    gradient, the axes' and colours' included, within 1e-3 relative L2 of
    the FP64 adjoint; tex gets none (the colours replace it)."""
    import torch
    from paper_2604_24994_gb300 import DeviceScene, Renderer
    from tests.gpu_util import rel_l2
    rng = np.random.default_rng(33)
    sc = f32(cluster_scene(rng, n=40, spread=0.15, r=(0.06, 0.12), tex_std=0.2))
    disp = random_disp(sc, 0.3, 12) if with_disp else None
    sv = random_sv(sc, 13)
    cams = [inputs.look_at((0.7, 0.2, 0.1), 48, 40, fov_y_deg=40),
            inputs.look_at((-0.5, 0.5, 0.3), 33, 21, fov_y_deg=50)]
    npx = sum(c.n_pixels for c in cams)
    gC = rng.normal(size=(npx, 3))
    gT = rng.normal(size=npx)
    ds = DeviceScene.from_numpy(sc, "cuda", disp=disp, sv=sv)
    r = Renderer(ds.n, ds.k, cams, hit_records=with_masks)
    rgb, T, last = r.forward(ds)
    g = r.backward(ds, torch.from_numpy(gC).float().cuda(), torch.from_numpy(gT).float().cuda(), T, last)
    torch.cuda.synchronize()
    G = {k: v.cpu().numpy().astype(np.float64) for k, v in g.items()}
    orc = oracle.Oracle(sc, disp=disp, sv=sv)
    Go = None
    o = 0
    for cam in cams:
        gg = orc.render_grad(cam, gC[o:o + cam.n_pixels], gT[o:o + cam.n_pixels])
        Go = gg if Go is None else {k: Go[k] + gg[k] for k in gg}
        o += cam.n_pixels
    for k in ("pos", "w", "R", "sigma", "rgb", "normal", "offset", "sv") + (("disp",) if with_disp else ()):
        a, b = G[k].reshape(-1), np.asarray(Go[k]).reshape(-1)
        assert np.linalg.norm(b) > 0, k
        assert rel_l2(a, b) < 1e-3, (k, rel_l2(a, b))
    assert np.abs(G["tex"]).max() == 0.0


# ------------------------------------------------- eight detail sites per face

def eight_site_scene(seed, n=40, spread=0.2, r=(0.06, 0.14)):
    """A cluster whose faces carry eight detail sites (Sec. 3.4's main
    configuration): tex [N,24]; displacements [N,8], learned positions
    [N,8,2] (the fixed 3 x 3 grid without its centre, jittered) and
    spherical-Voronoi colours [N,8,8,6] drawn for the cases that use them."""
    rng = np.random.default_rng(seed)
    sc = f32(cluster_scene(rng, n=n, spread=spread, r=r, tex_std=0.2))
    sc.tex = rng.normal(0, 0.2, (sc.n, 24)).astype(np.float32)
    disp = (rng.uniform(-0.3, 0.3, (sc.n, 8)) * sc.R[:, None]).astype(np.float32)
    grid = np.array([[-1, -1], [0, -1], [1, -1], [-1, 0], [1, 0], [-1, 1], [0, 1], [1, 1]], np.float64) / 3.0
    sites = (grid[None] + rng.uniform(-0.15, 0.15, (sc.n, 8, 2))).astype(np.float32)
    sv = np.concatenate([rng.normal(size=(sc.n, 8, 8, 3)), rng.uniform(0, 1, (sc.n, 8, 8, 3))], -1).astype(np.float32)
    return sc, disp, sites, sv


@pytest.mark.parametrize("with_disp,with_sites,with_sv", [(False, False, False), (True, False, False),
                                                          (True, True, False), (False, False, True),
                                                          (True, True, True)])
def test_eight_sites_forward(with_disp, with_sites, with_sv):
    """Eight detail sites per face on the GPU (the fixed grid or learned
    positions, with and without displacement and view-dependent colours),
    pinhole, inside and fisheye views, against the FP64 oracle with eight
    sites."""
    import torch
    from paper_2604_24994_gb300 import DeviceScene, Renderer
    sc, disp, sites, sv = eight_site_scene(21, n=50, spread=0.3, r=(0.08, 0.2))
    disp = disp if with_disp else None
    sites = sites if with_sites else None
    sv = sv if with_sv else None
    cams = [inputs.look_at((1.2, 0.4, 0.3), 80, 64),
            inputs.look_at((0.03, 0.02, 0.01), 41, 37, target=(1.0, 0.2, 0.1)),
            inputs.fisheye_look_at((0.9, -0.6, 0.2), 60, 60, fov_deg=150.0)]
    ds = DeviceScene.from_numpy(sc, "cuda", disp=disp, sites=sites, sv=sv)
    assert ds.n_sites == 8
    r = Renderer(ds.n, ds.k, cams)
    rgb, T, last = r.forward(ds)
    torch.cuda.synchronize()
    rgb = rgb.cpu().numpy().astype(np.float64)
    T = T.cpu().numpy().astype(np.float64)
    orc = oracle.Oracle(sc, disp=disp, sites=sites, sv=sv)
    assert orc.nsite == 8
    o = 0
    for cam in cams:
        n = cam.n_pixels
        rgb_o, T_o = orc.render(cam)
        assert_close_image(rgb[o:o + n], T[o:o + n], rgb_o, T_o, f"eight sites {cam.width}x{cam.height}")
        o += n
    # the eight-site texture is not the four-site one: the colours differ
    sc4 = sc.copy()
    sc4.tex = np.ascontiguousarray(sc.tex[:, :12])
    rgb4, _ = oracle.Oracle(sc4, disp=None if disp is None else disp[:, :4],
                            sites=None if sites is None else sites[:, :4],
                            sv=None if sv is None else sv[:, :4]).render(cams[0])
    assert np.abs(rgb4 - rgb[:cams[0].n_pixels]).max() > 1e-2


@pytest.mark.parametrize("with_masks,with_disp,with_sites,with_sv", [(True, True, True, False),
                                                                    (False, True, False, False),
                                                                    (True, False, False, False),
                                                                    (True, True, False, True)])
def test_eight_sites_backward(with_masks, with_disp, with_sites, with_sv):
    """The backward with eight detail sites: every parameter's gradient, the
    24 texture values, eight displacements, sixteen site coordinates and the
    spherical-Voronoi colours included, within 1e-3 relative L2 of the FP64
    adjoint (replaying recorded hits, or re-clipping)."""
    import torch
    from paper_2604_24994_gb300 import DeviceScene, Renderer
    from tests.gpu_util import rel_l2
    sc, disp, sites, sv = eight_site_scene(34)
    disp = disp if with_disp else None
    sites = sites if with_sites else None
    sv = sv if with_sv else None
    rng = np.random.default_rng(35)
    cams = [inputs.look_at((0.7, 0.2, 0.1), 48, 40, fov_y_deg=40),
            inputs.fisheye_look_at((-0.5, 0.5, 0.3), 33, 29, fov_deg=70.0)]
    npx = sum(c.n_pixels for c in cams)
    gC = rng.normal(size=(npx, 3))
    gT = rng.normal(size=npx)
    ds = DeviceScene.from_numpy(sc, "cuda", disp=disp, sites=sites, sv=sv)
    r = Renderer(ds.n, ds.k, cams, hit_records=with_masks)
    rgb, T, last = r.forward(ds)
    g = r.backward(ds, torch.from_numpy(gC).float().cuda(), torch.from_numpy(gT).float().cuda(), T, last)
    torch.cuda.synchronize()
    G = {k: v.cpu().numpy().astype(np.float64) for k, v in g.items()}
    orc = oracle.Oracle(sc, disp=disp, sites=sites, sv=sv)
    Go = None
    o = 0
    for cam in cams:
        gg = orc.render_grad(cam, gC[o:o + cam.n_pixels], gT[o:o + cam.n_pixels])
        Go = gg if Go is None else {k: Go[k] + gg[k] for k in gg}
        o += cam.n_pixels
    keys = ["pos", "w", "R", "sigma", "rgb", "normal", "offset"] + ([] if with_sv else ["tex"])
    keys += [k for k, on in (("disp", with_disp), ("sites", with_sites), ("sv", with_sv)) if on]
    for k in keys:
        a, b = G[k].reshape(-1), np.asarray(Go[k]).reshape(-1)
        assert a.size == b.size and np.linalg.norm(b) > 0, k
        assert rel_l2(a, b) < 1e-3, (k, rel_l2(a, b))
    if with_sv:
        assert np.abs(G["tex"]).max() == 0.0
