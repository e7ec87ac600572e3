"""Adversarial parity for the float segment ends (forward and backward
against the FP64 oracle).

The renderer computes the sphere's D = R^2 - |v|^2 in float, in the frame of
the ray's closest approach, and recomputes an end in FP64 only when its float
error bound could matter: |D| below a per-cell threshold, or a plane or face
end whose |d.a| is small against its error bound.  These scenes are built so
that those decisions are close:

- grazing rays: each cell's sphere is placed so that one pixel ray passes at
  R (1 + eps) from the site, eps from -1e-3 to +1e-4 (|D| -> 0 from both sides);
- near-parallel planes and faces: pairs of equal-weight sites straddle a
  pixel ray so that their radical plane is parallel to the ray up to a tilt
  of 0 to 1e-4, at 1e-4 to 3e-3 of the pair's half distance from it, and
  dipole faces are set parallel to the ray the same way;
- far cameras: cells of radius 5e-4 to 2e-3 seen from 1,000 to 30,000 radii
  through a narrow field of view.

Tolerances are the suite's: 1e-4 max abs per RGB channel, 1e-5 in T, 1e-3
relative L2 per gradient tensor."""
import numpy as np
import pytest

import oracle
from paper_2604_24994_gb300 import inputs
from tests.gpu_util import GRAD_TOL, assert_close_image, rel_l2
from tests.oracle_util import f32, make_scene, random_dirs

pytestmark = pytest.mark.gpu

PARAMS = ("pos", "w", "R", "sigma", "rgb", "normal", "offset", "tex")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2604_24994_gb300 import build
    build.build()


def pixel_ray(cam, u, v):
    o, d = oracle.Oracle(make_scene(np.zeros((1, 3)), [0.0], [0.0])).ray(cam, u, v)
    return o, d


def perp(d, rng):
    e = np.cross(d, rng.normal(size=3))
    return e / np.linalg.norm(e)


def grazing_scene(cam, rng):
    eps = [-1e-3, -1e-4, -1e-5, -1e-6, -1e-7, 0.0, 1e-7, 1e-6, 1e-5, 1e-4]
    pos, R = [], []
    us = np.linspace(6, cam.width - 7, 6).astype(int)
    vs = np.linspace(6, cam.height - 7, 5).astype(int)
    k = 0
    for v in vs:
        for u in us:
            o, d = pixel_ray(cam, u, v)
            t = rng.uniform(1.6, 2.4)
            r = rng.uniform(0.04, 0.09)
            p = (o + t * d + r * perp(d, rng)).astype(np.float32).astype(np.float64)
            # the pixel ray's distance from the float32 site, then R just around it
            m = o - p
            b = np.linalg.norm(m - np.dot(m, d) * d)
            pos.append(p)
            R.append(np.float32(b * (1.0 + eps[k % len(eps)])))
            k += 1
    pos = np.array(pos)
    R = np.array(R, np.float64)
    n = len(R)
    w = (R / 1.5) ** 2
    sigma = np.exp(rng.normal(2.0, 0.7, n))        # dense: chord errors show in T
    rgb = rng.uniform(0, 1, (n, 3))
    nrm = random_dirs(rng, n)
    off = np.where(np.arange(n) % 3 == 0, rng.uniform(-0.5, 0.5, n) * R, 10 * R)
    tex = rng.normal(0, 0.2, (n, 12))
    return f32(make_scene(pos, w, R, sigma, rgb, nrm, off, tex))


def near_parallel_scene(cam, rng):
    """Pairs of equal-weight sites straddle a pixel ray so that their radical
    plane (the bisector) is parallel to the ray up to a tilt of 0 to 1e-4 and
    lies at a small offset from it (1e-4 to 3e-3 of the pair's half
    distance); one site of each pair has its dipole face set the same way.
    The offsets are kept well above the float32 rounding of the inputs, so
    each ray lies on a definite side of every such plane (an offset at the
    inputs' rounding level would be a tie, which either side may take)."""
    tilts = [0.0, 1e-7, 1e-6, 1e-5, 1e-4]
    offs = [1e-4, -1e-4, 1e-3, -1e-3, 3e-3, -3e-3]
    pos, R, nrm, off = [], [], [], []
    us = np.linspace(8, cam.width - 9, 4).astype(int)
    vs = np.linspace(8, cam.height - 9, 3).astype(int)
    k = 0
    for v in vs:
        for u in us:
            o, d = pixel_ray(cam, u, v)
            x0 = o + rng.uniform(1.7, 2.3) * d
            e = perp(d, rng)
            h = rng.uniform(0.03, 0.06)
            tilt = tilts[k % len(tilts)] * (1 if k % 2 else -1)
            # equal weights: the bisector has normal a = e + tilt d and passes
            # through the pair's midpoint, offs * h from the ray along a
            a = e + tilt * d
            a /= np.linalg.norm(a)
            mid = x0 + offs[k % len(offs)] * h * a
            for sgn in (1.0, -1.0):
                pos.append(mid + sgn * h * a)
                rr = rng.uniform(1.4, 2.0) * h
                R.append(rr)
                # one face parallel to the ray (up to a tilt), offs * R from it; one far away
                f = perp(d, rng) + tilts[(k + 2) % len(tilts)] * d
                f /= np.linalg.norm(f)
                nrm.append(f if sgn > 0 else rng.normal(size=3))
                off.append(float(np.dot(f, x0 - pos[-1])) + offs[(k + 3) % len(offs)] * rr if sgn > 0 else 10 * rr)
            k += 1
    pos = np.array(pos)
    n = len(pos)
    R = np.array(R)
    w = np.full(n, 0.01)
    sigma = np.exp(rng.normal(1.5, 0.5, n))
    rgb = rng.uniform(0, 1, (n, 3))
    tex = rng.normal(0, 0.2, (n, 12))
    return f32(make_scene(pos, w, R, sigma, rgb, np.array(nrm), np.array(off), tex))


def far_scene(rng, n=60):
    pos = rng.uniform(-0.015, 0.015, (n, 3))
    r = rng.uniform(5e-4, 2e-3, n) / 1.5
    R = 1.5 * r
    sigma = np.exp(rng.normal(0, 0.7, n)) / R      # x = sigma l of order one
    rgb = rng.uniform(0, 1, (n, 3))
    nrm = random_dirs(rng, n)
    off = rng.uniform(-1, 1, n) * r
    tex = rng.normal(0, 0.2, (n, 12))
    return f32(make_scene(pos, r * r, R, sigma, rgb, nrm, off, tex))


def gpu_render_and_grads(sc, cams, gC, gT):
    import torch
    from paper_2604_24994_gb300 import DeviceScene, Renderer
    ds = DeviceScene.from_numpy(sc, "cuda")
    r = Renderer(ds.n, ds.k, cams)
    rgb, T, last = r.forward(ds)
    g = r.backward(ds, torch.from_numpy(gC).float().cuda(), torch.from_numpy(gT).float().cuda(), T, last)
    torch.cuda.synchronize()
    return (rgb.cpu().numpy().astype(np.float64), T.cpu().numpy().astype(np.float64),
            {k: v.cpu().numpy().astype(np.float64) for k, v in g.items()})


def check(sc, cams, seed):
    rng = np.random.default_rng(seed)
    npx = sum(c.n_pixels for c in cams)
    gC = rng.normal(size=(npx, 3))
    gT = rng.normal(size=npx)
    rgb, T, G = gpu_render_and_grads(sc, cams, gC, gT)
    orc = oracle.Oracle(sc)
    Go = None
    o = 0
    for v, cam in enumerate(cams):
        n = cam.n_pixels
        rgb_o, T_o = orc.render(cam)
        assert (T_o < 0.999).sum() > n // 20, "the scene must cover the view"
        assert_close_image(rgb[o:o + n], T[o:o + n], rgb_o, T_o, f"view {v}")
        g = orc.render_grad(cam, gC[o:o + n], gT[o:o + n])
        Go = g if Go is None else {k: Go[k] + g[k] for k in PARAMS}
        o += n
    errs = {k: rel_l2(G[k], Go[k]) for k in PARAMS if np.linalg.norm(Go[k]) > 0}
    bad = {k: e for k, e in errs.items() if e > GRAD_TOL}
    assert not bad, f"relative L2 above {GRAD_TOL}: {bad}; all: {errs}"


def test_grazing_rays_near_tangent_spheres():
    cam = inputs.look_at((2.0, 0.3, 0.2), 64, 48, fov_y_deg=40)
    sc = grazing_scene(cam, np.random.default_rng(31))
    check(sc, [cam], 1)


def test_planes_and_faces_parallel_to_the_ray():
    cam = inputs.look_at((-1.8, 0.6, 0.4), 56, 40, fov_y_deg=45)
    sc = near_parallel_scene(cam, np.random.default_rng(32))
    check(sc, [cam], 2)


def test_cells_seen_from_thousands_of_radii():
    sc = far_scene(np.random.default_rng(33))
    cams = [inputs.look_at((3.0, 0.4, -0.2), 48, 40, fov_y_deg=0.8),     # ~2,000-6,000 R
            inputs.look_at((0.0, -30.0, 5.0), 40, 40, fov_y_deg=0.08)]    # ~20,000-60,000 R
    check(sc, cams, 3)
