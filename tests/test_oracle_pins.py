"""Pins for the FP64 CPU oracle: each test checks it against something other
than itself (closed forms, library routines, invariants of the paper's
geometry, brute-force point classification, finite differences)."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle import ACT_CAMERA, ACT_DIPOLE, ACT_SPHERE
from tests.oracle_util import cam_at, cluster_scene, make_scene, random_dirs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def seg_dict(segs):
    return {c: (ta, tb) for c, ta, tb, _, _ in segs}


# ---------------------------------------------------------------- closed forms

def test_isolated_cell_chord_closed_form():
    """One cell, no neighbours, face outside the ball: the segment is the
    sphere chord 2 sqrt(R^2 - b^2) and T = exp(-sigma chord) (Sec. 3.1/3.2)."""
    R, sig = 0.3, 2.0
    rgb = np.array([0.2, 0.5, 0.9])
    orc = oracle.Oracle(make_scene([0, 0, 0], 0.04, R, sig, rgb))
    for b in (0.0, 0.1, 0.25, 0.299):
        o = np.array([[-2.0, b, 0.0]])
        d = np.array([[1.0, 0.0, 0.0]])
        c, T = orc.render_rays(o, d)
        chord = 2 * math.sqrt(R * R - b * b)
        assert T[0] == pytest.approx(math.exp(-sig * chord), rel=1e-13, abs=1e-15)
        np.testing.assert_allclose(c[0], (1 - math.exp(-sig * chord)) * rgb, rtol=1e-12, atol=1e-15)
    # through the centre the chord is the diameter
    segs = orc.ray_segments([-2.0, 0, 0], [1.0, 0, 0])
    assert segs[0][2] - segs[0][1] == pytest.approx(2 * R, rel=1e-14)
    assert segs[0][3] == ACT_SPHERE and segs[0][4] == ACT_SPHERE
    # a miss
    c, T = orc.render_rays([[-2.0, 0.31, 0.0]], [[1.0, 0, 0]])
    assert T[0] == 1.0 and np.all(c == 0)


def test_camera_inside_cell_clips_at_zero():
    """t >= 0: from inside the ball only the forward half-chord counts."""
    R = 0.5
    orc = oracle.Oracle(make_scene([0, 0, 0], 0.1, R, 1.0))
    segs = orc.ray_segments([0.1, 0.0, 0.0], [1.0, 0.0, 0.0])
    assert len(segs) == 1
    c, ta, tb, aa, ab = segs[0]
    assert ta == 0.0 and aa == ACT_CAMERA
    assert tb == pytest.approx(0.4, rel=1e-14) and ab == ACT_SPHERE


def test_two_cells_golden():
    g = json.load(open(os.path.join(GOLDEN, "two_cells_on_axis.json")))
    sc = make_scene([[0, 0, 0], [0.5, 0, 0]], [0.05, 0.03], [0.4, 0.4], [1.0, 2.0],
                    [[1, 0, 0], [0, 1, 0]])
    orc = oracle.Oracle(sc)
    segs = orc.ray_segments([-1.0, 0, 0], [1.0, 0, 0])
    assert len(segs) == len(g["segments"])
    for (c, ta, tb, _, _), (ce, tae, tbe) in zip(segs, g["segments"]):
        assert c == ce
        assert ta == pytest.approx(tae, abs=1e-13)
        assert tb == pytest.approx(tbe, abs=1e-13)
    assert segs[0][4] == 1 and segs[1][3] == 0       # the shared face is the radical plane
    rgb, T = orc.render_rays([[-1.0, 0, 0]], [[1.0, 0, 0]])
    assert T[0] == pytest.approx(g["T"], rel=1e-12)
    np.testing.assert_allclose(rgb[0], g["rgb"], rtol=1e-12, atol=1e-15)


def test_radical_plane_position_general():
    """Off-axis two-cell case: the shared boundary point satisfies
    pow(x,i) = pow(x,j) (the definition, Eq. pow_dist), for random weights."""
    rng = np.random.default_rng(5)
    for _ in range(20):
        D = rng.uniform(0.2, 0.6)
        wi, wj = rng.uniform(0.01, 0.08, 2)
        sc = make_scene([[0, 0, 0], [D, 0, 0]], [wi, wj], [0.7, 0.7])
        orc = oracle.Oracle(sc)
        o = np.array([-1.0, rng.uniform(-0.1, 0.1), rng.uniform(-0.1, 0.1)])
        d = np.array([1.0, rng.uniform(-0.05, 0.05), rng.uniform(-0.05, 0.05)])
        d /= np.linalg.norm(d)
        segs = orc.ray_segments(o, d)
        assert [s[0] for s in segs] == [0, 1]
        t = segs[0][2]
        assert segs[1][1] == pytest.approx(t, abs=1e-13)
        x = o + t * d
        pi = np.sum(x * x) - wi
        pj = np.sum((x - [D, 0, 0]) ** 2) - wj
        assert pi == pytest.approx(pj, abs=1e-13)


# ------------------------------------------------- point classification checks

def classify(sc, x):
    """Plain definition at a point: the power cell (argmin over all sites of
    |x - p|^2 - w), inside its ball, and on the dense side of its face."""
    P = np.asarray(sc.pos, np.float64)
    pw = np.sum((P - x) ** 2, axis=1) - np.asarray(sc.w, np.float64)
    i = int(np.argmin(pw))
    inside = np.sum((x - P[i]) ** 2) <= float(sc.R[i]) ** 2
    n = np.asarray(sc.normal[i], np.float64)
    n = n / np.linalg.norm(n)
    dense = float(np.dot(n, x - P[i])) <= float(sc.offset[i])
    return i, inside and dense


@pytest.mark.parametrize("seed,equal_w", [(1, False), (2, False), (3, True), (4, True)])
def test_segments_match_point_classification(seed, equal_w):
    """Every point inside segment k lies in cell k's bounded dense region,
    and every sampled point on the ray outside all segments lies in none."""
    rng = np.random.default_rng(seed)
    sc = cluster_scene(rng, n=14, equal_w=equal_w)
    orc = oracle.Oracle(sc)
    for _ in range(20):
        o = rng.uniform(-1, 1, 3)
        o = 1.2 * o / np.linalg.norm(o)
        d = -o / np.linalg.norm(o) + rng.normal(0, 0.08, 3)
        d /= np.linalg.norm(d)
        segs = orc.ray_segments(o, d)
        for c, ta, tb, _, _ in segs:
            for f in (0.02, 0.3, 0.5, 0.7, 0.98):
                x = o + (ta + f * (tb - ta)) * d
                i, ins = classify(sc, x)
                assert ins and i == c
        ts = np.linspace(0, 3, 1500)
        for t in ts:
            if any(ta - 1e-9 <= t <= tb + 1e-9 for _, ta, tb, _, _ in segs):
                continue
            _, ins = classify(sc, o + t * d)
            assert not ins


def test_equal_weights_reduce_to_voronoi_kdtree():
    """Equal weights: power cells are Voronoi cells (appendix), so the cell
    of a point is scipy's nearest site."""
    from scipy.spatial import cKDTree
    rng = np.random.default_rng(11)
    sc = cluster_scene(rng, n=30, spread=0.3, equal_w=True, dipole=False)
    tree = cKDTree(np.asarray(sc.pos, np.float64))
    orc = oracle.Oracle(sc)
    checked = 0
    for _ in range(40):
        o = random_dirs(rng, 1)[0] * 1.5
        d = -o / 1.5 + rng.normal(0, 0.1, 3)
        d /= np.linalg.norm(d)
        for c, ta, tb, _, _ in orc.ray_segments(o, d):
            x = o + 0.5 * (ta + tb) * d
            assert tree.query(x)[1] == c
            checked += 1
    assert checked > 50


# ----------------------------------------------------------------- invariants

def ball_union(sc, o, d):
    """Union of the ray's chords through all balls (t >= 0), merged."""
    P = np.asarray(sc.pos, np.float64)
    R = np.asarray(sc.R, np.float64)
    iv = []
    for p, r in zip(P, R):
        m = o - p
        b = m @ d
        disc = b * b - (m @ m - r * r)
        if disc <= 0:
            continue
        t0, t1 = -b - math.sqrt(disc), -b + math.sqrt(disc)
        t0 = max(t0, 0.0)
        if t1 > t0:
            iv.append([t0, t1])
    iv.sort()
    out = []
    for a, b in iv:
        if out and a <= out[-1][1]:
            out[-1][1] = max(out[-1][1], b)
        else:
            out.append([a, b])
    return out


@pytest.mark.parametrize("seed", [21, 22, 23])
def test_tied_scene_cells_tile_the_union_of_balls(seed):
    """R_i^2 - w_i equal for all cells: the bounded cells partition the
    union of the balls, so along any ray the segments neither overlap nor
    leave gaps inside the union, and their lengths sum to its length."""
    rng = np.random.default_rng(seed)
    sc = cluster_scene(rng, n=25, spread=0.25, tied=True, dipole=False)
    orc = oracle.Oracle(sc)
    for _ in range(30):
        o = random_dirs(rng, 1)[0] * 1.3
        d = -o / 1.3 + rng.normal(0, 0.15, 3)
        d /= np.linalg.norm(d)
        segs = orc.ray_segments(o, d)
        U = ball_union(sc, o, d)
        tot = sum(tb - ta for _, ta, tb, _, _ in segs)
        assert tot == pytest.approx(sum(b - a for a, b in U), abs=1e-12)
        for k in range(len(segs) - 1):
            gap = segs[k + 1][1] - segs[k][2]
            assert gap >= -1e-12                       # no overlap
            if gap > 1e-12:                            # a gap must be a gap of the union
                mid = 0.5 * (segs[k][2] + segs[k + 1][1])
                assert not any(a < mid < b for a, b in U)


@pytest.mark.parametrize("seed", [31, 32])
def test_untied_scene_segments_disjoint_and_bounded(seed):
    """R = 1.5 r: segments still never overlap and never exceed the union."""
    rng = np.random.default_rng(seed)
    sc = cluster_scene(rng, n=25, spread=0.25, dipole=False)
    orc = oracle.Oracle(sc)
    for _ in range(30):
        o = random_dirs(rng, 1)[0] * 1.3
        d = -o / 1.3 + rng.normal(0, 0.15, 3)
        d /= np.linalg.norm(d)
        segs = orc.ray_segments(o, d)
        for k in range(len(segs) - 1):
            assert segs[k + 1][1] - segs[k][2] >= -1e-12
        tot = sum(tb - ta for _, ta, tb, _, _ in segs)
        assert tot <= sum(b - a for a, b in ball_union(sc, o, d)) + 1e-12


@pytest.mark.parametrize("seed", [41, 42, 43])
def test_power_painter_order(seed):
    """Thm. power_painter: along any ray from the camera centre, the cells
    are met in increasing order of pow(o, p_i)."""
    rng = np.random.default_rng(seed)
    sc = cluster_scene(rng, n=30, spread=0.25)
    orc = oracle.Oracle(sc)
    P = np.asarray(sc.pos, np.float64)
    W = np.asarray(sc.w, np.float64)
    n_pairs = 0
    for q in range(40):
        # some cameras inside the cluster
        o = random_dirs(rng, 1)[0] * (1.3 if q % 2 else 0.1)
        d = random_dirs(rng, 1)[0]
        if q % 2:
            d = -o / 1.3 + 0.15 * d
            d /= np.linalg.norm(d)
        segs = orc.ray_segments(o, d)
        keys = [np.sum((o - P[c]) ** 2) - W[c] for c, *_ in segs]
        for a, b in zip(keys, keys[1:]):
            assert a < b
            n_pairs += 1
    assert n_pairs > 30


def test_cech_lists_equal_brute_force_for_tied_scene():
    """Sec. 3.2: with R = r, only overlapping balls can share a face, so
    clipping against the Cech neighbours (all overlapping spheres) renders
    the same image as clipping against every site."""
    rng = np.random.default_rng(51)
    sc = cluster_scene(rng, n=40, spread=0.3, tied=True)
    P = np.asarray(sc.pos, np.float64)
    R = np.asarray(sc.R, np.float64)
    lists = {i: [j for j in range(len(P)) if j != i and np.linalg.norm(P[i] - P[j]) < R[i] + R[j]]
             for i in range(len(P))}
    cam = cam_at([1.2, 0.3, 0.2], 24, 24)
    a = oracle.Oracle(sc)
    rgb0, T0 = a.render(cam)
    a.set_candidate_lists(lists)
    rgb1, T1 = a.render(cam)
    assert np.array_equal(rgb0, rgb1) and np.array_equal(T0, T1)
    assert np.any(T0 < 1)


def test_prune_matches_brute_force(tiny):
    sc, cam = tiny
    a = oracle.Oracle(sc)
    pix = np.stack(np.meshgrid(np.arange(0, 128, 3), np.arange(0, 128, 3)), -1).reshape(-1, 2)
    rgb0, T0 = a.render(cam, pix)
    a.prune_for(cam, pix)
    rgb1, T1 = a.render(cam, pix)
    assert np.array_equal(rgb0, rgb1) and np.array_equal(T0, T1)


# --------------------------------------------------------------------- dipole

def test_dipole_limits_and_complement():
    """Sec. 3.3: the face splits the cell; a face outside the ball (offset >=
    R) leaves the whole cell dense, offset <= -R makes it empty, and the two
    halves (n, o) and (-n, -o) add up to the whole cell."""
    rng = np.random.default_rng(61)
    base = cluster_scene(rng, n=12, spread=0.2, dipole=True)
    whole = base.copy()
    whole.offset = np.asarray(base.R, np.float64) * 1.0000001
    flip = base.copy()
    flip.normal = -np.asarray(base.normal)
    flip.offset = -np.asarray(base.offset)
    gone = base.copy()
    gone.offset = -np.asarray(base.R, np.float64) * 1.0000001
    big = base.copy()
    big.offset = np.full(base.n, 1e3)
    ob, of, ow, og, obig = (oracle.Oracle(s) for s in (base, flip, whole, gone, big))
    for _ in range(30):
        o = random_dirs(rng, 1)[0] * 1.2
        d = -o / 1.2 + rng.normal(0, 0.1, 3)
        d /= np.linalg.norm(d)
        sw = seg_dict(ow.ray_segments(o, d))
        assert sw == seg_dict(obig.ray_segments(o, d))
        assert og.ray_segments(o, d) == []
        sb = seg_dict(ob.ray_segments(o, d))
        sf = seg_dict(of.ray_segments(o, d))
        for c, (ta, tb) in sw.items():
            lb = sb.get(c, (0, 0))
            lf = sf.get(c, (0, 0))
            assert (lb[1] - lb[0]) + (lf[1] - lf[0]) == pytest.approx(tb - ta, abs=1e-12)


# -------------------------------------------------------------------- texture

def test_onb_properties():
    rng = np.random.default_rng(71)
    for n in list(random_dirs(rng, 50)) + [np.array([0, 0, 1.0]), np.array([0, 0, -1.0])]:
        e1, e2 = oracle.onb(n)
        M = np.stack([e1, e2, n])
        np.testing.assert_allclose(M @ M.T, np.eye(3), atol=1e-14)
        np.testing.assert_allclose(np.cross(e1, e2), n, atol=1e-14)
    e1, e2 = oracle.onb(np.array([0, 0, 1.0]))
    np.testing.assert_allclose(e1, [1, 0, 0])
    np.testing.assert_allclose(e2, [0, 1, 0])


def face_scene(tex, R=1.0):
    # cell at the origin, face = plane z = 0 through p, dense half z <= 0
    return make_scene([0, 0, 0], 0.2, R, 1.0, [0.1, 0.2, 0.3], [0, 0, 1.0], 0.0, tex)


def test_texture_closed_forms():
    """Eq. svrad on the face: zero texture gives the base colour; equal site
    values add a constant; at the face centre all four sites weigh 1/4; a
    sharp kernel picks the nearest site.  Sites (+-1/3, +-1/3) R in the
    (e1, e2) frame, site-major (k = 0: (-,-), 1: (+,-), 2: (-,+), 3: (+,+))."""
    rng = np.random.default_rng(81)
    tex = rng.normal(0, 0.2, 12)
    o_down, d_down = np.array([0.3, -0.35, 5.0]), np.array([0.0, 0.0, -1.0])
    # zero texture
    c = oracle.Oracle(face_scene(np.zeros(12))).cell_colour(0, o_down, d_down, 5.0, 5.5)
    np.testing.assert_allclose(c, [0.1, 0.2, 0.3], atol=1e-15)
    # equal site values
    v = np.array([0.05, -0.1, 0.2])
    c = oracle.Oracle(face_scene(np.tile(v, 4))).cell_colour(0, o_down, d_down, 5.0, 5.5)
    np.testing.assert_allclose(c, [0.15, 0.1, 0.5], atol=1e-14)
    # face centre: ray straight down the axis, entry at the face
    orc = oracle.Oracle(face_scene(tex))
    segs = orc.ray_segments([0, 0, 5.0], d_down)
    assert segs[0][3] == ACT_DIPOLE
    c = orc.cell_colour(0, [0, 0, 5.0], d_down, segs[0][1], segs[0][2])
    np.testing.assert_allclose(c, [0.1, 0.2, 0.3] + tex.reshape(4, 3).mean(0), atol=1e-14)
    # sharp kernel: nearest site to u = (0.3, -0.35) is k = 1
    sharp = oracle.Oracle(face_scene(tex), kappa=400.0)
    segs = sharp.ray_segments(o_down, d_down)
    c = sharp.cell_colour(0, o_down, d_down, segs[0][1], segs[0][2])
    np.testing.assert_allclose(c, [0.1, 0.2, 0.3] + tex[3:6], atol=1e-12)
    # the same face point seen from below (exit through the face)
    segs = sharp.ray_segments([0.3, -0.35, -5.0], [0, 0, 1.0])
    assert segs[0][4] == ACT_DIPOLE
    c2 = sharp.cell_colour(0, [0.3, -0.35, -5.0], [0, 0, 1.0], segs[0][1], segs[0][2])
    np.testing.assert_allclose(c2, c, atol=1e-14)


# -------------------------------------------------------------------- marching

def march(sc, o, d, h, tmax):
    """Midpoint marching with point classification only (the plain
    definition of the cells); texture-free colours."""
    T = 1.0
    C = np.zeros(3)
    P = np.asarray(sc.pos, np.float64)
    for k in range(int(tmax / h)):
        x = o + (k + 0.5) * h * d
        i, ins = classify(sc, x)
        if not ins:
            continue
        a = 1 - math.exp(-float(sc.sigma[i]) * h)
        C += T * a * np.asarray(sc.rgb[i], np.float64)
        T *= 1 - a
    return C, T


def test_compositing_matches_marching_on_ten_cells():
    """Sec. 3.1: the segment sum equals the volume rendering integral; a
    fine march with point-wise cell classification converges to it."""
    rng = np.random.default_rng(91)
    sc = cluster_scene(rng, n=10, spread=0.12)
    orc = oracle.Oracle(sc)
    for _ in range(4):
        o = random_dirs(rng, 1)[0] * 0.9
        d = -o / 0.9 + rng.normal(0, 0.05, 3)
        d /= np.linalg.norm(d)
        c_ref, T_ref = orc.render_rays(o[None], d[None])
        errs = []
        for h in (4e-3, 1e-3, 2.5e-4):
            c, T = march(sc, o, d, h, 2.0)
            errs.append(max(abs(T - T_ref[0]), np.max(np.abs(c - c_ref[0]))))
        assert errs[-1] < 2e-3
        assert errs[-1] <= errs[0] + 1e-12


# ------------------------------------------------------------------ gradients

def richardson_central(flat, j, h, loss):
    """d loss / d flat[j] by FP64 central differences at steps h and h/2,
    combined by Richardson extrapolation, (4 D(h/2) - D(h)) / 3, which
    cancels the h^2 term of the central difference's error.  flat[j] is
    restored."""
    old = flat[j]

    def central(step):
        flat[j] = old + step
        lp = loss()
        flat[j] = old - step
        lm = loss()
        flat[j] = old
        return (lp - lm) / (2 * step)
    return (4.0 * central(0.5 * h) - central(h)) / 3.0

def fd_scene(seed):
    rng = np.random.default_rng(seed)
    return cluster_scene(rng, n=9, spread=0.12, r=(0.06, 0.12), tex_std=0.2)


@pytest.mark.parametrize("seed", [101, 102])
def test_adjoint_matches_central_differences(seed):
    """The hand adjoint equals FP64 central differences of the forward for
    every parameter group, on a scene where cells clip each other."""
    sc = fd_scene(seed)
    cam = cam_at([0.55, 0.25, 0.15], 10, 10, fov=40.0)
    orc = oracle.Oracle(sc)
    rng = np.random.default_rng(seed + 1)
    npix = cam.width * cam.height
    gC = rng.normal(size=(npix, 3))
    gT = rng.normal(size=npix)
    G = orc.render_grad(cam, gC, gT)

    def loss():
        c, T = orc.render(cam)
        return float(np.sum(c * gC) + np.sum(T * gT))

    scale = {"pos": 1e-3, "w": 1e-4, "R": 1e-3, "sigma": 1e-3, "rgb": 1e-3, "normal": 1e-3,
             "offset": 1e-3, "tex": 1e-3}
    checked = 0
    for key, arr in orc.params.items():
        g = G[key]
        flat = arr.reshape(-1)
        gflat = np.asarray(g).reshape(-1)
        nz = np.nonzero(np.abs(gflat) > 1e-8)[0]
        assert nz.size > 0, key
        for j in rng.choice(nz, size=min(6, nz.size), replace=False):
            h = scale[key] * 1e-3
            fd = richardson_central(flat, j, h, loss)
            assert abs(fd - gflat[j]) <= 1e-6 * max(1.0, abs(fd)), (key, j, fd, gflat[j])
            checked += 1
    assert checked >= 40


def test_gradient_of_zero_upstream_is_zero():
    sc = fd_scene(103)
    cam = cam_at([0.55, 0.25, 0.15], 6, 6)
    G = oracle.Oracle(sc).render_grad(cam, np.zeros((36, 3)), np.zeros(36))
    assert all(np.all(v == 0) for v in G.values())


# -------------------------------------------------------------------- binning

def test_binning_is_conservative_and_keys_ordered(tiny):
    """Every pixel whose ray meets a cell's ball (t >= 0) lies in a tile of
    that cell's rectangle; keys order cells by pow(o, p_i)."""
    sc, cam = tiny
    orc = oracle.Oracle(sc)
    rect, key = orc.bin(cam)
    P = np.asarray(sc.pos, np.float64)
    R = np.asarray(sc.R, np.float64)
    us, vs = np.meshgrid(np.arange(cam.width), np.arange(cam.height))
    dirs = []
    for u, v in zip(us.ravel(), vs.ravel()):
        dirs.append(orc.ray(cam, u, v)[1])
    D = np.array(dirs)
    o = np.asarray(cam.origin, np.float64)
    m = o - P                                          # [N,3]
    b = D @ m.T                                        # [px, N]
    c = np.sum(m * m, 1) - R * R
    disc = b * b - c[None, :]
    hit = (disc > 0) & (-b + np.sqrt(np.maximum(disc, 0)) > 0)
    px, cell = np.nonzero(hit)
    tx = us.ravel()[px] // 16
    ty = vs.ravel()[px] // 16
    r = rect[cell]
    assert np.all((r[:, 0] <= tx) & (tx <= r[:, 2]) & (r[:, 1] <= ty) & (ty <= r[:, 3]))
    pw = np.sum((P - o) ** 2, 1) - np.asarray(sc.w, np.float64)
    assert np.array_equal(np.argsort(key, kind="stable"), np.argsort(pw, kind="stable"))


def test_tile_lists_equal_a_per_tile_brute_force():
    """The CPU tile lists (CSR, sorted per tile by (key, cell)), the
    reference of the bit-exact GPU binning tests, against a plain loop over
    tiles and cells: rectangles of every size, empty ones, ones on the grid
    border, and keys with many ties."""
    rng = np.random.default_rng(11)
    tx, ty, n = 7, 5, 300
    x0 = rng.integers(0, tx, n)
    y0 = rng.integers(0, ty, n)
    x1 = np.minimum(x0 + rng.integers(-1, 4, n), tx - 1)   # -1: an empty rectangle
    y1 = np.minimum(y0 + rng.integers(-1, 3, n), ty - 1)
    rect = np.stack([x0, y0, x1, y1], 1).astype(np.int32)
    key = rng.integers(0, 40, n).astype(np.uint64) << np.uint64(40)    # ties among the keys
    start, cells = oracle.tile_lists(rect, key, tx, ty)
    assert start[0] == 0 and start[-1] == cells.size and start.size == tx * ty + 1
    for t in range(tx * ty):
        u, v = t % tx, t // tx
        want = [i for i in range(n) if x0[i] <= u <= x1[i] and y0[i] <= v <= y1[i]]
        want.sort(key=lambda i: (int(key[i]), i))
        assert cells[start[t]:start[t + 1]].tolist() == want, t


def test_binning_rect_is_tight():
    """For a sphere in front of the camera the rectangle is the tile cover
    of its projected extent: sampled silhouette points reach every edge."""
    from paper_2604_24994_gb300.inputs import look_at
    rng = np.random.default_rng(7)
    cam = look_at([3.0, 0.5, 0.2], 320, 240)
    n = 200
    pos = rng.uniform(-0.8, 0.8, (n, 3))
    R = rng.uniform(0.02, 0.3, n)
    sc = make_scene(pos, R * R, R)
    rect, _ = oracle.Oracle(sc).bin(cam)
    sph = random_dirs(rng, 20000)
    Mr = np.asarray(cam.rot)
    for i in range(n):
        pts = pos[i] + R[i] * sph
        xc = (pts - cam.origin) @ Mr.T
        u = cam.fx * xc[:, 0] / xc[:, 2] + cam.cx
        v = cam.fy * xc[:, 1] / xc[:, 2] + cam.cy
        pu = np.ceil(u.min() - 0.5), np.floor(u.max() - 0.5)
        pv = np.ceil(v.min() - 0.5), np.floor(v.max() - 0.5)
        lo = np.array([max(pu[0], 0), max(pv[0], 0)])
        hi = np.array([min(pu[1], cam.width - 1), min(pv[1], cam.height - 1)])
        if np.any(lo > hi):
            continue
        # sampled extent inside the rect, and the rect at most one pixel row/column wider
        assert rect[i, 0] <= lo[0] // 16 and rect[i, 2] >= hi[0] // 16
        assert rect[i, 1] <= lo[1] // 16 and rect[i, 3] >= hi[1] // 16
        assert rect[i, 0] >= (lo[0] - 2) // 16 and rect[i, 2] <= (hi[0] + 2) // 16
        assert rect[i, 1] >= (lo[1] - 2) // 16 and rect[i, 3] <= (hi[1] + 2) // 16


# ------------------------------------------ per-cell contributions (Sec. 4)

def test_contributions_telescope_to_one_minus_T(tiny):
    """Per ray, sum_k T_k alpha_k = 1 - T_final (the product telescopes), so
    the per-cell L_sparse terms sum to sum over pixels of (1 - T); the
    L_normal terms lie between 0 and the L_sparse ones."""
    sc, cam = tiny
    orc = oracle.Oracle(sc)
    sp, nm = orc.contrib(cam)
    _, T = orc.render(cam)
    assert sp.sum() == pytest.approx((1 - T).sum(), rel=1e-12)
    assert np.all(nm >= 0) and np.all(nm <= sp * (1 + 1e-12))
    assert (sp > 0).sum() > 100


def test_contributions_of_an_isolated_cell_closed_form():
    """One cell, no neighbours, face outside the ball: each pixel adds
    w = 1 - exp(-sigma chord) to L_sparse, chord = 2 sqrt(R^2 - b^2) with b
    the ray's distance to the site, and w max(nh.d, 0)^2 to L_normal.
    Flipping the normal (the face stays outside the ball, so nothing else
    changes) moves the dot product to the other side: the two L_normal sum
    to sum w (nh.d)^2."""
    R, sig = 0.3, 2.0
    nrm = np.array([0.3, -0.5, 0.8])
    cam = cam_at((0.4, -2.0, 0.3), 24, 20, 30.0)
    orc = oracle.Oracle(make_scene([0, 0, 0], 0.04, R, sig, normal=nrm))
    sp, nm = orc.contrib(cam)
    nh = nrm / np.linalg.norm(nrm)
    ws, wn, wq = 0.0, 0.0, 0.0
    for v in range(cam.height):
        for u in range(cam.width):
            o, d = orc.ray(cam, u, v)
            tc = -np.dot(o, d)                      # closest approach to the site at the origin
            b2 = np.dot(o + tc * d, o + tc * d)
            if b2 >= R * R:
                continue
            half = math.sqrt(R * R - b2)
            ta, tb = max(tc - half, 0.0), tc + half
            if tb <= ta:
                continue
            w = 1 - math.exp(-sig * (tb - ta))
            nd = float(np.dot(nh, d))
            ws += w
            wn += w * max(nd, 0.0) ** 2
            wq += w * nd * nd
    assert ws > 1.0
    assert sp[0] == pytest.approx(ws, rel=1e-12)
    assert nm[0] == pytest.approx(wn, rel=1e-12)
    flipped = oracle.Oracle(make_scene([0, 0, 0], 0.04, R, sig, normal=-nrm))
    sp2, nm2 = flipped.contrib(cam)
    assert sp2[0] == pytest.approx(sp[0], rel=1e-14)
    assert nm[0] + nm2[0] == pytest.approx(wq, rel=1e-12)


# --------------------------------------- connectivity loss (Sec. 4, L_connect)

def test_connect_two_spheres_closed_form():
    """Two spheres at distance d with radii a, b: each lists the other, so
    L = 2 (a + b - d)^2 while they overlap and 0 once they do not."""
    from oracle.connect import connect
    for d, a, b in ((1.0, 0.7, 0.6), (0.5, 0.1, 0.3), (2.0, 0.5, 0.5)):
        pos = np.array([[0.0, 0.0, 0.0], [d, 0.0, 0.0]])
        loss, gp, gR = connect(pos, [a, b], [[1], [0]])
        o = max(a + b - d, 0.0)
        np.testing.assert_allclose(loss, [o * o, o * o], rtol=1e-15)
        np.testing.assert_allclose(gR, [4 * o, 4 * o], rtol=1e-15)
        # moving sphere 0 towards sphere 1 (+x) deepens the overlap
        np.testing.assert_allclose(gp[0], [4 * o, 0, 0], rtol=1e-15, atol=0)
        np.testing.assert_allclose(gp[1], [-4 * o, 0, 0], rtol=1e-15, atol=0)


def test_connect_gradient_matches_central_differences():
    from oracle.connect import connect
    rng = np.random.default_rng(5)
    n = 12
    pos = rng.uniform(-0.5, 0.5, (n, 3))
    R = rng.uniform(0.2, 0.5, n)
    nbr = np.array([[j for j in range(n) if j != i][:6] for i in range(n)])
    _, gp, gR = connect(pos, R, nbr)
    h = 1e-6
    for i in range(n):
        for c in range(3):
            p1, p2 = pos.copy(), pos.copy()
            p1[i, c] += h
            p2[i, c] -= h
            fd = (connect(p1, R, nbr)[0].sum() - connect(p2, R, nbr)[0].sum()) / (2 * h)
            assert fd == pytest.approx(gp[i, c], rel=1e-6, abs=1e-9)
        r1, r2 = R.copy(), R.copy()
        r1[i] += h
        r2[i] -= h
        fd = (connect(pos, r1, nbr)[0].sum() - connect(pos, r2, nbr)[0].sum()) / (2 * h)
        assert fd == pytest.approx(gR[i], rel=1e-6, abs=1e-9)


# ------------------------------------------------------------ neighbour lists

def _lattice(m, h):
    g = np.stack(np.meshgrid(*[np.arange(m)] * 3, indexing="ij"), -1).reshape(-1, 3)
    return (g * h).astype(np.float32), g


def test_neighbours_on_a_lattice_closed_form():
    """Equal weights: the radical plane is the bisector, t_ij = |p_j - p_i|/2
    (Sec. 3.2 with w_i = w_j).  On a cubic lattice of step h the centre's
    nearest planes are its 6 face neighbours (h/2), then 12 edge neighbours
    (h/sqrt 2), then 8 corners (h sqrt(3)/2); equal values go by index and
    R is clipped to the next shell."""
    h = 0.125
    pos, g = _lattice(5, h)
    n = len(pos)
    w = np.full(n, 0.01, np.float32)
    R = np.full(n, 0.3, np.float32)
    c = int(np.nonzero((g == 2).all(1))[0][0])
    off = np.abs(g - 2).sum(1)
    cheb = np.abs(g - 2).max(1)
    faces = np.sort(np.nonzero((off == 1))[0])
    edges = np.sort(np.nonzero((off == 2) & (cheb == 1))[0])
    for k, want, next_t in ((6, faces, h / math.sqrt(2)), (18, np.concatenate([faces, edges]),
                                                           h * math.sqrt(3) / 2)):
        nbr, Ro = oracle.neighbours(pos, w, R, k, cells=[c])
        assert list(nbr[0]) == list(want)
        # the clipped radius is the next shell's distance, rounded down to float
        assert Ro[0] <= next_t and next_t - Ro[0] < 1e-7
    # K beyond the shells that fit under R: no clip
    nbr, Ro = oracle.neighbours(pos, w, np.full(n, 0.05, np.float32), 6, cells=[c])
    assert Ro[0] == np.float32(0.05)


def test_neighbour_distance_is_where_the_power_distances_meet():
    """t_ij is the point on the ray from p_i to p_j where pow(x, i) =
    pow(x, j) (Eq. pow_dist; found here by root bracketing, not by the
    closed form): a heavier neighbour's plane moves towards p_i and comes
    first in the list."""
    from scipy.optimize import brentq
    rng = np.random.default_rng(7)
    pos = rng.uniform(-1, 1, (40, 3)).astype(np.float32)
    w = rng.uniform(0.0, 0.2, 40).astype(np.float32)
    R = np.full(40, 10.0, np.float32)
    nbr, _ = oracle.neighbours(pos, w, R, 39, cells=[0])
    P = pos.astype(np.float64)
    W = w.astype(np.float64)

    def t_root(j):
        a = P[j] - P[0]
        L = np.linalg.norm(a)
        u = a / L
        f = lambda s: (s * s - W[0]) - (np.sum((P[0] + s * u - P[j]) ** 2) - W[j])
        return brentq(f, -10.0, 10.0, xtol=1e-15, rtol=1e-15)

    ts = np.array([t_root(j) for j in nbr[0]])
    assert (np.diff(ts) > -1e-12).all()
    assert sorted(nbr[0]) == list(range(1, 40))


def test_neighbours_match_the_input_generators_kd_tree_build():
    """The brute-force oracle and the input module's KD-tree builder (a
    different search: Euclidean candidates plus a per-weight-group radius)
    give the same lists and radii on uniform and capture-shaped sites."""
    from paper_2604_24994_gb300 import inputs
    rng = np.random.default_rng(3)
    for pos, r, k in ((rng.uniform(-1, 1, (3000, 3)), rng.uniform(0.02, 0.08, 3000), 16),
                      (None, None, 32)):
        if pos is None:
            sc = inputs.capture_scene(3000, seed=4, K=4)
            pos, r = sc.pos.astype(np.float64), np.sqrt(sc.w.astype(np.float64))
        pos = pos.astype(np.float32)
        w = (r * r).astype(np.float32)
        R = (1.5 * r).astype(np.float32)
        nb_k, R_k, ncl = inputs.build_neighbours(pos, w, R, k)
        nb_o, R_o = oracle.neighbours(pos, w, R, k)
        np.testing.assert_array_equal(nb_o, nb_k)
        np.testing.assert_array_equal(R_o.view(np.int32), R_k.view(np.int32))
        assert ncl == int((R_o != R).sum())


def test_neighbour_lists_are_complete_and_ordered():
    """Invariants at any size: every listed site's plane is no farther than
    any unlisted one, and no unlisted site's plane cuts the clipped sphere
    (t_ij >= R_i); duplicate sites have no plane and never appear."""
    rng = np.random.default_rng(11)
    pos = rng.uniform(-1, 1, (400, 3)).astype(np.float32)
    pos[300:] = pos[:100]  # 100 duplicated sites
    w = rng.uniform(0.0, 0.01, 400).astype(np.float32)
    R = np.full(400, 0.5, np.float32)
    k = 12
    nbr, Ro = oracle.neighbours(pos, w, R, k)
    P = pos.astype(np.float64)
    for i in range(400):
        a = P - P[i]
        L = np.sqrt((a * a).sum(1))
        with np.errstate(divide="ignore", invalid="ignore"):
            t = (L * L + w[i] - w.astype(np.float64)) / (2 * L)
        t[L == 0] = np.inf
        listed = nbr[i][nbr[i] >= 0]
        assert i not in listed and not (L[listed] == 0).any()
        rest = np.setdiff1d(np.nonzero(np.isfinite(t))[0], listed)
        if len(listed) and len(rest):
            assert t[listed].max() <= t[rest].min() + 1e-12
        assert (t[rest] >= Ro[i] - 1e-6).all()


def test_neighbours_degenerate_sizes():
    """One site: nothing to list, R kept.  Fewer sites than K: all of them,
    then -1, R kept.  K = 0: an empty list, R still clipped by the nearest
    plane."""
    pos = np.array([[0, 0, 0], [1, 0, 0], [0, 2, 0]], np.float32)
    w = np.zeros(3, np.float32)
    R = np.full(3, 5.0, np.float32)
    nbr, Ro = oracle.neighbours(pos[:1], w[:1], R[:1], 4)
    assert list(nbr[0]) == [-1] * 4 and Ro[0] == 5.0
    nbr, Ro = oracle.neighbours(pos, w, R, 4)
    assert list(nbr[0]) == [1, 2, -1, -1] and Ro[0] == 5.0
    nbr, Ro = oracle.neighbours(pos, w, R, 0)
    assert nbr.shape == (3, 0) and Ro[0] == np.float32(0.5) and Ro[2] == np.float32(1.0)


# ------------------------------------------------------------- fisheye rays

def test_fisheye_ray_angle_is_the_pixel_radius():
    """Equidistant fisheye (appendix D's non-pinhole rasterization): the
    ray's angle from the optical axis equals the pixel's distance from the
    principal point over f (measured with arccos, not the sine/cosine the
    oracle builds the ray from), its azimuth follows the pixel offset, and
    pixels beyond pi have no ray."""
    from paper_2604_24994_gb300 import inputs
    cam = inputs.fisheye_look_at((3.0, 0.5, -0.2), 301, 200, fov_deg=300.0)
    orc = oracle.Oracle(make_scene([0, 0, 0], 0.01, 0.1, 1.0, [0, 0, 0]))
    rot = np.asarray(cam.rot)
    rng = np.random.default_rng(1)
    n_none = 0
    for u, v in zip(rng.integers(0, 301, 200), rng.integers(0, 200, 200)):
        a = np.array([(u + 0.5 - cam.cx) / cam.fx, (v + 0.5 - cam.cy) / cam.fy])
        th = np.linalg.norm(a)
        r = orc.ray(cam, u, v)
        if th > math.pi:
            assert r is None
            n_none += 1
            continue
        o, d = r
        dc = rot @ d                          # camera axes
        assert abs(np.linalg.norm(d) - 1) < 1e-14
        assert math.acos(np.clip(dc[2], -1, 1)) == pytest.approx(th, abs=1e-7)
        if th > 1e-3:
            # the image-plane part of the direction points along the pixel offset
            assert abs(dc[0] * a[1] - dc[1] * a[0]) < 1e-12 * (1 + th)
            assert dc[0] * a[0] + dc[1] * a[1] > 0
    assert n_none > 0
    # the principal point looks down the axis
    o, d = orc.ray(cam, cam.cx - 0.5, cam.cy - 0.5)
    np.testing.assert_allclose(rot @ d, [0, 0, 1], atol=1e-15)


def test_fisheye_renders_the_same_rays_as_a_pinhole(tiny):
    """Rendering is per ray: a fisheye pixel and a pinhole pixel that see the
    same direction get the same colour and transmittance (the paper's
    lossless non-pinhole claim), and a fisheye pixel without a ray is empty
    (T = 1, black)."""
    import dataclasses
    from paper_2604_24994_gb300 import inputs
    sc, _ = tiny
    orc = oracle.Oracle(sc)
    fe = inputs.fisheye_look_at((2.2, 0.4, 0.3), 96, 96, fov_deg=120.0)
    rot = np.asarray(fe.rot)
    for (u, v) in ((48, 48), (30, 61), (80, 20), (10, 50)):
        d = rot @ orc.ray(fe, u, v)[1]       # camera axes
        f = 400.0
        ph = dataclasses.replace(fe, model=0, fx=f, fy=f, cx=0.5 - f * d[0] / d[2],
                                 cy=0.5 - f * d[1] / d[2])
        c1, T1 = orc.render(fe, pix=np.array([[u, v]]))
        c2, T2 = orc.render(ph, pix=np.array([[0, 0]]))
        np.testing.assert_allclose(c1, c2, atol=1e-10)
        np.testing.assert_allclose(T1, T2, atol=1e-10)
    wide = inputs.fisheye_look_at((2.2, 0.4, 0.3), 64, 32, fov_deg=350.0)
    c, T = orc.render(wide, pix=np.array([[0, 0], [63, 31]]))
    assert np.all(T == 1.0) and np.all(c == 0.0)


# ----------------------------------------------------- face displacement

def test_zero_displacement_is_the_base_render(tiny):
    sc, cam = tiny
    pix = np.stack(np.meshgrid(np.arange(0, 128, 7), np.arange(0, 128, 5)), -1).reshape(-1, 2)
    c0, T0 = oracle.Oracle(sc).render(cam, pix=pix)
    c1, T1 = oracle.Oracle(sc, disp=np.zeros((sc.n, 4))).render(cam, pix=pix)
    assert np.array_equal(c0, c1) and np.array_equal(T0, T1)


def test_flat_displacement_is_an_offset_shift():
    """Eq. svdisp with every site displaced by the same c: the soft-Voronoi
    weights sum to one, so the face moves by c everywhere, exactly like an
    offset of off + c, images and gradients alike (the displacement's
    gradient summed over the sites is the offset's)."""
    rng = np.random.default_rng(21)
    sc = cluster_scene(rng, n=9, spread=0.12, r=(0.06, 0.12), tex_std=0.2)
    c = rng.uniform(-0.03, 0.03, sc.n)
    cam = cam_at([0.55, 0.25, 0.15], 12, 10, fov=40.0)
    shifted = sc.copy()
    shifted.offset = sc.offset + c
    od = oracle.Oracle(sc, disp=np.repeat(c[:, None], 4, 1))
    os_ = oracle.Oracle(shifted)
    c1, T1 = od.render(cam)
    c2, T2 = os_.render(cam)
    np.testing.assert_allclose(c1, c2, atol=1e-12)
    np.testing.assert_allclose(T1, T2, atol=1e-12)
    npix = cam.width * cam.height
    gC = rng.normal(size=(npix, 3))
    gT = rng.normal(size=npix)
    G1 = od.render_grad(cam, gC, gT)
    G2 = os_.render_grad(cam, gC, gT)
    np.testing.assert_allclose(G1["disp"].sum(1), G2["offset"], atol=1e-9)
    for k in ("pos", "w", "R", "sigma", "rgb", "normal", "offset", "tex"):
        np.testing.assert_allclose(G1[k], G2[k], atol=1e-9, err_msg=k)


def test_displacement_at_the_face_centre_is_the_mean():
    """A ray along the normal through the face centre crosses the base face
    at u = 0, equidistant from the four sites at (+-1/3, +-1/3) R: by symmetry
    each weighs 1/4, the face moves by the mean displacement, and the dense
    segment of an isolated cell runs from the sphere to that height."""
    R, sig, off = 0.5, 3.0, 0.1
    disp = np.array([[0.05, -0.02, 0.07, 0.0]])
    sc = make_scene([0, 0, 0], 0.04, R, sig, [0.3, 0.6, 0.9], normal=[0, 0, 1], offset=off)
    orc = oracle.Oracle(sc, disp=disp)
    c, T = orc.render_rays(np.array([[0.0, 0.0, -3.0]]), np.array([[0.0, 0.0, 1.0]]))
    length = (off + disp.mean()) - (-R)
    assert T[0] == pytest.approx(math.exp(-sig * length), rel=1e-13)
    segs = orc.ray_segments([0.0, 0, -3.0], [0.0, 0, 1.0])
    assert segs[0][2] == pytest.approx(3.0 + off + disp.mean(), abs=1e-14)
    assert segs[0][4] == ACT_DIPOLE


@pytest.mark.parametrize("seed", [111, 112])
def test_displacement_adjoint_matches_central_differences(seed):
    """The adjoint with displacement (Eq. svdisp: the face end moves with
    delta, delta with the site displacements and with u at the base
    crossing) equals FP64 central differences for every parameter group."""
    sc = fd_scene(seed)
    rng = np.random.default_rng(seed + 7)
    disp = rng.uniform(-0.04, 0.04, (sc.n, 4))
    cam = cam_at([0.55, 0.25, 0.15], 10, 10, fov=40.0)
    orc = oracle.Oracle(sc, disp=disp)
    npix = cam.width * cam.height
    gC = rng.normal(size=(npix, 3))
    gT = rng.normal(size=npix)
    G = orc.render_grad(cam, gC, gT)

    def loss():
        c, T = orc.render(cam)
        return float(np.sum(c * gC) + np.sum(T * gT))

    scale = {"pos": 1e-3, "w": 1e-4, "R": 1e-3, "sigma": 1e-3, "rgb": 1e-3, "normal": 1e-3,
             "offset": 1e-3, "tex": 1e-3, "disp": 1e-3}
    checked = 0
    for key, arr in orc.params.items():
        flat = arr.reshape(-1)
        gflat = np.asarray(G[key]).reshape(-1)
        nz = np.nonzero(np.abs(gflat) > 1e-8)[0]
        assert nz.size > 0, key
        for j in rng.choice(nz, size=min(6, nz.size), replace=False):
            h = scale[key] * 1e-3
            fd = richardson_central(flat, j, h, loss)
            assert abs(fd - gflat[j]) <= 1e-6 * max(1.0, abs(fd)), (key, j, fd, gflat[j])
            checked += 1
    assert checked >= 45


# ------------------------------------------------------- learned detail sites

def default_sites(n):
    return np.tile(np.array([[-1, -1], [1, -1], [-1, 1], [1, 1]], np.float64) / 3.0, (n, 1, 1))


def test_explicit_default_sites_are_the_fixed_ones(tiny):
    sc, cam = tiny
    pix = np.stack(np.meshgrid(np.arange(0, 128, 9), np.arange(0, 128, 7)), -1).reshape(-1, 2)
    disp = np.random.default_rng(2).uniform(-0.01, 0.01, (sc.n, 4))
    a = oracle.Oracle(sc, disp=disp)
    b = oracle.Oracle(sc, disp=disp, sites=default_sites(sc.n))
    ca, Ta = a.render(cam, pix=pix)
    cb, Tb = b.render(cam, pix=pix)
    assert np.array_equal(ca, cb) and np.array_equal(Ta, Tb)


def test_sites_around_the_crossing_weigh_equally():
    """Sec. 3.4 with learned sites: four sites placed symmetrically around
    the point where the ray crosses the face weigh 1/4 each, so the colour is
    the base colour plus the mean site colour and the face moves by the mean
    displacement, wherever the crossing lies on the face."""
    R, sig, off = 0.5, 3.0, 0.1
    rgb = np.array([0.2, 0.3, 0.4])
    tex = np.random.default_rng(5).uniform(-0.2, 0.2, 12)
    disp = np.array([[0.04, -0.01, 0.02, 0.03]])
    sc = make_scene([0, 0, 0], 0.04, R, sig, rgb, normal=[0, 0, 1], offset=off, tex=tex)
    x0, y0 = 0.12, -0.07                                  # the ray's crossing, world units
    c0 = np.array([x0, y0]) / R                           # in face units (e1 = x, e2 = y for n = z)
    a = 0.21
    sites = (c0 + a * np.array([[-1, -1], [1, -1], [-1, 1], [1, 1]]))[None]
    orc = oracle.Oracle(sc, disp=disp, sites=sites)
    c, T = orc.render_rays(np.array([[x0, y0, -3.0]]), np.array([[0.0, 0.0, 1.0]]))
    length = (off + disp.mean()) - (-math.sqrt(R * R - x0 * x0 - y0 * y0))
    alpha = 1 - math.exp(-sig * length)
    assert T[0] == pytest.approx(1 - alpha, rel=1e-13)
    np.testing.assert_allclose(c[0], alpha * (rgb + tex.reshape(4, 3).mean(0)), atol=1e-13)


@pytest.mark.parametrize("seed", [121, 122])
def test_site_adjoint_matches_central_differences(seed):
    """Gradients for learned site positions (through the texture weights and
    the displacement weights) equal FP64 central differences, with every
    other parameter group checked again alongside."""
    sc = fd_scene(seed)
    rng = np.random.default_rng(seed + 3)
    disp = rng.uniform(-0.04, 0.04, (sc.n, 4))
    sites = default_sites(sc.n) + rng.uniform(-0.15, 0.15, (sc.n, 4, 2))
    cam = cam_at([0.55, 0.25, 0.15], 10, 10, fov=40.0)
    orc = oracle.Oracle(sc, disp=disp, sites=sites)
    npix = cam.width * cam.height
    gC = rng.normal(size=(npix, 3))
    gT = rng.normal(size=npix)
    G = orc.render_grad(cam, gC, gT)

    def loss():
        c, T = orc.render(cam)
        return float(np.sum(c * gC) + np.sum(T * gT))

    scale = {"pos": 1e-3, "w": 1e-4, "R": 1e-3, "sigma": 1e-3, "rgb": 1e-3, "normal": 1e-3,
             "offset": 1e-3, "tex": 1e-3, "disp": 1e-3, "sites": 1e-3}
    checked = 0
    for key, arr in orc.params.items():
        flat = arr.reshape(-1)
        gflat = np.asarray(G[key]).reshape(-1)
        nz = np.nonzero(np.abs(gflat) > 1e-8)[0]
        assert nz.size > 0, key
        for j in rng.choice(nz, size=min(6 if key != "sites" else 12, nz.size), replace=False):
            h = scale[key] * 1e-3
            fd = richardson_central(flat, j, h, loss)
            assert abs(fd - gflat[j]) <= 1e-6 * max(1.0, abs(fd)), (key, j, fd, gflat[j])
            checked += 1
    assert checked >= 55


# ------------------------------------------- spherical-Voronoi site colours

def sv_from_tex(tex, rng):
    """Eight random axes per site, every colour equal to the site's tex colour."""
    n = tex.shape[0]
    axes = rng.normal(size=(n, 4, 8, 3))
    cols = np.repeat(tex.reshape(n, 4, 1, 3), 8, axis=2)
    return np.concatenate([axes, cols], -1)


def test_flat_spherical_voronoi_is_the_constant_colour():
    """A site whose eight spherical-Voronoi colours are all equal has that
    colour from every direction: the image and every gradient equal the
    constant-colour render's, and the colour gradients summed over the eight
    axes equal the tex gradient."""
    rng = np.random.default_rng(41)
    sc = cluster_scene(rng, n=9, spread=0.12, r=(0.06, 0.12), tex_std=0.2)
    sv = sv_from_tex(sc.tex, rng)
    cam = cam_at([0.55, 0.25, 0.15], 12, 10, fov=40.0)
    a = oracle.Oracle(sc)
    b = oracle.Oracle(sc, sv=sv)
    c1, T1 = a.render(cam)
    c2, T2 = b.render(cam)
    np.testing.assert_allclose(c2, c1, atol=1e-12)
    np.testing.assert_allclose(T2, T1, atol=1e-15)
    npix = cam.width * cam.height
    gC = rng.normal(size=(npix, 3))
    gT = rng.normal(size=npix)
    Ga = a.render_grad(cam, gC, gT)
    Gb = b.render_grad(cam, gC, gT)
    for k in ("pos", "w", "R", "sigma", "rgb", "normal", "offset"):
        np.testing.assert_allclose(Gb[k], Ga[k], atol=1e-9, err_msg=k)
    np.testing.assert_allclose(Gb["sv"][..., 3:].sum(2).reshape(sc.n, 12), Ga["tex"], atol=1e-9)
    np.testing.assert_allclose(Gb["sv"][..., :3], 0.0, atol=1e-9)   # no direction dependence to learn


def test_spherical_voronoi_closed_form_along_the_axis():
    """A ray along +z leaves towards -z.  A site whose axes are +-x, +-y, +-z
    and two more in the xy-plane weighs them by softmax(lambda a.wo):
    e^lambda for -z, e^-lambda for +z, 1 for the six others (axes need not be
    unit: they are normalised).  Through the face centre the four sites weigh
    1/4 each."""
    R, sig, off, lam = 0.5, 2.0, 0.1, 3.0
    sc = make_scene([0, 0, 0], 0.04, R, sig, [0.1, 0.2, 0.3], normal=[0, 0, 1], offset=off)
    axes = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1],
                     [1, 1, 0], [-1, 1, 0]], np.float64) * 2.0
    rng = np.random.default_rng(3)
    cols = rng.uniform(0, 1, (4, 8, 3))
    sv = np.concatenate([np.broadcast_to(axes, (4, 8, 3)), cols], -1)[None]
    orc = oracle.Oracle(sc, sv=sv, sv_lambda=lam)
    c, T = orc.render_rays(np.array([[0.0, 0.0, -3.0]]), np.array([[0.0, 0.0, 1.0]]))
    wgt = np.ones(8)
    wgt[5] = math.exp(lam)
    wgt[4] = math.exp(-lam)
    wgt /= wgt.sum()
    site_cols = (wgt[None, :, None] * cols).sum(1)          # [4, 3]
    alpha = 1 - math.exp(-sig * (off + R))
    np.testing.assert_allclose(c[0], alpha * (np.array([0.1, 0.2, 0.3]) + site_cols.mean(0)), atol=1e-13)


@pytest.mark.parametrize("seed", [131, 132])
def test_spherical_voronoi_adjoint_matches_central_differences(seed):
    sc = fd_scene(seed)
    rng = np.random.default_rng(seed + 5)
    sv = np.concatenate([rng.normal(size=(sc.n, 4, 8, 3)), rng.uniform(0, 1, (sc.n, 4, 8, 3))], -1)
    sites = default_sites(sc.n) + rng.uniform(-0.1, 0.1, (sc.n, 4, 2))
    cam = cam_at([0.55, 0.25, 0.15], 10, 10, fov=40.0)
    orc = oracle.Oracle(sc, sv=sv, sites=sites, sv_lambda=4.0)
    npix = cam.width * cam.height
    gC = rng.normal(size=(npix, 3))
    gT = rng.normal(size=npix)
    G = orc.render_grad(cam, gC, gT)

    def loss():
        c, T = orc.render(cam)
        return float(np.sum(c * gC) + np.sum(T * gT))

    checked = 0
    for key, arr in orc.params.items():
        if key == "tex":
            continue          # unused with view-dependent colours
        flat = arr.reshape(-1)
        gflat = np.asarray(G[key]).reshape(-1)
        nz = np.nonzero(np.abs(gflat) > 1e-8)[0]
        assert nz.size > 0, key
        for j in rng.choice(nz, size=min(16 if key == "sv" else 5, nz.size), replace=False):
            h = 1e-6 if key != "w" else 1e-7
            fd = richardson_central(flat, j, h, loss)
            assert abs(fd - gflat[j]) <= 1e-6 * max(1.0, abs(fd)), (key, j, fd, gflat[j])
            checked += 1
    assert checked >= 50


# ------------------------------------------------- contribution-loss adjoint

def test_sparse_loss_of_an_isolated_cell_closed_form():
    """One cell, one ray through its centre, face outside the ball: the
    sparse contribution is alpha = 1 - exp(-sigma 2R), so its derivative in
    sigma is 2R exp(-sigma 2R) and in R it is 2 sigma exp(-sigma 2R)."""
    R, sig = 0.3, 2.0
    sc = make_scene([0, 0, 0], 0.04, R, sig, [0.5, 0.5, 0.5])
    cam = cam_at([-2.0, 0.0, 0.0], 1, 1, fov=1.0)
    orc = oracle.Oracle(sc)
    sp, nm = orc.contrib(cam)
    assert sp[0] == pytest.approx(1 - math.exp(-sig * 2 * R), rel=1e-12)
    G = orc.contrib_grad(cam, 1.0, 0.0)
    assert G["sigma"][0] == pytest.approx(2 * R * math.exp(-sig * 2 * R), rel=1e-9)
    assert G["R"][0] == pytest.approx(2 * sig * math.exp(-sig * 2 * R), rel=1e-6)


@pytest.mark.parametrize("seed", [141, 142])
def test_contribution_adjoint_matches_central_differences(seed):
    """d/dtheta of sum_i (ws_i sparse_i + wn_i normal_i) equals FP64 central
    differences of the contributions for every parameter group (the normal
    weight reaches the normal through max(nh.d, 0)^2)."""
    sc = fd_scene(seed)
    rng = np.random.default_rng(seed + 9)
    disp = rng.uniform(-0.03, 0.03, (sc.n, 4))
    cam = cam_at([0.55, 0.25, 0.15], 10, 10, fov=40.0)
    orc = oracle.Oracle(sc, disp=disp)
    ws = rng.uniform(0.5, 1.5, sc.n)
    wn = rng.uniform(0.5, 1.5, sc.n)
    G = orc.contrib_grad(cam, ws, wn)

    def loss():
        sp, nm = orc.contrib(cam)
        return float(ws @ sp + wn @ nm)

    checked = 0
    for key, arr in orc.params.items():
        if key in ("rgb", "tex"):
            assert np.abs(G[key]).max() == 0.0      # colours do not enter the contributions
            continue
        flat = arr.reshape(-1)
        gflat = np.asarray(G[key]).reshape(-1)
        nz = np.nonzero(np.abs(gflat) > 1e-8)[0]
        assert nz.size > 0, key
        for j in rng.choice(nz, size=min(6, nz.size), replace=False):
            h = 1e-6 if key != "w" else 1e-7
            fd = richardson_central(flat, j, h, loss)
            assert abs(fd - gflat[j]) <= 1e-6 * max(1.0, abs(fd)), (key, j, fd, gflat[j])
            checked += 1
    assert checked >= 35


def test_radical_plane_contains_the_intersection_circle():
    """With R^2 = w (the sphere is the cell's bound), the radical plane of two
    overlapping spheres contains their intersection circle: a ray through a
    point of that circle leaves one cell and enters the other exactly there.
    For disjoint spheres the plane lies outside both, so each cell's segment
    is its full sphere chord."""
    r0, r1, L = 1.0, 0.8, 1.5
    x0 = (L * L + r0 * r0 - r1 * r1) / (2 * L)          # plane of the circle, from the sphere equations
    rho = math.sqrt(r0 * r0 - x0 * x0)                   # circle radius
    sc = make_scene([[0, 0, 0], [L, 0, 0]], [r0 * r0, r1 * r1], [r0, r1])
    orc = oracle.Oracle(sc)
    segs = seg_dict(orc.ray_segments([-3.0, rho, 0.0], [1.0, 0, 0]))
    assert segs[0][1] == pytest.approx(3.0 + x0, abs=1e-12)
    assert segs[1][0] == pytest.approx(3.0 + x0, abs=1e-12)
    # disjoint: full chords, the plane between them cuts neither
    sc2 = make_scene([[0, 0, 0], [2.5, 0, 0]], [r0 * r0, r1 * r1], [r0, r1])
    segs2 = seg_dict(oracle.Oracle(sc2).ray_segments([-3.0, 0.3, 0.0], [1.0, 0, 0]))
    assert segs2[0][1] - segs2[0][0] == pytest.approx(2 * math.sqrt(r0 * r0 - 0.09), abs=1e-12)
    assert segs2[1][1] - segs2[1][0] == pytest.approx(2 * math.sqrt(r1 * r1 - 0.09), abs=1e-12)


# --------------------------------------------------- eight detail sites

SITE8 = np.array([[-1, -1], [0, -1], [1, -1], [-1, 0], [1, 0], [-1, 1], [0, 1], [1, 1]], np.float64) / 3.0


def eight_site_scene(sc, tex8):
    s8 = sc.copy()
    s8.tex = tex8
    return s8


def test_eight_sites_with_duplicated_positions_reduce_to_four():
    """Eight detail sites (the paper's configuration) whose second four repeat
    the first four's positions, colours and displacements: each pair weighs
    what the single site weighed, so image and gradients equal the four-site
    scene's (the pairs' gradients summing to the single site's)."""
    rng = np.random.default_rng(51)
    sc = cluster_scene(rng, n=9, spread=0.12, r=(0.06, 0.12), tex_std=0.2)
    sites4 = default_sites(sc.n) + rng.uniform(-0.1, 0.1, (sc.n, 4, 2))
    disp4 = rng.uniform(-0.03, 0.03, (sc.n, 4))
    sc8 = eight_site_scene(sc, np.concatenate([sc.tex, sc.tex], 1))
    o4 = oracle.Oracle(sc, disp=disp4, sites=sites4)
    o8 = oracle.Oracle(sc8, disp=np.concatenate([disp4, disp4], 1), sites=np.concatenate([sites4, sites4], 1))
    assert o8.nsite == 8
    cam = cam_at([0.55, 0.25, 0.15], 12, 10, fov=40.0)
    c4, T4 = o4.render(cam)
    c8, T8 = o8.render(cam)
    np.testing.assert_allclose(c8, c4, atol=1e-12)
    np.testing.assert_allclose(T8, T4, atol=1e-13)
    npix = cam.width * cam.height
    gC = rng.normal(size=(npix, 3))
    gT = rng.normal(size=npix)
    G4 = o4.render_grad(cam, gC, gT)
    G8 = o8.render_grad(cam, gC, gT)
    for k in ("pos", "w", "R", "sigma", "rgb", "normal", "offset"):
        np.testing.assert_allclose(G8[k], G4[k], atol=1e-9, err_msg=k)
    np.testing.assert_allclose(G8["tex"][:, :12] + G8["tex"][:, 12:], G4["tex"], atol=1e-9)
    np.testing.assert_allclose(G8["disp"][:, :4] + G8["disp"][:, 4:], G4["disp"], atol=1e-9)
    np.testing.assert_allclose(G8["sites"][:, :4] + G8["sites"][:, 4:], G4["sites"], atol=1e-9)


def test_eight_fixed_sites_and_a_symmetric_ring():
    """The fixed eight sites are the 3 x 3 grid of step R/3 without its
    centre (explicit positions give the same image); eight sites on a circle
    around the ray's crossing weigh 1/8 each: the colour is the base plus the
    mean site colour and the face moves by the mean displacement."""
    rng = np.random.default_rng(52)
    sc = cluster_scene(rng, n=6, spread=0.1, r=(0.06, 0.12), tex_std=0.2)
    sc8 = eight_site_scene(sc, rng.normal(0, 0.1, (sc.n, 24)))
    cam = cam_at([0.5, 0.2, 0.1], 8, 8, fov=40.0)
    a = oracle.Oracle(sc8)
    b = oracle.Oracle(sc8, sites=np.tile(SITE8, (sc.n, 1, 1)))
    ca, Ta = a.render(cam)
    cb, Tb = b.render(cam)
    assert np.array_equal(ca, cb) and np.array_equal(Ta, Tb)
    R, sig, off = 0.5, 2.0, 0.1
    tex = rng.uniform(-0.2, 0.2, 24)
    disp = rng.uniform(-0.03, 0.03, (1, 8))
    one = make_scene([0, 0, 0], 0.04, R, sig, [0.2, 0.3, 0.4], normal=[0, 0, 1], offset=off)
    one = eight_site_scene(one, tex[None])
    x0, y0 = 0.1, 0.05
    ang = np.arange(8) * (2 * np.pi / 8) + 0.3
    ring = (np.array([x0, y0]) / R + 0.25 * np.stack([np.cos(ang), np.sin(ang)], 1))[None]
    orc = oracle.Oracle(one, disp=disp, sites=ring)
    c, T = orc.render_rays(np.array([[x0, y0, -3.0]]), np.array([[0.0, 0.0, 1.0]]))
    length = (off + disp.mean()) + math.sqrt(R * R - x0 * x0 - y0 * y0)
    alpha = 1 - math.exp(-sig * length)
    assert T[0] == pytest.approx(1 - alpha, rel=1e-12)
    np.testing.assert_allclose(c[0], alpha * (np.array([0.2, 0.3, 0.4]) + tex.reshape(8, 3).mean(0)), atol=1e-12)


def test_eight_site_adjoint_matches_central_differences():
    sc = fd_scene(153)
    rng = np.random.default_rng(154)
    sc8 = eight_site_scene(sc, rng.normal(0, 0.2, (sc.n, 24)))
    disp = rng.uniform(-0.04, 0.04, (sc.n, 8))
    sites = np.tile(SITE8, (sc.n, 1, 1)) + rng.uniform(-0.1, 0.1, (sc.n, 8, 2))
    cam = cam_at([0.55, 0.25, 0.15], 10, 10, fov=40.0)
    orc = oracle.Oracle(sc8, disp=disp, sites=sites)
    npix = cam.width * cam.height
    gC = rng.normal(size=(npix, 3))
    gT = rng.normal(size=npix)
    G = orc.render_grad(cam, gC, gT)

    def loss():
        c, T = orc.render(cam)
        return float(np.sum(c * gC) + np.sum(T * gT))

    checked = 0
    for key, arr in orc.params.items():
        flat = arr.reshape(-1)
        gflat = np.asarray(G[key]).reshape(-1)
        assert gflat.size == flat.size, key
        nz = np.nonzero(np.abs(gflat) > 1e-8)[0]
        assert nz.size > 0, key
        for j in rng.choice(nz, size=min(6, nz.size), replace=False):
            h = 1e-6 if key != "w" else 1e-7
            fd = richardson_central(flat, j, h, loss)
            assert abs(fd - gflat[j]) <= 1e-6 * max(1.0, abs(fd)), (key, j, fd, gflat[j])
            checked += 1
    assert checked >= 50


def test_displacement_beyond_the_ball_limits():
    """The dipole limits with displacement: faces pushed by +2R everywhere
    lie outside every ball, so the cells render as undipoled cells; pulled by
    -2R the dense halves miss the balls and nothing is rendered."""
    rng = np.random.default_rng(61)
    sc = cluster_scene(rng, n=9, spread=0.12, r=(0.06, 0.12), tex_std=0.2)
    sc.offset = np.zeros(sc.n)
    cam = cam_at([0.55, 0.25, 0.15], 10, 8, fov=40.0)
    up = oracle.Oracle(sc, disp=np.repeat(2 * sc.R[:, None], 4, 1))
    undipoled = sc.copy()
    undipoled.offset = 10 * sc.R
    c1, T1 = up.render(cam)
    c2, T2 = oracle.Oracle(undipoled).render(cam)
    np.testing.assert_allclose(c1, c2, atol=1e-12)
    np.testing.assert_allclose(T1, T2, atol=1e-13)
    down = oracle.Oracle(sc, disp=np.repeat(-2 * sc.R[:, None], 4, 1))
    c3, T3 = down.render(cam)
    assert np.all(T3 == 1.0) and np.all(c3 == 0.0)


def test_connect_over_the_cech_graph_and_over_lists():
    """L_connect is defined over the Cech graph (all overlapping bounding
    spheres).  Where the neighbour lists hold every overlapping pair, the
    list-based loss equals it; where they do not (K smaller than the number
    of overlaps), the list-based loss is smaller, never larger."""
    from oracle.connect import cech_lists, connect, connect_cech
    from paper_2604_24994_gb300 import inputs
    sc = inputs.uniform_scene(600, seed=9, r_range=(0.05, 0.12), K=8, box=0.5)
    full, _, _ = connect_cech(sc.pos, sc.R)
    lists, _, _ = connect(sc.pos, sc.R, sc.nbr)
    assert np.all(lists <= full + 1e-15)
    cl = cech_lists(sc.pos, sc.R)
    complete = np.array([set(c[c >= 0]) <= set(b[b >= 0]) for c, b in zip(cl, sc.nbr)])
    assert complete.any() and (~complete).any()       # this scene has both kinds of cells
    np.testing.assert_allclose(lists[complete], full[complete], rtol=1e-12, atol=0)
    assert np.all(lists[~complete] < full[~complete])


@pytest.mark.parametrize("dist,fov,seed", [(3.0, 90.0, 11), (60.0, 4.0, 12)])
def test_float_tile_box_contains_the_exact_box(dist, fov, seed):
    """The CPU binning evaluates the tile box of a sphere well in front of
    the camera in float, widened by a bound on its rounding.  Against the
    exact box (the tangent-line formula in FP64 from the same float32
    inputs) over 200k spheres, from just past the float path's Z > 2R limit
    to Z = 50 R and past the image edges: every tile of the exact box is in
    the rectangle, and the rectangle is at most one tile wider."""
    from tests.oracle_util import border_box_scene
    n = 200_000
    sc, cam = border_box_scene(dist, fov, seed, n)
    pos, R = sc.pos, sc.R
    Mr = np.asarray(cam.rot, np.float64)
    o = np.asarray(cam.origin, np.float64)
    rect, _ = oracle.Oracle(sc).bin(cam)
    d = (pos - o) @ Mr.T
    X, Y, Z = d[:, 0], d[:, 1], d[:, 2]
    sel = Z > 2.0 * R * (1 + 1e-3)
    zz = Z * Z - R * R
    sx = np.sqrt(X * X + zz)
    sy = np.sqrt(Y * Y + zz)
    box = np.stack([cam.fx * (X * Z - R * sx) / zz + cam.cx, cam.fy * (Y * Z - R * sy) / zz + cam.cy,
                    cam.fx * (X * Z + R * sx) / zz + cam.cx, cam.fy * (Y * Z + R * sy) / zz + cam.cy], 1)
    a0 = np.maximum(np.ceil(box[:, 0] - 0.5), 0)
    b0 = np.maximum(np.ceil(box[:, 1] - 0.5), 0)
    a1 = np.minimum(np.floor(box[:, 2] - 0.5), cam.width - 1)
    b1 = np.minimum(np.floor(box[:, 3] - 0.5), cam.height - 1)
    live = sel & (a0 <= a1) & (b0 <= b1)
    assert live.sum() > n // 4
    ex = np.stack([a0 // 16, b0 // 16, a1 // 16, b1 // 16], 1)[live]
    r = rect[live].astype(np.int64)
    assert np.all(r[:, 0] <= ex[:, 0]) and np.all(r[:, 1] <= ex[:, 1])
    assert np.all(r[:, 2] >= ex[:, 2]) and np.all(r[:, 3] >= ex[:, 3])
    assert np.all(r[:, 0] >= ex[:, 0] - 1) and np.all(r[:, 2] <= ex[:, 2] + 1)
    m16 = (box[live][:, [0, 2]] - 0.5) % 16.0
    assert (np.minimum(np.abs(m16 - 15.0), np.abs(m16)) < 2e-3).sum() > n // 10
