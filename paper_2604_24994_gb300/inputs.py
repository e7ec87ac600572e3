"""Seeded synthetic inputs: scenes of bounded power cells and pinhole cameras.

This module only draws inputs. It is shared by the CUDA path, the tests and
the FP64 CPU oracle, so it computes nothing that the renderer computes: no
ray, interval, colour or compositing arithmetic lives here.

One piece of geometry is unavoidable in an input generator for this method:
the neighbour lists.  The paper renders each cell against the radical planes
of its neighbours (Sec. 3.2, Eq. power_bisector) and builds those lists
outside the renderer (a Cech graph from collision detection).  The synthetic
workloads ask for "the K nearest sites by power distance".  Here a
neighbour j of cell i is ranked by the signed distance of the radical plane
between them from p_i,

    t_ij = (|p_j - p_i|^2 + w_i - w_j) / (2 |p_j - p_i|),

the K smallest are kept, and the bound radius is clipped to R_i <=
t_(K+1) so that no site missing from the list can cut the bounding sphere.
This makes every list complete by construction; the oracle never reads the
lists (it clips against every site), so it cannot inherit a mistake here.

Scene layout (all float32 except nbr):
    pos    [N,3]   site p_i
    w      [N]     power weight w_i = r_i^2
    R      [N]     bound radius of the cell's sphere
    sigma  [N]     density of the dense half
    rgb    [N,3]   base colour
    normal [N,3]   dipole normal n_i (any length; the renderer normalises it)
    offset [N]     dipole face offset along n_i from p_i
    tex    [N,12]  four texture sites x RGB, site-major (tex[i, 3k + c])
    nbr    [N,K]   int32 neighbour ids, sorted by t_ij, -1 padded
"""
from __future__ import annotations

import dataclasses
import itertools
import math

import numpy as np

TILE = 16


@dataclasses.dataclass
class Scene:
    pos: np.ndarray
    w: np.ndarray
    R: np.ndarray
    sigma: np.ndarray
    rgb: np.ndarray
    normal: np.ndarray
    offset: np.ndarray
    tex: np.ndarray
    nbr: np.ndarray
    n_clipped: int = 0          # cells whose R was clipped for list completeness
    # optional extended face model: displacement [N,4], learned site positions
    # [N,4,2] (units of R), view-dependent site colours [N,4,8,6]
    disp: np.ndarray | None = None
    sites: np.ndarray | None = None
    sv: np.ndarray | None = None

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])

    @property
    def k(self) -> int:
        return int(self.nbr.shape[1])

    PARAMS = ("pos", "w", "R", "sigma", "rgb", "normal", "offset", "tex")

    def params(self) -> dict:
        return {k: getattr(self, k) for k in self.PARAMS}

    def copy(self) -> "Scene":
        return Scene(**{f.name: (np.array(getattr(self, f.name), copy=True)
                                 if isinstance(getattr(self, f.name), np.ndarray)
                                 else getattr(self, f.name))
                        for f in dataclasses.fields(self)})

    FORMAT = "pf-scene-1"

    def save(self, path: str) -> None:
        """Write the scene to one uncompressed .npz file (the binary scene
        format: every array under its field name, plus `format` and
        `n_clipped`); `load_scene` reads it back unchanged."""
        arrays = {f.name: getattr(self, f.name) for f in dataclasses.fields(self)
                  if isinstance(getattr(self, f.name), np.ndarray)}
        np.savez(path, format=np.array(self.FORMAT), n_clipped=np.array(self.n_clipped, np.int64), **arrays)

    def subset_params(self, idx) -> "Scene":
        """A scene holding only cells `idx` (neighbour lists dropped)."""
        kw = {k: np.ascontiguousarray(getattr(self, k)[idx]) for k in self.PARAMS}
        return Scene(nbr=np.full((len(idx), 0), -1, np.int32), **kw)


@dataclasses.dataclass
class Camera:
    """Camera: x_cam = rot @ (x_world - origin); OpenCV axes (x right, y
    down, z forward); pixel (u, v) has its centre at (u+.5, v+.5).
    model 0: pinhole.  model 1: equidistant fisheye, the centre's offset
    ((u+.5-cx)/fx, (v+.5-cy)/fy) is the ray's angle from the optical axis
    (radians) towards that offset; beyond pi the pixel has no ray."""
    rot: np.ndarray        # [3,3] float64, world -> camera
    origin: np.ndarray     # [3] float64
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    model: int = 0

    @property
    def n_pixels(self) -> int:
        return self.width * self.height

    @property
    def tiles_x(self) -> int:
        return (self.width + TILE - 1) // TILE

    @property
    def tiles_y(self) -> int:
        return (self.height + TILE - 1) // TILE

    @property
    def n_tiles(self) -> int:
        return self.tiles_x * self.tiles_y


def load_scene(path: str) -> Scene:
    """Read a scene written by Scene.save."""
    with np.load(path, allow_pickle=False) as z:
        if str(z["format"]) != Scene.FORMAT:
            raise ValueError(f"{path}: not a {Scene.FORMAT} file")
        kw = {f.name: z[f.name] for f in dataclasses.fields(Scene) if f.name in z.files and f.name != "n_clipped"}
        return Scene(n_clipped=int(z["n_clipped"]), **kw)


def look_at(origin, width: int, height: int, fov_y_deg: float = 60.0,
            target=(0.0, 0.0, 0.0), up=(0.0, 0.0, 1.0)) -> Camera:
    """Camera at `origin` looking at `target`; vertical field of view; square
    pixels; principal point at the image centre; world up +z."""
    o = np.asarray(origin, np.float64)
    fwd = np.asarray(target, np.float64) - o
    fwd /= np.linalg.norm(fwd)
    right = np.cross(fwd, np.asarray(up, np.float64))
    nr = np.linalg.norm(right)
    if nr < 1e-12:  # looking along up: pick any perpendicular
        right = np.cross(fwd, np.array([1.0, 0.0, 0.0]))
        nr = np.linalg.norm(right)
    right /= nr
    down = np.cross(fwd, right)
    rot = np.stack([right, down, fwd])
    f = 0.5 * height / math.tan(math.radians(fov_y_deg) / 2)
    return Camera(rot=rot, origin=o, fx=f, fy=f, cx=width / 2.0, cy=height / 2.0,
                  width=int(width), height=int(height))


def fisheye_look_at(origin, width: int, height: int, fov_deg: float = 180.0,
                    target=(0.0, 0.0, 0.0), up=(0.0, 0.0, 1.0)) -> Camera:
    """Equidistant fisheye at `origin` looking at `target`: the circle
    inscribed in the image spans `fov_deg`; square pixels, principal point
    at the image centre."""
    c = look_at(origin, width, height, 60.0, target, up)
    f = 0.5 * min(width, height) / math.radians(fov_deg / 2)
    return dataclasses.replace(c, fx=f, fy=f, model=1)


def ring_cameras(n_views: int, radius: float, width: int, height: int,
                 fov_y_deg: float = 60.0):
    return [look_at((radius * math.cos(2 * math.pi * k / n_views),
                     radius * math.sin(2 * math.pi * k / n_views), 0.0),
                    width, height, fov_y_deg) for k in range(n_views)]


def random_sphere_cameras(rng, n: int, rmin: float, rmax: float, sizes, probs,
                          fov_y_deg: float = 60.0):
    """Cameras on spheres of random radius in [rmin, rmax] looking at the
    origin, with resolutions drawn from `sizes` with probabilities `probs`."""
    cams = []
    sidx = rng.choice(len(sizes), size=n, p=probs)
    dirs = rng.normal(size=(n, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    rad = rng.uniform(rmin, rmax, n)
    for i in range(n):
        w, h = sizes[sidx[i]]
        cams.append(look_at(dirs[i] * rad[i], w, h, fov_y_deg))
    return cams


# ----------------------------------------------------------------------------
# attributes and neighbour lists


def _attributes(rng, n: int, r: np.ndarray) -> dict:
    sigma = np.exp(rng.normal(0.0, 1.0, n))
    rgb = rng.uniform(0.0, 1.0, (n, 3))
    nrm = rng.normal(size=(n, 3))
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    offset = rng.uniform(-1.0, 1.0, n) * r
    tex = rng.normal(0.0, 0.1, (n, 12))
    f = np.float32
    return dict(sigma=sigma.astype(f), rgb=rgb.astype(f), normal=nrm.astype(f),
                offset=offset.astype(f), tex=tex.astype(f))


def _plane_dist(pi, wi, pj, wj):
    a = pj - pi
    L2 = np.einsum("...k,...k->...", a, a)
    L = np.sqrt(L2)
    with np.errstate(divide="ignore", invalid="ignore"):
        t = (L2 + wi - wj) / (2.0 * L)
    return np.where(L > 0, t, np.inf), L


def build_neighbours(pos: np.ndarray, w: np.ndarray, R: np.ndarray, K: int,
                     workers: int = -1, n_groups: int = 16):
    """Rank neighbours by radical-plane distance, keep K, clip R for
    completeness.  Returns (nbr int32 [N,K], R_clipped float32, n_clipped).

    Exact: the K+1 smallest t_ij over all sites.  Candidates are the
    Euclidean nearest sites; then, per group of sites of similar weight
    (largest weight W_g), every site closer than
        tau_i + sqrt(tau_i^2 - w_i + W_g)
    is added, where tau_i is the (K+1)-th smallest t among the first
    candidates (a site j with t_ij < tau_i must lie inside that radius)."""
    from scipy.spatial import cKDTree

    N = pos.shape[0]
    P = pos.astype(np.float64)
    W = w.astype(np.float64)
    Rn = R.astype(np.float64).copy()
    nbr = np.full((N, K), -1, np.int32)
    if N <= 1 or K == 0:
        return nbr, R.astype(np.float32), 0
    kq = min(N, K + 9)
    tree = cKDTree(P)
    best_t = np.full((N, K + 1), np.inf)
    best_j = np.full((N, K + 1), -1, np.int64)
    dmax = np.zeros(N)
    CH = 250_000
    for s0 in range(0, N, CH):
        idx = np.arange(s0, min(N, s0 + CH))
        dist, js = tree.query(P[idx], k=kq, workers=workers)
        dist = dist.reshape(len(idx), kq)
        js = js.reshape(len(idx), kq)
        t, _ = _plane_dist(P[idx][:, None, :], W[idx][:, None], P[js], W[js])
        t[js == idx[:, None]] = np.inf
        order = np.lexsort((js, t), axis=1)[:, :K + 1]
        m = min(K + 1, kq)
        best_t[idx, :m] = np.take_along_axis(t, order, 1)[:, :m]
        best_j[idx, :m] = np.take_along_axis(js, order, 1)[:, :m]
        dmax[idx] = dist[:, -1] if kq < N else np.inf
    tau = best_t[:, K]
    # weight groups, each with its own tree and largest weight
    order_w = np.argsort(W, kind="stable")
    extra_i, extra_j = [], []
    for g in np.array_split(order_w, max(1, min(n_groups, N))):
        if g.size == 0:
            continue
        Wg = float(W[g].max())
        disc = tau * tau - W + Wg
        rho = tau + np.sqrt(np.maximum(disc, 0.0))
        need = np.nonzero(np.isfinite(tau) & (disc >= 0) & (rho > dmax))[0]
        if need.size == 0:
            continue
        tg = cKDTree(P[g])
        cnt = tg.query_ball_point(P[need], rho[need], return_length=True, workers=workers)
        need = need[cnt > 0]
        if need.size == 0:
            continue
        lists = tg.query_ball_point(P[need], rho[need], workers=workers)
        lens = np.fromiter((len(l) for l in lists), np.int64, len(lists))
        flat = np.fromiter(itertools.chain.from_iterable(lists), np.int64, int(lens.sum()))
        ci = np.repeat(need, lens)
        js = g[flat]
        L = np.linalg.norm(P[js] - P[ci], axis=1)
        keep = (L > dmax[ci]) & (js != ci)
        extra_i.append(ci[keep])
        extra_j.append(js[keep])
    if extra_i and sum(a.size for a in extra_i):
        ei = np.concatenate(extra_i)
        ej = np.concatenate(extra_j)
        et, _ = _plane_dist(P[ei], W[ei], P[ej], W[ej])
        cells = np.unique(ei)
        # merge each affected cell's current best with its extra candidates
        bi = np.repeat(cells, K + 1)
        ai = np.concatenate([bi, ei])
        at = np.concatenate([best_t[cells].reshape(-1), et])
        aj = np.concatenate([best_j[cells].reshape(-1), ej])
        o = np.lexsort((aj, at, ai))
        ai, at, aj = ai[o], at[o], aj[o]
        start = np.searchsorted(ai, cells)
        rank = np.arange(ai.size) - np.repeat(start, np.diff(np.append(start, ai.size)))
        sel = rank < K + 1
        best_t[ai[sel], rank[sel]] = at[sel]
        best_j[ai[sel], rank[sel]] = aj[sel]
    nbr[:] = np.where(np.isfinite(best_t[:, :K]), best_j[:, :K], -1).astype(np.int32)
    tK1 = best_t[:, K]
    clip = tK1 < Rn
    Rn[clip] = np.maximum(tK1[clip], 0.0)
    Rf = Rn.astype(np.float32)
    # the float32 radius must not exceed t_(K+1)
    over = clip & (Rf.astype(np.float64) > np.maximum(tK1, 0.0))
    Rf[over] = np.nextafter(Rf[over], np.float32(0))
    return nbr, Rf, int(clip.sum())


# ----------------------------------------------------------------------------
# scene recipes


def uniform_scene(n: int, seed: int = 0, r_range=(0.02, 0.08), bound_factor=1.5,
                  K: int = 16, box: float = 1.0, tied: bool = False,
                  equal_weights: bool = False) -> Scene:
    """Sites uniform in [-box, box]^3, r ~ U(r_range), w = r^2, R = 1.5 r.
    `tied` sets R = r (so R^2 - w = 0 for every cell); `equal_weights` sets
    every w to the mean (power cells reduce to Voronoi cells)."""
    rng = np.random.default_rng(seed)
    pos = rng.uniform(-box, box, (n, 3))
    r = rng.uniform(r_range[0], r_range[1], n)
    attrs = _attributes(rng, n, r)
    w = r * r
    if equal_weights:
        w = np.full(n, float(np.mean(w)))
    R = r if tied else bound_factor * r
    pos = pos.astype(np.float32)
    w = w.astype(np.float32)
    nbr, Rc, ncl = build_neighbours(pos, w, R.astype(np.float32), K)
    return Scene(pos=pos, w=w, R=Rc, nbr=nbr, n_clipped=ncl, **attrs)


def capture_scene(n: int, seed: int = 0, K: int = 32, r_scale: float = 0.35,
                  bound_factor: float = 1.5, n_components: int = 64) -> Scene:
    """Shaped like an unbounded capture: 70% of sites from a Gaussian mixture
    inside the unit ball (centres uniform in the ball, component std ~
    U(0.02, 0.2), samples outside the ball redrawn), 30% on an outer shell
    with uniform directions and log-uniform radius in [1, 20].  r_i =
    r_scale * (distance to the 8th nearest site)."""
    from scipy.spatial import cKDTree

    rng = np.random.default_rng(seed)
    nin = int(0.7 * n)
    nout = n - nin
    cc = rng.normal(size=(n_components, 3))
    cc /= np.linalg.norm(cc, axis=1, keepdims=True)
    cc *= rng.uniform(0, 1, (n_components, 1)) ** (1 / 3)
    sc = rng.uniform(0.02, 0.2, n_components)
    comp = rng.integers(0, n_components, nin)
    pin = cc[comp] + rng.normal(size=(nin, 3)) * sc[comp, None]
    bad = np.linalg.norm(pin, axis=1) > 1
    while bad.any():
        k = int(bad.sum())
        q = rng.integers(0, n_components, k)
        pin[bad] = cc[q] + rng.normal(size=(k, 3)) * sc[q, None]
        bad = np.linalg.norm(pin, axis=1) > 1
    u = rng.normal(size=(nout, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    pout = u * np.exp(rng.uniform(0, math.log(20.0), nout))[:, None]
    pos = np.concatenate([pin, pout]).astype(np.float32)
    d8 = cKDTree(pos.astype(np.float64)).query(pos.astype(np.float64), k=9,
                                                workers=-1)[0][:, 8]
    r = r_scale * d8
    attrs = _attributes(rng, n, r)
    w = (r * r).astype(np.float32)
    nbr, Rc, ncl = build_neighbours(pos, w, (bound_factor * r).astype(np.float32), K)
    return Scene(pos=pos, w=w, R=Rc, nbr=nbr, n_clipped=ncl, **attrs)


def perturbed_sites(scene: Scene, std: float, seed: int = 1) -> Scene:
    """Copy with sites moved by N(0, std) (the training target of the
    forward+backward workload); everything else, lists included, is kept."""
    rng = np.random.default_rng(seed)
    s = scene.copy()
    s.pos = (scene.pos.astype(np.float64)
             + rng.normal(0.0, std, scene.pos.shape)).astype(np.float32)
    return s


# Workload recipes, named by what they are.
def tiny_scene(seed: int = 0) -> Scene:
    """2,000 cells uniform in [-1,1]^3, r ~ U(0.02, 0.08), 16 neighbours."""
    return uniform_scene(2000, seed=seed, r_range=(0.02, 0.08), K=16)


def tiny_camera() -> Camera:
    return look_at((3.0, 0.0, 0.0), 128, 128)


def train_scene(seed: int = 0) -> Scene:
    """100k cells uniform in [-1,1]^3, r ~ U(0.005, 0.02), 32 neighbours."""
    return uniform_scene(100_000, seed=seed, r_range=(0.005, 0.02), K=32)


def train_cameras(width: int = 800, height: int = 800):
    return ring_cameras(8, 3.0, width, height)


def capture_camera(width: int = 1920, height: int = 1080) -> Camera:
    return look_at((3.0, 0.0, 0.0), width, height)
