"""Small hand-built scenes for pinning the oracle (test helpers)."""
import numpy as np

from paper_2604_24994_gb300.inputs import Scene, look_at


def make_scene(pos, w, R, sigma=None, rgb=None, normal=None, offset=None, tex=None):
    pos = np.asarray(pos, np.float64).reshape(-1, 3)
    n = pos.shape[0]
    w = np.broadcast_to(np.asarray(w, np.float64), (n,)).copy()
    R = np.broadcast_to(np.asarray(R, np.float64), (n,)).copy()
    sigma = np.ones(n) if sigma is None else np.broadcast_to(np.asarray(sigma, np.float64), (n,)).copy()
    rgb = np.full((n, 3), 0.5) if rgb is None else np.asarray(rgb, np.float64).reshape(n, 3)
    if normal is None:
        normal = np.tile([0.0, 0.0, 1.0], (n, 1))
    normal = np.asarray(normal, np.float64).reshape(n, 3)
    # default: face far outside the ball, whole cell dense
    offset = (R * 10.0) if offset is None else np.broadcast_to(np.asarray(offset, np.float64), (n,)).copy()
    tex = np.zeros((n, 12)) if tex is None else np.asarray(tex, np.float64).reshape(n, 12)
    return Scene(pos=pos, w=w, R=R, sigma=sigma, rgb=rgb, normal=normal, offset=offset, tex=tex,
                 nbr=np.zeros((n, 0), np.int32))


def random_dirs(rng, n):
    d = rng.normal(size=(n, 3))
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def cluster_scene(rng, n=10, spread=0.15, r=(0.05, 0.12), bound=1.5, tied=False, equal_w=False,
                  dipole=True, tex_std=0.0):
    pos = rng.uniform(-spread, spread, (n, 3))
    rr = rng.uniform(r[0], r[1], n)
    w = rr * rr
    if equal_w:
        w = np.full(n, np.mean(w))
    R = rr if tied else bound * rr
    sigma = np.exp(rng.normal(0, 1, n))
    rgb = rng.uniform(0, 1, (n, 3))
    nrm = random_dirs(rng, n)
    off = rng.uniform(-1, 1, n) * rr if dipole else R * 10
    tex = rng.normal(0, tex_std, (n, 12)) if tex_std > 0 else np.zeros((n, 12))
    return make_scene(pos, w, R, sigma, rgb, nrm, off, tex)


def cam_at(o, w=16, h=16, fov=60.0):
    return look_at(o, w, h, fov)


def f32(scene):
    """The same scene with float32 parameters (what the CUDA path consumes;
    the oracle widens them exactly), and all-pairs neighbour lists if none."""
    s = scene.copy()
    for k in s.PARAMS:
        setattr(s, k, np.ascontiguousarray(np.asarray(getattr(s, k)), np.float32))
    if s.nbr.shape[1] == 0 and s.n > 1:
        s.nbr = np.array([[j for j in range(s.n) if j != i] for i in range(s.n)], np.int32)
    return s


def border_box_scene(dist, fov, seed, n):
    """Spheres seen by a 333x211 camera at distance `dist` (vertical field
    `fov`): camera depths Z from 0.05 to 1.5 dist, radii Z / U(2.02, 50) (the
    float tile box's domain, Z > 2R, from just past its limit), image-plane
    offsets up to 1.3x the half field; half of them placed so that the left
    (or right) edge of the exact box lies within 2e-3 px of the last (first)
    pixel centre of a tile, where an edge moved by rounding would change the
    tile.  Positions and radii are float32 values."""
    rng = np.random.default_rng(seed)
    cam = look_at([dist, 0.4, -0.3], 333, 211, fov_y_deg=fov)
    Mr = np.asarray(cam.rot, np.float64)
    o = np.asarray(cam.origin, np.float64)
    tanv = np.tan(np.radians(fov) / 2)
    Z = dist * rng.uniform(0.05, 1.5, n)
    R = Z / rng.uniform(2.02, 50.0, n)
    xy = rng.uniform(-1.3, 1.3, (n, 2)) * tanv * np.array([cam.width / cam.height, 1.0]) * Z[:, None]
    h = n // 2
    tile = rng.integers(1, cam.width // 16 - 1, h)
    left = rng.random(h) < 0.5
    target = np.where(left, 16 * tile - 0.5, 16 * tile + 0.5) + rng.uniform(-2e-3, 2e-3, h)
    kt = (target - cam.cx) / cam.fx
    Xh = kt * Z[:h]
    for _ in range(8):          # X with the tangent slope atan(kt) -+ asin(R / |(X, Z)|) equal to kt
        al = np.arcsin(R[:h] / np.hypot(Xh, Z[:h]))
        Xh = Z[:h] * np.tan(np.arctan(kt) + np.where(left, al, -al))
    xy[:h, 0] = Xh
    pc = np.stack([xy[:, 0], xy[:, 1], Z], 1)
    pos = (o + pc @ Mr).astype(np.float32).astype(np.float64)
    R = R.astype(np.float32).astype(np.float64)
    return make_scene(pos, R * R, R), cam
