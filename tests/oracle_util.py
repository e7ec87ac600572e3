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
