"""FP64 CPU oracle for the bounded-power-cell renderer (Power Foam, arxiv 2604.24994).

TEST INFRASTRUCTURE ONLY: only tests/, __graft_entry__.smoke() and the CPU
baseline legs of bench.py may import this package.  It shares no code with
the CUDA library; `pf_oracle.c` holds the arithmetic (see its header for the
definitions it writes out), this module builds it with gcc and calls it
through ctypes.

Optional exact prune: a cell i can only be cut by the radical plane of a
site j with |p_j - p_i| < R_i + sqrt(R_i^2 - w_i + w_j) (the plane's
distance from p_i, (|a|^2 + w_i - w_j) / (2|a|), must be below R_i).
`candidates()` gathers, per cell, every site inside that distance with
scipy's KD-tree (sites grouped by weight so each group uses its own maximum
w_j).  The C code then clips against those sites only; every other site's
plane lies outside the bounding sphere and can never bind, so pruned and
unpruned renders agree (checked by a test).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pf_oracle.c")
_LIB = os.path.join(_HERE, "liborc.so")
_lock = threading.Lock()
_lib = None

KAPPA = 6.0          # soft-Voronoi sharpness on the face, in units of 1/R
PARAM_COLS = {"pos": (0, 3), "w": (3, 1), "R": (4, 1), "sigma": (5, 1), "rgb": (6, 3),
              "normal": (9, 3), "offset": (12, 1), "tex": (13, 12), "disp": (37, 4), "sites": (45, 8),
              "sv": (61, 192)}
NPAR = 445          # the site blocks have room for eight sites
SV_LAMBDA = 10.0     # sharpness of the spherical-Voronoi site colours
ACT_SPHERE, ACT_CAMERA, ACT_DIPOLE = -1, -2, -3


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, no FMA contraction, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Scene(C.Structure):
    _fields_ = [("n", C.c_int64)] + [(k, C.POINTER(C.c_double)) for k in
                                     ("pos", "w", "R", "sigma", "rgb", "normal", "offset", "tex", "disp")] + \
               [("kappa_disp", C.c_double), ("sites", C.POINTER(C.c_double)), ("sv", C.POINTER(C.c_double)),
                ("sv_lambda", C.c_double), ("nsite", C.c_int32)]


class _Camera(C.Structure):
    _fields_ = [("rot", C.c_double * 9), ("origin", C.c_double * 3), ("fx", C.c_double),
                ("fy", C.c_double), ("cx", C.c_double), ("cy", C.c_double),
                ("width", C.c_int32), ("height", C.c_int32), ("model", C.c_int32)]


class _Cands(C.Structure):
    _fields_ = [("beg", C.POINTER(C.c_int64)), ("end", C.POINTER(C.c_int64)),
                ("idx", C.POINTER(C.c_int32))]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            P = C.POINTER
            d = C.c_double
            _lib.orc_render.argtypes = [P(_Scene), P(_Cands), P(_Camera), C.c_int64, P(C.c_int32), d,
                                        P(d), P(d), P(C.c_int32), C.c_int]
            _lib.orc_render_grad.argtypes = [P(_Scene), P(_Cands), P(_Camera), C.c_int64, P(C.c_int32), d,
                                             P(d), P(d), P(d), C.c_int]
            _lib.orc_ray_segments.argtypes = [P(_Scene), P(_Cands), P(d), P(d), C.c_int64, P(C.c_int32),
                                              P(d), P(d), P(C.c_int32), P(C.c_int32)]
            _lib.orc_ray_segments.restype = C.c_int64
            _lib.orc_cell_contrib.argtypes = [P(_Scene), P(_Cands), P(_Camera), C.c_int64, P(C.c_int32), P(d), P(d),
                                         C.c_int]
            _lib.orc_render_rays.argtypes = [P(_Scene), P(_Cands), C.c_int64, P(d), P(d), d, P(d), P(d)]
            _lib.orc_cell_colour.argtypes = [P(_Scene), C.c_int64, P(d), P(d), d, d, d, P(d)]
            _lib.orc_ray.argtypes = [P(_Camera), d, d, P(d), P(d)]
            _lib.orc_ray.restype = C.c_int
            _lib.orc_onb.argtypes = [P(d), P(d), P(d)]
            _lib.orc_hit_cells.argtypes = [P(_Scene), P(_Camera), C.c_int64, P(C.c_int32), P(C.c_uint8),
                                           C.c_int]
            _lib.orc_bin.argtypes = [P(_Camera), C.c_int64, P(d), P(d), P(d),
                                     P(C.c_int32), P(C.c_uint64)]
            f = C.c_float
            _lib.orc_contrib_grad.argtypes = [P(_Scene), P(_Cands), P(_Camera), C.c_int64, P(C.c_int32), P(d), P(d),
                                              P(d), C.c_int]
            _lib.orc_neighbours.argtypes = [P(f), P(f), P(f), C.c_int64, C.c_int32, C.c_int64, P(C.c_int64),
                                            P(C.c_int32), P(f), C.c_int]
            _lib.orc_render_tiles.argtypes = [P(_Scene), P(_Cands), P(_Camera), P(C.c_int64), P(C.c_int32),
                                              C.c_int64, P(C.c_int32), d, d, P(d), P(d), P(C.c_int32), C.c_int]
        return _lib


def neighbours(pos, w, R, k: int, cells=None, nthreads: int = 0):
    """Brute-force neighbour lists (orc_neighbours): for each cell in `cells`
    (default: all), the k sites with the smallest radical-plane distance
    t_ij (ties by j, -1 padded) and the clipped bound radius.  Returns
    (nbr int32 [m, k], R float32 [m])."""
    pos = np.ascontiguousarray(pos, np.float32)
    w = np.ascontiguousarray(w, np.float32)
    R = np.ascontiguousarray(R, np.float32)
    n = pos.shape[0]
    if cells is None:
        m, cp = n, None
    else:
        cells = np.ascontiguousarray(cells, np.int64)
        m, cp = cells.shape[0], _ptr(cells, C.c_int64)
    nbr = np.empty((m, k), np.int32)
    Ro = np.empty(m, np.float32)
    rc = lib().orc_neighbours(_ptr(pos, C.c_float), _ptr(w, C.c_float), _ptr(R, C.c_float), n, k, m, cp,
                              _ptr(nbr, C.c_int32), _ptr(Ro, C.c_float), nthreads)
    if rc != 0:
        raise ValueError("orc_neighbours: invalid k")
    return nbr, Ro


def _ptr(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def camera_struct(cam) -> _Camera:
    c = _Camera()
    c.rot[:] = [float(x) for x in np.asarray(cam.rot, np.float64).reshape(9)]
    c.origin[:] = [float(x) for x in np.asarray(cam.origin, np.float64)]
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.width, c.height = int(cam.width), int(cam.height)
    c.model = int(getattr(cam, "model", 0))
    return c


class Oracle:
    """Brute-force FP64 renderer and adjoint.  The scene's parameters are
    widened to float64 (exactly, for float32 inputs); `params` holds them and
    may be edited in place (finite differences do)."""

    def __init__(self, scene, kappa: float = KAPPA, nthreads: int = 0, disp=None, sites=None, sv=None,
                 sv_lambda: float = SV_LAMBDA):
        """`disp` [N,4] (or the scene's `disp` attribute): displacement of
        each face at its four texture sites (Eq. svdisp); None for none.
        `sites` [N,4,2] (or the scene's `sites`): learned positions of those
        sites in units of R; None for the fixed (+-1/3, +-1/3).  `sv`
        [N,4,8,6] (or the scene's `sv`): view-dependent site colours, per
        site eight (axis xyz, rgb) of a spherical-Voronoi function with
        sharpness `sv_lambda`; None for the constant colours `tex`."""
        self.kappa = float(kappa)
        self.nthreads = int(nthreads)
        self._arrs = {k: np.ascontiguousarray(np.asarray(getattr(scene, k), np.float64))
                      for k in ("pos", "w", "R", "sigma", "rgb", "normal", "offset", "tex")}
        # detail sites per face, from the texture's width: 4 (tex [N,12]) or 8 (tex [N,24])
        ns = self._arrs["tex"].shape[1] // 3 if self._arrs["tex"].ndim == 2 else 4
        if ns not in (4, 8):
            raise ValueError("tex must hold 4 or 8 RGB sites per cell")
        self.nsite = ns
        if disp is None:
            disp = getattr(scene, "disp", None)
        if disp is not None:
            self._arrs["disp"] = np.ascontiguousarray(np.asarray(disp, np.float64).reshape(-1, ns))
        if sites is None:
            sites = getattr(scene, "sites", None)
        if sites is not None:
            self._arrs["sites"] = np.ascontiguousarray(np.asarray(sites, np.float64).reshape(-1, ns, 2))
        if sv is None:
            sv = getattr(scene, "sv", None)
        if sv is not None:
            self._arrs["sv"] = np.ascontiguousarray(np.asarray(sv, np.float64).reshape(-1, ns, 8, 6))
        self.params = self._arrs
        self.n = int(self._arrs["pos"].shape[0])
        s = _Scene()
        s.n = self.n
        for k, a in self._arrs.items():
            setattr(s, k, _ptr(a, C.c_double))
        s.kappa_disp = self.kappa
        s.sv_lambda = float(sv_lambda)
        s.nsite = ns
        self._s = s
        self._cands = None      # (beg, end, idx) arrays, kept alive
        self._cs = None

    # -- exact prune ---------------------------------------------------------
    def set_candidates(self, cells=None, n_groups: int = 8):
        """Build candidate lists for `cells` (all cells if None)."""
        from scipy.spatial import cKDTree
        P = self._arrs["pos"].astype(np.float64)
        W = self._arrs["w"].astype(np.float64)
        R = self._arrs["R"].astype(np.float64)
        n = self.n
        cells = np.arange(n) if cells is None else np.asarray(cells, np.int64)
        beg = np.full(n, -1, np.int64)
        end = np.full(n, -1, np.int64)
        order = np.argsort(W, kind="stable")
        groups = np.array_split(order, max(1, min(n_groups, n)))
        trees = [(g, cKDTree(P[g]), float(W[g].max())) for g in groups if len(g)]
        per_cell = [[] for _ in range(len(cells))]
        for g, tree, wg in trees:
            disc = R[cells] ** 2 - W[cells] + wg
            ok = disc >= 0
            rad = R[cells] + np.sqrt(np.maximum(disc, 0.0))
            rad = rad * (1 + 1e-12) + 1e-12
            sel = np.nonzero(ok)[0]
            if sel.size == 0:
                continue
            res = tree.query_ball_point(P[cells[sel]], rad[sel], workers=-1)
            for q, lst in zip(sel, res):
                if lst:
                    per_cell[q].append(g[np.asarray(lst, np.int64)])
        idx_chunks = []
        off = 0
        for q, c in enumerate(cells):
            js = np.unique(np.concatenate(per_cell[q])) if per_cell[q] else np.zeros(0, np.int64)
            js = js[js != c]
            beg[c] = off
            off += js.size
            end[c] = off
            idx_chunks.append(js.astype(np.int32))
        idx = np.concatenate(idx_chunks) if idx_chunks else np.zeros(0, np.int32)
        if idx.size == 0:
            idx = np.zeros(1, np.int32)
        self._cands = (beg, end, idx)
        cs = _Cands()
        cs.beg = _ptr(beg, C.c_int64)
        cs.end = _ptr(end, C.c_int64)
        cs.idx = _ptr(idx, C.c_int32)
        self._cs = cs
        return int(off)

    def set_candidate_lists(self, lists: dict):
        """Explicit candidate lists {cell: iterable of sites}; other cells
        are clipped against every site."""
        n = self.n
        beg = np.full(n, -1, np.int64)
        end = np.full(n, -1, np.int64)
        chunks = []
        off = 0
        for c in sorted(lists):
            js = np.unique(np.asarray(list(lists[c]), np.int64))
            js = js[js != c]
            beg[c] = off
            off += js.size
            end[c] = off
            chunks.append(js.astype(np.int32))
        idx = np.concatenate(chunks) if chunks else np.zeros(0, np.int32)
        if idx.size == 0:
            idx = np.zeros(1, np.int32)
        self._cands = (beg, end, idx)
        cs = _Cands()
        cs.beg = _ptr(beg, C.c_int64)
        cs.end = _ptr(end, C.c_int64)
        cs.idx = _ptr(idx, C.c_int32)
        self._cs = cs

    def set_neighbour_lists(self, nbr):
        """Candidate lists from a neighbour array [N,K] (-1 padded): cell i
        is clipped against its K listed sites only, as the tiled renderer
        clips it."""
        nbr = np.asarray(nbr, np.int64)
        n = self.n
        valid = (nbr >= 0) & (nbr != np.arange(n)[:, None])
        cnt = valid.sum(1)
        end = np.cumsum(cnt).astype(np.int64)
        beg = (end - cnt).astype(np.int64)
        idx = nbr[valid].astype(np.int32)
        if idx.size == 0:
            idx = np.zeros(1, np.int32)
        self._cands = (beg, end, idx)
        cs = _Cands()
        cs.beg = _ptr(beg, C.c_int64)
        cs.end = _ptr(end, C.c_int64)
        cs.idx = _ptr(idx, C.c_int32)
        self._cs = cs

    def render_rays(self, o, d):
        """rgb [n,3] and T [n] for explicit rays (o [n,3], unit d [n,3])."""
        o = np.ascontiguousarray(np.asarray(o, np.float64).reshape(-1, 3))
        d = np.ascontiguousarray(np.asarray(d, np.float64).reshape(-1, 3))
        n = o.shape[0]
        rgb = np.zeros((n, 3))
        T = np.zeros(n)
        lib().orc_render_rays(C.byref(self._s), C.byref(self._cs) if self._cs else None, n,
                              _ptr(o, C.c_double), _ptr(d, C.c_double), self.kappa,
                              _ptr(rgb, C.c_double), _ptr(T, C.c_double))
        return rgb, T

    def clear_candidates(self):
        self._cands = None
        self._cs = None

    def hit_cells(self, cam, pix=None) -> np.ndarray:
        pixa, npix = self._pix(cam, pix)
        flag = np.zeros(self.n, np.uint8)
        lib().orc_hit_cells(C.byref(self._s), C.byref(camera_struct(cam)), npix,
                            _ptr(pixa, C.c_int32) if pixa is not None else None,
                            _ptr(flag, C.c_uint8), self.nthreads)
        return flag.astype(bool)

    def prune_for(self, cam, pix=None) -> int:
        """Candidate lists for the cells that these pixels' rays can meet.

        The hit test here is widened (a ray within 1e-6 relative of the
        sphere counts), and cells without a list fall back to brute force."""
        flag = self.hit_cells(cam, pix)
        return self.set_candidates(np.nonzero(flag)[0])

    # -- rendering -----------------------------------------------------------
    @staticmethod
    def _pix(cam, pix):
        if pix is None:
            return None, cam.width * cam.height
        pa = np.ascontiguousarray(np.asarray(pix, np.int32).reshape(-1, 2))
        return pa, pa.shape[0]

    def render(self, cam, pix=None, return_nseg: bool = False):
        """rgb [npix,3] and T [npix] (float64) for pixels `pix` ([npix,2] (u, v))
        or for the whole image in row-major order."""
        pixa, npix = self._pix(cam, pix)
        rgb = np.zeros((npix, 3), np.float64)
        T = np.zeros(npix, np.float64)
        nseg = np.zeros(npix, np.int32)
        lib().orc_render(C.byref(self._s), C.byref(self._cs) if self._cs else None,
                         C.byref(camera_struct(cam)), npix,
                         _ptr(pixa, C.c_int32) if pixa is not None else None, self.kappa,
                         _ptr(rgb, C.c_double), _ptr(T, C.c_double), _ptr(nseg, C.c_int32),
                         self.nthreads)
        return (rgb, T, nseg) if return_nseg else (rgb, T)

    def contrib(self, cam, pix=None):
        """Per-cell contributions [N] over the pixels (float64): sum of
        T alpha (L_sparse) and of T alpha max(nh . d, 0)^2 (L_normal)."""
        pixa, npix = self._pix(cam, pix)
        sp = np.zeros(self.n, np.float64)
        nm = np.zeros(self.n, np.float64)
        lib().orc_cell_contrib(C.byref(self._s), C.byref(self._cs) if self._cs else None, C.byref(camera_struct(cam)),
                          npix, _ptr(pixa, C.c_int32) if pixa is not None else None, _ptr(sp, C.c_double),
                          _ptr(nm, C.c_double), self.nthreads)
        return sp, nm

    def contrib_grad(self, cam, w_sparse, w_normal, pix=None) -> dict:
        """Gradient (float64 dict keyed like render_grad) of
        sum_i (w_sparse[i] sparse_i + w_normal[i] normal_i) over the pixels,
        sparse / normal the per-cell contributions of `contrib`."""
        pixa, npix = self._pix(cam, pix)
        ws = np.ascontiguousarray(np.broadcast_to(np.asarray(w_sparse, np.float64), (self.n,)))
        wn = np.ascontiguousarray(np.broadcast_to(np.asarray(w_normal, np.float64), (self.n,)))
        g = np.zeros((self.n, NPAR), np.float64)
        lib().orc_contrib_grad(C.byref(self._s), C.byref(self._cs) if self._cs else None,
                               C.byref(camera_struct(cam)), npix,
                               _ptr(pixa, C.c_int32) if pixa is not None else None, _ptr(ws, C.c_double),
                               _ptr(wn, C.c_double), _ptr(g, C.c_double), self.nthreads)
        return self._split_grad(g)

    def _split_grad(self, g) -> dict:
        out = {}
        per_site = {"tex": 3, "disp": 1, "sites": 2, "sv": 48}
        for k, (c0, w) in PARAM_COLS.items():
            if k in ("disp", "sites", "sv") and k not in self._arrs:
                continue
            if k in per_site:
                w = per_site[k] * self.nsite
            out[k] = g[:, c0:c0 + w] if w > 1 else g[:, c0].copy()
            if k == "sites":
                out[k] = out[k].reshape(-1, self.nsite, 2)
            if k == "sv":
                out[k] = out[k].reshape(-1, self.nsite, 8, 6)
            if k == "disp" and self.nsite != 4:
                out[k] = out[k].reshape(-1, self.nsite)
        return out

    def render_grad(self, cam, dL_dC, dL_dT, pix=None) -> dict:
        """dL/d(parameters) (float64 dict keyed like the scene) for upstream
        gradients dL/dC [npix,3] and dL/dT [npix] of the rendered pixels."""
        pixa, npix = self._pix(cam, pix)
        gC = np.ascontiguousarray(np.asarray(dL_dC, np.float64).reshape(npix, 3))
        gT = np.ascontiguousarray(np.asarray(dL_dT, np.float64).reshape(npix))
        g = np.zeros((self.n, NPAR), np.float64)
        lib().orc_render_grad(C.byref(self._s), C.byref(self._cs) if self._cs else None,
                              C.byref(camera_struct(cam)), npix,
                              _ptr(pixa, C.c_int32) if pixa is not None else None, self.kappa,
                              _ptr(gC, C.c_double), _ptr(gT, C.c_double), _ptr(g, C.c_double),
                              self.nthreads)
        return self._split_grad(g)

    def ray(self, cam, u, v):
        """(origin, unit direction) of pixel (u, v); None where the pixel has
        no ray (a fisheye pixel beyond theta = pi)."""
        o = np.zeros(3)
        d = np.zeros(3)
        ok = lib().orc_ray(C.byref(camera_struct(cam)), float(u), float(v), _ptr(o, C.c_double),
                           _ptr(d, C.c_double))
        return (o, d) if ok else None

    def ray_segments(self, o, d, maxn: int = 100000):
        """Non-empty segments of the ray o + t d, sorted by entry distance:
        list of (cell, ta, tb, act_a, act_b); act is a neighbour id or one
        of ACT_SPHERE / ACT_CAMERA / ACT_DIPOLE."""
        o = np.ascontiguousarray(o, np.float64)
        d = np.ascontiguousarray(d, np.float64)
        cell = np.zeros(maxn, np.int32)
        ta = np.zeros(maxn)
        tb = np.zeros(maxn)
        aa = np.zeros(maxn, np.int32)
        ab = np.zeros(maxn, np.int32)
        n = lib().orc_ray_segments(C.byref(self._s), C.byref(self._cs) if self._cs else None,
                                   _ptr(o, C.c_double), _ptr(d, C.c_double), maxn,
                                   _ptr(cell, C.c_int32), _ptr(ta, C.c_double), _ptr(tb, C.c_double),
                                   _ptr(aa, C.c_int32), _ptr(ab, C.c_int32))
        n = min(int(n), maxn)
        return [(int(cell[k]), float(ta[k]), float(tb[k]), int(aa[k]), int(ab[k])) for k in range(n)]

    def cell_colour(self, i, o, d, ta, tb):
        o = np.ascontiguousarray(o, np.float64)
        d = np.ascontiguousarray(d, np.float64)
        col = np.zeros(3)
        lib().orc_cell_colour(C.byref(self._s), int(i), _ptr(o, C.c_double), _ptr(d, C.c_double),
                              float(ta), float(tb), self.kappa, _ptr(col, C.c_double))
        return col

    def render_tiles(self, cam, start, cells, tiles=None, t_stop: float = 0.0, return_nseg: bool = False):
        """Full-frame render over per-tile lists (CSR `start`, `cells`, from
        tile_lists): each pixel composites its tile's cells in list order,
        each clipped against the current candidate lists; a ray stops once
        T < t_stop.  `tiles`: indices of the tiles to render (None: all).
        Returns row-major rgb [H*W,3], T [H*W] (and nseg), NaN outside the
        rendered tiles."""
        npx = cam.width * cam.height
        rgb = np.full((npx, 3), np.nan)
        T = np.full(npx, np.nan)
        nseg = np.full(npx, -1, np.int32)
        start = np.ascontiguousarray(start, np.int64)
        cells = np.ascontiguousarray(cells, np.int32)
        if cells.size == 0:
            cells = np.zeros(1, np.int32)
        tl = None if tiles is None else np.ascontiguousarray(tiles, np.int32)
        lib().orc_render_tiles(C.byref(self._s), C.byref(self._cs) if self._cs else None,
                               C.byref(camera_struct(cam)), _ptr(start, C.c_int64), _ptr(cells, C.c_int32),
                               0 if tl is None else tl.size, None if tl is None else _ptr(tl, C.c_int32),
                               self.kappa, float(t_stop), _ptr(rgb, C.c_double), _ptr(T, C.c_double),
                               _ptr(nseg, C.c_int32), self.nthreads)
        return (rgb, T, nseg) if return_nseg else (rgb, T)

    def bin(self, cam):
        """CPU binning: tile rectangles [N,4] (tx0, ty0, tx1, ty1; empty when
        tx0 > tx1) and painter keys [N] (uint64, order-preserving bits of
        pow(o, p_i) in FP64)."""
        rect = np.zeros((self.n, 4), np.int32)
        key = np.zeros(self.n, np.uint64)
        a = self._arrs
        lib().orc_bin(C.byref(camera_struct(cam)), self.n, _ptr(a["pos"], C.c_double),
                      _ptr(a["w"], C.c_double), _ptr(a["R"], C.c_double), _ptr(rect, C.c_int32),
                      _ptr(key, C.c_uint64))
        return rect, key


def onb(n):
    nn = np.ascontiguousarray(n, np.float64)
    e1 = np.zeros(3)
    e2 = np.zeros(3)
    lib().orc_onb(_ptr(nn, C.c_double), _ptr(e1, C.c_double), _ptr(e2, C.c_double))
    return e1, e2


def tile_lists(rect: np.ndarray, key: np.ndarray, tiles_x: int, tiles_y: int):
    """Per-tile cell lists from the CPU binning: for tile t, the cells whose
    rectangle covers it, sorted by (key, cell index).  Returns (start [T+1],
    cells [n_instances]) in CSR form."""
    nt = tiles_x * tiles_y
    rect = np.asarray(rect, np.int64)
    x0, y0, x1, y1 = rect[:, 0], rect[:, 1], rect[:, 2], rect[:, 3]
    live = np.nonzero((x0 <= x1) & (y0 <= y1))[0]
    wd = (x1 - x0 + 1)[live]
    ht = (y1 - y0 + 1)[live]
    cnt = wd * ht
    total = int(cnt.sum())
    # every (cell, tile) pair of every rectangle, row by row
    cells = np.repeat(live, cnt)
    k = np.arange(total, dtype=np.int64) - np.repeat(np.cumsum(cnt) - cnt, cnt)
    w_rep = np.repeat(wd, cnt)
    tiles = (np.repeat(y0[live], cnt) + k // w_rep) * tiles_x + np.repeat(x0[live], cnt) + k % w_rep
    order = np.lexsort((cells, key[cells], tiles))
    tiles = tiles[order]
    cells = cells[order]
    start = np.searchsorted(tiles, np.arange(nt + 1))
    return start.astype(np.int64), cells.astype(np.int32)
