"""Python-level API over the C ABI: device scenes, plans with workspaces,
forward/backward calls and a torch.autograd.Function.

PyTorch provides device memory and streams only; every step of the
rendering path runs in the library's kernels.
"""
from __future__ import annotations

import ctypes as C
import math

import numpy as np
import torch

from . import _lib
from ._lib import check, lib, ptr

PARAMS = ("pos", "w", "R", "sigma", "rgb", "normal", "offset", "tex")
EXTRA_PARAMS = ("disp", "sites", "sv")   # optional: face displacement, learned sites, view-dependent colours


class DeviceScene:
    """Scene parameters as contiguous float32 CUDA tensors (+ int32 lists)."""

    def __init__(self, params: dict, nbr: torch.Tensor):
        self.params = params
        self.nbr = nbr
        self.n = int(params["pos"].shape[0])
        self.k = int(nbr.shape[1]) if nbr.dim() == 2 else 0
        # detail sites per face (Sec. 3.4): 4, or 8 when tex holds 24 values per cell
        self.n_sites = 8 if params["tex"].numel() == 24 * self.n and self.n > 0 else 4

    @staticmethod
    def from_numpy(scene, device="cuda", requires_grad=False, disp=None, sites=None, sv=None) -> "DeviceScene":
        """`disp` [N,S] (or the scene's `disp` attribute): face displacement
        at the S texture sites (Eq. svdisp).  `sites` [N,S,2] (or the
        scene's `sites`): learned positions of those sites, in units of R.
        `sv` [N,S,8,6] (or the scene's `sv`): view-dependent site colours,
        eight (axis, rgb) per site.  S, the detail sites per face, is 4, or 8
        when the scene's tex is [N,24]."""
        params = {}
        tex = np.asarray(scene.tex)
        ns = 8 if tex.ndim == 2 and tex.shape[1] == 24 else 4
        for k in PARAMS:
            a = np.ascontiguousarray(getattr(scene, k), np.float32)
            t = torch.from_numpy(a).to(device)
            if requires_grad:
                t.requires_grad_(True)
            params[k] = t
        if disp is None:
            disp = getattr(scene, "disp", None)
        if disp is not None:
            params["disp"] = torch.from_numpy(np.ascontiguousarray(disp, np.float32).reshape(scene.n, ns)).to(device)
        if sites is None:
            sites = getattr(scene, "sites", None)
        if sites is not None:
            params["sites"] = torch.from_numpy(np.ascontiguousarray(sites, np.float32).reshape(scene.n, ns, 2)).to(device)
        if sv is None:
            sv = getattr(scene, "sv", None)
        if sv is not None:
            params["sv"] = torch.from_numpy(np.ascontiguousarray(sv, np.float32).reshape(scene.n, ns, 8, 6)).to(device)
        nbr = torch.from_numpy(np.ascontiguousarray(scene.nbr, np.int32)).to(device)
        return DeviceScene(params, nbr)

    def struct(self, params: dict | None = None) -> _lib.Scene:
        p = self.params if params is None else params
        s = _lib.Scene()
        for k in PARAMS:
            t = p[k]
            if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
                raise ValueError(f"scene parameter {k} must be a contiguous float32 CUDA tensor")
            setattr(s, k, t.data_ptr() if t.numel() else None)
        s.nbr = self.nbr.data_ptr() if self.nbr.numel() else None
        s.n_cells = self.n
        s.k_nbr = self.k
        ns = 8 if p["tex"].numel() == 24 * self.n and self.n > 0 else 4
        s.n_sites = ns
        for k, width in (("disp", ns), ("sites", 2 * ns), ("sv", 48 * ns)):
            d = p.get(k)
            if d is not None:
                if not (d.is_cuda and d.dtype == torch.float32 and d.is_contiguous() and d.numel() == width * self.n):
                    raise ValueError(f"{k} must be a contiguous float32 CUDA tensor with {width} values per cell")
                setattr(s, k, d.data_ptr() if d.numel() else None)
        return s


def connect_loss(scene: DeviceScene, grad: bool = True):
    """pf_connect: the per-cell connectivity loss [N] (Sec. 4, L_connect over
    the neighbour lists) and, if grad, the gradients (dL/dpos [N,3], dL/dR [N])
    of its sum; otherwise (loss, None, None)."""
    p = scene.params
    loss = torch.empty(scene.n, dtype=torch.float32, device=p["pos"].device)
    gp = torch.zeros_like(p["pos"]) if grad else None
    gR = torch.zeros_like(p["R"]) if grad else None
    check(lib().pf_connect(C.byref(scene.struct()), loss.data_ptr(), gp.data_ptr() if grad else None,
                           gR.data_ptr() if grad else None, _stream()), "pf_connect")
    return loss, gp, gR


def connect_loss_cech(pos, R, grad: bool = True):
    """pf_connect_cech: the per-cell connectivity loss [N] over the exact
    Cech adjacency (every pair of overlapping bounding spheres, Sec. 4 /
    appendix) and, if grad, the gradients (dL/dpos [N,3], dL/dR [N]) of its
    sum; otherwise (loss, None, None).  pos [N,3], R [N]: float32 CUDA
    tensors."""
    n = int(pos.shape[0])
    for t in (pos, R):
        if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous():
            raise ValueError("connect_loss_cech: float32 contiguous CUDA tensors expected")
    dev = pos.device
    loss = torch.empty(n, dtype=torch.float32, device=dev)
    gp = torch.zeros_like(pos) if grad else None
    gR = torch.zeros_like(R) if grad else None
    ws_bytes = int(lib().pf_connect_cech_workspace_bytes(n))
    ws = torch.empty(max(ws_bytes, 256), dtype=torch.uint8, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    check(lib().pf_connect_cech(pos.data_ptr(), R.data_ptr(), n, loss.data_ptr(), ptr(gp), ptr(gR),
                                status.data_ptr(), ws.data_ptr(), ws_bytes, _stream()), "pf_connect_cech")
    if int(status.item()):
        raise RuntimeError("pf_connect_cech: a tree walk ran out of stack or steps")
    return loss, gp, gR


def build_neighbours(pos, w, R, k: int, out_R=None):
    """pf_build_neighbours: per cell the k sites with the smallest
    radical-plane distance t_ij = (|p_j - p_i|^2 + w_i - w_j) / (2|p_j - p_i|)
    (Sec. 3.2; ties by j, -1 padded) and R clipped below t_(k+1).  pos [N,3],
    w [N], R [N]: float32 CUDA tensors.  Returns (nbr int32 [N,k], R_out
    float32 [N] (out_R if given; it may be R), n_clipped int)."""
    n = int(pos.shape[0])
    dev = pos.device
    for t in (pos, w, R):
        if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous():
            raise ValueError("build_neighbours: float32 contiguous CUDA tensors expected")
    nbr = torch.empty((n, k), dtype=torch.int32, device=dev)
    R_out = torch.empty_like(R) if out_R is None else out_R
    ws_bytes = int(lib().pf_neighbours_workspace_bytes(n))
    ws = torch.empty(max(ws_bytes, 256), dtype=torch.uint8, device=dev)
    info = torch.zeros(2, dtype=torch.int32, device=dev)  # n_clipped, status
    check(lib().pf_build_neighbours(pos.data_ptr(), w.data_ptr(), R.data_ptr(), n, k,
                                    nbr.data_ptr() if k > 0 else None, R_out.data_ptr(), info.data_ptr(),
                                    info.data_ptr() + 4, ws.data_ptr(), ws_bytes, _stream()),
          "pf_build_neighbours")
    ncl, status = (int(x) for x in info.cpu())
    if status:
        raise RuntimeError("pf_build_neighbours: a tree walk ran out of stack or steps")
    return nbr, R_out, ncl


class Plan:
    """A C plan (layout + cameras) with its device workspace."""

    def __init__(self, n: int, k: int, cams, capacity: int, device="cuda", hit_records: bool = True,
                 store_segments: int = 0):
        self.n, self.k = n, k
        self.cams = list(cams)
        self.capacity = int(capacity)
        self.handle = C.c_void_p()
        arr = _lib.camera_array(self.cams)
        check(lib().pf_plan_create(n, k, arr, len(self.cams), self.capacity, C.byref(self.handle)),
              "pf_plan_create")
        if not hit_records:
            check(lib().pf_plan_omit_hit_records(self.handle), "pf_plan_omit_hit_records")
        if store_segments:
            check(lib().pf_plan_store_segments(self.handle, int(store_segments)), "pf_plan_store_segments")
        b = C.c_uint64()
        check(lib().pf_plan_workspace_bytes(self.handle, C.byref(b)), "pf_plan_workspace_bytes")
        self.ws_bytes = int(b.value)
        self.ws = torch.empty(max(self.ws_bytes, 256), dtype=torch.uint8, device=device)
        px = C.c_uint64()
        check(lib().pf_plan_pixels(self.handle, C.byref(px)), "pf_plan_pixels")
        self.pixels = int(px.value)

    def set_cameras(self, cams):
        cams = list(cams)
        check(lib().pf_plan_set_cameras(self.handle, _lib.camera_array(cams), len(cams)), "pf_plan_set_cameras")
        self.cams = cams

    def __del__(self):
        try:
            if self.handle:
                lib().pf_plan_destroy(self.handle)
                self.handle = C.c_void_p()
        except Exception:
            pass

    @property
    def ws_ptr(self):
        return self.ws.data_ptr()


def _stream():
    return _lib.stream_ptr(torch.cuda.current_stream())


class Renderer:
    """Renders a DeviceScene from a fixed set of cameras (one or many views,
    any resolutions).  The instance capacity grows automatically."""

    def __init__(self, n: int, k: int, cams, capacity: int | None = None, device="cuda",
                 hit_records: bool = True, store_segments: int = 0):
        """hit_records=False lays the workspace out without the forward's hit
        records (smaller; the backward then always re-tests).
        store_segments=M > 0 also stores each pixel's first M segments
        (ends, transmittance in front, active constraints; 16 bytes each), which
        the backward reads instead of recomputing (pf_plan_store_segments)."""
        self.device = device
        self._hit_records = hit_records
        self._store = int(store_segments)
        cams = list(cams)
        if capacity is None:
            px = sum(c.width * c.height for c in cams)
            capacity = max(1 << 16, min(8 * n * len(cams) + px // 16, 0xE0000000))
        self._record = hit_records
        self._stats = False
        self.plan = self._make_plan(n, k, cams, capacity)
        self.generation = 0
        self.n_instances = 0

    def _make_plan(self, n, k, cams, capacity):
        P = Plan(n, k, cams, capacity, self.device, hit_records=self._hit_records, store_segments=self._store)
        check(lib().pf_plan_set_record_hits(P.handle, 1 if self._record else 0), "pf_plan_set_record_hits")
        check(lib().pf_plan_enable_stats(P.handle, 1 if self._stats else 0), "pf_plan_enable_stats")
        return P

    @property
    def cams(self):
        return self.plan.cams

    def set_cameras(self, cams):
        cams = list(cams)
        if [(c.width, c.height) for c in cams] == [(c.width, c.height) for c in self.plan.cams]:
            self.plan.set_cameras(cams)
        else:
            self.plan = self._make_plan(self.plan.n, self.plan.k, cams, self.plan.capacity)
        self.generation += 1

    def bin(self, scene: DeviceScene, params: dict | None = None, sync: bool = True):
        """pf_prepare + pf_project + pf_bin_sort (re-planning on overflow)."""
        s = scene.struct(params)
        st = _stream()
        for _ in range(3):
            P = self.plan
            check(lib().pf_prepare(C.byref(s), P.handle, P.ws_ptr, st), "pf_prepare")
            check(lib().pf_project(C.byref(s), P.handle, P.ws_ptr, st), "pf_project")
            if not sync:
                check(lib().pf_bin_sort(P.handle, P.ws_ptr, None, st), "pf_bin_sort")
                break
            n = C.c_uint64()
            r = lib().pf_bin_sort(P.handle, P.ws_ptr, C.byref(n), st)
            self.n_instances = int(n.value)
            if r == _lib.PF_ERR_CAPACITY:
                cap = min(int(n.value * 1.25) + 1024, 0xE0000000)
                self.plan = self._make_plan(P.n, P.k, P.cams, cap)
                continue
            check(r, "pf_bin_sort")
            break
        self.generation += 1
        return self.generation

    def _alloc_out(self):
        P = self.plan
        rgb = torch.empty((P.pixels, 3), dtype=torch.float32, device=self.device)
        T = torch.empty(P.pixels, dtype=torch.float32, device=self.device)
        last = torch.empty(P.pixels, dtype=torch.int32, device=self.device)
        return rgb, T, last

    def render_fwd(self, scene: DeviceScene, params: dict | None = None, out=None, contrib=None):
        """pf_render_fwd on the current bins: flat rgb [P,3], T [P], last [P].
        With contrib=(sparse [N], normal [N]) (float32 device tensors) it is
        pf_render_fwd_contrib, which also adds the per-cell contributions
        (sum of T alpha, and of T alpha max(n.d, 0)^2) into them."""
        rgb, T, last = out if out is not None else self._alloc_out()
        P = self.plan
        if contrib is None:
            check(lib().pf_render_fwd(C.byref(scene.struct(params)), P.handle, P.ws_ptr, rgb.data_ptr(),
                                      T.data_ptr(), last.data_ptr(), _stream()), "pf_render_fwd")
        else:
            cs, cn = contrib
            for t in (cs, cn):
                if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous() and t.numel() == P.n):
                    raise ValueError("contribution arrays must be contiguous float32 CUDA tensors of N cells")
            check(lib().pf_render_fwd_contrib(C.byref(scene.struct(params)), P.handle, P.ws_ptr, rgb.data_ptr(),
                                              T.data_ptr(), last.data_ptr(), cs.data_ptr(), cn.data_ptr(),
                                              _stream()), "pf_render_fwd_contrib")
        return rgb, T, last

    def forward(self, scene: DeviceScene, params: dict | None = None, sync: bool = True):
        self.bin(scene, params, sync=sync)
        return self.render_fwd(scene, params)

    def backward(self, scene: DeviceScene, dL_drgb, dL_dT, T, last, params: dict | None = None, grads=None,
                 contrib_weights=None):
        """pf_render_bwd: returns a dict of gradient tensors (added into
        `grads` when given).  With contrib_weights=(w_sparse [N], w_normal
        [N]) it is pf_render_bwd_contrib: the loss also holds
        sum_i w_sparse[i] sparse_i + w_normal[i] normal_i over the per-cell
        contributions of render_fwd(contrib=...)."""
        p = scene.params if params is None else params
        keys = PARAMS + tuple(k for k in EXTRA_PARAMS if p.get(k) is not None)
        if grads is None:
            grads = {k: torch.zeros_like(p[k]) for k in keys}
        g = _lib.SceneGrad()
        for k in keys:
            setattr(g, k, grads[k].data_ptr() if grads[k].numel() else None)
        dL_drgb = dL_drgb.contiguous().float()
        dL_dT = None if dL_dT is None else dL_dT.contiguous().float()
        P = self.plan
        if contrib_weights is None:
            check(lib().pf_render_bwd(C.byref(scene.struct(params)), P.handle, P.ws_ptr, dL_drgb.data_ptr(),
                                      ptr(dL_dT), T.data_ptr(), last.data_ptr(), C.byref(g), _stream()),
                  "pf_render_bwd")
        else:
            ws_, wn_ = (w.contiguous().float() for w in contrib_weights)
            for t in (ws_, wn_):
                if not (t.is_cuda and t.numel() == P.n):
                    raise ValueError("contribution weights must be float32 CUDA tensors of N cells")
            check(lib().pf_render_bwd_contrib(C.byref(scene.struct(params)), P.handle, P.ws_ptr, dL_drgb.data_ptr(),
                                              ptr(dL_dT), T.data_ptr(), last.data_ptr(), ws_.data_ptr(),
                                              wn_.data_ptr(), C.byref(g), _stream()), "pf_render_bwd_contrib")
        return grads

    def hit_counts(self):
        """Hits the last recording forward composited per pixel (numpy uint32 [P])."""
        P = self.plan
        out = np.zeros(P.pixels, np.uint32)
        check(lib().pf_read_hit_counts(P.handle, P.ws_ptr, out.ctypes.data, _stream()), "pf_read_hit_counts")
        return out

    def stats(self):
        s = _lib.Stats()
        P = self.plan
        check(lib().pf_plan_read_stats(P.handle, P.ws_ptr, C.byref(s), _stream()), "pf_plan_read_stats")
        return {f: int(getattr(s, f)) for f, _ in _lib.Stats._fields_}

    def record_hits(self, on: bool = True):
        """Hit recording in the forward (default on); off for rendering only."""
        self._record = bool(on)
        check(lib().pf_plan_set_record_hits(self.plan.handle, 1 if on else 0), "pf_plan_set_record_hits")

    def enable_stats(self, on: bool = True):
        self._stats = bool(on)
        check(lib().pf_plan_enable_stats(self.plan.handle, 1 if on else 0), "pf_plan_enable_stats")

    def read_bins(self):
        """Host copies of (tile_start [T+1], cells [capacity], keys [V*N], rects [V*N,4])."""
        P = self.plan
        T = sum(((c.width + 15) // 16) * ((c.height + 15) // 16) for c in P.cams)
        ts = np.zeros(T + 1, np.uint32)
        cells = np.zeros(max(P.capacity, 1), np.uint32)
        keys = np.zeros(max(P.n * len(P.cams), 1), np.uint64)
        rects = np.zeros((max(P.n * len(P.cams), 1), 4), np.uint16)
        check(lib().pf_read_bins(P.handle, P.ws_ptr, ts.ctypes.data, cells.ctypes.data, keys.ctypes.data,
                                 rects.ctypes.data, _stream()), "pf_read_bins")
        return ts, cells, keys, rects

    def split(self, flat):
        """Per-view images from a flat per-pixel tensor."""
        out = []
        o = 0
        for c in self.cams:
            n = c.width * c.height
            out.append(flat[o:o + n].view(c.height, c.width, *flat.shape[1:]))
            o += n
        return out


class RenderFunction(torch.autograd.Function):
    """(pos, w, R, sigma, rgb, normal, offset, tex[, disp][, sites][, sv]) ->
    (rgb [P,3], T [P]); `keys` names the parameter tensors that follow.

    The backward replays the forward's checkpoint (T, last) tile by tile,
    back to front, through pf_render_bwd."""

    @staticmethod
    def forward(ctx, renderer: Renderer, scene: DeviceScene, keys, *params):
        pd = dict(zip(keys, [p.detach() for p in params]))
        gen = renderer.bin(scene, pd)
        rgb, T, last = renderer.render_fwd(scene, pd)
        ctx.renderer = renderer
        ctx.scene = scene
        ctx.gen = gen
        ctx.keys = keys
        ctx.save_for_backward(T, last, *params)
        return rgb, T

    @staticmethod
    def backward(ctx, g_rgb, g_T):
        T, last, *params = ctx.saved_tensors
        r = ctx.renderer
        pd = dict(zip(ctx.keys, [p.detach() for p in params]))
        if r.generation != ctx.gen:  # the workspace was reused: rebuild the same bins
            r.bin(ctx.scene, pd)
        if g_rgb is None:
            g_rgb = torch.zeros((T.shape[0], 3), device=T.device)
        grads = r.backward(ctx.scene, g_rgb, g_T, T, last, pd)
        return (None, None, None, *[grads[k] for k in ctx.keys])


def render(renderer: Renderer, scene: DeviceScene, params: dict | None = None):
    """Differentiable render of all the renderer's views: flat rgb [P,3], T [P],
    with gradients for every parameter tensor of the scene (the optional
    displacement, learned sites and view-dependent colours included)."""
    p = scene.params if params is None else params
    keys = PARAMS + tuple(k for k in EXTRA_PARAMS if p.get(k) is not None)
    return RenderFunction.apply(renderer, scene, keys, *[p[k] for k in keys])
