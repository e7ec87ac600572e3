"""Benchmark: 1080p forward and forward+backward frames/s of the bounded
power-cell rasterizer on a synthetic 1M-cell capture-shaped scene, with the
render kernel's roofline fraction, an end-to-end number through host
buffers, and the FP64 CPU oracle timed on a pixel sample beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU: one process per GPU (torchrun); every rank renders its own
views (independent frames, no data-path collective): weak scaling.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "1080p fwd & fwd+bwd frames/s at 1M cells; serve p50/p99 ms; % roofline"
UNIT = "frames/s"
WORKLOAD = "capture-shaped scene, 1,000,000 cells (70% Gaussian mixture in the unit ball, 30% log-uniform shell to r=20), r=0.35*d8, R=1.5r, 32 neighbours; one 1920x1080 pinhole view (fov_y 60 deg) from (3,0,0)"

WORKLOAD_SMALL = "profiling case: the same recipe at 400,000 cells, one 1280x720 view from (3,0,0)"

# Algorithmic FP32 work of the forward per counted event, the per-unit
# figures of the path's cost model: a candidate (a listed cell a pixel
# examines) costs a sphere test of about 10 flops; a hit (a non-empty
# segment) about 140: about 9 relevant radical planes x 6, the dipole face
# 8, the soft-Voronoi texture about 60 and compositing 10.  The event counts
# come from the render kernel's stats pass over the same frame.
ALG_FLOPS_PER_CANDIDATE = 10
ALG_FLOPS_PER_HIT = 140

# The same frame counted operation by operation from the render kernel's
# source (FMA = 2, add / mul / compare / sqrt / exp / reciprocal = 1),
# reported beside the algorithmic figure: it includes the work this
# implementation adds (compensated products, refinement checks, the planes
# each ray needs on its own).
IMPL_FLOPS_PER_CANDIDATE = 15   # cheap sphere test: m x d (9), |v|^2 (5), compare (1)
IMPL_FLOPS_PER_PASS = 107       # compensated m x d (51), D (7), tangent check (9), sqrt (1),
                                # q = d x v (9), m.d (5), camera end (2), face clip (14),
                                # emptiness (1), refinement checks (8)
IMPL_FLOPS_PER_PLANE = 14       # q.a (5), g - q.a (1), d.a (5), sign test, divide, compare (3)
IMPL_FLOPS_PER_HIT = 92         # face point (6), face coordinates (10), site offsets (4),
                                # four sites x (|u - s| 3, sqrt, scale, exp, sum) (28),
                                # normalise (5), colour (24), compositing (15)


TRAFFIC_PROFILE = os.path.join(ROOT, "profiles", "render_fwd_pipe_dram_1080p_1M.md")
TRAFFIC_SOURCES = ("paper_2604_24994_gb300/csrc/pf_render_pipe.cu", "paper_2604_24994_gb300/csrc/pf_render_common.cuh",
                   "paper_2604_24994_gb300/csrc/pf_internal.cuh", "include/powerfoam.h")


def render_source_digest():
    import hashlib
    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def measured_traffic():
    """DRAM bytes (read + write) of one render_fwd_pipe_kernel launch on this
    workload from the committed ncu summary, or None when the kernel's
    sources changed since those counters were taken."""
    try:
        txt = open(TRAFFIC_PROFILE).read()
    except OSError:
        return None
    fields = dict(line.split(":", 1) for line in txt.splitlines() if line.startswith(("source_sha256:", "dram_bytes_per_launch:")))
    if fields.get("source_sha256", "").strip() != render_source_digest():
        return None
    return int(fields["dram_bytes_per_launch"].strip())


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for n, v in zip(names, r[5:9]):
                    if v.lower() == "active":
                        reasons.add(n)
            except Exception:
                pass
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def bench_config(workload: str, width: int, height: int, n_cells: int, n_nbr: int, ws: int = 1) -> dict:
    """The workload description both arms print (the same keys and values)."""
    return {"workload": WORKLOAD if workload == "full" else WORKLOAD_SMALL,
            "resolution": f"{width}x{height}", "cells": n_cells, "neighbours": n_nbr,
            "parallelism": f"replicas x{ws}",
            "l2": "256 MiB buffer written between timed steps (not timed)",
            "fwd_step": "pf_project + pf_bin_sort + pf_render_fwd (scene resident and prepared)",
            "fwd_bwd_step": "pf_prepare + pf_project + pf_bin_sort + pf_render_fwd + L2 loss grad + pf_render_bwd"}


def make_workload(rank: int = 0, small: bool = False):
    """The 1080p / 1M-cell capture workload, or (small=True) the same recipe
    at 400k cells and 1280x720 for profiler captures."""
    from paper_2604_24994_gb300 import inputs
    t0 = time.time()
    from paper_2604_24994_gb300.dataparallel import ring_view
    sc = inputs.capture_scene(400_000 if small else 1_000_000, seed=0, K=32)
    w, h = (1280, 720) if small else (1920, 1080)
    cam = inputs.capture_camera(w, h)
    if rank:  # every rank renders its own view of the same scene
        cam = ring_view(rank, w, h)
    return sc, cam, time.time() - t0


def cpu_baseline(sc, cam, seconds: float = 15.0):
    """The oracle as it stands, on a bounded pixel sample of the frame."""
    import oracle
    orc = oracle.Oracle(sc)
    rng = np.random.default_rng(0)
    n = 16
    done = 0
    t_spent = 0.0
    while t_spent < seconds and done < 4096:
        pix = np.stack([rng.integers(0, cam.width, n), rng.integers(0, cam.height, n)], 1).astype(np.int32)
        t0 = time.time()
        orc.prune_for(cam, pix)
        orc.render(cam, pix)
        t_spent += time.time() - t0
        done += n
        n = min(2 * n, 256)
    per_px = t_spent / done
    fps = 1.0 / (per_px * cam.width * cam.height)
    return {"value": fps, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{done} random pixels of the 1920x1080 frame ({t_spent:.1f} s, exact prune, "
                      f"OpenMP over pixels); frames/s = 1 / (time per pixel x 2,073,600)"}


def cpu_tile_baseline(sc, cam, t_stop: float = 1e-6):
    """Second, labelled CPU baseline: the oracle's full-frame FP64 renderer
    over per-tile lists and the scene's K-neighbour lists (the tiled
    renderer's own math, with its stop at T < 1e-6).  Timed: the CPU binning
    (single thread), the per-tile list sort (numpy) and the render (OpenMP
    over tiles); the neighbour lists are scene data, loaded before."""
    import oracle
    orc = oracle.Oracle(sc)
    orc.set_neighbour_lists(sc.nbr)
    t0 = time.time()
    rect, key = orc.bin(cam)
    start, cells = oracle.tile_lists(rect, key, cam.tiles_x, cam.tiles_y)
    t1 = time.time()
    orc.render_tiles(cam, start, cells, t_stop=t_stop)
    t2 = time.time()
    return {"value": 1.0 / (t2 - t0), "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle tile-list renderer",
            "s_bin_and_lists": round(t1 - t0, 3), "s_render": round(t2 - t1, 3),
            "sample": f"the full {cam.width}x{cam.height} frame: CPU binning, per-tile lists in painter order, "
                      f"each listed cell clipped against its {sc.k} neighbours in FP64, stop at T < {t_stop:g}"}


def run_reference(args):
    """The oracle as it stands on this host's cores: each step renders a
    bounded sample (64 random pixels) of the benchmark frame; frames/s is
    extrapolated from the time per pixel."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    small = args.workload == "small"
    sc, cam, _ = make_workload(0, small=small)
    import oracle
    orc = oracle.Oracle(sc)
    rng = np.random.default_rng(1)
    per, step_s = [], []
    for step in range(args.warmup + args.steps):
        pix = np.stack([rng.integers(0, cam.width, 64), rng.integers(0, cam.height, 64)], 1).astype(np.int32)
        t0 = time.time()
        orc.prune_for(cam, pix)
        orc.render(cam, pix)
        dt = time.time() - t0
        if step >= args.warmup:
            per.append(dt / 64)
            step_s.append(dt)
    per_px = float(np.mean(per))
    fps = 1.0 / (per_px * cam.width * cam.height)
    sample = (f"each step 64 random pixels of the {cam.width}x{cam.height} frame (exact prune, OpenMP over "
              f"pixels); frames/s extrapolated as 1 / (time per pixel x {cam.width * cam.height:,})")
    line = {"impl": "reference", "metric": METRIC, "value": fps, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(np.mean(step_s)) * 1e3,
            "ms_per_frame_extrapolated": per_px * cam.width * cam.height * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": bench_config(args.workload, cam.width, cam.height, sc.n, sc.k, args.gpus),
            "cpu_baseline": {"value": fps, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": fps, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2604_24994_gb300 import DeviceScene, Renderer, build
    from paper_2604_24994_gb300.dataparallel import sum_gradients
    build.build()

    sc, cam, gen_s = make_workload(rank, small=args.workload == "small")
    ds = DeviceScene.from_numpy(sc, "cuda")
    r = Renderer(ds.n, ds.k, [cam])
    stream = torch.cuda.current_stream()

    # size the instance capacity (synchronous once), then count work once
    r.bin(ds, sync=True)
    n_inst = r.n_instances
    r.enable_stats(True)
    rgb, T, last = r.render_fwd(ds)
    stats = r.stats()
    r.enable_stats(False)

    # target image for the fwd+bwd step: the same scene with sites moved by N(0, 0.002)
    from paper_2604_24994_gb300 import inputs
    tsc = inputs.perturbed_sites(sc, 0.002, seed=1)
    tds = DeviceScene.from_numpy(tsc, "cuda")
    rt = Renderer(tds.n, tds.k, [cam])
    target, _, _ = rt.forward(tds)
    target = target.clone()
    del rt, tds

    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    ev = lambda: torch.cuda.Event(enable_timing=True)

    def fwd_step(times=None):
        # a new view of a resident scene: project + bin/sort + render
        from paper_2604_24994_gb300._lib import check, lib
        import ctypes as C
        P = r.plan
        s = ds.struct()
        check(lib().pf_project(C.byref(s), P.handle, P.ws_ptr, stream.cuda_stream), "project")
        check(lib().pf_bin_sort(P.handle, P.ws_ptr, None, stream.cuda_stream), "bin_sort")
        if times is not None:
            a, b = ev(), ev()
            a.record(stream)
        out = r.render_fwd(ds, out=(rgb, T, last))
        if times is not None:
            b.record(stream)
            times.append((a, b))
        return out

    def train_step():
        r.bin(ds, sync=False)  # prepare + project + bin/sort
        c, t, l = r.render_fwd(ds, out=(rgb, T, last))
        g = 2.0 * (c - target)
        r.backward(ds, g, None, t, l, grads=grads)
        if ws > 1:  # data parallel over views: sum the per-view gradients (the one exchange step)
            sum_gradients(grads)
        return g

    grads = {k: torch.zeros_like(v) for k, v in ds.params.items()}
    # library kernels per forward step: project, the difference grids' sum, tile counts,
    # 2 scans x 3, expand, tile order, 2 tile sorts (shared-memory sizes), render
    kernels_fwd = 1 + 1 + 1 + 6 + 1 + 1 + 2 + 1

    def timed(fn, k, warm, per_kernel=None):
        for _ in range(warm):
            fn()
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        tot = 0.0
        for _ in range(k):
            flush.zero_()                      # L2 flush between steps (not timed)
            a, b = ev(), ev()
            a.record(stream)
            fn(per_kernel) if per_kernel is not None else fn()
            b.record(stream)
            b.synchronize()
            tot += a.elapsed_time(b)
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        return tot / k

    K, W = args.steps, args.warmup
    with ClockSampler(local) as clk:
        kt = []
        r.record_hits(False)   # rendering only: nothing for a backward to replay
        ms_fwd = timed(fwd_step, K, W, kt)
        ms_render = float(np.mean([a.elapsed_time(b) for a, b in kt]))
        r.record_hits(True)    # training: the forward records the hits the backward replays
        ms_train = timed(train_step, K, W)
        r.record_hits(False)
    clocks = clk.summary()

    # the forward with the per-cell contributions (T alpha, T alpha max(n.d,0)^2) added
    contrib = (torch.zeros(ds.n, device="cuda"), torch.zeros(ds.n, device="cuda"))
    ct = []
    for it in range(W + K):
        flush.zero_()
        a, b = ev(), ev()
        a.record(stream)
        r.render_fwd(ds, out=(rgb, T, last), contrib=contrib)
        b.record(stream)
        b.synchronize()
        if it >= W:
            ct.append(a.elapsed_time(b))
    ms_render_contrib = float(np.mean(ct))
    del contrib
    # the connectivity loss and its gradient over the neighbour lists
    from paper_2604_24994_gb300.api import connect_loss
    cc = []
    for it in range(W + K):
        a, b = ev(), ev()
        a.record(stream)
        connect_loss(ds)
        b.record(stream)
        b.synchronize()
        if it >= W:
            cc.append(a.elapsed_time(b))
    ms_connect = float(np.mean(cc))
    # the same loss over the exact Cech adjacency (every overlapping pair of bounding spheres)
    from paper_2604_24994_gb300.api import connect_loss_cech
    cc = []
    for it in range(W + K):
        a, b = ev(), ev()
        a.record(stream)
        connect_loss_cech(ds.params["pos"], ds.params["R"])
        b.record(stream)
        b.synchronize()
        if it >= W:
            cc.append(a.elapsed_time(b))
    ms_connect_cech = float(np.mean(cc))
    # a 180-degree equidistant fisheye view of the same scene through the same kernels
    from paper_2604_24994_gb300 import inputs as _inputs
    fcam = _inputs.fisheye_look_at(tuple(np.asarray(cam.origin)), cam.width, cam.height, fov_deg=180.0)
    rf = Renderer(ds.n, ds.k, [fcam], hit_records=False)
    rf.bin(ds, sync=True)                      # prepare once, size the instance capacity
    fo = rf.render_fwd(ds)
    from paper_2604_24994_gb300._lib import check, lib
    import ctypes as C
    sst = ds.struct()
    ft = []
    for it in range(W + K):
        flush.zero_()
        a, b = ev(), ev()
        a.record(stream)
        check(lib().pf_project(C.byref(sst), rf.plan.handle, rf.plan.ws_ptr, stream.cuda_stream), "project")
        check(lib().pf_bin_sort(rf.plan.handle, rf.plan.ws_ptr, None, stream.cuda_stream), "bin_sort")
        rf.render_fwd(ds, out=fo)
        b.record(stream)
        b.synchronize()
        if it >= W:
            ft.append(a.elapsed_time(b))
    ms_fisheye = float(np.mean(ft))
    del rf, fo
    # the same forward step with every face displaced (Eq. svdisp), up to 0.2 R at each texture site
    drng = np.random.default_rng(5)
    dsp = torch.from_numpy((drng.uniform(-0.2, 0.2, (ds.n, 4)) * sc.R[:, None]).astype(np.float32)).cuda()
    dparams = dict(ds.params, disp=dsp)
    dst = ds.struct(dparams)
    rd = Renderer(ds.n, ds.k, [cam], hit_records=False)
    rd.bin(ds, params=dparams, sync=True)   # prepare prunes planes against the displaced face
    do = rd.render_fwd(ds, params=dparams)
    dt = []
    for it in range(W + K):
        flush.zero_()
        a, b = ev(), ev()
        a.record(stream)
        check(lib().pf_project(C.byref(dst), rd.plan.handle, rd.plan.ws_ptr, stream.cuda_stream), "project")
        check(lib().pf_bin_sort(rd.plan.handle, rd.plan.ws_ptr, None, stream.cuda_stream), "bin_sort")
        check(lib().pf_render_fwd(C.byref(dst), rd.plan.handle, rd.plan.ws_ptr, do[0].data_ptr(), do[1].data_ptr(),
                                  do[2].data_ptr(), stream.cuda_stream), "render_fwd")
        b.record(stream)
        b.synchronize()
        if it >= W:
            dt.append(a.elapsed_time(b))
    ms_disp = float(np.mean(dt))
    # view-dependent site colours (spherical Voronoi, eight axes per site) on the same view
    svp = np.concatenate([drng.normal(size=(ds.n, 4, 8, 3)), drng.uniform(0, 1, (ds.n, 4, 8, 3))], -1)
    sparams = dict(ds.params, sv=torch.from_numpy(svp.astype(np.float32)).cuda())
    sst2 = ds.struct(sparams)
    del svp
    st_t = []
    for it in range(W + K):
        flush.zero_()
        a, b = ev(), ev()
        a.record(stream)
        check(lib().pf_project(C.byref(sst2), rd.plan.handle, rd.plan.ws_ptr, stream.cuda_stream), "project")
        check(lib().pf_bin_sort(rd.plan.handle, rd.plan.ws_ptr, None, stream.cuda_stream), "bin_sort")
        check(lib().pf_render_fwd(C.byref(sst2), rd.plan.handle, rd.plan.ws_ptr, do[0].data_ptr(), do[1].data_ptr(),
                                  do[2].data_ptr(), stream.cuda_stream), "render_fwd")
        b.record(stream)
        b.synchronize()
        if it >= W:
            st_t.append(a.elapsed_time(b))
    ms_sv = float(np.mean(st_t))
    # eight detail sites per face (Sec. 3.4's main configuration): 24 texture values, displacements up to
    # 0.2 R and learned positions (the fixed 3 x 3 grid without its centre, jittered) at every site
    grid8 = np.array([[-1, -1], [0, -1], [1, -1], [-1, 0], [1, 0], [-1, 1], [0, 1], [1, 1]], np.float32) / 3.0
    e8 = dict(ds.params,
              tex=torch.from_numpy(drng.normal(0, 0.1, (ds.n, 24)).astype(np.float32)).cuda(),
              disp=torch.from_numpy((drng.uniform(-0.2, 0.2, (ds.n, 8)) * sc.R[:, None]).astype(np.float32)).cuda(),
              sites=torch.from_numpy((grid8[None] + drng.uniform(-0.1, 0.1, (ds.n, 8, 2))).astype(np.float32)).cuda())
    est = ds.struct(e8)
    assert est.n_sites == 8
    rd.bin(ds, params=e8, sync=True)
    e8_t = []
    for it in range(W + K):
        flush.zero_()
        a, b = ev(), ev()
        a.record(stream)
        check(lib().pf_project(C.byref(est), rd.plan.handle, rd.plan.ws_ptr, stream.cuda_stream), "project")
        check(lib().pf_bin_sort(rd.plan.handle, rd.plan.ws_ptr, None, stream.cuda_stream), "bin_sort")
        check(lib().pf_render_fwd(C.byref(est), rd.plan.handle, rd.plan.ws_ptr, do[0].data_ptr(), do[1].data_ptr(),
                                  do[2].data_ptr(), stream.cuda_stream), "render_fwd")
        b.record(stream)
        b.synchronize()
        if it >= W:
            e8_t.append(a.elapsed_time(b))
    ms_e8 = float(np.mean(e8_t))
    del rd, do, dsp, dparams, sparams, e8, est
    # the neighbour lists of the same scene built on the GPU (pf_build_neighbours)
    from paper_2604_24994_gb300.api import build_neighbours
    pw, Rin = ds.params["pos"], ds.params["R"]
    nt = []
    for it in range(W + K):
        a, b = ev(), ev()
        a.record(stream)
        nb_gpu, R_gpu, _ = build_neighbours(pw, ds.params["w"], Rin, ds.k)
        b.record(stream)
        b.synchronize()
        if it >= W:
            nt.append(a.elapsed_time(b))
    ms_neighbours = float(np.mean(nt))
    nbr_same = bool(torch.equal(nb_gpu.cpu(), torch.from_numpy(sc.nbr)))
    del nb_gpu, R_gpu

    # end to end through the public API with host buffers: camera in, image out
    host_rgb = torch.empty((r.plan.pixels, 3), dtype=torch.float32, pin_memory=True)
    host_T = torch.empty(r.plan.pixels, dtype=torch.float32, pin_memory=True)

    def e2e_step():
        r.set_cameras([cam])                     # host camera -> plan (copied by pf_project)
        fwd_step()
        host_rgb.copy_(rgb, non_blocking=True)
        host_T.copy_(T, non_blocking=True)

    ms_e2e = timed(e2e_step, K, W)

    if ws > 1:
        import torch.distributed as dist
        t = torch.tensor([ms_fwd, ms_train, ms_e2e], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_fwd, ms_train, ms_e2e = [float(x) for x in t.cpu()]
    if rank != 0:
        return

    pk = peaks()
    sm_max = float(pk.get("sm_max_mhz", 2070.0))
    n_sms = torch.cuda.get_device_properties(local).multi_processor_count
    peak_tflops = n_sms * 128 * 2 * sm_max * 1e6 / 1e12   # FP32 FMA lanes x 2 flops x clock
    alg_flops = stats["candidates"] * ALG_FLOPS_PER_CANDIDATE + stats["hits"] * ALG_FLOPS_PER_HIT
    impl_flops = (stats["candidates"] * IMPL_FLOPS_PER_CANDIDATE + stats["sphere_pass"] * IMPL_FLOPS_PER_PASS
                  + stats["planes"] * IMPL_FLOPS_PER_PLANE + stats["hits"] * IMPL_FLOPS_PER_HIT)
    achieved = alg_flops / (ms_render * 1e-3) / 1e12
    achieved_impl = impl_flops / (ms_render * 1e-3) / 1e12
    cpu = cpu_baseline(sc, cam, seconds=args.cpu_seconds) if args.cpu_seconds > 0 else None
    cpu_tiles = cpu_tile_baseline(sc, cam) if args.cpu_seconds > 0 else None
    n_cells, n_nbr = ds.n, ds.k
    line = {
        "metric": METRIC, "value": ws * 1000.0 / ms_fwd, "unit": UNIT, "n_gpus": ws, "steps": K, "warmup": W,
        "ms_per_step": ms_fwd, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 (FP64 geometry)", "data": "synthetic",
        "config": bench_config(args.workload, cam.width, cam.height, n_cells, n_nbr, ws),
        "instances": n_inst, "scene_generation_s": round(gen_s, 1),
        "side_steps": {"fisheye_step": "the forward step for a 180-degree equidistant fisheye of the same size and position",
                       "displaced_step": "the forward step with every face displaced by up to 0.2 R at its four sites",
                       "view_dependent_step": "the forward step with spherical-Voronoi site colours (8 axes per site)",
                       "eight_site_step": "the forward step with eight detail sites per face: 24 texture values, "
                                          "displacements up to 0.2 R and learned positions"},
        "fwd_fps": ws * 1000.0 / ms_fwd, "fwd_bwd_fps": ws * 1000.0 / ms_train, "ms_fwd_bwd": ms_train,
        "ms_render_fwd_kernel": ms_render,
        "ms_render_fwd_contrib_kernel": ms_render_contrib,
        "ms_connect_loss_and_grad": ms_connect,
        "ms_connect_cech_loss_and_grad": ms_connect_cech,
        "fisheye_fwd_fps": 1000.0 / ms_fisheye,
        "displaced_fwd_fps": 1000.0 / ms_disp,
        "view_dependent_fwd_fps": 1000.0 / ms_sv,
        "eight_site_fwd_fps": 1000.0 / ms_e8,
        "ms_build_neighbours": ms_neighbours,
        "neighbours_equal_input_lists": nbr_same,
        "work": stats,
        "roofline": {"bound": "alu", "kernel": "render_fwd_pipe_kernel", "achieved": achieved, "peak": peak_tflops,
                     "unit": "TFLOP/s", "frac": achieved / peak_tflops,
                     "traffic": measured_traffic() if args.workload == "full" else None,
                     "work": f"{ALG_FLOPS_PER_CANDIDATE} flops x {stats['candidates']} candidates + "
                             f"{ALG_FLOPS_PER_HIT} flops x {stats['hits']} hits = {alg_flops:.4g} flops per launch",
                     "peak_source": f"{n_sms} SMs x 128 FP32 lanes x 2 flop x {sm_max:.0f} MHz (unit counts and "
                                    f"max clock; no FP32 figure is measured)",
                     "implementation_count": {"flops": impl_flops, "achieved": achieved_impl,
                                              "frac": achieved_impl / peak_tflops}},
        "e2e": {"value": ws * 1000.0 / ms_e2e, "unit": UNIT, "h2d_bytes_per_step": 184,
                "d2h_bytes_per_step": r.plan.pixels * 16},
        "gpu_launches": K * kernels_fwd,
        "clocks": clocks,
        "cpu_baseline": cpu,
        "cpu_baseline_tile_lists": cpu_tiles,
    }
    del r, ds, flush, grads, target, host_rgb, host_T, rgb, T, last
    torch.cuda.empty_cache()
    line["serve"] = None if args.no_serve else serve_bench(args, local)
    print(json.dumps(line), flush=True)


SERVE_SIZES = [(640, 360), (1280, 720), (1920, 1080), (3840, 2160)]
SERVE_PROBS = [0.3, 0.3, 0.3, 0.1]


def serve_bench(args, local: int):
    """Serving workload: a 2M-cell capture-shaped scene stays resident;
    requests arrive Poisson at `rate`/s with resolutions drawn from
    SERVE_SIZES; admission by a 40 GB tile/sort memory budget.  Both the
    continuous-batching server and the plain one-view-per-launch renderer
    (one request per batch, one in flight, no graphs) run the same arrival
    trace; then each runs a closed-loop burst to saturation."""
    import torch
    from paper_2604_24994_gb300 import DeviceScene, inputs
    from paper_2604_24994_gb300.serve import Server

    t0 = time.time()
    n_cells = 2_000_000 if args.workload in ("full", "serve") else 400_000
    sc = inputs.capture_scene(n_cells, seed=0, K=32)
    gen_s = time.time() - t0
    ds = DeviceScene.from_numpy(sc, "cuda")
    rng = np.random.default_rng(0)
    dur = args.serve_seconds
    rate = args.serve_rate
    n_req = int(rate * dur * 1.2) + 64
    arrivals = np.cumsum(rng.exponential(1.0 / rate, n_req))
    arrivals = arrivals[arrivals < dur]
    cams = inputs.random_sphere_cameras(rng, max(len(arrivals), args.serve_burst) + 400, 2.0, 6.0, SERVE_SIZES,
                                        SERVE_PROBS)
    ring = {}
    for (w, h) in SERVE_SIZES:  # output buffers, reused round-robin
        ring[(w, h)] = [(torch.empty((w * h, 3), device="cuda"), torch.empty(w * h, device="cuda"))
                        for _ in range(12 if w < 3840 else 4)]
    ctr = {k: 0 for k in ring}

    def outputs(cam):
        k = (cam.width, cam.height)
        o = ring[k][ctr[k] % len(ring[k])]
        ctr[k] += 1
        return o

    budget = int(args.serve_budget_gb * (1 << 30))

    def run(opts, open_loop: bool):
        srv = Server(ds, budget, **opts)
        # warm-up: every resolution alone and in a batch (graph capture, first launches)
        ids = [srv.submit(c, *outputs(c)) for c in cams[-40:]]
        for i in ids:
            srv.wait(i, 600000)
        srv.reset_stats()
        ids = []
        if open_loop:
            start = time.perf_counter()
            for a, cam in zip(arrivals, cams):
                delay = start + a - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
                st, rid = srv.try_submit(cam, *outputs(cam))
                if st == 0:
                    ids.append(rid)
        else:  # closed loop: a burst that keeps every slot busy
            for cam in cams[:args.serve_burst]:
                ids.append(srv.submit(cam, *outputs(cam)))
        for i in ids:
            srv.wait(i, 600000)
        rep = srv.report()
        srv.close()
        return rep

    q = int(2 * rate)  # at most two seconds of backlog are admitted; the rest is rejected (counted)
    batched = dict(max_batch_views=8, slots=3, use_graphs=True, max_queue=q)
    plain = dict(max_batch_views=1, slots=1, use_graphs=False, max_queue=q)
    out = {"workload": f"{n_cells:,}-cell capture-shaped scene resident; Poisson {rate}/s for {dur} s "
                       f"({len(arrivals)} requests); resolutions 640x360/1280x720/1920x1080/3840x2160 with "
                       f"p=.3/.3/.3/.1; cameras on spheres of radius 2-6 looking at the origin; "
                       f"{args.serve_budget_gb:.0f} GB tile/sort budget",
           "scene_generation_s": round(gen_s, 1)}
    keep = ("p50_ms", "p99_ms", "mean_ms", "requests_per_s", "mpix_per_s", "mean_batch_views", "completed",
            "rejected", "batches", "graph_replays", "graph_updates")
    for name, opts in (("batched", batched), ("plain", plain)):
        rep_open = run(opts, True)
        rep_sat = run(opts, False)
        out[name] = {"open_loop": {k: rep_open[k] for k in keep},
                     "saturation": {k: rep_sat[k] for k in ("requests_per_s", "mpix_per_s", "p50_ms", "p99_ms",
                                                            "mean_batch_views")},
                     "opts": opts}
    return out


def run_serve_only(args):
    """The serving workload alone (both servers, open loop for
    --serve-seconds, then a closed-loop burst of --serve-burst requests):
    one JSON line, not the benchmark line."""
    import torch
    from paper_2604_24994_gb300 import build
    torch.cuda.set_device(0)
    build.build()
    print(json.dumps({"workload": "serve", "serve": serve_bench(args, 0)}), flush=True)


def run_large(args):
    """The large differentiable workload: 5M cells (capture recipe), 48
    neighbours, four 3840x2160 views on a ring, forward+backward with the
    per-pixel (T, last) checkpoint.  Times the step and reports peak device
    memory for the default plan (checkpoint + the forward's hit records),
    for a plan laid out without hit records (checkpoint only: the backward
    re-tests every listed cell), and for the variant that stores every
    segment instead of replaying it (pf_plan_store_segments), which fits for
    one of the four views: the three plans are also measured on that view
    alone.  Prints one JSON line (not the benchmark line)."""
    import torch
    from paper_2604_24994_gb300 import DeviceScene, Renderer, build, inputs
    from paper_2604_24994_gb300.dataparallel import ring_view
    build.build()
    t0 = time.time()
    sc = inputs.capture_scene(5_000_000, seed=0, K=48)
    gen_s = time.time() - t0
    cams = [ring_view(v, 3840, 2160, radius=3.0, n_ring=4) for v in range(4)]
    ds = DeviceScene.from_numpy(sc, "cuda")
    del sc
    stream = torch.cuda.current_stream()
    free_total = torch.cuda.mem_get_info()

    def measure(name, views, rec, store=0):
        # size the instance capacity once, then lay the plan out at that size
        r = Renderer(ds.n, ds.k, views, hit_records=False)
        r.bin(ds, sync=True)
        cap = int(r.n_instances * 1.02) + 4096
        del r
        torch.cuda.empty_cache()
        torch.cuda.reset_peak_memory_stats()
        base = torch.cuda.memory_allocated()
        px = sum(c.width * c.height for c in views)
        gen = torch.Generator(device="cuda").manual_seed(0)
        target = torch.rand((px, 3), device="cuda", generator=gen)
        r = Renderer(ds.n, ds.k, views, capacity=cap, hit_records=rec, store_segments=store)
        rgb = torch.empty((px, 3), device="cuda")
        T = torch.empty(px, device="cuda")
        last = torch.empty(px, dtype=torch.int32, device="cuda")
        grads = {k: torch.zeros_like(v) for k, v in ds.params.items()}

        def step():
            r.bin(ds, sync=False)
            c, t, l = r.render_fwd(ds, out=(rgb, T, last))
            r.backward(ds, 2.0 * (c - target), None, t, l, grads=grads)

        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(args.steps):
            step()
        b.record(stream)
        b.synchronize()
        res = {"views": len(views), "ms_fwd_bwd": a.elapsed_time(b) / args.steps,
               "workspace_gb": r.plan.ws_bytes / 1e9,
               "peak_allocated_gb": torch.cuda.max_memory_allocated() / 1e9,
               "peak_above_scene_gb": (torch.cuda.max_memory_allocated() - base) / 1e9}
        if rec:
            hc = r.hit_counts()
            res["hits_per_pixel"] = float(hc.mean())
            res["max_hits_per_pixel"] = int(hc.max())
        if store:
            res["stored_segments_per_pixel"] = store
        del r, rgb, T, last, grads, target
        torch.cuda.empty_cache()
        return res

    out = {}
    out["checkpoint+hit_records"] = measure("checkpoint+hit_records", cams, True)
    out["checkpoint_only"] = measure("checkpoint_only", cams, False)
    one = cams[:1]
    out["one_view"] = {"checkpoint+hit_records": measure("1v hit records", one, True),
                       "checkpoint_only": measure("1v checkpoint", one, False)}
    # store every segment: the capacity per pixel is the largest hit count of that view
    mh = out["one_view"]["checkpoint+hit_records"]["max_hits_per_pixel"]
    need = one[0].width * one[0].height * mh * 16
    all4 = out["checkpoint+hit_records"]["max_hits_per_pixel"] * sum(c.width * c.height for c in cams) * 16
    try:
        out["one_view"]["store_every_segment"] = measure("1v store", one, True, store=mh)
    except torch.OutOfMemoryError:
        torch.cuda.empty_cache()
        out["one_view"]["store_every_segment"] = f"does not fit: {need / 1e9:.1f} GB of segments"
    if all4 <= free_total[1] * 0.6:
        out["store_every_segment"] = measure("store", cams, True,
                                             store=out["checkpoint+hit_records"]["max_hits_per_pixel"])
    line = {"workload": "5,000,000 cells (capture recipe), 48 neighbours, 4 views 3840x2160 on a ring of radius 3",
            "device_memory_gb": free_total[1] / 1e9,
            "checkpoint_bytes_per_pixel": 8, "store_bytes_per_segment": 16,
            "store_every_segment_one_view_gb": need / 1e9,
            "store_every_segment_four_views_gb": all4 / 1e9,
            "store_every_segment_four_views": "not run: the per-pixel store at the largest hit count of the "
                                              "four views exceeds the device's memory beside the scene and workspace"
            if all4 > free_total[1] * 0.6 else "fits",
            "steps": args.steps, "warmup": args.warmup, "scene_generation_s": round(gen_s, 1), **out}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--workload", default="full", choices=["full", "small", "large", "serve"])
    ap.add_argument("--serve-seconds", type=float, default=60.0)
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-budget-gb", type=float, default=40.0)
    ap.add_argument("--serve-burst", type=int, default=300)
    ap.add_argument("--no-serve", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "large":
        run_large(args)
    elif args.workload == "serve":
        run_serve_only(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
