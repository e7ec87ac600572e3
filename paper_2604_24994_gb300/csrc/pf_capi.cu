// C ABI entry points: plans, workspace layout, argument checks.
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <math.h>
#include <string.h>

#include <new>

#include "pf_internal.cuh"

namespace pf {

static thread_local char g_err[512];

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
}

pf_status cuda_status(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return PF_OK;
    set_error("%s: %s", what, cudaGetErrorString(e));
    return PF_ERR_CUDA;
}

WS Plan::ws(void *base) const {
    char *b = (char *)base;
    WS w;
    w.views = (ViewDev *)(b + L.views);
    w.cellrec = (float *)(b + L.cellrec);
    w.cellnp = (int32_t *)(b + L.cellnp);
    w.planes = (float4 *)(b + L.planes);
    w.planes_lo = (float4 *)(b + L.planes_lo);
    w.plane_nb = (int2 *)(b + L.plane_nb);
    w.viewrec = (float *)(b + L.viewrec);
    w.rect = (ushort4 *)(b + L.rect);
    w.key = (unsigned long long *)(b + L.key);
    w.cnt = (uint32_t *)(b + L.cnt);
    w.celloff = (uint32_t *)(b + L.celloff);
    w.diff = (int32_t *)(b + L.diff);
    w.tile_start = (uint32_t *)(b + L.tile_start);
    w.tile_cursor = (uint32_t *)(b + L.tile_cursor);
    w.tile_order = (uint32_t *)(b + L.tile_order);
    w.scan_tmp = (uint32_t *)(b + L.scan_tmp);
    w.inst_key = (unsigned long long *)(b + L.inst_key);
    w.inst_cell = (uint32_t *)(b + L.inst_cell);
    w.inst_sorted = (uint32_t *)(b + L.inst_sorted);
    w.sort_tmp_key = (unsigned long long *)(b + L.sort_tmp_key);
    w.sort_tmp_cell = (uint32_t *)(b + L.sort_tmp_cell);
    w.counters = (Counters *)(b + L.counters);
    w.acc = (float *)(b + L.acc);
    const bool rec = !fwd_only && !no_hit_records;
    w.hitmask = rec ? (uint32_t *)(b + L.hitmask) : nullptr;
    w.hitkind = rec ? (uint16_t *)(b + L.hitkind) : nullptr;
    w.hitcount = rec ? (uint32_t *)(b + L.hitcount) : nullptr;
    w.segrec = rec && seg_cap > 0 ? (float4 *)(b + L.segrec) : nullptr;
    w.pw = (float4 *)(b + L.pw);
    if (external_scene) {
        const SceneLayout S = make_scene_layout(n, k);
        char *sb = (char *)scene_ws;
        w.cellrec = (float *)(sb + S.cellrec);
        w.cellnp = (int32_t *)(sb + S.cellnp);
        w.planes = (float4 *)(sb + S.planes);
        w.planes_lo = (float4 *)(sb + S.planes_lo);
        w.plane_nb = (int2 *)(sb + S.plane_nb);
    }
    return w;
}

SceneLayout make_scene_layout(int32_t n, int32_t k) {
    SceneLayout S;
    uint64_t o = 0;
    auto take = [&](uint64_t bytes) {
        uint64_t at = o;
        o = align_up(o + bytes, 256);
        return at;
    };
    S.cellrec = take((uint64_t)n * CELLREC_F * 4);
    S.cellnp = take((uint64_t)n * 4);
    S.planes = take((uint64_t)n * k * 16);
    S.plane_nb = take((uint64_t)n * k * 8);
    S.planes_lo = take((uint64_t)n * k * 16);
    S.total = o;
    return S;
}

bool camera_ok(const pf_camera &c) {
    if (c.width < 1 || c.height < 1 || c.width > 16384 || c.height > 16384) return false;
    if (!(c.fx > 0) || !(c.fy > 0)) return false;
    if (c.model != PF_PINHOLE && c.model != PF_FISHEYE) return false;
    for (int i = 0; i < 9; i++)
        if (!isfinite(c.rot[i])) return false;
    for (int i = 0; i < 3; i++)
        if (!isfinite(c.origin[i])) return false;
    return isfinite(c.cx) && isfinite(c.cy) && isfinite(c.fx) && isfinite(c.fy);
}

void fill_views(Plan *p, const pf_camera *cams) {
    int64_t tb = 0, pb = 0, db = 0;
    for (int v = 0; v < p->nv; v++) {
        ViewDev &d = p->views_host[v];
        const pf_camera &c = cams[v];
        memcpy(d.rot, c.rot, sizeof d.rot);
        memcpy(d.origin, c.origin, sizeof d.origin);
        d.fx = c.fx;
        d.fy = c.fy;
        d.cx = c.cx;
        d.cy = c.cy;
        d.ifx = 1.0 / c.fx;
        d.ify = 1.0 / c.fy;
        // frustum side planes through the camera centre (host IEEE double,
        // no contraction: the CPU binning evaluates the same expressions)
        d.kl = (0.0 - c.cx) / c.fx;
        d.kr = ((double)c.width - c.cx) / c.fx;
        d.ku = (0.0 - c.cy) / c.fy;
        d.kd = ((double)c.height - c.cy) / c.fy;
        d.skl = sqrt(1.0 + d.kl * d.kl);
        d.skr = sqrt(1.0 + d.kr * d.kr);
        d.sku = sqrt(1.0 + d.ku * d.ku);
        d.skd = sqrt(1.0 + d.kd * d.kd);
        for (int k = 0; k < 9; k++) d.rotf[k] = (float)c.rot[k];
        d.fxf = (float)c.fx;
        d.fyf = (float)c.fy;
        d.cxf = (float)c.cx;
        d.cyf = (float)c.cy;
        for (int k = 0; k < 3; k++) {
            d.ohi[k] = (float)c.origin[k];
            d.olo[k] = (float)(c.origin[k] - (double)d.ohi[k]);
        }
        d.width = c.width;
        d.height = c.height;
        d.model = c.model;
        d.tiles_x = (c.width + TILE - 1) / TILE;
        d.tiles_y = (c.height + TILE - 1) / TILE;
        d.tile_base = tb;
        d.pix_base = pb;
        d.diff_base = db;
        d.out_rgb = nullptr;
        d.out_T = nullptr;
        d.out_last = nullptr;
        tb += (int64_t)d.tiles_x * d.tiles_y;
        pb += (int64_t)c.width * c.height;
        db += (int64_t)(d.tiles_x + 1) * (d.tiles_y + 1);
    }
    p->total_tiles = tb;
    p->total_pixels = pb;
    p->total_diff = db;
}

void make_layout(Plan *p) {
    Layout &L = p->L;
    uint64_t o = 0;
    auto take = [&](uint64_t bytes) {
        uint64_t at = o;
        o = align_up(o + bytes, 256);
        return at;
    };
    uint64_t n = (uint64_t)p->n, k = (uint64_t)p->k, nv = (uint64_t)p->nv, cap = p->cap;
    uint64_t T = (uint64_t)p->total_tiles;
    L.views = take(nv * sizeof(ViewDev));
    const uint64_t ns = p->external_scene ? 0 : n;
    L.cellrec = take(ns * CELLREC_F * 4);
    L.cellnp = take(ns * 4);
    L.planes = take(ns * k * 16);
    L.plane_nb = take(ns * k * 8);
    L.planes_lo = take(ns * k * 16);
    L.viewrec = take(nv * n * VIEWREC_F * 4);
    L.rect = take(nv * n * 8);
    L.key = take(nv * n * 8);
    L.cnt = take(nv * n * 4);
    L.celloff = take(nv * n * 4);
    L.diff = take((uint64_t)p->total_diff * 4 * DIFF_REP);
    L.tile_start = take((T + 1) * 4);
    L.tile_cursor = take(T * 4);
    L.tile_order = take(T * 4);
    uint64_t m = nv * n > T ? nv * n : T;
    L.scan_tmp_elems = m / 2048 + 2;
    L.scan_tmp = take(L.scan_tmp_elems * 4);
    L.inst_key = take(cap * 8);
    L.inst_cell = take(cap * 4);
    L.inst_sorted = take(cap * 4);
    L.sort_tmp_key = take(cap * 8);
    L.sort_tmp_cell = take(cap * 4);
    L.counters = take(sizeof(Counters));
    L.acc = take((p->fwd_only ? 0 : n) * ACC_F * 4);
    L.pw = take(n * 16);
    // hit records last, so that dropping them moves no other region
    const bool rec = !p->fwd_only && !p->no_hit_records;
    L.hitmask = take(rec ? (uint64_t)(TILE_PIX / 32) * mask_batches(*p) * 32 * 4 : 0);
    L.hitkind = take(rec ? (uint64_t)p->total_pixels * HIT_CAP * 2 : 0);
    L.hitcount = take(rec ? (uint64_t)p->total_pixels * 4 : 0);
    L.segrec = take(rec && p->seg_cap > 0 ? (uint64_t)p->total_pixels * (uint64_t)p->seg_cap * 16 : 0);
    L.total = o;
}

bool scene_ok(const pf_scene *s, const Plan *p) {
    if (!s) return false;
    if (s->n_cells != p->n || s->k_nbr != p->k) {
        set_error("scene has N=%d K=%d but the plan N=%d K=%d", s->n_cells, s->k_nbr, p->n, p->k);
        return false;
    }
    if (p->n == 0) return true;
    if (!s->pos || !s->w || !s->R || !s->sigma || !s->rgb || !s->normal || !s->offset || !s->tex ||
        (p->k > 0 && !s->nbr)) {
        set_error("null scene pointer");
        return false;
    }
    if (((uintptr_t)s->tex & 15) != 0 || ((uintptr_t)s->disp & 15) != 0 || ((uintptr_t)s->sites & 15) != 0) {
        set_error("tex, disp and sites must be 16-byte aligned");
        return false;
    }
    if (s->n_sites != 0 && s->n_sites != 4 && s->n_sites != 8) {
        set_error("n_sites must be 0 or 4 (four detail sites) or 8, not %d", s->n_sites);
        return false;
    }
    return true;
}

}  // namespace pf

using namespace pf;

struct pf_plan : public Plan {};

extern "C" {

const char *pf_status_string(pf_status s) {
    switch (s) {
        case PF_OK: return "ok";
        case PF_ERR_INVALID_ARG: return "invalid argument";
        case PF_ERR_CAPACITY: return "instance capacity exceeded";
        case PF_ERR_CUDA: return "CUDA error";
        case PF_ERR_TIMEOUT: return "timed out";
        case PF_ERR_BUSY: return "busy";
        case PF_ERR_NOT_FOUND: return "not found";
    }
    return "unknown status";
}

const char *pf_last_error_message(void) { return g_err; }

pf_status pf_plan_create(int32_t n_cells, int32_t k_nbr, const pf_camera *cams, int32_t n_views,
                         uint64_t inst_capacity, pf_plan **out) {
    g_err[0] = 0;
    if (!out || n_cells < 0 || k_nbr < 0 || k_nbr > MAX_K || n_views < 1 || !cams) {
        set_error("pf_plan_create: bad arguments");
        return PF_ERR_INVALID_ARG;
    }
    if (inst_capacity > 0xF0000000ull) {
        set_error("pf_plan_create: capacity above 2^32 - 2^28 instances");
        return PF_ERR_INVALID_ARG;
    }
    for (int v = 0; v < n_views; v++)
        if (!camera_ok(cams[v])) {
            set_error("pf_plan_create: camera %d invalid", v);
            return PF_ERR_INVALID_ARG;
        }
    pf_plan *p = new (std::nothrow) pf_plan();
    if (!p) return PF_ERR_INVALID_ARG;
    p->n = n_cells;
    p->k = k_nbr;
    p->nv = n_views;
    p->cap = inst_capacity;
    p->stats = 0;
    p->views_host = (ViewDev *)calloc((size_t)n_views, sizeof(ViewDev));
    if (!p->views_host) {
        delete p;
        set_error("pf_plan_create: host allocation failed");
        return PF_ERR_INVALID_ARG;
    }
    fill_views(p, cams);
    make_layout(p);
    *out = p;
    return PF_OK;
}

void pf_plan_destroy(pf_plan *p) {
    if (!p) return;
    free(p->views_host);
    delete p;
}

pf_status pf_plan_workspace_bytes(const pf_plan *p, uint64_t *bytes) {
    if (!p || !bytes) return PF_ERR_INVALID_ARG;
    *bytes = p->L.total;
    return PF_OK;
}

pf_status pf_plan_pixels(const pf_plan *p, uint64_t *pixels) {
    if (!p || !pixels) return PF_ERR_INVALID_ARG;
    *pixels = (uint64_t)p->total_pixels;
    return PF_OK;
}

pf_status pf_plan_set_cameras(pf_plan *p, const pf_camera *cams, int32_t n_views) {
    if (!p || !cams || n_views != p->nv) return PF_ERR_INVALID_ARG;
    for (int v = 0; v < n_views; v++) {
        if (!camera_ok(cams[v]) || cams[v].width != p->views_host[v].width ||
            cams[v].height != p->views_host[v].height) {
            set_error("pf_plan_set_cameras: camera %d invalid or resolution changed", v);
            return PF_ERR_INVALID_ARG;
        }
    }
    fill_views(p, cams);
    return PF_OK;
}

pf_status pf_plan_set_record_hits(pf_plan *p, int32_t enable) {
    if (!p) return PF_ERR_INVALID_ARG;
    if (enable && p->no_hit_records) {
        set_error("pf_plan_set_record_hits: the plan's workspace has no hit records (pf_plan_omit_hit_records)");
        return PF_ERR_INVALID_ARG;
    }
    p->record_hits = enable != 0;
    return PF_OK;
}

pf_status pf_plan_omit_hit_records(pf_plan *p) {
    if (!p) return PF_ERR_INVALID_ARG;
    p->no_hit_records = true;
    p->record_hits = false;
    p->masks_valid = false;
    make_layout(p);
    return PF_OK;
}

pf_status pf_plan_store_segments(pf_plan *p, int32_t max_hits) {
    if (!p || max_hits < 0) return PF_ERR_INVALID_ARG;
    if (max_hits > 0 && (p->no_hit_records || p->fwd_only)) {
        set_error("pf_plan_store_segments: the plan has no hit records (pf_plan_omit_hit_records)");
        return PF_ERR_INVALID_ARG;
    }
    p->seg_cap = max_hits;
    p->masks_valid = false;
    make_layout(p);
    return PF_OK;
}

pf_status pf_read_hit_counts(pf_plan *p, void *ws, uint32_t *counts, void *stream) {
    g_err[0] = 0;
    if (!p || !ws || !counts) return PF_ERR_INVALID_ARG;
    WS w = p->ws(ws);
    if (!w.hitcount) {
        set_error("pf_read_hit_counts: the plan has no hit records");
        return PF_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    pf_status s = cuda_status(cudaMemcpyAsync(counts, w.hitcount, 4 * (size_t)p->total_pixels, cudaMemcpyDeviceToHost, st),
                              "read hit counts");
    if (!s) s = cuda_status(cudaStreamSynchronize(st), "read hit counts sync");
    return s;
}

pf_status pf_plan_enable_stats(pf_plan *p, int32_t enable) {
    if (!p) return PF_ERR_INVALID_ARG;
    p->stats = enable ? 1 : 0;
    return PF_OK;
}

pf_status pf_plan_read_stats(pf_plan *p, void *ws, pf_stats *out, void *stream) {
    if (!p || !ws || !out) return PF_ERR_INVALID_ARG;
    WS w = p->ws(ws);
    Counters c;
    cudaStream_t st = (cudaStream_t)stream;
    pf_status s = cuda_status(cudaMemcpyAsync(&c, w.counters, sizeof c, cudaMemcpyDeviceToHost, st), "read stats");
    if (s) return s;
    s = cuda_status(cudaMemsetAsync(w.counters->stats, 0, sizeof c.stats, st), "reset stats");
    if (s) return s;
    s = cuda_status(cudaStreamSynchronize(st), "read stats sync");
    if (s) return s;
    out->instances = c.total_inst;
    out->candidates = c.stats[0];
    out->hits = c.stats[1];
    out->planes = c.stats[2];
    out->refined = c.stats[3];
    out->sphere_pass = c.stats[4];
    out->warp_candidates = c.stats[5];
    out->warp_passes = c.stats[6];
    out->warp_hits = c.stats[7];
    out->wait_errors = c.wait_errors;
    return PF_OK;
}

pf_status pf_prepare(const pf_scene *scene, pf_plan *p, void *ws, void *stream) {
    g_err[0] = 0;
    if (!p || !ws || !scene_ok(scene, p)) return PF_ERR_INVALID_ARG;
    p->masks_valid = false;
    WS w = p->ws(ws);
    return cuda_status(launch_prepare(*scene, *p, w, (cudaStream_t)stream), "pf_prepare");
}

pf_status pf_project(const pf_scene *scene, pf_plan *p, void *ws, void *stream) {
    g_err[0] = 0;
    if (!p || !ws || !scene_ok(scene, p)) return PF_ERR_INVALID_ARG;
    p->masks_valid = false;
    WS w = p->ws(ws);
    cudaStream_t st = (cudaStream_t)stream;
    pf_status s = cuda_status(
        cudaMemcpyAsync(w.views, p->views_host, sizeof(ViewDev) * p->nv, cudaMemcpyHostToDevice, st), "views");
    if (s) return s;
    return cuda_status(launch_project(*scene, *p, w, st), "pf_project");
}

pf_status pf_bin_sort(pf_plan *p, void *ws, uint64_t *n_instances, void *stream) {
    g_err[0] = 0;
    if (!p || !ws) return PF_ERR_INVALID_ARG;
    p->masks_valid = false;
    WS w = p->ws(ws);
    cudaStream_t st = (cudaStream_t)stream;
    pf_status s = cuda_status(launch_bin_sort(*p, w, st), "pf_bin_sort");
    if (s || !n_instances) return s;
    Counters c;
    s = cuda_status(cudaMemcpyAsync(&c, w.counters, sizeof c, cudaMemcpyDeviceToHost, st), "pf_bin_sort count");
    if (s) return s;
    s = cuda_status(cudaStreamSynchronize(st), "pf_bin_sort sync");
    if (s) return s;
    *n_instances = c.total_inst;
    if (c.overflow) {
        set_error("pf_bin_sort: %llu instances, capacity %llu", (unsigned long long)c.total_inst,
                  (unsigned long long)p->cap);
        return PF_ERR_CAPACITY;
    }
    return PF_OK;
}

pf_status pf_render_fwd(const pf_scene *scene, pf_plan *p, void *ws, float *rgb, float *T, uint32_t *last,
                        void *stream) {
    g_err[0] = 0;
    if (!p || !ws || !scene_ok(scene, p) || !rgb || !T || !last) return PF_ERR_INVALID_ARG;
    WS w = p->ws(ws);
    if (ext_face(*scene) && p->stats && p->n > 0) {
        set_error("pf_render_fwd: no stats pass for an extended face model");
        return PF_ERR_INVALID_ARG;
    }
    const bool record = p->record_hits && !p->stats && w.hitmask != nullptr;
    pf_status s =
        cuda_status(launch_render_fwd(*scene, *p, w, rgb, T, last, record, (cudaStream_t)stream), "pf_render_fwd");
    p->masks_valid = !s && record;
    return s;
}

pf_status pf_render_fwd_contrib(const pf_scene *scene, pf_plan *p, void *ws, float *rgb, float *T, uint32_t *last,
                                float *contrib_sparse, float *contrib_normal, void *stream) {
    g_err[0] = 0;
    if (!p || !ws || !scene_ok(scene, p) || !rgb || !T || !last) return PF_ERR_INVALID_ARG;
    if (p->n > 0 && (!contrib_sparse || !contrib_normal)) {
        set_error("pf_render_fwd_contrib: null contribution array");
        return PF_ERR_INVALID_ARG;
    }
    WS w = p->ws(ws);
    const bool record = p->record_hits && w.hitmask != nullptr;
    pf_status s = cuda_status(launch_render_fwd(*scene, *p, w, rgb, T, last, record, (cudaStream_t)stream,
                                                p->n > 0 ? contrib_sparse : nullptr, p->n > 0 ? contrib_normal : nullptr),
                              "pf_render_fwd_contrib");
    p->masks_valid = !s && record;
    return s;
}

static pf_status render_bwd(const char *who, const pf_scene *scene, pf_plan *p, void *ws, const float *dL_drgb,
                            const float *dL_dT, const float *T, const uint32_t *last, const float *w_sparse,
                            const float *w_normal, const pf_scene_grad *g, void *stream) {
    g_err[0] = 0;
    if (!p || !ws || !scene_ok(scene, p) || !dL_drgb || !T || !last || !g) return PF_ERR_INVALID_ARG;
    if (p->n > 0 && (!g->pos || !g->w || !g->R || !g->sigma || !g->rgb || !g->normal || !g->offset || !g->tex)) {
        set_error("%s: null gradient pointer", who);
        return PF_ERR_INVALID_ARG;
    }
    if (scene->disp && p->n > 0 && !g->disp) {
        set_error("%s: a displaced scene needs grad->disp", who);
        return PF_ERR_INVALID_ARG;
    }
    if (scene->sites && p->n > 0 && !g->sites) {
        set_error("%s: learned sites need grad->sites", who);
        return PF_ERR_INVALID_ARG;
    }
    if (scene->sv && p->n > 0 && !g->sv) {
        set_error("%s: view-dependent site colours need grad->sv", who);
        return PF_ERR_INVALID_ARG;
    }
    WS w = p->ws(ws);
    return cuda_status(launch_render_bwd(*scene, *p, w, dL_drgb, dL_dT, T, last, *g, p->masks_valid,
                                         (cudaStream_t)stream, w_sparse, w_normal),
                       who);
}

pf_status pf_render_bwd(const pf_scene *scene, pf_plan *p, void *ws, const float *dL_drgb, const float *dL_dT,
                        const float *T, const uint32_t *last, const pf_scene_grad *g, void *stream) {
    return render_bwd("pf_render_bwd", scene, p, ws, dL_drgb, dL_dT, T, last, nullptr, nullptr, g, stream);
}

pf_status pf_render_bwd_contrib(const pf_scene *scene, pf_plan *p, void *ws, const float *dL_drgb,
                                const float *dL_dT, const float *T, const uint32_t *last, const float *w_sparse,
                                const float *w_normal, const pf_scene_grad *g, void *stream) {
    if (p && p->n > 0 && (!w_sparse || !w_normal)) {
        g_err[0] = 0;
        set_error("pf_render_bwd_contrib: null contribution weights");
        return PF_ERR_INVALID_ARG;
    }
    return render_bwd("pf_render_bwd_contrib", scene, p, ws, dL_drgb, dL_dT, T, last, w_sparse, w_normal, g,
                      stream);
}

pf_status pf_connect(const pf_scene *scene, float *loss, float *grad_pos, float *grad_R, void *stream) {
    g_err[0] = 0;
    if (!scene || !loss || scene->n_cells < 0 || scene->k_nbr < 0 || (!grad_pos) != (!grad_R)) {
        set_error("pf_connect: invalid argument");
        return PF_ERR_INVALID_ARG;
    }
    if (scene->n_cells > 0 && (!scene->pos || !scene->R || (scene->k_nbr > 0 && !scene->nbr))) {
        set_error("pf_connect: null scene pointer");
        return PF_ERR_INVALID_ARG;
    }
    return cuda_status(launch_connect(*scene, loss, grad_pos, grad_R, (cudaStream_t)stream), "pf_connect");
}

pf_status pf_read_bins(pf_plan *p, void *ws, uint32_t *tile_start, uint32_t *cells, uint64_t *keys,
                       uint16_t *rects, void *stream) {
    g_err[0] = 0;
    if (!p || !ws || !tile_start || !cells) return PF_ERR_INVALID_ARG;
    WS w = p->ws(ws);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t VN = (size_t)p->n * p->nv;
    pf_status s = cuda_status(cudaMemcpyAsync(tile_start, w.tile_start, 4 * (size_t)(p->total_tiles + 1),
                                              cudaMemcpyDeviceToHost, st), "read tile_start");
    if (!s && p->cap)
        s = cuda_status(cudaMemcpyAsync(cells, w.inst_sorted, 4 * (size_t)p->cap, cudaMemcpyDeviceToHost, st),
                        "read cells");
    if (!s && keys && VN)
        s = cuda_status(cudaMemcpyAsync(keys, w.key, 8 * VN, cudaMemcpyDeviceToHost, st), "read keys");
    if (!s && rects && VN)
        s = cuda_status(cudaMemcpyAsync(rects, w.rect, 8 * VN, cudaMemcpyDeviceToHost, st), "read rects");
    if (!s) s = cuda_status(cudaStreamSynchronize(st), "read bins sync");
    return s;
}

}  // extern "C"
