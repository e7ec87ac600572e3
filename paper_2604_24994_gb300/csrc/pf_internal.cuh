// Internal definitions shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

#include "powerfoam.h"

namespace pf {

constexpr int TILE = 16;               // tile edge in pixels
constexpr int TILE_PIX = TILE * TILE;  // one thread per pixel
constexpr int BATCH = 32;              // cells staged per shared-memory batch
constexpr int MAX_K = 64;              // neighbour list width limit
constexpr int CELLREC_F = 32;          // floats per view-independent cell record
constexpr int VIEWREC_F = 8;           // floats per (view, cell) record: m hi, Rt^2, m lo, D threshold
constexpr int ACC_F = 32;              // gradient accumulator floats per cell
constexpr int HIT_CAP = 256;           // recorded hits per pixel (later ones are re-clipped)
constexpr float T_EPS = 1e-6f;         // forward stops once T drops below this
constexpr float X_CAP = 60.0f;         // sigma * l is capped (alpha = 1 - e^-60)
constexpr float KAPPA = 6.0f;          // soft-Voronoi sharpness, units of 1/R
constexpr float SITE = 1.0f / 3.0f;    // texture sites at (+-1/3, +-1/3) R
constexpr float SV_LAMBDA = 10.0f;     // sharpness of the spherical-Voronoi site colours

// Precision budget of the render's float segment ends (the rest of the
// budget for the forward's 1e-5 in T): an end whose float error bound could
// move sigma * l by more than REFINE_EPS is recomputed at higher precision.
constexpr float REFINE_EPS = 6e-6f;    // sigma * |error of a segment end| budget
constexpr float PLANE_ERR = 6e-7f;     // bound on |error| of a plane/face end, in units of (R + |s|)
constexpr float SPHERE_ERR = 6e-7f;    // bound on |error of D|, in units of R^2

// |D| below which the sphere's D = R^2 - |v|^2 is recomputed: where the
// chord 2 sqrt(D) moves sigma * l by more than REFINE_EPS for an error
// SPHERE_ERR R^2 in D, and never above the error itself.
__host__ __device__ inline float sphere_refine_threshold(float R, float sigma) {
    const float dthr = SPHERE_ERR * R * R * sigma * (1.0f / (2.0f * REFINE_EPS));
    const float t = SPHERE_ERR * R * R;
    return dthr * dthr > t ? dthr * dthr : t;
}

// Cell record layout (floats), one 128-byte line per cell.
enum : int {
    CR_N = 0,     // [0..2] unit normal, [3] offset
    CR_OFF = 3,
    CR_E1 = 4,    // [4..6] e1 / R,     [7] R
    CR_R = 7,
    CR_E2 = 8,    // [8..10] e2 / R,    [11] sigma
    CR_SIG = 11,
    CR_RGB = 12,  // [12..14] rgb,      [15] flags (bit 0: empty)
    CR_FLAGS = 15,
    CR_TEX = 16,  // [16..27] texture, site-major
    CR_NLO = 28,  // [28..30] low part of the unit normal (FP64 = hi + lo)
    CR_NLEN = 31  // [31] |n|
};

// Gradient accumulator layout (floats per cell).
enum : int {
    G_P = 0,     // [0..2] position
    G_W = 3,     // [3] weight
    G_R = 4,     // [4] bound radius
    G_SIG = 5,   // [5] density
    G_N = 6,     // [6..8] unit normal (projected to n in the finalize pass)
    G_OFF = 9,   // [9] offset
    G_TEX = 10,  // [10..21] texture (rgb is their sum)
    G_NB_A = 22, // [22..25] entry-side neighbour (p_j, w_j)
    G_NB_B = 26, // [26..29] exit-side neighbour
    G_USED = 22
};

// Copies of the per-view 2D difference grids that the projection's
// atomics are spread over (warp w of block b adds into copy (8 b + w) mod
// DIFF_REP); the tile-count pass sums them.
constexpr int DIFF_REP = 16;

// Per-view constants on the device.
struct ViewDev {
    double rot[9];
    double origin[3];
    double fx, fy, cx, cy;
    double ifx, ify;          // 1/fx, 1/fy
    double kl, kr, ku, kd;    // image-edge slopes x/z, y/z of the frustum side planes
    double skl, skr, sku, skd; // sqrt(1 + k^2) of each
    float rotf[9];            // rot, fx, fy, cx, cy rounded to float (the float tile box)
    float fxf, fyf, cxf, cyf;
    float ohi[3], olo[3];     // origin as a float pair: ohi = (float)origin, olo = (float)(origin - ohi)
    int32_t width, height;
    int32_t tiles_x, tiles_y;
    int32_t model;            // PF_PINHOLE or PF_FISHEYE
    int32_t pad_;
    int64_t tile_base;        // first global tile id of this view
    int64_t pix_base;         // first pixel of this view in the outputs
    int64_t diff_base;        // offset of this view's (tx+1)(ty+1) difference grid
    float *out_rgb;           // optional per-view outputs [H*W*3], [H*W], [H*W]
    float *out_T;             // (NULL: write into the concatenated outputs;
    uint32_t *out_last;       //  out_last NULL with out_rgb set: not written)
};

struct Counters {
    unsigned long long total_inst;  // instances required
    unsigned int overflow;          // 1 if total_inst > capacity
    unsigned int q_fwd;             // next entry of tile_order for the forward's CTAs
    unsigned int q_bwd;             // same for the backward
    unsigned int wait_errors;       // nonzero if a bounded wait of the pipelined forward ran out
    unsigned long long stats[8];    // pf_stats fields after `instances`
};

// Workspace layout (byte offsets into the caller's buffer).
struct Layout {
    uint64_t views, cellrec, cellnp, planes, plane_nb, viewrec, rect, key, cnt, celloff, diff, tile_start,
        tile_cursor, tile_order, scan_tmp, inst_key, inst_cell, inst_sorted, sort_tmp_key, sort_tmp_cell, counters,
        acc, planes_lo, hitmask, hitkind, hitcount, segrec, pw, total;
    uint64_t scan_tmp_elems;
};

struct Plan;

// Device pointers for one call, resolved from the layout.
struct WS {
    ViewDev *views;
    float *cellrec;        // [N][32]
    int32_t *cellnp;       // [N] relevant planes
    float4 *planes;        // [N][K] (unit a, plane distance g/|a|), float
    float4 *planes_lo;     // [N][K] low parts: FP64 plane = planes + planes_lo
    int2 *plane_nb;        // [N][K] (neighbour j, |a| as float bits)
    float *viewrec;        // [V][N][8]: m_hi.xyz, Rt^2, m_lo.xyz, pad
    ushort4 *rect;         // [V][N] tile rect (x0, y0, x1, y1), empty: x0 > x1
    unsigned long long *key;  // [V][N]
    uint32_t *cnt;         // [V][N] instances of the cell in the view
    uint32_t *celloff;     // [V][N] exclusive scan of cnt
    int32_t *diff;         // 2D difference grids of all views
    uint32_t *tile_start;  // [T+1]
    uint32_t *tile_cursor; // [T]
    uint32_t *tile_order;  // [T] tiles by decreasing list length (render order)
    uint32_t *scan_tmp;
    unsigned long long *inst_key;  // [cap]
    uint32_t *inst_cell;   // [cap]
    uint32_t *inst_sorted; // [cap]
    unsigned long long *sort_tmp_key;
    uint32_t *sort_tmp_cell;
    Counters *counters;
    float *acc;            // [N][32]
    float4 *pw;            // [N] (p, w) packed for prepare's neighbour gathers (scratch)
    uint16_t *hitkind;     // [pixels][HIT_CAP]: active constraints (entry, exit) of the pixel's
                           // first HIT_CAP hits in list order, 7 bits each, kind + 3
    uint32_t *hitcount;    // [pixels] hits the forward composited
    uint32_t *hitmask;     // [8][batch slots][32] per warp of a tile, batch of its list and
                           // pixel: bit j set if the forward's segment in cell j was non-empty
    float4 *segrec;        // [pixels][seg_cap] stored segments of the pixel's first hits in list
                           // order: (entry, exit, T before the segment, active constraints as bits)
};

struct Plan {
    int32_t n, k, nv;
    uint64_t cap;
    int64_t total_tiles, total_pixels, total_diff;
    ViewDev *views_host;   // host copy, uploaded by pf_project
    Layout L;
    int stats;
    // Optional: the view-independent cell records (cellrec, cellnp, planes,
    // plane_nb) live in a separate, shared buffer laid out by make_scene_layout
    // (the server prepares a resident scene once); then L omits them.
    void *scene_ws = nullptr;
    bool external_scene = false;
    bool fwd_only = false;   // omit the gradient accumulators and hit masks
    // hit masks in the workspace belong to the current bins: set by
    // pf_render_fwd, cleared by anything that changes the bins
    bool masks_valid = false;
    bool record_hits = true;   // pf_plan_set_record_hits
    bool no_hit_records = false;  // pf_plan_omit_hit_records: the layout has no hit-record regions
    int32_t seg_cap = 0;     // pf_plan_store_segments: stored segments per pixel (0: none)
    WS ws(void *base) const;
};

// Hit-mask batch slots per warp: every batch of every tile list gets one
// (see hitmask_slot in the renderer).
inline int64_t mask_batches(const Plan &p) { return (int64_t)(p.cap / BATCH) + p.total_tiles + 1; }

// Offsets of the view-independent records in a scene-only buffer.
struct SceneLayout {
    uint64_t cellrec, cellnp, planes, plane_nb, planes_lo, total;
};
SceneLayout make_scene_layout(int32_t n, int32_t k);

// ------------------------------------------------------------------ helpers
__host__ __device__ inline uint64_t align_up(uint64_t x, uint64_t a) { return (x + a - 1) / a * a; }

// Detail sites per face of a scene (Sec. 3.4): 4, or 8.
__host__ __device__ inline int scene_sites(const pf_scene &s) { return s.n_sites == 8 ? 8 : 4; }
// An extended face model: displacement, learned sites, view-dependent site
// colours or eight sites (the renderer's EXT kernels).
__host__ __device__ inline bool ext_face(const pf_scene &s) {
    return s.disp != nullptr || s.sites != nullptr || s.sv != nullptr || s.n_sites == 8;
}

void set_error(const char *fmt, ...);
pf_status cuda_status(cudaError_t e, const char *what);
bool camera_ok(const pf_camera &c);
bool scene_ok(const pf_scene *s, const Plan *p);
void fill_views(Plan *p, const pf_camera *cams);  // per-view constants and offsets
void make_layout(Plan *p);                        // workspace offsets

// kernels launched from the C API (defined in the .cu files)
cudaError_t launch_prepare(const pf_scene &s, const Plan &p, const WS &w, cudaStream_t st);
cudaError_t launch_connect(const pf_scene &s, float *loss, float *gpos, float *gR, cudaStream_t st);
cudaError_t launch_project(const pf_scene &s, const Plan &p, const WS &w, cudaStream_t st);
cudaError_t launch_bin_sort(const Plan &p, const WS &w, cudaStream_t st);
cudaError_t launch_render_fwd(const pf_scene &s, const Plan &p, const WS &w, float *rgb, float *T, uint32_t *last,
                              bool record, cudaStream_t st, float *contrib_sparse = nullptr,
                              float *contrib_normal = nullptr);
// The pipelined forward (pf_render_pipe.cu): the plain face model without
// hit recording, stats or contributions.
bool pipe_applies(const pf_scene &s, const Plan &p, bool record, bool contrib);
cudaError_t launch_render_fwd_pipe(const pf_scene &s, const Plan &p, const WS &w, float *rgb, float *T,
                                   uint32_t *last, bool record, cudaStream_t st, float *contrib_sparse,
                                   float *contrib_normal);
cudaError_t launch_render_bwd(const pf_scene &s, const Plan &p, const WS &w, const float *dL_drgb,
                              const float *dL_dT, const float *T, const uint32_t *last, const pf_scene_grad &g,
                              bool use_masks, cudaStream_t st, const float *w_sparse = nullptr,
                              const float *w_normal = nullptr);

}  // namespace pf
