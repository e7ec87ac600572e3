/*
 * powerfoam.h - C ABI of the GB300 (sm_103a) tile rasterizer for bounded
 * power-diagram cells (Power Foam, arxiv 2604.24994).
 *
 * Conventions for every entry point
 *   - All scene, image and gradient pointers are DEVICE pointers owned by the
 *     caller.  The library never allocates or frees device memory; scratch
 *     lives in a caller-provided workspace whose size pf_plan_workspace_bytes
 *     reports.  A plan (pf_plan) is a small host object (layout + cameras).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy stream).
 *     Calls only enqueue work on it and return; results are valid once the
 *     stream reaches them.  The exceptions say so (pf_bin_sort with a
 *     non-NULL n_instances, the pf_serve_* calls).
 *   - Nothing throws across the ABI.  Every call returns a pf_status;
 *     pf_status_string names it, pf_last_error_message gives detail for the
 *     calling thread's last failure.
 *   - Float data is IEEE binary32, little endian, C-contiguous.
 *
 * Scene parameters (Sec. 3.2-3.4 of the paper), N cells:
 *   pos    [N,3]  site p_i
 *   w      [N]    power weight w_i (pow(x,i) = |x - p_i|^2 - w_i, Eq. pow_dist)
 *   R      [N]    bound radius of cell i's sphere
 *   sigma  [N]    density of the dense half of the cell
 *   rgb    [N,3]  base colour
 *   normal [N,3]  dipole normal n_i (any non-zero length; used as n/|n|)
 *   offset [N]    the face is { x : n^.(x - p_i) = offset_i }; the dense
 *                 half is n^.(x - p_i) <= offset_i (Sec. 3.3)
 *   tex    [N,12] four texture sites x RGB, site-major, 16-byte aligned
 *                 (the soft-Voronoi radiance on the face, Eq. svrad)
 *   nbr    [N,K]  int32 neighbour ids (-1 padded): every site whose radical
 *                 plane can cut cell i's sphere must be listed (a Cech list,
 *                 Sec. 3.2, is enough); extra entries never change the result.
 */
#ifndef POWERFOAM_H
#define POWERFOAM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PF_OK = 0,
    PF_ERR_INVALID_ARG = 1, /* null pointer, bad size, bad camera */
    PF_ERR_CAPACITY = 2,    /* instance capacity too small; required size reported */
    PF_ERR_CUDA = 3,        /* a CUDA runtime call failed */
    PF_ERR_TIMEOUT = 4,     /* a bounded wait ran out */
    PF_ERR_BUSY = 5,        /* admission refused (serving) */
    PF_ERR_NOT_FOUND = 6    /* unknown request id (serving) */
} pf_status;

typedef struct {
    const float *pos, *w, *R, *sigma, *rgb, *normal, *offset, *tex;
    const int32_t *nbr;
    int32_t n_cells; /* N >= 0 */
    int32_t k_nbr;   /* K in [0, 64] */
    /* Optional face displacement [N][4] (NULL: none; 16-byte aligned):
     * disp[i][k] moves the face of cell i along its normal at texture site
     * k.  A ray crossing the base face at face coordinates u sees the face
     * moved by delta = sum_k W_k(u) disp[i][k], with the soft-Voronoi
     * weights of the texture (Eq. svdisp, one-step plane shift); a ray
     * parallel to the face sees no displacement.  pf_render_fwd (also
     * recording hits), pf_render_fwd_contrib, pf_render_fwd_static, the
     * server and pf_render_bwd (which then adds dL/ddisp into
     * pf_scene_grad.disp) honour it; stats passes return PF_ERR_INVALID_ARG
     * for a displaced scene. */
    const float *disp;
    /* Optional learned detail-site positions [N][4][2] (NULL: the fixed
     * sites (-1/3,-1/3), (1/3,-1/3), (-1/3,1/3), (1/3,1/3); 16-byte
     * aligned), in units of R in the face frame, in the site order of tex
     * and disp (Sec. 3.4: the detail sites are learnable).  They place both
     * the texture's and the displacement's soft-Voronoi weights; the same
     * entry points as disp honour them, and pf_render_bwd adds dL/dsites
     * into pf_scene_grad.sites. */
    const float *sites;
    /* Optional view-dependent site colours [N][4][8][6] (NULL: the constant
     * colours tex): per site a spherical-Voronoi function (Sec. 3.4) of
     * eight (axis xyz, rgb); seen along a ray with direction d the site's
     * colour is sum_j softmax_j(10 a_j.(-d) / |a_j|) rgb_j.  They replace
     * tex in the colour.  pf_render_fwd, pf_render_fwd_contrib,
     * pf_render_fwd_static, the server and pf_render_bwd (adding dL/dsv into
     * pf_scene_grad.sv) honour them; stats passes return PF_ERR_INVALID_ARG
     * for such a scene. */
    const float *sv;
    /* Detail sites per face (Sec. 3.4; the paper's main configuration has
     * eight): 0 or 4 for four, 8 for eight.  With eight, tex is [N,24],
     * disp [N][8], sites [N][8][2] and sv [N][8][8][6]; the fixed sites are
     * the 3 x 3 grid of step 1/3 (units of R) without its centre, row by row:
     * (-1,-1), (0,-1), (1,-1), (-1,0), (1,0), (-1,1), (0,1), (1,1) / 3.
     * pf_render_fwd, pf_render_fwd_contrib, pf_render_fwd_static, the
     * server and pf_render_bwd (its tex, disp, sites and sv gradients have the
     * same shapes) take either; stats passes return PF_ERR_INVALID_ARG for
     * eight. */
    int32_t n_sites;
} pf_scene;

/* Camera: x_cam = rot (x_world - origin), OpenCV axes (x right, y down,
 * z forward); pixel (u, v) is the ray through its centre (u + 0.5, v + 0.5).
 * model PF_PINHOLE (0): the ray through ((u+.5-cx)/fx, (v+.5-cy)/fy, 1).
 * model PF_FISHEYE (1), equidistant (non-pinhole rasterization, appendix D):
 * a = ((u+.5-cx)/fx, (v+.5-cy)/fy) is the ray's angle theta = |a| from the
 * optical axis, towards a/|a|: direction (sin(theta) a/|a|, cos(theta)).
 * Pixels with theta > pi have no ray: rgb 0, T 1, last 0.  The painter
 * order (power distance from the camera centre) is exact for every ray
 * through the centre, so both models render losslessly. */
#define PF_PINHOLE 0
#define PF_FISHEYE 1
typedef struct {
    double rot[9]; /* row-major world->camera rotation */
    double origin[3];
    double fx, fy, cx, cy;  /* fx, fy > 0 */
    int32_t width, height; /* 1..16384 each */
    int32_t model;         /* PF_PINHOLE or PF_FISHEYE */
} pf_camera;

/* Gradient outputs, same shapes as the scene parameters; the backward ADDS
 * into them (zero them first for a fresh gradient). */
typedef struct {
    float *pos, *w, *R, *sigma, *rgb, *normal, *offset, *tex;
    float *disp;  /* [N][4], required when the scene has a displacement, else ignored */
    float *sites; /* [N][4][2], required when the scene has learned sites, else ignored */
    float *sv;    /* [N][4][8][6], required when the scene has view-dependent site
                   * colours, else ignored (tex then gets no gradient) */
} pf_scene_grad;

typedef struct pf_plan pf_plan;

/* Work counters of one forward pass (filled when stats are enabled). */
typedef struct {
    uint64_t instances; /* (cell, tile) pairs after binning */
    uint64_t candidates; /* (pixel, listed cell) pairs examined */
    uint64_t hits;       /* non-empty (pixel, cell) segments */
    uint64_t planes;     /* radical-plane clips each ray needs on its own: per
                          * sphere pass, the planes up to the one that empties
                          * its segment (all of them if none does); the warp
                          * evaluates more, since it stops only when every
                          * lane's segment is empty */
    uint64_t refined;    /* segment ends recomputed in FP64 */
    uint64_t sphere_pass; /* candidates that passed the sphere test */
    /* the same events counted once per warp (32 pixels) that had at least
     * one of them: their ratio to the per-pixel counts is the SIMD use */
    uint64_t warp_candidates;
    uint64_t warp_passes;
    uint64_t warp_hits;
    /* nonzero if a bounded wait of the forward's shared-memory pipeline ran
     * out since the last pf_bin_sort (the image is then incomplete); always
     * 0 in correct operation, read whether or not stats are enabled */
    uint64_t wait_errors;
} pf_stats;

const char *pf_status_string(pf_status s);
/* Detail of the calling thread's last failed call ("" if none). */
const char *pf_last_error_message(void);

/*
 * Plans.  A plan fixes N, K, the views (their cameras and resolutions) and
 * the capacity of the (cell, tile) instance arrays.  Multi-view calls work
 * on all views at once; images of view v start at pixel offset
 * sum_{u<v} W_u H_u of the concatenated outputs.
 * Ownership: *out is owned by the caller and freed with pf_plan_destroy.
 */
pf_status pf_plan_create(int32_t n_cells, int32_t k_nbr, const pf_camera *cams, int32_t n_views,
                         uint64_t inst_capacity, pf_plan **out);
void pf_plan_destroy(pf_plan *plan);
/* Bytes of device workspace the plan needs (256-byte aligned base). */
pf_status pf_plan_workspace_bytes(const pf_plan *plan, uint64_t *bytes);
/* Total pixels over all views. */
pf_status pf_plan_pixels(const pf_plan *plan, uint64_t *pixels);
/* Replace the cameras; resolutions must equal the plan's.  The new values
 * are read by the next pf_project on any stream. */
pf_status pf_plan_set_cameras(pf_plan *plan, const pf_camera *cams, int32_t n_views);
/* Hit recording (default on).  While on, pf_render_fwd also writes, for
 * every pixel and every batch of 32 entries of its tile's list, a 32-bit
 * mask of the entries whose segment was non-empty, and the active
 * constraints (entry, exit) of the pixel's first 256 hits (in the
 * workspace); the next pf_render_bwd on the same bins then replays only
 * those (cell, pixel) pairs, without the plane loop for the recorded ones,
 * instead of re-testing every listed cell.  Turn it off for forward-only rendering (it saves one store per
 * warp and batch); the backward then re-tests.  The masks are dropped by
 * pf_prepare, pf_project and pf_bin_sort, and not written by a forward that
 * counts stats. */
pf_status pf_plan_set_record_hits(pf_plan *plan, int32_t enable);
/* Lay the plan's workspace out without the hit records (8 x (capacity/32 +
 * tiles + 1) x 128 bytes of masks, 516 bytes per pixel of records and
 * counts): a smaller workspace whose backward always re-tests.  Call it
 * before querying pf_plan_workspace_bytes and allocating; recording can then
 * no longer be enabled (PF_ERR_INVALID_ARG). */
pf_status pf_plan_omit_hit_records(pf_plan *plan);
/* Store every segment instead of replaying it: with max_hits > 0 the
 * forward (while recording hits) also stores, for each pixel's first
 * max_hits hits in list order, the segment's entry and exit, the
 * transmittance in front of it and its active constraints (16 bytes), and
 * the backward reads them instead of recomputing the ends and the
 * transmittance (the no-checkpoint variant of the large differentiable
 * workload; hits past max_hits are replayed as before).  It adds
 * pixels x max_hits x 16 bytes to the workspace: call it before querying
 * pf_plan_workspace_bytes and allocating.  0 turns it off.  Errors:
 * PF_ERR_INVALID_ARG (negative, or a plan laid out without hit records). */
pf_status pf_plan_store_segments(pf_plan *plan, int32_t max_hits);
/* Copy the hits the last recording forward composited per pixel [P] to a
 * HOST buffer (synchronises `stream`); PF_ERR_INVALID_ARG without hit
 * records. */
pf_status pf_read_hit_counts(pf_plan *plan, void *ws, uint32_t *counts, void *stream);
/* Count work in the next forward passes (adds to the counters; 0 disables). */
pf_status pf_plan_enable_stats(pf_plan *plan, int32_t enable);
/* Read the counters, then reset them (synchronises `stream`). */
pf_status pf_plan_read_stats(pf_plan *plan, void *ws, pf_stats *out, void *stream);

/*
 * View-independent cell records (Sec. 3.2-3.4).  For every cell, in FP64:
 * the unit normal and face frame, and the radical planes
 *   x.(p_j - p_i) <= (|p_j|^2 - |p_i|^2 + w_i - w_j) / 2
 * of its listed neighbours (the definition of pow gives +w_i - w_j; the
 * appendix's Eq. power_bisector prints the weights the other way round),
 * kept only where the plane reaches the bounding sphere (Sec. 3.2: other
 * planes never cut the cell) and where no single other plane or the dipole
 * face implies it inside the sphere.  Run after any scene change.
 */
pf_status pf_prepare(const pf_scene *scene, pf_plan *plan, void *ws, void *stream);

/*
 * Per view and cell: the camera-relative site offset as a float pair (an
 * error-free two-sum of the origin's float pair and the site), the painter
 * key pow(o, p_i) in FP64 (Thm. power_painter: ordering by power distance
 * from the camera centre is a valid painter's order), and the screen
 * bounding box of the sphere as a 16x16 tile rectangle: in float, widened by
 * a bound on its rounding, for a sphere well in front of the camera, in FP64
 * otherwise.  The rectangle covers every pixel whose ray meets the sphere.
 */
pf_status pf_project(const pf_scene *scene, pf_plan *plan, void *ws, void *stream);

/*
 * Duplicate every (cell, tile) pair, group by tile and sort each tile's list
 * by (key, cell index) (Sec. 3.2: all instances sorted by depth, as Gaussian
 * splatting does; here by power distance).  If n_instances is non-NULL the call
 * synchronises the stream and returns the instance count; then
 * PF_ERR_CAPACITY means the plan's capacity was too small (*n_instances is
 * the size needed; re-plan and repeat pf_prepare/pf_project/pf_bin_sort).
 * With NULL it stays asynchronous; an overflow is then only visible through
 * pf_plan_read_stats / a later synchronous call, and the lists are cut at
 * capacity (memory-safe, images wrong).
 */
pf_status pf_bin_sort(pf_plan *plan, void *ws, uint64_t *n_instances, void *stream);

/*
 * Forward render (Sec. 3.1-3.4): per pixel, walk the tile's sorted list,
 * cut the ray with each cell's sphere, radical planes and dense half,
 * composite alpha = 1 - exp(-sigma l) and the soft-Voronoi face colour front
 * to back over a black background; stop once T < 1e-6.
 * Outputs (device, concatenated over views): rgb [P,3], T [P] (final
 * transmittance) and last [P] (1 + list index of the last contributing
 * cell; 0 if none).  T and last are the checkpoint pf_render_bwd replays.
 */
pf_status pf_render_fwd(const pf_scene *scene, pf_plan *plan, void *ws, float *rgb, float *T, uint32_t *last,
                        void *stream);

/*
 * pf_render_fwd that also ADDS each cell's contributions over the views'
 * pixels (the per-primitive terms of Sec. 4's training): with T the
 * transmittance in front of the cell's segment on a ray and alpha its
 * opacity,
 *   contrib_sparse[i] += sum over rays of T alpha           (L_sparse, pruning EMA)
 *   contrib_normal[i] += sum over rays of T alpha max(nh_i . d, 0)^2   (L_normal)
 * Arrays [N] on the device, zeroed by the caller for a fresh sum.  Segments
 * behind a pixel's early termination (T < 1e-6) are not counted.  Records
 * hits like pf_render_fwd; does not count stats.  Takes every face model
 * (displacement, learned or eight sites, view-dependent colours).
 */
pf_status pf_render_fwd_contrib(const pf_scene *scene, pf_plan *plan, void *ws, float *rgb, float *T, uint32_t *last,
                                float *contrib_sparse, float *contrib_normal, void *stream);

/*
 * Adjoint of pf_render_fwd for upstream dL/drgb [P,3] and dL/dT [P]
 * (dL_dT may be NULL for zero).  Replays each tile back to front from the
 * checkpoint (T, last) and ADDS dL/d(parameter) into `grad` (every pointer
 * non-NULL).  Requires the same plan/workspace state as the forward (the
 * same scene, bins and views).  If the forward recorded hit masks on these
 * bins (pf_plan_set_record_hits) only the recorded (cell, pixel) pairs are
 * replayed; otherwise every listed cell is re-tested up to `last`.
 */
pf_status pf_render_bwd(const pf_scene *scene, pf_plan *plan, void *ws, const float *dL_drgb, const float *dL_dT,
                        const float *T, const uint32_t *last, const pf_scene_grad *grad, void *stream);

/*
 * pf_render_bwd for a loss that also holds the per-cell contributions of
 * pf_render_fwd_contrib (Sec. 4: L_sparse and L_normal are functions of
 * them; the caller's weights are their derivatives):
 *   L = L_image(rgb, T) + sum_i (w_sparse[i] sparse_i + w_normal[i] normal_i),
 *   sparse_i = sum over rays of T alpha,  normal_i = sum of T alpha max(nh_i.d, 0)^2,
 * the same sums as pf_render_fwd_contrib over the plan's views.  dL_drgb,
 * dL_dT, T and last as for pf_render_bwd (pass zeros in dL_drgb for the
 * contributions' gradient alone); w_sparse, w_normal: device [N].  Along a
 * ray the contributions composite the scalar w_sparse + w_normal
 * max(nh.d, 0)^2 like a colour channel, so the same replay gives their
 * gradient for every parameter the segments depend on, plus the normal's
 * share through max(nh.d, 0)^2.  ADDS into `grad`.  Errors as pf_render_bwd.
 */
pf_status pf_render_bwd_contrib(const pf_scene *scene, pf_plan *plan, void *ws, const float *dL_drgb,
                                const float *dL_dT, const float *T, const uint32_t *last, const float *w_sparse,
                                const float *w_normal, const pf_scene_grad *grad, void *stream);

/*
 * Connectivity loss of Sec. 4 / appendix (L_connect) over the neighbour
 * lists, which stand in for the Cech adjacency (pairs whose bounding spheres
 * do not overlap add nothing; pf_connect_cech below sums over the exact
 * adjacency):
 *   loss[i] = sum_{j in nbr(i)} max(R_i + R_j - |p_i - p_j|, 0)^2     (written)
 * With grad_pos [N,3] and grad_R [N] (both or neither) it ADDS the gradient
 * of sum_i loss[i] with respect to the sites and the bound radii.  Uses only
 * pos, R, nbr, n_cells and k_nbr of the scene; device pointers; no plan.
 */
pf_status pf_connect(const pf_scene *scene, float *loss, float *grad_pos, float *grad_R, void *stream);

/*
 * Connectivity loss of Sec. 4 / appendix (L_connect) over the exact Cech
 * adjacency of the bounding spheres: for every cell i, every j != i whose
 * sphere overlaps cell i's, |p_i - p_j| < R_i + R_j,
 *   loss[i] = sum_{j in Cech(i)} max(R_i + R_j - |p_i - p_j|, 0)^2   (written)
 * With grad_pos [N,3] and grad_R [N] (both or neither) it ADDS the gradient
 * of sum_i loss[i]: each overlapping pair appears in L(i) and in L(j), so
 * dR_i gets 4 o and dp_i gets 4 o (p_j - p_i) / d per pair, with
 * o = R_i + R_j - d > 0 and d = |p_j - p_i| (coincident sites add no
 * direction).  The pairs are found by a radix tree over the sites' Morton
 * codes refit with the spheres' boxes (the step the paper does with GPU
 * collision detection, Sec. 3.3); each pair's value is computed in FP64 from
 * the float inputs and each cell gathers its own sums (no atomics).
 * pos [N][3], R [N] (negative radii count as 0): device float32.  loss [N],
 * grad_pos, grad_R: device float32.  status: device uint32, optional: 1 if a
 * tree walk ran out of stack or steps (not expected below
 * PF_NEIGHBOURS_MAX_CELLS).  ws: device workspace of at least
 * pf_connect_cech_workspace_bytes(N) bytes (about 116 bytes per cell).
 * Errors: PF_ERR_INVALID_ARG (size, null pointer, only one gradient),
 * PF_ERR_CAPACITY (workspace too small).  Asynchronous on `stream`, no
 * allocation, no host synchronisation.
 */
uint64_t pf_connect_cech_workspace_bytes(int32_t n_cells);
pf_status pf_connect_cech(const float *pos, const float *R, int32_t n_cells, float *loss, float *grad_pos,
                          float *grad_R, uint32_t *status, void *ws, uint64_t ws_bytes, void *stream);

/*
 * Copy the binning results to HOST buffers (synchronises `stream`), for
 * inspection and tests.  tile_start [T+1] (T = tiles over all views, view v
 * first at its tile base, row-major tiles of 16x16 px): tile t's list is
 * cells[tile_start[t] .. tile_start[t+1]), cell indices sorted by (key,
 * index).  cells [capacity].  keys [V*N] painter keys (order-preserving bits
 * of pow(o, p_i) in FP64) and rects [V*N][4] (tx0, ty0, tx1, ty1 with
 * tx0 > tx1 when empty) may be NULL.
 */
pf_status pf_read_bins(pf_plan *plan, void *ws, uint32_t *tile_start, uint32_t *cells, uint64_t *keys,
                       uint16_t *rects, void *stream);

/*
 * Serving: continuous batching of render requests over one resident scene.
 *
 * The caller provides a device pool (the memory budget, 256-byte aligned).
 * The server keeps the scene's cell records there (prepared once), and
 * splits the rest into `slots` equal regions, one per batch in flight, each
 * with its own CUDA stream.  A worker thread admits queued requests in
 * arrival order into a free slot while the batch's per-view records, tile
 * arrays and instance buffers fit the slot (the admission test is memory),
 * up to max_batch_views.  A batch is projected, binned and rendered as one
 * multi-view plan with one persistent render launch; requests that arrive
 * while other batches run are admitted as slots free up, so their work
 * overlaps on the GPU.  With use_graphs each batch's launch sequence runs
 * as a CUDA graph: a slot keeps one executable graph per view count, replays
 * it for a repeated batch shape and updates it in place for a new one.  Results are the same as
 * rendering each view alone with pf_render_fwd.
 *
 * The scene pointers and the pool must stay valid until pf_serve_destroy.
 * Output buffers (device rgb [W*H,3], T [W*H]) belong to the caller and are
 * written when the request completes.  No call blocks longer than the
 * timeout it is given; pf_serve_destroy waits at most 10 s for batches in
 * flight and drops requests not yet started.
 */
typedef struct {
    int32_t max_batch_views; /* views per batch, 1..256 */
    int32_t slots;           /* batches in flight, 1..16 */
    int32_t use_graphs;      /* run each batch as a CUDA graph (replayed or updated per slot) */
    int32_t max_queue;       /* queued requests before submit returns PF_ERR_BUSY */
} pf_serve_opts;

typedef struct {
    /* graph_replays: batches that replayed their slot's graph as it was (the
     * same batch shape); graph_updates: batches written into an existing
     * graph of their view count (cudaGraphExecUpdate, no instantiation) */
    uint64_t submitted, completed, rejected, batches, graph_replays, requeued;
    double p50_ms, p99_ms, mean_ms, max_ms; /* submit -> result written */
    double elapsed_s;                        /* first submit -> last completion */
    double requests_per_s, mpix_per_s, mean_batch_views;
    uint64_t graph_updates;
} pf_serve_report;

typedef struct pf_server pf_server;

/* Prepares the scene (synchronously) and starts the worker.  Errors:
 * PF_ERR_INVALID_ARG, PF_ERR_CAPACITY (pool too small for the scene). */
pf_status pf_serve_create(const pf_scene *scene, void *pool, uint64_t pool_bytes, const pf_serve_opts *opts,
                          pf_server **out);
/* Non-blocking.  PF_ERR_CAPACITY if the view cannot fit a slot even alone,
 * PF_ERR_BUSY if the queue is full (the request is not taken). */
pf_status pf_serve_submit(pf_server *srv, const pf_camera *cam, float *rgb, float *T, uint64_t *req_id);
/* Waits up to timeout_ms (0: just check).  *done = 1 when the outputs are
 * written (the id is then released), 0 if not yet (PF_ERR_TIMEOUT when a
 * timeout was given), -1 with an error status if the request failed.
 * PF_ERR_NOT_FOUND for unknown or released ids. */
pf_status pf_serve_poll(pf_server *srv, uint64_t req_id, int32_t timeout_ms, int32_t *done);
pf_status pf_serve_stats(pf_server *srv, pf_serve_report *out);
pf_status pf_serve_reset_stats(pf_server *srv);
void pf_serve_destroy(pf_server *srv);

/*
 * Forward render of one small view WITHOUT a workspace and without any
 * device allocation (no cudaMalloc, cudaFree or allocating library call).
 * The paper has no counterpart: this exists for callers that cannot
 * allocate device memory (a host that has given its whole memory budget to
 * another allocator, a real-time loop that forbids allocation).  The caller
 * still passes the scene (device pointers), the camera (host struct) and
 * device outputs rgb [W*H,3], T [W*H], last [W*H], exactly as for
 * pf_render_fwd with a one-view plan; the results are the same.
 *
 * The scratch is one file-scope __device__ array of PF_STATIC_SCRATCH_BYTES
 * that every GPU loading the library keeps until the process exits.  With
 * CUDA's lazy module loading it is reserved inside the first call on a
 * device, so that call commits device memory and can fail with
 * out-of-memory (PF_ERR_CUDA): make it before giving the device's memory
 * away.  Each call looks up the array's address on the current device
 * (cudaGetSymbolAddress).  Limits (larger requests return
 * PF_ERR_INVALID_ARG, or PF_ERR_CAPACITY when the instance count is
 * exceeded, with a message from pf_last_error_message): at most
 * PF_STATIC_MAX_CELLS cells, PF_STATIC_MAX_K neighbours, an image of at most
 * PF_STATIC_MAX_SIDE x PF_STATIC_MAX_SIDE pixels and PF_STATIC_MAX_INSTANCES
 * (cell, tile) pairs.
 *
 * Every call reuses the same array and clears what must start at zero;
 * calls that overlap on the GPU (different streams or threads) race on it
 * and must be serialised by the caller.  The call synchronises `stream`
 * once, after binning, to check the instance count; on a stream that is
 * being captured into a CUDA graph it returns PF_ERR_INVALID_ARG without
 * enqueuing anything.
 */
#define PF_STATIC_MAX_CELLS 4096
#define PF_STATIC_MAX_K 32
#define PF_STATIC_MAX_SIDE 256
#define PF_STATIC_MAX_INSTANCES 65536
#define PF_STATIC_SCRATCH_BYTES (8u * 1024u * 1024u + 512u * 1024u)
pf_status pf_render_fwd_static(const pf_scene *scene, const pf_camera *cam, float *rgb, float *T, uint32_t *last,
                               void *stream);

/*
 * Neighbour lists on the GPU, the step before rendering that the paper does
 * with GPU collision detection over the bounding spheres (Sec. 3.3, the Cech
 * graph).  For cell i, with t_ij the signed distance from p_i of the radical
 * plane between sites i and j (Sec. 3.2, Eq. power bisector),
 *   t_ij = (|p_j - p_i|^2 + w_i - w_j) / (2 |p_j - p_i|)   (no plane if p_j == p_i),
 * nbr[i] lists the K sites j != i with the smallest t_ij, ascending, equal
 * values by ascending j, -1 after the last one when fewer than K exist; and
 * R_out[i] = R_in[i], except R_out[i] = the largest float <= max(t_(K+1), 0)
 * when the (K+1)-th smallest t_(K+1) < R_in[i] (so that no site left out can
 * cut the cell's sphere; t is evaluated in FP64 from the float inputs exactly
 * as written above: dx*dx + dy*dy, + dz*dz; sqrt; ((L^2 + w_i) - w_j) / (2L)).
 *
 * pos [N][3], w [N], R_in [N]: device, float32, finite.  nbr [N][K] int32
 * and R_out [N] float32: device, written (R_out may be R_in).  n_clipped and
 * status: device uint32, optional (NULL): the number of clipped radii, and 0
 * or 1 if a tree walk ran out of stack or steps (the lists may then be incomplete;
 * not expected below PF_NEIGHBOURS_MAX_CELLS).  ws: device workspace of at
 * least pf_neighbours_workspace_bytes(N) bytes (about 116 bytes per cell),
 * owned by the caller.  0 <= N <= PF_NEIGHBOURS_MAX_CELLS, 0 <= K <= 64,
 * otherwise PF_ERR_INVALID_ARG; a small workspace gives PF_ERR_CAPACITY.
 * Asynchronous on `stream`, no allocation, no host synchronisation (stream
 * capture is allowed).
 */
#define PF_NEIGHBOURS_MAX_CELLS (1 << 28)
uint64_t pf_neighbours_workspace_bytes(int32_t n_cells);
pf_status pf_build_neighbours(const float *pos, const float *w, const float *R_in, int32_t n_cells, int32_t k_nbr,
                              int32_t *nbr, float *R_out, uint32_t *n_clipped, uint32_t *status, void *ws,
                              uint64_t ws_bytes, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* POWERFOAM_H */
