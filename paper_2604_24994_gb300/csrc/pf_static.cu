// pf_render_fwd_static: one small view rendered with no caller workspace and
// no device allocation.  The scratch that pf_prepare / pf_project /
// pf_bin_sort / pf_render_fwd normally take from the caller's workspace
// lives here in one file-scope __device__ array instead.
//
// Who needs this: code that must not allocate device memory at all, for
// example a host that hands its whole memory budget to another allocator,
// or a real-time loop where an allocation (or the caching allocator
// growing) is not allowed.  Such a caller still owns and passes its scene,
// camera and output buffers.
//
// Costs and rules:
//   - The array is PF_STATIC_SCRATCH_BYTES (8.5 MiB).  It is reserved on a
//     device when the library's module is loaded there, which with CUDA's
//     lazy module loading happens inside the first call on that device
//     (its cudaGetSymbolAddress).  So the first call commits device memory
//     and can fail with out-of-memory: make it before handing the device's
//     memory to another allocator.  The array then stays until the process
//     exits.
//   - Host code cannot use the array's name as a device pointer: every call
//     looks up its device address on the current device with
//     cudaGetSymbolAddress (cheap once the module is loaded) and passes
//     that address to the kernels.  Looking it up each time keeps the call
//     correct after a cudaDeviceReset, which may place the array elsewhere.
//   - All calls share the one array and it keeps the previous call's data.
//     Everything that has to start at zero is cleared on every call.  Calls
//     that overlap on the GPU (other streams, other threads) race on it:
//     serialise them.
//   - The call synchronises `stream` once (to check the instance count),
//     so it cannot run while `stream` is being captured into a CUDA graph;
//     it returns PF_ERR_INVALID_ARG in that case without enqueuing work.
#include "pf_internal.cuh"

namespace pf {

constexpr size_t STATIC_SCRATCH_BYTES = PF_STATIC_SCRATCH_BYTES;

static __device__ __align__(256) unsigned char g_static_scratch[STATIC_SCRATCH_BYTES];

// Device address of the array on the current device.
static pf_status static_scratch(void **out) {
    void *p = nullptr;
    pf_status s = cuda_status(cudaGetSymbolAddress(&p, g_static_scratch), "pf_render_fwd_static: cudaGetSymbolAddress");
    if (s) return s;
    *out = p;
    return PF_OK;
}

}  // namespace pf

using namespace pf;

extern "C" pf_status pf_render_fwd_static(const pf_scene *scene, const pf_camera *cam, float *rgb, float *T,
                                          uint32_t *last, void *stream) {
    set_error("%s", "");
    if (!scene || !cam || !rgb || !T || !last) {
        set_error("pf_render_fwd_static: null argument");
        return PF_ERR_INVALID_ARG;
    }
    if (scene->n_cells < 0 || scene->n_cells > PF_STATIC_MAX_CELLS || scene->k_nbr < 0 ||
        scene->k_nbr > PF_STATIC_MAX_K) {
        set_error("pf_render_fwd_static: %d cells / %d neighbours exceed the limits %d / %d", scene->n_cells,
                  scene->k_nbr, PF_STATIC_MAX_CELLS, PF_STATIC_MAX_K);
        return PF_ERR_INVALID_ARG;
    }
    if (!camera_ok(*cam) || cam->width > PF_STATIC_MAX_SIDE || cam->height > PF_STATIC_MAX_SIDE) {
        set_error("pf_render_fwd_static: camera invalid or larger than %dx%d", PF_STATIC_MAX_SIDE,
                  PF_STATIC_MAX_SIDE);
        return PF_ERR_INVALID_ARG;
    }
    // a plan on the stack: no heap, no device allocation
    ViewDev view_host;
    Plan p;
    p.n = scene->n_cells;
    p.k = scene->k_nbr;
    p.nv = 1;
    p.cap = PF_STATIC_MAX_INSTANCES;
    p.stats = 0;
    p.fwd_only = true;
    p.views_host = &view_host;
    fill_views(&p, cam);
    make_layout(&p);
    if (!scene_ok(scene, &p)) return PF_ERR_INVALID_ARG;
    if (p.L.total > STATIC_SCRATCH_BYTES) {
        set_error("pf_render_fwd_static: layout %llu bytes exceeds the static scratch", (unsigned long long)p.L.total);
        return PF_ERR_CAPACITY;
    }
    cudaStream_t st = (cudaStream_t)stream;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    pf_status s = cuda_status(cudaStreamIsCapturing(st, &cap), "pf_render_fwd_static: cudaStreamIsCapturing");
    if (s) return s;
    if (cap != cudaStreamCaptureStatusNone) {
        set_error("pf_render_fwd_static: the stream is being captured; this call synchronises it and cannot be "
                  "captured");
        return PF_ERR_INVALID_ARG;
    }
    void *base = nullptr;
    s = static_scratch(&base);
    if (s) return s;
    WS w = p.ws(base);
    // the view constants: pageable copy, done before cudaMemcpyAsync returns
    s = cuda_status(cudaMemcpyAsync(w.views, &view_host, sizeof view_host, cudaMemcpyHostToDevice, st),
                    "pf_render_fwd_static: views");
    if (!s) s = cuda_status(launch_prepare(*scene, p, w, st), "pf_render_fwd_static: prepare");
    if (!s) s = cuda_status(launch_project(*scene, p, w, st), "pf_render_fwd_static: project");
    if (!s) s = cuda_status(launch_bin_sort(p, w, st), "pf_render_fwd_static: bin_sort");
    if (s) return s;
    Counters c;
    s = cuda_status(cudaMemcpyAsync(&c, w.counters, sizeof c, cudaMemcpyDeviceToHost, st),
                    "pf_render_fwd_static: counters");
    if (!s) s = cuda_status(cudaStreamSynchronize(st), "pf_render_fwd_static: sync");
    if (s) return s;
    if (c.overflow) {
        set_error("pf_render_fwd_static: %llu (cell, tile) instances exceed the limit %d",
                  (unsigned long long)c.total_inst, PF_STATIC_MAX_INSTANCES);
        return PF_ERR_CAPACITY;
    }
    return cuda_status(launch_render_fwd(*scene, p, w, rgb, T, last, false, st), "pf_render_fwd_static: render");
}
