// Continuous-batching render server over one resident scene.
//
// The caller gives a device memory pool (the budget).  The server lays it
// out once: the scene's view-independent records (prepared once at
// creation), then `slots` equal regions, one per in-flight batch, each with
// its own stream.  A worker thread takes queued requests in arrival order
// and, whenever a slot is free, admits as many as fit that slot's memory
// (the per-view records, tile arrays and (cell, tile) instance buffers of a
// multi-view plan) up to max_batch_views.  A batch is one multi-view plan:
// one projection over all its views, one binning/sort, and one persistent
// render launch whose CTAs take tiles of every view from a shared queue;
// each view writes straight into its request's output buffers.  Batches on
// different slots overlap on the GPU.  With use_graphs, the launch sequence
// of a batch is captured into a CUDA graph: each slot keeps one executable
// graph per view count, replayed as it is for a repeated batch shape and
// updated in place (cudaGraphExecUpdate) for a new one; the cameras and
// output pointers it reads live in the slot's pinned buffer.  Completion is
// signalled by a host function at the end of the batch's stream.
//
// Waits are bounded: pf_serve_poll takes a timeout, the worker wakes at
// least every millisecond, and destroy gives in-flight batches a bounded
// time to finish.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "pf_internal.cuh"

namespace pf {

using clk = std::chrono::steady_clock;

static double now_ms() {
    return std::chrono::duration<double, std::milli>(clk::now().time_since_epoch()).count();
}

struct Request {
    uint64_t id;
    pf_camera cam;
    float *rgb;
    float *T;
    double t_submit = 0, t_done = 0;
    int done = 0;    // 1 done, -1 failed
    int solo = 0;    // render alone (after an overflow in a batch)
};

struct Server;

struct Slot {
    Server *srv = nullptr;
    int index = 0;
    cudaStream_t stream = nullptr;
    char *ws = nullptr;          // device region
    uint64_t ws_bytes = 0;
    ViewDev *views_pinned = nullptr;   // cameras + outputs of the current batch
    Counters *ctr_pinned = nullptr;    // counters read back after the batch
    std::vector<Request *> batch;
    std::atomic<int> finished{0};
    double t_finished = 0;
    bool busy = false;
    // one executable graph per view count, and the batch shape it holds now
    std::map<int, std::pair<std::string, cudaGraphExec_t>> graphs;
};

struct Server {
    pf_scene scene;
    char *pool = nullptr;
    uint64_t pool_bytes = 0;
    char *scene_ws = nullptr;
    pf_serve_opts opts;
    int max_batch = 1;
    std::vector<Slot *> slots;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request *> queue;
    std::unordered_map<uint64_t, Request *> reqs;
    uint64_t next_id = 1;
    std::thread worker;
    std::atomic<bool> stop{false};
    std::atomic<int> pending_completions{0};
    pf_status worker_error = PF_OK;
    double t_stop = -1;
    // statistics
    std::vector<double> lat;
    uint64_t submitted = 0, completed = 0, rejected = 0, batches = 0, batch_views = 0, replays = 0, requeued = 0,
             updates = 0;
    double pixels_done = 0, t_first = -1, t_last = 0;
};

// Host function at the end of a batch's stream: record the time, wake the worker.
static void CUDART_CB batch_done(void *p) {
    Slot *s = (Slot *)p;
    s->t_finished = now_ms();
    s->finished.store(1);
    s->srv->pending_completions.fetch_add(1);
    s->srv->cv.notify_one();
}

// The multi-view plan of a batch placed in a slot's region.
static void plan_for(const Server &S, Slot &sl, const std::vector<Request *> &b, uint64_t cap, Plan &p,
                     std::vector<pf_camera> &cams) {
    p = Plan();
    cams.resize(b.size());
    for (size_t i = 0; i < b.size(); i++) cams[i] = b[i]->cam;
    p.n = S.scene.n_cells;
    p.k = S.scene.k_nbr;
    p.nv = (int)b.size();
    p.cap = cap;
    p.stats = 0;
    p.external_scene = true;
    p.scene_ws = S.scene_ws;
    p.fwd_only = true;
    p.views_host = sl.views_pinned;
    fill_views(&p, cams.data());
    make_layout(&p);
}

// Largest instance capacity for which the batch fits the slot, or 0.
static uint64_t fit_capacity(const Server &S, Slot &sl, const std::vector<Request *> &b) {
    Plan p;
    std::vector<pf_camera> cams;
    plan_for(S, sl, b, 0, p, cams);
    const uint64_t base = p.L.total + 4096;
    if (base >= sl.ws_bytes) return 0;
    uint64_t cap = (sl.ws_bytes - base) / 28;  // bytes per instance over the instance arrays
    if (cap > 0xE0000000ull) cap = 0xE0000000ull;
    // the layout rounds each region up to 256 bytes: step down until it fits
    while (cap > 0) {
        plan_for(S, sl, b, cap, p, cams);
        if (p.L.total <= sl.ws_bytes) return cap;
        cap = cap > 4096 ? cap - 4096 : 0;
    }
    return 0;
}

static std::string signature(const std::vector<Request *> &b, uint64_t cap) {
    std::string s;
    char buf[48];
    for (auto *r : b) {
        snprintf(buf, sizeof buf, "%dx%d,", r->cam.width, r->cam.height);
        s += buf;
    }
    snprintf(buf, sizeof buf, "|%llu", (unsigned long long)cap);
    return s + buf;
}

// Enqueue one batch's work on the slot's stream.
static cudaError_t enqueue_batch(Server &S, Slot &sl, const Plan &p) {
    const WS w = p.ws(sl.ws);
    cudaStream_t st = sl.stream;
    cudaError_t e = cudaMemcpyAsync(w.views, sl.views_pinned, sizeof(ViewDev) * p.nv, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_project(S.scene, p, w, st);
    if (e == cudaSuccess) e = launch_bin_sort(p, w, st);
    if (e == cudaSuccess) e = launch_render_fwd(S.scene, p, w, nullptr, nullptr, nullptr, false, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sl.ctr_pinned, w.counters, sizeof(Counters), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaLaunchHostFunc(st, batch_done, &sl);
    return e;
}

static cudaError_t launch_batch(Server &S, Slot &sl, uint64_t cap) {
    Plan p;
    std::vector<pf_camera> cams;
    plan_for(S, sl, sl.batch, cap, p, cams);
    for (int v = 0; v < p.nv; v++) {
        sl.views_pinned[v].out_rgb = sl.batch[v]->rgb;
        sl.views_pinned[v].out_T = sl.batch[v]->T;
        sl.views_pinned[v].out_last = nullptr;
    }
    sl.finished.store(0);
    if (!S.opts.use_graphs) return enqueue_batch(S, sl, p);
    // Each slot keeps one executable graph per view count.  A batch of the
    // shape (resolutions in order, capacity) that graph holds replays it as
    // it is.  A batch of another shape with the same number of views has the
    // same launch sequence with other grid sizes and arguments: it is
    // captured (cheap) and written into that executable graph with
    // cudaGraphExecUpdate, with no new instantiation; only a first batch of
    // its view count, or an update the runtime refuses, instantiates.
    const std::string key = signature(sl.batch, cap);
    const int nv = (int)sl.batch.size();
    auto it = sl.graphs.find(nv);
    if (it != sl.graphs.end() && it->second.first == key) {
        S.replays++;
        return cudaGraphLaunch(it->second.second, sl.stream);
    }
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(sl.stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    e = enqueue_batch(S, sl, p);
    cudaError_t e2 = cudaStreamEndCapture(sl.stream, &g);
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return e;
    }
    if (e2 != cudaSuccess) return e2;
    if (it != sl.graphs.end()) {
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(it->second.second, g, &info) == cudaSuccess) {
            cudaGraphDestroy(g);
            it->second.first = key;
            S.updates++;
            return cudaGraphLaunch(it->second.second, sl.stream);
        }
        cudaGetLastError();  // a refused update leaves no error behind
        cudaGraphExecDestroy(it->second.second);
        sl.graphs.erase(it);
    }
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return e;
    sl.graphs[nv] = std::make_pair(key, ex);
    return cudaGraphLaunch(ex, sl.stream);
}

// Complete finished batches (lock held).
static void reap(Server &S) {
    for (Slot *sl : S.slots) {
        if (!sl->busy || !sl->finished.load()) continue;
        S.pending_completions.fetch_sub(1);
        sl->busy = false;
        if (sl->ctr_pinned->overflow) {  // render the requests again, one per batch
            for (auto it = sl->batch.rbegin(); it != sl->batch.rend(); ++it) {
                if ((*it)->solo) {
                    (*it)->done = -1;  // does not fit even alone
                } else {
                    (*it)->solo = 1;
                    S.queue.push_front(*it);
                    S.requeued++;
                }
            }
        } else {
            for (Request *r : sl->batch) {
                r->t_done = sl->t_finished;
                r->done = 1;
                S.completed++;
                S.lat.push_back(r->t_done - r->t_submit);
                S.pixels_done += (double)r->cam.width * r->cam.height;
                S.t_last = std::max(S.t_last, r->t_done);
            }
        }
        sl->batch.clear();
    }
}

static void worker_main(Server *Sp) {
    Server &S = *Sp;
    std::unique_lock<std::mutex> lk(S.mu);
    while (true) {
        reap(S);
        bool launched = false;
        for (Slot *sl : S.slots) {
            if (sl->busy || S.queue.empty()) continue;
            // admit in arrival order while the batch fits this slot's memory
            std::vector<Request *> b;
            uint64_t cap = 0;
            while (!S.queue.empty() && (int)b.size() < S.max_batch) {
                Request *r = S.queue.front();
                if (r->solo && !b.empty()) break;
                b.push_back(r);
                const uint64_t c = fit_capacity(S, *sl, b);
                const uint64_t px = [&] {
                    uint64_t t = 0;
                    for (auto *q : b) t += (uint64_t)q->cam.width * q->cam.height;
                    return t;
                }();
                if (c < px / 4 + 1024) {  // too little room left for instances: stop here
                    b.pop_back();
                    break;
                }
                cap = c;
                S.queue.pop_front();
                if (r->solo) break;
            }
            if (b.empty()) {  // the head request does not fit an idle slot: fail it
                Request *r = S.queue.front();
                S.queue.pop_front();
                r->done = -1;
                S.cv.notify_all();
                continue;
            }
            sl->batch = b;
            sl->busy = true;
            S.batches++;
            S.batch_views += b.size();
            lk.unlock();
            cudaError_t e = launch_batch(S, *sl, cap);
            lk.lock();
            if (e != cudaSuccess) {
                S.worker_error = PF_ERR_CUDA;
                set_error("serve: %s", cudaGetErrorString(e));
                for (Request *r : sl->batch) r->done = -1;
                sl->batch.clear();
                sl->busy = false;
            }
            launched = true;
        }
        S.cv.notify_all();
        bool any_busy = false;
        for (Slot *sl : S.slots) any_busy |= sl->busy;
        if (S.stop.load()) {
            if (S.t_stop < 0) S.t_stop = now_ms();
            // in-flight batches get a bounded time to finish
            if (!any_busy || now_ms() - S.t_stop > 10000.0) break;
        }
        if (!launched)
            S.cv.wait_for(lk, std::chrono::milliseconds(1),
                          [&] { return S.stop.load() || S.pending_completions.load() > 0; });
    }
}

static uint64_t request_bytes_alone(const Server &S, const pf_camera &cam) {
    Plan p = Plan();
    ViewDev vh;
    p.n = S.scene.n_cells;
    p.k = S.scene.k_nbr;
    p.nv = 1;
    p.cap = (uint64_t)cam.width * cam.height / 4 + 1024;
    p.external_scene = true;
    p.fwd_only = true;
    p.views_host = &vh;
    fill_views(&p, &cam);
    make_layout(&p);
    return p.L.total;
}

}  // namespace pf

using namespace pf;

struct pf_server : public Server {};

extern "C" {

pf_status pf_serve_create(const pf_scene *scene, void *pool, uint64_t pool_bytes, const pf_serve_opts *opts,
                          pf_server **out) {
    set_error("%s", "");
    if (!scene || !pool || !opts || !out || opts->slots < 1 || opts->slots > 16 || opts->max_batch_views < 1 ||
        opts->max_batch_views > 256 || opts->max_queue < 1) {
        set_error("pf_serve_create: bad arguments");
        return PF_ERR_INVALID_ARG;
    }
    if (((uintptr_t)pool & 255) != 0) {
        set_error("pf_serve_create: pool must be 256-byte aligned");
        return PF_ERR_INVALID_ARG;
    }
    Plan chk;
    chk.n = scene->n_cells;
    chk.k = scene->k_nbr;
    if (scene->k_nbr < 0 || scene->k_nbr > MAX_K || scene->n_cells < 0 || !scene_ok(scene, &chk))
        return PF_ERR_INVALID_ARG;
    pf_server *S = new pf_server();
    S->scene = *scene;
    S->pool = (char *)pool;
    S->pool_bytes = pool_bytes;
    S->opts = *opts;
    S->max_batch = opts->max_batch_views;
    const SceneLayout SL = make_scene_layout(scene->n_cells, scene->k_nbr);
    if (SL.total >= pool_bytes) {
        set_error("pf_serve_create: pool of %llu bytes cannot hold the scene records (%llu)",
                  (unsigned long long)pool_bytes, (unsigned long long)SL.total);
        delete S;
        return PF_ERR_CAPACITY;
    }
    S->scene_ws = S->pool;
    const uint64_t per = align_up((pool_bytes - SL.total) / opts->slots, 256) - 256;
    pf_status st = PF_OK;
    for (int i = 0; i < opts->slots && !st; i++) {
        Slot *sl = new Slot();
        sl->srv = S;
        sl->index = i;
        sl->ws = S->pool + SL.total + (uint64_t)i * (per + 256);
        sl->ws_bytes = per;
        st = cuda_status(cudaStreamCreateWithFlags(&sl->stream, cudaStreamNonBlocking), "serve stream");
        if (!st) st = cuda_status(cudaHostAlloc((void **)&sl->views_pinned, sizeof(ViewDev) * opts->max_batch_views,
                                                cudaHostAllocDefault), "serve pinned views");
        if (!st) st = cuda_status(cudaHostAlloc((void **)&sl->ctr_pinned, sizeof(Counters), cudaHostAllocDefault),
                                  "serve pinned counters");
        S->slots.push_back(sl);
    }
    if (!st) {  // prepare the resident scene once
        Plan p = Plan();
        p.n = scene->n_cells;
        p.k = scene->k_nbr;
        p.external_scene = true;
        p.scene_ws = S->scene_ws;
        WS w = p.ws(S->slots[0]->ws);
        st = cuda_status(launch_prepare(*scene, p, w, S->slots[0]->stream), "serve prepare");
        if (!st) st = cuda_status(cudaStreamSynchronize(S->slots[0]->stream), "serve prepare sync");
    }
    if (st) {
        pf_serve_destroy(S);
        return st;
    }
    S->worker = std::thread(worker_main, S);
    *out = S;
    return PF_OK;
}

pf_status pf_serve_submit(pf_server *S, const pf_camera *cam, float *rgb, float *T, uint64_t *req_id) {
    if (!S || !cam || !rgb || !T || !req_id) return PF_ERR_INVALID_ARG;
    if (!camera_ok(*cam)) {
        set_error("pf_serve_submit: invalid camera");
        return PF_ERR_INVALID_ARG;
    }
    if (request_bytes_alone(*S, *cam) > S->slots[0]->ws_bytes) {
        set_error("pf_serve_submit: a %dx%d view does not fit a slot of %llu bytes", cam->width, cam->height,
                  (unsigned long long)S->slots[0]->ws_bytes);
        return PF_ERR_CAPACITY;
    }
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop.load()) return PF_ERR_INVALID_ARG;
    if ((int)S->queue.size() >= S->opts.max_queue) {
        S->rejected++;
        set_error("pf_serve_submit: queue full (%d)", S->opts.max_queue);
        return PF_ERR_BUSY;
    }
    Request *r = new Request();
    r->id = S->next_id++;
    r->cam = *cam;
    r->rgb = rgb;
    r->T = T;
    r->t_submit = now_ms();
    if (S->t_first < 0) S->t_first = r->t_submit;
    S->reqs[r->id] = r;
    S->queue.push_back(r);
    S->submitted++;
    *req_id = r->id;
    S->cv.notify_all();
    return PF_OK;
}

pf_status pf_serve_poll(pf_server *S, uint64_t id, int32_t timeout_ms, int32_t *done) {
    if (!S || !done) return PF_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(id);
    if (it == S->reqs.end()) return PF_ERR_NOT_FOUND;
    Request *r = it->second;
    if (!r->done && timeout_ms > 0)
        S->cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return r->done != 0; });
    *done = r->done;
    if (r->done) {
        S->reqs.erase(it);
        const int d = r->done;
        delete r;
        if (d < 0) {
            set_error("pf_serve_poll: request %llu failed", (unsigned long long)id);
            return S->worker_error ? S->worker_error : PF_ERR_CAPACITY;
        }
        return PF_OK;
    }
    return timeout_ms > 0 ? PF_ERR_TIMEOUT : PF_OK;
}

pf_status pf_serve_stats(pf_server *S, pf_serve_report *out) {
    if (!S || !out) return PF_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    memset(out, 0, sizeof *out);
    out->submitted = S->submitted;
    out->completed = S->completed;
    out->rejected = S->rejected;
    out->batches = S->batches;
    out->graph_replays = S->replays;
    out->graph_updates = S->updates;
    out->requeued = S->requeued;
    out->mean_batch_views = S->batches ? (double)S->batch_views / S->batches : 0;
    if (!S->lat.empty()) {
        std::vector<double> l = S->lat;
        std::sort(l.begin(), l.end());
        auto q = [&](double f) { return l[std::min(l.size() - 1, (size_t)(f * (l.size() - 1) + 0.5))]; };
        out->p50_ms = q(0.5);
        out->p99_ms = q(0.99);
        out->max_ms = l.back();
        double s = 0;
        for (double x : l) s += x;
        out->mean_ms = s / l.size();
        out->elapsed_s = (S->t_last - S->t_first) * 1e-3;
        if (out->elapsed_s > 0) {
            out->requests_per_s = S->completed / out->elapsed_s;
            out->mpix_per_s = S->pixels_done / out->elapsed_s * 1e-6;
        }
    }
    return PF_OK;
}

pf_status pf_serve_reset_stats(pf_server *S) {
    if (!S) return PF_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    S->lat.clear();
    S->submitted = S->completed = S->rejected = S->batches = S->batch_views = S->replays = S->requeued = 0;
    S->updates = 0;
    S->pixels_done = 0;
    S->t_first = -1;
    S->t_last = 0;
    return PF_OK;
}

void pf_serve_destroy(pf_server *S) {
    if (!S) return;
    if (S->worker.joinable()) {
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->stop.store(true);
            // queued requests that never launched are dropped
            for (Request *r : S->queue) r->done = -1;
            S->queue.clear();
        }
        S->cv.notify_all();
        S->worker.join();
    }
    for (Slot *sl : S->slots) {
        if (sl->stream) cudaStreamSynchronize(sl->stream);
        for (auto &kv : sl->graphs) cudaGraphExecDestroy(kv.second.second);
        if (sl->stream) cudaStreamDestroy(sl->stream);
        if (sl->views_pinned) cudaFreeHost(sl->views_pinned);
        if (sl->ctr_pinned) cudaFreeHost(sl->ctr_pinned);
        delete sl;
    }
    for (auto &kv : S->reqs) delete kv.second;
    delete S;
}

}  // extern "C"
