// pf_render_fwd for the plain face model without hit recording, stats or
// contributions (rendering a view: the benchmark's forward step, the server,
// the static entry point): the same per-pixel segments and compositing as
// render_fwd_kernel (Sec. 3.1-3.3), fed by a shared-memory ring instead of
// double buffers behind CTA barriers.
//
// Each persistent CTA streams batches through PIPE_S stages.  A batch holds
// up to 32 consecutive cells of one tile's sorted list whose kept radical
// planes fit the stage's plane budget (PIPE_PLANES; a cell keeps at most
// K <= 64 planes, so every batch holds at least one cell).  One warp fills a
// stage: one lane per cell issues cp.async.bulk copies of the cell's
// 128-byte record, its 32-byte view record and its planes (16 bytes each),
// all completing on the stage's mbarrier, whose expected transaction count
// the warp sets first.  Each warp waits for the stage's barrier, shades the
// batch for its 8 x 4 pixels, and signals that it is done with the stage;
// the last of the eight warps to do so refills that stage with the batch
// PIPE_S further on.  When a tile's list is exhausted, the refilling warp
// takes the next tile from the queue, so batches of consecutive tiles follow
// each other in the ring: a warp finishing a tile writes its pixels and
// moves on to the next tile's batches without waiting for the other warps,
// up to PIPE_S - 1 batches ahead of the slowest one.  No CTA barrier is
// taken inside the loop.  Batches are issued in order (a refill waits for
// the previous batch's issue, which fixes where its own batch starts); a
// tile whose pixels are all done (T below T_EPS) is cut short.
//
// Every wait is bounded: a wait that runs out sets the counters' error word
// and the CTA stops after waiting (bounded) for its copies in flight.
#include "pf_render_common.cuh"

namespace pf {

constexpr int PIPE_S = 4;                 // stages in the ring
constexpr int PIPE_PLANES = 320;          // planes one stage holds
constexpr int PIPE_WARPS = TILE_PIX / 32; // warps per CTA, all of them shade
constexpr int PIPE_SPIN = 1 << 22;        // polls before a wait gives up (about a second)

struct PipeStage {
    float cr[BATCH * CELLREC_F];   // cell records
    float vr[BATCH * VIEWREC_F];   // (view, cell) records
    float4 pl[PIPE_PLANES];        // the cells' kept planes, back to back
    int ids[BATCH];                // cell indices
    int poff[BATCH + 1];           // first plane of each cell in pl
    int nb, lo;                    // cells in the batch, list index of its first cell
    int ts;                        // sequence number of the batch's tile, -1: the end marker
    int pad_;
};
static_assert(sizeof(PipeStage) % 16 == 0, "stages must stay 16-byte aligned");

__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// One poll of the phase with the given parity; true once it has completed.
__device__ __forceinline__ bool mbar_test(uint64_t *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for a phase: false if it did not complete in PIPE_SPIN polls.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity) {
    for (int it = 0; it < PIPE_SPIN; it++) {
        if (mbar_test(bar, parity)) return true;
        if (it > 64) __nanosleep(128);
    }
    return false;
}

// size bytes from global src to shared dst, completing on bar (16-byte
// aligned addresses, size a multiple of 16)
__device__ __forceinline__ void bulk_copy(void *dst, const void *src, unsigned size, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(size), "r"(smem_addr(bar))
        : "memory");
}

// A tile in flight: the ring carries batches of several consecutive tiles.
struct PipeTile {
    int64_t tile;               // global tile id
    unsigned long long s0;      // its list's first instance
    int n;                      // its list's length
    int v;                      // its view
    int ndone;                  // warps whose every pixel of this tile is done
    int pad_;
};
constexpr int PIPE_TR = 8;      // tiles in flight at most (> PIPE_S: a warp is at most PIPE_S - 1 batches ahead)

struct PipeShared {
    uint64_t full[PIPE_S];      // stage filled (transaction-counted)
    int consumed[PIPE_S];       // warps done with the stage's batch
    unsigned fills[PIPE_S];     // fills of each stage (for the drain after an abort)
    PipeTile tiles[PIPE_TR];    // by tile sequence number modulo PIPE_TR
    int issued;                 // batches issued so far (or known not to exist)
    int tseq;                   // sequence number of the tile being issued, -1 before the first
    int next;                   // list index of that tile's next batch
    int ended;                  // the tile queue is exhausted and the end marker is issued
    int abort;                  // a wait ran out
    int pad_;
};

// Issue the next batch into stage `st` (by one warp): the next cells of the
// tile being issued, or, when its list is exhausted (or every pixel of it is
// done), the first batch of the next tile from the queue, or the end marker.
// A tile with an empty list gets one empty batch, so that its pixels are
// written.  Lanes take the next 32 entries; the prefix of them whose planes
// fit the stage forms the batch.
__device__ __forceinline__ void pipe_issue(PipeStage &st, uint64_t *full, PipeShared &S, const RenderArgs &A,
                                           int64_t n_tiles) {
    const int lane = threadIdx.x & 31;
    int ts = S.tseq, next = S.next;
    if (S.ended) {
        return;  // nothing follows the end marker
    }
    if (lane == 0) {
        bool fresh = ts < 0;
        if (!fresh) {
            const PipeTile &T = S.tiles[ts % PIPE_TR];
            fresh = next >= T.n || (T.ndone == PIPE_WARPS && next > 0);
        }
        if (fresh) {
            const int64_t q = atomicAdd(&A.w.counters->q_fwd, 1u);
            if (q >= n_tiles) {
                ts = -1;
                S.ended = 1;
            } else {
                ts++;
                PipeTile &T = S.tiles[ts % PIPE_TR];
                T.tile = A.w.tile_order[q];
                unsigned long long s0 = A.w.tile_start[T.tile], e0 = A.w.tile_start[T.tile + 1];
                if (s0 > A.cap) s0 = A.cap;
                if (e0 > A.cap) e0 = A.cap;
                if (A.w.counters->overflow != 0) e0 = s0;
                T.s0 = s0;
                T.n = (int)(e0 - s0);
                T.v = find_view(A.w.views, A.nv, T.tile);
                T.ndone = 0;
                next = 0;
            }
        }
    }
    ts = __shfl_sync(0xffffffffu, ts, 0);
    next = __shfl_sync(0xffffffffu, next, 0);
    __syncwarp();
    int n = 0, id = 0, np = 0;
    const uint32_t *list = nullptr;
    int64_t vbase = 0;
    if (ts >= 0) {
        const PipeTile &T = S.tiles[ts % PIPE_TR];
        n = T.n;
        list = A.w.inst_sorted + T.s0;
        vbase = (int64_t)T.v * A.n;
    }
    const bool valid = next + lane < n;
    if (valid) {
        id = (int)list[next + lane];
        np = A.w.cellnp[id];
    }
    int incl = np;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    const bool take = valid && incl <= PIPE_PLANES;
    const int nb = __popc(__ballot_sync(0xffffffffu, take));  // the taken lanes are a prefix
    const int planes = nb > 0 ? __shfl_sync(0xffffffffu, incl, nb - 1) : 0;
    if (take) {
        st.ids[lane] = id;
        st.poff[lane + 1] = incl;
    }
    if (lane == 0) {
        st.poff[0] = 0;
        st.nb = nb;
        st.lo = next;
        st.ts = ts;
        S.tseq = ts < 0 ? S.tseq : ts;
        S.next = n == 0 ? 1 : next + nb;  // an empty list: its one empty batch is issued
    }
    // the stage's previous contents were read through the generic proxy
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncwarp();
    if (lane == 0) mbar_arrive_expect_tx(full, (unsigned)(nb * (CELLREC_F + VIEWREC_F) * 4 + planes * 16));
    __syncwarp();
    if (take) {
        bulk_copy(st.cr + lane * CELLREC_F, A.w.cellrec + (int64_t)id * CELLREC_F, CELLREC_F * 4, full);
        bulk_copy(st.vr + lane * VIEWREC_F, A.w.viewrec + (vbase + id) * VIEWREC_F, VIEWREC_F * 4, full);
        if (np > 0) bulk_copy(st.pl + (incl - np), A.w.planes + (int64_t)id * A.K, (unsigned)np * 16u, full);
    }
}

// Ballot of the batch's cells whose sphere can meet the warp's cone (the
// test of warp_mask, on a stage).
__device__ __forceinline__ unsigned pipe_mask(const PipeStage &st, int nb, const Cone &cone) {
    const int lane = threadIdx.x & 31;
    bool ov = false;
    if (lane < nb) {
        const float *vr = st.vr + lane * VIEWREC_F;
        const float R = st.cr[lane * CELLREC_F + CR_R];
        const float3 m = f3(vr[0], vr[1], vr[2]);
        const float tc = -dot3(m, cone.dc);
        const float3 u = cross3(m, cone.dc);
        const float mm = sqrtf(dot3(m, m));
        const float rho = sqrtf(dot3(u, u));
        const float lim = fmaf(fmaxf(tc, 0.0f), cone.tan_t, R * (1.0f + cone.tan_t * cone.tan_t)) + 1e-5f * (mm + R);
        ov = (tc <= R * 1.01f + 1e-5f * mm) || (rho <= lim);
        ov = ov && (tc + R >= -1e-5f * mm);
    }
    return __ballot_sync(0xffffffffu, ov);
}

// A warp's pixels of one tile (8 x 4, one per lane).
struct PipePixels {
    int ts = -1;                // tile sequence number, -1: none yet
    const ViewDev *V = nullptr;
    int px = 0, py = 0;
    bool inside = false;
    Ray ray;
    Cone cone;
    float T = 1.0f;
    float3 C = float3{0.f, 0.f, 0.f};
    uint32_t last = 0;
    bool done = true;
    bool warp_done = true;      // counted in the tile's ndone
};

__device__ __forceinline__ void pipe_write(const PipePixels &P, float *__restrict__ rgb_out, float *__restrict__ T_out,
                                           uint32_t *__restrict__ last_out) {
    if (!P.inside) return;
    const ViewDev &V = *P.V;
    const int64_t lp = (int64_t)P.py * V.width + P.px;
    if (V.out_rgb) {  // per-view outputs (serving)
        V.out_rgb[3 * lp] = P.C.x;
        V.out_rgb[3 * lp + 1] = P.C.y;
        V.out_rgb[3 * lp + 2] = P.C.z;
        if (V.out_T) V.out_T[lp] = P.T;
        if (V.out_last) V.out_last[lp] = P.last;
    } else {
        const int64_t pix = V.pix_base + lp;
        rgb_out[3 * pix] = P.C.x;
        rgb_out[3 * pix + 1] = P.C.y;
        rgb_out[3 * pix + 2] = P.C.z;
        T_out[pix] = P.T;
        last_out[pix] = P.last;
    }
}

__global__ void __launch_bounds__(TILE_PIX, 4) render_fwd_pipe_kernel(RenderArgs A, int64_t n_tiles,
                                                                      float *__restrict__ rgb_out,
                                                                      float *__restrict__ T_out,
                                                                      uint32_t *__restrict__ last_out) {
    extern __shared__ float4 smem4[];
    __shared__ PipeShared S;
    PipeStage *stage = reinterpret_cast<PipeStage *>(smem4);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        for (int s = 0; s < PIPE_S; s++) {
            mbar_init(&S.full[s], 1);
            S.fills[s] = 0;
            S.consumed[s] = 0;
        }
        S.abort = 0;
        S.tseq = -1;
        S.next = 0;
        S.ended = 0;
        S.issued = PIPE_S;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // the first PIPE_S batches, by warp 0
    if (warp == 0) {
        for (int b = 0; b < PIPE_S; b++) {
            const int e = *(volatile int *)&S.ended;
            pipe_issue(stage[b], &S.full[b], S, A, n_tiles);
            if (lane == 0 && !e) S.fills[b]++;
        }
    }
    __syncthreads();

    PipePixels P;
    for (int k = 0;; k++) {
        const int sidx = k % PIPE_S;
        PipeStage &st = stage[sidx];
        if (!mbar_wait(&S.full[sidx], (unsigned)(k / PIPE_S) & 1u)) {
            if (lane == 0) {
                atomicOr(&A.w.counters->wait_errors, 1u);
                atomicExch(&S.abort, 1);
            }
            break;
        }
        const int ts = st.ts, nb = st.nb, lo = st.lo;
        if (ts != P.ts || ts < 0) {  // a new tile (or the end marker): the previous tile is finished
            if (P.ts >= 0) pipe_write(P, rgb_out, T_out, last_out);
            if (ts < 0) break;
            const PipeTile &T = S.tiles[ts % PIPE_TR];
            P.ts = ts;
            P.V = &A.w.views[T.v];
            int wx, wy;
            tile_pixel(*P.V, T.tile - P.V->tile_base, P.px, P.py, wx, wy);
            P.inside = P.px < P.V->width && P.py < P.V->height;
            P.ray = pixel_ray(*P.V, P.px, P.py);
            P.cone = warp_cone(P.ray);
            P.T = 1.0f;
            P.C = f3(0.f, 0.f, 0.f);
            P.last = 0;
            P.done = !P.inside || !pixel_has_ray(*P.V, P.px, P.py);
            P.warp_done = false;
        }
        if (!P.warp_done && __all_sync(0xffffffffu, P.done)) {
            P.warp_done = true;
            if (lane == 0) atomicAdd(&S.tiles[ts % PIPE_TR].ndone, 1);
        }
        if (!P.warp_done) {
            const Ray &ray = P.ray;
            unsigned mask = pipe_mask(st, nb, P.cone);
            while (mask) {
                const int j = __ffs(mask) - 1;
                mask &= mask - 1;
                if (__all_sync(0xffffffffu, P.done)) break;
                const float *cr = st.cr + j * CELLREC_F;
                const float *vr = st.vr + j * VIEWREC_F;
                Chord ch;
                bool cand = false, pass = false;
                if (!P.done) pass = sphere_chord<false>(cr, vr, ray, ch, cand);
                const unsigned pm = __ballot_sync(0xffffffffu, pass);
                bool hit = false;
                Seg seg;
                if (pm) {
                    const int o = st.poff[j];
                    const int np = st.poff[j + 1] - o;
                    if (pass)
                        hit = clip_chord<false>(cr, vr, st.pl + o, np, A.w.planes_lo + (int64_t)st.ids[j] * A.K, ray,
                                                ch, seg, pm);
                }
                if (!hit) continue;
                Tex tx;
                const float3 c = face_colour<4>(cr, seg, ray, tx);
                const float x = fminf(cr[CR_SIG] * (seg.sb - seg.sa), X_CAP);
                const float ex = __expf(-x);
                const float wgt = P.T * (1.0f - ex);
                P.C.x = fmaf(wgt, c.x, P.C.x);
                P.C.y = fmaf(wgt, c.y, P.C.y);
                P.C.z = fmaf(wgt, c.z, P.C.z);
                P.T *= ex;
                P.last = (uint32_t)(lo + j + 1);
                if (P.T < T_EPS) P.done = true;
            }
        }
        // done with the stage: the last warp refills it with the batch PIPE_S further on
        __syncwarp();
        int refill = 0;
        if (lane == 0) {
            __threadfence_block();
            const int c = atomicAdd(&S.consumed[sidx], 1);
            refill = c == PIPE_WARPS - 1;
            if (refill) {
                __threadfence_block();
                S.consumed[sidx] = 0;
            }
        }
        refill = __shfl_sync(0xffffffffu, refill, 0);
        if (refill) {
            const int b = k + PIPE_S;
            // batches are issued in order: wait for batch b - 1's issue (already
            // done in practice: its issuer finished batch k - 1 before it could
            // arrive here)
            int ok = 1;
            if (lane == 0) {
                int it = 0;
                while (*(volatile int *)&S.issued != b && !*(volatile int *)&S.abort) {
                    if (++it > PIPE_SPIN) {
                        ok = 0;
                        break;
                    }
                    __nanosleep(64);
                }
                __threadfence_block();
            }
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) {
                if (lane == 0) {
                    atomicOr(&A.w.counters->wait_errors, 2u);
                    atomicExch(&S.abort, 1);
                }
                break;
            }
            if (!*(volatile int *)&S.abort) {
                const int e = *(volatile int *)&S.ended;
                pipe_issue(st, &S.full[sidx], S, A, n_tiles);
                if (lane == 0 && !e) S.fills[sidx]++;
            }
            __syncwarp();
            if (lane == 0) {
                __threadfence_block();
                *(volatile int *)&S.issued = b + 1;
            }
        }
        if (*(volatile int *)&S.abort) break;
    }
    // after an abort, let every stage's last fill land (bounded) before the CTA exits
    __syncthreads();
    if (threadIdx.x == 0 && S.abort) {
        for (int s = 0; s < PIPE_S; s++)
            if (S.fills[s] > 0) mbar_wait(&S.full[s], (S.fills[s] - 1) & 1u);
    }
}

bool pipe_applies(const pf_scene &s, const Plan &p, bool record, bool contrib) {
    return !ext_face(s) && !record && !contrib && !p.stats;
}

cudaError_t launch_render_fwd_pipe(const pf_scene &s, const Plan &p, const WS &w, float *rgb, float *T,
                                   uint32_t *last, cudaStream_t st) {
    RenderArgs A;
    A.w = w;
    A.nv = p.nv;
    A.n = p.n;
    A.K = p.k;
    A.cap = p.cap;
    A.mask_batches = 0;
    A.contrib_sparse = A.contrib_normal = nullptr;
    A.disp = A.sites = A.sv = A.tex8 = nullptr;
    A.gdisp = A.gsites = A.gsv = A.gtex8 = nullptr;
    A.w_sparse = A.w_normal = nullptr;
    (void)s;
    const size_t smem = sizeof(PipeStage) * PIPE_S;
    cudaError_t e = cudaMemsetAsync(&w.counters->q_fwd, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess) return e;
    cudaFuncSetAttribute(render_fwd_pipe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    render_fwd_pipe_kernel<<<persistent_grid(render_fwd_pipe_kernel, smem, p.total_tiles), TILE_PIX, smem, st>>>(
        A, p.total_tiles, rgb, T, last);
    return cudaGetLastError();
}

}  // namespace pf
