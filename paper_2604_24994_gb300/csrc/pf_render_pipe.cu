// pf_render_fwd for the plain face model and the extended one with four
// detail sites, with or without hit recording (rendering a view: the
// benchmark's forward and training steps, the server, the static entry
// point; stats, contributions, stored segments and eight sites keep
// render_fwd_kernel): the same per-pixel segments and compositing as
// render_fwd_kernel (Sec. 3.1-3.4), fed by a shared-memory ring instead of
// double buffers behind CTA barriers.
//
// The tile's sorted list is cut into batches of at most 32 cells whose kept
// radical planes fit a stage's plane budget (PIPE_PLANES; a cell keeps at
// most K <= 64 planes, so every batch holds at least one cell).  PIPE_S
// stages hold consecutive batches.  One warp fills a stage: one lane per
// cell issues cp.async.bulk copies of the cell's 128-byte record, its
// 32-byte view record, its planes (16 bytes each) and, for the extended
// face model, its displacement and site rows, all completing on the
// stage's mbarrier, whose expected transaction count the warp sets first.
// Each warp waits for a stage's barrier, shades the batch, and signals that
// it is done with the stage; the last of the eight warps to do so refills
// that stage with the batch PIPE_S further on.  Batches are issued in list
// order (a refill waits for the previous batch's issue, which fixes where
// its own batch starts).  So warps only meet once per tile, and a warp can
// run up to PIPE_S - 1 batches ahead of the slowest one.
//
// Every wait is bounded: a wait that runs out sets the counters' error word
// and the CTA stops after waiting (bounded) for its copies in flight.
#include "pf_render_common.cuh"

namespace pf {

constexpr int PIPE_S = 4;                 // stages in the ring
constexpr int PIPE_PLANES = 320;          // planes one stage holds
constexpr int PIPE_WARPS = TILE_PIX / 32; // warps per CTA, all of them shade
constexpr int PIPE_SPIN = 1 << 22;        // polls before a wait gives up (about a second)

// XW: float4s of extended face model per cell (0: the plain model; 3: four
// sites, displacement then positions, as in the batch-staged kernel's
// stages).
template <int XW>
struct PipeStage {
    float cr[BATCH * CELLREC_F];   // cell records
    float vr[BATCH * VIEWREC_F];   // (view, cell) records
    float4 pl[PIPE_PLANES];        // the cells' kept planes, back to back
    float4 xt[XW > 0 ? BATCH * XW : 1];  // the cells' extended face model
    int ids[BATCH];                // cell indices
    int poff[BATCH + 1];           // first plane of each cell in pl
    int nb, lo;                    // cells in the batch, list index of its first cell
    int pad_[2];
};
static_assert(sizeof(PipeStage<0>) % 16 == 0 && sizeof(PipeStage<3>) % 16 == 0,
              "stages must stay 16-byte aligned");

// The extended face model's arrays (null where the scene has none).
struct PipeExt {
    const float *disp, *sites;
};

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

// Wait for batch k's stage (phase parity `parity`) unless the batch is known
// never to come (*stop <= k).  1: filled, 0: no such batch, -1: the wait ran out.
__device__ __forceinline__ int mbar_wait_or_stop(uint64_t *bar, unsigned parity, const int *stop, int k) {
    for (int it = 0; it < PIPE_SPIN; it++) {
        if (mbar_test(bar, parity)) return 1;
        if (*(const volatile int *)stop <= k) return 0;
        if (it > 64) __nanosleep(128);
    }
    return -1;
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

struct PipeShared {
    uint64_t full[PIPE_S];     // stage filled (transaction-counted)
    int consumed[PIPE_S];      // warps done with the stage's batch
    unsigned fills[PIPE_S];    // fills of each stage so far: the next fill completes phase fills & 1
    int issued;                // batches of this tile issued (or known not to exist)
    int next;                  // list index where the next batch starts
    int abort;                 // a wait ran out
    int ndone;                 // warps whose every pixel is done (T below T_EPS, or no pixel)
    int stop;                  // no batch of this tile from this index on will be issued
    int pad_;
    int64_t q;                 // the tile taken from the queue
};

// Issue the batch starting at list index `next` (< n) into stage `st`, by
// the calling warp; returns the index after it.  Lanes take the next 32
// entries; the prefix of them whose planes fit the stage forms the batch.
// With XW > 0 each cell's extended face model rows come along (16-byte
// aligned rows of 16 and 32 bytes, as the batch-staged kernel's copies need).
template <int XW>
__device__ __forceinline__ int pipe_issue(PipeStage<XW> &st, uint64_t *full, const uint32_t *__restrict__ list, int n,
                                          int next, const WS &w, int64_t vbase, int K, const PipeExt &x) {
    const int lane = threadIdx.x & 31;
    int id = 0, np = 0;
    const bool valid = next + lane < n;
    if (valid) {
        id = (int)list[next + lane];
        np = w.cellnp[id];
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
    }
    // the stage's previous contents were read through the generic proxy
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncwarp();
    // bytes of one cell's extended rows: displacement 16, positions 32
    constexpr unsigned DISP_B = 16u, SITE_B = 32u;
    const unsigned xb = XW > 0 ? (x.disp ? DISP_B : 0u) + (x.sites ? SITE_B : 0u) : 0u;
    if (lane == 0)
        mbar_arrive_expect_tx(full, (unsigned)(nb * ((CELLREC_F + VIEWREC_F) * 4 + xb) + planes * 16));
    __syncwarp();
    if (take) {
        bulk_copy(st.cr + lane * CELLREC_F, w.cellrec + (int64_t)id * CELLREC_F, CELLREC_F * 4, full);
        bulk_copy(st.vr + lane * VIEWREC_F, w.viewrec + (vbase + id) * VIEWREC_F, VIEWREC_F * 4, full);
        if (np > 0) bulk_copy(st.pl + (incl - np), w.planes + (int64_t)id * K, (unsigned)np * 16u, full);
        if (XW == 3) {
            float4 *xr = st.xt + 3 * lane;
            if (x.disp) bulk_copy(xr, x.disp + (int64_t)id * 4, DISP_B, full);
            if (x.sites) bulk_copy(xr + 1, x.sites + (int64_t)id * 8, SITE_B, full);
        }
    }
    return next + nb;
}

// Ballot of the batch's cells whose sphere can meet the warp's cone (the
// test of warp_mask, on a stage).
template <int XW>
__device__ __forceinline__ unsigned pipe_mask(const PipeStage<XW> &st, int nb, const Cone &cone) {
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

// REC: record hits for the backward.  EXT: the extended face model with
// four detail sites (displacement, learned site positions, view-dependent
// site colours), as in the batch-staged kernel.
// CONTRIB: also add the per-cell contributions (Sec. 4's L_sparse and
// L_normal terms) into A.contrib_sparse / A.contrib_normal, as the
// batch-staged kernel does.
template <bool REC, bool EXT = false, int NS = 4, bool CONTRIB = false>
__global__ void __launch_bounds__(TILE_PIX, 4) render_fwd_pipe_kernel(RenderArgs A, int64_t n_tiles,
                                                                      float *__restrict__ rgb_out,
                                                                      float *__restrict__ T_out,
                                                                      uint32_t *__restrict__ last_out) {
    static_assert(NS == 4, "eight detail sites take the batch-staged kernel");
    constexpr int XW = EXT ? 3 : 0;
    extern __shared__ float4 smem4[];
    __shared__ PipeShared S;
    PipeStage<XW> *stage = reinterpret_cast<PipeStage<XW> *>(smem4);
    const PipeExt xm{EXT ? A.disp : nullptr, EXT ? A.sites : nullptr};
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        for (int s = 0; s < PIPE_S; s++) {
            mbar_init(&S.full[s], 1);
            S.fills[s] = 0;
        }
        S.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    const bool overflow = A.w.counters->overflow != 0;

    for (;;) {
        __syncthreads();  // every warp is done with the previous tile
        if (threadIdx.x == 0) {
            // a tile whose warps all finished early may leave batches in flight that
            // nobody waited for: let every stage's last fill land before reusing it
            for (int s = 0; s < PIPE_S; s++)
                if (S.fills[s] > 0 && !mbar_wait(&S.full[s], (S.fills[s] - 1) & 1u)) {
                    atomicOr(&A.w.counters->wait_errors, 4u);
                    S.abort = 1;
                }
            S.q = S.abort ? n_tiles : (int64_t)atomicAdd(&A.w.counters->q_fwd, 1u);
            for (int b = 0; b < PIPE_S; b++) S.consumed[b] = 0;
            S.ndone = 0;
            S.stop = 0x7fffffff;
        }
        __syncthreads();
        if (S.q >= n_tiles) break;
        // the fill count of each stage at the start of this tile: batch k waits for
        // phase (fills + k / PIPE_S) of stage k % PIPE_S
        unsigned f0 = 0;
#pragma unroll
        for (int s = 0; s < PIPE_S; s++) f0 |= (S.fills[s] & 1u) << s;
        const int64_t tile = A.w.tile_order[S.q];
        const int v = find_view(A.w.views, A.nv, tile);
        const ViewDev &V = A.w.views[v];
        unsigned long long s0 = A.w.tile_start[tile], e0 = A.w.tile_start[tile + 1];
        if (s0 > A.cap) s0 = A.cap;
        if (e0 > A.cap) e0 = A.cap;
        if (overflow) e0 = s0;
        const int n = (int)(e0 - s0);
        const uint32_t *list = A.w.inst_sorted + s0;
        const int64_t vbase = (int64_t)v * A.n;
        __syncthreads();  // every warp has read the fill counts
        // the first PIPE_S batches, by warp 0, while the others set up their rays
        if (warp == 0) {
            int next = 0;
            for (int b = 0; b < PIPE_S; b++) {
                if (next < n) {
                    next = pipe_issue<XW>(stage[b], &S.full[b], list, n, next, A.w, vbase, A.K, xm);
                    if (lane == 0) S.fills[b]++;
                } else if (lane == 0 && S.stop > b) {
                    S.stop = b;
                }
            }
            if (lane == 0) {
                S.next = next;
                S.issued = PIPE_S;
            }
        }
        int px, py, wx, wy;
        tile_pixel(V, tile - V.tile_base, px, py, wx, wy);
        const bool inside = px < V.width && py < V.height;
        const Ray ray = pixel_ray(V, px, py);
        const Cone cone = warp_cone(ray);
        const bool has_ray = pixel_has_ray(V, px, py);
        __syncthreads();

        float T = 1.0f;
        float3 C = f3(0.f, 0.f, 0.f);
        uint32_t last = 0;
        // REC: this lane's hit bits of the 32-entry list groups hg and hg + 1
        // (a batch of at most 32 cells spans at most two), written to the hit
        // masks as the batches move past them; hit records in list order
        unsigned hb0 = 0u, hb1 = 0u;
        int hg = 0, pend = 0, nhit = 0;
        const int64_t s_slot = (int64_t)(s0 / BATCH) + tile;
        const int64_t rp = V.pix_base + (int64_t)py * V.width + px;
        bool done = !inside || !has_ray;
        bool warp_done = false;  // counted in S.ndone
        bool more = n > 0;
        // Every warp consumes every batch that is issued, done or not (a warp that
        // left early would leave a stage without its eighth arrival, and the batch
        // another warp waits for would never be refilled).  Once every warp is done
        // the refilling warp issues no further batch and publishes where the tile
        // stops; a warp waiting for a batch from there on leaves the loop.
        for (int k = 0; more; k++) {
            if (!warp_done && __all_sync(0xffffffffu, done)) {
                warp_done = true;
                if (lane == 0) atomicAdd(&S.ndone, 1);
            }
            const int sidx = k % PIPE_S;
            PipeStage<XW> &st = stage[sidx];
            // every lane waits itself (each observes the phase: acquire for the stage's
            // data); a batch that never comes cannot also complete, so the lanes agree
            // unless one of them ran out of polls
            const int got = __reduce_min_sync(
                0xffffffffu, mbar_wait_or_stop(&S.full[sidx], ((f0 >> sidx) + (unsigned)(k / PIPE_S)) & 1u, &S.stop, k));
            if (got == 0) break;  // the tile stops before batch k
            if (got < 0) {
                if (lane == 0) {
                    atomicOr(&A.w.counters->wait_errors, 1u);
                    atomicExch(&S.abort, 1);
                }
                break;
            }
            const int nb = st.nb, lo = st.lo;
            if (REC) {
                if ((lo >> 5) > hg) {  // group hg is complete: the next batches start past it
                    A.w.hitmask[((int64_t)warp * A.mask_batches + s_slot + hg) * 32 + lane] = hb0;
                    hb0 = hb1;
                    hb1 = 0u;
                    hg++;
                }
                pend = lo + nb;
            }
            more = lo + nb < n;
            if (!warp_done) {
                unsigned mask = pipe_mask(st, nb, cone);
                while (mask) {
                    const int j = __ffs(mask) - 1;
                    mask &= mask - 1;
                    const float *cr = st.cr + j * CELLREC_F;
                    const float *vr = st.vr + j * VIEWREC_F;
                    Chord ch;
                    bool cand = false, pass = false;
                    if (!done) pass = sphere_chord<false>(cr, vr, ray, ch, cand);
                    const unsigned pm = __ballot_sync(0xffffffffu, pass);
                    bool hit = false;
                    Seg seg;
                    // the cell's extended face model in the stage: displacement, then positions
                    const float *xj = EXT ? reinterpret_cast<const float *>(st.xt + XW * j) : nullptr;
                    const float *sj = EXT && xm.sites ? xj + 4 : nullptr;
                    if (pm) {
                        const int o = st.poff[j];
                        const int np = st.poff[j + 1] - o;
                        if (pass)
                            hit = clip_chord<false, false, EXT, NS>(
                                cr, vr, st.pl + o, np, A.w.planes_lo + (int64_t)st.ids[j] * A.K, ray, ch, seg, pm,
                                EXT && xm.disp && NS == 4 ? st.xt[3 * j] : float4{0.f, 0.f, 0.f, 0.f}, sj,
                                EXT && xm.disp, nullptr);
                    }
                    if (CONTRIB && __any_sync(0xffffffffu, hit)) {
                        // T alpha and T alpha max(nh.d, 0)^2 of the hit lanes, summed over the
                        // warp in 2^-24 fixed point, one atomic per value and cell
                        unsigned qw = 0u, qn = 0u;
                        if (hit) {
                            const float cw = T * (1.0f - __expf(-fminf(cr[CR_SIG] * (seg.sb - seg.sa), X_CAP)));
                            const float nd = dot3(f3(cr[CR_N], cr[CR_N + 1], cr[CR_N + 2]), ray.dh);
                            qw = __float2uint_rn(cw * 0x1p24f);
                            qn = __float2uint_rn((nd > 0.0f ? cw * nd * nd : 0.0f) * 0x1p24f);
                        }
                        qw = __reduce_add_sync(0xffffffffu, qw);
                        qn = __reduce_add_sync(0xffffffffu, qn);
                        if (lane < 2)
                            atomicAdd((lane ? A.contrib_normal : A.contrib_sparse) + st.ids[j],
                                      (float)(lane ? qn : qw) * 0x1p-24f);
                    }
                    if (!hit) continue;
                    if (REC) {
                        const int idx = lo + j;
                        if ((idx >> 5) == hg)
                            hb0 |= 1u << (idx & 31);
                        else
                            hb1 |= 1u << (idx & 31);
                        if (nhit < HIT_CAP)
                            A.w.hitkind[rp * HIT_CAP + nhit] = (uint16_t)((seg.ka + 3) | ((seg.kb + 3) << 7));
                        nhit++;
                    }
                    TexT<NS> tx;
                    const float3 c = face_colour<NS>(cr, seg, ray, tx, sj,
                                                     EXT && A.sv ? A.sv + 48 * NS * (int64_t)st.ids[j] : nullptr,
                                                     nullptr);
                    const float x = fminf(cr[CR_SIG] * (seg.sb - seg.sa), X_CAP);
                    const float ex = __expf(-x);
                    const float wgt = T * (1.0f - ex);
                    C.x = fmaf(wgt, c.x, C.x);
                    C.y = fmaf(wgt, c.y, C.y);
                    C.z = fmaf(wgt, c.z, C.z);
                    T *= ex;
                    last = (uint32_t)(lo + j + 1);
                    if (T < T_EPS) done = true;
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
                // batches are issued in list order: wait for batch b - 1's issue
                // (already done in practice: its issuer finished batch k - 1 before
                // it could arrive here)
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
                const int next = *(volatile int *)&S.next;
                int after = next;
                const bool go = next < n && !*(volatile int *)&S.abort &&
                                *(volatile int *)&S.ndone < PIPE_WARPS && *(volatile int *)&S.stop > b;
                if (go) {
                    after = pipe_issue<XW>(st, &S.full[sidx], list, n, next, A.w, vbase, A.K, xm);
                    if (lane == 0) S.fills[sidx]++;
                }
                __syncwarp();
                if (lane == 0) {
                    S.next = after;
                    if (!go && S.stop > b) *(volatile int *)&S.stop = b;  // no batch from b on
                    __threadfence_block();
                    *(volatile int *)&S.issued = b + 1;
                }
            }
            if (*(volatile int *)&S.abort) break;
        }
        if (REC && pend > 0) {  // the last one or two groups of the batches consumed
            A.w.hitmask[((int64_t)warp * A.mask_batches + s_slot + hg) * 32 + lane] = hb0;
            if (((pend - 1) >> 5) > hg) A.w.hitmask[((int64_t)warp * A.mask_batches + s_slot + hg + 1) * 32 + lane] = hb1;
        }
        if (inside) {
            const int64_t lp = (int64_t)py * V.width + px;
            if (V.out_rgb) {  // per-view outputs (serving)
                V.out_rgb[3 * lp] = C.x;
                V.out_rgb[3 * lp + 1] = C.y;
                V.out_rgb[3 * lp + 2] = C.z;
                if (V.out_T) V.out_T[lp] = T;
                if (V.out_last) V.out_last[lp] = last;
            } else {
                const int64_t pix = V.pix_base + lp;
                rgb_out[3 * pix] = C.x;
                rgb_out[3 * pix + 1] = C.y;
                rgb_out[3 * pix + 2] = C.z;
                T_out[pix] = T;
                last_out[pix] = last;
                if (REC) A.w.hitcount[pix] = (uint32_t)nhit;
            }
        }
    }
    // the loop ends after thread 0 let every stage's last fill land (or gave up
    // waiting, after an abort): no copy is in flight when the CTA exits
}

bool pipe_applies(const pf_scene &s, const Plan &p, bool record, bool contrib) {
    // the plain face model and the extended one with four sites, with or without
    // hit recording and contributions.  Stored segments, work counts and eight
    // sites take the batch-staged kernel (eight sites' 192-byte rows make a
    // stage 16.5 KB, and at three CTAs per SM the ring measured 7% slower).
    (void)contrib;
    return scene_sites(s) != 8 && !p.stats && !(record && p.seg_cap > 0);
}

template <bool REC, bool EXT, int NS, bool CONTRIB>
static cudaError_t launch_pipe(const RenderArgs &A, const Plan &p, float *rgb, float *T, uint32_t *last,
                               cudaStream_t st) {
    constexpr int XW = EXT ? 3 : 0;
    const size_t smem = sizeof(PipeStage<XW>) * PIPE_S;
    auto k = render_fwd_pipe_kernel<REC, EXT, NS, CONTRIB>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k<<<persistent_grid(k, smem, p.total_tiles), TILE_PIX, smem, st>>>(A, p.total_tiles, rgb, T, last);
    return cudaGetLastError();
}

template <bool REC, bool CONTRIB>
static cudaError_t launch_pipe_model(const pf_scene &s, const RenderArgs &A, const Plan &p, float *rgb, float *T,
                                     uint32_t *last, cudaStream_t st) {
    return ext_face(s) ? launch_pipe<REC, true, 4, CONTRIB>(A, p, rgb, T, last, st)
                       : launch_pipe<REC, false, 4, CONTRIB>(A, p, rgb, T, last, st);
}

cudaError_t launch_render_fwd_pipe(const pf_scene &s, const Plan &p, const WS &w, float *rgb, float *T,
                                   uint32_t *last, bool record, cudaStream_t st, float *contrib_sparse,
                                   float *contrib_normal) {
    RenderArgs A;
    A.w = w;
    A.nv = p.nv;
    A.n = p.n;
    A.K = p.k;
    A.cap = p.cap;
    A.mask_batches = record ? mask_batches(p) : 0;
    A.contrib_sparse = contrib_sparse;
    A.contrib_normal = contrib_normal;
    A.disp = s.disp;
    A.sites = s.sites;
    A.sv = s.sv;
    A.tex8 = nullptr;
    A.gdisp = A.gsites = A.gsv = A.gtex8 = nullptr;
    A.w_sparse = A.w_normal = nullptr;
    A.segrec = nullptr;
    A.seg_cap = 0;
    cudaError_t e = cudaMemsetAsync(&w.counters->q_fwd, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess) return e;
    if (scene_sites(s) == 8) return cudaErrorNotSupported;  // pipe_applies excludes it
    const bool contrib = contrib_sparse != nullptr;
    if (contrib) return record ? launch_pipe_model<true, true>(s, A, p, rgb, T, last, st)
                               : launch_pipe_model<false, true>(s, A, p, rgb, T, last, st);
    return record ? launch_pipe_model<true, false>(s, A, p, rgb, T, last, st)
                  : launch_pipe_model<false, false>(s, A, p, rgb, T, last, st);
}

}  // namespace pf
