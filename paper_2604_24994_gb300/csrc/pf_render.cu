// pf_render_fwd / pf_render_bwd: per-pixel ray/cell segments, front-to-back
// compositing, and the back-to-front adjoint replay.
//
// One CTA per 16x16 tile, one thread per pixel; each warp covers an 8x4
// pixel block.  The tile's sorted cell list is staged into shared memory in
// batches of 32 cells with cp.async (16-byte granules): the 128-byte cell
// record, the 32-byte view record and the cell's relevant radical planes.
// The segment model and the staging helpers are in pf_render_common.cuh.
#include "pf_render_common.cuh"

namespace pf {

// ---------------------------------------------------------------- forward
// STATS: count work (see pf_stats); REC: record the hit masks the backward
// replays (only with a hit-mask region in the workspace); CONTRIB: add each
// cell's contributions (Sec. 4: T alpha for L_sparse and the pruning EMA,
// T alpha max(nh.d, 0)^2 for L_normal) over the frame's pixels.
template <bool STATS, bool REC, bool CONTRIB, bool EXT = false, int NS = 4>
__global__ void __launch_bounds__(TILE_PIX, 4) render_fwd_kernel(RenderArgs A, int64_t n_tiles,
                                                                 float *__restrict__ rgb_out,
                                                                 float *__restrict__ T_out,
                                                                 uint32_t *__restrict__ last_out) {
    extern __shared__ float4 smem4[];
    __shared__ int64_t s_q, s_slot;
    constexpr int XW = NS == 8 ? 12 : 3;  // float4s of extended face model per staged cell
    const Stage sg = make_stage(smem4, A.K, false, XW);
    const int lane = threadIdx.x & 31;
    unsigned long long st_cand = 0, st_hit = 0, st_pl = 0, st_ref = 0, st_pass = 0;
    unsigned long long st_wcand = 0, st_wpass = 0, st_whit = 0;  // per warp (lane 0 counts)
    const bool overflow = A.w.counters->overflow != 0;

    // persistent CTAs take tiles from the queue, heaviest lists first
    for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_q = atomicAdd(&A.w.counters->q_fwd, 1u);
    __syncthreads();
    if (s_q >= n_tiles) break;
    const int64_t tile = A.w.tile_order[s_q];
    const int v = find_view(A.w.views, A.nv, tile);
    const ViewDev &V = A.w.views[v];
    int px, py, wx, wy;
    tile_pixel(V, tile - V.tile_base, px, py, wx, wy);
    const bool inside = px < V.width && py < V.height;
    const Ray ray = pixel_ray(V, px, py);
    const Cone cone = warp_cone(ray);
    const bool has_ray = pixel_has_ray(V, px, py);

    unsigned long long s = A.w.tile_start[tile], e = A.w.tile_start[tile + 1];
    if (s > A.cap) s = A.cap;
    if (e > A.cap) e = A.cap;
    if (overflow) e = s;
    const int64_t vbase = (int64_t)v * A.n;
    const int n = (int)(e - s);
    if (threadIdx.x == 0) s_slot = (int64_t)(s / BATCH) + tile;
    const int nbat = (n + BATCH - 1) / BATCH;

    float T = 1.0f;
    float3 C = f3(0.f, 0.f, 0.f);
    uint32_t last = 0;
    int nhit = 0;  // hits so far (hit recording)
    bool done = !inside || !has_ray;

    const float *disp = EXT ? A.disp : nullptr, *sites = EXT ? A.sites : nullptr;
    const float *tex8 = NS == 8 ? A.tex8 : nullptr;
    if (nbat > 0)
        issue_batch(sg, 0, A.w.inst_sorted + s, min(BATCH, n), A.w, vbase, A.K, false, disp, sites, tex8);
    for (int k = 0; k < nbat; k++) {
        // one barrier per batch: this thread's copies of batch k have landed, so
        // after it everyone's have, and every warp is done with batch k-1, whose
        // buffer batch k+1 (in flight while batch k is shaded) reuses
        cp_async_wait_all();
        if (__syncthreads_count(!done) == 0) break;
        if (k + 1 < nbat)
            issue_batch(sg, (k + 1) & 1, A.w.inst_sorted + s + (k + 1) * BATCH, min(BATCH, n - (k + 1) * BATCH),
                        A.w, vbase, A.K, false, disp, sites, tex8);
        const int buf = k & 1, nb = min(BATCH, n - k * BATCH);
        unsigned mask = warp_mask(sg, buf, nb, cone);
        unsigned my_hits = 0;  // bit j: this pixel's segment in cell j of the batch is non-empty
        while (mask) {
            const int j = __ffs(mask) - 1;
            mask &= mask - 1;
            const float *cr = sg.cr(buf) + j * CELLREC_F;
            const float *vr = sg.vr(buf) + j * VIEWREC_F;
            Chord ch;
            bool cand = false, pass = false;
            if (!done) pass = sphere_chord<false>(cr, vr, ray, ch, cand);
            const unsigned pm = __ballot_sync(0xffffffffu, pass);
            bool hit = false;
            Seg seg;
            int np = 0;
            // the cell's extended face model in shared memory: four sites,
            // displacement then positions; eight, texture, displacement, positions
            const float *xj = EXT ? reinterpret_cast<const float *>(sg.xtr(buf) + XW * j) : nullptr;
            const float *st = EXT && sites ? xj + (NS == 8 ? 32 : 4) : nullptr;
            if (pm) {
                const int o = sg.poff(buf)[j];
                np = sg.poff(buf)[j + 1] - o;
                if (pass)
                    hit = clip_chord<false, STATS, EXT, NS>(
                        cr, vr, sg.pl(buf) + o, np, A.w.planes_lo + (int64_t)sg.ids(buf)[j] * A.K, ray, ch, seg, pm,
                        EXT && disp && NS == 4 ? sg.xtr(buf)[3 * j] : float4{0.f, 0.f, 0.f, 0.f}, st, EXT && disp,
                        NS == 8 ? xj + 24 : nullptr);
            }
            if (STATS && !done) {
                const unsigned act = __ballot_sync(__activemask(), true);
                const bool l0 = lane == __ffs(act) - 1;
                const unsigned cm = __ballot_sync(act, cand), hm = __ballot_sync(act, hit);
                st_cand++;
                st_pass += cand;
                st_pl += pass ? seg.nplanes : 0;
                st_ref += pass ? (hit ? seg.refined : ch.refined) : 0;
                st_hit += hit;
                st_wcand += l0;
                st_wpass += l0 && cm;
                st_whit += l0 && hm;
            }
            if (CONTRIB && __any_sync(0xffffffffu, hit)) {
                // T alpha and T alpha max(nh.d, 0)^2 of the hit lanes, summed
                // over the warp in 2^-24 fixed point (integer warp reduction:
                // 32 terms <= 1 stay below 2^29), one atomic per value and cell
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
                    atomicAdd((lane ? A.contrib_normal : A.contrib_sparse) + sg.ids(buf)[j],
                              (float)(lane ? qn : qw) * 0x1p-24f);
            }
            if (!hit) continue;
            if (REC) {
                const int64_t rp = V.pix_base + (int64_t)py * V.width + px;
                const unsigned kinds = (unsigned)((seg.ka + 3) | ((seg.kb + 3) << 7));
                if (nhit < HIT_CAP) A.w.hitkind[rp * HIT_CAP + nhit] = (uint16_t)kinds;
                // stored segments (pf_plan_store_segments): the ends and the transmittance before
                if (A.segrec && nhit < A.seg_cap)
                    A.segrec[rp * A.seg_cap + nhit] = make_float4(seg.sa, seg.sb, T, __uint_as_float(kinds));
                nhit++;
            }
            TexT<NS> tx;
            const float3 c = face_colour<NS>(cr, seg, ray, tx, st,
                                             EXT && A.sv ? A.sv + 48 * NS * (int64_t)sg.ids(buf)[j] : nullptr,
                                             NS == 8 ? xj : nullptr);
            const float x = fminf(cr[CR_SIG] * (seg.sb - seg.sa), X_CAP);
            const float ex = __expf(-x);
            const float wgt = T * (1.0f - ex);
            C.x = fmaf(wgt, c.x, C.x);
            C.y = fmaf(wgt, c.y, C.y);
            C.z = fmaf(wgt, c.z, C.z);
            T *= ex;
            last = (uint32_t)(k * BATCH + j + 1);
            if (REC) my_hits |= 1u << j;
            if (T < T_EPS) done = true;
        }
        // the backward replays only the (cell, pixel) pairs recorded here
        if (REC) A.w.hitmask[((int64_t)(threadIdx.x >> 5) * A.mask_batches + s_slot + k) * 32 + (threadIdx.x & 31)] = my_hits;
    }
    cp_async_wait_all();  // a batch may still be in flight after an early exit
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
    }  // tile queue
    if (STATS) {
        unsigned long long *st = A.w.counters->stats;
        for (int o = 16; o > 0; o >>= 1) {
            st_cand += __shfl_xor_sync(0xffffffffu, st_cand, o);
            st_hit += __shfl_xor_sync(0xffffffffu, st_hit, o);
            st_pl += __shfl_xor_sync(0xffffffffu, st_pl, o);
            st_ref += __shfl_xor_sync(0xffffffffu, st_ref, o);
            st_pass += __shfl_xor_sync(0xffffffffu, st_pass, o);
            st_wcand += __shfl_xor_sync(0xffffffffu, st_wcand, o);
            st_wpass += __shfl_xor_sync(0xffffffffu, st_wpass, o);
            st_whit += __shfl_xor_sync(0xffffffffu, st_whit, o);
        }
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(&st[0], st_cand);
            atomicAdd(&st[1], st_hit);
            atomicAdd(&st[2], st_pl);
            atomicAdd(&st[3], st_ref);
            atomicAdd(&st[4], st_pass);
            atomicAdd(&st[5], st_wcand);
            atomicAdd(&st[6], st_wpass);
            atomicAdd(&st[7], st_whit);
        }
    }
}

// A stored hit (pf_plan_store_segments): the forward's segment ends, the
// transmittance in front of it and its active constraints, so the ends are
// not recomputed.  The d.a of the end constraints are formed in float, and
// from FP64 where the backward's criterion asks for it (the adjoint divides
// by them), as in segment_from_kinds.
template <bool EXT, int NS>
__device__ __forceinline__ bool segment_from_record(const float *__restrict__ cr, const float *__restrict__ vr,
                                                    const float4 *__restrict__ pl, const float4 *__restrict__ lo_glob,
                                                    const Ray &ray, const Chord &ch, float4 rec, Seg &sg, float4 dk,
                                                    const float *__restrict__ st, bool has_disp,
                                                    const float *__restrict__ dk8) {
    const unsigned kinds = __float_as_uint(rec.w);
    const int ka = (int)(kinds & 127u) - 3, kb = (int)(kinds >> 7) - 3;
    const float3 dh = ray.dh, q = ch.q;
    const float R = cr[CR_R];
    const float sig = cr[CR_SIG];
    const float3 n = f3(cr[CR_N], cr[CR_N + 1], cr[CR_N + 2]);
    float foff = cr[CR_OFF];
    const float fden = dot3(dh, n);
    if (EXT && has_disp) {  // the displaced face's offset, for an FP64 d.n at a face end
        const float fnum = foff - dot3(q, n);
        foff += NS == 8 ? face_delta8(cr, q, dh, fnum, fden, dk8, nullptr, st)
                        : face_delta(cr, q, dh, fnum, fden, dk, nullptr, st);
    }
    sg.dnd = fden;
    if (fabsf(fden) < 0x1p-20f) sg.dnd = face_side64(cr, ray);
    const float4 Pa = pl[max(ka, 0)], Pb = pl[max(kb, 0)];
    float dena = ka >= 0 ? dot3(dh, f3(Pa.x, Pa.y, Pa.z)) : (ka == K_FACE ? fden : CUDART_INF_F);
    float denb = kb >= 0 ? dot3(dh, f3(Pb.x, Pb.y, Pb.z)) : (kb == K_FACE ? fden : CUDART_INF_F);
    const float lim = PLANE_ERR * sig * (1.0f / REFINE_EPS);
    const float4 face_hi = make_float4(cr[CR_N], cr[CR_N + 1], cr[CR_N + 2], foff);
    const float4 face_lo = make_float4(cr[CR_NLO], cr[CR_NLO + 1], cr[CR_NLO + 2], 0.f);
    float d64;
    if (fabsf(dena) < fmaxf(lim * (R + fabsf(rec.x)), GRAD_DEN)) {
        refine_plane64(vr, ka >= 0 ? Pa : face_hi, ka >= 0 ? lo_glob[ka] : face_lo, ray, rec.x, d64);
        dena = d64;
    }
    if (fabsf(denb) < fmaxf(lim * (R + fabsf(rec.y)), GRAD_DEN)) {
        refine_plane64(vr, kb >= 0 ? Pb : face_hi, kb >= 0 ? lo_glob[kb] : face_lo, ray, rec.y, d64);
        denb = d64;
    }
    sg.sa = rec.x;
    sg.sb = rec.y;
    sg.ka = ka;
    sg.kb = kb;
    sg.dena = dena;
    sg.denb = denb;
    sg.q = q;
    sg.refined = 0;
    return true;
}

// --------------------------------------------------------------- backward
// A cell that at most this many lanes of a warp hit adds each lane's
// gradients with atomics; more hit lanes sum them over the warp first.
constexpr int BWD_DIRECT_LANES = 6;

// Sum v[0..31] over the warp with each lane ending up holding one index:
// after five exchange rounds lane l holds sum_lanes v[l] (31 shuffles).
__device__ __forceinline__ float warp_transpose_sum(float (&v)[32], int lane) {
#pragma unroll
    for (int k = 0; k < 16; k++) {
        const bool up = lane & 16;
        const float keep = up ? v[k + 16] : v[k];
        const float give = up ? v[k] : v[k + 16];
        v[k] = keep + __shfl_xor_sync(0xffffffffu, give, 16);
    }
#pragma unroll
    for (int k = 0; k < 8; k++) {
        const bool up = lane & 8;
        const float keep = up ? v[k + 8] : v[k];
        const float give = up ? v[k] : v[k + 8];
        v[k] = keep + __shfl_xor_sync(0xffffffffu, give, 8);
    }
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const bool up = lane & 4;
        const float keep = up ? v[k + 4] : v[k];
        const float give = up ? v[k] : v[k + 4];
        v[k] = keep + __shfl_xor_sync(0xffffffffu, give, 4);
    }
#pragma unroll
    for (int k = 0; k < 2; k++) {
        const bool up = lane & 2;
        const float keep = up ? v[k + 2] : v[k];
        const float give = up ? v[k] : v[k + 2];
        v[k] = keep + __shfl_xor_sync(0xffffffffu, give, 2);
    }
    {
        const bool up = lane & 1;
        const float keep = up ? v[1] : v[0];
        const float give = up ? v[0] : v[1];
        v[0] = keep + __shfl_xor_sync(0xffffffffu, give, 1);
    }
    return v[0];
}

// dL/dn through the face frame (Duff et al., JCGT 2017) for u = (e1.y, e2.y)/R
// with dL/du = (c1, c2) R: dL/de1 = c1 y, dL/de2 = c2 y, and
// e1 = (1 + s x^2 a, s b, -s x), e2 = (b, s + y^2 a, -y), b = x y a.
__device__ __forceinline__ float3 frame_grad(const float *__restrict__ cr, float c1, float c2, float3 y) {
    const float3 g1 = f3(c1 * y.x, c1 * y.y, c1 * y.z);
    const float3 g2 = f3(c2 * y.x, c2 * y.y, c2 * y.z);
    const float nx = cr[CR_N], ny = cr[CR_N + 1], nz = cr[CR_N + 2];
    const float sgn = nz >= 0.f ? 1.f : -1.f;
    const float ca = -rcp_approx(sgn + nz);
    const float da = ca * ca;
    const float db0 = ny * ca, db1 = nx * ca, db2 = nx * ny * da;
    return f3(g1.x * (2.f * sgn * nx * ca) + g1.y * sgn * db0 + g1.z * (-sgn) + g2.x * db0,
              g1.y * sgn * db1 + g2.x * db1 + g2.y * (2.f * ny * ca) + g2.z * (-1.f),
              g1.x * (sgn * nx * nx * da) + g1.y * sgn * db2 + g2.x * db2 + g2.y * (ny * ny * da));
}

// dL/ds of one segment end -> gradients of its active constraint, the same
// instructions for every kind (the lanes of a warp meet different kinds).
// y = q + s d is the end point relative to p_i; the constraint c(y) = rhs
// has normal nrm with d.nrm = dn, so ds/dm = -nrm/dn and ds/d(rhs) = 1/dn:
//   sphere |y|^2 = R^2:  nrm = y, dn = y.d = s,  rhs = R^2/2 (ds/dR = R/s)
//   face   n.y = off:    nrm = n, dn = d.n,      ds/dn = -y/dn
//   plane  a.y = g:      nrm = a, dn = d.a,      ds/da = -y/dn
//   camera (s = m.d):    no parameter of cell i; contributes nothing here.
// Lanes whose end is not of a kind see that kind's terms multiplied by 0,
// with their operands replaced by finite stand-ins first.
__device__ __forceinline__ void route_end(float gt, int kind, float s, float den, const Seg &sg, const Ray &ray,
                                          const float *cr, const float4 *pl, const int2 *nb, float3 &gm, float (&v)[32],
                                          float (&nbv)[4], int &nbj) {
    const bool sph = kind == K_SPHERE, face = kind == K_FACE, plane = kind >= 0;
    const float3 d = ray.dh;
    const float3 y = f3(fmaf(s, d.x, sg.q.x), fmaf(s, d.y, sg.q.y), fmaf(s, d.z, sg.q.z));
    float4 P = pl[max(kind, 0)];
    const int2 J = nb[max(kind, 0)];
    if (!plane) P = make_float4(0.f, 0.f, 0.f, 0.f);
    const float L = plane ? __int_as_float(J.y) : 1.0f;
    const float3 nf = f3(cr[CR_N], cr[CR_N + 1], cr[CR_N + 2]);
    const float3 nrm = sph ? y : (face ? nf : f3(P.x, P.y, P.z));
    const float dn = sph ? s : den;
    const float id = (sph || face || plane) ? gt * rcp_approx(dn) : 0.0f;
    gm.x -= id * nrm.x;
    gm.y -= id * nrm.y;
    gm.z -= id * nrm.z;
    v[G_R] += (sph ? id : 0.0f) * cr[CR_R];
    const float fid = face ? id : 0.0f;
    v[G_N] -= fid * y.x;
    v[G_N + 1] -= fid * y.y;
    v[G_N + 2] -= fid * y.z;
    v[G_OFF] += fid;
    // plane of neighbour j: dL/da_unit = -id y, dL/dg = id, with a_unit = A/L,
    // g = (L^2 + w_i - w_j)/(2L), A = p_j - p_i
    const float pid = plane ? id : 0.0f;
    const float3 a = f3(P.x, P.y, P.z);
    const float3 ga = f3(-pid * y.x, -pid * y.y, -pid * y.z);
    const float pa = dot3(a, ga);
    const float iL = rcp_approx(L);
    const float cg = pid * (1.0f - P.w * iL);
    const float3 dA = f3((ga.x - a.x * pa) * iL + cg * a.x, (ga.y - a.y * pa) * iL + cg * a.y,
                         (ga.z - a.z * pa) * iL + cg * a.z);
    v[G_P] -= dA.x;
    v[G_P + 1] -= dA.y;
    v[G_P + 2] -= dA.z;
    v[G_W] += 0.5f * pid * iL;
    nbv[0] = dA.x;
    nbv[1] = dA.y;
    nbv[2] = dA.z;
    nbv[3] = -0.5f * pid * iL;
    nbj = plane ? J.x : -1;
}

// MASKS: replay only the (cell, lane) pairs the forward recorded as hits
// (the hit masks of the current bins); otherwise re-test every listed cell.
// CONTRIB: also the adjoint of sum_i (w_sparse[i] sparse_i + w_normal[i]
// normal_i), the per-cell contributions of pf_render_fwd_contrib (Sec. 4's
// L_sparse / L_normal): along a ray they composite the scalar
// q_k = w_sparse + w_normal max(nh.d, 0)^2 like a fourth colour channel whose
// upstream gradient is 1, and q_k itself moves with the unit normal.
// STORE: read the segments the forward stored (pf_plan_store_segments)
// instead of recomputing their ends and the transmittance.
template <bool MASKS, bool EXT = false, int NS = 4, bool CONTRIB = false, bool STORE = false>
__global__ void __launch_bounds__(TILE_PIX, 3) render_bwd_kernel(RenderArgs A, int64_t n_tiles,
                                                                 const float *__restrict__ dL_drgb,
                                                                 const float *__restrict__ dL_dT,
                                                                 const float *__restrict__ T_in,
                                                                 const uint32_t *__restrict__ last_in) {
    extern __shared__ float4 smem4[];
    __shared__ int s_maxlast;
    __shared__ int64_t s_q;
    constexpr int XW = NS == 8 ? 12 : 3;  // float4s of extended face model per staged cell
    const Stage stg = make_stage(smem4, A.K, true, XW);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool overflow = A.w.counters->overflow != 0;

    for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) {
        s_q = atomicAdd(&A.w.counters->q_bwd, 1u);
        s_maxlast = 0;
    }
    __syncthreads();
    if (s_q >= n_tiles) break;
    const int64_t tile = A.w.tile_order[s_q];
    const int v = find_view(A.w.views, A.nv, tile);
    const ViewDev &V = A.w.views[v];
    int px, py, wx, wy;
    tile_pixel(V, tile - V.tile_base, px, py, wx, wy);
    const bool inside = px < V.width && py < V.height;
    const Ray ray = pixel_ray(V, px, py);
    const Cone cone = warp_cone(ray);
    unsigned long long s = A.w.tile_start[tile], e = A.w.tile_start[tile + 1];
    if (s > A.cap) s = A.cap;
    if (e > A.cap) e = A.cap;
    if (overflow) e = s;
    const int64_t vbase = (int64_t)v * A.n;

    float3 g = f3(0.f, 0.f, 0.f);
    float gT = 0.f, Tf = 1.f;
    int last = 0;
    int nrec = 0;  // the forward's hit count; hits are met in reverse order
    const int64_t pix = inside ? V.pix_base + (int64_t)py * V.width + px : 0;
    if (inside) {
        g = f3(dL_drgb[3 * pix], dL_drgb[3 * pix + 1], dL_drgb[3 * pix + 2]);
        gT = dL_dT ? dL_dT[pix] : 0.f;
        Tf = T_in[pix];
        last = (int)last_in[pix];
        if ((unsigned long long)last > e - s) last = (int)(e - s);
        if (MASKS) nrec = (int)A.w.hitcount[pix];
    }
    // the record of the next hit this lane meets (ordinal nrec - 1), loaded
    // one hit ahead so that its latency hides behind the current one
    unsigned kk_next = 0xffffu;
    if (MASKS && nrec > 0 && nrec - 1 < HIT_CAP) kk_next = A.w.hitkind[pix * HIT_CAP + nrec - 1];
    atomicMax(&s_maxlast, last);
    __syncthreads();
    const int maxlast = s_maxlast;

    float Tafter = Tf;
    float accQ = 0.f;  // CONTRIB: the contribution scalar composited behind the current cell
    float3 accC = f3(0.f, 0.f, 0.f);
    float *acc = A.w.acc;
    const uint32_t *list = A.w.inst_sorted + s;

    // batches of the list prefix [0, maxlast) in the forward's partition,
    // walked back to front; batch b-1 is copied while batch b is replayed
    const int nbat = (maxlast + BATCH - 1) / BATCH;
    if (nbat > 0)
        issue_batch(stg, (nbat - 1) & 1, list + (nbat - 1) * BATCH, maxlast - (nbat - 1) * BATCH, A.w, vbase, A.K,
                    true, EXT ? A.disp : nullptr, EXT ? A.sites : nullptr, NS == 8 ? A.tex8 : nullptr);
    for (int b = nbat - 1; b >= 0; b--) {
        // bit j: the forward found this pixel's segment in cell j non-empty
        const unsigned my_hits = MASKS ? A.w.hitmask[hitmask_slot(A, tile, s, b, warp) + lane] : 0u;
        // one barrier per batch: this thread's copies of batch b have landed, so
        // after it everyone's have, and batch b+1 (whose buffer batch b-1 reuses)
        // is done; batch b-1's copies are in flight while batch b is replayed
        cp_async_wait_all();
        __syncthreads();
        if (b > 0)
            issue_batch(stg, (b - 1) & 1, list + (b - 1) * BATCH, BATCH, A.w, vbase, A.K, true,
                        EXT ? A.disp : nullptr, EXT ? A.sites : nullptr, NS == 8 ? A.tex8 : nullptr);
        const int buf = b & 1, lo = b * BATCH, nb = min(BATCH, maxlast - lo);
        unsigned mask = MASKS ? __reduce_or_sync(0xffffffffu, my_hits) : warp_mask(stg, buf, nb, cone);
        const float *s_cr = stg.cr(buf);
        const float *s_vr = stg.vr(buf);
        const float4 *s_pl = stg.pl(buf);
        const int2 *s_nb = stg.nb(buf);
        const int *poff = stg.poff(buf);
        while (mask) {
            const int j = 31 - __clz(mask);
            mask &= ~(1u << j);
            const int idx = lo + j;
            const bool mine = MASKS ? ((my_hits >> j) & 1u) != 0 : idx < last;
            if (!MASKS && !__any_sync(0xffffffffu, mine)) continue;
            const int cell = stg.ids(buf)[j];
            const float *cr = s_cr + j * CELLREC_F;
            const float *vr = s_vr + j * VIEWREC_F;
            const bool has_disp = EXT && A.disp;
            // the cell's extended face model in shared memory (see Stage::xtr)
            const float *xj = EXT ? reinterpret_cast<const float *>(stg.xtr(buf) + XW * j) : nullptr;
            const float4 dk = has_disp && NS == 4 ? stg.xtr(buf)[3 * j] : float4{0.f, 0.f, 0.f, 0.f};
            const float *dk8 = NS == 8 && has_disp ? xj + 24 : nullptr;
            const float *st = EXT && A.sites ? xj + (NS == 8 ? 32 : 4) : nullptr;
            const int o = poff[j], np = poff[j + 1] - o;
            Seg sg;
            Chord ch;
            bool cand;
            bool hit = false;
            float4 srec = float4{0.f, 0.f, 0.f, 0.f};
            bool has_srec = false;  // the forward stored this hit's segment
            if (MASKS) {
                // the forward recorded this hit's active constraints: no plane loop
                unsigned kk = 0xffffu;
                if (mine) {
                    kk = kk_next;
                    --nrec;
                    kk_next = nrec > 0 && nrec - 1 < HIT_CAP ? A.w.hitkind[pix * HIT_CAP + nrec - 1] : 0xffffu;
                    if (STORE && A.segrec && nrec < A.seg_cap) {
                        srec = A.segrec[pix * A.seg_cap + nrec];
                        has_srec = true;
                    }
                }
                if (mine && sphere_chord<true>(cr, vr, ray, ch, cand)) {
                    if (STORE && has_srec)
                        hit = segment_from_record<EXT, NS>(cr, vr, s_pl + o, A.w.planes_lo + (int64_t)cell * A.K, ray,
                                                           ch, srec, sg, dk, st, has_disp, dk8);
                    else if (kk != 0xffffu)
                        hit = segment_from_kinds<true, EXT, NS>(cr, vr, s_pl + o,
                                                                A.w.planes_lo + (int64_t)cell * A.K, ray, ch,
                                                                (int)(kk & 127u) - 3, (int)(kk >> 7) - 3, sg, dk, st,
                                                                has_disp, dk8);
                    else  // beyond the recorded hits of this pixel: clip against every plane
                        hit = clip_chord<true, false, EXT, NS>(cr, vr, s_pl + o, np,
                                                               A.w.planes_lo + (int64_t)cell * A.K, ray, ch, sg, 0u, dk,
                                                               st, has_disp, dk8);
                }
            } else if (mine && sphere_chord<true>(cr, vr, ray, ch, cand)) {
                hit = clip_chord<true, false, EXT, NS>(cr, vr, s_pl + o, np, A.w.planes_lo + (int64_t)cell * A.K,
                                                       ray, ch, sg, 0u, dk, st, has_disp, dk8);
            }
            if (!__any_sync(0xffffffffu, hit)) continue;
            // Every lane runs the adjoint of this cell.  A lane without a hit
            // runs it on neutral inputs (an empty segment with camera ends at
            // the site, zero dL/dx and colour weight), so all its values are 0.
            if (!hit) {
                sg.sa = 0.f;
                sg.sb = 0.f;
                sg.ka = K_CAMERA;
                sg.kb = K_CAMERA;
                sg.dena = 1.f;
                sg.denb = 1.f;
                sg.q = f3(0.f, 0.f, 0.f);
                sg.dnd = 1.f;
            }
            float vv[32];
            float nba[4], nbb[4];
            int ja, jb;
            {
                TexT<NS> tx;
                const float *svc = EXT && A.sv ? A.sv + 48 * NS * (int64_t)cell : nullptr;
                const float3 c = face_colour<NS>(cr, sg, ray, tx, st, svc, NS == 8 ? xj : nullptr);
                const float sig = cr[CR_SIG];
                const float l = sg.sb - sg.sa;
                const float xr = sig * l;
                const float x = fminf(xr, X_CAP);
                const float ex = __expf(-x);
                const float alpha = 1.0f - ex;
                const float Tbefore = STORE && has_srec ? srec.z : Tafter * __expf(x);
                // x = sigma l, alpha = 1 - e^-x:  dL/dx = g.(T_{k+1} c - S_k) - gT T_final
                float dLdx = g.x * (Tafter * c.x - accC.x) + g.y * (Tafter * c.y - accC.y) +
                             g.z * (Tafter * c.z - accC.z) - gT * Tf;
                float qk = 0.f, ndq = 0.f;
                if (CONTRIB) {
                    ndq = dot3(f3(cr[CR_N], cr[CR_N + 1], cr[CR_N + 2]), ray.dh);
                    qk = __ldg(A.w_sparse + cell) + __ldg(A.w_normal + cell) * (ndq > 0.0f ? ndq * ndq : 0.0f);
                    dLdx += Tafter * qk - accQ;
                }
                if (xr > X_CAP || !hit) dLdx = 0.f;
                vv[G_SIG] = dLdx * l;
                const float gl = dLdx * sig;
                const float wc = hit ? Tbefore * alpha : 0.0f;
                const float3 gc = f3(wc * g.x, wc * g.y, wc * g.z);
                // texture values and soft-Voronoi weights
                float gW[NS], sW = 0.f;
                float gt8[NS == 8 ? 32 : 1];  // eight sites: the texture gradient, routed to memory below
                const float *tc = NS == 8 ? xj : cr + CR_TEX;
#pragma unroll
                for (int k = 0; k < NS; k++) {
                    // the site's colour weight (finalize: the tex gradient, and summed, the rgb one)
                    if constexpr (NS == 4) {
                        vv[G_TEX + 3 * k] = tx.W[k] * gc.x;
                        vv[G_TEX + 3 * k + 1] = tx.W[k] * gc.y;
                        vv[G_TEX + 3 * k + 2] = tx.W[k] * gc.z;
                    } else {
                        gt8[3 * k] = tx.W[k] * gc.x;
                        gt8[3 * k + 1] = tx.W[k] * gc.y;
                        gt8[3 * k + 2] = tx.W[k] * gc.z;
                    }
                    const float3 ck = svc ? sv_colour(svc, k, ray.dh) : f3(tc[3 * k], tc[3 * k + 1], tc[3 * k + 2]);
                    gW[k] = ck.x * gc.x + ck.y * gc.y + ck.z * gc.z;
                    sW += tx.W[k] * gW[k];
                }
                if constexpr (NS == 8) {
                    // the site weights sum to one: the rgb gradient is gc (finalize adds it);
                    // the 24 texture values are summed over the warp, one atomic each
#pragma unroll
                    for (int q = 0; q < 12; q++) vv[G_TEX + q] = q < 3 ? (q == 0 ? gc.x : (q == 1 ? gc.y : gc.z)) : 0.f;
                    if (!svc) {
#pragma unroll
                        for (int q = 24; q < 32; q++) gt8[q] = 0.f;
                        const float sum = warp_transpose_sum(gt8, lane);
                        if (lane < 24 && A.gtex8) atomicAdd(A.gtex8 + 24 * (int64_t)cell + lane, sum);
                    }
                }
                if (EXT && svc) {
                    // spherical-Voronoi site colours c_k = sum_j P_j rgb_j, P = softmax(lambda a_j.wo / |a_j|),
                    // wo = -d: dL/drgb_j = P_j W_k gc; dL/dlogit_j = P_j (gP_j - sum P gP) with
                    // gP_j = W_k gc.rgb_j; dL/da_j = (I - a a^T / |a|^2) lambda wo dL/dlogit_j / |a|.
                    // 48 values per site, summed over the warp in two transposed rounds of 24.
#pragma unroll 1
                    for (int k = 0; k < NS; k++) {
                        const float *pk = svc + 48 * k;
                        const float3 gck = f3(tx.W[k] * gc.x, tx.W[k] * gc.y, tx.W[k] * gc.z);
                        float P[8], gP[8], mx = -CUDART_INF_F, z = 0.f, sP = 0.f;
#pragma unroll
                        for (int j = 0; j < 8; j++) {
                            const float ax = __ldg(pk + 6 * j), ay = __ldg(pk + 6 * j + 1), az = __ldg(pk + 6 * j + 2);
                            P[j] = -SV_LAMBDA * (ax * ray.dh.x + ay * ray.dh.y + az * ray.dh.z) *
                                   rsqrtf(fmaf(ax, ax, fmaf(ay, ay, az * az)));
                            mx = fmaxf(mx, P[j]);
                            gP[j] = gck.x * __ldg(pk + 6 * j + 3) + gck.y * __ldg(pk + 6 * j + 4) +
                                    gck.z * __ldg(pk + 6 * j + 5);
                        }
#pragma unroll
                        for (int j = 0; j < 8; j++) {
                            P[j] = __expf(P[j] - mx);
                            z += P[j];
                        }
                        const float iz = 1.0f / z;
#pragma unroll
                        for (int j = 0; j < 8; j++) {
                            P[j] *= iz;
                            sP = fmaf(P[j], gP[j], sP);
                        }
#pragma unroll
                        for (int h = 0; h < 2; h++) {
                            float v[32];
#pragma unroll
                            for (int jj = 0; jj < 4; jj++) {
                                const int j = 4 * h + jj;
                                const float ax = __ldg(pk + 6 * j), ay = __ldg(pk + 6 * j + 1), az = __ldg(pk + 6 * j + 2);
                                const float ia = rsqrtf(fmaf(ax, ax, fmaf(ay, ay, az * az)));
                                const float3 ah = f3(ax * ia, ay * ia, az * ia);
                                const float gl = -SV_LAMBDA * P[j] * (gP[j] - sP);  // times wo = -d below
                                const float3 ga = f3(gl * ray.dh.x, gl * ray.dh.y, gl * ray.dh.z);
                                const float pa = dot3(ah, ga);
                                v[6 * jj] = (ga.x - ah.x * pa) * ia;
                                v[6 * jj + 1] = (ga.y - ah.y * pa) * ia;
                                v[6 * jj + 2] = (ga.z - ah.z * pa) * ia;
                                v[6 * jj + 3] = P[j] * gck.x;
                                v[6 * jj + 4] = P[j] * gck.y;
                                v[6 * jj + 5] = P[j] * gck.z;
                            }
#pragma unroll
                            for (int q = 24; q < 32; q++) v[q] = 0.f;
                            const float sum = warp_transpose_sum(v, lane);
                            if (lane < 24 && A.gsv)
                                atomicAdd(A.gsv + 48 * NS * (int64_t)cell + 48 * k + 24 * h + lane, sum);
                        }
                    }
                }
                float gu1 = 0.f, gu2 = 0.f;
                float gs[2 * NS];  // learned sites: r_k = |u - s_k|, so dL/ds_k = -dL/du through logit k
#pragma unroll
                for (int k = 0; k < NS; k++) {
                    const float gr = -KAPPA * tx.W[k] * (gW[k] - sW);
                    const float ir = tx.r[k] > 0.f ? gr * rcp_approx(tx.r[k]) : 0.0f;
                    const float dxk = st ? tx.u1 - st[2 * k] : (NS == 4 ? tx.ax[k & 1] : tx.u1 - site_x<NS>(k));
                    const float dyk = st ? tx.u2 - st[2 * k + 1] : (NS == 4 ? tx.ay[k >> 1] : tx.u2 - site_y<NS>(k));
                    gu1 = fmaf(ir, dxk, gu1);
                    gu2 = fmaf(ir, dyk, gu2);
                    gs[2 * k] = -ir * dxk;
                    gs[2 * k + 1] = -ir * dyk;
                }
                // u = (e1.y, e2.y)/R with e/R stored:  dL/dy, dL/dR, dL/dn via the frame
                const float3 E1 = f3(cr[CR_E1], cr[CR_E1 + 1], cr[CR_E1 + 2]);
                const float3 E2 = f3(cr[CR_E2], cr[CR_E2 + 1], cr[CR_E2 + 2]);
                const float R = cr[CR_R];
                const float3 gy = f3(gu1 * E1.x + gu2 * E2.x, gu1 * E1.y + gu2 * E2.y, gu1 * E1.z + gu2 * E2.z);
                const float iR = rcp_approx(R);
                vv[G_R] = -(gu1 * tx.u1 + gu2 * tx.u2) * iR;
                {
                    const float3 gn = frame_grad(cr, gu1 * iR, gu2 * iR, tx.ys);
                    vv[G_N] = gn.x;
                    vv[G_N + 1] = gn.y;
                    vv[G_N + 2] = gn.z;
                }
                vv[G_P] = 0.f;
                vv[G_P + 1] = 0.f;
                vv[G_P + 2] = 0.f;
                vv[G_W] = 0.f;
                vv[G_OFF] = 0.f;
                if (CONTRIB && ndq > 0.0f) {  // d(max(nh.d, 0)^2)/d nh = 2 (nh.d) d, weighted T alpha w_normal
                    const float gq = wc * __ldg(A.w_normal + cell) * 2.0f * ndq;
                    vv[G_N] = fmaf(gq, ray.dh.x, vv[G_N]);
                    vv[G_N + 1] = fmaf(gq, ray.dh.y, vv[G_N + 1]);
                    vv[G_N + 2] = fmaf(gq, ray.dh.z, vv[G_N + 2]);
                }
                // the texture point moves with its segment end: y_s = m + t_s d
                float3 gm = gy;
                const float gts = dot3(gy, ray.dh);
                const bool onb = sg.dnd > 0.f;
                const float gta = -gl + (onb ? 0.f : gts);
                const float gtb = gl + (onb ? gts : 0.f);
                const int2 *nbp = s_nb + o;
                const float4 *plp = s_pl + o;
                route_end(gta, sg.ka, sg.sa, sg.dena, sg, ray, cr, plp, nbp, gm, vv, nba, ja);
                route_end(gtb, sg.kb, sg.sb, sg.denb, sg, ray, cr, plp, nbp, gm, vv, nbb, jb);
                float gdk[NS];  // the site displacements' gradients
#pragma unroll
                for (int k = 0; k < NS; k++) gdk[k] = 0.f;
                if (EXT && has_disp) {
                    // the displaced face end moves with delta like with the offset
                    // (ds/d delta = 1/(d.n)); delta moves with the site displacements
                    // through W, and with u at the base crossing, whose point
                    // yb = q + sb d rides the base face (Eq. svdisp)
                    const float3 nf = f3(cr[CR_N], cr[CR_N + 1], cr[CR_N + 2]);
                    const bool fa = sg.ka == K_FACE, fb = sg.kb == K_FACE;
                    const float fden = dot3(ray.dh, nf);
                    TexT<NS> fd;
                    float dl;
                    if constexpr (NS == 8)
                        dl = face_delta8(cr, sg.q, ray.dh, cr[CR_OFF] - dot3(sg.q, nf), fden, dk8, &fd, st);
                    else
                        dl = face_delta(cr, sg.q, ray.dh, cr[CR_OFF] - dot3(sg.q, nf), fden, dk, &fd, st);
                    const float gd = (fa || fb) ? ((fa ? gta : 0.f) + (fb ? gtb : 0.f)) *
                                                      rcp_approx(fa ? sg.dena : sg.denb)
                                                : 0.f;
                    const float dk4[4] = {dk.x, dk.y, dk.z, dk.w};
                    float gv1 = 0.f, gv2 = 0.f;
#pragma unroll
                    for (int k = 0; k < NS; k++) {
                        gdk[k] = gd * fd.W[k];
                        const float gr = -KAPPA * gd * fd.W[k] * ((NS == 8 ? dk8[k] : dk4[k & 3]) - dl);
                        const float ir = fd.r[k] > 0.f ? gr * rcp_approx(fd.r[k]) : 0.0f;
                        const float dxk = st ? fd.u1 - st[2 * k] : (NS == 4 ? fd.ax[k & 1] : fd.u1 - site_x<NS>(k));
                        const float dyk = st ? fd.u2 - st[2 * k + 1] : (NS == 4 ? fd.ay[k >> 1] : fd.u2 - site_y<NS>(k));
                        gv1 = fmaf(ir, dxk, gv1);
                        gv2 = fmaf(ir, dyk, gv2);
                        gs[2 * k] -= ir * dxk;
                        gs[2 * k + 1] -= ir * dyk;
                    }
                    const float3 gyb = f3(gv1 * E1.x + gv2 * E2.x, gv1 * E1.y + gv2 * E2.y, gv1 * E1.z + gv2 * E2.z);
                    vv[G_R] -= (gv1 * fd.u1 + gv2 * fd.u2) * iR;
                    const float3 gn = frame_grad(cr, gv1 * iR, gv2 * iR, fd.ys);
                    const float id2 = fabsf(fden) > 0.f ? dot3(gyb, ray.dh) * rcp_approx(fden) : 0.f;
                    vv[G_N] += gn.x - id2 * fd.ys.x;
                    vv[G_N + 1] += gn.y - id2 * fd.ys.y;
                    vv[G_N + 2] += gn.z - id2 * fd.ys.z;
                    vv[G_OFF] += id2;
                    gm.x += gyb.x - id2 * nf.x;
                    gm.y += gyb.y - id2 * nf.y;
                    gm.z += gyb.z - id2 * nf.z;
                    if (NS == 4) {  // the four site displacements: summed over the warp, one atomic each
#pragma unroll
                        for (int k = 0; k < NS; k++) {
                            float v = gdk[k];
#pragma unroll
                            for (int o2 = 16; o2 > 0; o2 >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o2);
                            if (lane == 0 && A.gdisp) atomicAdd(A.gdisp + 4 * (int64_t)cell + k, v);
                        }
                    }
                }
                if (NS == 4 && EXT && st) {  // the eight site coordinates: summed over the warp, one atomic each
#pragma unroll
                    for (int k = 0; k < 2 * NS; k++) {
                        float v = gs[k];
#pragma unroll
                        for (int o2 = 16; o2 > 0; o2 >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o2);
                        if (lane == 0 && A.gsites) atomicAdd(A.gsites + 8 * (int64_t)cell + k, v);
                    }
                }
                if constexpr (NS == 8) {
                    // eight displacements and sixteen site coordinates in one transposed warp sum
                    if (has_disp || st) {
                        float e[32];
#pragma unroll
                        for (int q = 0; q < 8; q++) e[q] = has_disp ? gdk[q] : 0.f;
#pragma unroll
                        for (int q = 0; q < 16; q++) e[8 + q] = st ? gs[q] : 0.f;
#pragma unroll
                        for (int q = 24; q < 32; q++) e[q] = 0.f;
                        const float sum = warp_transpose_sum(e, lane);
                        if (lane < 8 && has_disp && A.gdisp) atomicAdd(A.gdisp + 8 * (int64_t)cell + lane, sum);
                        if (lane >= 8 && lane < 24 && st && A.gsites)
                            atomicAdd(A.gsites + 16 * (int64_t)cell + (lane - 8), sum);
                    }
                }
                // m = o - p
                vv[G_P] -= gm.x;
                vv[G_P + 1] -= gm.y;
                vv[G_P + 2] -= gm.z;
                accC.x = fmaf(wc, c.x, accC.x);
                accC.y = fmaf(wc, c.y, accC.y);
                accC.z = fmaf(wc, c.z, accC.z);
                if (CONTRIB) accQ = fmaf(wc, qk, accQ);
                if (hit) Tafter = Tbefore;
            }
            // few hit lanes: each adds its own values (cheaper than the transposed sum;
            // measured at 1080p / 1M: 6.63 -> 6.44 ms, best at up to six lanes)
            if (__popc(__ballot_sync(0xffffffffu, hit)) <= BWD_DIRECT_LANES) {
                if (hit) {
#pragma unroll
                    for (int q = 0; q < G_USED; q++) atomicAdd(acc + (int64_t)cell * ACC_F + q, vv[q]);
                    if (ja >= 0) {
                        float *d = acc + (int64_t)ja * ACC_F;
                        atomicAdd(d + G_P, nba[0]);
                        atomicAdd(d + G_P + 1, nba[1]);
                        atomicAdd(d + G_P + 2, nba[2]);
                        atomicAdd(d + G_W, nba[3]);
                    }
                    if (jb >= 0) {
                        float *d = acc + (int64_t)jb * ACC_F;
                        atomicAdd(d + G_P, nbb[0]);
                        atomicAdd(d + G_P + 1, nbb[1]);
                        atomicAdd(d + G_P + 2, nbb[2]);
                        atomicAdd(d + G_W, nbb[3]);
                    }
                }
                continue;
            }
            // neighbour gradients: fold into the warp sum when the warp agrees on j
            const unsigned ma = __ballot_sync(0xffffffffu, ja >= 0);
            const int ref_a = ma ? __shfl_sync(0xffffffffu, ja, __ffs(ma) - 1) : -1;
            const unsigned mb = __ballot_sync(0xffffffffu, jb >= 0);
            const int ref_b = mb ? __shfl_sync(0xffffffffu, jb, __ffs(mb) - 1) : -1;
            const bool fold_a = ja >= 0 && ja == ref_a, fold_b = jb >= 0 && jb == ref_b;
#pragma unroll
            for (int q = 0; q < 4; q++) {
                vv[G_NB_A + q] = fold_a ? nba[q] : 0.f;
                vv[G_NB_B + q] = fold_b ? nbb[q] : 0.f;
            }
            vv[30] = 0.f;
            vv[31] = 0.f;
            if (ja >= 0 && !fold_a) {
                float *d = acc + (int64_t)ja * ACC_F;
                atomicAdd(d + G_P, nba[0]);
                atomicAdd(d + G_P + 1, nba[1]);
                atomicAdd(d + G_P + 2, nba[2]);
                atomicAdd(d + G_W, nba[3]);
            }
            if (jb >= 0 && !fold_b) {
                float *d = acc + (int64_t)jb * ACC_F;
                atomicAdd(d + G_P, nbb[0]);
                atomicAdd(d + G_P + 1, nbb[1]);
                atomicAdd(d + G_P + 2, nbb[2]);
                atomicAdd(d + G_W, nbb[3]);
            }
            const float sum = warp_transpose_sum(vv, lane);
            if (lane < G_USED) {
                atomicAdd(acc + (int64_t)cell * ACC_F + lane, sum);
            } else if (lane < G_NB_B) {
                if (ref_a >= 0) atomicAdd(acc + (int64_t)ref_a * ACC_F + (lane - G_NB_A), sum);
            } else if (lane < G_NB_B + 4) {
                if (ref_b >= 0) atomicAdd(acc + (int64_t)ref_b * ACC_F + (lane - G_NB_B), sum);
            }
        }
    }
    cp_async_wait_all();
    }  // tile queue
}

// Accumulators -> parameter gradients.  n = |n| n^:  dL/dn = (I - n^ n^T) dL/dn^ / |n|;
// rgb enters the colour with weight 1, the texture sites with weights summing to 1.
__global__ void __launch_bounds__(256) finalize_kernel(int n, const float *__restrict__ acc,
                                                       const float *__restrict__ cellrec, pf_scene_grad G,
                                                       bool view_dependent, int nsite) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float *a = acc + (int64_t)i * ACC_F;
    const float *cr = cellrec + (int64_t)i * CELLREC_F;
    G.pos[3 * i] += a[G_P];
    G.pos[3 * i + 1] += a[G_P + 1];
    G.pos[3 * i + 2] += a[G_P + 2];
    G.w[i] += a[G_W];
    G.R[i] += a[G_R];
    G.sigma[i] += a[G_SIG];
    const float nx = cr[CR_N], ny = cr[CR_N + 1], nz = cr[CR_N + 2], nl = cr[CR_NLEN];
    const float gx = a[G_N], gy = a[G_N + 1], gz = a[G_N + 2];
    const float pr = nx * gx + ny * gy + nz * gz;
    const float inl = nl > 0.f ? 1.0f / nl : 0.f;
    G.normal[3 * i] += (gx - nx * pr) * inl;
    G.normal[3 * i + 1] += (gy - ny * pr) * inl;
    G.normal[3 * i + 2] += (gz - nz * pr) * inl;
    G.offset[i] += a[G_OFF];
    if (nsite == 8) {  // eight sites: the backward added tex itself and left the rgb gradient here
        G.rgb[3 * i] += a[G_TEX];
        G.rgb[3 * i + 1] += a[G_TEX + 1];
        G.rgb[3 * i + 2] += a[G_TEX + 2];
        return;
    }
    float r0 = 0.f, r1 = 0.f, r2 = 0.f;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const float t0 = a[G_TEX + 3 * k], t1 = a[G_TEX + 3 * k + 1], t2 = a[G_TEX + 3 * k + 2];
        if (!view_dependent) {  // (the spherical-Voronoi colours replace tex)
            G.tex[12 * i + 3 * k] += t0;
            G.tex[12 * i + 3 * k + 1] += t1;
            G.tex[12 * i + 3 * k + 2] += t2;
        }
        r0 += t0;
        r1 += t1;
        r2 += t2;
    }
    G.rgb[3 * i] += r0;
    G.rgb[3 * i + 1] += r1;
    G.rgb[3 * i + 2] += r2;
}

static RenderArgs make_args(const pf_scene &s, const Plan &p, const WS &w) {
    RenderArgs A;
    A.w = w;
    A.nv = p.nv;
    A.n = p.n;
    A.K = p.k;
    A.cap = p.cap;
    A.mask_batches = mask_batches(p);
    A.contrib_sparse = nullptr;
    A.contrib_normal = nullptr;
    A.disp = s.disp;
    A.gdisp = nullptr;
    A.sites = s.sites;
    A.gsites = nullptr;
    A.sv = s.sv;
    A.gsv = nullptr;
    A.tex8 = scene_sites(s) == 8 ? s.tex : nullptr;
    A.gtex8 = nullptr;
    A.w_sparse = nullptr;
    A.w_normal = nullptr;
    A.segrec = w.segrec;
    A.seg_cap = w.segrec ? p.seg_cap : 0;
    return A;
}

static size_t fwd_smem(int K) { return stage_bytes(K, false); }
static size_t bwd_smem(int K) { return stage_bytes(K, true); }

cudaError_t launch_render_fwd(const pf_scene &s, const Plan &p, const WS &w, float *rgb, float *T, uint32_t *last,
                              bool record, cudaStream_t st, float *contrib_sparse, float *contrib_normal) {
    if (p.total_tiles == 0) return cudaSuccess;
    if (pipe_applies(s, p, record, contrib_sparse != nullptr))
        return launch_render_fwd_pipe(s, p, w, rgb, T, last, record, st, contrib_sparse, contrib_normal);
    RenderArgs A = make_args(s, p, w);
    A.contrib_sparse = contrib_sparse;
    A.contrib_normal = contrib_normal;
    const bool contrib = contrib_sparse != nullptr;
    const bool disp = ext_face(s);  // an extended face model
    const bool eight = scene_sites(s) == 8;
    if (disp && p.stats) return cudaErrorNotSupported;  // the C API refuses this first
    const size_t smem = disp ? stage_bytes(p.k, false, true, eight ? 12 : 3) : fwd_smem(p.k);
    cudaError_t e = cudaMemsetAsync(&w.counters->q_fwd, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess) return e;
    auto k = disp && eight
                 ? (contrib ? (record ? render_fwd_kernel<false, true, true, true, 8>
                                      : render_fwd_kernel<false, false, true, true, 8>)
                            : (record ? render_fwd_kernel<false, true, false, true, 8>
                                      : render_fwd_kernel<false, false, false, true, 8>))
             : disp ? (contrib ? (record ? render_fwd_kernel<false, true, true, true>
                                         : render_fwd_kernel<false, false, true, true>)
                               : (record ? render_fwd_kernel<false, true, false, true>
                                         : render_fwd_kernel<false, false, false, true>))
             : contrib ? (record ? render_fwd_kernel<false, true, true> : render_fwd_kernel<false, false, true>)
             : p.stats ? render_fwd_kernel<true, false, false>
                       : (record ? render_fwd_kernel<false, true, false> : render_fwd_kernel<false, false, false>);
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k<<<persistent_grid(k, smem, p.total_tiles), TILE_PIX, smem, st>>>(A, p.total_tiles, rgb, T, last);
    return cudaGetLastError();
}

cudaError_t launch_render_bwd(const pf_scene &s, const Plan &p, const WS &w, const float *dL_drgb,
                              const float *dL_dT, const float *T, const uint32_t *last, const pf_scene_grad &g,
                              bool use_masks, cudaStream_t st, const float *w_sparse, const float *w_normal) {
    if (p.n == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(w.acc, 0, sizeof(float) * ACC_F * (size_t)p.n, st);
    if (e != cudaSuccess) return e;
    if (p.total_tiles > 0) {
        RenderArgs A = make_args(s, p, w);
        A.gdisp = g.disp;
        A.gsites = g.sites;
        A.gsv = g.sv;
        const bool disp = ext_face(s);  // an extended face model
        const bool eight = scene_sites(s) == 8;
        A.gtex8 = eight ? g.tex : nullptr;
        const size_t smem = disp ? stage_bytes(p.k, true, true, eight ? 12 : 3) : bwd_smem(p.k);
        e = cudaMemsetAsync(&w.counters->q_bwd, 0, sizeof(unsigned int), st);
        if (e != cudaSuccess) return e;
        const bool m = use_masks && w.hitmask;
        const bool cq = w_sparse != nullptr;  // the contributions' adjoint too
        A.w_sparse = w_sparse;
        A.w_normal = w_normal;
        const bool store = m && w.segrec != nullptr && !disp && !cq;  // stored segments to read
        auto kern =
            store ? render_bwd_kernel<true, false, 4, false, true>
            : cq ? (disp && eight ? (m ? render_bwd_kernel<true, true, 8, true> : render_bwd_kernel<false, true, 8, true>)
                  : disp        ? (m ? render_bwd_kernel<true, true, 4, true> : render_bwd_kernel<false, true, 4, true>)
                                : (m ? render_bwd_kernel<true, false, 4, true> : render_bwd_kernel<false, false, 4, true>))
               : (disp && eight ? (m ? render_bwd_kernel<true, true, 8> : render_bwd_kernel<false, true, 8>)
                  : disp        ? (m ? render_bwd_kernel<true, true> : render_bwd_kernel<false, true>)
                                : (m ? render_bwd_kernel<true> : render_bwd_kernel<false>));
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        kern<<<persistent_grid(kern, smem, p.total_tiles), TILE_PIX, smem, st>>>(A, p.total_tiles, dL_drgb, dL_dT, T,
                                                                                 last);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    finalize_kernel<<<(p.n + 255) / 256, 256, 0, st>>>(p.n, w.acc, w.cellrec, g, s.sv != nullptr, scene_sites(s));
    return cudaGetLastError();
}

}  // namespace pf
