// Device helpers of the renderer, shared by its translation units
// (pf_render.cu: the batch-staged forward, the backward; pf_render_pipe.cu:
// the pipelined forward).
//
// Segment of the ray x(t) = o + t d in cell i (Sec. 3.2-3.3), in the local
// frame of the ray's closest approach to p_i:  with m = o - p_i and
// v = m x d, the offset q = d x v satisfies |q| = |v| and x - p_i = q + s d,
// s = t + m.d.  Then
//   sphere:   s in [-sqrt(D), sqrt(D)],  D = R^2 - |v|^2
//   camera:   s >= m.d                   (t >= 0)
//   plane k:  s (d.a) <= g - q.a         (unit a, g = plane distance)
//   face:     s (d.n) <= off - q.n       (dense half)
// v is computed from the FP64 offset m (a float pair) and the FP64 ray
// direction (a float pair) with error-free products, so q is accurate to a
// few float ulps of |q| <= R no matter how far the camera is.  Segment ends
// whose float error bound could move sigma * l by more than REFINE_EPS are
// recomputed in FP64 from the original parameters (a near-tangent sphere or
// a near-parallel plane / face).
#pragma once

#include "pf_internal.cuh"

namespace pf {

struct Seg {
    float sa, sb;           // entry / exit in the local frame
    float dena, denb;       // d.a of the active plane or face at each end
    int ka, kb;             // active constraint: plane slot >= 0, or K_*
    float3 q;               // closest-approach offset from p_i
    float dnd;              // d . n (selects the texture end)
    int refined;            // ends recomputed in FP64
    int nplanes;            // radical planes evaluated (the warp may stop early)
};

enum : int { K_SPHERE = -1, K_CAMERA = -2, K_FACE = -3 };

__device__ __forceinline__ float3 f3(float x, float y, float z) { return make_float3(x, y, z); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }
// 1/x to about 1 ulp; +-0 gives +-inf (subnormals count as zero)
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
// sqrt(x) to a few ulp for x >= 0 (one hardware approximation, no
// correctly-rounded fix-up sequence)
__device__ __forceinline__ float sqrt_approx(float x) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
// 2^x by the hardware approximation (ex2.approx, about 2 ulp); the soft-
// Voronoi weights exp(-kappa r) = 2^(r * KAPPA_LOG2E) take one multiply.
__device__ __forceinline__ float exp2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
constexpr float KAPPA_LOG2E = (float)(-(double)KAPPA * 1.4426950408889634);

__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
    return f3(fmaf(a.y, b.z, -a.z * b.y), fmaf(a.z, b.x, -a.x * b.z), fmaf(a.x, b.y, -a.y * b.x));
}

// One component of (m x d) = m1 d2 - m2 d1 for float pairs m = mh + ml,
// d = dh + dl.  p2 = mh2 dh1 rounded, e2 its exact rounding error (FMA);
// fma(mh1, dh2, -p2) rounds the exact mh1 dh2 - p2 once, an error of half
// an ulp of the (small) result; then the first-order terms of the low parts.
__device__ __forceinline__ float cross_c(float mh1, float ml1, float dh2, float dl2, float mh2, float ml2, float dh1,
                                         float dl1) {
    const float p2 = mh2 * dh1;
    const float e2 = fmaf(mh2, dh1, -p2);
    const float hi = fmaf(mh1, dh2, -p2);
    float lo = fmaf(mh1, dl2, -e2);
    lo = fmaf(ml1, dh2, lo);
    lo = fmaf(-mh2, dl1, lo);
    lo = fmaf(-ml2, dh1, lo);
    return hi + lo;
}

struct Ray {
    float3 dh, dl;          // unit direction as a float pair
};

// Does pixel (u, v) have a ray?  (A fisheye pixel beyond theta = pi has none.)
__device__ __forceinline__ bool pixel_has_ray(const ViewDev &V, int u, int v) {
    if (V.model != PF_FISHEYE) return true;
    const double xc = ((double)u + 0.5 - V.cx) * V.ifx;
    const double yc = ((double)v + 0.5 - V.cy) * V.ify;
    return sqrt(xc * xc + yc * yc) <= CUDART_PI;
}

// Equidistant fisheye: the offset (xc, yc) is the angle from the axis
// (clamped at pi; pixels beyond have no ray and are never composited).  Out
// of line: the pinhole path never calls it.
static __device__ __noinline__ double3 fisheye_dir(double xc, double yc) {
    const double th = fmin(sqrt(xc * xc + yc * yc), CUDART_PI);
    double sn, cs;
    sincos(th, &sn, &cs);
    const double f = th > 0.0 ? sn / th : 1.0;
    return make_double3(xc * f, yc * f, cs);
}

__device__ __forceinline__ Ray pixel_ray(const ViewDev &V, int u, int v) {
    double xc = ((double)u + 0.5 - V.cx) * V.ifx;
    double yc = ((double)v + 0.5 - V.cy) * V.ify;
    double zc = 1.0;
    if (V.model == PF_FISHEYE) {
        const double3 c = fisheye_dir(xc, yc);
        xc = c.x;
        yc = c.y;
        zc = c.z;
    }
    const double *M = V.rot;
    double dx = M[0] * xc + M[3] * yc + M[6] * zc;
    double dy = M[1] * xc + M[4] * yc + M[7] * zc;
    double dz = M[2] * xc + M[5] * yc + M[8] * zc;
    const double n2 = dx * dx + dy * dy + dz * dz;
    double r = (double)rsqrtf((float)n2);
    r = r * (1.5 - 0.5 * n2 * r * r);
    r = r * (1.5 - 0.5 * n2 * r * r);
    dx *= r;
    dy *= r;
    dz *= r;
    Ray R;
    R.dh = f3((float)dx, (float)dy, (float)dz);
    R.dl = f3((float)(dx - (double)R.dh.x), (float)(dy - (double)R.dh.y), (float)(dz - (double)R.dh.z));
    return R;
}

// FP64 recomputation of segment ends, from float pairs already at hand (the
// view record's m = hi + lo, the ray's d = hi + lo, a plane's hi + lo parts
// written by prepare): no global gathers, no FP64 divide or sqrt sequence.
// q = m - (m.d) d is the closest-approach offset in FP64.
__device__ __forceinline__ double rcp64(double x) {
    double r = (double)(1.0f / (float)x);
    r = r * (2.0 - x * r);
    r = r * (2.0 - x * r);
    return r;
}

// A plane (or the face) end: s = (g - q.a) / (d.a); `fallback` if d.a == 0.
// `den` receives d.a in FP64, rounded once (the adjoint divides by it).
static __device__ __noinline__ float refine_plane64(const float *vr, float4 hi, float4 lo, Ray ray, float fallback,
                                             float &den_out) {
    const double dx = (double)ray.dh.x + (double)ray.dl.x, dy = (double)ray.dh.y + (double)ray.dl.y,
                 dz = (double)ray.dh.z + (double)ray.dl.z;
    const double mx = (double)vr[0] + (double)vr[4], my = (double)vr[1] + (double)vr[5],
                 mz = (double)vr[2] + (double)vr[6];
    const double b = mx * dx + my * dy + mz * dz;
    const double qx = mx - b * dx, qy = my - b * dy, qz = mz - b * dz;
    const double ax = (double)hi.x + (double)lo.x, ay = (double)hi.y + (double)lo.y, az = (double)hi.z + (double)lo.z;
    const double g = (double)hi.w + (double)lo.w;
    const double num = g - (qx * ax + qy * ay + qz * az);
    const double den = dx * ax + dy * ay + dz * az;
    den_out = (float)den;
    if (den == 0.0) return fallback;
    return (float)(num * rcp64(den));
}

// The sphere's D = R^2 - |q|^2.
static __device__ __noinline__ float refine_D64(const float *vr, float R, Ray ray) {
    const double dx = (double)ray.dh.x + (double)ray.dl.x, dy = (double)ray.dh.y + (double)ray.dl.y,
                 dz = (double)ray.dh.z + (double)ray.dl.z;
    const double mx = (double)vr[0] + (double)vr[4], my = (double)vr[1] + (double)vr[5],
                 mz = (double)vr[2] + (double)vr[6];
    const double b = mx * dx + my * dy + mz * dz;
    const double qx = mx - b * dx, qy = my - b * dy, qz = mz - b * dz;
    return (float)((double)R * (double)R - (qx * qx + qy * qy + qz * qz));
}

// Sign of d.n in FP64 (the side of the face the texture point is taken on).
static __device__ __noinline__ float face_side64(const float *cr, Ray ray) {
    const double dn = ((double)ray.dh.x + (double)ray.dl.x) * ((double)cr[CR_N] + (double)cr[CR_NLO]) +
                      ((double)ray.dh.y + (double)ray.dl.y) * ((double)cr[CR_N + 1] + (double)cr[CR_NLO + 1]) +
                      ((double)ray.dh.z + (double)ray.dl.z) * ((double)cr[CR_N + 2] + (double)cr[CR_NLO + 2]);
    return dn > 0.0 ? 1.0f : (dn < 0.0 ? -1.0f : 0.0f);
}

// The ray's segment in one cell.  cr: cell record, vr: view record,
// pl: the cell's planes, nb: their neighbour ids (global, for refinement).
// GRAD (the backward) also recomputes D in FP64 whenever D < GRAD_D R^2:
// the sphere end's derivatives scale with 1/sqrt(D), so near-tangent
// gradients need D to more digits than the forward's value does.  For the
// same reason it recomputes a plane or face end, and takes its d.a from
// FP64, whenever |d.a| < GRAD_DEN (the end's derivatives scale with 1/(d.a)).
constexpr float GRAD_D = 1e-3f;
constexpr float GRAD_DEN = 2e-3f;

// The ray against the cell's bounding sphere: the cheap candidate test
// (cand), then the exact chord in the closest-approach frame.
struct Chord {
    float3 q;      // closest-approach offset from p_i (x - p_i = q + s d)
    float sq;      // half chord: the sphere spans s in [-sq, sq]
    float b;       // s of the camera (the segment starts at s >= b)
    int refined;   // D recomputed in FP64
};

template <bool GRAD>
__device__ __forceinline__ bool sphere_chord(const float *__restrict__ cr, const float *__restrict__ vr,
                                             const Ray &ray, Chord &ch, bool &cand) {
    const float4 V0 = reinterpret_cast<const float4 *>(vr)[0];
    const float3 mh = f3(V0.x, V0.y, V0.z);
    const float3 v0 = cross3(mh, ray.dh);
    cand = dot3(v0, v0) <= V0.w;
    if (!cand) return false;
    const float4 V1 = reinterpret_cast<const float4 *>(vr)[1];
    const float3 ml = f3(V1.x, V1.y, V1.z);
    const float3 dh = ray.dh, dl = ray.dl;
    const float3 v = f3(cross_c(mh.y, ml.y, dh.z, dl.z, mh.z, ml.z, dh.y, dl.y),
                        cross_c(mh.z, ml.z, dh.x, dl.x, mh.x, ml.x, dh.z, dl.z),
                        cross_c(mh.x, ml.x, dh.y, dl.y, mh.y, ml.y, dh.x, dl.x));
    const float R = cr[CR_R];
    float D = fmaf(R, R, -dot3(v, v));
    ch.refined = 0;
    // near-tangent sphere: decide and measure D in FP64
    if (fabsf(D) < (GRAD ? fmaxf(V1.w, GRAD_D * R * R) : V1.w)) {
        D = refine_D64(vr, R, ray);
        ch.refined = 1;
    }
    if (!(D > 0.0f)) return false;
    ch.sq = sqrt_approx(D);
    ch.q = cross3(dh, v);
    ch.b = dot3(mh, dh);
    return true;
}

// Face coordinates of a point y (relative to the site) and the soft-Voronoi
// weights of the NS texture sites there.
template <int NS>
struct TexT {
    float3 ys;
    float u1, u2;
    float ax[2], ay[2];     // u - site offsets of the four fixed sites: ax[0] = u1 + 1/3, ax[1] = u1 - 1/3
    float r[NS], W[NS];
};
using Tex = TexT<4>;

// The fixed detail sites, in units of R: four at (+-1/3, +-1/3), site-major
// (-,-), (+,-), (-,+), (+,+); eight on the 3 x 3 grid of step 1/3 without its
// centre, row by row.
template <int NS>
__device__ __forceinline__ float site_x(int k) {
    if (NS == 4) return (k & 1) ? SITE : -SITE;
    return k < 3 ? (float)(k - 1) * SITE : (k == 3 ? -SITE : (k == 4 ? SITE : (float)(k - 6) * SITE));
}
template <int NS>
__device__ __forceinline__ float site_y(int k) {
    if (NS == 4) return (k >> 1) ? SITE : -SITE;
    return k < 3 ? -SITE : (k < 5 ? 0.0f : SITE);
}

// Displacement of the face for this ray (Eq. svdisp, one-step plane shift):
// the ray crosses the base face at s = num / fden from its closest approach,
// at y = q + s d from the site; there u = (e1.y, e2.y) / R, and the face
// moves by delta = sum_k W_k disp_k with the texture's soft-Voronoi weights.
// A ray parallel to the face sees no displacement.  s is kept within 1e6 R:
// the weights of a farther crossing are already the limit of the ray's
// direction.  With `tx` the crossing's coordinates and weights are returned
// (for the adjoint; its ax / ay hold u minus the fixed sites only).  `st`:
// the cell's learned site positions [4][2] in units of R, or null.
__device__ __forceinline__ float face_delta(const float *__restrict__ cr, float3 q, float3 dh, float num,
                                            float fden, float4 dk, Tex *tx = nullptr,
                                            const float *__restrict__ st = nullptr) {
    if (!(fabsf(fden) > 0.0f)) {
        if (tx) *tx = Tex{};
        return 0.0f;
    }
    const float big = 1e6f * cr[CR_R];
    const float s = fminf(fmaxf(num / fden, -big), big);
    const float3 y = f3(fmaf(s, dh.x, q.x), fmaf(s, dh.y, q.y), fmaf(s, dh.z, q.z));
    const float u0 = dot3(f3(cr[CR_E1], cr[CR_E1 + 1], cr[CR_E1 + 2]), y);
    const float u1 = dot3(f3(cr[CR_E2], cr[CR_E2 + 1], cr[CR_E2 + 2]), y);
    // the texture's sites: learned positions `st`, else (-,-), (+,-), (-,+),
    // (+,+) at a third of R
    const float a0 = u0 + SITE, a1 = u0 - SITE, b0 = u1 + SITE, b1 = u1 - SITE;
    float r0, r1, r2, r3;
    if (st) {
        r0 = sqrtf((u0 - st[0]) * (u0 - st[0]) + (u1 - st[1]) * (u1 - st[1]));
        r1 = sqrtf((u0 - st[2]) * (u0 - st[2]) + (u1 - st[3]) * (u1 - st[3]));
        r2 = sqrtf((u0 - st[4]) * (u0 - st[4]) + (u1 - st[5]) * (u1 - st[5]));
        r3 = sqrtf((u0 - st[6]) * (u0 - st[6]) + (u1 - st[7]) * (u1 - st[7]));
    } else {
        r0 = sqrtf(a0 * a0 + b0 * b0);
        r1 = sqrtf(a1 * a1 + b0 * b0);
        r2 = sqrtf(a0 * a0 + b1 * b1);
        r3 = sqrtf(a1 * a1 + b1 * b1);
    }
    const float l0 = -KAPPA * r0, l1 = -KAPPA * r1, l2 = -KAPPA * r2, l3 = -KAPPA * r3;
    const float mx = fmaxf(fmaxf(l0, l1), fmaxf(l2, l3));
    const float w0 = __expf(l0 - mx), w1 = __expf(l1 - mx), w2 = __expf(l2 - mx), w3 = __expf(l3 - mx);
    const float z = w0 + w1 + w2 + w3;
    if (tx) {
        const float iz = 1.0f / z;
        tx->ys = y;
        tx->u1 = u0;
        tx->u2 = u1;
        tx->ax[0] = a0;
        tx->ax[1] = a1;
        tx->ay[0] = b0;
        tx->ay[1] = b1;
        tx->r[0] = r0;
        tx->r[1] = r1;
        tx->r[2] = r2;
        tx->r[3] = r3;
        tx->W[0] = w0 * iz;
        tx->W[1] = w1 * iz;
        tx->W[2] = w2 * iz;
        tx->W[3] = w3 * iz;
    }
    return (w0 * dk.x + w1 * dk.y + w2 * dk.z + w3 * dk.w) / z;
}

// face_delta over eight sites (the fixed grid or learned positions st
// [8][2]): the same one-step plane shift, the weights taken relative to the
// nearest site; dk: the eight site displacements.
__device__ __forceinline__ float face_delta8(const float *__restrict__ cr, float3 q, float3 dh, float num, float fden,
                                             const float *__restrict__ dk, TexT<8> *tx = nullptr,
                                             const float *__restrict__ st = nullptr) {
    if (!(fabsf(fden) > 0.0f)) {
        if (tx) *tx = TexT<8>{};
        return 0.0f;
    }
    const float big = 1e6f * cr[CR_R];
    const float s = fminf(fmaxf(num / fden, -big), big);
    const float3 y = f3(fmaf(s, dh.x, q.x), fmaf(s, dh.y, q.y), fmaf(s, dh.z, q.z));
    const float u0 = dot3(f3(cr[CR_E1], cr[CR_E1 + 1], cr[CR_E1 + 2]), y);
    const float u1 = dot3(f3(cr[CR_E2], cr[CR_E2 + 1], cr[CR_E2 + 2]), y);
    float r[8], rmin = CUDART_INF_F;
#pragma unroll
    for (int k = 0; k < 8; k++) {
        const float ax = u0 - (st ? st[2 * k] : site_x<8>(k)), ay = u1 - (st ? st[2 * k + 1] : site_y<8>(k));
        r[k] = sqrtf(ax * ax + ay * ay);
        rmin = fminf(rmin, r[k]);
    }
    float w[8], z = 0.f, dl = 0.f;
#pragma unroll
    for (int k = 0; k < 8; k++) {
        w[k] = __expf(-KAPPA * (r[k] - rmin));
        z += w[k];
        dl = fmaf(w[k], dk[k], dl);
    }
    if (tx) {
        const float iz = 1.0f / z;
        tx->ys = y;
        tx->u1 = u0;
        tx->u2 = u1;
        tx->ax[0] = tx->ax[1] = tx->ay[0] = tx->ay[1] = 0.f;
#pragma unroll
        for (int k = 0; k < 8; k++) {
            tx->r[k] = r[k];
            tx->W[k] = w[k] * iz;
        }
    }
    return dl / z;
}

// Clip the chord with the cell's radical planes pl[0..np), the dipole face,
// then refine near-parallel ends.  False if the segment is empty.  NEED sets
// sg.nplanes to the planes this ray needs on its own (up to the one that
// empties its segment) instead of the planes the warp evaluated.  EXT:
// an extended face model; with has_disp the face moves by the ray's
// displacement (face_delta, from dk and the sites st).
template <bool GRAD, bool NEED = false, bool EXT = false, int NS = 4>
__device__ __forceinline__ bool clip_chord(const float *__restrict__ cr, const float *__restrict__ vr,
                                           const float4 *__restrict__ pl, int np,
                                           const float4 *__restrict__ lo_glob, const Ray &ray, const Chord &ch,
                                           Seg &sg, unsigned lanes = 0u, float4 dk = float4{0.f, 0.f, 0.f, 0.f},
                                           const float *__restrict__ st = nullptr, bool has_disp = false,
                                           const float *__restrict__ dk8 = nullptr) {
    const float3 dh = ray.dh, q = ch.q;
    const float R = cr[CR_R];
    const float sig = cr[CR_SIG];
    float sa = -ch.sq, sb = ch.sq;
    int ka = K_SPHERE, kb = K_SPHERE;
    if (ch.b > sa) {
        sa = ch.b;
        ka = K_CAMERA;
    }
    sg.refined = ch.refined;
    // d.a of the constraint at each end, carried along (+inf for sphere and camera ends)
    float dena = CUDART_INF_F, denb = CUDART_INF_F;
    // the dipole's dense half n.y <= offset first (it removes about half of
    // the ball): a bound from below when d.n < 0 (sign bit, so -0 counts as
    // below), from above otherwise; d.n = +-0 gives +-inf or NaN, which moves
    // no end unless the ray runs outside the half (num < 0): then it empties
    // the segment
    float fden;
    float foff = cr[CR_OFF];
    {
        const float3 n = f3(cr[CR_N], cr[CR_N + 1], cr[CR_N + 2]);
        float num = foff - dot3(q, n);
        fden = dot3(dh, n);
        if (EXT && has_disp) {
            const float dl = NS == 8 ? face_delta8(cr, q, dh, num, fden, dk8, nullptr, st)
                                     : face_delta(cr, q, dh, num, fden, dk, nullptr, st);
            foff += dl;
            num += dl;
        }
        const float t = num * rcp_approx(fden);
        const bool ent = __float_as_int(fden) < 0;
        const bool ua = ent && t > sa;
        const bool ub = !ent && t < sb;
        sa = ua ? t : sa;
        ka = ua ? K_FACE : ka;
        dena = ua ? fden : dena;
        sb = ub ? t : sb;
        kb = ub ? K_FACE : kb;
        denb = ub ? fden : denb;
        sg.dnd = fden;
        if (fabsf(fden) < 0x1p-20f) sg.dnd = face_side64(cr, ray);
    }
    // Radical planes the same way, branch free, nearest first (prepare sorts
    // them by distance).  With `lanes` (the lanes that run this call) the
    // warp stops once every one of them has an empty segment.
    int need = (NEED && !(sb > sa)) ? 0 : np;
    int k = (lanes && !__any_sync(lanes, sb > sa)) ? np : 0;  // the face alone may empty them all
    for (; k < np; k += 4) {
#pragma unroll
        for (int u = 0; u < 4; u++) {
            if (u >= 1 && k + u >= np) break;
            const float4 P = pl[k + u];
            const float3 a = f3(P.x, P.y, P.z);
            const float num = P.w - dot3(q, a);
            const float den = dot3(dh, a);
            const float t = num * rcp_approx(den);
            const bool ent = __float_as_int(den) < 0;
            const bool ua = ent && t > sa;
            const bool ub = !ent && t < sb;
            sa = ua ? t : sa;
            ka = ua ? k + u : ka;
            dena = ua ? den : dena;
            sb = ub ? t : sb;
            kb = ub ? k + u : kb;
            denb = ub ? den : denb;
            if (NEED && need == np && !(sb > sa)) need = k + u + 1;
        }
        if (lanes && !__any_sync(lanes, sb > sa)) {
            k += 4;
            break;
        }
    }
    sg.nplanes = NEED ? need : min(k, np);
    if (!(sb > sa)) return false;
    // near-parallel plane or face at an end: recompute that end in FP64
    const float lim = PLANE_ERR * sig * (1.0f / REFINE_EPS);
    // the adjoint divides by d.a: the backward also recomputes every end with
    // |d.a| < GRAD_DEN, so that 1/(d.a) has a relative error below ~1e-4
    const bool ra = fabsf(dena) < (GRAD ? fmaxf(lim * (R + fabsf(sa)), GRAD_DEN) : lim * (R + fabsf(sa)));
    const bool rb = fabsf(denb) < (GRAD ? fmaxf(lim * (R + fabsf(sb)), GRAD_DEN) : lim * (R + fabsf(sb)));
    if (ra || rb) {
        // and takes d.a from FP64 at the ends it recomputes
        float d64;
        if (ra) {
            sa = ka >= 0 ? refine_plane64(vr, pl[ka], lo_glob[ka], ray, sa, d64)
                         : refine_plane64(vr, make_float4(cr[CR_N], cr[CR_N + 1], cr[CR_N + 2], foff),
                                          make_float4(cr[CR_NLO], cr[CR_NLO + 1], cr[CR_NLO + 2], 0.f), ray, sa, d64);
            if (GRAD) dena = d64;
            sg.refined++;
        }
        if (rb) {
            sb = kb >= 0 ? refine_plane64(vr, pl[kb], lo_glob[kb], ray, sb, d64)
                         : refine_plane64(vr, make_float4(cr[CR_N], cr[CR_N + 1], cr[CR_N + 2], foff),
                                          make_float4(cr[CR_NLO], cr[CR_NLO + 1], cr[CR_NLO + 2], 0.f), ray, sb, d64);
            if (GRAD) denb = d64;
            sg.refined++;
        }
    }
    if (!(sb > sa)) return false;
    sg.sa = sa;
    sg.sb = sb;
    sg.ka = ka;
    sg.kb = kb;
    sg.dena = dena;
    sg.denb = denb;
    sg.q = q;
    return true;
}

// The segment of a recorded hit from its active constraints (ka, kb): the
// same float expressions as clip_chord for those two constraints and the
// face, then the same refinement, so the ends equal the forward's.
template <bool GRAD, bool EXT = false, int NS = 4>
__device__ __forceinline__ bool segment_from_kinds(const float *__restrict__ cr, const float *__restrict__ vr,
                                                   const float4 *__restrict__ pl,
                                                   const float4 *__restrict__ lo_glob, const Ray &ray,
                                                   const Chord &ch, int ka, int kb, Seg &sg,
                                                   float4 dk = float4{0.f, 0.f, 0.f, 0.f},
                                                   const float *__restrict__ st = nullptr, bool has_disp = false,
                                                   const float *__restrict__ dk8 = nullptr) {
    const float3 dh = ray.dh, q = ch.q;
    const float R = cr[CR_R];
    const float sig = cr[CR_SIG];
    sg.refined = ch.refined;
    const float3 n = f3(cr[CR_N], cr[CR_N + 1], cr[CR_N + 2]);
    float foff = cr[CR_OFF];
    float fnum = foff - dot3(q, n);
    const float fden = dot3(dh, n);
    if (EXT && has_disp) {  // the forward's displaced face, the same expressions
        const float dl = NS == 8 ? face_delta8(cr, q, dh, fnum, fden, dk8, nullptr, st)
                                 : face_delta(cr, q, dh, fnum, fden, dk, nullptr, st);
        foff += dl;
        fnum += dl;
    }
    const float tf = fnum * rcp_approx(fden);
    sg.dnd = fden;
    if (fabsf(fden) < 0x1p-20f) sg.dnd = face_side64(cr, ray);
    const float4 Pa = pl[max(ka, 0)], Pb = pl[max(kb, 0)];
    const float dpa = dot3(dh, f3(Pa.x, Pa.y, Pa.z)), dpb = dot3(dh, f3(Pb.x, Pb.y, Pb.z));
    const float tpa = (Pa.w - dot3(q, f3(Pa.x, Pa.y, Pa.z))) * rcp_approx(dpa);
    const float tpb = (Pb.w - dot3(q, f3(Pb.x, Pb.y, Pb.z))) * rcp_approx(dpb);
    float sa = ka >= 0 ? tpa : (ka == K_FACE ? tf : (ka == K_CAMERA ? ch.b : -ch.sq));
    float sb = kb >= 0 ? tpb : (kb == K_FACE ? tf : ch.sq);
    float dena = ka >= 0 ? dpa : (ka == K_FACE ? fden : CUDART_INF_F);
    float denb = kb >= 0 ? dpb : (kb == K_FACE ? fden : CUDART_INF_F);
    if (!(sb > sa)) return false;
    // near-parallel plane or face at an end: recompute that end in FP64
    const float lim = PLANE_ERR * sig * (1.0f / REFINE_EPS);
    // the adjoint divides by d.a: the backward also recomputes every end with
    // |d.a| < GRAD_DEN, so that 1/(d.a) has a relative error below ~1e-4
    const bool ra = fabsf(dena) < (GRAD ? fmaxf(lim * (R + fabsf(sa)), GRAD_DEN) : lim * (R + fabsf(sa)));
    const bool rb = fabsf(denb) < (GRAD ? fmaxf(lim * (R + fabsf(sb)), GRAD_DEN) : lim * (R + fabsf(sb)));
    if (ra || rb) {
        // and takes d.a from FP64 at the ends it recomputes
        float d64;
        if (ra) {
            sa = ka >= 0 ? refine_plane64(vr, pl[ka], lo_glob[ka], ray, sa, d64)
                         : refine_plane64(vr, make_float4(cr[CR_N], cr[CR_N + 1], cr[CR_N + 2], foff),
                                          make_float4(cr[CR_NLO], cr[CR_NLO + 1], cr[CR_NLO + 2], 0.f), ray, sa, d64);
            if (GRAD) dena = d64;
            sg.refined++;
        }
        if (rb) {
            sb = kb >= 0 ? refine_plane64(vr, pl[kb], lo_glob[kb], ray, sb, d64)
                         : refine_plane64(vr, make_float4(cr[CR_N], cr[CR_N + 1], cr[CR_N + 2], foff),
                                          make_float4(cr[CR_NLO], cr[CR_NLO + 1], cr[CR_NLO + 2], 0.f), ray, sb, d64);
            if (GRAD) denb = d64;
            sg.refined++;
        }
    }
    if (!(sb > sa)) return false;
    sg.sa = sa;
    sg.sb = sb;
    sg.ka = ka;
    sg.kb = kb;
    sg.dena = dena;
    sg.denb = denb;
    sg.q = q;
    return true;
}

// Soft-Voronoi face colour (Eq. svrad): weights of the four sites at the
// texture point y = q + s d (the dense segment's end on the face side).
// Colour of site k seen along the ray, a spherical-Voronoi function (Sec.
// 3.4): with wo = -d and the site's eight (axis, rgb), the colours weighed by
// softmax(SV_LAMBDA a.wo / |a|).  q: the cell's [4][8][6] floats in global
// memory (the lanes of a warp that hit the cell read the same lines).
__device__ __forceinline__ float3 sv_colour(const float *__restrict__ q, int k, float3 d) {
    const float *p = q + 48 * k;
    float lg[8], mx = -CUDART_INF_F;
#pragma unroll
    for (int j = 0; j < 8; j++) {
        const float ax = __ldg(p + 6 * j), ay = __ldg(p + 6 * j + 1), az = __ldg(p + 6 * j + 2);
        lg[j] = -SV_LAMBDA * (ax * d.x + ay * d.y + az * d.z) * rsqrtf(fmaf(ax, ax, fmaf(ay, ay, az * az)));
        mx = fmaxf(mx, lg[j]);
    }
    float z = 0.f;
    float3 c = f3(0.f, 0.f, 0.f);
#pragma unroll
    for (int j = 0; j < 8; j++) {
        const float w = __expf(lg[j] - mx);
        z += w;
        c.x = fmaf(w, __ldg(p + 6 * j + 3), c.x);
        c.y = fmaf(w, __ldg(p + 6 * j + 4), c.y);
        c.z = fmaf(w, __ldg(p + 6 * j + 5), c.z);
    }
    const float iz = 1.0f / z;
    return f3(c.x * iz, c.y * iz, c.z * iz);
}

// Colour at the texture point; `st`: the cell's learned site positions, or
// null for the fixed ones (then tx.ax / tx.ay hold u minus the sites); `sv`:
// the cell's view-dependent site colours, or null for the constant ones.
template <int NS>
__device__ __forceinline__ float3 face_colour(const float *__restrict__ cr, const Seg &sg, const Ray &ray, TexT<NS> &tx,
                                              const float *__restrict__ st = nullptr,
                                              const float *__restrict__ sv = nullptr,
                                              const float *__restrict__ tex = nullptr) {
    const float ss = sg.dnd > 0.0f ? sg.sb : sg.sa;
    tx.ys = f3(fmaf(ss, ray.dh.x, sg.q.x), fmaf(ss, ray.dh.y, sg.q.y), fmaf(ss, ray.dh.z, sg.q.z));
    tx.u1 = dot3(f3(cr[CR_E1], cr[CR_E1 + 1], cr[CR_E1 + 2]), tx.ys);
    tx.u2 = dot3(f3(cr[CR_E2], cr[CR_E2 + 1], cr[CR_E2 + 2]), tx.ys);
    tx.ax[0] = tx.u1 + SITE;
    tx.ax[1] = tx.u1 - SITE;
    tx.ay[0] = tx.u2 + SITE;
    tx.ay[1] = tx.u2 - SITE;
    float Z = 0.f;
    if (st || NS != 4) {  // learned sites may lie far off: weights relative to the nearest
        float rmin = CUDART_INF_F;
#pragma unroll
        for (int k = 0; k < NS; k++) {
            const float ax = tx.u1 - (st ? st[2 * k] : site_x<NS>(k)), ay = tx.u2 - (st ? st[2 * k + 1] : site_y<NS>(k));
            tx.r[k] = sqrt_approx(fmaf(ax, ax, ay * ay));
            rmin = fminf(rmin, tx.r[k]);
        }
#pragma unroll
        for (int k = 0; k < NS; k++) {
            tx.W[k] = exp2_approx((tx.r[k] - rmin) * KAPPA_LOG2E);
            Z += tx.W[k];
        }
    } else {
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const float ax = tx.ax[k & 1], ay = tx.ay[k >> 1];
            tx.r[k] = sqrt_approx(fmaf(ax, ax, ay * ay));
            tx.W[k] = exp2_approx(tx.r[k] * KAPPA_LOG2E);
            Z += tx.W[k];
        }
    }
    const float iz = __fdividef(1.0f, Z);
    // the weighted site colours summed unnormalised, then scaled once
    float3 c = f3(0.f, 0.f, 0.f);
    const float *tc = tex ? tex : cr + CR_TEX;  // eight sites: tex staged beside the record
#pragma unroll
    for (int k = 0; k < NS; k++) {
        const float3 ck = sv ? sv_colour(sv, k, ray.dh) : f3(tc[3 * k], tc[3 * k + 1], tc[3 * k + 2]);
        c.x = fmaf(tx.W[k], ck.x, c.x);
        c.y = fmaf(tx.W[k], ck.y, c.y);
        c.z = fmaf(tx.W[k], ck.z, c.z);
        tx.W[k] *= iz;  // the normalised weights, for the adjoint
    }
    return f3(fmaf(c.x, iz, cr[CR_RGB]), fmaf(c.y, iz, cr[CR_RGB + 1]), fmaf(c.z, iz, cr[CR_RGB + 2]));
}

// ------------------------------------------------------------ batch staging
// Tile lists are staged in batches of 32 cells, double buffered: while the
// warps work on batch k, the copies of batch k+1 are in flight (cp.async,
// 16-byte granules: the 128-byte cell record, the 32-byte view record and
// the cell's planes, plus the planes' neighbour ids for the backward).
struct Stage {
    char *base;        // dynamic shared memory
    int K;
    bool with_nb;
    int xw;            // float4s per cell in the extended face model region (3, or 12 for eight sites)
    // per buffer: cell records [BATCH][CELLREC_F], view records [BATCH][VIEWREC_F],
    // planes [BATCH * K], plane neighbours [BATCH * K]; then ids [2][BATCH], poff [2][BATCH + 1]
    __device__ __forceinline__ size_t kk() const { return K > 0 ? (size_t)K : 1; }
    __device__ __forceinline__ size_t buf_bytes() const {
        return (size_t)BATCH * (CELLREC_F + VIEWREC_F) * 4 + BATCH * kk() * (with_nb ? 24 : 16);
    }
    __device__ __forceinline__ float *cr(int b) const { return reinterpret_cast<float *>(base + b * buf_bytes()); }
    __device__ __forceinline__ float *vr(int b) const { return cr(b) + BATCH * CELLREC_F; }
    __device__ __forceinline__ float4 *pl(int b) const { return reinterpret_cast<float4 *>(vr(b) + BATCH * VIEWREC_F); }
    __device__ __forceinline__ int2 *nb(int b) const { return reinterpret_cast<int2 *>(pl(b) + BATCH * kk()); }
    __device__ __forceinline__ int *ids(int b) const {
        return reinterpret_cast<int *>(base + 2 * buf_bytes()) + b * BATCH;
    }
    __device__ __forceinline__ int *poff(int b) const {
        return reinterpret_cast<int *>(base + 2 * buf_bytes()) + 2 * BATCH + b * (BATCH + 1);
    }
    // extended face model [2][BATCH][xw] (16-byte aligned).  Four sites: the
    // displacement, then the four learned site positions (x, y) (scenes with
    // either only).  Eight sites: the texture (24 floats), the displacement
    // (8), the learned positions (16).
    __device__ __forceinline__ float4 *xtr(int b) const {
        return reinterpret_cast<float4 *>(base + ((2 * buf_bytes() + (4 * BATCH + 2) * 4 + 15) & ~(size_t)15)) +
               b * BATCH * xw;
    }
};

__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(src));
}
__device__ __forceinline__ void cp_async8(void *dst, const void *src) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(src));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_one() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// Start the copies of list entries [0, nb) into buffer `buf`.  Every warp
// reads the 32 ids and plane counts itself (no barrier before the copies);
// warp 0 also publishes them for the consumers.
__device__ __forceinline__ void issue_batch(const Stage &sg, int buf, const uint32_t *__restrict__ list, int nb,
                                            const WS &w, int64_t vbase, int K, bool with_nb,
                                            const float *__restrict__ disp = nullptr,
                                            const float *__restrict__ sites = nullptr,
                                            const float *__restrict__ tex8 = nullptr) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int id = 0, np = 0;
    if (lane < nb) {
        id = (int)list[lane];
        np = w.cellnp[id];
    }
    int incl = np;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (warp == 0) {
        sg.ids(buf)[lane] = id;
        sg.poff(buf)[lane + 1] = incl;
        if (lane == 0) sg.poff(buf)[0] = 0;
    }
    // records: nb x (8 + 2 (+ 3, or 12 with eight sites, extended)) chunks
    // over all threads (uniform trip count: the shuffles need every lane)
    const int parts = tex8 ? 22 : ((disp || sites) ? 13 : 10);
    const int nrec = nb * parts;
    for (int q0 = 0; q0 < nrec; q0 += TILE_PIX) {
        const int q = q0 + tid;
        const int j = (q < nrec ? q : 0) / parts, part = q - j * parts;
        const int c = __shfl_sync(0xffffffffu, id, j);
        if (q < nrec) {
            if (part < 8)
                cp_async16(sg.cr(buf) + j * CELLREC_F + part * 4, w.cellrec + (int64_t)c * CELLREC_F + part * 4);
            else if (part < 10)
                cp_async16(sg.vr(buf) + j * VIEWREC_F + (part - 8) * 4,
                           w.viewrec + (vbase + c) * VIEWREC_F + (part - 8) * 4);
            else if (tex8) {  // eight sites: texture 6, displacement 2, positions 4 granules
                const int e = part - 10;
                if (e < 6)
                    cp_async16(sg.xtr(buf) + 12 * j + e, tex8 + (int64_t)c * 24 + e * 4);
                else if (e < 8 && disp)
                    cp_async16(sg.xtr(buf) + 12 * j + e, disp + (int64_t)c * 8 + (e - 6) * 4);
                else if (e >= 8 && sites)
                    cp_async16(sg.xtr(buf) + 12 * j + e, sites + (int64_t)c * 16 + (e - 8) * 4);
            } else if (part == 10 && disp)
                cp_async16(sg.xtr(buf) + 3 * j, disp + (int64_t)c * 4);
            else if (part > 10 && sites)
                cp_async16(sg.xtr(buf) + 3 * j + (part - 10), sites + (int64_t)c * 8 + (part - 11) * 4);
        }
    }
    // planes: warp w copies the planes of cells w, w + 8, ...
    for (int j = warp; j < nb; j += TILE_PIX / 32) {
        const int c = __shfl_sync(0xffffffffu, id, j);
        const int end = __shfl_sync(0xffffffffu, incl, j);
        const int cnt = __shfl_sync(0xffffffffu, np, j);
        const int o = end - cnt;
        for (int k = lane; k < cnt; k += 32) {
            cp_async16(sg.pl(buf) + o + k, w.planes + (int64_t)c * K + k);
            if (with_nb) cp_async8(sg.nb(buf) + o + k, w.plane_nb + (int64_t)c * K + k);
        }
    }
    cp_async_commit();
}

__device__ __forceinline__ int find_view(const ViewDev *views, int nv, int64_t tile) {
    int lo = 0, hi = nv - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (views[mid].tile_base <= tile) lo = mid; else hi = mid - 1;
    }
    return lo;
}

struct RenderArgs {
    WS w;
    int nv, n, K;
    unsigned long long cap;
    int64_t mask_batches;   // batch slots per warp in the hit-mask array
    float *contrib_sparse;  // [N] sum of T alpha per cell (pf_render_fwd_contrib), or null
    float *contrib_normal;  // [N] sum of T alpha max(nh.d, 0)^2 per cell, or null
    const float *disp;      // [N][4] face displacement at the texture sites, or null
    float *gdisp;           // [N][4] its gradient (the backward adds into it), or null
    const float *sites;     // [N][4][2] learned texture / detail site positions, or null
    float *gsites;          // [N][4][2] their gradient, or null
    const float *sv;        // [N][S][8][6] view-dependent site colours, or null
    float *gsv;             // [N][S][8][6] their gradient, or null
    const float *tex8;      // eight sites: the texture [N][24] (four: in the cell record), else null
    float *gtex8;           // eight sites: its gradient (the backward adds into it), else null
    const float *w_sparse;  // [N] upstream weights of the contributions' adjoint (pf_render_bwd_contrib), or null
    const float *w_normal;  // [N]
    float4 *segrec;         // [pixels][seg_cap] stored segments (pf_plan_store_segments), or null
    int seg_cap;
};

// Hit masks: one 32-bit word per (warp of the tile, batch, pixel of the
// warp).  Batch k of the tile whose list starts at instance s gets the
// unique slot floor(s / 32) + tile + k (a list of n entries has at most
// ceil(n / 32) batches, so consecutive tiles' slots never overlap).
__device__ __forceinline__ int64_t hitmask_slot(const RenderArgs &A, int64_t tile, unsigned long long s, int k,
                                                int warp) {
    return ((int64_t)warp * A.mask_batches + (int64_t)(s / BATCH) + tile + k) * 32;
}

__device__ __forceinline__ void tile_pixel(const ViewDev &V, int64_t lt, int &px, int &py, int &wx, int &wy) {
    const int tx = (int)(lt % V.tiles_x), ty = (int)(lt / V.tiles_x);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    wx = tx * TILE + (warp & 1) * 8;   // the warp's 8x4 block
    wy = ty * TILE + (warp >> 1) * 4;
    px = wx + (lane & 7);
    py = wy + (lane >> 3);
}

// The warp's view cone: centre ray through the middle of its 8x4 block and
// the tangent of the largest angle to any of its 32 pixel rays.
struct Cone {
    float3 dc;
    float tan_t;
};

__device__ __forceinline__ Cone warp_cone(const Ray &ray) {
    Cone c;
    // the ray of pixel (wx + 4, wy + 2), near the block's centre, is lane 20's
    // own (lanes run x fastest, 8 to a row); the cone is measured from it
    c.dc = f3(__shfl_sync(0xffffffffu, ray.dh.x, 20), __shfl_sync(0xffffffffu, ray.dh.y, 20),
              __shfl_sync(0xffffffffu, ray.dh.z, 20));
    const float3 d = ray.dh;
    const float3 x = cross3(d, c.dc);
    const float sn = sqrtf(dot3(x, x));
    const float cs = dot3(d, c.dc);
    float t = sn / fmaxf(cs, 1e-3f);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t = fmaxf(t, __shfl_xor_sync(0xffffffffu, t, o));
    c.tan_t = t * 1.001f + 1e-5f;
    return c;
}

// Ballot of the batch's cells whose bounding sphere can meet the warp's
// cone: lane j tests cell j (conservative: a sphere near or behind the
// camera plane always counts).
__device__ __forceinline__ unsigned warp_mask(const Stage &sg, int buf, int nb, const Cone &cone) {
    const int lane = threadIdx.x & 31;
    bool ov = false;
    if (lane < nb) {
        const float *vr = sg.vr(buf) + lane * VIEWREC_F;
        const float R = sg.cr(buf)[lane * CELLREC_F + CR_R];
        const float3 m = f3(vr[0], vr[1], vr[2]);      // o - p
        const float tc = -dot3(m, cone.dc);              // site depth along the centre ray
        const float3 u = cross3(m, cone.dc);
        const float mm = sqrtf(dot3(m, m));
        const float rho = sqrtf(dot3(u, u));
        const float lim = fmaf(fmaxf(tc, 0.0f), cone.tan_t, R * (1.0f + cone.tan_t * cone.tan_t)) + 1e-5f * (mm + R);
        ov = (tc <= R * 1.01f + 1e-5f * mm) || (rho <= lim);
        ov = ov && (tc + R >= -1e-5f * mm);
    }
    return __ballot_sync(0xffffffffu, ov);
}

__host__ __device__ inline size_t stage_bytes(int K, bool with_nb, bool ext = false, int xw = 3) {
    const size_t k = K > 0 ? (size_t)K : 1;
    const size_t buf = (size_t)BATCH * (CELLREC_F + VIEWREC_F) * 4 + BATCH * k * (with_nb ? 24 : 16);
    const size_t ids = 2 * buf + (2 * BATCH + 2 * (BATCH + 1)) * 4;
    return ext ? ((ids + 15) & ~(size_t)15) + 2 * BATCH * 16 * (size_t)xw : ids;
}

__device__ __forceinline__ Stage make_stage(float4 *smem, int K, bool with_nb, int xw = 3) {
    Stage sg;
    sg.base = reinterpret_cast<char *>(smem);
    sg.K = K;
    sg.with_nb = with_nb;
    sg.xw = xw;
    return sg;
}

// Enough CTAs to fill every SM at the kernel's occupancy, at most one per tile.
template <typename Kernel>
static unsigned persistent_grid(Kernel k, size_t smem, int64_t tiles) {
    int dev = 0, sms = 1, per_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, TILE_PIX, smem);
    if (per_sm < 1) per_sm = 1;
    const int64_t g = (int64_t)sms * per_sm;
    return (unsigned)(g < tiles ? g : tiles);
}

}  // namespace pf
