// pf_render_fwd / pf_render_bwd: per-pixel ray/cell segments, front-to-back
// compositing, and the back-to-front adjoint replay.
//
// One CTA per 16x16 tile, one thread per pixel; each warp covers an 8x4
// pixel block.  The tile's sorted cell list is staged into shared memory in
// batches of 32 cells with cp.async (16-byte granules): the 128-byte cell
// record, the 32-byte view record and the cell's relevant radical planes.
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
__device__ __noinline__ double3 fisheye_dir(double xc, double yc) {
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
__device__ __noinline__ float refine_plane64(const float *vr, float4 hi, float4 lo, Ray ray, float fallback,
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
__device__ __noinline__ float refine_D64(const float *vr, float R, Ray ray) {
    const double dx = (double)ray.dh.x + (double)ray.dl.x, dy = (double)ray.dh.y + (double)ray.dl.y,
                 dz = (double)ray.dh.z + (double)ray.dl.z;
    const double mx = (double)vr[0] + (double)vr[4], my = (double)vr[1] + (double)vr[5],
                 mz = (double)vr[2] + (double)vr[6];
    const double b = mx * dx + my * dy + mz * dz;
    const double qx = mx - b * dx, qy = my - b * dy, qz = mz - b * dz;
    return (float)((double)R * (double)R - (qx * qx + qy * qy + qz * qz));
}

// Sign of d.n in FP64 (the side of the face the texture point is taken on).
__device__ __noinline__ float face_side64(const float *cr, Ray ray) {
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
        sb = ub ? t : sb;
        kb = ub ? K_FACE : kb;
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
            sb = ub ? t : sb;
            kb = ub ? k + u : kb;
            if (NEED && need == np && !(sb > sa)) need = k + u + 1;
        }
        if (lanes && !__any_sync(lanes, sb > sa)) {
            k += 4;
            break;
        }
    }
    sg.nplanes = NEED ? need : min(k, np);
    // d.a of the constraints at the ends (+inf for sphere / camera ends); a
    // cell without planes reads some other slot of the batch and discards it
    const float4 Pa = pl[max(ka, 0)], Pb = pl[max(kb, 0)];
    float dena = ka >= 0 ? dot3(dh, f3(Pa.x, Pa.y, Pa.z)) : (ka == K_FACE ? fden : CUDART_INF_F);
    float denb = kb >= 0 ? dot3(dh, f3(Pb.x, Pb.y, Pb.z)) : (kb == K_FACE ? fden : CUDART_INF_F);
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
            tx.W[k] = __expf(-KAPPA * (tx.r[k] - rmin));
            Z += tx.W[k];
        }
    } else {
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const float ax = tx.ax[k & 1], ay = tx.ay[k >> 1];
            tx.r[k] = sqrt_approx(fmaf(ax, ax, ay * ay));
            tx.W[k] = __expf(-KAPPA * tx.r[k]);
            Z += tx.W[k];
        }
    }
    const float iz = __fdividef(1.0f, Z);
    float3 c = f3(cr[CR_RGB], cr[CR_RGB + 1], cr[CR_RGB + 2]);
    const float *tc = tex ? tex : cr + CR_TEX;  // eight sites: tex staged beside the record
#pragma unroll
    for (int k = 0; k < NS; k++) {
        tx.W[k] *= iz;
        const float3 ck = sv ? sv_colour(sv, k, ray.dh) : f3(tc[3 * k], tc[3 * k + 1], tc[3 * k + 2]);
        c.x = fmaf(tx.W[k], ck.x, c.x);
        c.y = fmaf(tx.W[k], ck.y, c.y);
        c.z = fmaf(tx.W[k], ck.z, c.z);
    }
    return c;
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
        // every warp is done with batch k-1, whose buffer batch k+1 reuses
        if (__syncthreads_count(!done) == 0) break;
        if (k + 1 < nbat) {
            issue_batch(sg, (k + 1) & 1, A.w.inst_sorted + s + (k + 1) * BATCH, min(BATCH, n - (k + 1) * BATCH),
                        A.w, vbase, A.K, false, disp, sites, tex8);
            cp_async_wait_one();
        } else {
            cp_async_wait_all();
        }
        __syncthreads();
        const int buf = k & 1, nb = min(BATCH, n - k * BATCH);
        unsigned mask = warp_mask(sg, buf, nb, cone);
        unsigned my_hits = 0;  // bit j: this pixel's segment in cell j of the batch is non-empty
        while (mask) {
            const int j = __ffs(mask) - 1;
            mask &= mask - 1;
            if (__all_sync(0xffffffffu, done)) break;
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
                if (nhit < HIT_CAP)
                    A.w.hitkind[(V.pix_base + (int64_t)py * V.width + px) * HIT_CAP + nhit] =
                        (uint16_t)((seg.ka + 3) | ((seg.kb + 3) << 7));
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

// --------------------------------------------------------------- backward
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
template <bool MASKS, bool EXT = false, int NS = 4, bool CONTRIB = false>
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
        __syncthreads();  // batch b+1, whose buffer batch b-1 reuses, is done
        if (b > 0) {
            issue_batch(stg, (b - 1) & 1, list + (b - 1) * BATCH, BATCH, A.w, vbase, A.K, true,
                        EXT ? A.disp : nullptr, EXT ? A.sites : nullptr, NS == 8 ? A.tex8 : nullptr);
            cp_async_wait_one();
        } else {
            cp_async_wait_all();
        }
        __syncthreads();
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
            if (MASKS) {
                // the forward recorded this hit's active constraints: no plane loop
                unsigned kk = 0xffffu;
                if (mine) {
                    kk = kk_next;
                    --nrec;
                    kk_next = nrec > 0 && nrec - 1 < HIT_CAP ? A.w.hitkind[pix * HIT_CAP + nrec - 1] : 0xffffu;
                }
                if (mine && sphere_chord<true>(cr, vr, ray, ch, cand)) {
                    if (kk != 0xffffu)
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
                const float Tbefore = Tafter * __expf(x);
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
    return A;
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

static size_t fwd_smem(int K) { return stage_bytes(K, false); }
static size_t bwd_smem(int K) { return stage_bytes(K, true); }

cudaError_t launch_render_fwd(const pf_scene &s, const Plan &p, const WS &w, float *rgb, float *T, uint32_t *last,
                              bool record, cudaStream_t st, float *contrib_sparse, float *contrib_normal) {
    if (p.total_tiles == 0) return cudaSuccess;
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
        auto kern =
            cq ? (disp && eight ? (m ? render_bwd_kernel<true, true, 8, true> : render_bwd_kernel<false, true, 8, true>)
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
