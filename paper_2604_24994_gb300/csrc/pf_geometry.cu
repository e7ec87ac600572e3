// pf_prepare / pf_project kernels: FP64 geometry per cell and per (view, cell).
#include <math_constants.h>

#include "pf_internal.cuh"

namespace pf {

// ---------------------------------------------------------------------------
// View-independent cell records.
//
// Per cell, in FP64: unit normal, face frame (e1, e2) / R, and the radical
// planes of the listed neighbours, each stored as float + low part.  The
// plane between i and j is
//   (x - p_i).a <= g,  a = p_j - p_i,  g = (|a|^2 + w_i - w_j) / 2
// (pow(x,i) <= pow(x,j) with pow = |x - p|^2 - w, Eq. pow_dist); it is
// stored normalised, (a/|a|, g/|a|), so g/|a| is the signed distance of
// the plane from p_i.  A plane at distance >= R_i never reaches the ball
// and is dropped (Sec. 3.2: it cannot cut the cell); one at distance
// < -R_i excludes the whole ball and marks the cell empty.  Planes whose
// facet is shown empty by a single other plane or the dipole face are
// dropped as well (drop_implied_planes; a displaced face is taken at its
// highest, the offset plus the largest site displacement).
// ---------------------------------------------------------------------------

// FP64 1/sqrt(x): float estimate refined by two Newton steps (relative
// error ~1e-15; avoids the FP64 divide and square root sequences).
__device__ __forceinline__ double rsqrt64(double x) {
    double r = (double)rsqrtf((float)x);
    r = r * (1.5 - 0.5 * x * r * r);
    r = r * (1.5 - 0.5 * x * r * r);
    return r;
}

// Drop the planes that another constraint implies inside the ball B (radius
// R about p_i).  Plane k's disk B.(plane k) lies entirely outside the
// half-space H_j of a witness j (a plane or the dipole's dense half) when
//   min over the disk of a_j.y - g_j = g_k (a_j.a_k) - rho_k |a_j x a_k| - g_j > 0,
// rho_k = sqrt(R^2 - g_k^2).  Then the convex set B n H_j misses plane k, so
// it lies on one side of it; the point y = -R a_j of B n H_j shows which:
// if a_k.y < g_k, B n H_j is inside H_k and plane k changes no segment.
// Both tests keep a margin of 1e-5 R above the float error.  Witnesses are
// the planes still kept (earlier survivors, later ones not yet examined), so
// a dropped plane is always implied through a chain ending at a kept one.
// Planes are compacted in place; returns the new count.
__device__ int drop_implied_planes(float4 *__restrict__ P, float4 *__restrict__ PL, int2 *__restrict__ NB, int cnt,
                                   float4 face, float R) {
    const float tol = 1e-5f * R;
    int kept = 0;
    for (int k = 0; k < cnt; k++) {
        const float4 ak = P[k];
        const float rho = sqrtf(fmaxf(R * R - ak.w * ak.w, 0.0f));
        bool implied = false;
        for (int j = -1; j < cnt && !implied; j++) {
            if (j >= kept && j <= k) continue;   // slots [kept, k) are vacated, k is the plane itself
            const float4 aj = j < 0 ? face : P[j];
            const float c = ak.x * aj.x + ak.y * aj.y + ak.z * aj.z;
            // sin of the angle from the cross product (accurate for near-parallel normals)
            const float cx = ak.y * aj.z - ak.z * aj.y, cy = ak.z * aj.x - ak.x * aj.z, cz = ak.x * aj.y - ak.y * aj.x;
            const float sn = sqrtf(cx * cx + cy * cy + cz * cz);
            const float gap = ak.w * c - rho * sn - aj.w;
            implied = gap > tol && -R * c < ak.w - tol;
        }
        if (!implied) {
            if (kept != k) {
                P[kept] = ak;
                PL[kept] = PL[k];
                NB[kept] = NB[k];
            }
            kept++;
        }
    }
    return kept;
}

// (p, w) of every cell in one 16-byte word, so that each neighbour gather
// in prepare_kernel is a single load.
__global__ void __launch_bounds__(256) pack_sites_kernel(pf_scene s, float4 *__restrict__ pw) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= s.n_cells) return;
    pw[i] = make_float4(s.pos[3 * i], s.pos[3 * i + 1], s.pos[3 * i + 2], s.w[i]);
}

__global__ void __launch_bounds__(256) prepare_kernel(pf_scene s, const float4 *__restrict__ pw,
                                                      float *__restrict__ cellrec, int32_t *__restrict__ cellnp,
                                                      float4 *__restrict__ planes, float4 *__restrict__ planes_lo,
                                                      int2 *__restrict__ plane_nb) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= s.n_cells) return;
    const int K = s.k_nbr;
    const float pxf = s.pos[3 * i], pyf = s.pos[3 * i + 1], pzf = s.pos[3 * i + 2];
    const double px = pxf, py = pyf, pz = pzf;
    const float wif = s.w[i];
    const double wi = wif;
    const float Rf = s.R[i];
    const double R = Rf;
    const double nx0 = s.normal[3 * i], ny0 = s.normal[3 * i + 1], nz0 = s.normal[3 * i + 2];
    const double n2 = nx0 * nx0 + ny0 * ny0 + nz0 * nz0;
    const double inl = n2 > 0.0 ? rsqrt64(n2) : 0.0;
    const double nxd = nx0 * inl, nyd = ny0 * inl, nzd = nz0 * inl;
    const float nx = (float)nxd, ny = (float)nyd, nz = (float)nzd;
    // orthonormal face frame from the unit normal, branchless construction of
    // Duff et al. (JCGT 2017); divided by R so that u = (e1.y, e2.y) / R
    const float sg = nz >= 0.0f ? 1.0f : -1.0f;
    const float ca = -1.0f / (sg + nz);
    const float cb = nx * ny * ca;
    const float iR = Rf > 0.0f ? 1.0f / Rf : 0.0f;
    const float e1x = (1.0f + sg * nx * nx * ca) * iR, e1y = sg * cb * iR, e1z = -sg * nx * iR;
    const float e2x = cb * iR, e2y = (sg + ny * ny * ca) * iR, e2z = -ny * iR;

    bool empty = !(R > 0.0) || !(n2 > 0.0);
    int cnt = 0;
    for (int k = 0; k < K; k++) {
        const int j = s.nbr[(int64_t)i * K + k];
        if (j < 0 || j >= s.n_cells || j == i) continue;
        const float4 pj = pw[j];
        const float qx = pj.x, qy = pj.y, qz = pj.z;
        const float wjf = pj.w;
        // float pre-test with a wide margin: only planes that may reach the
        // ball (distance (|a|^2 + w_i - w_j) / (2|a|) < R) go on to FP64
        {
            const float ax = qx - pxf, ay = qy - pyf, az = qz - pzf;
            const float L2 = ax * ax + ay * ay + az * az;
            const float num = L2 + wif - wjf;
            const float mag = L2 + fabsf(wif) + fabsf(wjf);
            const float Lf = sqrtf(L2);
            if (L2 > 0.0f && num > 2.0f * Lf * Rf * 1.001f + 1e-4f * mag) continue;
        }
        const double ax = (double)qx - px, ay = (double)qy - py, az = (double)qz - pz;
        const double wj = wjf;
        const double L2 = ax * ax + ay * ay + az * az;
        if (L2 == 0.0) {  // coincident sites: pow(x,i) <= pow(x,j) iff w_i >= w_j
            if (wi < wj) empty = true;
            continue;
        }
        const double iL = rsqrt64(L2);
        const double g = 0.5 * (L2 + wi - wj) * iL;  // plane distance from p_i
        if (g < -R * (1.0 + 1e-6)) empty = true;
        if (g < R * (1.0 + 1e-6)) {
            const double ux = ax * iL, uy = ay * iL, uz = az * iL;
            const float4 hi = make_float4((float)ux, (float)uy, (float)uz, (float)g);
            planes[(int64_t)i * K + cnt] = hi;
            planes_lo[(int64_t)i * K + cnt] = make_float4((float)(ux - (double)hi.x), (float)(uy - (double)hi.y),
                                                          (float)(uz - (double)hi.z), (float)(g - (double)hi.w));
            plane_nb[(int64_t)i * K + cnt] = make_int2(j, __float_as_int((float)(L2 * iL)));
            cnt++;
        }
    }
    // the face as a witness at its widest: a displaced face (Eq. svdisp) moves
    // by a convex combination of the site displacements, at most their maximum
    float face_off = s.offset[i];
    if (s.disp) {
        const int ns = scene_sites(s);
        float mx = s.disp[(int64_t)ns * i];
        for (int k = 1; k < ns; k++) mx = fmaxf(mx, s.disp[(int64_t)ns * i + k]);
        face_off += mx;
    }
    if (!empty) cnt = drop_implied_planes(planes + (int64_t)i * K, planes_lo + (int64_t)i * K,
                                          plane_nb + (int64_t)i * K, cnt, make_float4(nx, ny, nz, face_off), Rf);
    // nearest planes first: they cut the most of the ball, so a warp whose
    // segments all become empty stops the plane loop earliest
    {
        float4 *P = planes + (int64_t)i * K, *PL = planes_lo + (int64_t)i * K;
        int2 *NB = plane_nb + (int64_t)i * K;
        for (int a = 1; a < cnt; a++) {
            const float4 p = P[a], pl = PL[a];
            const int2 nb = NB[a];
            int b = a - 1;
            for (; b >= 0 && P[b].w > p.w; b--) {
                P[b + 1] = P[b];
                PL[b + 1] = PL[b];
                NB[b + 1] = NB[b];
            }
            P[b + 1] = p;
            PL[b + 1] = pl;
            NB[b + 1] = nb;
        }
    }
    cellnp[i] = cnt;
    float4 *cr = reinterpret_cast<float4 *>(cellrec + (int64_t)i * CELLREC_F);
    cr[0] = make_float4(nx, ny, nz, s.offset[i]);
    cr[1] = make_float4(e1x, e1y, e1z, Rf);
    cr[2] = make_float4(e2x, e2y, e2z, s.sigma[i]);
    cr[3] = make_float4(s.rgb[3 * i], s.rgb[3 * i + 1], s.rgb[3 * i + 2], __int_as_float(empty ? 1 : 0));
    if (s.n_sites == 8) {  // eight sites: the renderer stages tex [N,24] beside the record
        cr[4] = cr[5] = cr[6] = make_float4(0.f, 0.f, 0.f, 0.f);
    } else {
        const float4 *tx = reinterpret_cast<const float4 *>(s.tex + (int64_t)i * 12);
        cr[4] = tx[0];
        cr[5] = tx[1];
        cr[6] = tx[2];
    }
    cr[7] = make_float4((float)(nxd - (double)nx), (float)(nyd - (double)ny), (float)(nzd - (double)nz),
                        (float)(n2 * inl));
}

// ---------------------------------------------------------------------------
// Per (view, cell) projection.
//
// Painter key: pow(o, p_i) = |p_i - o|^2 - w_i in FP64 (Thm. power_painter),
// mapped to order-preserving unsigned bits.
//
// Tile rectangle: the image-plane bounding box of the sphere (p_i, R_i),
// from the tangent lines through the camera centre in the camera's x-z and
// y-z planes, covering every pixel whose centre lies inside it.  For a
// sphere well in front of the camera plane (camera-frame Z > 2 R) the box
// is evaluated in float from the camera-frame centre rounded to float, and
// widened by 2^-18 (|f| (|X| / Z + 1) + |c|) pixels per axis, a bound on the
// float evaluation's rounding (about 32 ulps of those magnitudes); closer
// spheres take the same box in double, widened by 1e-6 px.  A sphere
// reaching z <= 0 gets the whole image unless it lies entirely outside one
// side plane of the frustum; one entirely behind is dropped.  Every
// operation is an explicitly rounded IEEE operation (no contraction), so a
// CPU evaluating the same rule in the same order gets the same rectangles
// bit for bit.
//
// Site offset m = o - p_i is stored as a float pair (hi + lo ~ 48 bits) for
// the renderer's compensated products; Rt^2 is a conservative radius^2 for
// the cheap single-float sphere test (covers its rounding); the last slot
// holds the cell's near-tangent threshold on |D|.
// ---------------------------------------------------------------------------
#define DADD __dadd_rn
#define DSUB __dsub_rn
#define DMUL __dmul_rn
#define DDIV __ddiv_rn
#define DSQRT __dsqrt_rn

// Widening (pixels) of one edge of the float tile box: 2^-17 (|f| ((1 + k^2)
// |c|_1 / Z + |X| / Z + 1) + |c0|) for an edge of slope k, focal length f and
// principal point c0, with |c|_1 / Z = (|X| + |Y| + Z) / Z.  It bounds, with a
// factor of four to spare, the float error of the edge: about 32 ulps of
// |f| (|X| / Z + 1) from evaluating the tangent slopes (Z > 2 R keeps
// Z^2 - R^2 >= 3 Z^2 / 4), and 23 ulps of |f| (1 + k^2) |c|_1 / Z from the
// camera-frame centre's own rounding (about 10 ulps of |c|_1, moving the
// slope by (1 + k^2) times the angle it subtends).
__device__ __forceinline__ float box_margin(float f, float c0, float k, float L1z, float az) {
    return __fmul_rn(0x1p-17f,
                     __fadd_rn(__fmul_rn(fabsf(f), __fadd_rn(__fmul_rn(__fadd_rn(1.0f, __fmul_rn(k, k)), L1z), az)),
                               fabsf(c0)));
}

__global__ void __launch_bounds__(256) project_kernel(pf_scene s, const ViewDev *__restrict__ views, int nv,
                                                      const float *__restrict__ cellrec, float *__restrict__ viewrec,
                                                      ushort4 *__restrict__ rect_out,
                                                      unsigned long long *__restrict__ key_out,
                                                      uint32_t *__restrict__ cnt_out, int32_t *__restrict__ diff,
                                                      int64_t diff_total) {
    const int64_t N = s.n_cells;
    // the views of this block's cells (one or two unless the scene has fewer
    // cells than the block has threads), staged in shared memory: every
    // thread reads some thirty of their fields
    __shared__ ViewDev sv[2];
    const int64_t first = (int64_t)blockIdx.x * blockDim.x;
    const int v0 = (int)(first / N);
    const int v1 = (int)min((int64_t)nv - 1, (first + blockDim.x - 1) / N);
    const bool staged = v1 - v0 < 2;
    if (staged) {
        constexpr int WORDS = (int)(sizeof(ViewDev) / 4);
        static_assert(sizeof(ViewDev) % 4 == 0, "ViewDev is copied as 32-bit words");
        for (int q = threadIdx.x; q < WORDS * (v1 - v0 + 1); q += blockDim.x)
            reinterpret_cast<uint32_t *>(sv)[q] = reinterpret_cast<const uint32_t *>(views + v0)[q];
    }
    __syncthreads();
    const int64_t idx = first + threadIdx.x;
    if (idx >= N * nv) return;
    const int v = (int)(idx / N);
    const int64_t i = idx - (int64_t)v * N;
    const ViewDev &V = staged ? sv[v - v0] : views[v];
    const double px = s.pos[3 * i], py = s.pos[3 * i + 1], pz = s.pos[3 * i + 2];
    const double dx = DSUB(px, V.origin[0]);
    const double dy = DSUB(py, V.origin[1]);
    const double dz = DSUB(pz, V.origin[2]);
    const double pw = DSUB(DADD(DADD(DMUL(dx, dx), DMUL(dy, dy)), DMUL(dz, dz)), (double)s.w[i]);
    unsigned long long bits = (unsigned long long)__double_as_longlong(pw);
    key_out[idx] = (bits >> 63) ? ~bits : (bits | 0x8000000000000000ull);

    // camera-relative offset m = o - p as a float pair: Knuth's two-sum of
    // the origin's high part and -p, then the origin's low part added
    float hm[3], lm[3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const float p = s.pos[3 * i + c];
        const float a = V.ohi[c];
        const float s0 = __fsub_rn(a, p);
        const float bb = __fsub_rn(s0, a);
        const float e0 = __fadd_rn(__fsub_rn(a, __fsub_rn(s0, bb)), __fsub_rn(-p, bb));
        const float t0 = __fadd_rn(e0, V.olo[c]);
        hm[c] = __fadd_rn(s0, t0);
        lm[c] = __fsub_rn(t0, __fsub_rn(hm[c], s0));
    }
    {
        // |m| only sets the margin 2^-19 |m| of the bound radius: float is plenty
        const float mlen = sqrtf(fmaf(hm[0], hm[0], fmaf(hm[1], hm[1], hm[2] * hm[2])));
        const float Rt = __fmaf_ru(mlen, 0x1p-19f, __fmul_ru(s.R[i], 1.0f + 0x1p-20f));
        const float rt2 = __fmul_ru(__fmul_ru(Rt, Rt), 1.0f + 0x1p-20f);
        float4 *vr = reinterpret_cast<float4 *>(viewrec + idx * VIEWREC_F);
        vr[0] = make_float4(hm[0], hm[1], hm[2], rt2);
        vr[1] = make_float4(lm[0], lm[1], lm[2], sphere_refine_threshold(s.R[i], s.sigma[i]));
    }

    ushort4 rc = make_ushort4(1, 1, 0, 0);
    uint32_t count = 0;
    // camera-frame centre in float from the rounded offset (d = -m)
    const float *Mf = V.rotf;
    const float Xf = -__fadd_rn(__fadd_rn(__fmul_rn(Mf[0], hm[0]), __fmul_rn(Mf[1], hm[1])), __fmul_rn(Mf[2], hm[2]));
    const float Yf = -__fadd_rn(__fadd_rn(__fmul_rn(Mf[3], hm[0]), __fmul_rn(Mf[4], hm[1])), __fmul_rn(Mf[5], hm[2]));
    const float Zf = -__fadd_rn(__fadd_rn(__fmul_rn(Mf[6], hm[0]), __fmul_rn(Mf[7], hm[1])), __fmul_rn(Mf[8], hm[2]));
    const float rf = s.R[i];
    const double W = V.width, H = V.height;
    double ulo = -CUDART_INF, uhi = CUDART_INF, vlo = -CUDART_INF, vhi = CUDART_INF;
    // well in front of the camera and within 89.9 degrees of its axis: the
    // float tile box below; otherwise the double one from the double centre
    const bool fast = V.model != PF_FISHEYE && Zf > __fmul_rn(2.0f, rf) &&
                      __fmul_rn(Zf, 1024.0f) > __fadd_rn(fabsf(Xf), fabsf(Yf));
    bool vis = true;
    float fa0 = 0.f, fa1 = 0.f, fb0 = 0.f, fb1 = 0.f;
    double X = 0.0, Y = 0.0, Z = 0.0;
    const double r = rf;
    if (fast) {
        const float rr = __fmul_rn(rf, rf), zz = __fmul_rn(Zf, Zf);
        const float izr = __fdiv_rn(1.0f, __fsub_rn(zz, rr));
        const float sx = __fsqrt_rn(__fsub_rn(__fadd_rn(__fmul_rn(Xf, Xf), zz), rr));
        const float sy = __fsqrt_rn(__fsub_rn(__fadd_rn(__fmul_rn(Yf, Yf), zz), rr));
        const float xz = __fmul_rn(Xf, Zf), yz = __fmul_rn(Yf, Zf);
        const float rsx = __fmul_rn(rf, sx), rsy = __fmul_rn(rf, sy);
        const float kxl = __fmul_rn(__fsub_rn(xz, rsx), izr), kxh = __fmul_rn(__fadd_rn(xz, rsx), izr);
        const float kyl = __fmul_rn(__fsub_rn(yz, rsy), izr), kyh = __fmul_rn(__fadd_rn(yz, rsy), izr);
        const float L1z = __fdiv_rn(__fadd_rn(__fadd_rn(fabsf(Xf), fabsf(Yf)), Zf), Zf);
        const float axz = __fadd_rn(__fdiv_rn(fabsf(Xf), Zf), 1.0f), ayz = __fadd_rn(__fdiv_rn(fabsf(Yf), Zf), 1.0f);
        fa0 = ceilf(__fsub_rn(__fsub_rn(__fadd_rn(__fmul_rn(V.fxf, kxl), V.cxf), 0.5f),
                              box_margin(V.fxf, V.cxf, kxl, L1z, axz)));
        fa1 = floorf(__fadd_rn(__fsub_rn(__fadd_rn(__fmul_rn(V.fxf, kxh), V.cxf), 0.5f),
                               box_margin(V.fxf, V.cxf, kxh, L1z, axz)));
        fb0 = ceilf(__fsub_rn(__fsub_rn(__fadd_rn(__fmul_rn(V.fyf, kyl), V.cyf), 0.5f),
                              box_margin(V.fyf, V.cyf, kyl, L1z, ayz)));
        fb1 = floorf(__fadd_rn(__fsub_rn(__fadd_rn(__fmul_rn(V.fyf, kyh), V.cyf), 0.5f),
                               box_margin(V.fyf, V.cyf, kyh, L1z, ayz)));
    } else {
        const double *M = V.rot;
        X = DADD(DADD(DMUL(M[0], dx), DMUL(M[1], dy)), DMUL(M[2], dz));
        Y = DADD(DADD(DMUL(M[3], dx), DMUL(M[4], dy)), DMUL(M[5], dz));
        Z = DADD(DADD(DMUL(M[6], dx), DMUL(M[7], dy)), DMUL(M[8], dz));
        vis = !(DADD(Z, r) <= 0.0);
    }
    if (fast) {
        // the box is fa0..fb1
    } else if (V.model == PF_FISHEYE) {
        // equidistant fisheye: the directions that meet the sphere form a cap
        // of angular radius asin(r/|c|) around c; its pixels lie in the box
        // of the annular sector theta in [thc - b, thc + b], phi in
        // [phc - dphi, phc + dphi] (image offsets theta (cos phi, sin phi)
        // scaled by fx, fy), or of the disc of radius thc + b when the cap
        // holds the optical axis.  Conservative; the renderer tests each ray.
        vis = true;
        const double L = sqrt(X * X + Y * Y + Z * Z);
        if (L > r) {
            const double b = asin(r / L) * (1.0 + 1e-12) + 1e-12;
            const double rho = sqrt(X * X + Y * Y);
            const double thc = atan2(rho, Z);
            const double th0 = thc - b, th1 = fmin(thc + b, CUDART_PI);
            double xl, xh, yl, yh;
            const double st = sin(thc);
            if (th0 <= 0.0 || thc + b >= CUDART_PI || !(r / L < st * (1.0 - 1e-12))) {
                // the cap holds a pole, or spans every azimuth: a disc
                xl = yl = -th1;
                xh = yh = th1;
            } else {
                const double dphi = asin(fmin(r / L / st, 1.0)) * (1.0 + 1e-12) + 1e-12;
                const double phc = atan2(Y, X);
                const double p0 = phc - dphi, p1 = phc + dphi;
                double c0, s0, c1, s1;
                sincos(p0, &s0, &c0);
                sincos(p1, &s1, &c1);
                xl = fmin(fmin(th0 * c0, th1 * c0), fmin(th0 * c1, th1 * c1));
                xh = fmax(fmax(th0 * c0, th1 * c0), fmax(th0 * c1, th1 * c1));
                yl = fmin(fmin(th0 * s0, th1 * s0), fmin(th0 * s1, th1 * s1));
                yh = fmax(fmax(th0 * s0, th1 * s0), fmax(th0 * s1, th1 * s1));
                // the outer arc's extremes where it crosses an axis direction
                for (int q = -4; q <= 4; q++) {
                    const double psi = q * (0.5 * CUDART_PI);
                    if (psi < p0 || psi > p1) continue;
                    const int m = ((q % 4) + 4) % 4;
                    if (m == 0) xh = fmax(xh, th1);
                    if (m == 1) yh = fmax(yh, th1);
                    if (m == 2) xl = fmin(xl, -th1);
                    if (m == 3) yl = fmin(yl, -th1);
                }
            }
            ulo = V.cx + V.fx * xl;
            uhi = V.cx + V.fx * xh;
            vlo = V.cy + V.fy * yl;
            vhi = V.cy + V.fy * yh;
        }
    } else if (vis && Z > r) {
        // tangent lines from the camera centre to the sphere's x-z and y-z circles
        const double rr = DMUL(r, r);
        const double izr = DDIV(1.0, DSUB(DMUL(Z, Z), rr));
        const double sx = DSQRT(DSUB(DADD(DMUL(X, X), DMUL(Z, Z)), rr));
        const double sy = DSQRT(DSUB(DADD(DMUL(Y, Y), DMUL(Z, Z)), rr));
        const double kxl = DMUL(DSUB(DMUL(X, Z), DMUL(r, sx)), izr);
        const double kxh = DMUL(DADD(DMUL(X, Z), DMUL(r, sx)), izr);
        const double kyl = DMUL(DSUB(DMUL(Y, Z), DMUL(r, sy)), izr);
        const double kyh = DMUL(DADD(DMUL(Y, Z), DMUL(r, sy)), izr);
        ulo = DADD(DMUL(V.fx, kxl), V.cx);
        uhi = DADD(DMUL(V.fx, kxh), V.cx);
        vlo = DADD(DMUL(V.fy, kyl), V.cy);
        vhi = DADD(DMUL(V.fy, kyh), V.cy);
    } else if (vis) {
        // reaches z <= 0: whole image unless outside a side plane x = k z
        if (DSUB(X, DMUL(V.kr, Z)) > DMUL(r, V.skr)) vis = false;
        if (DSUB(DMUL(V.kl, Z), X) > DMUL(r, V.skl)) vis = false;
        if (DSUB(Y, DMUL(V.kd, Z)) > DMUL(r, V.skd)) vis = false;
        if (DSUB(DMUL(V.ku, Z), Y) > DMUL(r, V.sku)) vis = false;
    }
    if (vis) {
        double a0, a1, b0, b1;
        if (fast) {  // whole numbers (or +-inf) in float: exact in double
            a0 = fa0;
            a1 = fa1;
            b0 = fb0;
            b1 = fb1;
        } else {
            a0 = ceil(DSUB(DSUB(ulo, 0.5), 1e-6));
            a1 = floor(DADD(DSUB(uhi, 0.5), 1e-6));
            b0 = ceil(DSUB(DSUB(vlo, 0.5), 1e-6));
            b1 = floor(DADD(DSUB(vhi, 0.5), 1e-6));
        }
        if (a0 < 0.0) a0 = 0.0;
        if (b0 < 0.0) b0 = 0.0;
        if (a1 > W - 1.0) a1 = W - 1.0;
        if (b1 > H - 1.0) b1 = H - 1.0;
        if (!(a0 > a1 || b0 > b1)) {
            const int x0 = (int)a0 / TILE, y0 = (int)b0 / TILE, x1 = (int)a1 / TILE, y1 = (int)b1 / TILE;
            rc = make_ushort4((unsigned short)x0, (unsigned short)y0, (unsigned short)x1, (unsigned short)y1);
            count = (uint32_t)(x1 - x0 + 1) * (uint32_t)(y1 - y0 + 1);
            // 2D difference grid: +1 at (x0,y0), -1 at (x1+1,y0) and (x0,y1+1), +1 at (x1+1,y1+1)
            const int gw = V.tiles_x + 1;
            int32_t *g = diff + diff_total * (int64_t)((blockIdx.x * 8 + (threadIdx.x >> 5)) % DIFF_REP) + V.diff_base;
            atomicAdd(&g[y0 * gw + x0], 1);
            atomicAdd(&g[y0 * gw + x1 + 1], -1);
            atomicAdd(&g[(y1 + 1) * gw + x0], -1);
            atomicAdd(&g[(y1 + 1) * gw + x1 + 1], 1);
        }
    }
    rect_out[idx] = rc;
    cnt_out[idx] = count;
}

// Connectivity loss (Sec. 4, L_connect) over the neighbour lists: per cell
// sum_j max(R_i + R_j - |p_i - p_j|, 0)^2, and, when asked, the gradient of
// the sum over cells: with o = R_i + R_j - d > 0, dR_i = dR_j = 2 o and
// dp_i = -dp_j = 2 o (p_j - p_i) / d.  One thread per cell; the neighbour
// side goes through atomics.
__global__ void __launch_bounds__(256) connect_kernel(pf_scene s, float *__restrict__ loss, float *__restrict__ gpos,
                                                      float *__restrict__ gR) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= s.n_cells) return;
    const int K = s.k_nbr;
    const float px = s.pos[3 * i], py = s.pos[3 * i + 1], pz = s.pos[3 * i + 2], Ri = s.R[i];
    float li = 0.f, gx = 0.f, gy = 0.f, gz = 0.f, gr = 0.f;
    for (int k = 0; k < K; k++) {
        const int j = s.nbr[(int64_t)i * K + k];
        if (j < 0 || j >= s.n_cells || j == i) continue;
        const float ax = s.pos[3 * j] - px, ay = s.pos[3 * j + 1] - py, az = s.pos[3 * j + 2] - pz;
        const float d = sqrtf(ax * ax + ay * ay + az * az);
        const float o = Ri + s.R[j] - d;
        if (!(o > 0.0f)) continue;
        li += o * o;
        if (gpos) {
            gr += 2.0f * o;
            atomicAdd(gR + j, 2.0f * o);
            if (d > 0.0f) {
                const float f = 2.0f * o / d;
                gx += f * ax;
                gy += f * ay;
                gz += f * az;
                atomicAdd(gpos + 3 * j, -f * ax);
                atomicAdd(gpos + 3 * j + 1, -f * ay);
                atomicAdd(gpos + 3 * j + 2, -f * az);
            }
        }
    }
    loss[i] = li;
    if (gpos) {
        atomicAdd(gR + i, gr);
        atomicAdd(gpos + 3 * i, gx);
        atomicAdd(gpos + 3 * i + 1, gy);
        atomicAdd(gpos + 3 * i + 2, gz);
    }
}

cudaError_t launch_connect(const pf_scene &s, float *loss, float *gpos, float *gR, cudaStream_t st) {
    if (s.n_cells == 0) return cudaSuccess;
    connect_kernel<<<(s.n_cells + 255) / 256, 256, 0, st>>>(s, loss, gpos, gR);
    return cudaGetLastError();
}

cudaError_t launch_prepare(const pf_scene &s, const Plan &p, const WS &w, cudaStream_t st) {
    if (p.n == 0) return cudaSuccess;
    const int threads = 256;
    const int blocks = (p.n + threads - 1) / threads;
    pack_sites_kernel<<<blocks, threads, 0, st>>>(s, w.pw);
    prepare_kernel<<<blocks, threads, 0, st>>>(s, w.pw, w.cellrec, w.cellnp, w.planes, w.planes_lo, w.plane_nb);
    return cudaGetLastError();
}

cudaError_t launch_project(const pf_scene &s, const Plan &p, const WS &w, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(w.diff, 0, sizeof(int32_t) * (size_t)p.total_diff * DIFF_REP, st);
    if (e != cudaSuccess) return e;
    const int64_t total = (int64_t)p.n * p.nv;
    if (total == 0) return cudaSuccess;
    const int threads = 256;
    const int64_t blocks = (total + threads - 1) / threads;
    project_kernel<<<(unsigned)blocks, threads, 0, st>>>(s, w.views, p.nv, w.cellrec, w.viewrec, w.rect, w.key,
                                                         w.cnt, w.diff, p.total_diff);
    return cudaGetLastError();
}

}  // namespace pf
