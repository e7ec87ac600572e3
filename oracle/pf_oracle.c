/*
 * FP64 CPU oracle for the bounded-power-cell renderer of Power Foam
 * (arxiv 2604.24994).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file; only the tests, the smoke check and the benchmark's CPU
 * baseline do.  It shares no code, header or constant with the CUDA library.
 *
 * Everything is the plain definition, in double precision, brute force:
 *
 *   ray        x(t) = o + t d, |d| = 1, through the pixel centre (u+.5, v+.5)
 *              of a pinhole camera (x_cam = rot (x - o)).
 *   power      pow(x, i) = |x - p_i|^2 - w_i                (Eq. pow_dist)
 *   power cell P_i = { x : pow(x,i) <= pow(x,j) for all j }  (Eq. power_cell)
 *   bound      B_i = { x : |x - p_i| <= R_i }                (Sec. 3.2)
 *   dense half D_i = { x : nh_i . (x - p_i) <= off_i },  nh = n/|n|
 *              (Sec. 3.3: the oriented face splits the cell; the outer half
 *              has zero density)
 *   segment    [ta, tb] = { t >= 0 : x(t) in B_i, P_i, D_i },  l = tb - ta
 *   colour     c_i = rgb_i + sum_k W_k tex_ik with soft-Voronoi weights
 *              W_k = softmax_k(-kappa |u - s_k|)               (Eq. svrad)
 *              evaluated at the end of the dense segment that lies on the
 *              face side, u = (e1.(x_s - p_i), e2.(x_s - p_i)) / R_i.
 *   opacity    alpha = 1 - exp(-sigma l)
 *   composite  segments sorted by entry distance ta (they are disjoint):
 *              C = sum_k T_k alpha_k c_k, T_{k+1} = T_k (1 - alpha_k),
 *              black background; T_final is returned separately.
 *              (Sec. 3.1: the volume rendering integral is a sum over the
 *              segments of the ray inside the cells.)
 *
 * The radical plane between i and j is  pow(x,i) = pow(x,j), i.e.
 *     2 x.(p_j - p_i) = |p_j|^2 - |p_i|^2 + w_i - w_j
 * (the definition of pow gives +w_i - w_j; the appendix's Eq.
 * power_bisector prints the weights the other way round).
 *
 * The adjoint (orc_render_grad) differentiates exactly this, in FP64, by
 * the implicit function theorem on whichever constraint is active at each
 * segment end.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* parameters as double arrays (the float32 inputs widen exactly; finite
 * differences perturb them in double) */
typedef struct {
    int64_t n;
    const double *pos, *w, *R, *sigma, *rgb, *normal, *offset, *tex;
    /* optional (NULL: none): displacement of the face at the four texture
     * sites, [n][nsite] (Eq. svdisp), with soft-Voronoi sharpness kappa_disp */
    const double *disp;
    double kappa_disp;
    /* optional (NULL: the fixed sites (+-1/3, +-1/3)): positions of the four
     * texture / detail sites on the face, [n][nsite][2], in units of R, in the
     * site order of tex and disp (Sec. 3.4: learnable detail sites) */
    const double *sites;
    /* optional (NULL: the constant site colours tex): view-dependent site
     * colours, a spherical-Voronoi function per site (Sec. 3.4): [n][nsite][8][6],
     * per site eight (axis xyz, rgb); sharpness sv_lambda */
    const double *sv;
    double sv_lambda;
    /* detail sites per face: 4 (also when 0) or 8; tex is [n][3 nsite], and
     * disp, sites and sv have nsite sites per cell */
    int32_t nsite;
} orc_scene;

/* model 0: pinhole.  model 1: equidistant fisheye (non-pinhole rasterization,
 * appendix D): the pixel centre's offset a = ((u+.5-cx)/fx, (v+.5-cy)/fy)
 * is the direction's angle from the optical axis, theta = |a|, towards
 * a/|a|; pixels with theta > pi have no ray. */
typedef struct {
    double rot[9];
    double origin[3];
    double fx, fy, cx, cy;
    int32_t width, height;
    int32_t model;
} orc_camera;

/* optional candidate lists: cell i is clipped against idx[beg[i]..end[i])
 * only (ascending, i excluded).  A NULL list, or beg[i] < 0, means against
 * every other site.  A candidate list must contain every j whose radical
 * plane can cut B_i; the others can never bind, so the result is the same. */
typedef struct {
    const int64_t *beg, *end;
    const int32_t *idx;
} orc_cands;

enum { ACT_SPHERE = -1, ACT_CAMERA = -2, ACT_DIPOLE = -3 };

typedef struct {
    int32_t cell;
    double ta, tb;
    int32_t act_a, act_b;
} orc_seg;

static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

static void load3(const double *p, int64_t i, double *o) {
    o[0] = p[3 * i];
    o[1] = p[3 * i + 1];
    o[2] = p[3 * i + 2];
}

/* pixel-centre ray; 0 if the pixel has none (fisheye beyond theta = pi) */
int orc_ray(const orc_camera *cam, double u, double v, double *o, double *d) {
    double dc[3] = {(u + 0.5 - cam->cx) / cam->fx, (v + 0.5 - cam->cy) / cam->fy, 1.0};
    if (cam->model == 1) {
        double th = sqrt(dc[0] * dc[0] + dc[1] * dc[1]);
        if (th > 3.14159265358979323846) return 0;
        double f = th > 0.0 ? sin(th) / th : 1.0;
        dc[0] *= f;
        dc[1] *= f;
        dc[2] = cos(th);
    }
    double dw[3];
    for (int r = 0; r < 3; r++)
        dw[r] = cam->rot[0 * 3 + r] * dc[0] + cam->rot[1 * 3 + r] * dc[1] + cam->rot[2 * 3 + r] * dc[2];
    double nn = sqrt(dot3(dw, dw));
    for (int r = 0; r < 3; r++) {
        d[r] = dw[r] / nn;
        o[r] = cam->origin[r];
    }
    return 1;
}

/* unit dipole normal */
static void unit_normal(const orc_scene *s, int64_t i, double *nh, double *len) {
    double n[3];
    load3(s->normal, i, n);
    double L = sqrt(dot3(n, n));
    for (int r = 0; r < 3; r++) nh[r] = n[r] / L;
    *len = L;
}

static double face_disp(const orc_scene *s, int64_t i, const double *o, const double *d, double *W, double *u,
                        double *tbar);

/*
 * Segment of the ray inside cell i (brute force over every other site, or
 * over the given candidates).  Returns 1 when non-empty.
 */
static int cell_segment(const orc_scene *s, const orc_cands *cd, int64_t i, const double *o, const double *d,
                        orc_seg *out) {
    double p[3], m[3];
    load3(s->pos, i, p);
    for (int r = 0; r < 3; r++) m[r] = o[r] - p[r];
    double R = s->R[i];
    /* sphere |m + t d|^2 = R^2:  t^2 + 2 b t + c = 0 */
    double b = dot3(m, d);
    double c = dot3(m, m) - R * R;
    double disc = b * b - c;
    if (disc < 0.0) return 0;
    double sq = sqrt(disc);
    /* numerically stable roots */
    double q = (b >= 0.0) ? -(b + sq) : -(b - sq);
    double t0, t1;
    if (q == 0.0) {
        t0 = t1 = 0.0;
    } else {
        double r1 = q, r2 = c / q;
        t0 = r1 < r2 ? r1 : r2;
        t1 = r1 < r2 ? r2 : r1;
    }
    double ta = t0, tb = t1;
    int aa = ACT_SPHERE, ab = ACT_SPHERE;
    if (ta < 0.0) {
        ta = 0.0;
        aa = ACT_CAMERA;
    }
    if (tb <= ta) return 0;
    double wi = s->w[i];
    /* radical planes:  x.a <= (|p_j|^2 - |p_i|^2 + w_i - w_j)/2  with a = p_j - p_i,
     * written for x = o + t d as  t (d.a) <= h,  h = (|a|^2 + w_i - w_j)/2 - a.m */
    int64_t jb = 0, je = s->n;
    int use_list = (cd && cd->beg && cd->beg[i] >= 0);
    if (use_list) {
        jb = cd->beg[i];
        je = cd->end[i];
    }
    for (int64_t jj = jb; jj < je; jj++) {
        int64_t j = use_list ? (int64_t)cd->idx[jj] : jj;
        if (j == i) continue;
        double pj[3], a[3];
        load3(s->pos, j, pj);
        for (int r = 0; r < 3; r++) a[r] = pj[r] - p[r];
        double h = 0.5 * (dot3(a, a) + wi - (double)s->w[j]) - dot3(a, m);
        double den = dot3(d, a);
        if (den > 0.0) {
            double t = h / den;
            if (t < tb) {
                tb = t;
                ab = (int)j;
            }
        } else if (den < 0.0) {
            double t = h / den;
            if (t > ta) {
                ta = t;
                aa = (int)j;
            }
        } else if (h < 0.0) {
            return 0;
        }
        if (tb <= ta) return 0;
    }
    /* dense half:  nh.(x - p) <= off  ->  t (nh.d) <= off - nh.m */
    double nh[3], nl;
    unit_normal(s, i, nh, &nl);
    double den = dot3(nh, d);
    double h = (double)s->offset[i] - dot3(nh, m);
    if (s->disp) h += face_disp(s, i, o, d, NULL, NULL, NULL);
    if (den > 0.0) {
        double t = h / den;
        if (t < tb) {
            tb = t;
            ab = ACT_DIPOLE;
        }
    } else if (den < 0.0) {
        double t = h / den;
        if (t > ta) {
            ta = t;
            aa = ACT_DIPOLE;
        }
    } else if (h < 0.0) {
        return 0;
    }
    if (tb <= ta) return 0;
    out->cell = (int32_t)i;
    out->ta = ta;
    out->tb = tb;
    out->act_a = aa;
    out->act_b = ab;
    return 1;
}

/*
 * Orthonormal frame (e1, e2) of the face with unit normal nh, by the
 * branchless construction of Duff et al., "Building an Orthonormal Basis,
 * Revisited" (JCGT 2017).  J1/J2 (optional) receive de/dnh as 3x3
 * row-major matrices J[r][c] = d e_r / d nh_c, treating the three
 * components of nh as independent.
 */
static void onb(const double *n, double *e1, double *e2, double *J1, double *J2) {
    double sg = n[2] >= 0.0 ? 1.0 : -1.0;
    double a = -1.0 / (sg + n[2]);
    double b = n[0] * n[1] * a;
    e1[0] = 1.0 + sg * n[0] * n[0] * a;
    e1[1] = sg * b;
    e1[2] = -sg * n[0];
    e2[0] = b;
    e2[1] = sg + n[1] * n[1] * a;
    e2[2] = -n[1];
    if (J1) {
        double da = a * a; /* d a / d nz */
        double db[3] = {n[1] * a, n[0] * a, n[0] * n[1] * da};
        double J1v[9] = {2.0 * sg * n[0] * a, 0.0, sg * n[0] * n[0] * da,
                         sg * db[0], sg * db[1], sg * db[2],
                         -sg, 0.0, 0.0};
        double J2v[9] = {db[0], db[1], db[2],
                         0.0, 2.0 * n[1] * a, n[1] * n[1] * da,
                         0.0, -1.0, 0.0};
        memcpy(J1, J1v, sizeof J1v);
        memcpy(J2, J2v, sizeof J2v);
    }
}

void orc_onb(const double *n, double *e1, double *e2) { onb(n, e1, e2, NULL, NULL); }

/* the four texture sites, in units of R on the face, site-major */
static const double SITE[4][2] = {{-1.0 / 3.0, -1.0 / 3.0}, {1.0 / 3.0, -1.0 / 3.0}, {-1.0 / 3.0, 1.0 / 3.0}, {1.0 / 3.0, 1.0 / 3.0}};

/* eight fixed sites: the 3 x 3 grid of step 1/3 without its centre, row by row */
static const double SITE8[8][2] = {{-1.0 / 3.0, -1.0 / 3.0}, {0.0, -1.0 / 3.0}, {1.0 / 3.0, -1.0 / 3.0},
                                   {-1.0 / 3.0, 0.0},        {1.0 / 3.0, 0.0},  {-1.0 / 3.0, 1.0 / 3.0},
                                   {0.0, 1.0 / 3.0},         {1.0 / 3.0, 1.0 / 3.0}};
enum { MAXS = 8 };

static int nsites(const orc_scene *s) { return s->nsite == 8 ? 8 : 4; }

/* site k of cell i: the scene's learned position, else the fixed one */
static double site_x(const orc_scene *s, int64_t i, int k) {
    const int ns = nsites(s);
    return s->sites ? s->sites[2 * ns * i + 2 * k] : (ns == 8 ? SITE8[k][0] : SITE[k][0]);
}
static double site_y(const orc_scene *s, int64_t i, int k) {
    const int ns = nsites(s);
    return s->sites ? s->sites[2 * ns * i + 2 * k + 1] : (ns == 8 ? SITE8[k][1] : SITE[k][1]);
}

/*
 * Displacement of the face for one ray (Eq. svdisp, with the one-step plane
 * shift): the ray crosses the base face nh.(x - p) = off at
 * tbar = (off - nh.m)/(nh.d), m = o - p; there, u = (e1.y, e2.y)/R with
 * y = m + tbar d, and delta = sum_k W_k disp_k with the soft-Voronoi weights
 * W_k = softmax_k(-kappa_disp |u - s_k|) over the four texture sites.  The
 * ray then meets the displaced face nh.(x - p) = off + delta.  A ray
 * parallel to the face (nh.d = 0) has no crossing: delta = 0.
 */
static double face_disp(const orc_scene *s, int64_t i, const double *o, const double *d, double *W, double *u,
                        double *tbar) {
    double nh[3], nl, p[3], m[3], y[3], e1[3], e2[3];
    unit_normal(s, i, nh, &nl);
    double den = dot3(nh, d);
    const int ns = nsites(s);
    if (!s->disp || den == 0.0) {
        if (W)
            for (int k = 0; k < ns; k++) W[k] = 0.0;
        if (tbar) *tbar = 0.0;
        return 0.0;
    }
    load3(s->pos, i, p);
    for (int r = 0; r < 3; r++) m[r] = o[r] - p[r];
    double tb = ((double)s->offset[i] - dot3(nh, m)) / den;
    for (int r = 0; r < 3; r++) y[r] = m[r] + tb * d[r];
    onb(nh, e1, e2, NULL, NULL);
    double R = s->R[i];
    double uu[2] = {dot3(e1, y) / R, dot3(e2, y) / R};
    double lg[MAXS], mx = -INFINITY, Wk[MAXS], Z = 0.0, delta = 0.0;
    for (int k = 0; k < ns; k++) {
        double dx = uu[0] - site_x(s, i, k), dy = uu[1] - site_y(s, i, k);
        lg[k] = -s->kappa_disp * sqrt(dx * dx + dy * dy);
        if (lg[k] > mx) mx = lg[k];
    }
    for (int k = 0; k < ns; k++) {
        Wk[k] = exp(lg[k] - mx);
        Z += Wk[k];
    }
    for (int k = 0; k < ns; k++) {
        Wk[k] /= Z;
        delta += Wk[k] * s->disp[(int64_t)ns * i + k];
    }
    if (W) memcpy(W, Wk, sizeof(double) * (size_t)ns);
    if (u) memcpy(u, uu, sizeof uu);
    if (tbar) *tbar = tb;
    return delta;
}

/*
 * Colour of site k of cell i seen along the ray (reading of Sec. 3.4's
 * spherical-Voronoi radiance): with the outgoing direction wo = -d and the
 * site's eight axes a_j (normalised) and colours c_j,
 * c_k(wo) = sum_j P_j c_j, P_j = softmax_j(sv_lambda a_j.wo).
 * P (optional) receives the eight weights.
 */
static void sv_colour(const orc_scene *s, int64_t i, int k, const double *d, double *c, double *P) {
    const double *q = s->sv + (((int64_t)i * nsites(s) + k) * 8) * 6;
    double lg[8], mx = -INFINITY, Z = 0.0;
    for (int j = 0; j < 8; j++) {
        const double *a = q + 6 * j;
        double L = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
        lg[j] = -s->sv_lambda * (a[0] * d[0] + a[1] * d[1] + a[2] * d[2]) / L;
        if (lg[j] > mx) mx = lg[j];
    }
    double Pj[8];
    for (int j = 0; j < 8; j++) {
        Pj[j] = exp(lg[j] - mx);
        Z += Pj[j];
    }
    c[0] = c[1] = c[2] = 0.0;
    for (int j = 0; j < 8; j++) {
        Pj[j] /= Z;
        for (int ch = 0; ch < 3; ch++) c[ch] += Pj[j] * q[6 * j + 3 + ch];
    }
    if (P) memcpy(P, Pj, sizeof Pj);
}

/* colour of cell i for the segment (Eq. svrad, see header) */
static void cell_colour(const orc_scene *s, int64_t i, const double *o, const double *d, const orc_seg *sg,
                        double kappa, double *col, double *Wout, double *uout, double *ts_out) {
    double nh[3], nl;
    unit_normal(s, i, nh, &nl);
    double ts = (dot3(nh, d) > 0.0) ? sg->tb : sg->ta;
    double p[3], y[3], e1[3], e2[3];
    load3(s->pos, i, p);
    for (int r = 0; r < 3; r++) y[r] = o[r] + ts * d[r] - p[r];
    onb(nh, e1, e2, NULL, NULL);
    double R = s->R[i];
    double u[2] = {dot3(e1, y) / R, dot3(e2, y) / R};
    const int ns = nsites(s);
    double lg[MAXS], mx = -INFINITY;
    for (int k = 0; k < ns; k++) {
        double dx = u[0] - site_x(s, i, k), dy = u[1] - site_y(s, i, k);
        lg[k] = -kappa * sqrt(dx * dx + dy * dy);
        if (lg[k] > mx) mx = lg[k];
    }
    double W[MAXS], Z = 0.0;
    for (int k = 0; k < ns; k++) {
        W[k] = exp(lg[k] - mx);
        Z += W[k];
    }
    for (int k = 0; k < ns; k++) W[k] /= Z;
    double ck[MAXS][3];
    for (int k = 0; k < ns; k++) {
        if (s->sv)
            sv_colour(s, i, k, d, ck[k], NULL);
        else
            for (int ch = 0; ch < 3; ch++) ck[k][ch] = (double)s->tex[3 * ns * i + 3 * k + ch];
    }
    for (int ch = 0; ch < 3; ch++) {
        double v = s->rgb[3 * i + ch];
        for (int k = 0; k < ns; k++) v += W[k] * ck[k][ch];
        col[ch] = v;
    }
    if (Wout) memcpy(Wout, W, sizeof(double) * (size_t)ns);
    if (uout) memcpy(uout, u, sizeof u);
    if (ts_out) *ts_out = ts;
}

static int cmp_seg(const void *a, const void *b) {
    const orc_seg *x = a, *y = b;
    if (x->ta < y->ta) return -1;
    if (x->ta > y->ta) return 1;
    return (x->cell > y->cell) - (x->cell < y->cell);
}

/* all non-empty segments of one ray, sorted by entry distance */
static int64_t ray_segments(const orc_scene *s, const orc_cands *cd, const double *o, const double *d, orc_seg **buf,
                            int64_t *cap) {
    int64_t n = 0;
    for (int64_t i = 0; i < s->n; i++) {
        orc_seg sg;
        if (!cell_segment(s, cd, i, o, d, &sg)) continue;
        if (n == *cap) {
            *cap = *cap ? 2 * *cap : 64;
            *buf = realloc(*buf, (size_t)*cap * sizeof(orc_seg));
        }
        (*buf)[n++] = sg;
    }
    if (n > 1) qsort(*buf, (size_t)n, sizeof(orc_seg), cmp_seg);
    return n;
}

/* exported for the tests: segments of an explicit ray */
int64_t orc_ray_segments(const orc_scene *s, const orc_cands *cd, const double *o, const double *d, int64_t maxn,
                         int32_t *cell, double *ta, double *tb, int32_t *act_a, int32_t *act_b) {
    orc_seg *buf = NULL;
    int64_t cap = 0;
    int64_t n = ray_segments(s, cd, o, d, &buf, &cap);
    for (int64_t k = 0; k < n && k < maxn; k++) {
        cell[k] = buf[k].cell;
        ta[k] = buf[k].ta;
        tb[k] = buf[k].tb;
        act_a[k] = buf[k].act_a;
        act_b[k] = buf[k].act_b;
    }
    free(buf);
    return n;
}

/* exported for the tests: colour of cell i for an explicit segment */
void orc_cell_colour(const orc_scene *s, int64_t i, const double *o, const double *d, double ta, double tb,
                     double kappa, double *col) {
    orc_seg sg = {(int32_t)i, ta, tb, ACT_SPHERE, ACT_SPHERE};
    cell_colour(s, i, o, d, &sg, kappa, col, NULL, NULL, NULL);
}

static void pixel_of(const orc_camera *cam, int64_t k, const int32_t *pix, double *u, double *v) {
    if (pix) {
        *u = pix[2 * k];
        *v = pix[2 * k + 1];
    } else {
        *u = (double)(k % cam->width);
        *v = (double)(k / cam->width);
    }
}

/* composite one ray: C = sum_k T_k alpha_k c_k over its sorted segments */
static int64_t render_ray(const orc_scene *s, const orc_cands *cd, const double *o, const double *d, double kappa,
                          orc_seg **buf, int64_t *cap, double *C, double *Tout) {
    int64_t n = ray_segments(s, cd, o, d, buf, cap);
    double T = 1.0;
    C[0] = C[1] = C[2] = 0.0;
    for (int64_t q = 0; q < n; q++) {
        int64_t i = (*buf)[q].cell;
        double l = (*buf)[q].tb - (*buf)[q].ta;
        double surv = exp(-s->sigma[i] * l);
        double alpha = 1.0 - surv;
        double col[3];
        cell_colour(s, i, o, d, &(*buf)[q], kappa, col, NULL, NULL, NULL);
        for (int ch = 0; ch < 3; ch++) C[ch] += T * alpha * col[ch];
        T *= surv;
    }
    *Tout = T;
    return n;
}

/* explicit rays: o [n][3], d [n][3] (unit) */
int orc_render_rays(const orc_scene *s, const orc_cands *cd, int64_t nray, const double *o, const double *d,
                    double kappa, double *out_rgb, double *out_T) {
    orc_seg *buf = NULL;
    int64_t cap = 0;
    for (int64_t k = 0; k < nray; k++) render_ray(s, cd, &o[3 * k], &d[3 * k], kappa, &buf, &cap, &out_rgb[3 * k], &out_T[k]);
    free(buf);
    return 0;
}

/*
 * Render npix pixels (pix = [npix][2] (u, v) or NULL for the whole image in
 * row-major order).  out_rgb [npix][3], out_T [npix], out_nseg [npix] (nullable).
 */
int orc_render(const orc_scene *s, const orc_cands *cd, const orc_camera *cam, int64_t npix, const int32_t *pix,
               double kappa, double *out_rgb, double *out_T, int32_t *out_nseg, int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
    {
        orc_seg *buf = NULL;
        int64_t cap = 0;
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int64_t k = 0; k < npix; k++) {
            double u, v, o[3], d[3];
            pixel_of(cam, k, pix, &u, &v);
            double T = 1.0, C[3] = {0.0, 0.0, 0.0};
            int64_t n = 0;
            if (orc_ray(cam, u, v, o, d)) n = render_ray(s, cd, o, d, kappa, &buf, &cap, C, &T);
            for (int ch = 0; ch < 3; ch++) out_rgb[3 * k + ch] = C[ch];
            out_T[k] = T;
            if (out_nseg) out_nseg[k] = (int32_t)n;
        }
        free(buf);
    }
    return 0;
}

/*
 * Per-cell contributions over npix pixels (Sec. 4 training terms): with
 * T_k the transmittance in front of the cell's segment k on a ray and
 * alpha_k its opacity,
 *   sparse[i] = sum over rays of T_k alpha_k                   (L_sparse)
 *   normal[i] = sum over rays of T_k alpha_k max(nh_i . d, 0)^2 (L_normal)
 * accumulated over the same composited segments as orc_render.
 */
int orc_cell_contrib(const orc_scene *s, const orc_cands *cd, const orc_camera *cam, int64_t npix, const int32_t *pix,
                double *sparse, double *normal, int nthreads) {
    memset(sparse, 0, sizeof(double) * (size_t)s->n);
    memset(normal, 0, sizeof(double) * (size_t)s->n);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
    {
        orc_seg *buf = NULL;
        int64_t cap = 0;
        double *ls = calloc((size_t)s->n, sizeof(double)), *ln = calloc((size_t)s->n, sizeof(double));
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int64_t k = 0; k < npix; k++) {
            double u, v, o[3], d[3];
            pixel_of(cam, k, pix, &u, &v);
            if (!orc_ray(cam, u, v, o, d)) continue;
            int64_t n = ray_segments(s, cd, o, d, &buf, &cap);
            double T = 1.0;
            for (int64_t q = 0; q < n; q++) {
                int64_t i = buf[q].cell;
                double surv = exp(-s->sigma[i] * (buf[q].tb - buf[q].ta));
                double w = T * (1.0 - surv);
                double nh[3], len;
                unit_normal(s, i, nh, &len);
                double nd = dot3(nh, d);
                ls[i] += w;
                ln[i] += w * (nd > 0.0 ? nd * nd : 0.0);
                T *= surv;
            }
        }
#ifdef _OPENMP
#pragma omp critical
#endif
        for (int64_t i = 0; i < s->n; i++) {
            sparse[i] += ls[i];
            normal[i] += ln[i];
        }
        free(ls);
        free(ln);
        free(buf);
    }
    return 0;
}

/* cells whose bounding sphere the given pixels' rays meet at t >= 0 (flag per cell) */
int orc_hit_cells(const orc_scene *s, const orc_camera *cam, int64_t npix, const int32_t *pix, uint8_t *flag,
                  int nthreads) {
    memset(flag, 0, (size_t)s->n);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int64_t i = 0; i < s->n; i++) {
        double p[3], m[3];
        load3(s->pos, i, p);
        double R = s->R[i];
        for (int64_t k = 0; k < npix; k++) {
            double u, v, o[3], d[3];
            pixel_of(cam, k, pix, &u, &v);
            if (!orc_ray(cam, u, v, o, d)) continue;
            for (int r = 0; r < 3; r++) m[r] = o[r] - p[r];
            double b = dot3(m, d), c = dot3(m, m) - R * R;
            double disc = b * b - c;
            /* widened: a ray passing within ~1e-6 R of the sphere also counts */
            if (disc >= -1e-12 * R * R && -b + sqrt(fabs(disc)) >= -1e-6 * R) {
                flag[i] = 1;
                break;
            }
        }
    }
    return 0;
}

/*
 * Accumulate d t_end / d(params) * g into the per-pixel contribution list,
 * for the constraint `act` active at ray parameter t.
 * Parameter columns (25 per cell): pos 0-2, w 3, R 4, sigma 5, rgb 6-8,
 * normal 9-11, offset 12, tex 13-24.
 */
/* gradient columns; the site blocks have room for eight sites (tex 24, disp 8,
 * sites 16, sv 384), a four-site scene uses the first half of each */
enum { P_POS = 0, P_W = 3, P_R = 4, P_SIG = 5, P_RGB = 6, P_N = 9, P_OFF = 12, P_TEX = 13, P_DISP = 37, P_SITE = 45,
       P_SV = 61, NPAR = 445 };

typedef struct {
    int32_t cell, col;
    double v;
} orc_contrib;

typedef struct {
    orc_contrib *c;
    int64_t n, cap;
} clist;

static void push(clist *L, int32_t cell, int col, double v) {
    if (v == 0.0) return;
    if (L->n == L->cap) {
        L->cap = L->cap ? 2 * L->cap : 256;
        L->c = realloc(L->c, (size_t)L->cap * sizeof(orc_contrib));
    }
    L->c[L->n].cell = cell;
    L->c[L->n].col = col;
    L->c[L->n].v = v;
    L->n++;
}

/*
 * dL/dt for a segment end on the face of cell i at t:
 * F = nh.(x - p) - off - delta = 0 gives dt/dp = nh/(nh.d),
 * dt/doff = dt/ddelta = 1/(nh.d), dt/dnh = -(x - p)/(nh.d) at fixed delta.
 * With displacement, delta (see face_disp) depends on disp_k through W_k,
 * and on p, R and nh through u at the base crossing tbar, which itself
 * moves like a face end without displacement.
 */
static void route_face(const orc_scene *s, int64_t i, double t, const double *o, const double *d, double g,
                       clist *L, int with_disp) {
    double nh[3], nl, p[3], y[3];
    unit_normal(s, i, nh, &nl);
    load3(s->pos, i, p);
    for (int r = 0; r < 3; r++) y[r] = o[r] + t * d[r] - p[r];
    double nd = dot3(nh, d);
    double gnh[3];
    for (int r = 0; r < 3; r++) {
        push(L, (int32_t)i, P_POS + r, g * nh[r] / nd);
        gnh[r] = -g * y[r] / nd;
    }
    push(L, (int32_t)i, P_OFF, g / nd);
    if (with_disp && s->disp && nd != 0.0) {
        double W[MAXS], u[2], tb;
        double delta = face_disp(s, i, o, d, W, u, &tb);
        double gd = g / nd; /* dL/ddelta */
        double gu[2] = {0.0, 0.0};
        for (int k = 0; k < nsites(s); k++) {
            push(L, (int32_t)i, P_DISP + k, gd * W[k]);
            /* d delta / d u = sum_k W_k (disp_k - delta) d lg_k / du,  lg_k = -kappa |u - s_k| */
            double dx = u[0] - site_x(s, i, k), dy = u[1] - site_y(s, i, k);
            double rr = sqrt(dx * dx + dy * dy);
            if (rr > 0.0) {
                double c = gd * W[k] * (s->disp[(int64_t)nsites(s) * i + k] - delta) * (-s->kappa_disp) / rr;
                gu[0] += c * dx;
                gu[1] += c * dy;
                /* the logit depends on u - s_k: the site moves opposite to u */
                if (s->sites) {
                    push(L, (int32_t)i, P_SITE + 2 * k, -c * dx);
                    push(L, (int32_t)i, P_SITE + 2 * k + 1, -c * dy);
                }
            }
        }
        /* u = (e1.yb, e2.yb)/R, yb = o + tbar d - p */
        double e1[3], e2[3], J1[9], J2[9], yb[3], gy[3];
        onb(nh, e1, e2, J1, J2);
        double R = s->R[i];
        for (int r = 0; r < 3; r++) yb[r] = o[r] + tb * d[r] - p[r];
        for (int r = 0; r < 3; r++) gy[r] = (gu[0] * e1[r] + gu[1] * e2[r]) / R;
        for (int r = 0; r < 3; r++) push(L, (int32_t)i, P_POS + r, -gy[r]);
        push(L, (int32_t)i, P_R, -(gu[0] * u[0] + gu[1] * u[1]) / R);
        for (int c = 0; c < 3; c++)
            for (int r = 0; r < 3; r++)
                gnh[c] += J1[3 * r + c] * gu[0] * yb[r] / R + J2[3 * r + c] * gu[1] * yb[r] / R;
        /* the base crossing moves with the base face */
        route_face(s, i, tb, o, d, dot3(gy, d), L, 0);
    }
    /* nh = n/|n|:  dL/dn = (I - nh nh^T) dL/dnh / |n| */
    double pr = dot3(nh, gnh);
    for (int r = 0; r < 3; r++) push(L, (int32_t)i, P_N + r, (gnh[r] - nh[r] * pr) / nl);
}

/* dL/dt for the end of a segment given by constraint act on cell i */
static void route_t(const orc_scene *s, int64_t i, int act, double t, const double *o, const double *d, double g,
                    clist *L) {
    if (g == 0.0 || act == ACT_CAMERA) return;
    double p[3], x[3], y[3];
    load3(s->pos, i, p);
    for (int r = 0; r < 3; r++) {
        x[r] = o[r] + t * d[r];
        y[r] = x[r] - p[r];
    }
    if (act == ACT_SPHERE) {
        /* F = |x - p|^2 - R^2 = 0:  dt/dp = y/(y.d), dt/dR = R/(y.d) */
        double yd = dot3(y, d);
        for (int r = 0; r < 3; r++) push(L, (int32_t)i, P_POS + r, g * y[r] / yd);
        push(L, (int32_t)i, P_R, g * (double)s->R[i] / yd);
    } else if (act == ACT_DIPOLE) {
        route_face(s, i, t, o, d, g, L, 1);
    } else {
        /* F = 2 x.(p_j - p_i) - |p_j|^2 + |p_i|^2 - w_i + w_j
         * dF/dt = 2 d.(p_j - p_i), dF/dp_i = -2(x - p_i), dF/dp_j = 2(x - p_j),
         * dF/dw_i = -1, dF/dw_j = 1  ->  dt/dtheta = -dF/dtheta / dF/dt */
        int64_t j = act;
        double pj[3], a[3];
        load3(s->pos, j, pj);
        for (int r = 0; r < 3; r++) a[r] = pj[r] - p[r];
        double Ft = 2.0 * dot3(d, a);
        for (int r = 0; r < 3; r++) {
            push(L, (int32_t)i, P_POS + r, g * (2.0 * (x[r] - p[r])) / Ft);
            push(L, (int32_t)j, P_POS + r, g * (-2.0 * (x[r] - pj[r])) / Ft);
        }
        push(L, (int32_t)i, P_W, g * 1.0 / Ft);
        push(L, (int32_t)j, P_W, g * -1.0 / Ft);
    }
}

/*
 * Gradient of L with respect to every cell parameter, given dL/dC [npix][3]
 * and dL/dT_final [npix] for the rendered pixels.  grad [n][229] is
 * overwritten.  Contributions are summed in pixel order, so the result does
 * not depend on the thread count.
 */
int orc_render_grad(const orc_scene *s, const orc_cands *cd, const orc_camera *cam, int64_t npix, const int32_t *pix,
                    double kappa, const double *dL_dC, const double *dL_dT, double *grad, int nthreads) {
    clist *lists = calloc((size_t)npix, sizeof(clist));
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
    {
        orc_seg *buf = NULL;
        int64_t cap = 0;
        double *alpha = NULL, *surv = NULL, *Tin = NULL, *col = NULL;
        int64_t acap = 0;
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int64_t k = 0; k < npix; k++) {
            double u, v, o[3], d[3];
            pixel_of(cam, k, pix, &u, &v);
            if (!orc_ray(cam, u, v, o, d)) continue;
            int64_t n = ray_segments(s, cd, o, d, &buf, &cap);
            if (n > acap) {
                acap = n;
                alpha = realloc(alpha, (size_t)n * sizeof(double));
                surv = realloc(surv, (size_t)n * sizeof(double));
                Tin = realloc(Tin, (size_t)n * sizeof(double));
                col = realloc(col, (size_t)n * 3 * sizeof(double));
            }
            double T = 1.0;
            for (int64_t q = 0; q < n; q++) {
                int64_t i = buf[q].cell;
                double l = buf[q].tb - buf[q].ta;
                surv[q] = exp(-(double)s->sigma[i] * l);
                alpha[q] = 1.0 - surv[q];
                Tin[q] = T;
                cell_colour(s, i, o, d, &buf[q], kappa, &col[3 * q], NULL, NULL, NULL);
                T *= surv[q];
            }
            double Tf = T;
            const double *gC = &dL_dC[3 * k];
            double gT = dL_dT[k];
            clist *L = &lists[k];
            /* S = sum over segments behind q of T_j alpha_j c_j */
            double S[3] = {0, 0, 0};
            for (int64_t q = n - 1; q >= 0; q--) {
                int64_t i = buf[q].cell;
                double sig = s->sigma[i];
                double l = buf[q].tb - buf[q].ta;
                double Tout = Tin[q] * surv[q];
                /* x = sigma l, alpha = 1 - e^-x:
                 * dL/dx = gC.(T_{q+1} c_q - S_q) - gT T_final */
                double dLdx = -gT * Tf;
                for (int ch = 0; ch < 3; ch++) dLdx += gC[ch] * (Tout * col[3 * q + ch] - S[ch]);
                push(L, (int32_t)i, P_SIG, dLdx * l);
                double gl = dLdx * sig;
                /* colour: dL/dc = T alpha gC */
                double wc = Tin[q] * alpha[q];
                double gc[3] = {wc * gC[0], wc * gC[1], wc * gC[2]};
                double W[MAXS], uu[2], ts;
                const int ns = nsites(s);
                double cc[3];
                cell_colour(s, i, o, d, &buf[q], kappa, cc, W, uu, &ts);
                for (int ch = 0; ch < 3; ch++) push(L, (int32_t)i, P_RGB + ch, gc[ch]);
                /* site colours: constant (tex), or view dependent (spherical Voronoi) */
                double gW[MAXS], sW = 0.0;
                for (int kk = 0; kk < ns; kk++) {
                    gW[kk] = 0.0;
                    if (!s->sv) {
                        for (int ch = 0; ch < 3; ch++) {
                            push(L, (int32_t)i, P_TEX + 3 * kk + ch, W[kk] * gc[ch]);
                            gW[kk] += (double)s->tex[3 * ns * i + 3 * kk + ch] * gc[ch];
                        }
                    } else {
                        /* c_k = sum_j P_j c_j, P = softmax(lambda a_j.wo / |a_j|), wo = -d */
                        double ck[3], P[8], gP[8], sP = 0.0;
                        const double *qv = s->sv + (((int64_t)i * ns + kk) * 8) * 6;
                        const int base = P_SV + kk * 48;
                        sv_colour(s, i, kk, d, ck, P);
                        for (int ch = 0; ch < 3; ch++) gW[kk] += ck[ch] * gc[ch];
                        for (int j = 0; j < 8; j++) {
                            gP[j] = 0.0;
                            for (int ch = 0; ch < 3; ch++) {
                                double gck = W[kk] * gc[ch];
                                push(L, (int32_t)i, base + 6 * j + 3 + ch, P[j] * gck);
                                gP[j] += gck * qv[6 * j + 3 + ch];
                            }
                            sP += P[j] * gP[j];
                        }
                        for (int j = 0; j < 8; j++) {
                            double glg = P[j] * (gP[j] - sP);   /* dL/dlogit_j */
                            const double *a = qv + 6 * j;
                            double La = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
                            double ah[3] = {a[0] / La, a[1] / La, a[2] / La};
                            double ga[3] = {-glg * s->sv_lambda * d[0], -glg * s->sv_lambda * d[1],
                                            -glg * s->sv_lambda * d[2]};   /* dL/d(a hat), wo = -d */
                            double pa = dot3(ah, ga);
                            for (int r = 0; r < 3; r++) push(L, (int32_t)i, base + 6 * j + r, (ga[r] - ah[r] * pa) / La);
                        }
                    }
                    sW += W[kk] * gW[kk];
                }
                double gu[2] = {0.0, 0.0};
                for (int kk = 0; kk < ns; kk++) {
                    double glog = W[kk] * (gW[kk] - sW);          /* dL/dlogit */
                    double dx = uu[0] - site_x(s, i, kk), dy = uu[1] - site_y(s, i, kk);
                    double r = sqrt(dx * dx + dy * dy);
                    if (r > 0.0) {
                        double gr = -kappa * glog;                  /* logit = -kappa r */
                        gu[0] += gr * dx / r;
                        gu[1] += gr * dy / r;
                        if (s->sites) {                             /* r = |u - s_k| */
                            push(L, (int32_t)i, P_SITE + 2 * kk, -gr * dx / r);
                            push(L, (int32_t)i, P_SITE + 2 * kk + 1, -gr * dy / r);
                        }
                    }
                }
                /* u = (e1.y_s, e2.y_s)/R, y_s = o + ts d - p */
                double nh[3], nl, e1[3], e2[3], J1[9], J2[9], p[3], ys[3];
                unit_normal(s, i, nh, &nl);
                onb(nh, e1, e2, J1, J2);
                load3(s->pos, i, p);
                for (int r = 0; r < 3; r++) ys[r] = o[r] + ts * d[r] - p[r];
                double R = s->R[i];
                double gy[3];
                for (int r = 0; r < 3; r++) gy[r] = (gu[0] * e1[r] + gu[1] * e2[r]) / R;
                for (int r = 0; r < 3; r++) push(L, (int32_t)i, P_POS + r, -gy[r]);
                push(L, (int32_t)i, P_R, -(gu[0] * uu[0] + gu[1] * uu[1]) / R);
                /* through the frame: dL/de1 = gu0 y/R, dL/dnh = J1^T dL/de1 + J2^T dL/de2 */
                double gnh[3] = {0, 0, 0};
                for (int c = 0; c < 3; c++)
                    for (int r = 0; r < 3; r++)
                        gnh[c] += J1[3 * r + c] * gu[0] * ys[r] / R + J2[3 * r + c] * gu[1] * ys[r] / R;
                double pr = dot3(nh, gnh);
                for (int r = 0; r < 3; r++) push(L, (int32_t)i, P_N + r, (gnh[r] - nh[r] * pr) / nl);
                /* the texture point moves with its segment end */
                double gts = dot3(gy, d);
                int on_b = (dot3(nh, d) > 0.0);
                double gta = -gl + (on_b ? 0.0 : gts);
                double gtb = gl + (on_b ? gts : 0.0);
                route_t(s, i, buf[q].act_a, buf[q].ta, o, d, gta, L);
                route_t(s, i, buf[q].act_b, buf[q].tb, o, d, gtb, L);
                for (int ch = 0; ch < 3; ch++) S[ch] += Tin[q] * alpha[q] * col[3 * q + ch];
            }
        }
        free(buf);
        free(alpha);
        free(surv);
        free(Tin);
        free(col);
    }
    memset(grad, 0, (size_t)s->n * NPAR * sizeof(double));
    for (int64_t k = 0; k < npix; k++) {
        for (int64_t q = 0; q < lists[k].n; q++) {
            orc_contrib *c = &lists[k].c[q];
            grad[(int64_t)c->cell * NPAR + c->col] += c->v;
        }
        free(lists[k].c);
    }
    free(lists);
    return 0;
}

/* ------------------------------------------------------------------------
 * CPU binning: which 16x16 tiles each cell's bounding sphere can touch, and
 * the painter key pow(o, p_i) (Sec. 3.2; Thm. power_painter orders cells by
 * the power distance of the camera centre).
 *
 * The rectangle is the image-plane bounding box of the projected sphere
 * (the tangent lines from the camera centre in the x-z and y-z planes,
 * slopes (X Z -+ r sqrt(X^2 + Z^2 - r^2)) / (Z^2 - r^2)), clipped to the
 * image.  For a centre at camera depth Z > 2 r it is evaluated in float from
 * X, Y, Z rounded to float and widened by e = 2^-18 (|f| (|X| / Z + 1) + |c|)
 * pixels per axis (twice a bound on that evaluation's rounding error, about
 * 32 ulps of those magnitudes); nearer spheres take the same box in double,
 * widened by 1e-6 px.  A sphere that reaches the plane z = 0 gets the whole
 * image unless it lies entirely outside a side plane of the view frustum.
 * Every step is one IEEE operation, in the order written (the library
 * evaluates the same rule), so the tile sets can be compared bit for bit.
 * ------------------------------------------------------------------------ */
#define ORC_TILE 16

static double orc_ceil(double x) { return ceil(x); }
static double orc_floor(double x) { return floor(x); }

/* widening of one edge of the float box (pixels): 2^-17 (|f| ((1 + k^2) L1z + az) + |c0|) */
static float orc_box_margin(float f, float c0, float k, float L1z, float az) {
    return 0x1p-17f * (fabsf(f) * ((1.0f + k * k) * L1z + az) + fabsf(c0));
}

/* rect[4] = {tx0, ty0, tx1, ty1} (empty: tx0 > tx1), key = order-preserving bits of pow */
void orc_bin_cell(const orc_camera *cam, const double *pos, const double *w, const double *R, int64_t i,
                  int32_t *rect, uint64_t *key) {
    double px = pos[3 * i], py = pos[3 * i + 1], pz = pos[3 * i + 2];
    double dx = px - cam->origin[0];
    double dy = py - cam->origin[1];
    double dz = pz - cam->origin[2];
    double pw = ((dx * dx + dy * dy) + dz * dz) - (double)w[i];
    uint64_t bits;
    memcpy(&bits, &pw, 8);
    *key = (bits >> 63) ? ~bits : (bits | 0x8000000000000000ULL);

    rect[0] = 1;
    rect[1] = 1;
    rect[2] = 0;
    rect[3] = 0;
    double W = cam->width, H = cam->height;
    double ulo = -INFINITY, uhi = INFINITY, vlo = -INFINITY, vhi = INFINITY;
    double a0, a1, b0, b1;
    {
        /* m = o - p as a float pair (two-sum of the origin's float high part
         * and -p, plus its low part), then the camera-frame centre in float */
        float hm[3];
        for (int c = 0; c < 3; c++) {
            float p = (float)pos[3 * i + c];
            float a = (float)cam->origin[c];
            float ol = (float)(cam->origin[c] - (double)a);
            float s0 = a - p;
            float bb = s0 - a;
            float e0 = (a - (s0 - bb)) + (-p - bb);
            float t0 = e0 + ol;
            hm[c] = s0 + t0;
        }
        float Mf[9];
        for (int k = 0; k < 9; k++) Mf[k] = (float)cam->rot[k];
        float Xf = -((Mf[0] * hm[0] + Mf[1] * hm[1]) + Mf[2] * hm[2]);
        float Yf = -((Mf[3] * hm[0] + Mf[4] * hm[1]) + Mf[5] * hm[2]);
        float Zf = -((Mf[6] * hm[0] + Mf[7] * hm[1]) + Mf[8] * hm[2]);
        float rf = (float)R[i];
        if (Zf > 2.0f * rf && Zf * 1024.0f > fabsf(Xf) + fabsf(Yf)) {
            /* well in front, within 89.9 degrees of the axis: the box in
             * float, each edge widened by a bound on its rounding error */
            float fxf = (float)cam->fx, fyf = (float)cam->fy, cxf = (float)cam->cx, cyf = (float)cam->cy;
            float rr = rf * rf, zz = Zf * Zf;
            float izr = 1.0f / (zz - rr);
            float sx = sqrtf((Xf * Xf + zz) - rr);
            float sy = sqrtf((Yf * Yf + zz) - rr);
            float xz = Xf * Zf, yz = Yf * Zf;
            float rsx = rf * sx, rsy = rf * sy;
            float kxl = (xz - rsx) * izr, kxh = (xz + rsx) * izr;
            float kyl = (yz - rsy) * izr, kyh = (yz + rsy) * izr;
            float L1z = ((fabsf(Xf) + fabsf(Yf)) + Zf) / Zf;
            float axz = fabsf(Xf) / Zf + 1.0f, ayz = fabsf(Yf) / Zf + 1.0f;
            a0 = ceilf(((fxf * kxl + cxf) - 0.5f) - orc_box_margin(fxf, cxf, kxl, L1z, axz));
            a1 = floorf(((fxf * kxh + cxf) - 0.5f) + orc_box_margin(fxf, cxf, kxh, L1z, axz));
            b0 = ceilf(((fyf * kyl + cyf) - 0.5f) - orc_box_margin(fyf, cyf, kyl, L1z, ayz));
            b1 = floorf(((fyf * kyh + cyf) - 0.5f) + orc_box_margin(fyf, cyf, kyh, L1z, ayz));
            goto clip;
        }
    }
    const double *M = cam->rot;
    double X = (M[0] * dx + M[1] * dy) + M[2] * dz;
    double Y = (M[3] * dx + M[4] * dy) + M[5] * dz;
    double Z = (M[6] * dx + M[7] * dy) + M[8] * dz;
    double r = R[i];
    if (Z + r <= 0.0) return; /* entirely behind the camera */
    if (Z > r) {
        /* tangent lines from the camera centre to the sphere's x-z and y-z circles */
        double rr = r * r;
        double izr = 1.0 / (Z * Z - rr);
        double sx = sqrt((X * X + Z * Z) - rr);
        double sy = sqrt((Y * Y + Z * Z) - rr);
        double kxl = (X * Z - r * sx) * izr, kxh = (X * Z + r * sx) * izr;
        double kyl = (Y * Z - r * sy) * izr, kyh = (Y * Z + r * sy) * izr;
        ulo = cam->fx * kxl + cam->cx;
        uhi = cam->fx * kxh + cam->cx;
        vlo = cam->fy * kyl + cam->cy;
        vhi = cam->fy * kyh + cam->cy;
    } else {
        /* reaches z <= 0: whole image unless entirely outside a side plane
         * x = k z of the frustum (through the camera centre) */
        double kl = (0.0 - cam->cx) / cam->fx, kr = (W - cam->cx) / cam->fx;
        double ku = (0.0 - cam->cy) / cam->fy, kd = (H - cam->cy) / cam->fy;
        if (X - kr * Z > r * sqrt(1.0 + kr * kr)) return;
        if (kl * Z - X > r * sqrt(1.0 + kl * kl)) return;
        if (Y - kd * Z > r * sqrt(1.0 + kd * kd)) return;
        if (ku * Z - Y > r * sqrt(1.0 + ku * ku)) return;
    }
    /* pixel centres u + 0.5 inside [ulo, uhi], widened by 1e-6 px */
    a0 = orc_ceil((ulo - 0.5) - 1e-6);
    a1 = orc_floor((uhi - 0.5) + 1e-6);
    b0 = orc_ceil((vlo - 0.5) - 1e-6);
    b1 = orc_floor((vhi - 0.5) + 1e-6);
clip:
    if (a0 < 0.0) a0 = 0.0;
    if (b0 < 0.0) b0 = 0.0;
    if (a1 > W - 1.0) a1 = W - 1.0;
    if (b1 > H - 1.0) b1 = H - 1.0;
    if (a0 > a1 || b0 > b1) return;
    rect[0] = (int32_t)a0 / ORC_TILE;
    rect[1] = (int32_t)b0 / ORC_TILE;
    rect[2] = (int32_t)a1 / ORC_TILE;
    rect[3] = (int32_t)b1 / ORC_TILE;
}

int orc_bin(const orc_camera *cam, int64_t n, const double *pos, const double *w, const double *R, int32_t *rect,
            uint64_t *key) {
    for (int64_t i = 0; i < n; i++) orc_bin_cell(cam, pos, w, R, i, &rect[4 * i], &key[i]);
    return 0;
}

/*
 * Neighbour lists (the radical planes of Sec. 3.2, Eq. power_bisector, read
 * as above): the signed distance from p_i of the plane between sites i and j
 * is t_ij = (|a|^2 + w_i - w_j) / (2|a|), a = p_j - p_i (no plane when
 * a = 0).  For each listed cell i: the K sites j != i with the smallest
 * t_ij, ascending, equal values by ascending j, -1 after the last; and the
 * bound radius, clipped to the largest float <= max(t_(K+1), 0) when the
 * (K+1)-th smallest value t_(K+1) is below R_i (every site left out then
 * has its plane outside the sphere).  Brute force over all sites; t in
 * double from the float inputs as written, left to right, no contraction.
 * cells: NULL for all n cells in order, else ncells indices; nbr
 * [ncells][k], R_out [ncells].
 */
int orc_neighbours(const float *pos, const float *w, const float *R, int64_t n, int32_t k, int64_t ncells,
                   const int64_t *cells, int32_t *nbr, float *R_out, int nthreads) {
    if (k < 0) return -1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
    {
        double *bt = malloc(((size_t)k + 1) * sizeof(double));
        int64_t *bj = malloc(((size_t)k + 1) * sizeof(int64_t));
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 16)
#endif
        for (int64_t q = 0; q < ncells; q++) {
            const int64_t i = cells ? cells[q] : q;
            int m = 0;
            for (int64_t j = 0; j < n; j++) {
                if (j == i) continue;
                double dx = (double)pos[3 * j] - (double)pos[3 * i];
                double dy = (double)pos[3 * j + 1] - (double)pos[3 * i + 1];
                double dz = (double)pos[3 * j + 2] - (double)pos[3 * i + 2];
                double L2 = dx * dx + dy * dy + dz * dz;
                if (!(L2 > 0.0)) continue;
                double L = sqrt(L2);
                double t = (L2 + (double)w[i] - (double)w[j]) / (2.0 * L);
                if (!(t < INFINITY)) continue;
                /* keep the k+1 smallest (t, j) in ascending order */
                if (m == k + 1 && !(t < bt[k] || (t == bt[k] && j < bj[k]))) continue;
                int p = m < k + 1 ? m++ : k;
                while (p > 0 && (bt[p - 1] > t || (bt[p - 1] == t && bj[p - 1] > j))) {
                    bt[p] = bt[p - 1];
                    bj[p] = bj[p - 1];
                    p--;
                }
                bt[p] = t;
                bj[p] = j;
            }
            for (int r = 0; r < k; r++) nbr[q * k + r] = r < m ? (int32_t)bj[r] : -1;
            double tk1 = m == k + 1 ? bt[k] : INFINITY;
            float Ri = R[i];
            if (tk1 < (double)Ri) {
                double x = tk1 > 0.0 ? tk1 : 0.0;
                float f = (float)x;
                if ((double)f > x) f = nextafterf(f, 0.0f);
                R_out[q] = f;
            } else {
                R_out[q] = Ri;
            }
        }
        free(bt);
        free(bj);
    }
    return 0;
}

/*
 * Gradient of L = sum_i (ws_i sparse_i + wn_i normal_i), the per-cell
 * contributions of orc_cell_contrib (Sec. 4's L_sparse and L_normal with
 * per-cell weights), with respect to every cell parameter.  Along one ray
 * the contributions composite the scalar c_k = ws_i + wn_i max(nh.d, 0)^2 of
 * each segment: L_ray = sum_k T_k alpha_k c_k.  So, as in the colour adjoint,
 * dL/dx_k (x = sigma l) = T_{k+1} c_k - S_k with S_k the part of the sum
 * behind segment k, routed to the segment ends; and c_k moves with the unit
 * normal: dc/dnh = 2 wn max(nh.d, 0) d.  grad [n][NPAR] is overwritten;
 * contributions are summed in pixel order.
 */
int orc_contrib_grad(const orc_scene *s, const orc_cands *cd, const orc_camera *cam, int64_t npix, const int32_t *pix,
                     const double *ws, const double *wn, double *grad, int nthreads) {
    clist *lists = calloc((size_t)npix, sizeof(clist));
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
    {
        orc_seg *buf = NULL;
        int64_t cap = 0;
        double *alpha = NULL, *Tin = NULL, *cv = NULL;
        int64_t acap = 0;
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int64_t k = 0; k < npix; k++) {
            double u, v, o[3], d[3];
            pixel_of(cam, k, pix, &u, &v);
            if (!orc_ray(cam, u, v, o, d)) continue;
            int64_t n = ray_segments(s, cd, o, d, &buf, &cap);
            if (n > acap) {
                acap = n;
                alpha = realloc(alpha, (size_t)n * sizeof(double));
                Tin = realloc(Tin, (size_t)n * sizeof(double));
                cv = realloc(cv, (size_t)n * sizeof(double));
            }
            double T = 1.0;
            for (int64_t q = 0; q < n; q++) {
                int64_t i = buf[q].cell;
                double nh[3], nl;
                unit_normal(s, i, nh, &nl);
                double nd = dot3(nh, d);
                alpha[q] = 1.0 - exp(-(double)s->sigma[i] * (buf[q].tb - buf[q].ta));
                Tin[q] = T;
                cv[q] = ws[i] + wn[i] * (nd > 0.0 ? nd * nd : 0.0);
                T *= 1.0 - alpha[q];
            }
            clist *L = &lists[k];
            double S = 0.0;
            for (int64_t q = n - 1; q >= 0; q--) {
                int64_t i = buf[q].cell;
                double sig = s->sigma[i];
                double l = buf[q].tb - buf[q].ta;
                double Tout = Tin[q] * (1.0 - alpha[q]);
                double dLdx = Tout * cv[q] - S;
                push(L, (int32_t)i, P_SIG, dLdx * l);
                double gl = dLdx * sig;
                route_t(s, i, buf[q].act_a, buf[q].ta, o, d, -gl, L);
                route_t(s, i, buf[q].act_b, buf[q].tb, o, d, gl, L);
                /* the normal-loss weight: dc/dnh = 2 wn (nh.d) d where nh.d > 0; n = |n| nh */
                double nh[3], nl;
                unit_normal(s, i, nh, &nl);
                double nd = dot3(nh, d);
                if (nd > 0.0 && wn[i] != 0.0) {
                    double f = Tin[q] * alpha[q] * 2.0 * wn[i] * nd;
                    double gnh[3] = {f * d[0], f * d[1], f * d[2]};
                    double pr = dot3(nh, gnh);
                    for (int r = 0; r < 3; r++) push(L, (int32_t)i, P_N + r, (gnh[r] - nh[r] * pr) / nl);
                }
                S += Tin[q] * alpha[q] * cv[q];
            }
        }
        free(buf);
        free(alpha);
        free(Tin);
        free(cv);
    }
    memset(grad, 0, (size_t)s->n * NPAR * sizeof(double));
    for (int64_t k = 0; k < npix; k++) {
        for (int64_t q = 0; q < lists[k].n; q++) {
            orc_contrib *c = &lists[k].c[q];
            grad[(int64_t)c->cell * NPAR + c->col] += c->v;
        }
        free(lists[k].c);
    }
    free(lists);
    return 0;
}

/*
 * Full-frame renderer over per-tile lists (the CPU counterpart of the tiled
 * renderer, Sec. 3.4): every pixel of a tile walks the tile's cell list in
 * the given order (the painter order of Sec. 3.4: ascending power distance
 * from the camera centre, then cell index), clips each listed cell's ray
 * segment against that cell's candidates (its K neighbour list when `cd`
 * holds one), and composites the non-empty segments in list order:
 *   C = sum_k T_k alpha_k c_k,  T_{k+1} = T_k (1 - alpha_k).
 * A ray stops once T < t_stop (t_stop = 0: never).  In a power diagram the
 * segments of one ray are disjoint and the painter order is their order
 * along the ray, so with complete lists this equals orc_render.
 *
 * tile_start [ntx*nty+1], tile_cells: CSR lists, tile t = ty*ntx + tx of
 * ORC_TILE x ORC_TILE pixels.  tiles: ntile indices to render (NULL: all).
 * out_rgb [H*W][3], out_T [H*W], out_nseg [H*W] (nullable): row-major,
 * written for the pixels of the rendered tiles only.  OpenMP over tiles.
 */
int orc_render_tiles(const orc_scene *s, const orc_cands *cd, const orc_camera *cam, const int64_t *tile_start,
                     const int32_t *tile_cells, int64_t ntile, const int32_t *tiles, double kappa, double t_stop,
                     double *out_rgb, double *out_T, int32_t *out_nseg, int nthreads) {
    const int64_t ntx = (cam->width + ORC_TILE - 1) / ORC_TILE;
    const int64_t nty = (cam->height + ORC_TILE - 1) / ORC_TILE;
    if (!tiles) ntile = ntx * nty;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t q = 0; q < ntile; q++) {
        const int64_t t = tiles ? (int64_t)tiles[q] : q;
        if (t < 0 || t >= ntx * nty) continue;
        const int64_t tx = t % ntx, ty = t / ntx;
        for (int64_t v = ty * ORC_TILE; v < (ty + 1) * ORC_TILE && v < cam->height; v++) {
            for (int64_t u = tx * ORC_TILE; u < (tx + 1) * ORC_TILE && u < cam->width; u++) {
                const int64_t k = v * cam->width + u;
                double o[3], d[3], C[3] = {0.0, 0.0, 0.0}, T = 1.0;
                int32_t nseg = 0;
                if (orc_ray(cam, (double)u, (double)v, o, d)) {
                    for (int64_t e = tile_start[t]; e < tile_start[t + 1] && !(T < t_stop); e++) {
                        const int64_t i = tile_cells[e];
                        orc_seg sg;
                        if (!cell_segment(s, cd, i, o, d, &sg)) continue;
                        double surv = exp(-s->sigma[i] * (sg.tb - sg.ta));
                        double col[3];
                        cell_colour(s, i, o, d, &sg, kappa, col, NULL, NULL, NULL);
                        for (int ch = 0; ch < 3; ch++) C[ch] += T * (1.0 - surv) * col[ch];
                        T *= surv;
                        nseg++;
                    }
                }
                for (int ch = 0; ch < 3; ch++) out_rgb[3 * k + ch] = C[ch];
                out_T[k] = T;
                if (out_nseg) out_nseg[k] = nseg;
            }
        }
    }
    return 0;
}
