/*
 * Memory- and UB-checked run of the FP64 oracle: this file includes the
 * oracle's source and is compiled with -fsanitize=address,undefined by
 * tests/test_oracle_sanitize.py.  It exercises every exported function on a
 * small deterministic scene (with displacement, learned sites, eight sites,
 * view-dependent colours, a fisheye camera and candidate lists) and checks
 * only that results are finite: the pins check the values.
 */
#include <stdio.h>

#include "../oracle/pf_oracle.c"

static uint64_t rs = 88172645463325252ull;
static double urand(void) { /* xorshift64 in [0, 1) */
    rs ^= rs << 13;
    rs ^= rs >> 7;
    rs ^= rs << 17;
    return (double)(rs >> 11) * (1.0 / 9007199254740992.0);
}

static int finite_all(const double *a, int64_t n) {
    for (int64_t i = 0; i < n; i++)
        if (!isfinite(a[i])) return 0;
    return 1;
}

int main(void) {
    enum { N = 24, NS = 8, W = 9, H = 7 };
    static double pos[3 * N], w[N], R[N], sig[N], rgb[3 * N], nrm[3 * N], off[N], tex[3 * NS * N];
    static double disp[NS * N], sites[2 * NS * N], sv[NS * 8 * 6 * N];
    for (int i = 0; i < N; i++) {
        for (int r = 0; r < 3; r++) {
            pos[3 * i + r] = 0.3 * (urand() - 0.5);
            rgb[3 * i + r] = urand();
            nrm[3 * i + r] = urand() - 0.5;
        }
        double r0 = 0.05 + 0.05 * urand();
        w[i] = r0 * r0;
        R[i] = 1.5 * r0;
        sig[i] = 1.0 + 2.0 * urand();
        off[i] = r0 * (urand() - 0.5);
    }
    for (int q = 0; q < 3 * NS * N; q++) tex[q] = 0.2 * (urand() - 0.5);
    for (int q = 0; q < NS * N; q++) disp[q] = 0.02 * (urand() - 0.5);
    for (int q = 0; q < 2 * NS * N; q++) sites[q] = 0.6 * (urand() - 0.5);
    for (int q = 0; q < NS * 8 * 6 * N; q++) sv[q] = urand() - 0.5;
    orc_scene s = {N, pos, w, R, sig, rgb, nrm, off, tex, disp, 6.0, sites, sv, 10.0, NS};
    orc_camera cams[2];
    for (int c = 0; c < 2; c++) {
        double rot[9] = {0, 1, 0, 0, 0, -1, -1, 0, 0}; /* looking along -x */
        memcpy(cams[c].rot, rot, sizeof rot);
        cams[c].origin[0] = 0.6;
        cams[c].origin[1] = 0.05;
        cams[c].origin[2] = 0.02;
        cams[c].fx = cams[c].fy = c ? 2.5 : 12.0;
        cams[c].cx = W / 2.0;
        cams[c].cy = H / 2.0;
        cams[c].width = W;
        cams[c].height = H;
        cams[c].model = c; /* pinhole, then a fisheye with pixels beyond pi */
    }
    /* candidate lists: every other site */
    static int64_t beg[N], end[N];
    static int32_t idx[N * N];
    int64_t m = 0;
    for (int i = 0; i < N; i++) {
        beg[i] = m;
        for (int j = 0; j < N; j++)
            if (j != i) idx[m++] = j;
        end[i] = m;
    }
    orc_cands cd = {beg, end, idx};
    static double out_rgb[3 * W * H], out_T[W * H], gC[3 * W * H], gT[W * H], grad[(int64_t)N * NPAR];
    static double sp[N], nm[N], ws[N], wn[N];
    static int32_t nseg[W * H];
    static uint8_t flag[N];
    for (int q = 0; q < 3 * W * H; q++) gC[q] = urand() - 0.5;
    for (int q = 0; q < W * H; q++) gT[q] = urand() - 0.5;
    for (int i = 0; i < N; i++) {
        ws[i] = urand();
        wn[i] = urand();
    }
    int ok = 1;
    for (int c = 0; c < 2; c++) {
        for (int with_list = 0; with_list < 2; with_list++) {
            const orc_cands *cdp = with_list ? &cd : NULL;
            ok &= orc_render(&s, cdp, &cams[c], W * H, NULL, 6.0, out_rgb, out_T, nseg, 2) == 0;
            ok &= finite_all(out_rgb, 3 * W * H) && finite_all(out_T, W * H);
            ok &= orc_render_grad(&s, cdp, &cams[c], W * H, NULL, 6.0, gC, gT, grad, 2) == 0;
            ok &= finite_all(grad, (int64_t)N * NPAR);
            ok &= orc_cell_contrib(&s, cdp, &cams[c], W * H, NULL, sp, nm, 2) == 0;
            ok &= orc_contrib_grad(&s, cdp, &cams[c], W * H, NULL, ws, wn, grad, 2) == 0;
            ok &= finite_all(grad, (int64_t)N * NPAR) && finite_all(sp, N) && finite_all(nm, N);
        }
        ok &= orc_hit_cells(&s, &cams[c], W * H, NULL, flag, 2) == 0;
    }
    static int32_t rect[4 * N];
    static uint64_t key[N];
    ok &= orc_bin(&cams[0], N, pos, w, R, rect, key) == 0;
    static float pf[3 * N], wf[N], Rf[N], Ro[N];
    static int32_t nbr[N * 6];
    for (int q = 0; q < 3 * N; q++) pf[q] = (float)pos[q];
    for (int i = 0; i < N; i++) {
        wf[i] = (float)w[i];
        Rf[i] = (float)R[i];
    }
    ok &= orc_neighbours(pf, wf, Rf, N, 6, N, NULL, nbr, Ro, 2) == 0;
    double o[3], d[3], ta[64], tb[64];
    int32_t cell[64], act[128];
    orc_ray(&cams[0], 4.0, 3.0, o, d);
    int64_t ns = orc_ray_segments(&s, NULL, o, d, 64, cell, ta, tb, act, act + 64);
    ok &= ns >= 0;
    printf(ok ? "sanitized oracle ok\n" : "sanitized oracle FAILED\n");
    return ok ? 0 : 1;
}
