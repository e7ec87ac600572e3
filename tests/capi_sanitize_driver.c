/*
 * The library's host code under AddressSanitizer (built by
 * tests/test_capi_sanitize.py with -fsanitize=address on the host side of
 * every translation unit): plan creation, layout, camera updates, flags,
 * validation errors and the neighbour build's argument checks.  None of
 * these calls touches a GPU.
 */
#include <stdio.h>
#include <string.h>
#include "powerfoam.h"
int main(void) {
    pf_camera c[2];
    memset(c, 0, sizeof c);
    for (int v = 0; v < 2; v++) {
        double rot[9] = {0, 1, 0, 0, 0, -1, -1, 0, 0};
        memcpy(c[v].rot, rot, sizeof rot);
        c[v].origin[0] = 3;
        c[v].fx = c[v].fy = 100;
        c[v].cx = 50; c[v].cy = 40;
        c[v].width = 100 + 7 * v; c[v].height = 80;
        c[v].model = v;
    }
    pf_plan *p = 0;
    int ok = pf_plan_create(1000, 16, c, 2, 5000, &p) == PF_OK;
    uint64_t b = 0, px = 0;
    ok &= pf_plan_workspace_bytes(p, &b) == PF_OK && b > 0;
    ok &= pf_plan_pixels(p, &px) == PF_OK && px == 100 * 80 + 107 * 80;
    ok &= pf_plan_set_cameras(p, c, 2) == PF_OK;
    ok &= pf_plan_enable_stats(p, 1) == PF_OK && pf_plan_enable_stats(p, 0) == PF_OK;
    ok &= pf_plan_omit_hit_records(p) == PF_OK;
    ok &= pf_plan_set_record_hits(p, 1) == PF_ERR_INVALID_ARG;
    pf_plan_destroy(p);
    c[0].model = 7;
    ok &= pf_plan_create(10, 4, c, 1, 100, &p) == PF_ERR_INVALID_ARG;
    ok &= strlen(pf_last_error_message()) > 0;
    ok &= pf_neighbours_workspace_bytes(1000) > 0;
    ok &= pf_build_neighbours(0, 0, 0, 10, 65, 0, 0, 0, 0, 0, 0, 0) == PF_ERR_INVALID_ARG;
    for (int s = 0; s < 7; s++) ok &= pf_status_string((pf_status)s) != 0;
    printf(ok ? "capi ok\n" : "capi FAILED\n");
    return ok ? 0 : 1;
}
