/* A program that uses the library through its C ABI alone (include/lbhb.h), with
 * no Python: three G = 0 Couette cells started from the linear profile, the
 * exact steady state of halfway bounce-back, in FP32 and FP64.  The time-averaged
 * wall stress must be rho nu 2U/ny and the shear rate 2U/ny, with
 * nu = (tau - 1/2)/3 for the BGK cells (tau = 1 and 0.8) and (1/s_nu - 1/2)/3 for
 * the cell with multiple relaxation times (tau = 1, s_nu = 1.6).
 * Exit status: 0 all values right, 1 a value wrong, 2 an ABI call failed, 3 no
 * CUDA device (lb_create reports a CUDA error; the message is printed). */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "lbhb.h"

static int check(const char* what, double got, double want, double rel, double abs_tol)
{
    if (fabs(got - want) <= rel * fabs(want) + abs_tol) return 0;
    fprintf(stderr, "%s: %.9g, expected %.9g (tolerance %g relative + %g)\n", what, got, want, rel, abs_tol);
    return 1;
}

int main(void)
{
    enum { NX = 64, NY = 32, NC = 3, STEPS = 3000 };
    /* the multiple-relaxation-time cell at a small wall speed: its profile is linear
       only up to a relative O(U^2) deviation (1e-8 at U = 1e-3) */
    const double u_wall[NC] = {1e-3, 1e-4, 1e-4};
    lb_cell_params cells[NC];
    memset(cells, 0, sizeof cells);
    for (int c = 0; c < NC; ++c) {
        cells[c].nx = NX;
        cells[c].ny = NY;
        cells[c].tau = c == 1 ? 0.8 : 1.0;
        cells[c].rho0 = 0.83;
        cells[c].u_wall = u_wall[c];
        cells[c].rho_bar_a = cells[c].rho_bar_b = 0.6;
        cells[c].bc = LB_BC_COUETTE;
    }
    cells[2].s_nu = 1.6;
    const double nu[NC] = {0.5 / 3.0, 0.3 / 3.0, (1.0 / 1.6 - 0.5) / 3.0};

    static double rho[NC * NY * NX], ux[NC * NY * NX];
    for (int c = 0; c < NC; ++c)
        for (int y = 0; y < NY; ++y)
            for (int x = 0; x < NX; ++x) {
                rho[(c * NY + y) * NX + x] = 0.6;
                ux[(c * NY + y) * NX + x] = u_wall[c] * (2.0 * (y + 0.5) / NY - 1.0);
            }
    if (lb_step(NULL, 1) != LB_ERR_INVALID) return 2;  /* a NULL handle is refused, not dereferenced */

    const lb_precision precs[2] = {LB_FP32, LB_FP64};
    /* FP32: the wall stress is a sum of FP32 population differences, an absolute
       error of order 1e-8 on stresses of 3e-7 .. 1e-5 */
    const double tol[2] = {2e-2, 1e-8}, abs_tol[2] = {2e-8, 0.0};
    int bad = 0;
    for (int k = 0; k < 2; ++k) {
        lb_handle* h = NULL;
        lb_status st = lb_create(cells, NC, precs[k], NULL, &h);
        if (st != LB_OK) {
            fprintf(stderr, "lb_create: %s\n", lb_last_error(NULL));
            return st == LB_ERR_CUDA ? 3 : 2;
        }
        double sigma[NC], shear[NC];
        if (lb_init_fields(h, rho, rho, ux, NULL) != LB_OK || lb_set_sampling(h, STEPS - 300, 10) != LB_OK ||
            lb_step(h, STEPS) != LB_OK || lb_shear_stress(h, sigma, shear, NULL) != LB_OK) {
            fprintf(stderr, "ABI call failed: %s\n", lb_last_error(h));
            lb_destroy(h);
            return 2;
        }
        for (int c = 0; c < NC; ++c) {
            char what[64];
            snprintf(what, sizeof what, "precision %d cell %d sigma_xy", (int)precs[k], c);
            bad |= check(what, sigma[c], 1.2 * nu[c] * 2.0 * u_wall[c] / NY, tol[k], abs_tol[k]);
            snprintf(what, sizeof what, "precision %d cell %d shear rate", (int)precs[k], c);
            bad |= check(what, shear[c], 2.0 * u_wall[c] / NY, tol[k], 0.0);
        }
        lb_destroy(h);
    }
    if (!bad) printf("ok\n");
    return bad;
}
