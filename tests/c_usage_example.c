/* c_usage_example.c -- the C usage shown to library users: one 256x128x128
 * shear cell with a spheroid, 1000 steps, the hydrodynamic force read back.
 * The ABI tests compile and link it against the headers and the library
 * (it is not run there: it needs a GPU). */
#include <stdio.h>
#include <string.h>
#include "lbm.h"

int main(void) {
    lbm_grid_desc d;
    memset(&d, 0, sizeof d);                   /* NULL stream, library-owned device memory */
    d.nx = 256; d.ny = 128; d.nz = 128;
    d.tau = 0.8; d.magic = 3.0 / 16.0; d.rho0 = 1.0;
    d.periodic[0] = d.periodic[2] = 1;         /* walls at y = 0 and y = ny - 1 */
    d.wall_u_lo[0] = -0.02; d.wall_u_hi[0] = 0.02;
    d.prec = LBM_F32;
    lbm_ctx *ctx = NULL;
    if (lbm_create(&d, &ctx) != LBM_OK) return 1;

    lbm_particle p;
    memset(&p, 0, sizeof p);
    p.pos[0] = 127.5; p.pos[1] = 63.5; p.pos[2] = 63.5;
    p.quat[0] = 1.0;                           /* body x along world x */
    p.semi_axes[0] = 24; p.semi_axes[1] = 3; p.semi_axes[2] = 3;
    p.density = 2.0;
    p.shape = LBM_SHAPE_ELLIPSOID;
    lbm_status s = lbm_set_particles(ctx, &p, 1);
    if (s == LBM_OK) s = lbm_step(ctx, 1000);  /* asynchronous */
    double F[3], M[3];
    if (s == LBM_OK) s = lbm_get_forces(ctx, F, M, 1);
    if (s != LBM_OK) fprintf(stderr, "%s: %s\n", lbm_status_string(s), lbm_last_error(ctx));
    else printf("F = (%g, %g, %g)\n", F[0], F[1], F[2]);
    lbm_destroy(ctx);
    return s != LBM_OK;
}
