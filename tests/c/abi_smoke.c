/* A plain C program against include/cmlbm.h and libcmlbm.so: create a D3Q27 FP32 handle,
 * initialise a small shear wave from host arrays, step it, read the FP64 sums and the fields
 * back into host memory, and check mass conservation and the decay of the wave.
 * Usage: abi_smoke [nsteps]. Exit status 0 on success. */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include "cmlbm.h"

int main(int argc, char** argv) {
    const int nsteps = argc > 1 ? atoi(argv[1]) : 20;
    const int nx = 64, ny = 16, nz = 8;
    const size_t n = (size_t)nx * ny * nz;
    cmlbm_config cfg;
    if (cmlbm_config_default(&cfg) != CMLBM_OK) return 1;
    cfg.lattice = CMLBM_D3Q27;
    cfg.nx = nx;
    cfg.ny = ny;
    cfg.nz = nz;
    cfg.storage = CMLBM_F32;
    cfg.tau = 0.6;
    cmlbm_t* h = NULL;
    int rc = cmlbm_create(&cfg, &h);
    if (rc != CMLBM_OK) {
        fprintf(stderr, "create failed (%d): %s\n", rc, cmlbm_last_error(NULL));
        return 1;
    }
    double* rho = (double*)malloc(n * sizeof(double));
    double* u = (double*)calloc(3 * n, sizeof(double));
    const double pi = 3.14159265358979323846, amp = 0.02;
    for (size_t c = 0; c < n; ++c) {
        const int y = (int)((c / nx) % ny);
        rho[c] = 1.0;
        u[c] = amp * sin(2.0 * pi * (y + 0.5) / ny);    /* u_x(y): a decaying shear wave */
    }
    rc = cmlbm_init(h, rho, u, CMLBM_HOST);
    double s0[5], s1[5];
    if (rc == CMLBM_OK) rc = cmlbm_reduce(h, s0);
    if (rc == CMLBM_OK) rc = cmlbm_step(h, nsteps);
    if (rc == CMLBM_OK) rc = cmlbm_reduce(h, s1);
    if (rc == CMLBM_OK) rc = cmlbm_moments(h, rho, u, CMLBM_HOST);
    if (rc != CMLBM_OK) {
        fprintf(stderr, "call failed (%d): %s\n", rc, cmlbm_last_error(h));
        return 1;
    }
    /* the wave decays at the rate nu k^2 (nu = (tau - 1/2) / 3), to leading order */
    const double nu = (cfg.tau - 0.5) / 3.0, k = 2.0 * pi / ny;
    const double expect = exp(-2.0 * nu * k * k * nsteps);
    const double ratio = s1[4] / s0[4];
    double umax = 0.0;
    for (size_t c = 0; c < n; ++c) umax = fmax(umax, fabs(u[c]));
    printf("kernel %d, mass %.9f -> %.9f, energy ratio %.6f (viscous decay %.6f), max |u_x| %.6f\n",
           cmlbm_step_kernel(h), s0[0], s1[0], ratio, expect, umax);
    int ok = fabs(s1[0] - s0[0]) < 1e-6 * s0[0] && fabs(ratio - expect) < 0.03 * expect && umax < amp;
    cmlbm_destroy(h);
    free(rho);
    free(u);
    return ok ? 0 : 2;
}
