/* A solve through the C ABI alone (no Python): the four-fracture unit square
 * of 64 x 64 cells (k_m = 1; fractures on the face planes x = 16, 48 and
 * y = 19, 45, full length, k_f = 1e4, a = 1e-4; p = 1 at x = 0, p = 0 at
 * x = 1), the block lower preconditioner M_L of Algorithm 1 with FGMRES(30)
 * to a relative residual of 1e-8 from x0 = 0, solution returned in host
 * memory.
 *
 *   gcc -std=c99 -I include solve_c.c -L <dir> -l:libmdsolve.so -Wl,-rpath,<dir> -o solve_c
 *
 * Prints the status, iterations and residual; exit status 0 when the solve
 * converged, 1 when it did not, 2 when no context could be created (no GPU). */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include "mdsolve.h"

static int fail(mds_ctx ctx, const char *what, int code) {
    fprintf(stderr, "%s failed: %s (%s)\n", what, mds_error_string(code), ctx ? mds_last_error(ctx) : "");
    return code;
}

int main(void) {
    const int n = 64;
    const int planes_x[2] = {16, 48}, planes_y[2] = {19, 45};
    const int64_t nf = 4 * (int64_t)n;
    double *km = malloc(sizeof(double) * n * n);
    int32_t *axis = malloc(sizeof(int32_t) * nf);
    int32_t *pos = malloc(sizeof(int32_t) * 3 * nf);
    double *kf = malloc(sizeof(double) * nf), *ap = malloc(sizeof(double) * nf);
    double *pl = malloc(sizeof(double) * n), *pr = malloc(sizeof(double) * n);
    double *x = calloc((size_t)(n * n + nf), sizeof(double));
    if (!km || !axis || !pos || !kf || !ap || !pl || !pr || !x) return 3;
    for (int i = 0; i < n * n; i++) km[i] = 1.0;
    int64_t k = 0;
    for (int q = 0; q < 2; q++)
        for (int y = 0; y < n; y++, k++) {  /* normal x: (plane, cell y) */
            axis[k] = 0;
            pos[3 * k] = planes_x[q];
            pos[3 * k + 1] = y;
            pos[3 * k + 2] = 0;
        }
    for (int q = 0; q < 2; q++)
        for (int xc = 0; xc < n; xc++, k++) {  /* normal y: (cell x, plane) */
            axis[k] = 1;
            pos[3 * k] = xc;
            pos[3 * k + 1] = planes_y[q];
            pos[3 * k + 2] = 0;
        }
    for (k = 0; k < nf; k++) {
        kf[k] = 1e4;
        ap[k] = 1e-4;
    }
    for (int y = 0; y < n; y++) {
        pl[y] = 1.0;
        pr[y] = 0.0;
    }

    mds_ctx ctx = NULL;
    int code = mds_create(&ctx, 0, NULL, NULL);
    if (code != MDS_OK) {
        fail(NULL, "mds_create", code);
        return 2;
    }
    mds_instance in = {2, n, km, nf, axis, pos, kf, ap, 1, pl, pr, 0, MDS_JUNCTION_PAIRWISE, NULL};
    mds_system sys = NULL;
    mds_precond prec = NULL;
    mds_setup_opts so;
    mds_solve_opts vo;
    mds_rhs_stats st;
    int64_t n_m = 0, n_f = 0;
    int nrhs = 0;
    int64_t nnz[5];
    if ((code = mds_assemble(ctx, &in, &sys)) != MDS_OK) return fail(ctx, "mds_assemble", code), 1;
    mds_system_info(sys, &n_m, &n_f, &nrhs, nnz);
    mds_setup_opts_default(&so);
    if ((code = mds_setup(ctx, sys, &so, &prec)) != MDS_OK) return fail(ctx, "mds_setup", code), 1;
    mds_solve_opts_default(&vo);
    code = mds_solve(ctx, sys, prec, NULL, x, 1, &vo, &st);
    printf("n_m %lld n_f %lld nnz %lld status %d iterations %d relres %.3e p(32,32) %.6f\n", (long long)n_m,
           (long long)n_f, (long long)nnz[4], st.status, st.iterations, st.relres_true, x[32 + n * 32]);
    mds_precond_destroy(prec);
    mds_system_destroy(sys);
    mds_destroy(ctx);
    free(km);
    free(axis);
    free(pos);
    free(kf);
    free(ap);
    free(pl);
    free(pr);
    free(x);
    return code == MDS_OK ? 0 : 1;
}
