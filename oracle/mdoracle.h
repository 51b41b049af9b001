/* Oracle for the mixed-dimensional block solver: TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, sequential FP64 CPU implementation of what the GPU path
 * computes.  Only the tests, the smoke check and the benchmark's CPU-baseline
 * leg may load it.  It shares no code, header, table or helper with the CUDA
 * library; the two meet only in the seeded instance arrays.
 *
 * Paper: Hu, Keilegavlen, Nordbotten, "Effective preconditioners for
 * mixed-dimensional scalar elliptic problems" (arXiv:2206.03203).
 *   assembly ........ Sec. 2.1 Eq. (1)-(3), Sec. 3.1 Eq. (4) (block order [m; f])
 *   Schur ........... Sec. 3.2 Eq. (7)
 *   M_L ............. Sec. 3.2 Eq. (8), Sec. 3.3 Algorithm 1
 *   AMG V-cycle ..... Sec. 3.3 (one V-cycle per diagonal block)
 *   GMRES ........... Sec. 3.2 (right preconditioning), Sec. 4 (x0 = 0,
 *                     relative-residual stopping rule)
 * Parity status of each function is listed in its comment.
 */
#ifndef MDORACLE_H
#define MDORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int64_t nrow, ncol, nnz;
    int64_t *rp;   /* [nrow+1] */
    int32_t *ci;   /* [nnz], ascending within a row */
    double *v;     /* [nnz] */
} ocsr;

ocsr *orc_csr_new(int64_t nrow, int64_t ncol, int64_t nnz);
void orc_csr_free(ocsr *A);

/* Two-point-flux assembly of the full system [A_mm A_mf; A_fm A_ff] and the
 * right-hand sides b[r*(n_m+n_f) + i].  Returns NULL on invalid input. */
ocsr *orc_assemble(int dim, int n, const double *km, int64_t nf,
                   const int32_t *fc_axis, const int32_t *fc_pos,
                   const double *fc_kf, const double *fc_a, int nrhs,
                   const double *pD_left, const double *pD_right, double *b);

/* The paper's own partition (Sec. 3.1, Eq. (4)): unknowns [all cell
 * pressures (matrix, then fracture); interface fluxes, 2 per fracture cell],
 * a symmetric saddle-point system whose flux block is diag(-1/T).  b has
 * n_m + 3 n_f entries per right-hand side (zero on the flux rows). */
ocsr *orc_assemble_flux(int dim, int n, const double *km, int64_t nf,
                        const int32_t *fc_axis, const int32_t *fc_pos,
                        const double *fc_kf, const double *fc_a, int nrhs,
                        const double *pD_left, const double *pD_right, double *b);

/* Either form with either junction rule (0: pairwise links between the
 * fracture cells of a junction; 1: each junction of >= 3 cells a node joined
 * by half transmissibilities, eliminated by star-delta in the primal form,
 * an intersection cell with interface fluxes in the flux form).  Allocates
 * the right-hand sides (*b_out, nrhs x NT, free with orc_free);
 * *n_omega = the size of the first block (matrix cells in the primal form,
 * all pressures in the flux form).  fc_kn: the fractures' normal
 * permeabilities (kappa = 2 k_n / a in the matrix-fracture coupling), NULL
 * for k_n = k_f. */
ocsr *orc_assemble_ex(int dim, int n, const double *km, int64_t nf,
                      const int32_t *fc_axis, const int32_t *fc_pos,
                      const double *fc_kf, const double *fc_a, int nrhs,
                      const double *pD_left, const double *pD_right, int flux, int junction,
                      int64_t *n_omega, double **b_out, const double *fc_kn);
void orc_free(void *p);

/* Slice a full CSR at row/column n_m into its four blocks. */
int orc_split(const ocsr *A, int64_t n_m, ocsr **Amm, ocsr **Amf, ocsr **Afm, ocsr **Aff);

/* Eq. (7): S~ = A_mm - A_mf diag(A_ff)^-1 A_fm.  NULL on a zero diagonal. */
ocsr *orc_schur(const ocsr *Amm, const ocsr *Amf, const ocsr *Afm, const ocsr *Aff);

/* y = A x */
void orc_spmv(const ocsr *A, const double *x, double *y);

/* Symmetrised strength graph (pattern only, no diagonal). */
ocsr *orc_strength(const ocsr *A, double theta);

/* MIS-2 priority key of vertex i on level l. */
uint64_t orc_mis_key(uint64_t seed, int level, int64_t i);

typedef struct orc_amg orc_amg;
typedef struct {
    double theta;
    int64_t n_coarse;    /* dense Cholesky once n <= n_coarse */
    int max_levels;
    double stall_ratio;  /* stop when n_{l+1} > stall_ratio n_l */
    uint64_t seed;
    int smoother;        /* 0 = L1-Jacobi, 1 = Chebyshev, 2 = Gauss-Seidel (oracle only) */
    int prec;            /* 64, 32 (float storage), 16 / 17 (bf16 / fp16 row-scaled levels, float vectors) */
    int lowp_from_level; /* for prec 16/17: first level stored in bf16/fp16 */
    int sweeps;          /* smoother applications before and after the coarse correction */
    int smoothed;        /* 0 = piecewise-constant P, 1 = smoothed aggregation P */
    int cheb_degree;     /* Chebyshev degree (0 = 2) */
} orc_amg_opts;

/* Storage rounding used by the precision emulation: 32 -> float,
 * 16 -> bfloat16 of the float, 17 -> binary16 of the float (all round to
 * nearest even); 64 -> x. */
double orc_round_lowp(double x, int prec);

orc_amg *orc_amg_setup(const ocsr *A, const orc_amg_opts *o);
/* A packed batch: K instances whose rows are the segments [off[k], off[k+1])
 * of a block-diagonal matrix (off[0] = 0, off[K] = rows).  Every instance is
 * coarsened as if it were alone: MIS-2 keys use a row's index within its
 * segment, the next level's segments are each instance's aggregates, the
 * coarsening stops once every segment has at most n_coarse rows, and the
 * coarsest level is solved with each segment's own dense Cholesky factor.
 * orc_amg_setup is the case K = 1.  NULL on failure. */
orc_amg *orc_amg_setup_seg(const ocsr *A, const orc_amg_opts *o, int K, const int64_t *off);
/* Segment offsets of level l (K + 1 values); returns K, or -1. */
int orc_amg_level_seg(const orc_amg *h, int l, int64_t *out);
void orc_amg_free(orc_amg *h);
int orc_amg_nlevels(const orc_amg *h);
int64_t orc_amg_level_n(const orc_amg *h, int l);
const ocsr *orc_amg_level_A(const orc_amg *h, int l);
int orc_amg_level_agg(const orc_amg *h, int l, int32_t *out);  /* -1 = not aggregated */
int orc_amg_level_roots(const orc_amg *h, int l, int8_t *out);
int orc_amg_level_l1(const orc_amg *h, int l, double *out);
/* The level's stored operator as the V-cycle applies it: values in CSR order
 * of orc_amg_level_A (each the FP32, or the bf16/fp16 value times its row
 * scale, as a double), the row scales s_i (1 on levels not stored in
 * bf16/fp16) and 1/D1 rounded to the vector precision.  Any pointer may be
 * NULL. */
int orc_amg_level_stored(const orc_amg *h, int l, double *av, double *rs, double *dinv);
/* 16 / 17 when the level is stored in bf16 / fp16 with row scales, else 0. */
int orc_amg_level_lowp(const orc_amg *h, int l);
/* Prolongator of level l (fine rows x coarse columns) when smoothed; NULL otherwise. */
const ocsr *orc_amg_level_P(const orc_amg *h, int l);
int orc_amg_coarsest_dense(const orc_amg *h);  /* 1: the last level is a dense solve; 2: it has no
                                                   couplings and is solved by x = b / a_ii; 0: smoothed */
/* One V-cycle x = V(b) on level 0. */
void orc_vcycle(orc_amg *h, const double *b, double *x);

/* Preconditioner callback: z = M r. Returns 0 on success. */
typedef int (*orc_prec_fn)(void *ctx, const double *r, double *z);

typedef struct orc_ml orc_ml;
/* kind 0 = block lower triangular M_L (Alg. 1), 1 = block diagonal, 2 = block upper. */
orc_ml *orc_ml_new(const ocsr *A, int64_t n_m, const orc_amg_opts *o, int kind);
/* M_L of a packed batch: S~ coarsened with the matrix-row segments moff and
 * A_ff with the fracture-row segments foff (offsets within the fracture
 * rows), K + 1 values each (see orc_amg_setup_seg). */
orc_ml *orc_ml_new_seg(const ocsr *A, int64_t n_m, const orc_amg_opts *o, int kind, int K, const int64_t *moff,
                       const int64_t *foff);
void orc_ml_free(orc_ml *m);
int orc_ml_apply(void *ml, const double *r, double *z);
const orc_amg *orc_ml_amg(const orc_ml *m, int block);  /* 0 = S~, 1 = A_ff */
const ocsr *orc_ml_schur(const orc_ml *m);
int orc_identity_apply(void *ctx, const double *r, double *z);

typedef struct {
    int iterations;     /* preconditioner applications */
    int restarts;
    int converged;
    double relres_true; /* ||b - A x|| / ||b|| at exit */
    int history_len;
} orc_stats;

/* Right-preconditioned flexible GMRES(m) with modified Gram-Schmidt.
 * x holds x0 on entry.  hist (optional, length >= maxit+1) receives the
 * residual-norm estimates after each preconditioner application, relative
 * to ||b||, with hist[0] the initial one. */
int orc_fgmres(const ocsr *A, orc_prec_fn prec, void *pctx, const double *b, double *x,
               int restart, double rtol, int maxit, double *hist, orc_stats *st);
/* Preconditioned conjugate gradients (symmetric preconditioner). */
int orc_pcg(const ocsr *A, orc_prec_fn prec, void *pctx, const double *b, double *x,
            double rtol, int maxit, double *hist, orc_stats *st);
/* Preconditioned MINRES for symmetric A and a symmetric positive definite
 * preconditioner (the block-diagonal B_D of Sec. 3.2 with symmetric
 * V-cycles); same stopping rule and iteration count as orc_pcg. */
int orc_minres(const ocsr *A, orc_prec_fn prec, void *pctx, const double *b, double *x,
               double rtol, int maxit, double *hist, orc_stats *st);

#ifdef __cplusplus
}
#endif
#endif
