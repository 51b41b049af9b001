/* mdsolve: GB300 solver for mixed-dimensional scalar elliptic problems.
 *
 * C ABI of the CUDA library libmdsolve.so.  It implements the block-
 * factorisation preconditioner of Hu, Keilegavlen and Nordbotten,
 * "Effective preconditioners for mixed-dimensional scalar elliptic problems"
 * (arXiv:2206.03203) on one GPU:
 *   - the 2x2 block system  [A_mm A_mf; A_fm A_ff] [p_m; p_f] = [f_m; f_f]
 *     (Sec. 3.1, Eq. (4)), here with matrix-cell pressures m and fracture-cell
 *     pressures f from a cell-centred two-point-flux discretisation of the
 *     model of Sec. 2.1 (Eq. (1)-(3));
 *   - the approximate Schur complement S~ = A_mm - A_mf diag(A_ff)^-1 A_fm
 *     (Sec. 3.2, Eq. (7));
 *   - the inexact block lower-triangular preconditioner M_L (Sec. 3.2,
 *     Eq. (8)) applied by Algorithm 1 (Sec. 3.3), each diagonal block
 *     approximately inverted by one aggregation-AMG V-cycle (Sec. 3.3);
 *   - right-preconditioned flexible GMRES with zero initial guess and a
 *     relative-residual stopping rule (Sec. 3.2 and Sec. 4), or PCG with the
 *     block-diagonal preconditioner B_D (Sec. 3.2).
 *
 * Conventions (all entry points):
 *   - Every call returns an int status: MDS_OK (0), a warning (> 0) or an
 *     error (< 0).  mds_error_string() names a status; mds_last_error()
 *     returns the context's last detailed message.  No call aborts or traps.
 *   - Handles are owned by the library and freed by their _destroy call.
 *     Host arrays passed in are copied before the call returns.  Device
 *     pointers passed in stay owned by the caller and must stay valid for
 *     the duration stated at each call.
 *   - All GPU work is enqueued on the context's CUDA stream.  Calls that
 *     return sizes or statistics synchronise that stream.
 *   - A context is not thread-safe; use one context per host thread.
 *   - Sparse matrices are CSR with int32 row pointers and column indices
 *     (columns ascending within a row) and FP64 values; vectors are FP64.
 */
#ifndef MDSOLVE_H
#define MDSOLVE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define MDS_OK 0
#define MDS_WARN_NOT_CONVERGED 1   /* some right-hand side hit max_iters */
#define MDS_ERR_INVALID (-1)       /* bad argument, size or handle */
#define MDS_ERR_CUDA (-2)          /* a CUDA runtime call failed */
#define MDS_ERR_OOM (-3)           /* device allocation failed */
#define MDS_ERR_NOT_SPD (-4)       /* coarsest Cholesky met a pivot <= 0 */
#define MDS_ERR_BREAKDOWN (-5)     /* Krylov breakdown (non-finite or zero norm) */
#define MDS_ERR_NONFINITE (-6)     /* NaN/Inf in the right-hand side or residual */
#define MDS_ERR_CAPACITY (-7)      /* a sparse row exceeded a kernel's row capacity */
#define MDS_ERR_TIMEOUT (-8)       /* an iterative setup loop exceeded its bound */
#define MDS_ERR_ZERO_DIAG (-9)     /* zero diagonal in A_ff (Eq. (7) undefined) */

typedef struct mds_ctx_s *mds_ctx;
typedef struct mds_system_s *mds_system;
typedef struct mds_precond_s *mds_precond;

/* Optional device allocator (for example a framework's caching allocator).
 * alloc returns a device pointer of at least `bytes` bytes aligned to 256
 * bytes or NULL on failure; free releases it.  Both are called on the host
 * thread that calls into the library, with the context's stream current
 * for stream-ordered allocators. */
typedef struct {
    void *(*alloc)(size_t bytes, void *user);
    void (*free)(void *ptr, void *user);
    void *user;
} mds_allocator;

/* Create a context on CUDA device `device` that enqueues on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  `alloc` may be NULL
 * for stream-ordered allocation from a memory pool the context owns: blocks
 * freed by one set-up or solve stay mapped in that pool for the next one
 * (the pool holds the largest working set the context has used), and
 * mds_destroy returns the pool to the driver.  The allocator struct is
 * copied; its callbacks must stay valid for the context's lifetime.  The
 * environment variable MDS_PDL=0 makes the context launch its kernels in
 * plain stream order, without programmatic dependent launch (for diagnosis;
 * the results are the same). */
int mds_create(mds_ctx *out, int device, void *cuda_stream, const mds_allocator *alloc);
/* Systems and preconditioners keep their context alive: destroying a context
 * that still has some only marks it, and it is released when the last of them
 * is destroyed (in any order).  A context must not be used after this call. */
int mds_destroy(mds_ctx ctx);
/* Change the stream later calls enqueue on. */
int mds_set_stream(mds_ctx ctx, void *cuda_stream);
const char *mds_error_string(int status);
/* Detailed message of the last failing call on this context (static storage
 * owned by the context, valid until its next call). */
const char *mds_last_error(mds_ctx ctx);

/* ---- problem input ----
 * A Cartesian instance on the unit square (dim 2) or cube (dim 3) with n
 * cells per side (h = 1/n), matrix cells indexed x-fastest.  Fracture cells
 * are interior grid faces (codimension-1 subdomains, Sec. 2.1) given by their
 * normal axis and position (x, y, z): the coordinate along the normal axis is
 * the face-plane index 1..n-1, the others are cell indices.  Each has a
 * tangential permeability k_f and an aperture a.  Dirichlet data lives on the
 * x = 0 (pD_left) and x = 1 (pD_right) faces, one value per boundary face
 * (index y + n z) and right-hand side; other boundary faces are no-flow.
 * Transmissibilities (two-point flux, Eq. (1)-(3)):
 *   matrix-matrix      |F| / (h/(2 k_i) + h/(2 k_j))
 *   matrix-fracture    |F| / (h/(2 k_i) + 1/kappa),  kappa = 2 k_n / a (k_n = k_f unless
 *                      fc_kn is given: the paper's normal permeability, Eq. (2))
 *   fracture-fracture  t_i t_j / (t_i + t_j) for every pair of fracture cells
 *                      meeting at a vertex (2D) / edge (3D) e,
 *                      t = k_f a |e| / (h/2)
 *   Dirichlet          matrix |F| 2 k / h; fracture end on x = 0/1: t, with
 *                      the mean of the two boundary faces at that end.
 * `junction` selects the rule at junctions of three or more fracture cells
 * (intersections, Sec. 2.1): MDS_JUNCTION_PAIRWISE (0) links every pair as
 * above; MDS_JUNCTION_STAR (1) joins the cells of such a junction to a node
 * by their half transmissibilities t_l, eliminated in the primal system
 * (star-delta: t_i t_j / sum_l t_l, the sum over the members in ascending
 * order; two-cell junctions keep t_i t_j / (t_i + t_j)) and an intersection
 * cell with its own pressure and interface fluxes in mds_assemble_flux.
 * `on_device` = 1 means every array pointer below is a device pointer that
 * must stay valid until mds_assemble returns; 0 means host arrays. */
#define MDS_JUNCTION_PAIRWISE 0
#define MDS_JUNCTION_STAR 1
typedef struct {
    int dim;
    int n;
    const double *km;        /* [n^dim] */
    int64_t n_f;
    const int32_t *fc_axis;  /* [n_f]   normal axis 0..dim-1 */
    const int32_t *fc_pos;   /* [3 n_f] (x, y, z) per fracture cell */
    const double *fc_kf;     /* [n_f] */
    const double *fc_a;      /* [n_f] */
    int nrhs;                /* >= 1 */
    const double *pD_left;   /* [nrhs n^(dim-1)] */
    const double *pD_right;  /* [nrhs n^(dim-1)] */
    int on_device;
    int junction;            /* MDS_JUNCTION_* */
    const double *fc_kn;     /* [n_f] normal permeability (kappa = 2 k_n / a), NULL: k_n = k_f */
} mds_instance;

/* Device CSR view.  row_ptr [nrow+1], col/val [nnz]. */
typedef struct {
    int64_t nrow, ncol, nnz;
    int32_t *row_ptr;
    int32_t *col;
    double *val;
} mds_csr;

/* Assemble the block system of one instance on the GPU (Eq. (4)): the four
 * blocks, the full matrix and the nrhs right-hand sides b (column r at
 * b + r (n_m + n_f)).  Fails with MDS_ERR_INVALID on a fracture cell outside
 * the interior faces or two fracture cells on one face. */
int mds_assemble(mds_ctx ctx, const mds_instance *inst, mds_system *out);

/* Assemble one instance in the paper's own partition (Sec. 3.1, Eq. (4)):
 * Omega = the pressures of all N = n_m + n_f cells (matrix cells, then
 * fracture cells), Gamma = the 2 n_f interface fluxes, flux j = 2k + s of
 * fracture cell k on side s (side 0 toward the lower coordinate along the
 * fracture's normal).  Flux row N + j holds +1 at its matrix cell i, -1 at
 * fracture cell n_m + k and -1/T_j at itself (the interface law
 * p_i - p_k - lambda_j / T_j = 0, T_j the matrix-fracture transmissibility
 * of the primal system); its transpose is the flux columns of the pressure
 * rows, whose diagonals keep only the cell-cell and boundary
 * transmissibilities.  The system is symmetric and indefinite; the
 * mds_system reports n_m = N and n_f = 2 n_f, so the Omega/Gamma blocks of
 * every preconditioner are the pressure and flux blocks.  b: the primal
 * right-hand side in the pressure rows, 0 in the flux rows, column r at
 * b + r (N + 2 n_f).  Eliminating the fluxes gives mds_assemble's matrix.
 * With junction = MDS_JUNCTION_STAR each junction of m >= 3 fracture cells
 * (a vertex in 2D, a grid edge in 3D) is an intersection cell appended to
 * Omega after the fracture cells (ordered by its lowest member cell, then by
 * that cell's junction: tangential axes ascending, low end first), and each
 * member l gets a flux lambda = t_l (p_l - p_I) appended to Gamma after the
 * matrix-fracture fluxes (by intersection, then ascending member): its row
 * holds +1 at fracture cell l, -1 at the intersection cell and -1/t_l; the
 * intersection row holds an explicit zero diagonal and -1 per member flux.
 * n_m and n_f of the system then count these as well; eliminating the
 * fluxes and the intersection pressures gives the star-delta primal system.
 * Errors as mds_assemble. */
int mds_assemble_flux(mds_ctx ctx, const mds_instance *inst, mds_system *out);

/* Assemble n_inst independent instances (uneven sizes allowed, equal nrhs)
 * into one packed block-diagonal system.  Unknowns are ordered
 * [matrix cells of instance 0..n_inst-1; fracture cells of instance
 * 0..n_inst-1], so the packed system keeps the 2x2 block structure of
 * Eq. (4) with block-diagonal blocks, and every preconditioner set up on it
 * acts on each instance separately.  mds_solve on such a system solves every
 * (instance, right-hand side) pair as its own problem. */
int mds_assemble_batch(mds_ctx ctx, const mds_instance *inst, int n_inst, mds_system *out);
/* Instances of a packed system: instance k owns matrix rows
 * [m_off[k], m_off[k+1]) and fracture rows n_m + [f_off[k], f_off[k+1]);
 * m_off and f_off have n_inst + 1 entries (either may be NULL). */
int mds_system_instances(mds_system sys, int *n_inst, int64_t *m_off, int64_t *f_off);

/* Wrap caller CSR blocks (device, borrowed until mds_system_destroy) and an
 * optional device right-hand side b [n_m + n_f] (NULL: zero).  The library
 * builds its own merged copy of the full matrix. */
int mds_system_from_csr(mds_ctx ctx, const mds_csr *Amm, const mds_csr *Amf,
                        const mds_csr *Afm, const mds_csr *Aff, const double *b,
                        mds_system *out);
/* Frees the system's own storage (borrowed caller blocks stay the caller's).
 * Preconditioners set up on it must be destroyed first; the context is
 * released here if it was destroyed while this was its last dependent. */
int mds_system_destroy(mds_system sys);
/* Sizes: n_m, n_f, nrhs and nnz of (A_mm, A_mf, A_fm, A_ff, full). */
int mds_system_info(mds_system sys, int64_t *n_m, int64_t *n_f, int *nrhs, int64_t nnz[5]);
/* Borrowed device views of the blocks (index 0..3 = mm, mf, fm, ff), the full
 * matrix (index 4) and the right-hand sides; valid until the system is
 * destroyed. */
int mds_system_view(mds_system sys, mds_csr blocks[5], const double **b);

/* ---- preconditioner set-up ---- */
#define MDS_SMOOTHER_L1JACOBI 0
#define MDS_SMOOTHER_CHEBYSHEV 1
#define MDS_PREC_FP64 64        /* V-cycles stored and applied in FP64 */
#define MDS_PREC_FP32 32        /* FP32 values and vectors */
#define MDS_PREC_BF16 16        /* FP32 vectors; levels >= lowp_from_level stored in BF16 with
                                   power-of-two row scales, finer levels in FP32 */
#define MDS_PREC_FP16 17        /* as MDS_PREC_BF16 with FP16 storage */
#define MDS_PROLONG_PIECEWISE 0 /* piecewise-constant aggregate injection */
#define MDS_PROLONG_SMOOTHED 1  /* smoothed aggregation: P = (I - 4/3 D1F^-1 AF) P0 */
#define MDS_FORMAT_AUTO 0       /* timed choice per level (autotuner) */
#define MDS_FORMAT_CSR 1
#define MDS_FORMAT_SELL 2       /* sliced ELLPACK, slice height sell_c, sort window sell_sigma */
#define MDS_FORMAT_STENCIL 3    /* the finest level of S~ of a primal system assembled by this library
                                   (a 5- or 7-point stencil per Cartesian instance) stored by
                                   diagonals, no column indices; CSR on the other levels.
                                   MDS_FORMAT_AUTO uses it there too when it times fastest */
#define MDS_FORMAT_STENCIL_BULK 4  /* MDS_FORMAT_STENCIL whose kernel stages each 256-row block's
                                      coefficient planes and the window of the vector its
                                      neighbours at +-1 and +-s read into shared memory by bulk
                                      asynchronous copies (cp.async.bulk, mbarrier completion);
                                      the same results bit for bit, where it applies (vectors of
                                      16-byte rows; the direct kernel otherwise).  Slower than
                                      MDS_FORMAT_STENCIL in a solve, so MDS_FORMAT_AUTO does not
                                      choose it */
#define MDS_FORM_AUTO 0         /* the fused form, or the stored one on a level where the storage
                                   autotuner (MDS_FORMAT_AUTO) times it faster */
#define MDS_FORM_FUSED 1        /* a level with a coarser one applies its one L1-Jacobi sweep before
                                   and after the coarse correction in two launches, the smoothed
                                   iterate D1^-1 b (+ P x_c) formed per neighbour, never stored */
#define MDS_FORM_STORED 2       /* the iterate stored: y = D1^-1 b, r = b - A y, y += P x_c,
                                   x = y + D1^-1 (b - A y), four launches; one gather per neighbour
                                   instead of two to four.  The same roundings as the fused form: the
                                   results are equal bit for bit */
#define MDS_BLOCK_LOWER 0       /* M_L, Eq. (8), Algorithm 1 */
#define MDS_BLOCK_DIAG 1        /* block diagonal B_D with Q blocks */
#define MDS_BLOCK_UPPER 2       /* block upper triangular B_U with Q blocks */

typedef struct {
    double theta;            /* strength threshold; < 0 (the default) = 0.08 with piecewise-constant
                                and 0.04 with smoothed prolongation (with 0.04 smoothed aggregation
                                keeps its iteration counts flat over contrast and refinement) */
    int64_t n_coarse;        /* dense Cholesky once a level has <= n_coarse rows (512) */
    int max_levels;          /* (25) */
    double stall_ratio;      /* stop coarsening when n_{l+1} > stall_ratio n_l (0.9) */
    uint64_t seed;           /* MIS-2 hash seed */
    int smoother;            /* MDS_SMOOTHER_* */
    int precision;           /* MDS_PREC_* */
    int lowp_from_level;     /* first BF16/FP16 level for MDS_PREC_BF16/FP16 (1) */
    int kind;                /* MDS_BLOCK_* */
    int format;              /* MDS_FORMAT_* for the V-cycle level matrices (MDS_FORMAT_CSR) */
    int sell_c;              /* SELL slice height: 8, 16 or 32 (32) */
    int sell_sigma;          /* SELL sort window in rows: 1 or a multiple of sell_c up to 1024 (1) */
    int sweeps;              /* smoother applications before and after the coarse correction (1) */
    int prolongation;        /* MDS_PROLONG_* (MDS_PROLONG_PIECEWISE).  Smoothed: AF keeps the
                                strong couplings and adds the weak ones to its diagonal, D1F is
                                its L1 diagonal, A_c = P^T (A P) */
    int coarse_tail;         /* 1: the coarse end of each V-cycle (levels of at most 8192 rows,
                                one L1-Jacobi sweep, unsmoothed, values in the vector type, and
                                the dense solve) runs as one kernel on a thread block cluster;
                                0: one launch per level operation (0: on GB300 the separate
                                launches, overlapped by programmatic dependent launch, measured
                                faster) */
    int cheb_degree;         /* degree of the Chebyshev smoother, 1..8 (2): residual polynomial
                                T_k((theta - t)/delta) / T_k(theta/delta) of D1^-1 A on
                                [0.3, 1] (Saad, Iterative Methods, Alg. 12.1) */
    int level_form;          /* MDS_FORM_* (MDS_FORM_AUTO); levels with one L1-Jacobi sweep, unsmoothed
                                prolongation, FP32 / BF16 / FP16 values or FP64 values of at most
                                65,536 rows (larger FP64 levels always store the iterate) */
} mds_setup_opts;

/* Fill `o` with the defaults listed above. */
int mds_setup_opts_default(mds_setup_opts *o);

/* Build S~ (Eq. (7)) and one aggregation-AMG hierarchy for each of S~ and
 * A_ff: strength graph, MIS-2 with SplitMix64 priorities, aggregates,
 * piecewise-constant P, Galerkin P^T A P, L1 diagonals, coarsest dense
 * Cholesky; then the per-level storage (precision, format) used by the
 * V-cycle, chosen by timing when format = MDS_FORMAT_AUTO.  A level whose
 * rows hold only their diagonal entry (of either sign: the flux block of
 * mds_assemble_flux) ends its hierarchy and is solved exactly, x = b / a_ii.
 * With kind = MDS_BLOCK_DIAG and every diagonal entry of A_ff negative the
 * interface block of B_D is -Q_ff, so that B_D stays positive definite for
 * PCG and MINRES.  The system must outlive the preconditioner. */
int mds_setup(mds_ctx ctx, mds_system sys, const mds_setup_opts *opts, mds_precond *out);
int mds_precond_destroy(mds_precond prec);
/* Hierarchy of block 0 (S~) or 1 (A_ff): number of levels, and per level the
 * rows and nonzeros (arrays of length >= 32).  *dense = 1 when the last level
 * is solved by dense Cholesky, 2 when it has no couplings and is solved by
 * x = b / a_ii, 0 when it is smoothed only. */
int mds_precond_info(mds_precond prec, int block, int *nlevels, int64_t *level_n,
                     int64_t *level_nnz, int *dense);
/* Borrowed device views of level `level` of a block: its FP64 matrix, the
 * aggregate map to the next level (int32 [n], -1 = not aggregated; NULL on
 * the last level) and the MIS-2 root flags (int8 [n]). */
int mds_precond_level(mds_precond prec, int block, int level, mds_csr *A,
                      const int32_t **agg, const int8_t **roots);
/* Borrowed device view of the smoothed prolongator of a level (fine rows x
 * coarse columns); P->nnz = 0 and null arrays when the level uses injection. */
int mds_precond_prolongator(mds_precond prec, int block, int level, mds_csr *P);
/* Borrowed device views of what the V-cycle of a level multiplies by (the
 * storage readings of Sec. 3.3's V-cycle in reduced precision): the value
 * type (MDS_PREC_FP64 / FP32 / BF16 / FP16), the values in the CSR order of
 * mds_precond_level's matrix (for BF16 / FP16: q_ij with a_ij ~ s_i q_ij;
 * NULL on a last level applied through its dense inverse), the float row
 * scales s_i (NULL unless BF16 / FP16), 1/D1 (double for FP64
 * hierarchies, float otherwise) and the storage format the V-cycle reads
 * (MDS_FORMAT_CSR, MDS_FORMAT_SELL or MDS_FORMAT_STENCIL).  Any output
 * pointer may be NULL.  MDS_ERR_INVALID for a block or level that does not
 * exist. */
int mds_precond_level_storage(mds_precond prec, int block, int level, int *value_type,
                              const void **values, const float **row_scale, const void **dinv, int *format);
/* z = M r for device FP64 vectors of length n_m + n_f. */
int mds_precond_apply(mds_ctx ctx, mds_precond prec, const double *r, double *z);
/* x = V(b): one V-cycle of block 0 or 1 on device FP64 vectors. */
int mds_vcycle(mds_ctx ctx, mds_precond prec, int block, const double *b, double *x);
/* y = A x with the full system matrix (device FP64 vectors). */
int mds_spmv(mds_ctx ctx, mds_system sys, const double *x, double *y);

/* ---- solve ---- */
#define MDS_KRYLOV_FGMRES 0  /* right-preconditioned flexible GMRES(restart) (Sec. 3.2) */
#define MDS_KRYLOV_PCG 1     /* preconditioned CG: SPD system and SPD preconditioner (B_D) */
#define MDS_KRYLOV_MINRES 2  /* preconditioned MINRES: symmetric system, SPD preconditioner (B_D);
                                iterations = preconditioner applications after the first */

typedef struct {
    int krylov;          /* MDS_KRYLOV_* */
    int restart;         /* FGMRES restart length (30) */
    double rtol;         /* stop when ||b - A x|| <= rtol ||b|| (1e-8) */
    int max_iters;       /* preconditioner applications per right-hand side (1000) */
    int use_precond;     /* 1 = the set-up preconditioner, 0 = identity */
    int graphs;          /* 1 = capture each Krylov step as a CUDA graph on its first use and
                            replay it (1); 0 = launch every kernel directly */
    int batched;         /* 1 = solve the nrhs columns together in lockstep, each as its own
                            FGMRES problem with shared matrix reads (1); packed multi-instance
                            systems are always solved this way */
    double reorth_eta2;  /* FGMRES runs a second classical Gram-Schmidt pass when
                            ||w_new||^2 < reorth_eta2 ||w||^2 (1e-8; 0.5 = the DGKS rule,
                            >= 1 always); batched solves decide per problem */
    int x0_zero;         /* 1 = the initial guess is zero (the paper's x0, Sec. 4) and x is
                            output only: its contents are not read, and a host x is not
                            copied to the device (0: x holds x0) */
} mds_solve_opts;

typedef struct {
    int iterations;      /* preconditioner applications */
    int restarts;
    int status;          /* MDS_OK, MDS_WARN_NOT_CONVERGED or an error */
    double relres_est;   /* last Arnoldi / recurrence estimate */
    double relres_true;  /* ||b - A x|| / ||b|| recomputed at exit */
} mds_rhs_stats;

int mds_solve_opts_default(mds_solve_opts *o);

/* Solve A x = b for nrhs right-hand sides.  b: [nrhs][n] FP64 (column r at
 * b + r n), NULL = the assembled right-hand sides.  On a packed batch every
 * (instance k, column r) pair is an independent problem with its own
 * stopping test, and stats has n_inst * nrhs entries (index k nrhs + r).  x: [nrhs][n], holds the
 * initial guess on entry (zeros give the x0 = 0 of Sec. 4) and the solution on
 * return.  b and x may be device or host pointers (host ones are staged
 * through device buffers inside the call).  `prec` may be NULL when
 * use_precond = 0.  stats: host array [nrhs], may be NULL.  Returns MDS_OK,
 * MDS_WARN_NOT_CONVERGED or an error. */
int mds_solve(mds_ctx ctx, mds_system sys, mds_precond prec, const double *b, double *x,
              int nrhs, const mds_solve_opts *opts, mds_rhs_stats *stats);

/* ---- solver tuner ----
 * The storage autotuner of mds_setup times kernels; the options that also
 * change convergence (smoother, sweeps, Chebyshev degree, level precision)
 * can only be judged by time to solution.  mds_tune runs, for each
 * candidate, mds_setup with the base options and the candidate's four
 * fields, then mds_solve of b (NULL: the assembled first right-hand side)
 * from x0 = 0 with the given solve options, and records the wall times of
 * both and the outcome.  *best = the converged candidate with the least
 * set-up + solve time (-1 if none converged: MDS_WARN_NOT_CONVERGED).  The
 * trial solution lives in a device buffer of the call; no preconditioner
 * is kept.  Meant for workloads that solve many systems alike (a parameter
 * sweep, many right-hand sides): tune once on a representative one. */
typedef struct {
    int smoother;       /* in: MDS_SMOOTHER_* */
    int sweeps;         /* in: 1..8 */
    int cheb_degree;    /* in: 1..8 */
    int precision;      /* in: MDS_PREC_* */
    int status;         /* out: set-up error, or the solve's status */
    int iterations;     /* out */
    double setup_ms;    /* out: wall time of mds_setup */
    double solve_ms;    /* out: wall time of mds_solve */
    int64_t n_coarse;   /* in: coarsest-level size N_c (dense Cholesky once every instance has at
                           most N_c rows; 1..8192), 0 = the base options' value */
} mds_tune_candidate;
int mds_tune(mds_ctx ctx, mds_system sys, const mds_setup_opts *base, const mds_solve_opts *sopts,
             const double *b, mds_tune_candidate *cands, int n_cands, int *best);

/* The same solve without blocking the calling thread: the solve's host
 * control loop runs on a library thread and mds_solve_async returns at once
 * (MDS_OK when started, or an error for invalid arguments or an uncollected
 * previous solve).  b, x, the system and the preconditioner must stay valid
 * until mds_solve_wait returns.  Any other call on the context (or on a
 * system or preconditioner of it) first waits for the solve to finish, so
 * the context is never used by two threads at once; mds_last_error is
 * meaningful after mds_solve_wait.  Several contexts, each on its own CUDA
 * stream, can thus solve concurrently on one GPU from one host thread: the
 * latency-bound phases of one solve (coarse levels, the host round trip of
 * each Krylov step) overlap with the kernels of the others.  This has no
 * counterpart in the paper; it serves throughput over many independent
 * solves. */
int mds_solve_async(mds_ctx ctx, mds_system sys, mds_precond prec, const double *b, double *x,
                    int nrhs, const mds_solve_opts *opts);
/* 1 when the asynchronous solve has finished, 0 while it runs,
 * MDS_ERR_INVALID when none was started (or it was already collected). */
int mds_solve_done(mds_ctx ctx);
/* Waits for the asynchronous solve, copies its statistics (up to `count`
 * entries, as mds_solve's stats; may be NULL) and returns its status (as
 * mds_solve would).  MDS_ERR_INVALID when no solve is pending. */
int mds_solve_wait(mds_ctx ctx, mds_rhs_stats *stats, int count);

/* ---- solve without device allocation ----
 * The paper has no counterpart to this entry point; it serves callers that
 * cannot allocate device memory while solving: code running inside a
 * framework that owns every allocation (a memory-capped serving process, a
 * caller between pool resets) or a caller that must not synchronise on the
 * allocator.  It runs the same FGMRES as mds_solve (nrhs = 1, kernels
 * launched directly, no CUDA graphs) with its Krylov workspace (bases V and
 * Z, Hessenberg matrix, reduction partials) in one file-scope static device
 * array of MDS_NOALLOC_SCRATCH_BYTES, which every GPU that loads the library
 * holds until the process exits.  It calls no cudaMalloc, cudaFree or other
 * allocating routine.
 *   - n_m + n_f must be <= MDS_NOALLOC_MAX_N and restart <= 30; larger
 *     problems are rejected with MDS_ERR_INVALID, and so is a packed batch
 *     of several instances (mds_solve solves those).
 *   - b (NULL: the assembled right-hand side) and x must be device pointers;
 *     x holds x0 on entry and the solution on return.
 *   - The array exists from the first mds_create on a device onwards:
 *     mds_create resolves its device address (which loads the part of the
 *     library that holds it) with that device current, so a call of this
 *     entry point performs no set-up of its own.
 *   - Every call on a device shares the one array and leaves its contents
 *     behind (the parts that must start at zero are cleared on entry); calls
 *     whose GPU work overlaps, from any context or stream, race on it.
 *   - The preconditioner's own work vectors were allocated by mds_setup. */
#define MDS_NOALLOC_MAX_N 16384
#define MDS_NOALLOC_SCRATCH_BYTES (8u * 1024u * 1024u)
int mds_solve_noalloc(mds_ctx ctx, mds_system sys, mds_precond prec, const double *b, double *x,
                      const mds_solve_opts *opts, mds_rhs_stats *stats);

/* ---- measurement ----
 * Kernel classes timed with CUDA events on the context stream when enabled:
 * 0 = full-system SpMV, 1 = V-cycle residual (pre-smooth + residual),
 * 2 = V-cycle post-smooth (prolongation + correction + smoothing),
 * 3 = Gram-Schmidt dot products, 4 = Gram-Schmidt updates, 5 = all V-cycle
 * kernels together, 6 = restriction.  Classes 1, 2 and 6 count the kernels of
 * the finest level of hierarchies with at least 65536 rows (the coarser
 * levels' kernels are counted in no class).  Bytes are algorithmic (each
 * matrix and vector byte counted once per launch). */
#define MDS_KCLASS_COUNT 8
int mds_timing_enable(mds_ctx ctx, int kclass, int enable);
int mds_timing_reset(mds_ctx ctx);
/* Synchronises the stream; returns launches, summed event time (ms), summed
 * algorithmic bytes and summed algorithmic floating-point operations of a
 * class since the last reset (any output pointer may be NULL). */
int mds_timing_query(mds_ctx ctx, int kclass, int64_t *launches, double *ms, double *bytes, double *flops);
/* Event brackets cost a few microseconds of pipeline time each (they end the
 * programmatic overlap of neighbouring kernels).  With every = k > 1, FGMRES
 * brackets the timed classes only in every k-th restart cycle (its Arnoldi
 * steps are replayed from a second, bracketed CUDA graph); other launches run
 * unbracketed.  Default 1: every launch of a timed class is bracketed. */
int mds_timing_sample_every(mds_ctx ctx, int every);
/* Like mds_timing_query, restricted to the launches that were bracketed:
 * their count, event time, algorithmic bytes and operations.  Their ratios
 * are the measured per-launch averages when sampling. */
int mds_timing_sampled(mds_ctx ctx, int kclass, int64_t *launches, double *ms, double *bytes, double *flops);
/* Copy `bytes` bytes from src to dst (each a host or device pointer) on the
 * context stream and synchronise it.  A convenience for callers without
 * their own CUDA runtime binding. */
int mds_memcpy(mds_ctx ctx, void *dst, const void *src, size_t bytes);

/* Number of kernels the library launched since the last reset (all classes). */
int mds_launch_count(mds_ctx ctx, int64_t *launches);

#ifdef __cplusplus
}
#endif
#endif
