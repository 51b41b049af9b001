/* Oracle for the mixed-dimensional block solver: TEST INFRASTRUCTURE ONLY.
 *
 * Plain sequential FP64 C.  Loaded only by the tests, the smoke check and the
 * benchmark's CPU-baseline leg and reference arm.  Nothing here is shared with
 * the CUDA library.
 * Compiled with -ffp-contract=off so every product and sum is rounded exactly
 * as written.
 *
 * Citations are to Hu, Keilegavlen, Nordbotten, arXiv:2206.03203.
 */
#include "mdoracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ CSR */

ocsr *orc_csr_new(int64_t nrow, int64_t ncol, int64_t nnz) {
    ocsr *A = (ocsr *)calloc(1, sizeof(ocsr));
    if (!A) return NULL;
    A->nrow = nrow;
    A->ncol = ncol;
    A->nnz = nnz;
    A->rp = (int64_t *)calloc((size_t)nrow + 1, sizeof(int64_t));
    A->ci = (int32_t *)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int32_t));
    A->v = (double *)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(double));
    if (!A->rp || !A->ci || !A->v) {
        orc_csr_free(A);
        return NULL;
    }
    return A;
}

void orc_csr_free(ocsr *A) {
    if (!A) return;
    free(A->rp);
    free(A->ci);
    free(A->v);
    free(A);
}

void orc_spmv(const ocsr *A, const double *x, double *y) {
    for (int64_t i = 0; i < A->nrow; i++) {
        double s = 0.0;
        for (int64_t p = A->rp[i]; p < A->rp[i + 1]; p++) s += A->v[p] * x[A->ci[p]];
        y[i] = s;
    }
}

static double dot(int64_t n, const double *a, const double *b) {
    double s = 0.0;
    for (int64_t i = 0; i < n; i++) s += a[i] * b[i];
    return s;
}

static double nrm2(int64_t n, const double *a) { return sqrt(dot(n, a, a)); }

/* Growable (col, T) list used while building one row. */
typedef struct {
    int32_t c;
    double t;
} entry;

static int cmp_entry(const void *a, const void *b) {
    int32_t x = ((const entry *)a)->c, y = ((const entry *)b)->c;
    return (x > y) - (x < y);
}

/* ------------------------------------------------------------ assembly */
/* Two-point flux approximation on the Cartesian grid (Sec. 2.1: Eq. (1) in
 * each subdomain, Eq. (2)-(3) across each matrix-fracture interface), with
 * the interface flux eliminated into a matrix-fracture transmissibility:
 *   matrix-matrix     T = |F| / (h/(2k_i) + h/(2k_j))        (harmonic mean)
 *   matrix-fracture   T = |F| / (h/(2k_i) + 1/kappa), kappa = 2 k_n / a
 *                     (Eq. (2): interface law, kappa from the normal
 *                     permeability k_n, which is k_f unless given)
 *   fracture-fracture half transmissibilities t = k_f a |e| / (h/2) at the
 *                     shared vertex (2D) / edge (3D) e, every pair of cells at
 *                     e linked by t_i t_j / (t_i + t_j)
 *   Dirichlet         matrix: T_b = |F| 2k/h; fracture end: T_b = t
 * Rows: A_ii = sum of the row's T (ascending column, then Dirichlet terms),
 * A_ij = -T_ij; unknowns ordered [matrix cells (x fastest); fracture cells]
 * as the 2x2 block system of Eq. (4).  Parity pins: linear-field exactness,
 * series and parallel closed forms, symmetry, row sums, SPD. */

typedef struct {
    int dim, n;
    int64_t ext[3][3]; /* face-array extents per normal axis */
    int32_t *map[3];   /* face -> fracture cell, -1 if none */
} facemap;

static int64_t face_id(const facemap *fm, int d, int64_t x, int64_t y, int64_t z) {
    const int64_t *e = fm->ext[d];
    if (x < 0 || y < 0 || z < 0 || x >= e[0] || y >= e[1] || z >= e[2]) return -1;
    return x + e[0] * (y + e[1] * z);
}

static int32_t face_frac(const facemap *fm, int d, const int64_t c[3]) {
    int64_t f = face_id(fm, d, c[0], c[1], c[2]);
    return f < 0 ? -1 : fm->map[d][f];
}

/* Junction q of fracture cell k: the vertex (2D) or edge (3D) closing the
 * cell along its (q/2)-th tangential axis e (ascending axes), on the low
 * (q even) or high (q odd) side.  The fracture cells incident to it are the
 * faces normal to the cell's own axis d on either side along e and the faces
 * normal to e on either side along d.  Writes them (k included) ascending to
 * J and returns their number, or 0 for an end on a Dirichlet face (x = 0 or
 * x = 1), which joins no other cell; *e_out = e. */
static int junction_members(const facemap *fm, const int32_t *fc_axis, const int32_t *fc_pos, int64_t k, int q,
                            int *e_out, int32_t J[5]) {
    const int dim = fm->dim, n = fm->n;
    const int d = fc_axis[k];
    const int32_t *p = fc_pos + 3 * k;
    int64_t c[3] = {p[0], p[1], dim == 3 ? p[2] : 0};
    int e = -1;
    for (int a = 0, seen = 0; a < dim; a++) {
        if (a == d) continue;
        if (seen++ == q / 2) {
            e = a;
            break;
        }
    }
    *e_out = e;
    int64_t u = c[e] + (q & 1);
    if (e == 0 && (u == 0 || u == n)) return 0;
    int64_t cand[4][3];
    int cd[4];
    for (int r = 0; r < 4; r++) {
        cand[r][0] = c[0];
        cand[r][1] = c[1];
        cand[r][2] = c[2];
    }
    cand[0][e] = u - 1; cd[0] = d;
    cand[1][e] = u;     cd[1] = d;
    cand[2][e] = u; cand[2][d] = c[d] - 1; cd[2] = e;
    cand[3][e] = u; cand[3][d] = c[d];     cd[3] = e;
    int m = 0;
    J[m++] = (int32_t)k;
    for (int r = 0; r < 4; r++) {
        int32_t l = face_frac(fm, cd[r], cand[r]);
        if (l >= 0 && l != k) J[m++] = l;
    }
    for (int a = 1; a < m; a++) /* insertion sort, ascending */
        for (int b2 = a; b2 > 0 && J[b2 - 1] > J[b2]; b2--) {
            int32_t t = J[b2];
            J[b2] = J[b2 - 1];
            J[b2 - 1] = t;
        }
    return m;
}

/* flux = 0: the primal system above.  flux = 1: the paper's own partition
 * (Sec. 3.1, Eq. (4)): unknowns [pressures of all cells; interface fluxes],
 * one flux lambda_j per matrix-fracture face side, j = 2k + side (side 0 =
 * the matrix cell below the fracture face, 1 = above), in the order of the
 * fracture cells.  The pressure rows keep the matrix-matrix,
 * fracture-fracture and Dirichlet terms (diagonal = their sum, same order);
 * matrix cell i gets +lambda_j and fracture cell k gets -lambda_j (mass
 * leaving i enters k); row j is the interface law of Eq. (2) written as
 * p_i - p_k - lambda_j / T_j = 0 with T_j the series transmissibility of the
 * matrix half cell and the normal coupling.  A_{Gamma Omega} = A_{Omega
 * Gamma}^T and A_{Gamma Gamma} = diag(-1/T_j): symmetric indefinite;
 * eliminating lambda gives the primal system.
 *
 * junction = 0: every pair of fracture cells at a junction is linked by
 * t_i t_j / (t_i + t_j).  junction = 1: a junction of m >= 3 cells is a node
 * joined to each of its cells by the cell's half transmissibility t_l.
 * Primal form: the node is eliminated (star-delta), T_ij = t_i t_j / sum_l
 * t_l with the sum in ascending cell order (equal to the pairwise rule when
 * m = 2).  Flux form: the node is an intersection cell (a subdomain of
 * dimension N-2, Sec. 2.1) with its own pressure, appended to Omega after the
 * fracture cells, and each member l gets an interface flux
 * lambda = t_l (p_l - p_I) (the fracture is the higher-dimensional side),
 * appended to Gamma after the matrix-fracture fluxes.  Intersection cells are
 * numbered by their lowest member cell, then by that cell's junction index;
 * their fluxes by intersection, then ascending member.  An intersection row
 * holds an explicit zero diagonal (no pressure-pressure term) and -1 per
 * flux.  Eliminating the fluxes and then the intersection pressures gives the
 * star-delta primal system.  *n_omega = the number of pressure unknowns; b
 * is written to the caller's array, or allocated (*b_out) when b is NULL. */
static ocsr *assemble_impl(int dim, int n, const double *km, int64_t nf,
                           const int32_t *fc_axis, const int32_t *fc_pos,
                           const double *fc_kf, const double *fc_a, int nrhs,
                           const double *pD_left, const double *pD_right, double *b, int flux, int junction,
                           int64_t *n_omega, double **b_out, const double *fc_kn) {
    /* normal permeability of each fracture cell (kappa = 2 k_n / a); the
     * tangential one k_f when not given */
    const double *kn = fc_kn ? fc_kn : fc_kf;
    if ((dim != 2 && dim != 3) || n < 1 || nrhs < 1 || junction < 0 || junction > 1) return NULL;
    const double h = 1.0 / (double)n;
    const double F = dim == 2 ? h : h * h;      /* face measure |F| */
    const double elen = dim == 2 ? 1.0 : h;     /* fracture edge measure |e| */
    const int64_t nz = dim == 3 ? n : 1;
    const int64_t n_m = (int64_t)n * n * nz;
    const int64_t N = n_m + nf;             /* matrix and fracture cells */
    const int nslot = 2 * (dim - 1);        /* junctions per fracture cell */
    ocsr *A = NULL;
    int32_t *jid = NULL, *isz = NULL, *imem = NULL;
    int64_t *ioff = NULL;
    int64_t nI = 0, nIF = 0;

    facemap fm;
    memset(&fm, 0, sizeof fm);
    fm.dim = dim;
    fm.n = n;
    for (int d = 0; d < 3; d++) {
        for (int a = 0; a < 3; a++) fm.ext[d][a] = (a < dim) ? (a == d ? n + 1 : n) : 1;
        if (d >= dim) continue;
        int64_t sz = fm.ext[d][0] * fm.ext[d][1] * fm.ext[d][2];
        fm.map[d] = (int32_t *)malloc((size_t)sz * sizeof(int32_t));
        for (int64_t q = 0; q < sz; q++) fm.map[d][q] = -1;
    }
    for (int64_t k = 0; k < nf; k++) {
        int d = fc_axis[k];
        const int32_t *p = fc_pos + 3 * k;
        if (d < 0 || d >= dim || p[d] < 1 || p[d] > n - 1) goto bad;
        int64_t f = face_id(&fm, d, p[0], p[1], dim == 3 ? p[2] : 0);
        if (f < 0 || fm.map[d][f] != -1) goto bad; /* outside, or a duplicate face */
        fm.map[d][f] = (int32_t)k;
    }

    /* intersection cells: junctions of >= 3 fracture cells, created by their
     * lowest member; every member's junction slot is found by comparing
     * member sets (two cells share at most one junction) */
    if (flux && junction) {
        jid = (int32_t *)malloc((size_t)(nf > 0 ? nf : 1) * 4 * sizeof(int32_t));
        isz = (int32_t *)malloc((size_t)(nf > 0 ? 2 * nf : 1) * sizeof(int32_t));
        imem = (int32_t *)malloc((size_t)(nf > 0 ? 2 * nf : 1) * 4 * sizeof(int32_t));
        for (int64_t q = 0; q < nf * 4; q++) jid[q] = -1;
        int32_t J[5], J2[5];
        int e;
        for (int64_t k = 0; k < nf; k++)
            for (int q = 0; q < nslot; q++) {
                int m = junction_members(&fm, fc_axis, fc_pos, k, q, &e, J);
                if (m >= 3 && J[0] == k) {
                    isz[nI] = m;
                    for (int r = 0; r < m; r++) imem[nI * 4 + r] = J[r];
                    nI++;
                }
            }
        ioff = (int64_t *)malloc((size_t)(nI + 1) * sizeof(int64_t));
        ioff[0] = 0;
        for (int64_t id = 0; id < nI; id++) {
            ioff[id + 1] = ioff[id] + isz[id];
            for (int r = 0; r < isz[id]; r++) {
                int32_t l = imem[id * 4 + r];
                for (int ql = 0; ql < nslot; ql++) {
                    int m2 = junction_members(&fm, fc_axis, fc_pos, l, ql, &e, J2);
                    if (m2 != isz[id]) continue;
                    int same = 1;
                    for (int t = 0; t < m2; t++) same &= J2[t] == imem[id * 4 + t];
                    if (same) {
                        jid[(int64_t)l * 4 + ql] = (int32_t)id;
                        break;
                    }
                }
            }
        }
        nIF = ioff[nI];
    }
    const int64_t NO = N + nI;                        /* pressure unknowns (Omega) */
    const int64_t GF = NO + 2 * nf;                   /* first intersection flux */
    const int64_t NT = flux ? GF + nIF : N;           /* all unknowns */
    const int64_t nb = dim == 3 ? (int64_t)n * n : n; /* boundary faces per x side */
    if (n_omega) *n_omega = flux ? NO : n_m;
    if (!b) {
        b = (double *)malloc((size_t)(NT * nrhs > 0 ? NT * nrhs : 1) * sizeof(double));
        if (!b) goto bad;
        *b_out = b;
    }

    /* count pass: an upper bound per row, then exact fill */
    int64_t cap = n_m * (1 + 2 * dim) + nf * (1 + 2 + 4 * 3) + (flux ? 6 * nf : 0) + 5 * nI + 3 * nIF;
    A = orc_csr_new(NT, NT, cap);
    if (!A) goto bad;
    for (int r = 0; r < nrhs; r++)
        for (int64_t i = 0; i < NT; i++) b[(int64_t)r * NT + i] = 0.0;

    /* entries: t is the transmissibility of a pressure column (written as
     * -t) or the value itself of a flux column (+1 / -1) */
    entry row[32];
    int64_t pos = 0;
    /* matrix rows */
    for (int64_t cz = 0; cz < nz; cz++)
        for (int64_t cy = 0; cy < n; cy++)
            for (int64_t cx = 0; cx < n; cx++) {
                int64_t i = cx + n * (cy + n * cz);
                int64_t c[3] = {cx, cy, cz};
                double ki = km[i];
                int cnt = 0;
                double tb[2] = {0.0, 0.0};
                int has_tb[2] = {0, 0};
                for (int d = 0; d < dim; d++) {
                    for (int s = 0; s < 2; s++) {
                        int64_t plane = c[d] + s;
                        int64_t fc[3] = {c[0], c[1], c[2]};
                        fc[d] = plane;
                        if (plane == 0 || plane == n) {
                            if (d == 0) { /* Dirichlet face x=0 (s=0) or x=1 (s=1) */
                                tb[s] = (F * (2.0 * ki)) / h;
                                has_tb[s] = 1;
                            }
                            continue;
                        }
                        int32_t k = face_frac(&fm, d, fc);
                        if (k >= 0) {
                            double kappa = (2.0 * kn[k]) / fc_a[k];
                            if (flux) {
                                /* the interface flux column, side 0 when the
                                 * face is above this cell (s = 1) */
                                row[cnt].c = (int32_t)(NO + 2 * k + (s ? 0 : 1));
                                row[cnt].t = 1.0;
                            } else {
                                row[cnt].c = (int32_t)(n_m + k);
                                row[cnt].t = F / (h / (2.0 * ki) + 1.0 / kappa);
                            }
                        } else {
                            int64_t nc[3] = {c[0], c[1], c[2]};
                            nc[d] = c[d] + (s ? 1 : -1);
                            int64_t j = nc[0] + n * (nc[1] + n * nc[2]);
                            row[cnt].c = (int32_t)j;
                            row[cnt].t = F / (h / (2.0 * ki) + h / (2.0 * km[j]));
                        }
                        cnt++;
                    }
                }
                qsort(row, (size_t)cnt, sizeof(entry), cmp_entry);
                double diag = 0.0;
                for (int q = 0; q < cnt; q++)
                    if (row[q].c < NO) diag += row[q].t; /* flux columns carry no transmissibility */
                for (int s = 0; s < 2; s++)
                    if (has_tb[s]) diag += tb[s];
                int64_t bf = cy + n * cz;
                for (int r = 0; r < nrhs; r++) {
                    double acc = 0.0;
                    if (has_tb[0]) acc += tb[0] * pD_left[(int64_t)r * nb + bf];
                    if (has_tb[1]) acc += tb[1] * pD_right[(int64_t)r * nb + bf];
                    b[(int64_t)r * NT + i] = acc;
                }
                int placed = 0;
                for (int q = 0; q < cnt; q++) {
                    if (!placed && row[q].c > i) {
                        A->ci[pos] = (int32_t)i;
                        A->v[pos++] = diag;
                        placed = 1;
                    }
                    A->ci[pos] = row[q].c;
                    A->v[pos++] = row[q].c < NO ? -row[q].t : row[q].t;
                }
                if (!placed) {
                    A->ci[pos] = (int32_t)i;
                    A->v[pos++] = diag;
                }
                A->rp[i + 1] = pos;
            }
    /* fracture rows */
    for (int64_t k = 0; k < nf; k++) {
        int d = fc_axis[k];
        const int32_t *p = fc_pos + 3 * k;
        int64_t c[3] = {p[0], p[1], dim == 3 ? p[2] : 0};
        int64_t plane = c[d];
        double kappa = (2.0 * kn[k]) / fc_a[k];
        double tk = ((fc_kf[k] * fc_a[k]) * elen) / (0.5 * h);
        int cnt = 0;
        /* the two matrix cells on either side of the face */
        for (int s = 0; s < 2; s++) {
            int64_t mc[3] = {c[0], c[1], c[2]};
            mc[d] = plane - 1 + s;
            int64_t j = mc[0] + n * (mc[1] + n * mc[2]);
            if (flux) {
                row[cnt].c = (int32_t)(NO + 2 * k + s);
                row[cnt].t = -1.0;
            } else {
                row[cnt].c = (int32_t)j;
                row[cnt].t = F / (h / (2.0 * km[j]) + 1.0 / kappa);
            }
            cnt++;
        }
        /* junctions: along each tangential axis, low (s=0) and high (s=1) end */
        double tb[2] = {0.0, 0.0};
        int has_tb[2] = {0, 0};
        int64_t bfa[2] = {0, 0}, bfb[2] = {0, 0};
        for (int q = 0; q < nslot; q++) {
            int32_t J[5];
            int e;
            int m = junction_members(&fm, fc_axis, fc_pos, k, q, &e, J);
            if (m == 0) {
                int side = q & 1; /* x = 0 (low end) or x = 1 (high end) */
                tb[side] = tk;
                has_tb[side] = 1;
                /* boundary faces sharing the end: d-cells plane-1 and plane */
                int64_t fa[3] = {c[0], c[1], c[2]}, fb[3] = {c[0], c[1], c[2]};
                fa[d] = plane - 1;
                fb[d] = plane;
                bfa[side] = fa[1] + n * fa[2];
                bfb[side] = fb[1] + n * fb[2];
                continue;
            }
            if (flux && junction && m >= 3) {
                /* the flux to this junction's intersection cell */
                int32_t id = jid[k * 4 + q];
                int rank = 0;
                while (J[rank] != k) rank++;
                row[cnt].c = (int32_t)(GF + ioff[id] + rank);
                row[cnt].t = 1.0;
                cnt++;
                continue;
            }
            double S = 0.0;
            if (junction)
                for (int r = 0; r < m; r++) S += ((fc_kf[J[r]] * fc_a[J[r]]) * elen) / (0.5 * h);
            for (int r = 0; r < m; r++) {
                int32_t l = J[r];
                if (l == k) continue;
                double tl = ((fc_kf[l] * fc_a[l]) * elen) / (0.5 * h);
                row[cnt].c = (int32_t)(n_m + l);
                row[cnt].t = junction ? (tk * tl) / S : (tk * tl) / (tk + tl);
                cnt++;
            }
        }
        qsort(row, (size_t)cnt, sizeof(entry), cmp_entry);
        double diag = 0.0;
        for (int q = 0; q < cnt; q++)
            if (row[q].c < NO) diag += row[q].t;
        for (int s = 0; s < 2; s++)
            if (has_tb[s]) diag += tb[s];
        for (int r = 0; r < nrhs; r++) {
            double acc = 0.0;
            for (int s = 0; s < 2; s++) {
                if (!has_tb[s]) continue;
                const double *pd = (s == 0 ? pD_left : pD_right) + (int64_t)r * nb;
                double pv = (pd[bfa[s]] + pd[bfb[s]]) * 0.5;
                acc += tb[s] * pv;
            }
            b[(int64_t)r * NT + n_m + k] = acc;
        }
        int64_t self = n_m + k;
        int placed = 0;
        for (int q = 0; q < cnt; q++) {
            if (!placed && row[q].c > self) {
                A->ci[pos] = (int32_t)self;
                A->v[pos++] = diag;
                placed = 1;
            }
            A->ci[pos] = row[q].c;
            A->v[pos++] = row[q].c < NO ? -row[q].t : row[q].t;
        }
        if (!placed) {
            A->ci[pos] = (int32_t)self;
            A->v[pos++] = diag;
        }
        A->rp[self + 1] = pos;
    }
    /* intersection rows: zero diagonal, -1 per flux (mass entering from each
     * member fracture cell) */
    for (int64_t id = 0; id < nI; id++) {
        int64_t self = N + id;
        A->ci[pos] = (int32_t)self;
        A->v[pos++] = 0.0;
        for (int r = 0; r < isz[id]; r++) {
            A->ci[pos] = (int32_t)(GF + ioff[id] + r);
            A->v[pos++] = -1.0;
        }
        A->rp[self + 1] = pos;
    }
    /* flux rows: lambda_j (fracture k, side s): p_i - p_k - lambda_j / T_j = 0 */
    for (int64_t k = 0; flux && k < nf; k++) {
        int d = fc_axis[k];
        const int32_t *p = fc_pos + 3 * k;
        double kappa = (2.0 * kn[k]) / fc_a[k];
        for (int s = 0; s < 2; s++) {
            int64_t mc[3] = {p[0], p[1], dim == 3 ? p[2] : 0};
            mc[d] = p[d] - 1 + s;
            int64_t i = mc[0] + n * (mc[1] + n * mc[2]);
            double t = F / (h / (2.0 * km[i]) + 1.0 / kappa);
            int64_t j = NO + 2 * k + s;
            A->ci[pos] = (int32_t)i;
            A->v[pos++] = 1.0;
            A->ci[pos] = (int32_t)(n_m + k);
            A->v[pos++] = -1.0;
            A->ci[pos] = (int32_t)j;
            A->v[pos++] = -1.0 / t;
            A->rp[j + 1] = pos;
        }
    }
    /* intersection fluxes: lambda (member l of intersection I):
     * p_l - p_I - lambda / t_l = 0 */
    for (int64_t id = 0; id < nI; id++)
        for (int r = 0; r < isz[id]; r++) {
            int32_t l = imem[id * 4 + r];
            double tl = ((fc_kf[l] * fc_a[l]) * elen) / (0.5 * h);
            int64_t j = GF + ioff[id] + r;
            A->ci[pos] = (int32_t)(n_m + l);
            A->v[pos++] = 1.0;
            A->ci[pos] = (int32_t)(N + id);
            A->v[pos++] = -1.0;
            A->ci[pos] = (int32_t)j;
            A->v[pos++] = -1.0 / tl;
            A->rp[j + 1] = pos;
        }
    A->nnz = pos;
    for (int d = 0; d < 3; d++) free(fm.map[d]);
    free(jid);
    free(isz);
    free(imem);
    free(ioff);
    return A;
bad:
    for (int d = 0; d < 3; d++) free(fm.map[d]);
    free(jid);
    free(isz);
    free(imem);
    free(ioff);
    orc_csr_free(A);
    return NULL;
}

ocsr *orc_assemble(int dim, int n, const double *km, int64_t nf,
                   const int32_t *fc_axis, const int32_t *fc_pos,
                   const double *fc_kf, const double *fc_a, int nrhs,
                   const double *pD_left, const double *pD_right, double *b) {
    return assemble_impl(dim, n, km, nf, fc_axis, fc_pos, fc_kf, fc_a, nrhs, pD_left, pD_right, b, 0, 0, NULL,
                         NULL, NULL);
}

ocsr *orc_assemble_flux(int dim, int n, const double *km, int64_t nf,
                        const int32_t *fc_axis, const int32_t *fc_pos,
                        const double *fc_kf, const double *fc_a, int nrhs,
                        const double *pD_left, const double *pD_right, double *b) {
    return assemble_impl(dim, n, km, nf, fc_axis, fc_pos, fc_kf, fc_a, nrhs, pD_left, pD_right, b, 1, 0, NULL,
                         NULL, NULL);
}

ocsr *orc_assemble_ex(int dim, int n, const double *km, int64_t nf,
                      const int32_t *fc_axis, const int32_t *fc_pos,
                      const double *fc_kf, const double *fc_a, int nrhs,
                      const double *pD_left, const double *pD_right, int flux, int junction,
                      int64_t *n_omega, double **b_out, const double *fc_kn) {
    *b_out = NULL;
    ocsr *A = assemble_impl(dim, n, km, nf, fc_axis, fc_pos, fc_kf, fc_a, nrhs, pD_left, pD_right, NULL, flux,
                            junction, n_omega, b_out, fc_kn);
    if (!A) {
        free(*b_out);
        *b_out = NULL;
    }
    return A;
}

void orc_free(void *p) { free(p); }

/* Slice the full system into the blocks of Eq. (4). */
int orc_split(const ocsr *A, int64_t n_m, ocsr **Amm, ocsr **Amf, ocsr **Afm, ocsr **Aff) {
    int64_t N = A->nrow, n_f = N - n_m;
    int64_t cnt[4] = {0, 0, 0, 0};
    for (int64_t i = 0; i < N; i++)
        for (int64_t p = A->rp[i]; p < A->rp[i + 1]; p++)
            cnt[(i >= n_m) * 2 + (A->ci[p] >= n_m)]++;
    ocsr *B[4];
    B[0] = orc_csr_new(n_m, n_m, cnt[0]);
    B[1] = orc_csr_new(n_m, n_f, cnt[1]);
    B[2] = orc_csr_new(n_f, n_m, cnt[2]);
    B[3] = orc_csr_new(n_f, n_f, cnt[3]);
    int64_t at[4] = {0, 0, 0, 0};
    for (int64_t i = 0; i < N; i++) {
        int rb = i >= n_m;
        int64_t li = i - (rb ? n_m : 0);
        for (int64_t p = A->rp[i]; p < A->rp[i + 1]; p++) {
            int cb = A->ci[p] >= n_m;
            ocsr *T = B[rb * 2 + cb];
            int64_t q = at[rb * 2 + cb]++;
            T->ci[q] = A->ci[p] - (int32_t)(cb ? n_m : 0);
            T->v[q] = A->v[p];
        }
        B[rb * 2 + 0]->rp[li + 1] = at[rb * 2 + 0];
        B[rb * 2 + 1]->rp[li + 1] = at[rb * 2 + 1];
    }
    *Amm = B[0];
    *Amf = B[1];
    *Afm = B[2];
    *Aff = B[3];
    return 0;
}

/* --------------------------------------------------------------- Schur */
/* Eq. (7): S~ = A_mm - A_mf diag(A_ff)^-1 A_fm.  Entry (i,j) starts from
 * (A_mm)_ij (0 if absent) and subtracts (A_mf)_ik (A_fm)_kj / d_k for each k
 * of row i of A_mf in ascending order.  Pinned against a dense product. */
ocsr *orc_schur(const ocsr *Amm, const ocsr *Amf, const ocsr *Afm, const ocsr *Aff) {
    int64_t nm = Amm->nrow, nf = Aff->nrow;
    double *dk = (double *)malloc((size_t)(nf > 0 ? nf : 1) * sizeof(double));
    for (int64_t k = 0; k < nf; k++) {
        dk[k] = 0.0;
        for (int64_t p = Aff->rp[k]; p < Aff->rp[k + 1]; p++)
            if (Aff->ci[p] == k) dk[k] = Aff->v[p];
        if (dk[k] == 0.0) {
            free(dk);
            return NULL;
        }
    }
    /* dense accumulator per row */
    double *acc = (double *)calloc((size_t)nm, sizeof(double));
    int8_t *mark = (int8_t *)calloc((size_t)nm, 1);
    int32_t *cols = (int32_t *)malloc((size_t)nm * sizeof(int32_t));
    int64_t cap = Amm->nnz + 4 * Amf->nnz + 16;
    ocsr *S = orc_csr_new(nm, nm, cap);
    int64_t pos = 0;
    for (int64_t i = 0; i < nm; i++) {
        int ncols = 0;
        for (int64_t p = Amm->rp[i]; p < Amm->rp[i + 1]; p++) {
            int32_t j = Amm->ci[p];
            acc[j] = Amm->v[p];
            mark[j] = 1;
            cols[ncols++] = j;
        }
        for (int64_t p = Amf->rp[i]; p < Amf->rp[i + 1]; p++) {
            int32_t k = Amf->ci[p];
            for (int64_t q = Afm->rp[k]; q < Afm->rp[k + 1]; q++) {
                int32_t j = Afm->ci[q];
                if (!mark[j]) {
                    mark[j] = 1;
                    acc[j] = 0.0;
                    cols[ncols++] = j;
                }
                acc[j] = acc[j] - (Amf->v[p] * Afm->v[q]) / dk[k];
            }
        }
        /* sort columns (insertion sort; rows are short) */
        for (int a = 1; a < ncols; a++) {
            int32_t x = cols[a];
            int q = a - 1;
            while (q >= 0 && cols[q] > x) {
                cols[q + 1] = cols[q];
                q--;
            }
            cols[q + 1] = x;
        }
        if (pos + ncols > cap) { /* grow */
            cap = 2 * cap + ncols;
            S->ci = (int32_t *)realloc(S->ci, (size_t)cap * sizeof(int32_t));
            S->v = (double *)realloc(S->v, (size_t)cap * sizeof(double));
        }
        for (int a = 0; a < ncols; a++) {
            S->ci[pos] = cols[a];
            S->v[pos++] = acc[cols[a]];
            mark[cols[a]] = 0;
        }
        S->rp[i + 1] = pos;
    }
    S->nnz = pos;
    free(dk);
    free(acc);
    free(mark);
    free(cols);
    return S;
}

/* ----------------------------------------------------------------- AMG */
/* One V-cycle of aggregation AMG per diagonal block (Sec. 3.3).  The paper
 * uses smoothed aggregation with Gauss-Seidel; this follows the variant the
 * GPU path implements: strength graph, greedy maximal independent set on the
 * square of the strength graph (MIS-2) in hash-priority order, aggregates of
 * roots plus distance-1 and distance-2 vertices, piecewise-constant P, and
 * Galerkin coarse operators P^T A P; L1-Jacobi smoothing; dense Cholesky on
 * the coarsest level.  Pins: aggregate partition/connectivity, MIS-2
 * distance/maximality, brute-force P^T A P, exact solve with one level. */

static uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

#define GOLDEN 0x9E3779B97F4A7C15ULL

uint64_t orc_mis_key(uint64_t seed, int level, int64_t i) {
    uint64_t lk = mix64(seed + GOLDEN * (uint64_t)(level + 1));
    uint64_t hv = mix64(lk + GOLDEN * (uint64_t)(i + 1));
    return (hv & 0xFFFFFFFF00000000ULL) | (uint64_t)(uint32_t)i;
}

static double find_val(const ocsr *A, int64_t i, int64_t j, int *found) {
    for (int64_t p = A->rp[i]; p < A->rp[i + 1]; p++)
        if (A->ci[p] == j) {
            *found = 1;
            return A->v[p];
        }
    *found = 0;
    return 0.0;
}

/* j != i is strong for i when a_ij^2 >= (theta^2 a_ii) a_jj; the graph
 * links i and j when either direction is strong. */
ocsr *orc_strength(const ocsr *A, double theta) {
    int64_t n = A->nrow;
    double th2 = theta * theta;
    double *dg = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    for (int64_t i = 0; i < n; i++) {
        int f;
        dg[i] = find_val(A, i, i, &f);
    }
    int8_t *s = (int8_t *)calloc((size_t)(A->nnz > 0 ? A->nnz : 1), 1);
    for (int64_t i = 0; i < n; i++)
        for (int64_t p = A->rp[i]; p < A->rp[i + 1]; p++) {
            int64_t j = A->ci[p];
            if (j == i) continue;
            double a = A->v[p];
            s[p] = (a * a) >= (th2 * dg[i]) * dg[j];
        }
    int64_t cnt = 0;
    int8_t *g = (int8_t *)calloc((size_t)(A->nnz > 0 ? A->nnz : 1), 1);
    for (int64_t i = 0; i < n; i++)
        for (int64_t p = A->rp[i]; p < A->rp[i + 1]; p++) {
            int64_t j = A->ci[p];
            if (j == i) continue;
            int sym = 0;
            for (int64_t q = A->rp[j]; q < A->rp[j + 1]; q++)
                if (A->ci[q] == i) sym = s[q];
            g[p] = s[p] || sym;
            cnt += g[p];
        }
    ocsr *G = orc_csr_new(n, n, cnt);
    int64_t pos = 0;
    for (int64_t i = 0; i < n; i++) {
        for (int64_t p = A->rp[i]; p < A->rp[i + 1]; p++)
            if (g[p]) {
                G->ci[pos] = A->ci[p];
                G->v[pos++] = A->v[p];
            }
        G->rp[i + 1] = pos;
    }
    free(dg);
    free(s);
    free(g);
    return G;
}

#define MAXLEV 32

struct orc_amg {
    orc_amg_opts o;
    int nlev;
    ocsr *A[MAXLEV];
    int32_t *agg[MAXLEV];  /* level l -> level l+1 map; NULL on the last level */
    int8_t *root[MAXLEV];
    double *l1[MAXLEV];    /* L1 diagonal a_ii + sum_{j!=i} |a_ij| */
    double *av[MAXLEV];    /* matrix values as the smoother/residual use them */
    double *dinv[MAXLEV];  /* 1 / l1, rounded to the storage precision */
    double *rs[MAXLEV];    /* row scales s_i of a bf16/fp16 level (1 on other levels) */
    int lowp[MAXLEV];      /* level stored with bf16 row-scaled values */
    ocsr *P[MAXLEV];       /* smoothed prolongator of level l (NULL: injection by agg) */
    ocsr *R[MAXLEV];       /* its transpose */
    int dense;             /* last level solved by dense Cholesky */
    int diagonal;          /* last level has no couplings: solved by x = b / a_ii */
    double *L;             /* dense Cholesky factors of the coarsest segments (each row-major, lower) */
    int64_t nd;
    int K;                 /* instances (segments) of a packed batch; 1 for one instance */
    int64_t *seg[MAXLEV];  /* segment offsets of each level [K + 1] */
    int64_t *loff;         /* start of each coarsest segment's factor in L [K + 1] */
    double *vb[MAXLEV], *vx[MAXLEV], *vr[MAXLEV];
};

typedef struct {
    uint64_t key;
    int32_t v;
} keyed;

static int cmp_keyed_desc(const void *a, const void *b) {
    uint64_t x = ((const keyed *)a)->key, y = ((const keyed *)b)->key;
    return (x < y) - (x > y);
}

/* Greedy MIS on G^2 in descending key order; returns roots[] (1 = root) and
 * the number of roots.  Vertices without a strong neighbour take no part. */
/* The segment holding row i (segments [off[k], off[k+1]), k < K). */
static int seg_of(const int64_t *off, int K, int64_t i) {
    int lo = 0, hi = K - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) / 2;
        if (off[mid] <= i)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

/* Greedy MIS-2 in descending key order.  A vertex's key uses its index within
 * its segment, so every instance of a packed batch draws the keys it would
 * draw alone (vertices of different instances are never within distance
 * two, so their relative order does not matter). */
static int64_t mis2_greedy(const ocsr *G, uint64_t seed, int level, int8_t *roots, int K, const int64_t *off) {
    int64_t n = G->nrow;
    int8_t *state = (int8_t *)calloc((size_t)(n > 0 ? n : 1), 1); /* 0 undecided, 1 root, 2 out */
    keyed *order = (keyed *)malloc((size_t)(n > 0 ? n : 1) * sizeof(keyed));
    int64_t m = 0;
    for (int64_t i = 0; i < n; i++) {
        roots[i] = 0;
        if (G->rp[i + 1] == G->rp[i]) {
            state[i] = 2;
            continue;
        }
        order[m].key = orc_mis_key(seed, level, i - off[seg_of(off, K, i)]);
        order[m].v = (int32_t)i;
        m++;
    }
    qsort(order, (size_t)m, sizeof(keyed), cmp_keyed_desc);
    int64_t nroots = 0;
    for (int64_t q = 0; q < m; q++) {
        int32_t v = order[q].v;
        if (state[v] != 0) continue;
        state[v] = 1;
        roots[v] = 1;
        nroots++;
        for (int64_t p = G->rp[v]; p < G->rp[v + 1]; p++) {
            int32_t u = G->ci[p];
            if (state[u] == 0) state[u] = 2;
            for (int64_t r = G->rp[u]; r < G->rp[u + 1]; r++) {
                int32_t w = G->ci[r];
                if (state[w] == 0) state[w] = 2;
            }
        }
    }
    free(state);
    free(order);
    return nroots;
}

/* Aggregates: roots numbered by ascending index; a vertex with a root among
 * its strong neighbours joins it; a remaining vertex joins the aggregate of
 * the strong neighbour (aggregated in the first pass) with the largest
 * |a_ij|, ties to the smaller aggregate id.  Vertices without strong
 * neighbours stay unaggregated (-1). */
static int64_t aggregate(const ocsr *G, const int8_t *roots, int32_t *agg) {
    int64_t n = G->nrow, nc = 0;
    for (int64_t i = 0; i < n; i++) agg[i] = roots[i] ? (int32_t)(nc++) : -1;
    int32_t *first = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    for (int64_t i = 0; i < n; i++) {
        first[i] = agg[i];
        if (roots[i]) continue;
        for (int64_t p = G->rp[i]; p < G->rp[i + 1]; p++)
            if (roots[G->ci[p]]) first[i] = agg[G->ci[p]];
    }
    for (int64_t i = 0; i < n; i++) {
        if (first[i] >= 0 || G->rp[i + 1] == G->rp[i]) {
            agg[i] = first[i];
            continue;
        }
        double best = -1.0;
        int32_t ba = -1;
        for (int64_t p = G->rp[i]; p < G->rp[i + 1]; p++) {
            int32_t j = G->ci[p];
            if (roots[j] || first[j] < 0) continue;
            double w = fabs(G->v[p]);
            if (w > best || (w == best && first[j] < ba)) {
                best = w;
                ba = first[j];
            }
        }
        agg[i] = ba; /* -1 only if MIS-2 maximality failed */
    }
    free(first);
    return nc;
}

/* Galerkin product A_c = P^T A P for the 0/1 injection P of agg: entry
 * (I,J) = sum of a_ij over agg(i)=I, agg(j)=J, accumulated over i ascending
 * and, within a row, in CSR order. */
static ocsr *galerkin(const ocsr *A, const int32_t *agg, int64_t nc) {
    int64_t n = A->nrow;
    /* members of each aggregate, ascending */
    int64_t *cnt = (int64_t *)calloc((size_t)nc + 1, sizeof(int64_t));
    for (int64_t i = 0; i < n; i++)
        if (agg[i] >= 0) cnt[agg[i] + 1]++;
    for (int64_t I = 0; I < nc; I++) cnt[I + 1] += cnt[I];
    int64_t *fill = (int64_t *)malloc((size_t)(nc > 0 ? nc : 1) * sizeof(int64_t));
    for (int64_t I = 0; I < nc; I++) fill[I] = cnt[I];
    int32_t *mem = (int32_t *)malloc((size_t)(cnt[nc] > 0 ? cnt[nc] : 1) * sizeof(int32_t));
    for (int64_t i = 0; i < n; i++)
        if (agg[i] >= 0) mem[fill[agg[i]]++] = (int32_t)i;
    double *acc = (double *)calloc((size_t)(nc > 0 ? nc : 1), sizeof(double));
    int8_t *mark = (int8_t *)calloc((size_t)(nc > 0 ? nc : 1), 1);
    int32_t *cols = (int32_t *)malloc((size_t)(nc > 0 ? nc : 1) * sizeof(int32_t));
    int64_t cap = A->nnz + 16;
    ocsr *C = orc_csr_new(nc, nc, cap);
    int64_t pos = 0;
    for (int64_t I = 0; I < nc; I++) {
        int64_t ncols = 0;
        for (int64_t q = cnt[I]; q < cnt[I + 1]; q++) {
            int32_t i = mem[q];
            for (int64_t p = A->rp[i]; p < A->rp[i + 1]; p++) {
                int32_t J = agg[A->ci[p]];
                if (J < 0) continue;
                if (!mark[J]) {
                    mark[J] = 1;
                    acc[J] = 0.0;
                    cols[ncols++] = J;
                }
                acc[J] = acc[J] + A->v[p];
            }
        }
        for (int64_t a = 1; a < ncols; a++) {
            int32_t x = cols[a];
            int64_t q = a - 1;
            while (q >= 0 && cols[q] > x) {
                cols[q + 1] = cols[q];
                q--;
            }
            cols[q + 1] = x;
        }
        if (pos + ncols > cap) {
            cap = 2 * cap + ncols;
            C->ci = (int32_t *)realloc(C->ci, (size_t)cap * sizeof(int32_t));
            C->v = (double *)realloc(C->v, (size_t)cap * sizeof(double));
        }
        for (int64_t a = 0; a < ncols; a++) {
            C->ci[pos] = cols[a];
            C->v[pos++] = acc[cols[a]];
            mark[cols[a]] = 0;
        }
        C->rp[I + 1] = pos;
    }
    C->nnz = pos;
    free(cnt);
    free(fill);
    free(mem);
    free(acc);
    free(mark);
    free(cols);
    return C;
}

/* Smoothed aggregation (Sec. 3.3 uses smoothed-aggregation AMG;
 * Vanek, Mandel, Brezina 1996): P = P0 - w D1F^-1 AF P0, with P0 the 0/1
 * aggregate injection, AF the filtered matrix (weak off-diagonals removed and
 * added to the diagonal, so row sums are kept; a row whose lumped diagonal
 * would not be positive keeps a_ii instead), D1F the L1 diagonal of AF and
 * w = 4/3 (lambda_max(D1F^-1 AF) <= 1, so w / lambda_max >= 4/3 needs no
 * eigenvalue estimate).  Row i: (agg(i), 1) when aggregated, then for each
 * entry of row i kept in AF, in CSR order, with J = agg(col) >= 0:
 * P_iJ = P_iJ - (c_i aF_ij), c_i = (4/3) / d1f_i.  Parity pins: dense formula,
 * dense P^T A P, two-grid error propagation. */
static ocsr *smoothed_prolongator(const ocsr *A, const ocsr *G, const int32_t *agg, int64_t nc) {
    int64_t n = A->nrow;
    int64_t cap = A->nnz + n + 16;
    ocsr *P = orc_csr_new(n, nc, cap);
    int32_t *cols = (int32_t *)malloc(sizeof(int32_t) * 4096);
    double *vals = (double *)malloc(sizeof(double) * 4096);
    int64_t pos = 0;
    for (int64_t i = 0; i < n; i++) {
        /* strong flags of row i by merging the sorted rows of A and G */
        int64_t g = G->rp[i];
        double afd = 0.0, d1 = 0.0;
        int found_d = 0;
        for (int64_t p = A->rp[i]; p < A->rp[i + 1]; p++)
            if (A->ci[p] == i) {
                afd = A->v[p];
                found_d = 1;
            }
        (void)found_d;
        /* filtered diagonal: a_ii + sum of weak off-diagonals (CSR order);
         * where that is not positive (coarse operators have positive
         * off-diagonals) the row keeps a_ii and drops its weak entries
         * without lumping them */
        const double aii = afd;
        for (int64_t p = A->rp[i]; p < A->rp[i + 1]; p++) {
            int32_t j = A->ci[p];
            if (j == i) continue;
            while (g < G->rp[i + 1] && G->ci[g] < j) g++;
            int strong = g < G->rp[i + 1] && G->ci[g] == j;
            if (!strong) afd = afd + A->v[p];
        }
        if (!(afd > 0.0)) afd = aii;
        d1 = afd;
        g = G->rp[i];
        for (int64_t p = A->rp[i]; p < A->rp[i + 1]; p++) {
            int32_t j = A->ci[p];
            if (j == i) continue;
            while (g < G->rp[i + 1] && G->ci[g] < j) g++;
            if (g < G->rp[i + 1] && G->ci[g] == j) d1 = d1 + fabs(A->v[p]);
        }
        double ci = (4.0 / 3.0) / d1;
        int m = 0;
        if (agg[i] >= 0) {
            cols[m] = agg[i];
            vals[m++] = 1.0;
        }
        g = G->rp[i];
        for (int64_t p = A->rp[i]; p < A->rp[i + 1]; p++) {
            int32_t j = A->ci[p];
            double a;
            if (j == i) {
                a = afd;
            } else {
                while (g < G->rp[i + 1] && G->ci[g] < j) g++;
                if (!(g < G->rp[i + 1] && G->ci[g] == j)) continue;
                a = A->v[p];
            }
            int32_t J = agg[j];
            if (J < 0) continue;
            int t = 0;
            while (t < m && cols[t] != J) t++;
            if (t == m) {
                cols[m] = J;
                vals[m++] = 0.0;
            }
            vals[t] = vals[t] - ci * a;
        }
        for (int a2 = 1; a2 < m; a2++) {
            int32_t x = cols[a2];
            double y = vals[a2];
            int q = a2 - 1;
            while (q >= 0 && cols[q] > x) {
                cols[q + 1] = cols[q];
                vals[q + 1] = vals[q];
                q--;
            }
            cols[q + 1] = x;
            vals[q + 1] = y;
        }
        if (pos + m > cap) {
            cap = 2 * cap + m;
            P->ci = (int32_t *)realloc(P->ci, (size_t)cap * sizeof(int32_t));
            P->v = (double *)realloc(P->v, (size_t)cap * sizeof(double));
        }
        for (int a2 = 0; a2 < m; a2++) {
            P->ci[pos] = cols[a2];
            P->v[pos++] = vals[a2];
        }
        P->rp[i + 1] = pos;
    }
    P->nnz = pos;
    free(cols);
    free(vals);
    return P;
}

/* R = P^T with the entries of each row in ascending fine index. */
static ocsr *transpose_csr(const ocsr *P) {
    ocsr *R = orc_csr_new(P->ncol, P->nrow, P->nnz);
    for (int64_t p = 0; p < P->nnz; p++) R->rp[P->ci[p] + 1]++;
    for (int64_t I = 0; I < P->ncol; I++) R->rp[I + 1] += R->rp[I];
    int64_t *at = (int64_t *)malloc(sizeof(int64_t) * (size_t)(P->ncol > 0 ? P->ncol : 1));
    for (int64_t I = 0; I < P->ncol; I++) at[I] = R->rp[I];
    for (int64_t i = 0; i < P->nrow; i++)
        for (int64_t p = P->rp[i]; p < P->rp[i + 1]; p++) {
            int64_t q = at[P->ci[p]]++;
            R->ci[q] = (int32_t)i;
            R->v[q] = P->v[p];
        }
    free(at);
    return R;
}

/* C = X Y: entry (i, k) accumulates x_ij y_jk over the entries of row i of X
 * in order, then the entries of row j of Y in order. */
static ocsr *spgemm(const ocsr *X, const ocsr *Y) {
    int64_t n = X->nrow, nc = Y->ncol;
    double *acc = (double *)calloc((size_t)(nc > 0 ? nc : 1), sizeof(double));
    int8_t *mark = (int8_t *)calloc((size_t)(nc > 0 ? nc : 1), 1);
    int32_t *cols = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nc > 0 ? nc : 1));
    int64_t cap = X->nnz + Y->nnz + 16;
    ocsr *C = orc_csr_new(n, nc, cap);
    int64_t pos = 0;
    for (int64_t i = 0; i < n; i++) {
        int64_t m = 0;
        for (int64_t p = X->rp[i]; p < X->rp[i + 1]; p++) {
            int32_t j = X->ci[p];
            for (int64_t q = Y->rp[j]; q < Y->rp[j + 1]; q++) {
                int32_t k = Y->ci[q];
                if (!mark[k]) {
                    mark[k] = 1;
                    acc[k] = 0.0;
                    cols[m++] = k;
                }
                acc[k] = acc[k] + X->v[p] * Y->v[q];
            }
        }
        for (int64_t a = 1; a < m; a++) {
            int32_t x = cols[a];
            int64_t q = a - 1;
            while (q >= 0 && cols[q] > x) {
                cols[q + 1] = cols[q];
                q--;
            }
            cols[q + 1] = x;
        }
        if (pos + m > cap) {
            cap = 2 * cap + m;
            C->ci = (int32_t *)realloc(C->ci, (size_t)cap * sizeof(int32_t));
            C->v = (double *)realloc(C->v, (size_t)cap * sizeof(double));
        }
        for (int64_t a = 0; a < m; a++) {
            C->ci[pos] = cols[a];
            C->v[pos++] = acc[cols[a]];
            mark[cols[a]] = 0;
        }
        C->rp[i + 1] = pos;
    }
    C->nnz = pos;
    free(acc);
    free(mark);
    free(cols);
    return C;
}

/* bf16 rounding: round to nearest even on the top 16 bits of a float. */
static float to_bf16(float x) {
    uint32_t u;
    memcpy(&u, &x, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) return x;
    uint32_t lsb = (u >> 16) & 1u;
    u = (u + 0x7fffu + lsb) & 0xffff0000u;
    float y;
    memcpy(&y, &u, 4);
    return y;
}

/* fp16 rounding of a float: round to nearest even with 10 fraction bits,
 * subnormals down to 2^-24, overflow to infinity (IEEE 754 binary16). */
static double to_fp16(float xf) {
    double x = (double)xf;
    if (x == 0.0 || !isfinite(x)) return x;
    double ax = fabs(x);
    if (ax >= 65520.0) return copysign(INFINITY, x);
    int e;
    frexp(ax, &e); /* ax = f 2^e, f in [0.5, 1): exponent of the leading bit is e-1 */
    int E = e - 1;
    double ulp = E >= -14 ? ldexp(1.0, E - 10) : ldexp(1.0, -24);
    double q = nearbyint(ax / ulp);
    return copysign(q * ulp, x);
}

double orc_round_lowp(double x, int prec) {
    if (prec == 16) return (double)to_bf16((float)x);
    if (prec == 17) return to_fp16((float)x);
    if (prec == 32) return (double)(float)x;
    return x;
}

static double rnd(double x, int prec) {
    if (prec == 64) return x;
    return (double)(float)x;
}

orc_amg *orc_amg_setup(const ocsr *A0, const orc_amg_opts *o) {
    int64_t off[2] = {0, A0->nrow};
    return orc_amg_setup_seg(A0, o, 1, off);
}

/* Rows of the largest segment of level l. */
static int64_t seg_max(const orc_amg *h, int l) {
    int64_t m = 0;
    for (int k = 0; k < h->K; k++)
        if (h->seg[l][k + 1] - h->seg[l][k] > m) m = h->seg[l][k + 1] - h->seg[l][k];
    return m;
}

orc_amg *orc_amg_setup_seg(const ocsr *A0, const orc_amg_opts *o, int K, const int64_t *off0) {
    if (K < 1 || off0[0] != 0 || off0[K] != A0->nrow) return NULL;
    orc_amg *h = (orc_amg *)calloc(1, sizeof(orc_amg));
    h->o = *o;
    h->K = K;
    h->seg[0] = (int64_t *)malloc((size_t)(K + 1) * sizeof(int64_t));
    memcpy(h->seg[0], off0, (size_t)(K + 1) * sizeof(int64_t));
    int maxl = o->max_levels < MAXLEV ? o->max_levels : MAXLEV;
    if (maxl < 1) maxl = 1;
    ocsr *A = orc_csr_new(A0->nrow, A0->ncol, A0->nnz);
    memcpy(A->rp, A0->rp, (size_t)(A0->nrow + 1) * sizeof(int64_t));
    memcpy(A->ci, A0->ci, (size_t)A0->nnz * sizeof(int32_t));
    memcpy(A->v, A0->v, (size_t)A0->nnz * sizeof(double));
    int l = 0;
    for (;;) {
        h->A[l] = A;
        int64_t n = A->nrow;
        h->root[l] = (int8_t *)calloc((size_t)(n > 0 ? n : 1), 1);
        /* a matrix without couplings (every row holds only its diagonal, of
         * either sign) is the last level and is solved exactly by x = b / a_ii:
         * neither coarsened nor factored */
        int diagonal = A->nnz == n;
        for (int64_t i = 0; diagonal && i < n; i++)
            if (A->rp[i + 1] - A->rp[i] != 1 || A->ci[A->rp[i]] != i) diagonal = 0;
        if (diagonal) {
            h->diagonal = 1;
            break;
        }
        /* the coarsening stops once every instance has at most n_coarse rows */
        if (seg_max(h, l) <= o->n_coarse) {
            h->dense = 1;
            break;
        }
        if (l == maxl - 1) break;
        ocsr *G = orc_strength(A, o->theta);
        int64_t nr = mis2_greedy(G, o->seed, l, h->root[l], K, h->seg[l]);
        (void)nr;
        h->agg[l] = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
        int64_t nc = aggregate(G, h->root[l], h->agg[l]);
        if (nc == 0 || (double)nc > o->stall_ratio * (double)n) {
            orc_csr_free(G);
            free(h->agg[l]);
            h->agg[l] = NULL;
            break;
        }
        /* aggregates are numbered by ascending root, so the next level's
         * segment k starts at the number of roots before segment k */
        h->seg[l + 1] = (int64_t *)malloc((size_t)(K + 1) * sizeof(int64_t));
        {
            int64_t cnt = 0;
            int k = 0;
            for (int64_t i = 0; i <= n; i++) {
                while (k <= K && h->seg[l][k] == i) h->seg[l + 1][k++] = cnt;
                if (i < n && h->root[l][i]) cnt++;
            }
        }
        if (o->smoothed) {
            h->P[l] = smoothed_prolongator(A, G, h->agg[l], nc);
            h->R[l] = transpose_csr(h->P[l]);
            ocsr *B = spgemm(A, h->P[l]);
            A = spgemm(h->R[l], B);
            orc_csr_free(B);
        } else {
            A = galerkin(A, h->agg[l], nc);
        }
        orc_csr_free(G);
        l++;
    }
    h->nlev = l + 1;
    for (int q = 0; q < h->nlev; q++) {
        ocsr *M = h->A[q];
        int64_t n = M->nrow;
        int lp = ((o->prec == 16 || o->prec == 17) && q >= o->lowp_from_level) ? o->prec : 0;
        h->lowp[q] = lp;
        h->l1[q] = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
        h->dinv[q] = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
        h->av[q] = (double *)malloc((size_t)(M->nnz > 0 ? M->nnz : 1) * sizeof(double));
        h->rs[q] = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
        for (int64_t i = 0; i < n; i++) {
            h->rs[q][i] = 1.0;
            int f;
            double s = find_val(M, i, i, &f);
            for (int64_t p = M->rp[i]; p < M->rp[i + 1]; p++)
                if (M->ci[p] != i) s = s + fabs(M->v[p]);
            h->l1[q][i] = s;
            h->dinv[q][i] = rnd(1.0 / s, o->prec == 64 ? 64 : 32);
            if (lp) {
                /* row scale s_i = 2^ceil(log2 max_j |a_ij|), values bf16(a/s) */
                double mx = 0.0;
                for (int64_t p = M->rp[i]; p < M->rp[i + 1]; p++)
                    if (fabs(M->v[p]) > mx) mx = fabs(M->v[p]);
                int e = 0;
                double fr = frexp(mx, &e); /* mx = fr 2^e, fr in [0.5,1) */
                if (fr == 0.5) e -= 1;     /* exact power of two */
                double sc = ldexp(1.0, e);
                h->rs[q][i] = sc;
                for (int64_t p = M->rp[i]; p < M->rp[i + 1]; p++) {
                    float t = (float)(M->v[p] / sc);
                    h->av[q][p] = (lp == 16 ? (double)to_bf16(t) : to_fp16(t)) * sc;
                }
            } else {
                for (int64_t p = M->rp[i]; p < M->rp[i + 1]; p++)
                    h->av[q][p] = rnd(M->v[p], o->prec == 64 ? 64 : 32);
            }
        }
        h->vb[q] = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
        h->vx[q] = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
        h->vr[q] = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    }
    if (h->dense) {
        /* textbook Cholesky A_k = L_k L_k^T of each segment's diagonal block of
         * the coarsest matrix (FP64); a packed matrix couples no segments */
        ocsr *M = h->A[h->nlev - 1];
        const int64_t *sg = h->seg[h->nlev - 1];
        h->nd = M->nrow;
        h->loff = (int64_t *)malloc((size_t)(K + 1) * sizeof(int64_t));
        h->loff[0] = 0;
        for (int k = 0; k < K; k++) h->loff[k + 1] = h->loff[k] + (sg[k + 1] - sg[k]) * (sg[k + 1] - sg[k]);
        h->L = (double *)calloc((size_t)(h->loff[K] > 0 ? h->loff[K] : 1), sizeof(double));
        for (int k = 0; k < K; k++) {
            int64_t s0 = sg[k], n = sg[k + 1] - sg[k];
            double *Lk = h->L + h->loff[k];
            for (int64_t i = 0; i < n; i++)
                for (int64_t p = M->rp[s0 + i]; p < M->rp[s0 + i + 1]; p++) {
                    int64_t j = M->ci[p] - s0;
                    if (j < 0 || j >= n) {
                        orc_amg_free(h);
                        return NULL;
                    }
                    Lk[i * n + j] = M->v[p];
                }
            for (int64_t j = 0; j < n; j++) {
                double s = Lk[j * n + j];
                for (int64_t q = 0; q < j; q++) s -= Lk[j * n + q] * Lk[j * n + q];
                if (!(s > 0.0)) {
                    orc_amg_free(h);
                    return NULL;
                }
                double ljj = sqrt(s);
                Lk[j * n + j] = ljj;
                for (int64_t i = j + 1; i < n; i++) {
                    double t = Lk[i * n + j];
                    for (int64_t q = 0; q < j; q++) t -= Lk[i * n + q] * Lk[j * n + q];
                    Lk[i * n + j] = t / ljj;
                }
                for (int64_t i = 0; i < j; i++) Lk[i * n + j] = 0.0;
            }
        }
    }
    return h;
}

void orc_amg_free(orc_amg *h) {
    if (!h) return;
    for (int q = 0; q < MAXLEV; q++) {
        orc_csr_free(h->A[q]);
        orc_csr_free(h->P[q]);
        orc_csr_free(h->R[q]);
        free(h->agg[q]);
        free(h->root[q]);
        free(h->l1[q]);
        free(h->dinv[q]);
        free(h->av[q]);
        free(h->rs[q]);
        free(h->vb[q]);
        free(h->vx[q]);
        free(h->vr[q]);
        free(h->seg[q]);
    }
    free(h->L);
    free(h->loff);
    free(h);
}

int orc_amg_nlevels(const orc_amg *h) { return h->nlev; }
int64_t orc_amg_level_n(const orc_amg *h, int l) { return h->A[l]->nrow; }
const ocsr *orc_amg_level_A(const orc_amg *h, int l) { return h->A[l]; }
int orc_amg_coarsest_dense(const orc_amg *h) { return h->dense ? 1 : (h->diagonal ? 2 : 0); }

int orc_amg_level_agg(const orc_amg *h, int l, int32_t *out) {
    if (l < 0 || l >= h->nlev || !h->agg[l]) return -1;
    memcpy(out, h->agg[l], (size_t)h->A[l]->nrow * sizeof(int32_t));
    return 0;
}

/* The values the level's smoother and residual multiply by, in CSR order of
 * the level matrix (FP64, or the FP32 / bf16 / fp16 storage value as a
 * double), its row scales and its stored 1/D1. */
int orc_amg_level_stored(const orc_amg *h, int l, double *av, double *rs, double *dinv) {
    if (l < 0 || l >= h->nlev) return -1;
    if (av) memcpy(av, h->av[l], (size_t)h->A[l]->nnz * sizeof(double));
    if (rs) memcpy(rs, h->rs[l], (size_t)h->A[l]->nrow * sizeof(double));
    if (dinv) memcpy(dinv, h->dinv[l], (size_t)h->A[l]->nrow * sizeof(double));
    return 0;
}

int orc_amg_level_seg(const orc_amg *h, int l, int64_t *out) {
    if (l < 0 || l >= h->nlev) return -1;
    memcpy(out, h->seg[l], (size_t)(h->K + 1) * sizeof(int64_t));
    return h->K;
}

int orc_amg_level_lowp(const orc_amg *h, int l) { return (l < 0 || l >= h->nlev) ? -1 : h->lowp[l]; }

const ocsr *orc_amg_level_P(const orc_amg *h, int l) {
    if (l < 0 || l >= h->nlev) return NULL;
    return h->P[l];
}

int orc_amg_level_roots(const orc_amg *h, int l, int8_t *out) {
    if (l < 0 || l >= h->nlev) return -1;
    memcpy(out, h->root[l], (size_t)h->A[l]->nrow);
    return 0;
}

int orc_amg_level_l1(const orc_amg *h, int l, double *out) {
    if (l < 0 || l >= h->nlev) return -1;
    memcpy(out, h->l1[l], (size_t)h->A[l]->nrow * sizeof(double));
    return 0;
}

/* r = b - A x with the level's stored values */
static void level_residual(const orc_amg *h, int l, const double *b, const double *x, double *r) {
    const ocsr *M = h->A[l];
    const double *av = h->av[l];
    for (int64_t i = 0; i < M->nrow; i++) {
        double s = 0.0;
        for (int64_t p = M->rp[i]; p < M->rp[i + 1]; p++) s += av[p] * x[M->ci[p]];
        r[i] = b[i] - s;
    }
}

/* The smoothers.  0: L1-Jacobi, x <- x + D1^{-1} (b - A x) (omega = 1).
 * 1: Chebyshev of degree cheb_degree (2 when 0) for D1^{-1} A on the
 * interval [0.3, 1] (lambda_max(D1^{-1} A) <= 1 for L1 diagonals), by the
 * three-term recurrence of Saad, Iterative Methods, Alg. 12.1: the residual
 * polynomial is T_k((theta - t)/delta) / T_k(theta/delta).  2: Gauss-Seidel
 * with the level's own diagonal, as in the paper's experiments (Sec. 4):
 * ascending rows before the coarse correction, descending after it, so that
 * the V-cycle stays symmetric.  Gauss-Seidel is sequential; it exists only
 * here, to compare iteration counts with the paper's smoother. */
static void smooth(orc_amg *h, int l, const double *b, double *x, int zero_guess, int post) {
    int64_t n = h->A[l]->nrow;
    int pv = h->o.prec == 64 ? 64 : 32;
    double *r = h->vr[l];
    const double *dv = h->dinv[l];
    if (h->o.smoother == 0) {
        if (zero_guess) {
            for (int64_t i = 0; i < n; i++) x[i] = rnd(dv[i] * b[i], pv);
        } else {
            level_residual(h, l, b, x, r);
            for (int64_t i = 0; i < n; i++) x[i] = rnd(x[i] + dv[i] * r[i], pv);
        }
        return;
    }
    if (h->o.smoother == 2) {
        const ocsr *M = h->A[l];
        const double *av = h->av[l];
        if (zero_guess)
            for (int64_t i = 0; i < n; i++) x[i] = 0.0;
        for (int64_t q = 0; q < n; q++) {
            int64_t i = post ? n - 1 - q : q;
            double s = b[i], aii = 0.0;
            for (int64_t p = M->rp[i]; p < M->rp[i + 1]; p++) {
                if (M->ci[p] == i)
                    aii = av[p];
                else
                    s -= av[p] * x[M->ci[p]];
            }
            x[i] = rnd(s / aii, pv);
        }
        return;
    }
    const int deg = h->o.cheb_degree < 1 ? 2 : h->o.cheb_degree;
    const double lo = 0.3, hi = 1.0;
    double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo);
    double sigma = theta / delta, rho = 1.0 / sigma;
    double *d = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    if (zero_guess) {
        for (int64_t i = 0; i < n; i++) r[i] = b[i];
    } else {
        level_residual(h, l, b, x, r);
    }
    for (int64_t i = 0; i < n; i++) {
        d[i] = rnd((dv[i] * r[i]) / theta, pv);
        x[i] = rnd((zero_guess ? 0.0 : x[i]) + d[i], pv);
    }
    for (int j = 2; j <= deg; j++) {
        double rho_new = 1.0 / (2.0 * sigma - rho);
        level_residual(h, l, b, x, r);
        for (int64_t i = 0; i < n; i++) {
            d[i] = rnd(rho_new * rho * d[i] + (2.0 * rho_new / delta) * (dv[i] * r[i]), pv);
            x[i] = rnd(x[i] + d[i], pv);
        }
        rho = rho_new;
    }
    free(d);
}

static void vcycle_level(orc_amg *h, int l, const double *b, double *x) {
    int64_t n = h->A[l]->nrow;
    int pv = h->o.prec == 64 ? 64 : 32;
    if (l == h->nlev - 1 && h->dense) {
        /* per segment: L_k y = b_k, L_k^T x_k = y */
        const int64_t *sg = h->seg[l];
        for (int k = 0; k < h->K; k++) {
            const double *L = h->L + h->loff[k];
            int64_t s0 = sg[k], m = sg[k + 1] - sg[k];
            const double *bk = b + s0;
            double *xk = x + s0;
            for (int64_t i = 0; i < m; i++) {
                double s = bk[i];
                for (int64_t q = 0; q < i; q++) s -= L[i * m + q] * xk[q];
                xk[i] = s / L[i * m + i];
            }
            for (int64_t i = m - 1; i >= 0; i--) {
                double s = xk[i];
                for (int64_t q = i + 1; q < m; q++) s -= L[q * m + i] * xk[q];
                xk[i] = s / L[i * m + i];
            }
        }
        for (int64_t i = 0; i < n; i++) x[i] = rnd(x[i], pv);
        return;
    }
    if (l == h->nlev - 1 && h->diagonal) {
        /* the stored 1/a_ii (1/l1 of a row without off-diagonals) */
        for (int64_t i = 0; i < n; i++) x[i] = rnd(h->dinv[l][i] * b[i], pv);
        return;
    }
    int ns = h->o.sweeps < 1 ? 1 : h->o.sweeps;
    for (int s = 0; s < ns; s++) smooth(h, l, b, x, s == 0, 0);
    if (h->agg[l]) {
        int64_t nc = h->A[l + 1]->nrow;
        double *r = h->vr[l];
        level_residual(h, l, b, x, r);
        for (int64_t i = 0; i < n; i++) r[i] = rnd(r[i], pv);
        double *bc = h->vb[l + 1], *xc = h->vx[l + 1];
        if (h->P[l]) {
            /* b_c = R r, x += P x_c (values rounded to the storage precision) */
            const ocsr *R = h->R[l], *P = h->P[l];
            for (int64_t I = 0; I < nc; I++) {
                double s = 0.0;
                for (int64_t p = R->rp[I]; p < R->rp[I + 1]; p++) s += rnd(R->v[p], pv) * r[R->ci[p]];
                bc[I] = rnd(s, pv);
            }
            vcycle_level(h, l + 1, bc, xc);
            for (int64_t i = 0; i < n; i++) {
                double s = 0.0;
                for (int64_t p = P->rp[i]; p < P->rp[i + 1]; p++) s += rnd(P->v[p], pv) * xc[P->ci[p]];
                x[i] = rnd(x[i] + s, pv);
            }
        } else {
            for (int64_t I = 0; I < nc; I++) bc[I] = 0.0;
            for (int64_t i = 0; i < n; i++)
                if (h->agg[l][i] >= 0) bc[h->agg[l][i]] += r[i];
            for (int64_t I = 0; I < nc; I++) bc[I] = rnd(bc[I], pv);
            vcycle_level(h, l + 1, bc, xc);
            for (int64_t i = 0; i < n; i++)
                if (h->agg[l][i] >= 0) x[i] = rnd(x[i] + xc[h->agg[l][i]], pv);
        }
    }
    for (int s = 0; s < ns; s++) smooth(h, l, b, x, 0, 1);
}

void orc_vcycle(orc_amg *h, const double *b, double *x) {
    int64_t n = h->A[0]->nrow;
    int pv = h->o.prec == 64 ? 64 : 32;
    double *bb = h->vb[0];
    for (int64_t i = 0; i < n; i++) bb[i] = rnd(b[i], pv);
    vcycle_level(h, 0, bb, x);
}

/* ------------------------------------------------------------------ M_L */
/* Eq. (8) / Algorithm 1: z_m = Q_mm r_m; r_f <- r_f - A_fm z_m;
 * z_f = Q_ff r_f, with Q_mm one V-cycle on S~ (Eq. (7)) and Q_ff one V-cycle
 * on A_ff.  kind 1 (block diagonal D^{-1} of Sec. 3.2) skips the update;
 * kind 2 (block upper (UD)^{-1}) solves the interface first and then
 * updates the domain residual with A_mf. */
struct orc_ml {
    int64_t n_m, n_f;
    int kind;
    int ff_negative; /* every diagonal entry of A_ff is negative (flux block of the paper's partition) */
    ocsr *Amm, *Amf, *Afm, *Aff, *S;
    orc_amg *amg[2];
    double *t, *u;
};

orc_ml *orc_ml_new(const ocsr *A, int64_t n_m, const orc_amg_opts *o, int kind) {
    int64_t mo[2] = {0, n_m}, fo[2] = {0, A->nrow - n_m};
    return orc_ml_new_seg(A, n_m, o, kind, 1, mo, fo);
}

orc_ml *orc_ml_new_seg(const ocsr *A, int64_t n_m, const orc_amg_opts *o, int kind, int K, const int64_t *moff,
                       const int64_t *foff) {
    orc_ml *m = (orc_ml *)calloc(1, sizeof(orc_ml));
    m->n_m = n_m;
    m->n_f = A->nrow - n_m;
    m->kind = kind;
    orc_split(A, n_m, &m->Amm, &m->Amf, &m->Afm, &m->Aff);
    m->S = orc_schur(m->Amm, m->Amf, m->Afm, m->Aff);
    if (!m->S) {
        orc_ml_free(m);
        return NULL;
    }
    m->amg[0] = orc_amg_setup_seg(m->S, o, K, moff);
    m->amg[1] = m->n_f > 0 ? orc_amg_setup_seg(m->Aff, o, K, foff) : NULL;
    m->ff_negative = m->n_f > 0;
    for (int64_t k = 0; k < m->n_f; k++) {
        int f;
        if (!(find_val(m->Aff, k, k, &f) < 0.0)) m->ff_negative = 0;
    }
    if (!m->amg[0] || (m->n_f > 0 && !m->amg[1])) {
        orc_ml_free(m);
        return NULL;
    }
    int64_t mx = m->n_m > m->n_f ? m->n_m : m->n_f;
    m->t = (double *)calloc((size_t)(mx > 0 ? mx : 1), sizeof(double));
    m->u = (double *)calloc((size_t)(mx > 0 ? mx : 1), sizeof(double));
    return m;
}

void orc_ml_free(orc_ml *m) {
    if (!m) return;
    orc_csr_free(m->Amm);
    orc_csr_free(m->Amf);
    orc_csr_free(m->Afm);
    orc_csr_free(m->Aff);
    orc_csr_free(m->S);
    orc_amg_free(m->amg[0]);
    orc_amg_free(m->amg[1]);
    free(m->t);
    free(m->u);
    free(m);
}

const orc_amg *orc_ml_amg(const orc_ml *m, int block) { return m->amg[block ? 1 : 0]; }
const ocsr *orc_ml_schur(const orc_ml *m) { return m->S; }

int orc_ml_apply(void *ctx, const double *r, double *z) {
    orc_ml *m = (orc_ml *)ctx;
    int64_t nm = m->n_m, nf = m->n_f;
    const double *rm = r, *rf = r + nm;
    double *zm = z, *zf = z + nm;
    if (m->kind == 2) {
        /* block upper: z_f = Q_ff r_f; r_m <- r_m - A_mf z_f; z_m = Q_mm r_m */
        if (nf > 0) orc_vcycle(m->amg[1], rf, zf);
        for (int64_t i = 0; i < nm; i++) {
            double s = 0.0;
            for (int64_t p = m->Amf->rp[i]; p < m->Amf->rp[i + 1]; p++) s += m->Amf->v[p] * zf[m->Amf->ci[p]];
            m->t[i] = rm[i] - s;
        }
        orc_vcycle(m->amg[0], m->t, zm);
        return 0;
    }
    orc_vcycle(m->amg[0], rm, zm);
    if (nf == 0) return 0;
    if (m->kind == 1) {
        /* B_D is used with CG and MINRES, which need it positive definite:
         * for a negative definite A_ff (the flux block) its block is -Q_ff */
        orc_vcycle(m->amg[1], rf, zf);
        if (m->ff_negative)
            for (int64_t k = 0; k < nf; k++) zf[k] = -zf[k];
        return 0;
    }
    for (int64_t k = 0; k < nf; k++) {
        double s = 0.0;
        for (int64_t p = m->Afm->rp[k]; p < m->Afm->rp[k + 1]; p++) s += m->Afm->v[p] * zm[m->Afm->ci[p]];
        m->t[k] = rf[k] - s;
    }
    orc_vcycle(m->amg[1], m->t, zf);
    return 0;
}

int orc_identity_apply(void *ctx, const double *r, double *z) {
    int64_t n = *(const int64_t *)ctx;
    memcpy(z, r, (size_t)n * sizeof(double));
    return 0;
}

/* --------------------------------------------------------------- Krylov */
/* Flexible GMRES(m) (Saad, SIAM J. Sci. Comput. 14, 1993) with right
 * preconditioning as in Sec. 3.2 (A B_L is the operator whose spectrum the
 * paper studies), modified Gram-Schmidt, Givens rotations; x0 given (zero in
 * Sec. 4); convergence when the true relative residual ||b - A x|| / ||b||
 * is <= rtol.  The Arnoldi estimate ends a cycle early; the true residual
 * decides.  Pins: <= 2 iterations with exact block inverses, <= n steps with
 * the identity preconditioner, orthonormal basis, monotone estimates. */
int orc_fgmres(const ocsr *A, orc_prec_fn prec, void *pctx, const double *b, double *x,
               int restart, double rtol, int maxit, double *hist, orc_stats *st) {
    int64_t n = A->nrow;
    int m = restart;
    double *V = (double *)calloc((size_t)(m + 1) * (size_t)n, sizeof(double));
    double *Z = (double *)calloc((size_t)m * (size_t)n, sizeof(double));
    double *H = (double *)calloc((size_t)(m + 1) * (size_t)m, sizeof(double));
    double *cs = (double *)calloc((size_t)m, sizeof(double));
    double *sn = (double *)calloc((size_t)m, sizeof(double));
    double *g = (double *)calloc((size_t)m + 1, sizeof(double));
    double *y = (double *)calloc((size_t)m, sizeof(double));
    double *w = (double *)calloc((size_t)n, sizeof(double));
    int it = 0, restarts = 0, conv = 0, hl = 0, err = 0;
    double bn = nrm2(n, b);
    if (bn == 0.0) bn = 1.0;
    for (;;) {
        orc_spmv(A, x, w);
        for (int64_t i = 0; i < n; i++) V[i] = b[i] - w[i];
        double beta = nrm2(n, V);
        if (hist && hl == 0) hist[hl++] = beta / bn;
        if (beta / bn <= rtol) {
            conv = 1;
            break;
        }
        if (it >= maxit) break;
        for (int64_t i = 0; i < n; i++) V[i] /= beta;
        for (int q = 0; q <= m; q++) g[q] = 0.0;
        g[0] = beta;
        int j, kdone = 0;
        for (j = 0; j < m; j++) {
            double *vj = V + (size_t)j * n, *zj = Z + (size_t)j * n, *vn = V + (size_t)(j + 1) * n;
            if (prec(pctx, vj, zj) != 0) {
                err = 1;
                break;
            }
            it++;
            orc_spmv(A, zj, vn);
            for (int q = 0; q <= j; q++) {
                const double *vq = V + (size_t)q * n;
                double hq = dot(n, vn, vq);
                H[q * m + j] = hq;
                for (int64_t i = 0; i < n; i++) vn[i] -= hq * vq[i];
            }
            double hn = nrm2(n, vn);
            H[(j + 1) * m + j] = hn;
            if (hn != 0.0)
                for (int64_t i = 0; i < n; i++) vn[i] /= hn;
            for (int q = 0; q < j; q++) {
                double a = H[q * m + j], c = H[(q + 1) * m + j];
                H[q * m + j] = cs[q] * a + sn[q] * c;
                H[(q + 1) * m + j] = -sn[q] * a + cs[q] * c;
            }
            double a = H[j * m + j], c = H[(j + 1) * m + j];
            double rr = sqrt(a * a + c * c);
            cs[j] = rr == 0.0 ? 1.0 : a / rr;
            sn[j] = rr == 0.0 ? 0.0 : c / rr;
            H[j * m + j] = rr;
            H[(j + 1) * m + j] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            if (hist) hist[hl++] = fabs(g[j + 1]) / bn;
            kdone = j + 1;
            if (fabs(g[j + 1]) / bn <= rtol || it >= maxit || hn == 0.0) break;
        }
        if (err) break;
        /* back substitution H y = g, then x += Z y */
        for (int q = kdone - 1; q >= 0; q--) {
            double s = g[q];
            for (int p = q + 1; p < kdone; p++) s -= H[q * m + p] * y[p];
            y[q] = H[q * m + q] == 0.0 ? 0.0 : s / H[q * m + q];
        }
        for (int q = 0; q < kdone; q++) {
            const double *zq = Z + (size_t)q * n;
            for (int64_t i = 0; i < n; i++) x[i] += y[q] * zq[i];
        }
        restarts++;
    }
    orc_spmv(A, x, w);
    for (int64_t i = 0; i < n; i++) w[i] = b[i] - w[i];
    if (st) {
        st->iterations = it;
        st->restarts = restarts;
        st->converged = conv;
        st->relres_true = nrm2(n, w) / bn;
        st->history_len = hl;
    }
    free(V);
    free(Z);
    free(H);
    free(cs);
    free(sn);
    free(g);
    free(y);
    free(w);
    return err ? -1 : (conv ? 0 : 1);
}

/* Preconditioned CG (Hestenes-Stiefel) for the symmetric positive definite
 * system with a symmetric preconditioner (the block-diagonal B_D of
 * Sec. 3.2 with symmetric V-cycles). */
int orc_pcg(const ocsr *A, orc_prec_fn prec, void *pctx, const double *b, double *x,
            double rtol, int maxit, double *hist, orc_stats *st) {
    int64_t n = A->nrow;
    double *r = (double *)calloc((size_t)n, sizeof(double));
    double *z = (double *)calloc((size_t)n, sizeof(double));
    double *p = (double *)calloc((size_t)n, sizeof(double));
    double *q = (double *)calloc((size_t)n, sizeof(double));
    int it = 0, conv = 0, hl = 0, err = 0;
    double bn = nrm2(n, b);
    if (bn == 0.0) bn = 1.0;
    orc_spmv(A, x, q);
    for (int64_t i = 0; i < n; i++) r[i] = b[i] - q[i];
    double rn = nrm2(n, r);
    if (hist) hist[hl++] = rn / bn;
    double rz = 0.0;
    while (rn / bn > rtol && it < maxit) {
        if (prec(pctx, r, z) != 0) {
            err = 1;
            break;
        }
        it++;
        double rz_new = dot(n, r, z);
        if (it == 1) {
            for (int64_t i = 0; i < n; i++) p[i] = z[i];
        } else {
            double beta = rz_new / rz;
            for (int64_t i = 0; i < n; i++) p[i] = z[i] + beta * p[i];
        }
        rz = rz_new;
        orc_spmv(A, p, q);
        double alpha = rz / dot(n, p, q);
        for (int64_t i = 0; i < n; i++) {
            x[i] += alpha * p[i];
            r[i] -= alpha * q[i];
        }
        rn = nrm2(n, r);
        if (hist) hist[hl++] = rn / bn;
    }
    orc_spmv(A, x, q);
    for (int64_t i = 0; i < n; i++) q[i] = b[i] - q[i];
    double tr = nrm2(n, q) / bn;
    conv = tr <= rtol;
    if (st) {
        st->iterations = it;
        st->restarts = 0;
        st->converged = conv;
        st->relres_true = tr;
        st->history_len = hl;
    }
    free(r);
    free(z);
    free(p);
    free(q);
    return err ? -1 : (conv ? 0 : 1);
}

/* Preconditioned MINRES (Paige and Saunders 1975), in the three-term form of
 * Elman, Silvester and Wathen (Finite Elements and Fast Iterative Solvers,
 * preconditioned MINRES): Lanczos vectors v with z = M v normalised in the
 * M-inner product, Givens rotations (c, s) on the tridiagonal matrix, search
 * directions w, and eta the M^-1-norm of the residual.  The 2-norm residual
 * r is carried along by the same recurrence as x (A w is formed from A z, so
 * no extra product is needed); when it reaches rtol ||b|| the true residual
 * decides, and the iteration restarts from x if it is not yet small enough.
 * Iterations count preconditioner applications after the first. */
int orc_minres(const ocsr *A, orc_prec_fn prec, void *pctx, const double *b, double *x,
               double rtol, int maxit, double *hist, orc_stats *st) {
    int64_t n = A->nrow;
    double *r = (double *)calloc((size_t)n, sizeof(double));
    double *v0 = (double *)calloc((size_t)n, sizeof(double));
    double *v1 = (double *)calloc((size_t)n, sizeof(double));
    double *z = (double *)calloc((size_t)n, sizeof(double));
    double *az = (double *)calloc((size_t)n, sizeof(double));
    double *w0 = (double *)calloc((size_t)n, sizeof(double));
    double *w1 = (double *)calloc((size_t)n, sizeof(double));
    double *aw0 = (double *)calloc((size_t)n, sizeof(double));
    double *aw1 = (double *)calloc((size_t)n, sizeof(double));
    double *t = (double *)calloc((size_t)n, sizeof(double));
    int it = 0, conv = 0, hl = 0, err = 0, restarts = 0;
    double bn = nrm2(n, b);
    if (bn == 0.0) bn = 1.0;
    for (;;) {
        orc_spmv(A, x, t);
        for (int64_t i = 0; i < n; i++) r[i] = b[i] - t[i];
        double rn = nrm2(n, r);
        if (hist && hl == 0) hist[hl++] = rn / bn;
        if (rn / bn <= rtol || it >= maxit) break;
        /* v1 = r, z = M v1, gamma1 = sqrt(z . v1) */
        for (int64_t i = 0; i < n; i++) {
            v1[i] = r[i];
            v0[i] = 0.0;
            w0[i] = w1[i] = aw0[i] = aw1[i] = 0.0;
        }
        if (prec(pctx, v1, z) != 0) {
            err = 1;
            break;
        }
        double g1 = sqrt(dot(n, z, v1));
        if (!(g1 > 0.0)) {
            err = 1;
            break;
        }
        double g0 = 1.0, eta = g1, c0 = 1.0, c1 = 1.0, s0 = 0.0, s1 = 0.0;
        int restart = 0;
        while (it < maxit) {
            it++;
            /* z_j = z / gamma_j; delta_j = (A z_j) . z_j */
            for (int64_t i = 0; i < n; i++) z[i] /= g1;
            orc_spmv(A, z, az);
            double delta = dot(n, az, z);
            /* v_{j+1} = A z_j - (delta/gamma_j) v_j - (gamma_j/gamma_{j-1}) v_{j-1} */
            for (int64_t i = 0; i < n; i++) {
                double vn = az[i] - (delta / g1) * v1[i] - (g1 / g0) * v0[i];
                v0[i] = v1[i];
                v1[i] = vn;
            }
            /* Givens rotations on the new column of the tridiagonal matrix */
            double a0 = c1 * delta - c0 * s1 * g1;
            double a2 = s1 * delta + c0 * c1 * g1;
            double a3 = s0 * g1;
            /* z_{j+1} = M v_{j+1}, gamma_{j+1}; t keeps z_j for w */
            for (int64_t i = 0; i < n; i++) t[i] = z[i];
            if (prec(pctx, v1, z) != 0) {
                err = 1;
                break;
            }
            double zv = dot(n, z, v1);
            double g2 = zv > 0.0 ? sqrt(zv) : 0.0;
            double a1 = sqrt(a0 * a0 + g2 * g2);
            if (!(a1 > 0.0)) {
                err = 1;
                break;
            }
            double c2 = a0 / a1, s2 = g2 / a1;
            /* w_{j+1} = (z_j - a3 w_{j-1} - a2 w_j) / a1, and A w likewise */
            double step = c2 * eta;
            for (int64_t i = 0; i < n; i++) {
                double wn = (t[i] - a3 * w0[i] - a2 * w1[i]) / a1;
                double awn = (az[i] - a3 * aw0[i] - a2 * aw1[i]) / a1;
                w0[i] = w1[i];
                w1[i] = wn;
                aw0[i] = aw1[i];
                aw1[i] = awn;
                x[i] += step * wn;
                r[i] -= step * awn;
            }
            eta = -s2 * eta;
            g0 = g1;
            g1 = g2;
            c0 = c1;
            c1 = c2;
            s0 = s1;
            s1 = s2;
            double rr = nrm2(n, r);
            if (hist) hist[hl++] = rr / bn;
            if (rr / bn <= rtol) break;
            if (!(g2 > 0.0)) { /* invariant subspace: exact within the Krylov space */
                restart = 1;
                break;
            }
        }
        if (err) break;
        (void)restart;
        restarts++;
        if (it >= maxit) {
            orc_spmv(A, x, t);
            break;
        }
    }
    orc_spmv(A, x, t);
    for (int64_t i = 0; i < n; i++) t[i] = b[i] - t[i];
    double tr = nrm2(n, t) / bn;
    conv = tr <= rtol;
    if (st) {
        st->iterations = it;
        st->restarts = restarts > 0 ? restarts - 1 : 0;
        st->converged = conv;
        st->relres_true = tr;
        st->history_len = hl;
    }
    free(r);
    free(v0);
    free(v1);
    free(z);
    free(az);
    free(w0);
    free(w1);
    free(aw0);
    free(aw1);
    free(t);
    return err ? -1 : (conv ? 0 : 1);
}
