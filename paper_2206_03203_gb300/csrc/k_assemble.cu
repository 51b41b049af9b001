// Two-point-flux assembly of the mixed-dimensional block system on the GPU.
//
// Sec. 2.1 of the paper (Eq. (1) per subdomain, Eq. (2)-(3) across each
// matrix-fracture interface) discretised cell-centred on a Cartesian grid;
// the interface flux is eliminated into a matrix-fracture transmissibility.
// Unknowns are ordered [matrix cells (x fastest); fracture cells], giving the
// 2x2 block structure of Eq. (4).  Compiled with -fmad=false: every product
// and sum is rounded as written, so values are reproducible to the bit.
#include "internal.cuh"

namespace mds {

struct GridD {
    int dim, n;
    int64_t ext[3][3];
    int64_t off[3];
    double h, F, elen;
    int64_t n_m, nf, N, nb;
    int flux;      // 1: the paper's partition, interface fluxes as unknowns
    int junction;  // 0: pairwise links at junctions; 1: node of >= 3 cells (star)
    int64_t nI;    // intersection cells (flux form with junction 1)
    int64_t nIF;   // their fluxes
    int64_t NO;    // pressure unknowns: N + nI
    int64_t GF;    // first intersection flux: NO + 2 nf
    int64_t NT;    // all unknowns: N (primal) or GF + nIF (flux form)
    // intersection tables (flux form with junction 1)
    const int32_t *own_base;  // [nf+1] first intersection owned by each fracture cell
    const int32_t *ioff;      // [nI+1] first flux of each intersection (relative to GF)
    const int32_t *imem;      // [4 nI] members of each intersection, ascending
    const int32_t *phi_int;   // [nIF] intersection of each flux
    const double *kn;         // [nf] normal permeability (kappa = 2 kn / a)
    const double *hk;         // [n_m] h / (2 k_m) of each matrix cell, or null (computed per use)
};

__device__ __forceinline__ int64_t face_id(const GridD &g, int d, int64_t x, int64_t y, int64_t z) {
    const int64_t *e = g.ext[d];
    if (x < 0 || y < 0 || z < 0 || x >= e[0] || y >= e[1] || z >= e[2]) return -1;
    return g.off[d] + x + e[0] * (y + e[1] * z);
}

__device__ __forceinline__ int32_t frac_at(const GridD &g, const int32_t *map, int d, const int64_t c[3]) {
    int64_t f = face_id(g, d, c[0], c[1], c[2]);
    return f < 0 ? -1 : map[f];
}

__device__ __forceinline__ int64_t cell_id(const GridD &g, const int64_t c[3]) {
    return c[0] + (int64_t)g.n * (c[1] + (int64_t)g.n * c[2]);
}

// Half-cell resistance h / (2 k_m) of matrix cell j, the term each side of
// a face contributes to the two-point transmissibility (the same division as
// written inline, so the values are identical to the bit).
__device__ __forceinline__ double half_res(const GridD &g, const double *km, int64_t j) {
    return g.hk ? g.hk[j] : g.h / (2.0 * km[j]);
}

// Fracture cell k claims its face in the face map (error bits on a bad or
// doubly claimed face).
__device__ __forceinline__ void scatter_face(const GridD &g, const int32_t *axis, const int32_t *pos, int32_t *map,
                                             int *err, int64_t k) {
    int d = axis[k];
    int64_t x = pos[3 * k], y = pos[3 * k + 1], z = g.dim == 3 ? pos[3 * k + 2] : 0;
    int64_t c[3] = {x, y, z};
    if (d < 0 || d >= g.dim || c[d] < 1 || c[d] > g.n - 1) {
        atomicOr(err, DERR_BAD_FRACTURE);
        return;
    }
    int64_t f = face_id(g, d, x, y, z);
    if (f < 0) {
        atomicOr(err, DERR_BAD_FRACTURE);
        return;
    }
    if (atomicCAS(map + f, -1, (int32_t)k) != -1) atomicOr(err, DERR_DUP_FACE);
}

__global__ void k_map_scatter(GridD g, const int32_t *__restrict__ axis, const int32_t *__restrict__ pos,
                              int32_t *__restrict__ map, int *err) {
    mds_pdl_entry();
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= g.nf) return;
    scatter_face(g, axis, pos, map, err, k);
}

struct Ent {
    int32_t c;
    double t;
};

__device__ __forceinline__ void sort_ents(Ent *e, int cnt) {
    for (int a = 1; a < cnt; a++) {
        Ent x = e[a];
        int q = a - 1;
        while (q >= 0 && e[q].c > x.c) {
            e[q + 1] = e[q];
            q--;
        }
        e[q + 1] = x;
    }
}

// Entries of matrix row i (without the diagonal); returns their count and the
// Dirichlet coefficients of the x=0 / x=1 faces.
__device__ int matrix_entries(const GridD &g, const int32_t *map, const double *km, const double *kf,
                              const double *ap, int64_t i, Ent *row, double tb[2], int has[2]) {
    int64_t n = g.n;
    int64_t c[3] = {i % n, (i / n) % n, g.dim == 3 ? i / (n * n) : 0};
    double ki = km[i];
    int cnt = 0;
    has[0] = has[1] = 0;
    tb[0] = tb[1] = 0.0;
    for (int d = 0; d < g.dim; d++) {
        for (int s = 0; s < 2; s++) {
            int64_t plane = c[d] + s;
            if (plane == 0 || plane == n) {
                if (d == 0) {
                    tb[s] = (g.F * (2.0 * ki)) / g.h;
                    has[s] = 1;
                }
                continue;
            }
            int64_t fc[3] = {c[0], c[1], c[2]};
            fc[d] = plane;
            int32_t k = frac_at(g, map, d, fc);
            if (k >= 0) {
                double kappa = (2.0 * g.kn[k]) / ap[k];
                // flux form: the interface flux of this face side (side 0 when
                // the face is above the cell, s = 1)
                if (g.flux) {
                    row[cnt].c = (int32_t)(g.NO + 2 * k + (s ? 0 : 1));
                    row[cnt].t = 1.0;
                } else {
                    row[cnt].c = (int32_t)(g.n_m + k);
                    row[cnt].t = g.F / (g.h / (2.0 * ki) + 1.0 / kappa);
                }
            } else {
                int64_t nc[3] = {c[0], c[1], c[2]};
                nc[d] = c[d] + (s ? 1 : -1);
                int64_t j = cell_id(g, nc);
                row[cnt].c = (int32_t)j;
                row[cnt].t = g.F / (g.h / (2.0 * ki) + g.h / (2.0 * km[j]));
            }
            cnt++;
        }
    }
    return cnt;
}

__device__ __forceinline__ double half_t(const GridD &g, const double *kf, const double *ap, int64_t k) {
    return ((kf[k] * ap[k]) * g.elen) / (0.5 * g.h);
}

// Junction q of fracture cell k (normal d): the vertex (2D) / grid edge (3D)
// closing the cell along its (q/2)-th tangential axis e, low end for even q.
// The cells incident to it: faces normal to d at e-cells u-1 and u, faces
// normal to e at plane u with d-cells plane-1 and plane.  J gets them, k
// included, ascending; returns their count, 0 at a Dirichlet end (x = 0/1).
__device__ int junction_members(const GridD &g, const int32_t *map, const int32_t *axis, const int32_t *pos,
                                int64_t k, int q, int *e_out, int32_t J[5]) {
    const int d = axis[k];
    int64_t c[3] = {pos[3 * k], pos[3 * k + 1], g.dim == 3 ? pos[3 * k + 2] : 0};
    int e = q / 2 == 0 ? (d == 0 ? 1 : 0) : (d == 2 ? 1 : 2);  // tangential axes ascending
    *e_out = e;
    const int64_t u = c[e] + (q & 1);
    if (e == 0 && (u == 0 || u == g.n)) return 0;
    int m = 0;
    J[m++] = (int32_t)k;
#pragma unroll
    for (int r = 0; r < 4; r++) {
        int64_t f[3] = {c[0], c[1], c[2]};
        int fd;
        if (r < 2) {
            f[e] = u - 1 + r;
            fd = d;
        } else {
            f[e] = u;
            f[d] = c[d] - 1 + (r - 2);
            fd = e;
        }
        int32_t l = frac_at(g, map, fd, f);
        if (l >= 0 && l != k) J[m++] = l;
    }
    for (int a = 1; a < m; a++) {
        int32_t x = J[a];
        int b2 = a - 1;
        while (b2 >= 0 && J[b2] > x) {
            J[b2 + 1] = J[b2];
            b2--;
        }
        J[b2 + 1] = x;
    }
    return m;
}

// Intersection id of the junction with members J (m >= 3): it was created
// by its lowest member J[0], in that cell's junction order.
__device__ int64_t intersection_of(const GridD &g, const int32_t *map, const int32_t *axis, const int32_t *pos,
                                   const int32_t *J, int m) {
    const int64_t k0 = J[0];
    const int nslot = 2 * (g.dim - 1);
    int ord = 0;
    for (int q = 0; q < nslot; q++) {
        int32_t J0[5];
        int e;
        int m0 = junction_members(g, map, axis, pos, k0, q, &e, J0);
        if (m0 < 3 || J0[0] != k0) continue;
        bool same = m0 == m;
        for (int r = 0; same && r < m; r++) same = J0[r] == J[r];
        if (same) return g.own_base[k0] + ord;
        ord++;
    }
    return -1;
}

// Entries of fracture row k (without the diagonal).  bfa/bfb are the two
// boundary faces sharing a Dirichlet end edge.  Pressure columns carry their
// transmissibility t (written -t), flux columns their value.
__device__ int fracture_entries(const GridD &g, const int32_t *map, const double *km, const int32_t *axis,
                                const int32_t *pos, const double *kf, const double *ap, int64_t k, Ent *row,
                                double tb[2], int has[2], int64_t bfa[2], int64_t bfb[2]) {
    int d = axis[k];
    int64_t c[3] = {pos[3 * k], pos[3 * k + 1], g.dim == 3 ? pos[3 * k + 2] : 0};
    int64_t plane = c[d];
    double kappa = (2.0 * g.kn[k]) / ap[k];
    double tk = half_t(g, kf, ap, k);
    int cnt = 0;
    has[0] = has[1] = 0;
    tb[0] = tb[1] = 0.0;
    bfa[0] = bfa[1] = bfb[0] = bfb[1] = 0;
    for (int s = 0; s < 2; s++) {
        int64_t mc[3] = {c[0], c[1], c[2]};
        mc[d] = plane - 1 + s;
        int64_t j = cell_id(g, mc);
        if (g.flux) {
            row[cnt].c = (int32_t)(g.NO + 2 * k + s);
            row[cnt].t = -1.0;
        } else {
            row[cnt].c = (int32_t)j;
            row[cnt].t = g.F / (half_res(g, km, j) + 1.0 / kappa);
        }
        cnt++;
    }
    const int nslot = 2 * (g.dim - 1);
    for (int q = 0; q < nslot; q++) {
        int32_t J[5];
        int e;
        int m = junction_members(g, map, axis, pos, k, q, &e, J);
        if (m == 0) {
            int side = q & 1;
            tb[side] = tk;
            has[side] = 1;
            int64_t fa[3] = {c[0], c[1], c[2]}, fb[3] = {c[0], c[1], c[2]};
            fa[d] = plane - 1;
            fb[d] = plane;
            bfa[side] = fa[1] + (int64_t)g.n * fa[2];
            bfb[side] = fb[1] + (int64_t)g.n * fb[2];
            continue;
        }
        if (g.flux && g.junction && m >= 3) {  // the flux to the intersection cell
            int64_t id = intersection_of(g, map, axis, pos, J, m);
            if (id < 0) continue;  // unreachable: the lowest member owns every such junction
            int rank = 0;
            while (J[rank] != k) rank++;
            row[cnt].c = (int32_t)(g.GF + g.ioff[id] + rank);
            row[cnt].t = 1.0;
            cnt++;
            continue;
        }
        double S = 0.0;
        if (g.junction)
            for (int r = 0; r < m; r++) S += half_t(g, kf, ap, J[r]);
        for (int r = 0; r < m; r++) {
            const int32_t l = J[r];
            if (l == k) continue;
            double tl = half_t(g, kf, ap, l);
            row[cnt].c = (int32_t)(g.n_m + l);
            row[cnt].t = g.junction ? (tk * tl) / S : (tk * tl) / (tk + tl);
            cnt++;
        }
    }
    return cnt;
}

// ---- intersection tables (flux form, junction rule 1)

// junctions of >= 3 cells owned (lowest member) by each fracture cell
__global__ void k_junc_own(GridD g, const int32_t *__restrict__ map, const int32_t *__restrict__ axis,
                           const int32_t *__restrict__ pos, int32_t *__restrict__ cnt) {
    mds_pdl_entry();
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= g.nf) return;
    int own = 0;
    for (int q = 0; q < 2 * (g.dim - 1); q++) {
        int32_t J[5];
        int e;
        int m = junction_members(g, map, axis, pos, k, q, &e, J);
        own += (m >= 3 && J[0] == k) ? 1 : 0;
    }
    cnt[k] = own;
}

__global__ void k_junc_list(GridD g, const int32_t *__restrict__ map, const int32_t *__restrict__ axis,
                            const int32_t *__restrict__ pos, const int32_t *__restrict__ own_base,
                            int32_t *__restrict__ isz, int32_t *__restrict__ imem) {
    mds_pdl_entry();
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= g.nf) return;
    int64_t id = own_base[k];
    for (int q = 0; q < 2 * (g.dim - 1); q++) {
        int32_t J[5];
        int e;
        int m = junction_members(g, map, axis, pos, k, q, &e, J);
        if (m < 3 || J[0] != k) continue;
        isz[id] = m;
        for (int r = 0; r < 4; r++) imem[4 * id + r] = r < m ? J[r] : -1;
        id++;
    }
}

__global__ void k_junc_phi(int64_t nI, const int32_t *__restrict__ ioff, int32_t *__restrict__ phi_int) {
    mds_pdl_entry();
    int64_t I = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nI) return;
    for (int32_t p = ioff[I]; p < ioff[I + 1]; p++) phi_int[p] = (int32_t)I;
}

// Position of a local unknown of an instance in the output system: the
// identity for a single instance; in a packed batch, matrix rows at mo + i and
// fracture rows at fbase + (i - n_m).  Monotone, so sorted rows stay sorted.
struct Remap {
    int64_t n_m, mo, fbase;
    __device__ __forceinline__ int64_t operator()(int64_t j) const { return j < n_m ? mo + j : fbase + (j - n_m); }
};

__global__ void k_half_res(int64_t n_m, double h, const double *__restrict__ km, double *__restrict__ hk) {
    mds_pdl_entry();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_m) hk[i] = h / (2.0 * km[i]);
}

// Matrix row i: the faces are visited in ascending order of the neighbour
// they lead to (-z, -y, -x, +x, +y, +z), so the matrix columns come out
// sorted without a sort; fracture (or flux) columns, all above the matrix
// block, follow in ascending order.  The diagonal sums the transmissibilities
// in ascending column order and then the Dirichlet faces, as the general
// path does.  Everything is held in registers (fixed slot per face).
__device__ void fill_matrix_row(const GridD &g, const int32_t *map, const double *km, const double *ap, int nrhs,
                                const double *pL, const double *pR, int64_t i, const Remap &rm, int64_t NT,
                                const int32_t *rp, int32_t *ci, double *val, double *b) {
    const int64_t n = g.n;
    const int64_t c[3] = {i % n, (i / n) % n, g.dim == 3 ? i / (n * n) : 0};
    const double ki = km[i];
    const double ri = half_res(g, km, i);
    int64_t col[6];
    double t[6];
    bool fr[6];
    double tb[2] = {0.0, 0.0};
    bool has[2] = {false, false};
    int nmat = 0, nlow = 0, nfr = 0;
#pragma unroll
    for (int q = 0; q < 6; q++) {
        const int d = q < 3 ? 2 - q : q - 3;
        const int s = q < 3 ? 0 : 1;
        col[q] = -1;
        t[q] = 0.0;
        fr[q] = false;
        if (d >= g.dim) continue;
        const int64_t plane = c[d] + s;
        if (plane == 0 || plane == n) {
            if (d == 0) {
                tb[s] = (g.F * (2.0 * ki)) / g.h;
                has[s] = true;
            }
            continue;
        }
        int64_t fc[3] = {c[0], c[1], c[2]};
        fc[d] = plane;
        const int32_t k = frac_at(g, map, d, fc);
        if (k >= 0) {
            const double kappa = (2.0 * g.kn[k]) / ap[k];
            fr[q] = true;
            nfr++;
            if (g.flux) {
                col[q] = g.NO + 2 * (int64_t)k + (s ? 0 : 1);
                t[q] = 1.0;
            } else {
                col[q] = g.n_m + k;
                t[q] = g.F / (ri + 1.0 / kappa);
            }
        } else {
            int64_t nc[3] = {c[0], c[1], c[2]};
            nc[d] = c[d] + (s ? 1 : -1);
            const int64_t j = cell_id(g, nc);
            col[q] = j;
            t[q] = g.F / (ri + half_res(g, km, j));
            nmat++;
            nlow += s == 0 ? 1 : 0;
        }
    }
    const int64_t oi = rm(i);
    const int64_t p0 = rp[oi];
    double diag = 0.0;
    int64_t p = p0;
#pragma unroll
    for (int q = 0; q < 6; q++) {
        if (col[q] < 0 || fr[q]) continue;
        if (p == p0 + nlow) p++;  // the diagonal's place
        ci[p] = (int32_t)rm(col[q]);
        val[p++] = -t[q];
        diag += t[q];
    }
    // fracture / flux columns: selection in ascending order (at most six)
    int64_t last = -1;
    for (int r = 0; r < nfr; r++) {
        int64_t best = INT64_MAX;
        double bt = 0.0;
#pragma unroll
        for (int q = 0; q < 6; q++)
            if (fr[q] && col[q] > last && col[q] < best) {
                best = col[q];
                bt = t[q];
            }
        ci[p0 + nmat + 1 + r] = (int32_t)rm(best);
        val[p0 + nmat + 1 + r] = best < g.NO ? -bt : bt;
        if (best < g.NO) diag += bt;
        last = best;
    }
    for (int s = 0; s < 2; s++)
        if (has[s]) diag += tb[s];
    ci[p0 + nlow] = (int32_t)oi;
    val[p0 + nlow] = diag;
    const int64_t bf = (i / n) % n + (g.dim == 3 ? n * (i / (n * n)) : 0);
    for (int r = 0; r < nrhs; r++) {
        const double *L = pL + (int64_t)r * g.nb, *R = pR + (int64_t)r * g.nb;
        double acc = 0.0;
        if (has[0]) acc += tb[0] * L[bf];
        if (has[1]) acc += tb[1] * R[bf];
        b[(int64_t)r * NT + oi] = acc;
    }
}

// Row i of the primal system (a matrix or a fracture cell): its entries in
// ascending column order, the diagonal, and its right-hand sides, written at
// the remapped row and columns (entries from rp[row], b[r NT + row]).
__device__ void fill_primal_row(const GridD &g, const int32_t *map, const double *km, const int32_t *axis,
                                const int32_t *pos, const double *kf, const double *ap, int nrhs, const double *pL,
                                const double *pR, int64_t i, const Remap &rm, int64_t NT, const int32_t *rp,
                                int32_t *ci, double *val, double *b) {
    if (i < g.n_m) {
        fill_matrix_row(g, map, km, ap, nrhs, pL, pR, i, rm, NT, rp, ci, val, b);
        return;
    }
    Ent row[16];
    double tb[2];
    int has[2];
    int64_t bfa[2] = {0, 0}, bfb[2] = {0, 0};
    bool is_m = i < g.n_m;
    int cnt = is_m ? matrix_entries(g, map, km, kf, ap, i, row, tb, has)
                   : fracture_entries(g, map, km, axis, pos, kf, ap, i - g.n_m, row, tb, has, bfa, bfb);
    sort_ents(row, cnt);
    // diagonal: the transmissibilities of the row (flux columns carry none)
    double diag = 0.0;
    for (int q = 0; q < cnt; q++)
        if (row[q].c < g.NO) diag += row[q].t;
    for (int s = 0; s < 2; s++)
        if (has[s]) diag += tb[s];
    const int64_t oi = rm(i);
    int64_t p = rp[oi];
    bool placed = false;
    for (int q = 0; q < cnt; q++) {
        if (!placed && row[q].c > i) {
            ci[p] = (int32_t)oi;
            val[p++] = diag;
            placed = true;
        }
        ci[p] = (int32_t)rm(row[q].c);
        val[p++] = row[q].c < g.NO ? -row[q].t : row[q].t;
    }
    if (!placed) {
        ci[p] = (int32_t)oi;
        val[p] = diag;
    }
    for (int r = 0; r < nrhs; r++) {
        const double *L = pL + (int64_t)r * g.nb, *R = pR + (int64_t)r * g.nb;
        double acc = 0.0;
        if (is_m) {
            int64_t n = g.n;
            int64_t bf = (i / n) % n + (g.dim == 3 ? n * (i / (n * n)) : 0);
            if (has[0]) acc += tb[0] * L[bf];
            if (has[1]) acc += tb[1] * R[bf];
        } else {
            for (int s = 0; s < 2; s++) {
                if (!has[s]) continue;
                const double *P = s == 0 ? L : R;
                double pv = (P[bfa[s]] + P[bfb[s]]) * 0.5;
                acc += tb[s] * pv;
            }
        }
        b[(int64_t)r * NT + oi] = acc;
    }
}


// Entries (diagonal included) of row i of the primal system.
__device__ __forceinline__ int count_primal_row(const GridD &g, const int32_t *map, const double *km,
                                                const int32_t *axis, const int32_t *pos, const double *kf,
                                                const double *ap, int64_t i) {
    Ent row[16];
    double tb[2];
    int has[2];
    int64_t bfa[2], bfb[2];
    int m = i < g.n_m ? matrix_entries(g, map, km, kf, ap, i, row, tb, has)
                      : fracture_entries(g, map, km, axis, pos, kf, ap, i - g.n_m, row, tb, has, bfa, bfb);
    return m + 1;
}

__global__ void k_count(GridD g, const int32_t *__restrict__ map, const double *__restrict__ km,
                        const int32_t *__restrict__ axis, const int32_t *__restrict__ pos,
                        const double *__restrict__ kf, const double *__restrict__ ap, int32_t *__restrict__ cnt) {
    mds_pdl_entry();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.NT) return;
    if (i >= g.NO) {  // interface flux row: higher-dimensional cell, lower one, itself
        cnt[i] = 3;
        return;
    }
    if (i >= g.N) {  // intersection cell: zero diagonal and its member fluxes
        int64_t I = i - g.N;
        cnt[i] = 1 + (g.ioff[I + 1] - g.ioff[I]);
        return;
    }
    cnt[i] = count_primal_row(g, map, km, axis, pos, kf, ap, i);
}

__global__ void k_fill(GridD g, const int32_t *__restrict__ map, const double *__restrict__ km,
                       const int32_t *__restrict__ axis, const int32_t *__restrict__ pos,
                       const double *__restrict__ kf, const double *__restrict__ ap, int nrhs,
                       const double *__restrict__ pL, const double *__restrict__ pR, const int32_t *__restrict__ rp,
                       int32_t *__restrict__ ci, double *__restrict__ val, double *__restrict__ b) {
    mds_pdl_entry();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.NT) return;
    if (i >= g.GF) {
        // intersection flux (member l of intersection I): p_l - p_I - lambda / t_l = 0
        int64_t phi = i - g.GF;
        int64_t I = g.phi_int[phi];
        int32_t l = g.imem[4 * I + (phi - g.ioff[I])];
        int64_t p = rp[i];
        ci[p] = (int32_t)(g.n_m + l);
        val[p] = 1.0;
        ci[p + 1] = (int32_t)(g.N + I);
        val[p + 1] = -1.0;
        ci[p + 2] = (int32_t)i;
        val[p + 2] = -1.0 / half_t(g, kf, ap, l);
        for (int r = 0; r < nrhs; r++) b[(int64_t)r * g.NT + i] = 0.0;
        return;
    }
    if (i >= g.N && i < g.NO) {  // intersection cell
        int64_t I = i - g.N;
        int64_t p = rp[i];
        ci[p] = (int32_t)i;
        val[p++] = 0.0;
        for (int32_t f = g.ioff[I]; f < g.ioff[I + 1]; f++) {
            ci[p] = (int32_t)(g.GF + f);
            val[p++] = -1.0;
        }
        for (int r = 0; r < nrhs; r++) b[(int64_t)r * g.NT + i] = 0.0;
        return;
    }
    if (i >= g.NO) {
        // interface law of flux j = 2k + s: p_i - p_k - lambda_j / T_j = 0
        int64_t j = i - g.NO, k = j / 2;
        int s = (int)(j % 2);
        int d = axis[k];
        int64_t mc[3] = {pos[3 * k], pos[3 * k + 1], g.dim == 3 ? pos[3 * k + 2] : 0};
        mc[d] = mc[d] - 1 + s;
        int64_t m = cell_id(g, mc);
        double kappa = (2.0 * g.kn[k]) / ap[k];
        double t = g.F / (g.h / (2.0 * km[m]) + 1.0 / kappa);
        int64_t p = rp[i];
        ci[p] = (int32_t)m;
        val[p] = 1.0;
        ci[p + 1] = (int32_t)(g.n_m + k);
        val[p + 1] = -1.0;
        ci[p + 2] = (int32_t)i;
        val[p + 2] = -1.0 / t;
        for (int r = 0; r < nrhs; r++) b[(int64_t)r * g.NT + i] = 0.0;
        return;
    }
    fill_primal_row(g, map, km, axis, pos, kf, ap, nrhs, pL, pR, i, Remap{g.n_m, 0, g.n_m}, g.NT, rp, ci, val, b);
}

// ---------------------------------------------------------------- block split / merge

__global__ void k_split_count(int64_t N, int64_t n_m, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                              int32_t *__restrict__ lo, int32_t *__restrict__ hi) {
    mds_pdl_entry();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    int32_t a = rp[i], e = rp[i + 1], m = a;
    while (m < e && ci[m] < n_m) m++;
    lo[i] = m - a;
    hi[i] = e - m;
}

__global__ void k_split_fill(int64_t N, int64_t n_m, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                             const double *__restrict__ v, const int32_t *__restrict__ rp_mm,
                             int32_t *__restrict__ c_mm, double *__restrict__ v_mm, const int32_t *__restrict__ rp_mf,
                             int32_t *__restrict__ c_mf, double *__restrict__ v_mf, const int32_t *__restrict__ rp_fm,
                             int32_t *__restrict__ c_fm, double *__restrict__ v_fm, const int32_t *__restrict__ rp_ff,
                             int32_t *__restrict__ c_ff, double *__restrict__ v_ff) {
    mds_pdl_entry();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    bool mrow = i < n_m;
    int64_t li = mrow ? i : i - n_m;
    int32_t plo = mrow ? rp_mm[li] : rp_fm[li];
    int32_t phi = mrow ? rp_mf[li] : rp_ff[li];
    int32_t *clo = mrow ? c_mm : c_fm, *chi = mrow ? c_mf : c_ff;
    double *vlo = mrow ? v_mm : v_fm, *vhi = mrow ? v_mf : v_ff;
    for (int32_t p = rp[i]; p < rp[i + 1]; p++) {
        int32_t j = ci[p];
        if (j < n_m) {
            clo[plo] = j;
            vlo[plo++] = v[p];
        } else {
            chi[phi] = (int32_t)(j - n_m);
            vhi[phi++] = v[p];
        }
    }
}

void split_blocks(Ctx &c, const mds_csr &full, int64_t n_m, DCsr blk[4]) {
    int64_t N = full.nrow, n_f = N - n_m;
    Buf lo(&c, sizeof(int32_t) * (size_t)(N + 1)), hi(&c, sizeof(int32_t) * (size_t)(N + 1));
    MDS_LAUNCH(c, KC_NONE, 0, k_split_count, grid_for(N, 256), 256, 0, N, n_m, full.row_ptr, full.col,
               lo.as<int32_t>(), hi.as<int32_t>());
    int64_t rows[4] = {n_m, n_m, n_f, n_f};
    int64_t cols[4] = {n_m, n_f, n_m, n_f};
    const int32_t *src[4] = {lo.as<int32_t>(), hi.as<int32_t>(), lo.as<int32_t>() + n_m, hi.as<int32_t>() + n_m};
    for (int q = 0; q < 4; q++) {
        Buf rp(&c, sizeof(int32_t) * (size_t)(rows[q] + 1));
        int64_t nnz = scan_counts(c, src[q], rp.as<int32_t>(), rows[q]);
        blk[q].nrow = rows[q];
        blk[q].ncol = cols[q];
        blk[q].nnz = nnz;
        blk[q].rp = std::move(rp);
        blk[q].ci = Buf(&c, sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
        blk[q].v = Buf(&c, sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
    }
    MDS_LAUNCH(c, KC_NONE, 0, k_split_fill, grid_for(N, 256), 256, 0, N, n_m, full.row_ptr, full.col, full.val,
               blk[0].rowp(), blk[0].cols(), blk[0].vals(), blk[1].rowp(), blk[1].cols(), blk[1].vals(),
               blk[2].rowp(), blk[2].cols(), blk[2].vals(), blk[3].rowp(), blk[3].cols(), blk[3].vals());
}

__global__ void k_merge_count(int64_t N, int64_t n_m, const int32_t *rp0, const int32_t *rp1, const int32_t *rp2,
                              const int32_t *rp3, int32_t *cnt) {
    mds_pdl_entry();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    if (i < n_m)
        cnt[i] = (rp0[i + 1] - rp0[i]) + (rp1[i + 1] - rp1[i]);
    else {
        int64_t k = i - n_m;
        cnt[i] = (rp2[k + 1] - rp2[k]) + (rp3[k + 1] - rp3[k]);
    }
}

__global__ void k_merge_fill(int64_t N, int64_t n_m, mds_csr b0, mds_csr b1, mds_csr b2, mds_csr b3,
                             const int32_t *__restrict__ rp, int32_t *__restrict__ ci, double *__restrict__ v) {
    mds_pdl_entry();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const mds_csr &L = i < n_m ? b0 : b2;
    const mds_csr &R = i < n_m ? b1 : b3;
    int64_t li = i < n_m ? i : i - n_m;
    int32_t p = rp[i];
    for (int32_t q = L.row_ptr[li]; q < L.row_ptr[li + 1]; q++) {
        ci[p] = L.col[q];
        v[p++] = L.val[q];
    }
    for (int32_t q = R.row_ptr[li]; q < R.row_ptr[li + 1]; q++) {
        ci[p] = (int32_t)(R.col[q] + n_m);
        v[p++] = R.val[q];
    }
}

void merge_blocks(Ctx &c, const mds_csr blk[4], int64_t n_m, int64_t n_f, DCsr &full) {
    int64_t N = n_m + n_f;
    Buf cnt(&c, sizeof(int32_t) * (size_t)(N + 1));
    MDS_LAUNCH(c, KC_NONE, 0, k_merge_count, grid_for(N, 256), 256, 0, N, n_m, blk[0].row_ptr, blk[1].row_ptr,
               blk[2].row_ptr, blk[3].row_ptr, cnt.as<int32_t>());
    full.nrow = N;
    full.ncol = N;
    full.rp = Buf(&c, sizeof(int32_t) * (size_t)(N + 1));
    full.nnz = scan_counts(c, cnt.as<int32_t>(), full.rowp(), N);
    full.ci = Buf(&c, sizeof(int32_t) * (size_t)(full.nnz > 0 ? full.nnz : 1));
    full.v = Buf(&c, sizeof(double) * (size_t)(full.nnz > 0 ? full.nnz : 1));
    MDS_LAUNCH(c, KC_NONE, 0, k_merge_fill, grid_for(N, 256), 256, 0, N, n_m, blk[0], blk[1], blk[2], blk[3],
               full.rowp(), full.cols(), full.vals());
}

// ---------------------------------------------------------------- packing of instances

// rows of one block of one instance into the packed block: row r goes to
// row_off + r, its entries to nnz_off + ..., columns shifted by col_off
__global__ void k_concat_rows(int64_t nrow, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                              const double *__restrict__ v, int64_t row_off, int64_t nnz_off, int64_t col_off,
                              int32_t *__restrict__ rp_dst, int32_t *__restrict__ ci_dst, double *__restrict__ v_dst) {
    mds_pdl_entry();
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrow) return;
    rp_dst[row_off + r] = (int32_t)(nnz_off + rp[r]);
    for (int32_t p = rp[r]; p < rp[r + 1]; p++) {
        ci_dst[nnz_off + p] = (int32_t)(ci[p] + col_off);
        v_dst[nnz_off + p] = v[p];
    }
}

// Block-diagonal packing: unknowns [m_0 .. m_{K-1}; f_0 .. f_{K-1}], so the
// packed system keeps the 2x2 block structure of Eq. (4) and each diagonal
// block is block diagonal over the instances.
void pack_instances(Ctx &c, std::vector<SystemData> &parts, SystemData &out) {
    const int K = (int)parts.size();
    MDS_REQUIRE(K >= 1, MDS_ERR_INVALID, "no instances");
    out.nrhs = parts[0].nrhs;
    out.moff.assign(K + 1, 0);
    out.foff.assign(K + 1, 0);
    for (int k = 0; k < K; k++) {
        MDS_REQUIRE(parts[k].nrhs == out.nrhs, MDS_ERR_INVALID, "instances of a batch need the same nrhs");
        out.moff[k + 1] = out.moff[k] + parts[k].n_m;
        out.foff[k + 1] = out.foff[k] + parts[k].n_f;
    }
    const int64_t NM = out.moff[K], NF = out.foff[K], N = NM + NF;
    MDS_REQUIRE(N < INT32_MAX, MDS_ERR_INVALID, "packed batch exceeds int32 indices");
    out.stencil = true;
    out.dim = parts[0].dim;
    out.side.clear();
    for (int k = 0; k < K; k++) {
        out.stencil = out.stencil && parts[k].stencil && parts[k].dim == out.dim && parts[k].side.size() == 1;
        out.side.push_back(parts[k].side.empty() ? 0 : parts[k].side[0]);
    }
    out.n_m = NM;
    out.n_f = NF;
    for (int q = 0; q < 4; q++) {
        bool mrow = q < 2, mcol = q % 2 == 0;
        int64_t nrow = mrow ? NM : NF, ncol = mcol ? NM : NF, nnz = 0;
        for (int k = 0; k < K; k++) nnz += parts[k].blk[q].nnz;
        MDS_REQUIRE(nnz < INT32_MAX, MDS_ERR_INVALID, "packed batch exceeds 2^31-1 nonzeros");
        out.blk[q] = csr_alloc(c, nrow, ncol, nnz);
        int64_t at = 0;
        for (int k = 0; k < K; k++) {
            const DCsr &B = parts[k].blk[q];
            int64_t roff = mrow ? out.moff[k] : out.foff[k], coff = mcol ? out.moff[k] : out.foff[k];
            if (B.nrow > 0)
                MDS_LAUNCH(c, KC_NONE, 0, k_concat_rows, grid_for(B.nrow, 256), 256, 0, B.nrow, B.rowp(), B.cols(),
                           B.vals(), roff, at, coff, out.blk[q].rowp(), out.blk[q].cols(), out.blk[q].vals());
            at += B.nnz;
        }
        int32_t last = (int32_t)nnz;
        std::memcpy(c.h_pin, &last, sizeof last);
        MDS_CUDA(cudaMemcpyAsync(out.blk[q].rowp() + nrow, c.h_pin, sizeof last, cudaMemcpyHostToDevice, c.stream));
        c.sync();
    }
    mds_csr views[4] = {out.blk[0].view(), out.blk[1].view(), out.blk[2].view(), out.blk[3].view()};
    merge_blocks(c, views, NM, NF, out.full);
    out.b = Buf(&c, sizeof(double) * (size_t)(N * out.nrhs));
    for (int k = 0; k < K; k++) {
        const SystemData &S = parts[k];
        int64_t Nk = S.n_m + S.n_f;
        for (int r = 0; r < out.nrhs; r++) {
            const double *src = S.b.as<double>() + (int64_t)r * Nk;
            double *dst = out.b.as<double>() + (int64_t)r * N;
            if (S.n_m)
                MDS_CUDA(cudaMemcpyAsync(dst + out.moff[k], src, sizeof(double) * (size_t)S.n_m,
                                         cudaMemcpyDeviceToDevice, c.stream));
            if (S.n_f)
                MDS_CUDA(cudaMemcpyAsync(dst + NM + out.foff[k], src + S.n_m, sizeof(double) * (size_t)S.n_f,
                                         cudaMemcpyDeviceToDevice, c.stream));
        }
    }
    c.sync();
}

// ---------------------------------------------------------------- packed batches (primal form)
//
// Every instance of a batch is assembled straight into the packed system
// [m_0 .. m_K-1; f_0 .. f_K-1]: one launch per phase for all instances
// (blockIdx.y = instance), one prefix sum over the packed rows.  Each row is
// computed by the same functions as for a single instance, its row and
// columns remapped to their packed positions.

struct BInst {
    GridD g;
    const double *km, *kf, *ap, *pL, *pR;
    const int32_t *ax, *ps;
    int32_t *map;          // the instance's face map
    double *hk;            // its half-cell resistances (g.hk points here)
    int64_t mo, fbase;     // packed rows of its first matrix cell and first fracture cell
};

__global__ void k_half_res_b(const BInst *__restrict__ bi) {
    mds_pdl_entry();
    const BInst &B = bi[blockIdx.y];
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < B.g.n_m) B.hk[i] = B.g.h / (2.0 * B.km[i]);
}

__global__ void k_map_scatter_b(const BInst *__restrict__ bi, int *err) {
    mds_pdl_entry();
    const BInst &B = bi[blockIdx.y];
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= B.g.nf) return;
    scatter_face(B.g, B.ax, B.ps, B.map, err, k);
}

__global__ void k_count_b(const BInst *__restrict__ bi, int32_t *__restrict__ cnt) {
    mds_pdl_entry();
    const BInst &B = bi[blockIdx.y];
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B.g.N) return;
    const Remap rm{B.g.n_m, B.mo, B.fbase};
    cnt[rm(i)] = count_primal_row(B.g, B.map, B.km, B.ax, B.ps, B.kf, B.ap, i);
}

__global__ void k_fill_b(const BInst *__restrict__ bi, int nrhs, int64_t NT, const int32_t *__restrict__ rp,
                         int32_t *__restrict__ ci, double *__restrict__ val, double *__restrict__ b) {
    mds_pdl_entry();
    const BInst &B = bi[blockIdx.y];
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B.g.N) return;
    fill_primal_row(B.g, B.map, B.km, B.ax, B.ps, B.kf, B.ap, nrhs, B.pL, B.pR, i, Remap{B.g.n_m, B.mo, B.fbase}, NT,
                    rp, ci, val, b);
}

// ---------------------------------------------------------------- driver

template <class T>
static const T *stage(Ctx &c, const T *p, size_t count, bool on_device, Buf &hold) {
    if (on_device || count == 0) return p;
    hold = Buf(&c, sizeof(T) * count);
    MDS_CUDA(cudaMemcpyAsync(hold.p, p, sizeof(T) * count, cudaMemcpyHostToDevice, c.stream));
    return hold.as<T>();
}

// The grid description of an instance (faces counted in *faces); checks the
// instance's sizes and arrays.
static GridD grid_of(const mds_instance &in, bool flux, int64_t *faces) {
    MDS_REQUIRE(in.dim == 2 || in.dim == 3, MDS_ERR_INVALID, "dim must be 2 or 3");
    MDS_REQUIRE(in.n >= 1 && in.nrhs >= 1 && in.n_f >= 0, MDS_ERR_INVALID, "bad instance sizes");
    MDS_REQUIRE(in.km && in.pD_left && in.pD_right, MDS_ERR_INVALID, "missing instance arrays");
    MDS_REQUIRE(in.n_f == 0 || (in.fc_axis && in.fc_pos && in.fc_kf && in.fc_a), MDS_ERR_INVALID,
                "missing fracture arrays");
    GridD g{};
    g.dim = in.dim;
    g.n = in.n;
    int64_t n = in.n;
    int64_t total = 0;
    for (int d = 0; d < 3; d++) {
        for (int a = 0; a < 3; a++) g.ext[d][a] = (a < in.dim) ? (a == d ? n + 1 : n) : 1;
        g.off[d] = total;
        if (d < in.dim) total += g.ext[d][0] * g.ext[d][1] * g.ext[d][2];
    }
    g.h = 1.0 / (double)in.n;
    g.F = in.dim == 2 ? g.h : g.h * g.h;
    g.elen = in.dim == 2 ? 1.0 : g.h;
    g.n_m = in.dim == 3 ? n * n * n : n * n;
    g.nf = in.n_f;
    g.N = g.n_m + g.nf;
    g.flux = flux ? 1 : 0;
    MDS_REQUIRE(in.junction == MDS_JUNCTION_PAIRWISE || in.junction == MDS_JUNCTION_STAR, MDS_ERR_INVALID,
                "unknown junction rule");
    g.junction = in.junction;
    g.nb = in.dim == 3 ? n * n : n;
    MDS_REQUIRE(g.N + 2 * g.nf < INT32_MAX, MDS_ERR_INVALID, "too many unknowns for int32 indices");
    // the primal form has no intersection unknowns nor fluxes
    g.NO = g.N;
    g.GF = g.NO;
    g.NT = g.N;
    *faces = total;
    return g;
}

// One copy segment of the batched host-to-device gather.
struct CopySeg {
    const uint4 *src;  // device address of page-locked host memory (16-byte aligned)
    uint4 *dst;        // 16-byte aligned
    int64_t bytes;
};

// All segments in one launch: block b copies segment b, its threads striding
// over 16-byte units (the host arrays are read once over the host link) and
// the last thread copying the bytes after the last full unit.
__global__ void k_gather_segments(const CopySeg *__restrict__ seg) {
    mds_pdl_entry();
    const CopySeg g = seg[blockIdx.x];
    const int64_t n16 = g.bytes / 16;
    for (int64_t i = threadIdx.x; i < n16; i += blockDim.x) g.dst[i] = g.src[i];
    if (threadIdx.x == blockDim.x - 1)
        for (int64_t b = n16 * 16; b < g.bytes; b++)
            reinterpret_cast<char *>(g.dst)[b] = reinterpret_cast<const char *>(g.src)[b];
}

void assemble_batch_primal(Ctx &c, const mds_instance *inst, int K, SystemData &out) {
    MDS_REQUIRE(K >= 1 && K <= 65535, MDS_ERR_INVALID, "a batch holds 1 to 65535 instances");
    std::vector<BInst> hb(K);
    std::vector<int64_t> faces(K);
    std::vector<Buf> hold;
    hold.reserve((size_t)K * 8);
    // Host arrays in page-locked memory the device can address are gathered
    // by one kernel into one device buffer (instead of one copy call per
    // array); the others are staged one copy each.
    struct Pend {
        const void *src;
        size_t bytes;
        const void **slot;
    };
    std::vector<Pend> pend;
    size_t pend_bytes = 0;
    // *dst = a device copy of p[0 .. count) (p itself when on the device)
    auto stg = [&](auto **dst, auto p, size_t count, bool dev) {
        using T = std::remove_const_t<std::remove_pointer_t<decltype(p)>>;
        if (!dev && count > 0) {
            cudaPointerAttributes a;
            if (cudaPointerGetAttributes(&a, p) == cudaSuccess && a.type == cudaMemoryTypeHost && a.devicePointer &&
                (reinterpret_cast<uintptr_t>(a.devicePointer) & 15) == 0) {
                pend.push_back(Pend{a.devicePointer, sizeof(T) * count, reinterpret_cast<const void **>(dst)});
                pend_bytes += (sizeof(T) * count + 15) / 16 * 16;
                *dst = nullptr;  // set after the gather
                return;
            }
            cudaGetLastError();
        }
        hold.emplace_back();
        *dst = stage<T>(c, p, count, dev, hold.back());
    };
    out.nrhs = inst[0].nrhs;
    out.moff.assign(K + 1, 0);
    out.foff.assign(K + 1, 0);
    out.stencil = true;
    out.dim = inst[0].dim;
    out.side.assign(K, 0);
    int64_t total_faces = 0, maxN = 0, maxf = 0;
    for (int k = 0; k < K; k++) {
        const mds_instance &in = inst[k];
        MDS_REQUIRE(in.nrhs == out.nrhs, MDS_ERR_INVALID, "instances of a batch need the same nrhs");
        GridD g = grid_of(in, false, &faces[k]);
        bool dev = in.on_device != 0;
        BInst &B = hb[k];
        B.g = g;
        stg(&B.km, in.km, (size_t)g.n_m, dev);
        stg(&B.ax, in.fc_axis, (size_t)g.nf, dev);
        stg(&B.ps, in.fc_pos, (size_t)(3 * g.nf), dev);
        stg(&B.kf, in.fc_kf, (size_t)g.nf, dev);
        stg(&B.ap, in.fc_a, (size_t)g.nf, dev);
        stg(&B.pL, in.pD_left, (size_t)(in.nrhs * g.nb), dev);
        stg(&B.pR, in.pD_right, (size_t)(in.nrhs * g.nb), dev);
        if (in.fc_kn) stg(&B.g.kn, in.fc_kn, (size_t)g.nf, dev);
        out.moff[k + 1] = out.moff[k] + g.n_m;
        out.foff[k + 1] = out.foff[k] + g.nf;
        out.stencil = out.stencil && in.dim == out.dim;
        out.side[k] = in.n;
        total_faces += faces[k];
        maxN = std::max(maxN, g.N);
        maxf = std::max(maxf, g.nf);
    }
    if (!pend.empty()) {
        Buf gath(&c, pend_bytes);
        std::vector<CopySeg> segs;
        size_t o = 0;
        for (const Pend &q : pend) {
            char *d = static_cast<char *>(gath.p) + o;
            segs.push_back(CopySeg{static_cast<const uint4 *>(q.src), reinterpret_cast<uint4 *>(d), (int64_t)q.bytes});
            *q.slot = d;
            o += (q.bytes + 15) / 16 * 16;
        }
        Buf dseg(&c, sizeof(CopySeg) * segs.size());
        MDS_CUDA(cudaMemcpyAsync(dseg.p, segs.data(), sizeof(CopySeg) * segs.size(), cudaMemcpyHostToDevice, c.stream));
        MDS_LAUNCH(c, KC_NONE, 0, k_gather_segments, (unsigned)segs.size(), 256, 0, dseg.as<CopySeg>());
        c.sync();  // the segment table is released on return
        hold.push_back(std::move(gath));
    }
    for (int k = 0; k < K; k++)
        if (!inst[k].fc_kn) hb[k].g.kn = hb[k].kf;  // the normal permeability defaults to k_f
    const int64_t NM = out.moff[K], NF = out.foff[K], N = NM + NF;
    MDS_REQUIRE(N < INT32_MAX, MDS_ERR_INVALID, "packed batch exceeds int32 indices");
    Buf map(&c, sizeof(int32_t) * (size_t)(total_faces > 0 ? total_faces : 1));
    fill_i32(c, map.as<int32_t>(), -1, total_faces);
    Buf hk(&c, sizeof(double) * (size_t)(NM > 0 ? NM : 1));
    int64_t at = 0, maxm = 0;
    for (int k = 0; k < K; k++) {
        hb[k].map = map.as<int32_t>() + at;
        hb[k].hk = hk.as<double>() + out.moff[k];
        hb[k].g.hk = hb[k].hk;
        maxm = std::max(maxm, hb[k].g.n_m);
        at += faces[k];
        hb[k].mo = out.moff[k];
        hb[k].fbase = NM + out.foff[k];
    }
    Buf bi(&c, sizeof(BInst) * (size_t)K);
    MDS_CUDA(cudaMemcpyAsync(bi.p, hb.data(), sizeof(BInst) * (size_t)K, cudaMemcpyHostToDevice, c.stream));
    const BInst *B = bi.as<BInst>();
    c.clear_err();
    if (maxf > 0)
        MDS_LAUNCH(c, KC_NONE, 0, k_map_scatter_b, dim3(grid_for(maxf, 256), K), 256, 0, B, c.d_err);
    c.check_err("fracture list");
    if (maxm > 0) MDS_LAUNCH(c, KC_NONE, 0, k_half_res_b, dim3(grid_for(maxm, 256), K), 256, 0, B);
    Buf cnt(&c, sizeof(int32_t) * (size_t)(N + 1));
    MDS_LAUNCH(c, KC_NONE, 0, k_count_b, dim3(grid_for(maxN, 128), K), 128, 0, B, cnt.as<int32_t>());
    DCsr &A = out.full;
    A.nrow = A.ncol = N;
    A.rp = Buf(&c, sizeof(int32_t) * (size_t)(N + 1));
    A.nnz = scan_counts(c, cnt.as<int32_t>(), A.rowp(), N);
    A.ci = Buf(&c, sizeof(int32_t) * (size_t)A.nnz);
    A.v = Buf(&c, sizeof(double) * (size_t)A.nnz);
    out.b = Buf(&c, sizeof(double) * (size_t)(N * out.nrhs));
    MDS_LAUNCH(c, KC_NONE, 0, k_fill_b, dim3(grid_for(maxN, 128), K), 128, 0, B, out.nrhs, N, A.rowp(), A.cols(),
               A.vals(), out.b.as<double>());
    out.n_m = NM;
    out.n_f = NF;
    split_blocks(c, A.view(), NM, out.blk);
    c.sync();  // staged host copies are released on return
}

void assemble_instance(Ctx &c, const mds_instance &in, SystemData &out, bool flux) {
    int64_t total = 0;
    GridD g = grid_of(in, flux, &total);

    bool dev = in.on_device != 0;
    Buf h0, h1, h2, h3, h4, h5, h6;
    const double *km = stage(c, in.km, (size_t)g.n_m, dev, h0);
    const int32_t *ax = stage(c, in.fc_axis, (size_t)g.nf, dev, h1);
    const int32_t *ps = stage(c, in.fc_pos, (size_t)(3 * g.nf), dev, h2);
    const double *kf = stage(c, in.fc_kf, (size_t)g.nf, dev, h3);
    const double *ap = stage(c, in.fc_a, (size_t)g.nf, dev, h4);
    const double *pL = stage(c, in.pD_left, (size_t)(in.nrhs * g.nb), dev, h5);
    const double *pR = stage(c, in.pD_right, (size_t)(in.nrhs * g.nb), dev, h6);
    Buf h7;
    g.kn = in.fc_kn ? stage(c, in.fc_kn, (size_t)g.nf, dev, h7) : kf;

    Buf map(&c, sizeof(int32_t) * (size_t)total);
    fill_i32(c, map.as<int32_t>(), -1, total);
    c.clear_err();
    if (g.nf > 0)
        MDS_LAUNCH(c, KC_NONE, 0, k_map_scatter, grid_for(g.nf, 256), 256, 0, g, ax, ps, map.as<int32_t>(), c.d_err);
    c.check_err("fracture list");

    // intersection cells and their fluxes (flux form, junction rule 1)
    Buf own_cnt, own_base, isz, ioff, imem, phi;
    int64_t nI = 0, nIF = 0;
    if (flux && g.junction && g.nf > 0) {
        own_cnt = Buf(&c, sizeof(int32_t) * (size_t)(g.nf + 1));
        own_base = Buf(&c, sizeof(int32_t) * (size_t)(g.nf + 1));
        MDS_LAUNCH(c, KC_NONE, 0, k_junc_own, grid_for(g.nf, 128), 128, 0, g, map.as<int32_t>(), ax, ps,
                   own_cnt.as<int32_t>());
        nI = scan_counts(c, own_cnt.as<int32_t>(), own_base.as<int32_t>(), g.nf);
        if (nI > 0) {
            isz = Buf(&c, sizeof(int32_t) * (size_t)(nI + 1));
            imem = Buf(&c, sizeof(int32_t) * (size_t)(4 * nI));
            MDS_LAUNCH(c, KC_NONE, 0, k_junc_list, grid_for(g.nf, 128), 128, 0, g, map.as<int32_t>(), ax, ps,
                       own_base.as<int32_t>(), isz.as<int32_t>(), imem.as<int32_t>());
            ioff = Buf(&c, sizeof(int32_t) * (size_t)(nI + 1));
            nIF = scan_counts(c, isz.as<int32_t>(), ioff.as<int32_t>(), nI);
            phi = Buf(&c, sizeof(int32_t) * (size_t)(nIF > 0 ? nIF : 1));
            MDS_LAUNCH(c, KC_NONE, 0, k_junc_phi, grid_for(nI, 128), 128, 0, nI, ioff.as<int32_t>(),
                       phi.as<int32_t>());
        }
    }
    g.nI = nI;
    g.nIF = nIF;
    g.NO = g.N + nI;
    g.GF = g.NO + 2 * g.nf;
    g.NT = flux ? g.GF + nIF : g.N;
    g.own_base = own_base.p ? own_base.as<int32_t>() : nullptr;
    g.ioff = ioff.p ? ioff.as<int32_t>() : nullptr;
    g.imem = imem.p ? imem.as<int32_t>() : nullptr;
    g.phi_int = phi.p ? phi.as<int32_t>() : nullptr;
    MDS_REQUIRE(g.NT < INT32_MAX, MDS_ERR_INVALID, "too many unknowns for int32 indices");

    Buf hk(&c, sizeof(double) * (size_t)(g.n_m > 0 ? g.n_m : 1));
    if (g.n_m > 0) MDS_LAUNCH(c, KC_NONE, 0, k_half_res, grid_for(g.n_m, 256), 256, 0, g.n_m, g.h, km, hk.as<double>());
    g.hk = hk.as<double>();
    Buf cnt(&c, sizeof(int32_t) * (size_t)(g.NT + 1));
    MDS_LAUNCH(c, KC_NONE, 0, k_count, grid_for(g.NT, 128), 128, 0, g, map.as<int32_t>(), km, ax, ps, kf, ap,
               cnt.as<int32_t>());
    DCsr &A = out.full;
    A.nrow = A.ncol = g.NT;
    A.rp = Buf(&c, sizeof(int32_t) * (size_t)(g.NT + 1));
    A.nnz = scan_counts(c, cnt.as<int32_t>(), A.rowp(), g.NT);
    A.ci = Buf(&c, sizeof(int32_t) * (size_t)A.nnz);
    A.v = Buf(&c, sizeof(double) * (size_t)A.nnz);
    out.b = Buf(&c, sizeof(double) * (size_t)(g.NT * in.nrhs));
    MDS_LAUNCH(c, KC_NONE, 0, k_fill, grid_for(g.NT, 128), 128, 0, g, map.as<int32_t>(), km, ax, ps, kf, ap, in.nrhs,
               pL, pR, A.rowp(), A.cols(), A.vals(), out.b.as<double>());
    // blocks: [matrix; fracture] cells, or [all pressures; interface fluxes]
    const int64_t nm = flux ? g.NO : g.n_m, nfb = flux ? 2 * g.nf + nIF : g.nf;
    out.n_m = nm;
    out.n_f = nfb;
    out.nrhs = in.nrhs;
    out.moff = {0, nm};
    out.foff = {0, nfb};
    out.stencil = !flux;
    out.dim = in.dim;
    out.side = {in.n};
    split_blocks(c, A.view(), nm, out.blk);
    c.sync();  // staged host copies are released on return
}

}  // namespace mds
