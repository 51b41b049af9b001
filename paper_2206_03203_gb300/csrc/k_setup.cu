// Set-up on the GPU: the approximate Schur complement of Eq. (7) and the
// aggregation-AMG hierarchy used for one V-cycle per diagonal block
// (Sec. 3.3): strength graph, deterministic parallel MIS-2 with hash
// priorities, aggregates, piecewise-constant P, Galerkin P^T A P, L1
// diagonals.  Compiled with -fmad=false and a fixed summation order so that
// sparsity, aggregates and FP64 values are reproducible to the bit.
#include "internal.cuh"

namespace mds {

constexpr int SCHUR_CAP = 64;
constexpr int RAP_CAP = 512;

__device__ __forceinline__ int32_t find_col(const int32_t *ci, int32_t a, int32_t e, int32_t j) {
    // binary search in a sorted row segment; -1 if absent
    int32_t lo = a, hi = e - 1;
    while (lo <= hi) {
        int32_t m = (lo + hi) >> 1;
        int32_t c = ci[m];
        if (c == j) return m;
        if (c < j)
            lo = m + 1;
        else
            hi = m - 1;
    }
    return -1;
}

__global__ void k_diag(int64_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                       const double *__restrict__ v, double *__restrict__ d, int need_nonzero, int *err) {
    mds_pdl_entry();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t p = find_col(ci, rp[i], rp[i + 1], (int32_t)i);
    double x = p >= 0 ? v[p] : 0.0;
    d[i] = x;
    if (need_nonzero && x == 0.0) atomicOr(err, DERR_ZERO_DIAG);
}

// ---------------------------------------------------------------- Schur (Eq. 7)

// Row i of S~: start from row i of A_mm, then for each k of row i of A_mf in
// ascending order subtract (A_mf)_ik (A_fm)_kj / d_k from entry j.
template <bool FILL>
__global__ void k_schur(int64_t nm, mds_csr Amm, mds_csr Amf, mds_csr Afm, const double *__restrict__ dk,
                        int32_t *__restrict__ cnt, const int32_t *__restrict__ rp, int32_t *__restrict__ ci,
                        double *__restrict__ val, int *err) {
    mds_pdl_entry();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nm) return;
    int32_t cols[SCHUR_CAP];
    double acc[SCHUR_CAP];
    int m = 0;
    for (int32_t p = Amm.row_ptr[i]; p < Amm.row_ptr[i + 1]; p++) {
        if (m >= SCHUR_CAP) {
            atomicOr(err, DERR_CAPACITY);
            return;
        }
        cols[m] = Amm.col[p];
        acc[m++] = Amm.val[p];
    }
    for (int32_t p = Amf.row_ptr[i]; p < Amf.row_ptr[i + 1]; p++) {
        int32_t k = Amf.col[p];
        double a = Amf.val[p];
        double d = dk[k];
        for (int32_t q = Afm.row_ptr[k]; q < Afm.row_ptr[k + 1]; q++) {
            int32_t j = Afm.col[q];
            int t = 0;
            while (t < m && cols[t] != j) t++;
            if (t == m) {
                if (m >= SCHUR_CAP) {
                    atomicOr(err, DERR_CAPACITY);
                    return;
                }
                cols[m] = j;
                acc[m++] = 0.0;
            }
            acc[t] = acc[t] - (a * Afm.val[q]) / d;
        }
    }
    if constexpr (!FILL) {
        cnt[i] = m;
        return;
    } else {
    for (int a = 1; a < m; a++) {
        int32_t x = cols[a];
        double y = acc[a];
        int q = a - 1;
        while (q >= 0 && cols[q] > x) {
            cols[q + 1] = cols[q];
            acc[q + 1] = acc[q];
            q--;
        }
        cols[q + 1] = x;
        acc[q + 1] = y;
    }
    int32_t o = rp[i];
    for (int a = 0; a < m; a++) {
        ci[o + a] = cols[a];
        val[o + a] = acc[a];
    }
    }
}

DCsr schur_build(Ctx &c, const mds_csr &Amm, const mds_csr &Amf, const mds_csr &Afm, const mds_csr &Aff, Buf &dk) {
    int64_t nm = Amm.nrow, nf = Aff.nrow;
    dk = Buf(&c, sizeof(double) * (size_t)(nf > 0 ? nf : 1));
    c.clear_err();
    if (nf > 0)
        MDS_LAUNCH(c, KC_NONE, 0, k_diag, grid_for(nf, 256), 256, 0, nf, Aff.row_ptr, Aff.col, Aff.val,
                   dk.as<double>(), 1, c.d_err);
    c.check_err("diag(A_ff)");
    Buf cnt(&c, sizeof(int32_t) * (size_t)(nm + 1));
    MDS_LAUNCH(c, KC_NONE, 0, k_schur<false>, grid_for(nm, 128), 128, 0, nm, Amm, Amf, Afm, dk.as<double>(),
               cnt.as<int32_t>(), nullptr, nullptr, nullptr, c.d_err);
    c.check_err("Schur complement (symbolic)");
    DCsr S;
    S.nrow = S.ncol = nm;
    S.rp = Buf(&c, sizeof(int32_t) * (size_t)(nm + 1));
    S.nnz = scan_counts(c, cnt.as<int32_t>(), S.rowp(), nm);
    S.ci = Buf(&c, sizeof(int32_t) * (size_t)(S.nnz > 0 ? S.nnz : 1));
    S.v = Buf(&c, sizeof(double) * (size_t)(S.nnz > 0 ? S.nnz : 1));
    MDS_LAUNCH(c, KC_NONE, 0, k_schur<true>, grid_for(nm, 128), 128, 0, nm, Amm, Amf, Afm, dk.as<double>(), nullptr,
               S.rowp(), S.cols(), S.vals(), c.d_err);
    c.check_err("Schur complement");
    return S;
}

// ---------------------------------------------------------------- strength

// j != i is strong for i when a_ij^2 >= (theta^2 a_ii) a_jj; i and j are
// linked in the graph G when either direction is strong.
__global__ void k_strength(int64_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                           const double *__restrict__ v, const double *__restrict__ dg, double th2,
                           int8_t *__restrict__ g, int32_t *__restrict__ deg) {
    mds_pdl_entry();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int cnt = 0;
    for (int32_t p = rp[i]; p < rp[i + 1]; p++) {
        int32_t j = ci[p];
        int8_t s = 0;
        if (j != i) {
            double a = v[p];
            s = (a * a) >= (th2 * dg[i]) * dg[j];
            if (!s) {
                int32_t q = find_col(ci, rp[j], rp[j + 1], (int32_t)i);
                if (q >= 0) {
                    double b = v[q];
                    s = (b * b) >= (th2 * dg[j]) * dg[i];
                }
            }
        }
        g[p] = s;
        cnt += s;
    }
    deg[i] = cnt;
}

// ---------------------------------------------------------------- MIS-2

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// Priority of vertex i on a level: high 32 bits of a SplitMix64 hash, low 32
// bits the index (unique).  Stored +1 so that 0 means "no undecided vertex".
__device__ __forceinline__ uint64_t mis_key1(uint64_t lkey, int64_t i) {
    uint64_t hv = mix64(lkey + 0x9E3779B97F4A7C15ULL * (uint64_t)(i + 1));
    return ((hv & 0xFFFFFFFF00000000ULL) | (uint64_t)(uint32_t)i) + 1ULL;
}

__global__ void k_mis_init(int64_t n, const int32_t *__restrict__ deg, int8_t *__restrict__ state) {
    mds_pdl_entry();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) state[i] = deg[i] == 0 ? 2 : 0;
}

// Index of row i within its instance (packed batches: lid; else i): the keys
// of an instance do not depend on the other instances packed with it.
__device__ __forceinline__ int64_t key_index(const int32_t *lid, int64_t i) { return lid ? (int64_t)lid[i] : i; }

// lid[i] = i - seg[k] for the instance k holding row i (seg ascending, K + 1)
__global__ void k_local_index(int64_t n, const int64_t *__restrict__ seg, int K, int32_t *__restrict__ lid) {
    mds_pdl_entry();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int lo = 0, hi = K - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (seg[mid] <= i)
            lo = mid;
        else
            hi = mid - 1;
    }
    lid[i] = (int32_t)(i - seg[lo]);
}

// The rounds below run on 256-row blocks; act[b] = 0 marks a block that
// holds no undecided vertex nor a strong neighbour of one, whose keys and
// flags no later step reads (it returns at once).

// m1_i = max key over undecided vertices of {i} and its strong neighbours
__global__ void k_mis_max1(int64_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                           const int8_t *__restrict__ g, const int8_t *__restrict__ state, uint64_t lkey,
                           const int32_t *__restrict__ lid, const int8_t *__restrict__ act,
                           uint64_t *__restrict__ m1) {
    mds_pdl_entry();
    if (!act[blockIdx.x]) return;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t m = state[i] == 0 ? mis_key1(lkey, key_index(lid, i)) : 0;
    for (int32_t p = rp[i]; p < rp[i + 1]; p++) {
        if (!g[p]) continue;
        int32_t j = ci[p];
        if (state[j] == 0) {
            uint64_t k = mis_key1(lkey, key_index(lid, j));
            m = k > m ? k : m;
        }
    }
    m1[i] = m;
}

// a vertex whose key is the largest among undecided vertices within distance
// two becomes a root
__global__ void k_mis_select(int64_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                             const int8_t *__restrict__ g, const uint64_t *__restrict__ m1, uint64_t lkey,
                             const int32_t *__restrict__ lid, const int8_t *__restrict__ act,
                             int8_t *__restrict__ state) {
    mds_pdl_entry();
    if (!act[blockIdx.x]) return;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || state[i] != 0) return;
    uint64_t m = m1[i];
    for (int32_t p = rp[i]; p < rp[i + 1]; p++)
        if (g[p]) {
            uint64_t k = m1[ci[p]];
            m = k > m ? k : m;
        }
    if (m == mis_key1(lkey, key_index(lid, i))) state[i] = 1;
}

__global__ void k_mis_near_root(int64_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                const int8_t *__restrict__ g, const int8_t *__restrict__ state,
                                const int8_t *__restrict__ act, int8_t *__restrict__ e1) {
    mds_pdl_entry();
    if (!act[blockIdx.x]) return;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int8_t e = state[i] == 1;
    for (int32_t p = rp[i]; p < rp[i + 1] && !e; p++)
        if (g[p] && state[ci[p]] == 1) e = 1;
    e1[i] = e;
}

__global__ void k_mis_exclude(int64_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                              const int8_t *__restrict__ g, const int8_t *__restrict__ e1, int8_t *__restrict__ state,
                              const int8_t *__restrict__ act, int8_t *__restrict__ act_next,
                              int32_t *__restrict__ undecided) {
    mds_pdl_entry();
    if (!act[blockIdx.x]) return;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || state[i] != 0) return;
    bool ex = e1[i];
    for (int32_t p = rp[i]; p < rp[i + 1] && !ex; p++)
        if (g[p] && e1[ci[p]]) ex = true;
    if (ex) {
        state[i] = 2;
    } else {
        atomicAdd(undecided, 1);
        // the next round reads the keys and flags of i and its strong neighbours
        act_next[i >> 8] = 1;
        for (int32_t p = rp[i]; p < rp[i + 1]; p++)
            if (g[p]) act_next[ci[p] >> 8] = 1;
    }
}

// ---------------------------------------------------------------- aggregation

__global__ void k_root_flags(int64_t n, const int8_t *__restrict__ state, int8_t *__restrict__ roots,
                             int32_t *__restrict__ flag) {
    mds_pdl_entry();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int8_t r = state[i] == 1;
    roots[i] = r;
    flag[i] = r;
}

__global__ void k_agg_first(int64_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                            const int8_t *__restrict__ g, const int8_t *__restrict__ roots,
                            const int32_t *__restrict__ rootid, int32_t *__restrict__ first) {
    mds_pdl_entry();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t f = -1;
    if (roots[i]) {
        f = rootid[i];
    } else {
        for (int32_t p = rp[i]; p < rp[i + 1]; p++)
            if (g[p] && roots[ci[p]]) f = rootid[ci[p]];
    }
    first[i] = f;
}

__global__ void k_agg_second(int64_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                             const double *__restrict__ v, const int8_t *__restrict__ g,
                             const int8_t *__restrict__ roots, const int32_t *__restrict__ deg,
                             const int32_t *__restrict__ first, int32_t *__restrict__ agg) {
    mds_pdl_entry();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (first[i] >= 0 || deg[i] == 0) {
        agg[i] = first[i];
        return;
    }
    double best = -1.0;
    int32_t ba = -1;
    for (int32_t p = rp[i]; p < rp[i + 1]; p++) {
        if (!g[p]) continue;
        int32_t j = ci[p];
        if (roots[j] || first[j] < 0) continue;
        double w = fabs(v[p]);
        if (w > best || (w == best && first[j] < ba)) {
            best = w;
            ba = first[j];
        }
    }
    agg[i] = ba;
}

// ---------------------------------------------------------------- Galerkin P^T A P

__global__ void k_agg_count(int64_t n, const int32_t *__restrict__ agg, int32_t *__restrict__ cnt) {
    mds_pdl_entry();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && agg[i] >= 0) atomicAdd(cnt + agg[i], 1);
}

__global__ void k_agg_scatter(int64_t n, const int32_t *__restrict__ agg, const int32_t *__restrict__ off,
                              int32_t *__restrict__ cursor, int32_t *__restrict__ mem) {
    mds_pdl_entry();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && agg[i] >= 0) {
        int32_t q = atomicAdd(cursor + agg[i], 1);
        mem[off[agg[i]] + q] = (int32_t)i;
    }
}

__global__ void k_agg_sort(int64_t nc, const int32_t *__restrict__ off, int32_t *__restrict__ mem) {
    mds_pdl_entry();
    int64_t I = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nc) return;
    int32_t a = off[I], e = off[I + 1];
    for (int32_t p = a + 1; p < e; p++) {
        int32_t x = mem[p];
        int32_t q = p - 1;
        while (q >= a && mem[q] > x) {
            mem[q + 1] = mem[q];
            q--;
        }
        mem[q + 1] = x;
    }
}

// Upper bound of the entries of coarse row I: those of its members' rows.
__global__ void k_rap_bound(int64_t nc, const int32_t *__restrict__ off, const int32_t *__restrict__ mem,
                            const int32_t *__restrict__ rp, int32_t *__restrict__ ub) {
    mds_pdl_entry();
    int64_t I = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nc) return;
    int32_t u = 0;
    for (int32_t q = off[I]; q < off[I + 1]; q++) u += rp[mem[q] + 1] - rp[mem[q]];
    ub[I] = u;
}

// Coarse row I = sum over members i of I (ascending) of row i of A mapped
// through agg, accumulated in CSR order; its entries, sorted by column, go to
// the scratch rows starting at uoff[I] (room for the bound above) and their
// count to cnt[I], in one pass (no separate symbolic pass).
__global__ void k_rap(int64_t nc, const int32_t *__restrict__ off, const int32_t *__restrict__ mem,
                      const int32_t *__restrict__ rp, const int32_t *__restrict__ ci, const double *__restrict__ v,
                      const int32_t *__restrict__ agg, const int32_t *__restrict__ uoff, int32_t *__restrict__ cnt,
                      int32_t *__restrict__ tci, double *__restrict__ tv, int *err) {
    mds_pdl_entry();
    int64_t I = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nc) return;
    int32_t cols[RAP_CAP];
    double acc[RAP_CAP];
    int m = 0;
    for (int32_t q = off[I]; q < off[I + 1]; q++) {
        int32_t i = mem[q];
        for (int32_t p = rp[i]; p < rp[i + 1]; p++) {
            int32_t J = agg[ci[p]];
            if (J < 0) continue;
            int t = 0;
            while (t < m && cols[t] != J) t++;
            if (t == m) {
                if (m >= RAP_CAP) {
                    atomicOr(err, DERR_CAPACITY);
                    cnt[I] = 0;
                    return;
                }
                cols[m] = J;
                acc[m++] = 0.0;
            }
            acc[t] = acc[t] + v[p];
        }
    }
    for (int a = 1; a < m; a++) {
        int32_t x = cols[a];
        double y = acc[a];
        int q = a - 1;
        while (q >= 0 && cols[q] > x) {
            cols[q + 1] = cols[q];
            acc[q + 1] = acc[q];
            q--;
        }
        cols[q + 1] = x;
        acc[q + 1] = y;
    }
    const int32_t o = uoff[I];
    for (int a = 0; a < m; a++) {
        tci[o + a] = cols[a];
        tv[o + a] = acc[a];
    }
    cnt[I] = m;
}

// The scratch rows moved to the coarse CSR arrays, one warp per row.
__global__ void k_rap_compact(int64_t nc, const int32_t *__restrict__ uoff, const int32_t *__restrict__ crp,
                              const int32_t *__restrict__ tci, const double *__restrict__ tv,
                              int32_t *__restrict__ cci, double *__restrict__ cv) {
    mds_pdl_entry();
    const int64_t I = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    const int lane = threadIdx.x % 32;
    if (I >= nc) return;
    const int32_t s = uoff[I], d = crp[I], m = crp[I + 1] - crp[I];
    for (int32_t a = lane; a < m; a += 32) {
        cci[d + a] = tci[s + a];
        cv[d + a] = tv[s + a];
    }
}

// ---------------------------------------------------------------- smoothed aggregation

constexpr int SA_P_CAP = 64;
constexpr int SPGEMM_CAP = 512;

// Filtered diagonal aF_ii = a_ii + sum of weak off-diagonals (a_ii itself
// where that sum is not positive), and the L1 diagonal of the filtered
// matrix d1f_i = aF_ii + sum of strong |a_ij| (both summed in CSR order).
__global__ void k_sa_diag(int64_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                          const double *__restrict__ v, const int8_t *__restrict__ g, double *__restrict__ afd,
                          double *__restrict__ d1f) {
    mds_pdl_entry();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t pd = find_col(ci, rp[i], rp[i + 1], (int32_t)i);
    const double aii = pd >= 0 ? v[pd] : 0.0;
    double a = aii;
    for (int32_t p = rp[i]; p < rp[i + 1]; p++)
        if (ci[p] != i && !g[p]) a = a + v[p];
    // lumping the weak entries must leave a positive diagonal (coarse
    // operators have positive off-diagonals): otherwise the row keeps a_ii
    if (!(a > 0.0)) a = aii;
    double d = a;
    for (int32_t p = rp[i]; p < rp[i + 1]; p++)
        if (ci[p] != i && g[p]) d = d + fabs(v[p]);
    afd[i] = a;
    d1f[i] = d;
}

// Smoothed prolongator P = P0 - (4/3) D1F^-1 AF P0, row i: (agg(i), 1) when
// aggregated, then for each entry kept in AF, in CSR order, with
// J = agg(col) >= 0: P_iJ = P_iJ - c_i aF_ij, c_i = (4/3) / d1f_i.
template <bool FILL>
__global__ void k_sa_prolongator(int64_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                 const double *__restrict__ v, const int8_t *__restrict__ g,
                                 const double *__restrict__ afd, const double *__restrict__ d1f,
                                 const int32_t *__restrict__ agg, int32_t *__restrict__ cnt,
                                 const int32_t *__restrict__ prp, int32_t *__restrict__ pci, double *__restrict__ pv,
                                 int *err) {
    mds_pdl_entry();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t cols[SA_P_CAP];
    double acc[SA_P_CAP];
    int m = 0;
    if (agg[i] >= 0) {
        cols[0] = agg[i];
        acc[0] = 1.0;
        m = 1;
    }
    double c = (4.0 / 3.0) / d1f[i];
    for (int32_t p = rp[i]; p < rp[i + 1]; p++) {
        int32_t j = ci[p];
        double a;
        if (j == i)
            a = afd[i];
        else if (g[p])
            a = v[p];
        else
            continue;
        int32_t J = agg[j];
        if (J < 0) continue;
        int t = 0;
        while (t < m && cols[t] != J) t++;
        if (t == m) {
            if (m >= SA_P_CAP) {
                atomicOr(err, DERR_CAPACITY);
                return;
            }
            cols[m] = J;
            acc[m++] = 0.0;
        }
        acc[t] = acc[t] - c * a;
    }
    if constexpr (!FILL) {
        cnt[i] = m;
    } else {
        for (int a2 = 1; a2 < m; a2++) {
            int32_t x = cols[a2];
            double y = acc[a2];
            int q = a2 - 1;
            while (q >= 0 && cols[q] > x) {
                cols[q + 1] = cols[q];
                acc[q + 1] = acc[q];
                q--;
            }
            cols[q + 1] = x;
            acc[q + 1] = y;
        }
        int32_t o = prp[i];
        for (int a2 = 0; a2 < m; a2++) {
            pci[o + a2] = cols[a2];
            pv[o + a2] = acc[a2];
        }
    }
}

// Transpose: counts per column, scatter with an atomic cursor, then each row
// sorted by column so that the result is deterministic.
__global__ void k_tr_count(int64_t nnz, const int32_t *__restrict__ ci, int32_t *__restrict__ cnt) {
    mds_pdl_entry();
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < nnz) atomicAdd(cnt + ci[p], 1);
}

__global__ void k_tr_fill(int64_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                          const double *__restrict__ v, const int32_t *__restrict__ trp, int32_t *__restrict__ cur,
                          int32_t *__restrict__ tci, double *__restrict__ tv) {
    mds_pdl_entry();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int32_t p = rp[i]; p < rp[i + 1]; p++) {
        int32_t J = ci[p];
        int32_t q = trp[J] + atomicAdd(cur + J, 1);
        tci[q] = (int32_t)i;
        tv[q] = v[p];
    }
}

__global__ void k_sort_rows(int64_t n, const int32_t *__restrict__ rp, int32_t *__restrict__ ci,
                            double *__restrict__ v) {
    mds_pdl_entry();
    int64_t I = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= n) return;
    int32_t a = rp[I], e = rp[I + 1];
    for (int32_t p = a + 1; p < e; p++) {
        int32_t x = ci[p];
        double y = v[p];
        int32_t q = p - 1;
        while (q >= a && ci[q] > x) {
            ci[q + 1] = ci[q];
            v[q + 1] = v[q];
            q--;
        }
        ci[q + 1] = x;
        v[q + 1] = y;
    }
}

// C = X Y, one thread per row: entry (i, k) accumulates x_ij y_jk over row i
// of X in order and row j of Y in order.
template <bool FILL>
__global__ void k_spgemm(int64_t n, mds_csr X, mds_csr Y, int32_t *__restrict__ cnt, const int32_t *__restrict__ crp,
                         int32_t *__restrict__ cci, double *__restrict__ cv, int *err) {
    mds_pdl_entry();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t cols[SPGEMM_CAP];
    double acc[SPGEMM_CAP];
    int m = 0;
    for (int32_t p = X.row_ptr[i]; p < X.row_ptr[i + 1]; p++) {
        int32_t j = X.col[p];
        double x = X.val[p];
        for (int32_t q = Y.row_ptr[j]; q < Y.row_ptr[j + 1]; q++) {
            int32_t k = Y.col[q];
            int t = 0;
            while (t < m && cols[t] != k) t++;
            if (t == m) {
                if (m >= SPGEMM_CAP) {
                    atomicOr(err, DERR_CAPACITY);
                    return;
                }
                cols[m] = k;
                acc[m++] = 0.0;
            }
            acc[t] = acc[t] + x * Y.val[q];
        }
    }
    if constexpr (!FILL) {
        cnt[i] = m;
    } else {
        for (int a2 = 1; a2 < m; a2++) {
            int32_t xk = cols[a2];
            double y = acc[a2];
            int q = a2 - 1;
            while (q >= 0 && cols[q] > xk) {
                cols[q + 1] = cols[q];
                acc[q + 1] = acc[q];
                q--;
            }
            cols[q + 1] = xk;
            acc[q + 1] = y;
        }
        int32_t o = crp[i];
        for (int a2 = 0; a2 < m; a2++) {
            cci[o + a2] = cols[a2];
            cv[o + a2] = acc[a2];
        }
    }
}

static DCsr spgemm_gpu(Ctx &c, const mds_csr &X, const mds_csr &Y) {
    int64_t n = X.nrow;
    Buf cnt(&c, sizeof(int32_t) * (size_t)(n + 1));
    c.clear_err();
    MDS_LAUNCH(c, KC_NONE, 0, k_spgemm<false>, grid_for(n, 64), 64, 0, n, X, Y, cnt.as<int32_t>(), nullptr, nullptr,
               nullptr, c.d_err);
    c.check_err("sparse product (symbolic)");
    DCsr C;
    C.nrow = n;
    C.ncol = Y.ncol;
    C.rp = Buf(&c, sizeof(int32_t) * (size_t)(n + 1));
    C.nnz = scan_counts(c, cnt.as<int32_t>(), C.rowp(), n);
    C.ci = Buf(&c, sizeof(int32_t) * (size_t)(C.nnz > 0 ? C.nnz : 1));
    C.v = Buf(&c, sizeof(double) * (size_t)(C.nnz > 0 ? C.nnz : 1));
    MDS_LAUNCH(c, KC_NONE, 0, k_spgemm<true>, grid_for(n, 64), 64, 0, n, X, Y, nullptr, C.rowp(), C.cols(), C.vals(),
               c.d_err);
    c.check_err("sparse product");
    return C;
}

static DCsr transpose_gpu(Ctx &c, const DCsr &P) {
    DCsr R;
    R.nrow = P.ncol;
    R.ncol = P.nrow;
    R.nnz = P.nnz;
    Buf cnt(&c, sizeof(int32_t) * (size_t)(R.nrow + 1));
    MDS_CUDA(cudaMemsetAsync(cnt.p, 0, cnt.bytes, c.stream));
    if (P.nnz) MDS_LAUNCH(c, KC_NONE, 0, k_tr_count, grid_for(P.nnz, 256), 256, 0, P.nnz, P.cols(), cnt.as<int32_t>());
    R.rp = Buf(&c, sizeof(int32_t) * (size_t)(R.nrow + 1));
    scan_counts(c, cnt.as<int32_t>(), R.rowp(), R.nrow);
    R.ci = Buf(&c, sizeof(int32_t) * (size_t)(R.nnz > 0 ? R.nnz : 1));
    R.v = Buf(&c, sizeof(double) * (size_t)(R.nnz > 0 ? R.nnz : 1));
    MDS_CUDA(cudaMemsetAsync(cnt.p, 0, cnt.bytes, c.stream));
    MDS_LAUNCH(c, KC_NONE, 0, k_tr_fill, grid_for(P.nrow, 256), 256, 0, P.nrow, P.rowp(), P.cols(), P.vals(),
               R.rowp(), cnt.as<int32_t>(), R.cols(), R.vals());
    MDS_LAUNCH(c, KC_NONE, 0, k_sort_rows, grid_for(R.nrow, 128), 128, 0, R.nrow, R.rowp(), R.cols(), R.vals());
    return R;
}

// ---------------------------------------------------------------- per-level data

// L1 diagonal a_ii + sum_{j != i} |a_ij| and its reciprocal
template <class DT>
__global__ void k_l1(int64_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                     const double *__restrict__ v, double *__restrict__ l1, DT *__restrict__ dinv) {
    mds_pdl_entry();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t p = find_col(ci, rp[i], rp[i + 1], (int32_t)i);
    double s = p >= 0 ? v[p] : 0.0;
    for (int32_t q = rp[i]; q < rp[i + 1]; q++)
        if (ci[q] != i) s = s + fabs(v[q]);
    l1[i] = s;
    dinv[i] = (DT)(1.0 / s);
}

// bit 1: row i holds more than its diagonal entry; bit 2: a_ii is missing
// or not negative
__global__ void k_row_kinds(int64_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                            const double *__restrict__ v, int *flag) {
    mds_pdl_entry();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t b = rp[i], e = rp[i + 1];
    int f = (e - b != 1 || ci[b] != (int32_t)i) ? 1 : 0;
    int32_t p = find_col(ci, b, e, (int32_t)i);
    if (!(p >= 0 && v[p] < 0.0)) f |= 2;
    if (f) atomicOr(flag, f);
}

int row_kinds(Ctx &c, const mds_csr &A) {
    if (A.nrow <= 0) return 0;
    Buf f(&c, sizeof(int));
    MDS_CUDA(cudaMemsetAsync(f.p, 0, sizeof(int), c.stream));
    MDS_LAUNCH(c, KC_NONE, 0, k_row_kinds, grid_for(A.nrow, 256), 256, 0, A.nrow, A.row_ptr, A.col, A.val,
               f.as<int>());
    return c.read(f.as<int32_t>());
}

static DCsr copy_csr(Ctx &c, const mds_csr &A) {
    DCsr B = csr_alloc(c, A.nrow, A.ncol, A.nnz);
    MDS_CUDA(cudaMemcpyAsync(B.rowp(), A.row_ptr, sizeof(int32_t) * (size_t)(A.nrow + 1), cudaMemcpyDeviceToDevice,
                             c.stream));
    if (A.nnz > 0) {
        MDS_CUDA(cudaMemcpyAsync(B.cols(), A.col, sizeof(int32_t) * (size_t)A.nnz, cudaMemcpyDeviceToDevice, c.stream));
        MDS_CUDA(cudaMemcpyAsync(B.vals(), A.val, sizeof(double) * (size_t)A.nnz, cudaMemcpyDeviceToDevice, c.stream));
    }
    return B;
}

// out[k] = rootid[seg[k]] for k <= K: the first aggregate of each instance
__global__ void k_seg_next(int K, const int64_t *__restrict__ seg, const int32_t *__restrict__ rootid,
                           int64_t *__restrict__ out) {
    mds_pdl_entry();
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k <= K) out[k] = rootid[seg[k]];
}

static uint64_t host_mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// MIS-2 on the strength graph of level l: fills roots, returns their count.
static int64_t mis2(Ctx &c, const DCsr &A, const int8_t *g, const int32_t *deg, uint64_t seed, int level,
                    const int32_t *lid, Buf &state) {
    int64_t n = A.nrow;
    unsigned gr = grid_for(n, 256);
    state = Buf(&c, (size_t)(n > 0 ? n : 1));
    Buf m1(&c, sizeof(uint64_t) * (size_t)(n > 0 ? n : 1));
    Buf e1(&c, (size_t)(n > 0 ? n : 1));
    Buf und(&c, sizeof(int32_t));
    // active-block flags of this round and the next (every block in the first)
    Buf act[2] = {Buf(&c, (size_t)gr + 1), Buf(&c, (size_t)gr + 1)};
    MDS_CUDA(cudaMemsetAsync(act[0].p, 1, (size_t)gr + 1, c.stream));
    uint64_t lkey = host_mix64(seed + 0x9E3779B97F4A7C15ULL * (uint64_t)(level + 1));
    MDS_LAUNCH(c, KC_NONE, 0, k_mis_init, gr, 256, 0, n, deg, state.as<int8_t>());
    for (int round = 0;; round++) {
        MDS_REQUIRE(round < 10000, MDS_ERR_TIMEOUT, "MIS-2 did not terminate");
        const int8_t *a = act[round & 1].as<int8_t>();
        int8_t *an = act[(round + 1) & 1].as<int8_t>();
        MDS_CUDA(cudaMemsetAsync(und.p, 0, sizeof(int32_t), c.stream));
        MDS_CUDA(cudaMemsetAsync(an, 0, (size_t)gr + 1, c.stream));
        MDS_LAUNCH(c, KC_NONE, 0, k_mis_max1, gr, 256, 0, n, A.rowp(), A.cols(), g, state.as<int8_t>(), lkey, lid,
                   a, m1.as<uint64_t>());
        MDS_LAUNCH(c, KC_NONE, 0, k_mis_select, gr, 256, 0, n, A.rowp(), A.cols(), g, m1.as<uint64_t>(), lkey, lid,
                   a, state.as<int8_t>());
        MDS_LAUNCH(c, KC_NONE, 0, k_mis_near_root, gr, 256, 0, n, A.rowp(), A.cols(), g, state.as<int8_t>(), a,
                   e1.as<int8_t>());
        MDS_LAUNCH(c, KC_NONE, 0, k_mis_exclude, gr, 256, 0, n, A.rowp(), A.cols(), g, e1.as<int8_t>(),
                   state.as<int8_t>(), a, an, und.as<int32_t>());
        if (c.read(und.as<int32_t>()) == 0) break;
    }
    return 0;
}

void amg_setup(Ctx &c, const mds_csr &A0, const mds_setup_opts &o, Hierarchy &h, const std::vector<int64_t> *seg0) {
    h.lv.clear();
    h.dense = false;
    h.diagonal = false;
    h.seg.clear();
    if (seg0 && seg0->size() >= 2) {
        MDS_REQUIRE(seg0->front() == 0 && seg0->back() == A0.nrow, MDS_ERR_INVALID, "instance segments do not cover the matrix");
        h.seg.push_back(*seg0);
    } else {
        h.seg.push_back(std::vector<int64_t>{0, A0.nrow});
    }
    h.K = (int)h.seg[0].size() - 1;
    h.prec = o.precision == MDS_PREC_FP64 ? 64 : 32;
    h.smoother = o.smoother;
    h.sweeps = o.sweeps < 1 ? 1 : o.sweeps;
    h.cheb_degree = o.cheb_degree < 1 ? 2 : o.cheb_degree;
    h.form = o.level_form;
    h.use_tail = o.coarse_tail != 0 && h.K == 1;
    int maxl = o.max_levels < 1 ? 1 : (o.max_levels > 32 ? 32 : o.max_levels);
    h.lv.emplace_back();
    h.lv[0].A = copy_csr(c, A0);
    double th2 = o.theta * o.theta;
    for (int l = 0;; l++) {
        Level &L = h.lv[l];
        int64_t n = L.A.nrow;
        L.roots = Buf(&c, (size_t)(n > 0 ? n : 1));
        MDS_CUDA(cudaMemsetAsync(L.roots.p, 0, (size_t)(n > 0 ? n : 1), c.stream));
        // a level without couplings (each row only its diagonal, of either
        // sign) is the last one and is solved exactly by x = b / a_ii
        if (L.A.nnz == n && !(row_kinds(c, L.A.view()) & 1)) {
            h.diagonal = true;
            break;
        }
        // the coarsening stops once every instance has at most n_coarse rows
        const std::vector<int64_t> &sg = h.seg[l];
        int64_t smax = 0;
        for (int k = 0; k < h.K; k++) smax = std::max(smax, sg[k + 1] - sg[k]);
        if (smax <= o.n_coarse) {
            h.dense = true;
            break;
        }
        if (l == maxl - 1) break;
        unsigned gr = grid_for(n, 256);
        Buf lid;
        if (h.K > 1) {
            L.K = h.K;
            L.seg_h = sg;
            L.seg_d = Buf(&c, sizeof(int64_t) * (size_t)(h.K + 1));
            MDS_CUDA(cudaMemcpyAsync(L.seg_d.p, sg.data(), sizeof(int64_t) * (size_t)(h.K + 1),
                                     cudaMemcpyHostToDevice, c.stream));
            lid = Buf(&c, sizeof(int32_t) * (size_t)n);
            MDS_LAUNCH(c, KC_NONE, 0, k_local_index, gr, 256, 0, n, L.seg_d.as<int64_t>(), h.K, lid.as<int32_t>());
        }
        Buf dg(&c, sizeof(double) * (size_t)n), gf(&c, (size_t)(L.A.nnz > 0 ? L.A.nnz : 1));
        Buf deg(&c, sizeof(int32_t) * (size_t)(n + 1));
        MDS_LAUNCH(c, KC_NONE, 0, k_diag, gr, 256, 0, n, L.A.rowp(), L.A.cols(), L.A.vals(), dg.as<double>(), 0,
                   c.d_err);
        MDS_LAUNCH(c, KC_NONE, 0, k_strength, gr, 256, 0, n, L.A.rowp(), L.A.cols(), L.A.vals(), dg.as<double>(), th2,
                   gf.as<int8_t>(), deg.as<int32_t>());
        Buf state;
        mis2(c, L.A, gf.as<int8_t>(), deg.as<int32_t>(), o.seed, l, h.K > 1 ? lid.as<int32_t>() : nullptr, state);
        Buf flag(&c, sizeof(int32_t) * (size_t)(n + 1)), rootid(&c, sizeof(int32_t) * (size_t)(n + 1));
        MDS_LAUNCH(c, KC_NONE, 0, k_root_flags, gr, 256, 0, n, state.as<int8_t>(), L.roots.as<int8_t>(),
                   flag.as<int32_t>());
        int64_t nc = scan_counts(c, flag.as<int32_t>(), rootid.as<int32_t>(), n);
        Buf first(&c, sizeof(int32_t) * (size_t)n);
        L.agg = Buf(&c, sizeof(int32_t) * (size_t)n);
        MDS_LAUNCH(c, KC_NONE, 0, k_agg_first, gr, 256, 0, n, L.A.rowp(), L.A.cols(), gf.as<int8_t>(),
                   L.roots.as<int8_t>(), rootid.as<int32_t>(), first.as<int32_t>());
        MDS_LAUNCH(c, KC_NONE, 0, k_agg_second, gr, 256, 0, n, L.A.rowp(), L.A.cols(), L.A.vals(), gf.as<int8_t>(),
                   L.roots.as<int8_t>(), deg.as<int32_t>(), first.as<int32_t>(), L.agg.as<int32_t>());
        if (nc == 0 || (double)nc > o.stall_ratio * (double)n) {
            L.agg.reset();
            break;
        }
        // the next level's instance segments: aggregates are numbered by
        // ascending root, so instance k's first aggregate is the number of
        // roots before its first row
        {
            std::vector<int64_t> nx(h.K + 1, 0);
            if (h.K > 1) {
                Buf o_d(&c, sizeof(int64_t) * (size_t)(h.K + 1));
                MDS_LAUNCH(c, KC_NONE, 0, k_seg_next, grid_for(h.K + 1, 128), 128, 0, h.K, L.seg_d.as<int64_t>(),
                           rootid.as<int32_t>(), o_d.as<int64_t>());
                MDS_CUDA(cudaMemcpyAsync(nx.data(), o_d.p, sizeof(int64_t) * (size_t)(h.K + 1), cudaMemcpyDeviceToHost,
                                         c.stream));
                c.sync();
            } else {
                nx[1] = nc;
            }
            h.seg.push_back(nx);
        }
        // members of each aggregate, ascending
        Buf acnt(&c, sizeof(int32_t) * (size_t)(nc + 1));
        MDS_CUDA(cudaMemsetAsync(acnt.p, 0, sizeof(int32_t) * (size_t)(nc + 1), c.stream));
        MDS_LAUNCH(c, KC_NONE, 0, k_agg_count, gr, 256, 0, n, L.agg.as<int32_t>(), acnt.as<int32_t>());
        L.mem_off = Buf(&c, sizeof(int32_t) * (size_t)(nc + 1));
        int64_t nmem = scan_counts(c, acnt.as<int32_t>(), L.mem_off.as<int32_t>(), nc);
        L.mem = Buf(&c, sizeof(int32_t) * (size_t)(nmem > 0 ? nmem : 1));
        L.mem_count = nmem;
        MDS_CUDA(cudaMemsetAsync(acnt.p, 0, sizeof(int32_t) * (size_t)(nc + 1), c.stream));
        MDS_LAUNCH(c, KC_NONE, 0, k_agg_scatter, gr, 256, 0, n, L.agg.as<int32_t>(), L.mem_off.as<int32_t>(),
                   acnt.as<int32_t>(), L.mem.as<int32_t>());
        MDS_LAUNCH(c, KC_NONE, 0, k_agg_sort, grid_for(nc, 128), 128, 0, nc, L.mem_off.as<int32_t>(),
                   L.mem.as<int32_t>());
        if (o.prolongation == MDS_PROLONG_SMOOTHED) {
            Buf afd(&c, sizeof(double) * (size_t)n), d1f(&c, sizeof(double) * (size_t)n);
            MDS_LAUNCH(c, KC_NONE, 0, k_sa_diag, gr, 256, 0, n, L.A.rowp(), L.A.cols(), L.A.vals(), gf.as<int8_t>(),
                       afd.as<double>(), d1f.as<double>());
            Buf pcnt(&c, sizeof(int32_t) * (size_t)(n + 1));
            c.clear_err();
            MDS_LAUNCH(c, KC_NONE, 0, k_sa_prolongator<false>, grid_for(n, 128), 128, 0, n, L.A.rowp(), L.A.cols(),
                       L.A.vals(), gf.as<int8_t>(), afd.as<double>(), d1f.as<double>(), L.agg.as<int32_t>(),
                       pcnt.as<int32_t>(), nullptr, nullptr, nullptr, c.d_err);
            c.check_err("smoothed prolongator (symbolic)");
            L.P.nrow = n;
            L.P.ncol = nc;
            L.P.rp = Buf(&c, sizeof(int32_t) * (size_t)(n + 1));
            L.P.nnz = scan_counts(c, pcnt.as<int32_t>(), L.P.rowp(), n);
            L.P.ci = Buf(&c, sizeof(int32_t) * (size_t)(L.P.nnz > 0 ? L.P.nnz : 1));
            L.P.v = Buf(&c, sizeof(double) * (size_t)(L.P.nnz > 0 ? L.P.nnz : 1));
            MDS_LAUNCH(c, KC_NONE, 0, k_sa_prolongator<true>, grid_for(n, 128), 128, 0, n, L.A.rowp(), L.A.cols(),
                       L.A.vals(), gf.as<int8_t>(), afd.as<double>(), d1f.as<double>(), L.agg.as<int32_t>(), nullptr,
                       L.P.rowp(), L.P.cols(), L.P.vals(), c.d_err);
            c.check_err("smoothed prolongator");
            L.R = transpose_gpu(c, L.P);
            DCsr B = spgemm_gpu(c, L.A.view(), L.P.view());
            DCsr Ac = spgemm_gpu(c, L.R.view(), B.view());
            L.smoothed = true;
            L.has_coarse = true;
            L.nc = nc;
            h.lv.emplace_back();
            h.lv.back().A = std::move(Ac);
            continue;
        }
        // Galerkin product
        c.clear_err();
        Buf ub(&c, sizeof(int32_t) * (size_t)(nc + 1)), uoff(&c, sizeof(int32_t) * (size_t)(nc + 1));
        MDS_LAUNCH(c, KC_NONE, 0, k_rap_bound, grid_for(nc, 256), 256, 0, nc, L.mem_off.as<int32_t>(),
                   L.mem.as<int32_t>(), L.A.rowp(), ub.as<int32_t>());
        const int64_t utot = scan_counts(c, ub.as<int32_t>(), uoff.as<int32_t>(), nc);
        Buf tci(&c, sizeof(int32_t) * (size_t)(utot > 0 ? utot : 1)), tv(&c, sizeof(double) * (size_t)(utot > 0 ? utot : 1));
        Buf ccnt(&c, sizeof(int32_t) * (size_t)(nc + 1));
        MDS_LAUNCH(c, KC_NONE, 0, k_rap, grid_for(nc, 64), 64, 0, nc, L.mem_off.as<int32_t>(), L.mem.as<int32_t>(),
                   L.A.rowp(), L.A.cols(), L.A.vals(), L.agg.as<int32_t>(), uoff.as<int32_t>(), ccnt.as<int32_t>(),
                   tci.as<int32_t>(), tv.as<double>(), c.d_err);
        c.check_err("Galerkin product");
        DCsr Ac;
        Ac.nrow = Ac.ncol = nc;
        Ac.rp = Buf(&c, sizeof(int32_t) * (size_t)(nc + 1));
        Ac.nnz = scan_counts(c, ccnt.as<int32_t>(), Ac.rowp(), nc);
        Ac.ci = Buf(&c, sizeof(int32_t) * (size_t)(Ac.nnz > 0 ? Ac.nnz : 1));
        Ac.v = Buf(&c, sizeof(double) * (size_t)(Ac.nnz > 0 ? Ac.nnz : 1));
        MDS_LAUNCH(c, KC_NONE, 0, k_rap_compact, grid_for(nc * 32, 256), 256, 0, nc, uoff.as<int32_t>(), Ac.rowp(),
                   tci.as<int32_t>(), tv.as<double>(), Ac.cols(), Ac.vals());
        L.has_coarse = true;
        L.nc = nc;
        h.lv.emplace_back();
        h.lv.back().A = std::move(Ac);
    }
    // per-level smoother data and work vectors
    size_t vb = h.prec == 64 ? sizeof(double) : sizeof(float);
    for (auto &L : h.lv) {
        int64_t n = L.A.nrow;
        unsigned gr = grid_for(n, 256);
        size_t nb = vb * (size_t)(n > 0 ? n : 1);
        L.l1 = Buf(&c, sizeof(double) * (size_t)(n > 0 ? n : 1));
        L.dinv = Buf(&c, nb);
        if (h.prec == 64)
            MDS_LAUNCH(c, KC_NONE, 0, k_l1<double>, gr, 256, 0, n, L.A.rowp(), L.A.cols(), L.A.vals(),
                       L.l1.as<double>(), L.dinv.as<double>());
        else
            MDS_LAUNCH(c, KC_NONE, 0, k_l1<float>, gr, 256, 0, n, L.A.rowp(), L.A.cols(), L.A.vals(),
                       L.l1.as<double>(), L.dinv.as<float>());
    }
    h.nr_cap = 0;
    // work vectors for the columns the solves will use (the autotuner times
    // the level kernels with them)
    hierarchy_reserve(c, h, h.tune_nr >= 8 ? 8 : h.tune_nr >= 4 ? 4 : h.tune_nr >= 2 ? 2 : 1);
    if (h.dense) {
        Level &L = h.lv.back();
        h.nd = L.A.nrow;
        dense_spd_inverse(c, L.A.view(), h.seg[h.lv.size() - 1], h.Ainv, h.db);
    }
    // per-level instance offsets on the device (every level of a packed batch)
    if (h.K > 1)
        for (size_t l = 0; l < h.lv.size(); l++) {
            Level &L = h.lv[l];
            L.K = h.K;
            L.seg_h = h.seg[l];
            L.ck = live_chunks(c, L.A.nrow, h.seg[l]);
            if (L.seg_d.p) continue;
            L.seg_d = Buf(&c, sizeof(int64_t) * (size_t)(h.K + 1));
            MDS_CUDA(cudaMemcpyAsync(L.seg_d.p, h.seg[l].data(), sizeof(int64_t) * (size_t)(h.K + 1),
                                     cudaMemcpyHostToDevice, c.stream));
        }
    level_storage(c, h, o);
    c.sync();
}

}  // namespace mds
