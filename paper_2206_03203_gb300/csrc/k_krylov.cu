// Krylov solvers in FP64: right-preconditioned flexible GMRES(m) with
// classical Gram-Schmidt applied twice (CGS2) and device-side Givens
// rotations, and preconditioned conjugate gradients.  Sec. 3.2 studies the
// right-preconditioned operator A B_L; Sec. 4 fixes x0 = 0 and a relative-
// residual stopping rule.  All reductions are two-stage with a fixed order,
// so results are run-to-run reproducible.
#include <algorithm>
#include <cmath>
#include <functional>
#include <memory>
#include <mutex>

#include "conv.cuh"
#include "internal.cuh"
#include "krylov.cuh"

namespace mds {

constexpr int QMAX = 32;
constexpr int RED_BLOCK = 256;

static unsigned red_grid(int64_t n) {
    int64_t g = (n + RED_BLOCK * 4 - 1) / (RED_BLOCK * 4);
    if (g < 1) g = 1;
    if (g > 1216) g = 1216;  // 8 blocks per SM on 152 SMs
    return (unsigned)g;
}

// True in exactly one block of the grid: the last to arrive after every
// block has written its partial sums (each thread fences its writes first).
// That block then reduces the partials in a fixed order, so the result does
// not depend on which block it is.  The counter is reset for the next launch.
__device__ __forceinline__ bool last_block(unsigned *counter) {
    __shared__ bool is_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned total = gridDim.x * gridDim.y;
        unsigned t = atomicAdd(counter, 1u);
        is_last = t == total - 1;
        if (is_last) *counter = 0u;
    }
    __syncthreads();
    return is_last;
}

// Sum of v over the block (fixed order: lane tree, then warps ascending);
// valid in thread 0.
__device__ __forceinline__ double block_sum(double v) {
    __shared__ double ws[RED_BLOCK / 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();  // ws may still be read by an earlier call
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < RED_BLOCK / 32; k++) t += ws[k];
    return t;
}

// Gram-Schmidt dot products in one launch: out[q] = V[q] . w for q < nq and,
// when nout = nq + 1, out[nq] = w . w.  Grid (row blocks, nout): block (b, q)
// writes the partial sum of its rows to partial[q][b]; the last block sums
// each q's partials.  Rows of V are 16-byte aligned (ldv even); w is a row
// of V.  w is re-read once per q from L2, V once from HBM.
__global__ void __launch_bounds__(RED_BLOCK) k_gs_dot(int64_t n, const double *__restrict__ V, int64_t ldv, int nq,
                                                       const double *__restrict__ w, double *__restrict__ partial,
                                                       unsigned *__restrict__ counter, double *__restrict__ out) {
    mds_pdl_entry();
    const int q = blockIdx.y;
    const double *v = q < nq ? V + (int64_t)q * ldv : w;
    const double2 *v2 = reinterpret_cast<const double2 *>(v);
    const double2 *w2 = reinterpret_cast<const double2 *>(w);
    int64_t n2 = n >> 1;
    double s0 = 0.0, s1 = 0.0;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + stride < n2; i += 2 * stride) {
        double2 a = v2[i], b = w2[i], c = v2[i + stride], d = w2[i + stride];
        s0 += a.x * b.x;
        s1 += a.y * b.y;
        s0 += c.x * d.x;
        s1 += c.y * d.y;
    }
    for (; i < n2; i += stride) {
        double2 a = v2[i], b = w2[i];
        s0 += a.x * b.x;
        s1 += a.y * b.y;
    }
    if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) s0 += v[n - 1] * w[n - 1];
    double t = block_sum(s0 + s1);
    if (threadIdx.x == 0) partial[(int64_t)q * gridDim.x + blockIdx.x] = t;
    if (!last_block(counter)) return;
    const int nblk = gridDim.x, lane = threadIdx.x & 31;
    for (int qq = threadIdx.x >> 5; qq < (int)gridDim.y; qq += RED_BLOCK / 32) {
        double u = 0.0;
        for (int b = lane; b < nblk; b += 32) u += __ldcg(partial + (int64_t)qq * nblk + b);
        for (int o = 16; o > 0; o >>= 1) u += __shfl_down_sync(0xffffffffu, u, o);
        if (lane == 0) out[qq] = u;
    }
}

// out[q] (+)= sum over blocks of partial[blk][q] (stride QMAX); one warp per q,
// fixed order
__global__ void k_reduce_cols(const double *__restrict__ partial, int nblk, int nq, double *__restrict__ out,
                              int accumulate) {
    mds_pdl_entry();
    int q = blockIdx.x;
    if (q >= nq) return;
    double s = 0.0;
    for (int b = threadIdx.x; b < nblk; b += 32) s += partial[(int64_t)b * QMAX + q];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) out[q] = accumulate ? out[q] + s : s;
}

// w_i += sign * sum_q coef_q V[q][i]; optional block partials of w_i^2.
// VEC: w and the rows of V are 16-byte aligned, two elements per thread.
template <int SIGN, bool VEC>
__global__ void __launch_bounds__(RED_BLOCK) k_maxpy(int64_t n, const double *__restrict__ V, int64_t ldv, int nq,
                                                      const double *__restrict__ coef, double *__restrict__ w,
                                                      double *__restrict__ partial, const double *__restrict__ run_flag) {
    mds_pdl_entry();
    if (run_flag && *run_flag == 0.0) return;
    __shared__ double cs[QMAX];
    __shared__ double ws[RED_BLOCK / 32];
    if (threadIdx.x < QMAX) cs[threadIdx.x] = threadIdx.x < nq ? coef[threadIdx.x] : 0.0;
    __syncthreads();
    double nrm = 0.0;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if (VEC) {
        int64_t n2 = n >> 1;
        double2 *w2 = reinterpret_cast<double2 *>(w);
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += stride) {
            double s0 = 0.0, s1 = 0.0;
            for (int q = 0; q < nq; q++) {
                double2 a = reinterpret_cast<const double2 *>(V + (int64_t)q * ldv)[i];
                s0 += cs[q] * a.x;
                s1 += cs[q] * a.y;
            }
            double2 x = w2[i];
            x.x = SIGN > 0 ? x.x + s0 : x.x - s0;
            x.y = SIGN > 0 ? x.y + s1 : x.y - s1;
            w2[i] = x;
            nrm += x.x * x.x + x.y * x.y;
        }
        if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
            double s = 0.0;
            for (int q = 0; q < nq; q++) s += cs[q] * V[(int64_t)q * ldv + n - 1];
            double x = SIGN > 0 ? w[n - 1] + s : w[n - 1] - s;
            w[n - 1] = x;
            nrm += x * x;
        }
    } else {
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
            double s = 0.0;
            for (int q = 0; q < nq; q++) s += cs[q] * V[(int64_t)q * ldv + i];
            double wi = SIGN > 0 ? w[i] + s : w[i] - s;
            w[i] = wi;
            nrm += wi * wi;
        }
    }
    if (partial) {
        for (int o = 16; o > 0; o >>= 1) nrm += __shfl_down_sync(0xffffffffu, nrm, o);
        if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = nrm;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int k = 0; k < RED_BLOCK / 32; k++) s += ws[k];
            partial[(int64_t)blockIdx.x * QMAX] = s;
        }
    }
}

// block partials of sum a_i b_i
__global__ void __launch_bounds__(RED_BLOCK) k_dot(int64_t n, const double *__restrict__ a, const double *__restrict__ b,
                                                    double *__restrict__ partial) {
    mds_pdl_entry();
    __shared__ double ws[RED_BLOCK / 32];
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s += a[i] * b[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < RED_BLOCK / 32; k++) t += ws[k];
        partial[(int64_t)blockIdx.x * QMAX] = t;
    }
}

__global__ void k_scale(int64_t n, const double *w, const double *__restrict__ f, double *o) {
    mds_pdl_entry();
    double s = *f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        o[i] = w[i] * s;
}

// scal[0] = beta = sqrt(normsq); g = (beta, 0, ...); scal[1] = 1/beta
__global__ void k_cycle_start(const double *__restrict__ normsq, double *__restrict__ g, int m,
                              double *__restrict__ scal) {
    mds_pdl_entry();
    double beta = sqrt(normsq[0]);
    scal[0] = beta;
    scal[1] = beta > 0.0 ? 1.0 / beta : 0.0;
    g[0] = beta;
    for (int q = 1; q <= m; q++) g[q] = 0.0;
}

// Arnoldi column j, by all threads of one block: H[0..j][j] = h (+ h2 after
// a second pass), H[j+1][j] = hn = ||w||; apply the previous rotations, form
// the new one, update g.  The column and the rotations are staged in shared
// memory so that the sequential rotation chain does not wait on global
// memory.  scal[2] = |g_{j+1}|, scal[3] = 1/H[j+1][j] (0 on breakdown),
// scal[4] = breakdown flag (1 lucky, 2 non-finite).
__device__ void arnoldi_column(int j, int m, double *H, const double *h, const double *h2, double hn, double *cs,
                               double *sn, double *g, double *scal) {
    __shared__ double col[QMAX + 1], csq[QMAX], snq[QMAX];
    const int t = threadIdx.x;
    if (t <= j) col[t] = h2 ? h[t] + h2[t] : h[t];
    if (t < j) {
        csq[t] = cs[t];
        snq[t] = sn[t];
    }
    __syncthreads();
    if (t == 0) {
        col[j + 1] = hn;
        for (int q = 0; q < j; q++) {
            double a = col[q], c = col[q + 1];
            col[q] = csq[q] * a + snq[q] * c;
            col[q + 1] = -snq[q] * a + csq[q] * c;
        }
        double a = col[j], c = col[j + 1];
        double rr = sqrt(a * a + c * c);
        double cj = rr == 0.0 ? 1.0 : a / rr, sj = rr == 0.0 ? 0.0 : c / rr;
        cs[j] = cj;
        sn[j] = sj;
        col[j] = rr;
        col[j + 1] = 0.0;
        double gj = g[j];
        g[j + 1] = -sj * gj;
        g[j] = cj * gj;
        scal[2] = fabs(sj * gj);
        bool bad = !(hn > 0.0) || !isfinite(hn) || !isfinite(rr);
        scal[3] = bad ? 0.0 : 1.0 / hn;
        scal[4] = !isfinite(hn) || !isfinite(rr) ? 2.0 : (hn == 0.0 ? 1.0 : 0.0);
    }
    __syncthreads();
    if (t <= j + 1) H[t * m + j] = col[t];
}

// One Arnoldi step after the products V^T w are known.
struct GsStep {
    int j, m, pass;  // Arnoldi column, restart length, Gram-Schmidt pass (1 or 2)
    double eta2;     // second-pass threshold on ||w_new||^2 / ||w||^2
    double *H, *h, *cs, *sn, *g, *scal;
};

// w -= sum_q coef_q V[q] (unrolled over q so several rows load at once) and
// ||w||^2; the last block finishes the step.  Pass 1 (coef = h): when
// ||w_new||^2 < eta2 ||w||^2, with ||w||^2 = ||w_new||^2 + ||h||^2, one classical
// pass may have left an orthogonality error of order eps ||w|| / ||w_new||,
// so scal[5] = 1 asks the host for a second pass; otherwise the Arnoldi
// column is formed and scal[5] = 0.  Pass 2 (coef = h2): the column uses
// h + h2 and the norm after the second pass.  eta2 = 1/2 is the DGKS "twice
// is enough" rule; eta2 >= 1 always runs two passes.
__global__ void __launch_bounds__(RED_BLOCK) k_gs_update(int64_t n, const double *__restrict__ V, int64_t ldv, int nq,
                                                          const double *__restrict__ coef, double *__restrict__ w,
                                                          double *__restrict__ partial, unsigned *__restrict__ counter,
                                                          GsStep st) {
    mds_pdl_entry();
    __shared__ double cq[QMAX];
    if (threadIdx.x < QMAX) cq[threadIdx.x] = (int)threadIdx.x < nq ? coef[threadIdx.x] : 0.0;
    __syncthreads();
    double nrm = 0.0;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t n2 = n >> 1;
    double2 *w2 = reinterpret_cast<double2 *>(w);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += stride) {
        // w_i - sum_q c_q V[q][i], accumulated from w_i (one FMA per term)
        double2 x = w2[i];
        int q = 0;
        for (; q + 4 <= nq; q += 4) {
            double2 a0 = reinterpret_cast<const double2 *>(V + (int64_t)q * ldv)[i];
            double2 a1 = reinterpret_cast<const double2 *>(V + (int64_t)(q + 1) * ldv)[i];
            double2 a2 = reinterpret_cast<const double2 *>(V + (int64_t)(q + 2) * ldv)[i];
            double2 a3 = reinterpret_cast<const double2 *>(V + (int64_t)(q + 3) * ldv)[i];
            x.x -= cq[q] * a0.x;
            x.y -= cq[q] * a0.y;
            x.x -= cq[q + 1] * a1.x;
            x.y -= cq[q + 1] * a1.y;
            x.x -= cq[q + 2] * a2.x;
            x.y -= cq[q + 2] * a2.y;
            x.x -= cq[q + 3] * a3.x;
            x.y -= cq[q + 3] * a3.y;
        }
        for (; q < nq; q++) {
            double2 a = reinterpret_cast<const double2 *>(V + (int64_t)q * ldv)[i];
            x.x -= cq[q] * a.x;
            x.y -= cq[q] * a.y;
        }
        w2[i] = x;
        nrm += x.x * x.x + x.y * x.y;
    }
    if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
        double x = w[n - 1];
        for (int q = 0; q < nq; q++) x -= cq[q] * V[(int64_t)q * ldv + n - 1];
        w[n - 1] = x;
        nrm += x * x;
    }
    double t = block_sum(nrm);
    if (threadIdx.x == 0) partial[blockIdx.x] = t;
    if (!last_block(counter)) return;
    double u = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += RED_BLOCK) u += __ldcg(partial + b);
    __shared__ double nsq_s;
    __shared__ int second;
    double nsq = block_sum(u);
    if (threadIdx.x == 0) {
        // ||w||^2 before the pass = ||w_new||^2 + ||h||^2 (w_new is orthogonal
        // to the orthonormal basis up to rounding)
        double hh = 0.0;
        for (int q = 0; q < nq; q++) hh += cq[q] * cq[q];
        nsq_s = nsq;
        second = st.pass == 1 && nsq < st.eta2 * (nsq + hh);
        st.scal[5] = second ? 1.0 : 0.0;
    }
    __syncthreads();
    if (second) return;
    arnoldi_column(st.j, st.m, st.H, st.h, st.pass == 2 ? coef : nullptr, sqrt(nsq_s), st.cs, st.sn, st.g, st.scal);
}

// v_{j+1} = w / H[j+1][j], unless a second Gram-Schmidt pass is pending
__global__ void k_scale_step(int64_t n, double *__restrict__ w, const double *__restrict__ scal) {
    mds_pdl_entry();
    if (scal[5] != 0.0) return;
    double s = scal[3];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        w[i] *= s;
}

// upper-triangular solve H y = g (k columns)
__global__ void k_backsolve(int k, int m, const double *__restrict__ H, const double *__restrict__ g,
                            double *__restrict__ y) {
    mds_pdl_entry();
    for (int q = k - 1; q >= 0; q--) {
        double s = g[q];
        for (int p = q + 1; p < k; p++) s -= H[q * m + p] * y[p];
        y[q] = H[q * m + q] == 0.0 ? 0.0 : s / H[q * m + q];
    }
}

// PCG helpers
__global__ void k_pcg_p(int64_t n, const double *__restrict__ z, double *__restrict__ p, const double *__restrict__ sc,
                        int first) {
    mds_pdl_entry();
    double beta = first ? 0.0 : sc[0] / sc[1];  // rz_new / rz
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = first ? z[i] : z[i] + beta * p[i];
}

__global__ void __launch_bounds__(RED_BLOCK) k_pcg_xr(int64_t n, double *__restrict__ x, double *__restrict__ r,
                                                       const double *__restrict__ p, const double *__restrict__ q,
                                                       const double *__restrict__ sc, double *__restrict__ partial) {
    mds_pdl_entry();
    __shared__ double ws[RED_BLOCK / 32];
    double alpha = sc[0] / sc[2];  // rz / (p, q)
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        x[i] += alpha * p[i];
        double ri = r[i] - alpha * q[i];
        r[i] = ri;
        s += ri * ri;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < RED_BLOCK / 32; k++) t += ws[k];
        partial[(int64_t)blockIdx.x * QMAX] = t;
    }
}

// ---- preconditioned MINRES (three-term Lanczos in the M-inner product with
// Givens rotations; Paige and Saunders 1975, in the recurrence of Elman,
// Silvester and Wathen).  Device scalars, indices into sc[]:
enum { MR_G0 = 0, MR_G1, MR_C0, MR_C1, MR_S0, MR_S1, MR_ETA, MR_DELTA, MR_ZV, MR_RR, MR_A1, MR_A2, MR_A3, MR_STEP,
       MR_FLAG, MR_G2, MR_COUNT };

// t = z / gamma_j (the normalised z_j)
__global__ void k_mr_scale(int64_t n, const double *__restrict__ z, const double *__restrict__ sc,
                           double *__restrict__ t) {
    mds_pdl_entry();
    double g = sc[MR_G1];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        t[i] = z[i] / g;
}

// v_old <- A z_j - (delta / gamma_j) v_cur - (gamma_j / gamma_{j-1}) v_old
__global__ void k_mr_lanczos(int64_t n, const double *__restrict__ az, const double *__restrict__ vcur,
                             double *__restrict__ vold, const double *__restrict__ sc) {
    mds_pdl_entry();
    double a = sc[MR_DELTA] / sc[MR_G1], b = sc[MR_G1] / sc[MR_G0];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        vold[i] = az[i] - a * vcur[i] - b * vold[i];
}

// Rotations for the new column of the tridiagonal matrix; the step length
// along w_{j+1}; the scalars shifted for the next step.  MR_FLAG = 1 when the
// rotation is undefined (breakdown).
__global__ void k_mr_rotate(double *__restrict__ sc) {
    mds_pdl_entry();
    double g0 = sc[MR_G0], g1 = sc[MR_G1], c0 = sc[MR_C0], c1 = sc[MR_C1], s0 = sc[MR_S0], s1 = sc[MR_S1];
    double delta = sc[MR_DELTA], zv = sc[MR_ZV], eta = sc[MR_ETA];
    double a0 = c1 * delta - c0 * s1 * g1;
    double a2 = s1 * delta + c0 * c1 * g1;
    double a3 = s0 * g1;
    double g2 = zv > 0.0 ? sqrt(zv) : 0.0;
    double a1 = sqrt(a0 * a0 + g2 * g2);
    bool bad = !(a1 > 0.0) || !isfinite(a1);
    double c2 = bad ? 1.0 : a0 / a1, s2 = bad ? 0.0 : g2 / a1;
    sc[MR_A1] = bad ? 1.0 : a1;
    sc[MR_A2] = a2;
    sc[MR_A3] = a3;
    sc[MR_STEP] = bad ? 0.0 : c2 * eta;
    sc[MR_ETA] = -s2 * eta;
    sc[MR_FLAG] = bad ? 1.0 : 0.0;
    sc[MR_G2] = g2;
    sc[MR_G0] = g1;
    sc[MR_G1] = g2 > 0.0 ? g2 : 1.0;
    sc[MR_C0] = c1;
    sc[MR_C1] = c2;
    sc[MR_S0] = s1;
    sc[MR_S1] = s2;
    (void)g0;
}

// w_old <- (z_j - a3 w_old - a2 w_cur) / a1, the same for A w, then
// x += step w_new, r -= step A w_new, and block partials of ||r||^2.
__global__ void __launch_bounds__(RED_BLOCK) k_mr_update(int64_t n, const double *__restrict__ t,
                                                         const double *__restrict__ az, double *__restrict__ wold,
                                                         const double *__restrict__ wcur, double *__restrict__ awold,
                                                         const double *__restrict__ awcur, double *__restrict__ x,
                                                         double *__restrict__ r, const double *__restrict__ sc,
                                                         double *__restrict__ partial) {
    mds_pdl_entry();
    __shared__ double ws[RED_BLOCK / 32];
    const double a1 = sc[MR_A1], a2 = sc[MR_A2], a3 = sc[MR_A3], step = sc[MR_STEP];
    double nrm = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double wn = (t[i] - a3 * wold[i] - a2 * wcur[i]) / a1;
        double awn = (az[i] - a3 * awold[i] - a2 * awcur[i]) / a1;
        wold[i] = wn;
        awold[i] = awn;
        x[i] += step * wn;
        double ri = r[i] - step * awn;
        r[i] = ri;
        nrm += ri * ri;
    }
    for (int o = 16; o > 0; o >>= 1) nrm += __shfl_down_sync(0xffffffffu, nrm, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = nrm;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < RED_BLOCK / 32; k++) s += ws[k];
        partial[(int64_t)blockIdx.x * QMAX] = s;
    }
}

// start of a cycle: gamma_1 = sqrt(z . v), eta = gamma_1, rotations reset
__global__ void k_mr_start(double *__restrict__ sc) {
    mds_pdl_entry();
    double zv = sc[MR_ZV];
    double g1 = zv > 0.0 ? sqrt(zv) : 0.0;
    sc[MR_G0] = 1.0;
    sc[MR_G1] = g1 > 0.0 ? g1 : 1.0;
    sc[MR_G2] = g1;
    sc[MR_C0] = sc[MR_C1] = 1.0;
    sc[MR_S0] = sc[MR_S1] = 0.0;
    sc[MR_ETA] = g1;
}

__global__ void k_copy1(const double *__restrict__ a, double *__restrict__ b) { mds_pdl_entry(); *b = *a; }

// ---------------------------------------------------------------- host side

struct Red {
    Buf partial;
    double *pp = nullptr;  // the partials buffer in use
    unsigned grid = 1;     // blocks of the single-vector reductions
    int slots = 1;         // resident blocks of k_gs_dot on the device
    unsigned ugrid = 1;    // blocks of k_gs_update: at most one wave
};

// Partial sums one k_gs_dot launch may write (row blocks x outputs).
constexpr int GS_MAX_BLOCKS = 4096;

// Row blocks per output of k_gs_dot for nout outputs: one wave of resident
// blocks in total (equal work per block, and the fewest per-block
// reductions, which cost FP64 operations), at least two elements per thread.
static unsigned gs_dot_grid(const Red &R, int64_t n, int nout) {
    int64_t g = (int64_t)R.slots / nout;
    int64_t cap = (n + 2 * RED_BLOCK - 1) / (2 * RED_BLOCK);
    if (g > cap) g = cap;
    if (g * nout > GS_MAX_BLOCKS) g = GS_MAX_BLOCKS / nout;
    if (g < 1) g = 1;
    return (unsigned)g;
}

static void gs_grids(Ctx &c, Red &R, int64_t n) {
    int sms = 0, occ = 0, uocc = 0;
    MDS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c.device));
    MDS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_gs_dot, RED_BLOCK, 0));
    MDS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&uocc, k_gs_update, RED_BLOCK, 0));
    int s = sms * (occ > 0 ? occ : 1);
    R.slots = s > GS_MAX_BLOCKS / 2 - QMAX ? GS_MAX_BLOCKS / 2 - QMAX : s;
    unsigned us = (unsigned)(sms * (uocc > 0 ? uocc : 1));
    R.ugrid = red_grid(n) < us ? red_grid(n) : us;
}

static void dot_dev(Ctx &c, Red &R, int64_t n, const double *a, const double *b, double *out) {
    MDS_LAUNCH(c, KC_NONE, 16.0 * n, k_dot, R.grid, RED_BLOCK, 0, n, a, b, R.pp);
    MDS_LAUNCH(c, KC_NONE, 0, k_reduce_cols, 1, 32, 0, R.pp, (int)R.grid, 1, out, 0);
}

static size_t round256(size_t doubles) { return (doubles + 31) / 32 * 32; }

// Workspace parts in order: reduction partials, V ((m+1) rows), Z (m rows),
// Hessenberg ((m+1) x m), small scalars (256).
static size_t partial_doubles(int64_t n) {
    size_t a = (size_t)red_grid(n) * QMAX;
    return a > (size_t)GS_MAX_BLOCKS ? a : (size_t)GS_MAX_BLOCKS;
}

size_t fgmres_workspace_doubles(int64_t n, int m) {
    const int64_t ld = (n + 63) / 64 * 64;
    return round256(partial_doubles(n)) + round256((size_t)(m + 1) * ld) + round256((size_t)m * ld) +
           round256((size_t)(m + 1) * m) + 256;
}

FgmresWorkspace fgmres_workspace_carve(double *base, int64_t n, int m) {
    const int64_t ld = (n + 63) / 64 * 64;
    FgmresWorkspace w;
    w.partial = base;
    w.V = w.partial + round256(partial_doubles(n));
    w.Z = w.V + round256((size_t)(m + 1) * ld);
    w.H = w.Z + round256((size_t)m * ld);
    w.small = w.H + round256((size_t)(m + 1) * m);
    return w;
}

KrylovResult fgmres(Ctx &c, const mds_csr &A, const PrecFn &M, const double *b, double *x, int64_t n,
                    const mds_solve_opts &o, const FgmresWorkspace *ws) {
    KrylovResult res;
    const int m = o.restart < 1 ? 1 : (o.restart > QMAX - 1 ? QMAX - 1 : o.restart);
    Red R;
    R.grid = red_grid(n);
    gs_grids(c, R, n);
    // basis rows padded to 64 elements: 16-byte aligned rows for vector loads
    const int64_t ld = (n + 63) / 64 * 64;
    Buf V, Z, H, small;
    double *Vp, *Zp, *Hp, *d, *partial;
    if (ws) {
        partial = ws->partial;
        Vp = ws->V;
        Zp = ws->Z;
        Hp = ws->H;
        d = ws->small;
    } else {
        R.partial = Buf(&c, sizeof(double) * partial_doubles(n));
        V = Buf(&c, sizeof(double) * (size_t)(m + 1) * (size_t)ld);
        Z = Buf(&c, sizeof(double) * (size_t)m * (size_t)ld);
        H = Buf(&c, sizeof(double) * (size_t)(m + 1) * m);
        small = Buf(&c, sizeof(double) * 256);
        partial = R.partial.as<double>();
        Vp = V.as<double>();
        Zp = Z.as<double>();
        Hp = H.as<double>();
        d = small.as<double>();
    }
    R.pp = partial;
    MDS_REQUIRE(partial && Vp && Zp && Hp && d, MDS_ERR_INVALID, "FGMRES workspace pointer missing");
    MDS_CUDA(cudaMemsetAsync(d, 0, sizeof(double) * 256, c.stream));
    // cs, sn, g, y, h (first Gram-Schmidt pass), h2 (second
    // pass), scal (step scalars; scal[5] = second pass pending), nsq, and two
    // block-arrival counters of the fused reductions
    double *cs = d, *sn = d + 32, *g = d + 64, *y = d + 96, *h = d + 128, *h2 = d + 160, *scal = d + 192,
           *nsq = d + 224;
    unsigned *cnt = reinterpret_cast<unsigned *>(d + 240);
    // ||b||
    dot_dev(c, R, n, b, b, nsq);
    double bn = std::sqrt(c.read(nsq));
    if (!(bn < INFINITY)) {
        res.status = MDS_ERR_NONFINITE;
        return res;
    }
    if (bn == 0.0) bn = 1.0;
    auto gs_pass = [&](int j, int pass) {
        double *w = Vp + (size_t)(j + 1) * ld;
        int nq = j + 1;
        int nout = nq;
        double *hh = pass == 1 ? h : h2;
        unsigned mg = gs_dot_grid(R, n, nout);
        GsStep st{j, m, pass, o.reorth_eta2, Hp, h, cs, sn, g, scal};
        int cls_dot = pass == 1 ? KC_GS_DOT : KC_NONE, cls_upd = pass == 1 ? KC_GS_AXPY : KC_NONE;
        MDS_LAUNCH_F(c, cls_dot, 8.0 * n * (nq + 1), 2.0 * n * nq, k_gs_dot, dim3(mg, nout), RED_BLOCK, 0, n, Vp,
                     ld, nq, w, R.pp, cnt, hh);
        MDS_LAUNCH_F(c, cls_upd, 8.0 * n * (nq + 2), 2.0 * n * (nq + 1), k_gs_update, R.ugrid, RED_BLOCK, 0, n, Vp, ld,
                     nq, hh, w, R.pp, cnt + 1, st);
        MDS_LAUNCH(c, KC_NONE, 16.0 * n, k_scale_step, red_grid(n), RED_BLOCK, 0, n, w, scal);
        MDS_CUDA(cudaMemcpyAsync(c.h_pin, scal, 6 * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    };
    // One Arnoldi step j: z_j = M v_j, w = A z_j, one classical Gram-Schmidt
    // pass with its reductions, cancellation test and Givens update fused into
    // two launches, the scaled v_{j+1}, and the step's scalars copied to
    // pinned host memory.  Captured as a CUDA graph on first use and replayed
    // on later restart cycles.  A second pass, when the cancellation test asks
    // for it, is launched directly by the host (rare).
    auto body = [&](int j) {
        double *vj = Vp + (size_t)j * ld, *zj = Zp + (size_t)j * ld;
        M(vj, zj);
        spmv_f64(c, A, zj, Vp + (size_t)(j + 1) * ld, KC_SPMV);
        gs_pass(j, 1);
    };
    // Step graphs: one set, or with timing sampled, an unbracketed set and a
    // bracketed set used in every sample_every-th restart cycle.
    bool any_timed = false;
    for (int k = 0; k < MDS_KCLASS_COUNT; k++) any_timed = any_timed || c.timing[k];
    const bool sampled = any_timed && c.sample_every > 1;
    std::vector<std::unique_ptr<Graph>> graphs(m), graphs_timed(sampled ? m : 0);
    bool graphs_ok = o.graphs != 0;
    int restarts = 0;
    auto run_step = [&](int j) {
        Graph *gj = nullptr;
        bool bracket = !sampled || restarts % c.sample_every == 0;
        if (graphs_ok) {
            auto &slot = sampled && bracket ? graphs_timed[j] : graphs[j];
            if (!slot) {
                slot.reset(new Graph);
                c.timing_suspended = !bracket;
                bool ok = graph_capture(c, *slot, [&] { body(j); });
                c.timing_suspended = false;
                if (!ok) {
                    slot.reset();
                    graphs_ok = false;
                }
            }
            gj = slot.get();
        }
        if (gj) {
            graph_launch(c, *gj);
        } else {
            c.timing_suspended = !bracket;
            try {
                body(j);
            } catch (...) {
                c.timing_suspended = false;
                throw;
            }
            c.timing_suspended = false;
        }
        c.sync();
        if (gj) graph_collect(c, *gj);
    };
    int it = 0;
    double est = 0.0;
    for (;;) {
        spmv_sub_f64(c, A, b, x, Vp);  // V0 = b - A x
        dot_dev(c, R, n, Vp, Vp, nsq);
        MDS_LAUNCH(c, KC_NONE, 0, k_cycle_start, 1, 1, 0, nsq, g, m, scal);
        double beta = c.read(scal);
        if (!std::isfinite(beta)) {
            res.status = MDS_ERR_NONFINITE;
            break;
        }
        est = beta / bn;
        if (est <= o.rtol) {
            res.status = MDS_OK;
            break;
        }
        if (it >= o.max_iters) {
            res.status = MDS_WARN_NOT_CONVERGED;
            break;
        }
        MDS_LAUNCH(c, KC_NONE, 16.0 * n, k_scale, red_grid(n), RED_BLOCK, 0, n, Vp, scal + 1, Vp);
        int kdone = 0;
        int flag = 0;
        for (int j = 0; j < m; j++) {
            run_step(j);
            double sv[6];
            std::memcpy(sv, c.h_pin, sizeof sv);
            if (sv[5] != 0.0) {
                gs_pass(j, 2);
                c.sync();
                std::memcpy(sv, c.h_pin, sizeof sv);
            }
            it++;
            est = sv[2] / bn;
            kdone = j + 1;
            if (sv[4] == 2.0 || !std::isfinite(est)) {
                flag = 2;
                break;
            }
            if (est <= o.rtol || it >= o.max_iters || sv[4] == 1.0) break;
        }
        if (flag == 2) {
            res.status = MDS_ERR_BREAKDOWN;
            break;
        }
        MDS_LAUNCH(c, KC_NONE, 0, k_backsolve, 1, 1, 0, kdone, m, Hp, g, y);
        MDS_LAUNCH(c, KC_NONE, 8.0 * n * (kdone + 2), (k_maxpy<1, false>), R.grid, RED_BLOCK, 0, n, Zp, ld, kdone,
                   y, x, nullptr, (const double *)nullptr);
        restarts++;
    }
    // true residual at exit
    spmv_sub_f64(c, A, b, x, Vp);
    dot_dev(c, R, n, Vp, Vp, nsq);
    res.relres_true = std::sqrt(c.read(nsq)) / bn;
    res.iterations = it;
    res.restarts = restarts;
    res.relres_est = est;
    return res;
}

KrylovResult pcg(Ctx &c, const mds_csr &A, const PrecFn &M, const double *b, double *x, int64_t n,
                 const mds_solve_opts &o) {
    KrylovResult res;
    Red R;
    R.grid = red_grid(n);
    R.partial = Buf(&c, sizeof(double) * (size_t)R.grid * QMAX);
    R.pp = R.partial.as<double>();
    Buf rb(&c, sizeof(double) * (size_t)n), zb(&c, sizeof(double) * (size_t)n), pb(&c, sizeof(double) * (size_t)n),
        qb(&c, sizeof(double) * (size_t)n);
    Buf small(&c, sizeof(double) * 8);
    double *sc = small.as<double>();  // [rz_new, rz, pq, rn2, bn2]
    double *r = rb.as<double>(), *z = zb.as<double>(), *p = pb.as<double>(), *q = qb.as<double>();
    dot_dev(c, R, n, b, b, sc + 4);
    double bn = std::sqrt(c.read(sc + 4));
    if (!(bn < INFINITY)) {
        res.status = MDS_ERR_NONFINITE;
        return res;
    }
    if (bn == 0.0) bn = 1.0;
    spmv_sub_f64(c, A, b, x, r);
    dot_dev(c, R, n, r, r, sc + 3);
    double rn = std::sqrt(c.read(sc + 3));
    int it = 0;
    // one PCG iteration; graph 0 is the first iteration (p = z), graph 1 the rest
    auto body = [&](int first) {
        M(r, z);
        dot_dev(c, R, n, r, z, sc);  // rz_new
        MDS_LAUNCH(c, KC_NONE, 24.0 * n, k_pcg_p, red_grid(n), RED_BLOCK, 0, n, z, p, sc, first);
        MDS_LAUNCH(c, KC_NONE, 0, k_copy1, 1, 1, 0, sc, sc + 1);  // rz = rz_new
        spmv_f64(c, A, p, q, KC_SPMV);
        dot_dev(c, R, n, p, q, sc + 2);
        MDS_LAUNCH(c, KC_NONE, 56.0 * n, k_pcg_xr, R.grid, RED_BLOCK, 0, n, x, r, p, q, sc, R.pp);
        MDS_LAUNCH(c, KC_NONE, 0, k_reduce_cols, 1, 32, 0, R.pp, (int)R.grid, 1, sc + 3, 0);
        MDS_CUDA(cudaMemcpyAsync(c.h_pin, sc + 3, sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    };
    std::unique_ptr<Graph> graphs[2];
    bool graphs_ok = o.graphs != 0;
    while (rn / bn > o.rtol && it < o.max_iters) {
        int first = it == 0 ? 1 : 0;
        Graph *gj = nullptr;
        if (graphs_ok) {
            if (!graphs[first]) {
                graphs[first].reset(new Graph);
                if (!graph_capture(c, *graphs[first], [&] { body(first); })) {
                    graphs[first].reset();
                    graphs_ok = false;
                }
            }
            gj = graphs[first].get();
        }
        if (gj)
            graph_launch(c, *gj);
        else
            body(first);
        c.sync();
        if (gj) graph_collect(c, *gj);
        it++;
        double rn2;
        std::memcpy(&rn2, c.h_pin, sizeof rn2);
        rn = std::sqrt(rn2);
        if (!std::isfinite(rn)) {
            res.status = MDS_ERR_BREAKDOWN;
            break;
        }
    }
    spmv_sub_f64(c, A, b, x, r);
    dot_dev(c, R, n, r, r, sc + 3);
    res.relres_true = std::sqrt(c.read(sc + 3)) / bn;
    res.relres_est = rn / bn;
    res.iterations = it;
    if (res.status != MDS_ERR_BREAKDOWN) res.status = res.relres_true <= o.rtol ? MDS_OK : MDS_WARN_NOT_CONVERGED;
    return res;
}

KrylovResult minres(Ctx &c, const mds_csr &A, const PrecFn &M, const double *b, double *x, int64_t n,
                    const mds_solve_opts &o) {
    KrylovResult res;
    Red R;
    R.grid = red_grid(n);
    R.partial = Buf(&c, sizeof(double) * (size_t)R.grid * QMAX);
    R.pp = R.partial.as<double>();
    // r, z, t (= z_j), A z_j, v[2], w[2], A w[2]
    Buf buf(&c, sizeof(double) * (size_t)n * 10);
    double *r = buf.as<double>(), *z = r + n, *t = z + n, *az = t + n;
    double *v[2] = {az + n, az + 2 * n}, *w[2] = {az + 3 * n, az + 4 * n}, *aw[2] = {az + 5 * n, az + 6 * n};
    Buf small(&c, sizeof(double) * 32);
    double *sc = small.as<double>();
    const unsigned eg = red_grid(n);
    dot_dev(c, R, n, b, b, sc + MR_RR);
    double bn = std::sqrt(c.read(sc + MR_RR));
    if (!(bn < INFINITY)) {
        res.status = MDS_ERR_NONFINITE;
        return res;
    }
    if (bn == 0.0) bn = 1.0;
    // one Lanczos step with parity p: v[p], w[p], aw[p] hold the older
    // vectors and receive the new ones
    auto body = [&](int p) {
        const int q = 1 - p;
        MDS_LAUNCH(c, KC_NONE, 16.0 * n, k_mr_scale, eg, RED_BLOCK, 0, n, z, sc, t);
        spmv_f64(c, A, t, az, KC_SPMV);
        dot_dev(c, R, n, az, t, sc + MR_DELTA);
        MDS_LAUNCH(c, KC_NONE, 32.0 * n, k_mr_lanczos, eg, RED_BLOCK, 0, n, az, v[q], v[p], sc);
        M(v[p], z);
        dot_dev(c, R, n, z, v[p], sc + MR_ZV);
        MDS_LAUNCH(c, KC_NONE, 0, k_mr_rotate, 1, 1, 0, sc);
        MDS_LAUNCH(c, KC_NONE, 104.0 * n, k_mr_update, R.grid, RED_BLOCK, 0, n, t, az, w[p], w[q], aw[p], aw[q], x, r,
                   sc, R.pp);
        MDS_LAUNCH(c, KC_NONE, 0, k_reduce_cols, 1, 32, 0, R.pp, (int)R.grid, 1, sc + MR_RR, 0);
        MDS_CUDA(cudaMemcpyAsync(c.h_pin, sc, sizeof(double) * MR_COUNT, cudaMemcpyDeviceToHost, c.stream));
    };
    std::unique_ptr<Graph> graphs[2];
    bool graphs_ok = o.graphs != 0;
    int it = 0, cycles = 0;
    double rr = 0.0;
    for (;;) {
        spmv_sub_f64(c, A, b, x, r);
        dot_dev(c, R, n, r, r, sc + MR_RR);
        rr = std::sqrt(c.read(sc + MR_RR));
        if (!std::isfinite(rr)) {
            res.status = MDS_ERR_NONFINITE;
            break;
        }
        if (rr / bn <= o.rtol || it >= o.max_iters) break;
        cycles++;
        // v[1] = r, v[0] = w = A w = 0, z = M v[1], gamma_1
        MDS_CUDA(cudaMemcpyAsync(v[1], r, sizeof(double) * (size_t)n, cudaMemcpyDeviceToDevice, c.stream));
        MDS_CUDA(cudaMemsetAsync(v[0], 0, sizeof(double) * (size_t)n, c.stream));
        MDS_CUDA(cudaMemsetAsync(w[0], 0, sizeof(double) * (size_t)n * 2, c.stream));
        MDS_CUDA(cudaMemsetAsync(aw[0], 0, sizeof(double) * (size_t)n * 2, c.stream));
        M(v[1], z);
        dot_dev(c, R, n, z, v[1], sc + MR_ZV);
        MDS_LAUNCH(c, KC_NONE, 0, k_mr_start, 1, 1, 0, sc);
        if (!(c.read(sc + MR_G2) > 0.0)) {
            res.status = MDS_ERR_BREAKDOWN;
            break;
        }
        int p = 0;
        bool stop = false;
        while (it < o.max_iters) {
            Graph *gj = nullptr;
            if (graphs_ok) {
                if (!graphs[p]) {
                    graphs[p].reset(new Graph);
                    if (!graph_capture(c, *graphs[p], [&] { body(p); })) {
                        graphs[p].reset();
                        graphs_ok = false;
                    }
                }
                gj = graphs[p].get();
            }
            if (gj)
                graph_launch(c, *gj);
            else
                body(p);
            c.sync();
            if (gj) graph_collect(c, *gj);
            it++;
            p = 1 - p;
            double s[MR_COUNT];
            std::memcpy(s, c.h_pin, sizeof s);
            rr = std::sqrt(s[MR_RR]);
            if (s[MR_FLAG] != 0.0 || !std::isfinite(rr)) {
                res.status = MDS_ERR_BREAKDOWN;
                stop = true;
                break;
            }
            if (rr / bn <= o.rtol) break;
            if (!(s[MR_G2] > 0.0)) break;  // invariant subspace: restart from x
        }
        if (stop) break;
    }
    spmv_sub_f64(c, A, b, x, r);
    dot_dev(c, R, n, r, r, sc + MR_RR);
    res.relres_true = std::sqrt(c.read(sc + MR_RR)) / bn;
    res.relres_est = rr / bn;
    res.iterations = it;
    res.restarts = cycles > 0 ? cycles - 1 : 0;
    if (res.status == MDS_OK) res.status = res.relres_true <= o.rtol ? MDS_OK : MDS_WARN_NOT_CONVERGED;
    return res;
}

// ---------------------------------------------------------------- no-allocation workspace

// Static FGMRES workspace for mds_solve_noalloc: 8 MiB in every device that
// loads the library, enough for n <= MDS_NOALLOC_MAX_N and restart <= 30.
constexpr size_t NOALLOC_DOUBLES = (size_t)MDS_NOALLOC_SCRATCH_BYTES / sizeof(double);
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_DOUBLES];

size_t noalloc_scratch_doubles() { return NOALLOC_DOUBLES; }

// The symbol's device address on the current device.  mds_create calls this
// with the context's device current and keeps the result in the context: the
// host-side name is only a stand-in, never a device address, and resolving it
// loads the module that holds the array, so that happens while the context
// is created rather than in the middle of a solve.
double *noalloc_scratch_lookup() {
    void *p = nullptr;
    MDS_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    return static_cast<double *>(p);
}

double *noalloc_scratch(Ctx &c) {
    MDS_REQUIRE(c.noalloc_scratch != nullptr, MDS_ERR_INVALID, "context has no static workspace address");
    return c.noalloc_scratch;
}

}  // namespace mds

// ================================================================ batched lockstep FGMRES
//
// P = K instances x NR columns independent problems on one packed system:
// instance k owns the matrix rows [moff_k, moff_k+1) and the fracture rows
// [NM + foff_k, NM + foff_k+1); vectors hold NR interleaved columns.  Every
// problem runs its own right-preconditioned FGMRES(m) (own Krylov basis,
// Hessenberg matrix, rotations, restarts and convergence); the SpMV, the
// V-cycles and the Gram-Schmidt passes of all problems share one launch each,
// so every matrix entry is read once per NR columns.  A problem whose
// estimate has converged sits out (mask) until the common restart; its x is
// updated with its own step count.

namespace mds {

struct Chunk {
    int64_t b, e;  // row range
    int32_t inst;
};

// partial[(q * nchunk + chunk) * NR + c] = sum over the chunk's rows of
// V_q(i, c) W(i, c); row q == nq is W itself (squared norm).
// Chunk-level skip for the masked second Gram-Schmidt pass: true when no
// column of the chunk's instance is flagged.
template <int NR> __device__ __forceinline__ bool chunk_skipped(const int8_t *mask, int32_t inst) {
    if (!mask) return false;
#pragma unroll
    for (int c = 0; c < NR; c++)
        if (mask[(int64_t)inst * NR + c]) return false;
    return true;
}

template <int NR>
__global__ void __launch_bounds__(RED_BLOCK) k_bdot(const Chunk *__restrict__ ch, int nchunk, const double *__restrict__ V,
                                                     int64_t ldq, int nq, const double *__restrict__ W,
                                                     double *__restrict__ partial, const int8_t *__restrict__ mask,
                                                     const int32_t *__restrict__ lc) {
    mds_pdl_entry();
    __shared__ double ws[RED_BLOCK / 32][NR];
    // the nq blocks of one chunk are adjacent in launch order, so they run
    // together and the chunk of W is read from DRAM once (a grid-stride loop
    // over a resident grid loses this order, measured slower)
    const int nqb = nq > 0 ? nq : 1;
    const int64_t chunk = lc ? lc[blockIdx.x / nqb] : blockIdx.x / nqb;  // lc: the live chunks only
    const int q = (int)(blockIdx.x % nqb);
    Chunk k = ch[chunk];
    if (chunk_skipped<NR>(mask, k.inst)) return;
    const double *v = q < nq ? V + (int64_t)q * ldq : W;
    double s[NR];
#pragma unroll
    for (int c = 0; c < NR; c++) s[c] = 0.0;
    for (int64_t i = k.b + threadIdx.x; i < k.e; i += blockDim.x)
#pragma unroll
        for (int c = 0; c < NR; c++) s[c] += v[i * NR + c] * W[i * NR + c];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < NR; c++) {
        double t = s[c];
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        if (lane == 0) ws[w][c] = t;
    }
    __syncthreads();
    if (threadIdx.x < NR) {
        double t = 0.0;
        for (int k2 = 0; k2 < RED_BLOCK / 32; k2++) t += ws[k2][threadIdx.x];
        partial[((int64_t)q * nchunk + chunk) * NR + threadIdx.x] = t;
    }
}

// out[p * 32 + q] (+)= sum over instance k's chunks of partial[q][chunk][c],
// p = k NR + c; one warp per (q, p), fixed order.
__global__ void k_breduce(const double *__restrict__ partial, int nchunk, int nq, int NR,
                          const int32_t *__restrict__ ioff, const int32_t *__restrict__ ichunk, int P,
                          double *__restrict__ out, int accumulate, const int8_t *__restrict__ mask) {
    mds_pdl_entry();
    int q = blockIdx.y;
    int p = blockIdx.x;
    if (p >= P || q >= nq || (mask && !mask[p])) return;
    int k = p / NR, c = p % NR;
    double s = 0.0;
    for (int t = ioff[k] + threadIdx.x; t < ioff[k + 1]; t += 32)
        s += partial[((int64_t)q * nchunk + ichunk[t]) * NR + c];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) out[(int64_t)p * 32 + q] = accumulate ? out[(int64_t)p * 32 + q] + s : s;
}

// W(i, c) += SIGN sum_q coef[p][q] V_q(i, c) over one chunk per block;
// optional partials of W(i, c)^2 as partial[chunk][c] (q = 0 layout).
// qlim (optional): the chunk's instance uses V_q for q < max over its
// columns of qlim[p] only (the coefficients beyond a column's own count are
// zero; later V_q rows of an instance that stopped were never computed).
template <int NR, int SIGN>
__global__ void __launch_bounds__(RED_BLOCK) k_bmaxpy(const Chunk *__restrict__ ch, const double *__restrict__ V,
                                                       int64_t ldq, int nq, const double *__restrict__ coef,
                                                       double *__restrict__ W, double *__restrict__ partial,
                                                       const int8_t *__restrict__ mask,
                                                       const int32_t *__restrict__ qlim, const int32_t *__restrict__ lc) {
    mds_pdl_entry();
    __shared__ double cs[NR][32];
    __shared__ double ws[RED_BLOCK / 32][NR];
    const int64_t chunk = lc ? lc[blockIdx.x] : blockIdx.x;  // lc: the live chunks only
    Chunk k = ch[chunk];
    if (chunk_skipped<NR>(mask, k.inst)) return;
    if (qlim) {
        int q1 = 0;
#pragma unroll
        for (int c = 0; c < NR; c++) q1 = max(q1, qlim[(int64_t)k.inst * NR + c]);
        if (q1 == 0) return;
        nq = min(nq, q1);
    }
    // the coefficients carry the sign, so W(i, c) itself starts each row's
    // chain of fused multiply-adds
    for (int t = threadIdx.x; t < NR * 32; t += blockDim.x) {
        int c = t / 32, q = t % 32;
        const double a = q < nq ? coef[((int64_t)k.inst * NR + c) * 32 + q] : 0.0;
        cs[c][q] = SIGN > 0 ? a : -a;
    }
    __syncthreads();
    double nrm[NR];
#pragma unroll
    for (int c = 0; c < NR; c++) nrm[c] = 0.0;
    for (int64_t i = k.b + threadIdx.x; i < k.e; i += blockDim.x) {
        double s[NR];
#pragma unroll
        for (int c = 0; c < NR; c++) s[c] = W[i * NR + c];
        for (int q = 0; q < nq; q++) {
            const double *v = V + (int64_t)q * ldq + i * NR;
#pragma unroll
            for (int c = 0; c < NR; c++) s[c] = fma(cs[c][q], v[c], s[c]);
        }
#pragma unroll
        for (int c = 0; c < NR; c++) {
            W[i * NR + c] = s[c];
            nrm[c] += s[c] * s[c];
        }
    }
    if (partial) {
        int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
        for (int c = 0; c < NR; c++) {
            double t = nrm[c];
            for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
            if (lane == 0) ws[w][c] = t;
        }
        __syncthreads();
        if (threadIdx.x < NR) {
            double t = 0.0;
            for (int k2 = 0; k2 < RED_BLOCK / 32; k2++) t += ws[k2][threadIdx.x];
            partial[chunk * NR + threadIdx.x] = t;
        }
    }
}

// Per problem after the first Gram-Schmidt pass: flag[p] = 1 when the pass
// cancelled severely (||w_new||^2 < eta2 (||w_new||^2 + ||h||^2)), the
// second-pass coefficients start at 0.
__global__ void k_bflag(int P, int nq, const int8_t *__restrict__ active, const double *__restrict__ h1,
                        const double *__restrict__ nsq, double eta2, int8_t *__restrict__ flag,
                        double *__restrict__ h2) {
    mds_pdl_entry();
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    double hh = 0.0;
    for (int q = 0; q < nq; q++) hh += h1[(int64_t)p * 32 + q] * h1[(int64_t)p * 32 + q];
    double w2 = nsq[(int64_t)p * 32];
    flag[p] = active[p] && w2 < eta2 * (w2 + hh) ? 1 : 0;
    for (int q = 0; q < 32; q++) h2[(int64_t)p * 32 + q] = 0.0;
}

// W(i, c) *= f[p]  (f = sc[p * 8 + slot]) for active problems; inactive ones
// get exact zeros, so the vectors of a problem that has stopped stay bounded
// (and 0 * their entries stays 0 in the shared kernels).
// The chunk is scaled element by element (entry (i, c) at i * NR + c): the
// block size is a multiple of NR, so each thread keeps one column c and one
// factor, and a warp's loads and stores are contiguous.  With st, the
// entries of rows below st_rows are also written in FP32 to st (same
// layout): the preconditioner's FP32 input, rounded to nearest as its own
// conversion rounds, by integer operations (the FP64 unit does the scaling).
template <int NR>
__global__ void __launch_bounds__(RED_BLOCK) k_bscale(const Chunk *__restrict__ ch, double *__restrict__ W,
                                                       const double *__restrict__ sc, int slot,
                                                       const int8_t *__restrict__ active, const int32_t *__restrict__ lc,
                                                       float *__restrict__ st, int64_t st_rows) {
    static_assert(RED_BLOCK % NR == 0, "block size must be a multiple of the column count");
    mds_pdl_entry();
    Chunk k = ch[lc ? lc[blockIdx.x] : blockIdx.x];  // lc: the live chunks only
    if (chunk_skipped<NR>(active, k.inst)) return;  // a finished instance: its rows are no longer used
    const int64_t p = (int64_t)k.inst * NR + threadIdx.x % NR;
    const double f = active[p] ? sc[p * 8 + slot] : 0.0;
    double *w = W + k.b * NR;
    const int64_t m = (k.e - k.b) * NR;
    // entries of this chunk that are also staged in FP32
    const int64_t ms = st ? (st_rows > k.e ? m : st_rows > k.b ? (st_rows - k.b) * NR : 0) : 0;
    float *s = st ? st + k.b * NR : nullptr;
    constexpr int B = RED_BLOCK;
    int64_t i = threadIdx.x;
    for (; i + 3 * B < m; i += 4 * B) {
        const double a0 = w[i], a1 = w[i + B], a2 = w[i + 2 * B], a3 = w[i + 3 * B];
        const double v0 = f == 0.0 ? 0.0 : a0 * f, v1 = f == 0.0 ? 0.0 : a1 * f, v2 = f == 0.0 ? 0.0 : a2 * f,
                     v3 = f == 0.0 ? 0.0 : a3 * f;
        w[i] = v0;
        w[i + B] = v1;
        w[i + 2 * B] = v2;
        w[i + 3 * B] = v3;
        if (i + 3 * B < ms) {
            s[i] = d2f_int(v0);
            s[i + B] = d2f_int(v1);
            s[i + 2 * B] = d2f_int(v2);
            s[i + 3 * B] = d2f_int(v3);
        } else if (i < ms) {
            s[i] = d2f_int(v0);
            if (i + B < ms) s[i + B] = d2f_int(v1);
            if (i + 2 * B < ms) s[i + 2 * B] = d2f_int(v2);
        }
    }
    for (; i < m; i += B) {
        const double v = f == 0.0 ? 0.0 : w[i] * f;
        w[i] = v;
        if (i < ms) s[i] = d2f_int(v);
    }
}

// per problem: beta = sqrt(nsq), g = (beta, 0, ...), sc[1] = 1/beta
__global__ void k_bcycle_start(int P, const double *__restrict__ nsq, int m, double *__restrict__ g,
                               double *__restrict__ sc) {
    mds_pdl_entry();
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    double beta = sqrt(nsq[(int64_t)p * 32]);
    sc[p * 8 + 0] = beta;
    sc[p * 8 + 1] = beta > 0.0 ? 1.0 / beta : 0.0;
    g[p * 32] = beta;
    for (int q = 1; q <= m; q++) g[p * 32 + q] = 0.0;
}

// per active problem: Hessenberg column j from h1 + h2 and ||w||, rotations,
// g; sc[2] = |g_{j+1}|, sc[3] = 1/H[j+1][j], sc[4] = breakdown (1 lucky, 2 bad)
__global__ void k_barnoldi(int P, int j, int m, const int8_t *__restrict__ active, double *__restrict__ H,
                           const double *__restrict__ h1, const double *__restrict__ h2,
                           const double *__restrict__ nsq, double *__restrict__ cs, double *__restrict__ sn,
                           double *__restrict__ g, double *__restrict__ sc) {
    mds_pdl_entry();
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P || !active[p]) return;
    double *Hp = H + (int64_t)p * (m + 1) * m;
    const double *a1 = h1 + (int64_t)p * 32, *a2 = h2 + (int64_t)p * 32;
    double *c_ = cs + (int64_t)p * 32, *s_ = sn + (int64_t)p * 32, *gp = g + (int64_t)p * 32, *scp = sc + p * 8;
    for (int q = 0; q <= j; q++) Hp[q * m + j] = a1[q] + a2[q];
    double hn = sqrt(nsq[(int64_t)p * 32]);
    Hp[(j + 1) * m + j] = hn;
    for (int q = 0; q < j; q++) {
        double a = Hp[q * m + j], c = Hp[(q + 1) * m + j];
        Hp[q * m + j] = c_[q] * a + s_[q] * c;
        Hp[(q + 1) * m + j] = -s_[q] * a + c_[q] * c;
    }
    double a = Hp[j * m + j], c = Hp[(j + 1) * m + j];
    double rr = sqrt(a * a + c * c);
    c_[j] = rr == 0.0 ? 1.0 : a / rr;
    s_[j] = rr == 0.0 ? 0.0 : c / rr;
    Hp[j * m + j] = rr;
    Hp[(j + 1) * m + j] = 0.0;
    gp[j + 1] = -s_[j] * gp[j];
    gp[j] = c_[j] * gp[j];
    scp[2] = fabs(gp[j + 1]);
    bool bad = !(hn > 0.0) || !isfinite(hn) || !isfinite(rr);
    scp[3] = bad ? 0.0 : 1.0 / hn;
    scp[4] = !isfinite(hn) || !isfinite(rr) ? 2.0 : (hn == 0.0 ? 1.0 : 0.0);
}

// per problem: solve H y = g with its own step count kdone[p]; y zero beyond
__global__ void k_bbacksolve(int P, const int32_t *__restrict__ kdone, int m, const double *__restrict__ H,
                             const double *__restrict__ g, double *__restrict__ y) {
    mds_pdl_entry();
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    int k = kdone[p];
    const double *Hp = H + (int64_t)p * (m + 1) * m;
    const double *gp = g + (int64_t)p * 32;
    double *yp = y + (int64_t)p * 32;
    for (int q = 0; q < 32; q++) yp[q] = 0.0;
    for (int q = k - 1; q >= 0; q--) {
        double s = gp[q];
        for (int t = q + 1; t < k; t++) s -= Hp[q * m + t] * yp[t];
        yp[q] = Hp[q * m + q] == 0.0 ? 0.0 : s / Hp[q * m + q];
    }
}

// interleave NR columns of a column-major [ncol][N] array / scatter back,
// RED_BLOCK rows per block through shared memory, so that both the column
// runs and the interleaved rows move in whole contiguous segments (the
// column-major side may be page-locked host memory read or written in place)
constexpr int IL_PAD = 1;  // shared row stride NR + 1: conflict-free column walks
template <int NR>
__global__ void __launch_bounds__(RED_BLOCK) k_to_interleaved(int64_t N, const double *__restrict__ src, int c0,
                                                              double *__restrict__ dst) {
    __shared__ double t[RED_BLOCK * (NR + IL_PAD)];
    mds_pdl_entry();
    const int64_t nb = (N + RED_BLOCK - 1) / RED_BLOCK;
    for (int64_t blk = blockIdx.x; blk < nb; blk += gridDim.x) {
        const int64_t r0 = blk * RED_BLOCK, rows = N - r0 < RED_BLOCK ? N - r0 : RED_BLOCK;
        if ((int64_t)threadIdx.x < rows)
#pragma unroll
            for (int c = 0; c < NR; c++) t[threadIdx.x * (NR + IL_PAD) + c] = src[(int64_t)(c0 + c) * N + r0 + threadIdx.x];
        __syncthreads();
        for (int e = threadIdx.x; e < rows * NR; e += RED_BLOCK)
            dst[r0 * NR + e] = t[(e / NR) * (NR + IL_PAD) + e % NR];
        __syncthreads();
    }
}
template <int NR>
__global__ void __launch_bounds__(RED_BLOCK) k_from_interleaved(int64_t N, const double *__restrict__ src, int c0,
                                                                double *__restrict__ dst) {
    __shared__ double t[RED_BLOCK * (NR + IL_PAD)];
    mds_pdl_entry();
    const int64_t nb = (N + RED_BLOCK - 1) / RED_BLOCK;
    for (int64_t blk = blockIdx.x; blk < nb; blk += gridDim.x) {
        const int64_t r0 = blk * RED_BLOCK, rows = N - r0 < RED_BLOCK ? N - r0 : RED_BLOCK;
        for (int e = threadIdx.x; e < rows * NR; e += RED_BLOCK) t[(e / NR) * (NR + IL_PAD) + e % NR] = src[r0 * NR + e];
        __syncthreads();
        if ((int64_t)threadIdx.x < rows)
#pragma unroll
            for (int c = 0; c < NR; c++) dst[(int64_t)(c0 + c) * N + r0 + threadIdx.x] = t[threadIdx.x * (NR + IL_PAD) + c];
        __syncthreads();
    }
}

template <int NR>
static void fgmres_group(Ctx &c, const mds_csr &A, const BatchPrecFn &M, const std::vector<int64_t> &moff,
                         const std::vector<int64_t> &foff, const double *Bcol, double *Xcol, int c0,
                         const mds_solve_opts &o, std::vector<KrylovResult> &out) {
    const int K = (int)moff.size() - 1;
    const int64_t NM = moff[K], N = NM + foff[K];
    const int P = K * NR;
    const int m = o.restart < 1 ? 1 : (o.restart > QMAX - 1 ? QMAX - 1 : o.restart);
    // chunks of at most CH rows, never crossing an instance's segment
    int64_t CH = std::max<int64_t>(1024, std::min<int64_t>(16384, N / (4 * 152) + 1));
    std::vector<Chunk> chunks;
    std::vector<std::vector<int32_t>> per(K);
    auto add = [&](int64_t b, int64_t e, int k) {
        for (int64_t s = b; s < e; s += CH) {
            per[k].push_back((int32_t)chunks.size());
            chunks.push_back(Chunk{s, std::min(e, s + CH), k});
        }
    };
    for (int k = 0; k < K; k++) add(moff[k], moff[k + 1], k);
    for (int k = 0; k < K; k++) add(NM + foff[k], NM + foff[k + 1], k);
    std::vector<int32_t> ioff(K + 1, 0), ilist;
    for (int k = 0; k < K; k++) {
        ioff[k + 1] = ioff[k] + (int32_t)per[k].size();
        ilist.insert(ilist.end(), per[k].begin(), per[k].end());
    }
    const int nch = (int)chunks.size();
    Buf dch(&c, sizeof(Chunk) * chunks.size()), dioff(&c, sizeof(int32_t) * ioff.size()),
        dil(&c, sizeof(int32_t) * (ilist.size() ? ilist.size() : 1));
    MDS_CUDA(cudaMemcpyAsync(dch.p, chunks.data(), sizeof(Chunk) * chunks.size(), cudaMemcpyHostToDevice, c.stream));
    MDS_CUDA(cudaMemcpyAsync(dioff.p, ioff.data(), sizeof(int32_t) * ioff.size(), cudaMemcpyHostToDevice, c.stream));
    if (ilist.size())
        MDS_CUDA(cudaMemcpyAsync(dil.p, ilist.data(), sizeof(int32_t) * ilist.size(), cudaMemcpyHostToDevice, c.stream));
    const Chunk *CHp = dch.as<Chunk>();
    const int32_t *IO = dioff.as<int32_t>(), *IL = dil.as<int32_t>();
    // Finer chunks (2,048 rows) for the kernels whose block walks a chunk's
    // rows for every basis vector (the Gram-Schmidt update, the x update, the
    // scaling and the squared norms): once most instances have finished, the
    // few live ones still spread over many blocks.
    constexpr int64_t CHF = 2048;
    std::vector<Chunk> fchunks;
    std::vector<std::vector<int32_t>> fper(K);
    auto fadd = [&](int64_t b, int64_t e, int k) {
        for (int64_t s = b; s < e; s += CHF) {
            fper[k].push_back((int32_t)fchunks.size());
            fchunks.push_back(Chunk{s, std::min(e, s + CHF), k});
        }
    };
    for (int k = 0; k < K; k++) fadd(moff[k], moff[k + 1], k);
    for (int k = 0; k < K; k++) fadd(NM + foff[k], NM + foff[k + 1], k);
    std::vector<int32_t> fioff(K + 1, 0), filist;
    for (int k = 0; k < K; k++) {
        fioff[k + 1] = fioff[k] + (int32_t)fper[k].size();
        filist.insert(filist.end(), fper[k].begin(), fper[k].end());
    }
    const int nchf = (int)fchunks.size();
    Buf dchf(&c, sizeof(Chunk) * fchunks.size()), dfioff(&c, sizeof(int32_t) * fioff.size()),
        dfil(&c, sizeof(int32_t) * (filist.size() ? filist.size() : 1));
    MDS_CUDA(cudaMemcpyAsync(dchf.p, fchunks.data(), sizeof(Chunk) * fchunks.size(), cudaMemcpyHostToDevice, c.stream));
    MDS_CUDA(cudaMemcpyAsync(dfioff.p, fioff.data(), sizeof(int32_t) * fioff.size(), cudaMemcpyHostToDevice, c.stream));
    if (filist.size())
        MDS_CUDA(cudaMemcpyAsync(dfil.p, filist.data(), sizeof(int32_t) * filist.size(), cudaMemcpyHostToDevice,
                                 c.stream));
    const Chunk *CHFp = dchf.as<Chunk>();
    const int32_t *IOF = dfioff.as<int32_t>(), *ILF = dfil.as<int32_t>();

    const int64_t ld = (N + 63) / 64 * 64, ldq = ld * NR;
    Buf Bi(&c, sizeof(double) * (size_t)(N * NR)), Xi(&c, sizeof(double) * (size_t)(N * NR));
    Buf V(&c, sizeof(double) * (size_t)(m + 1) * ldq), Z(&c, sizeof(double) * (size_t)m * ldq);
    Buf H(&c, sizeof(double) * (size_t)P * (m + 1) * m);
    Buf part(&c, sizeof(double) * (size_t)(std::max<int64_t>((int64_t)QMAX * nch, nchf) * NR));
    // per-problem arrays with stride 32: cs, sn, g, y, h1, h2, nsq; scalars stride 8
    Buf pa(&c, sizeof(double) * (size_t)P * 32 * 7), psc(&c, sizeof(double) * (size_t)P * 8);
    // act: P problem flags, then K instance flags (an instance is live while
    // one of its columns iterates; the kernels skip the rows of the others)
    Buf act(&c, (size_t)(P + K)), kd(&c, sizeof(int32_t) * (size_t)P), f2(&c, (size_t)P);
    const int8_t *ilive = act.as<int8_t>() + P;
    LiveMap sysmap;
    Buf sys_ck, sys_rt;
    // the chunks (coarse and fine) of the live instances, for the compacted
    // Gram-Schmidt, scaling and update launches
    struct LiveChunks {
        Ctx &c;
        const std::vector<Chunk> &coarse, &fine;
        Buf dcoarse, dfine;
        int64_t nc = 0, nf = 0;
        bool on = false;
        void build(const std::vector<int8_t> &live) {
            std::vector<int32_t> a, b;
            for (size_t i = 0; i < coarse.size(); i++)
                if (live[coarse[i].inst]) a.push_back((int32_t)i);
            for (size_t i = 0; i < fine.size(); i++)
                if (live[fine[i].inst]) b.push_back((int32_t)i);
            // never empty: chunk 0 stands in, and the kernels' masks skip it
            if (a.empty()) a.push_back(0);
            if (b.empty()) b.push_back(0);
            if (!dcoarse.p) dcoarse = Buf(&c, sizeof(int32_t) * (coarse.size() + 1));
            if (!dfine.p) dfine = Buf(&c, sizeof(int32_t) * (fine.size() + 1));
            MDS_CUDA(cudaMemcpyAsync(dcoarse.p, a.data(), sizeof(int32_t) * a.size(), cudaMemcpyHostToDevice, c.stream));
            MDS_CUDA(cudaMemcpyAsync(dfine.p, b.data(), sizeof(int32_t) * b.size(), cudaMemcpyHostToDevice, c.stream));
            nc = (int64_t)a.size();
            nf = (int64_t)b.size();
            on = true;
        }
        const int32_t *lcoarse() const { return on ? dcoarse.as<int32_t>() : nullptr; }
        const int32_t *lfine() const { return on ? dfine.as<int32_t>() : nullptr; }
        int64_t ncoarse(int64_t all) const { return on ? nc : all; }
        int64_t nfine(int64_t all) const { return on ? nf : all; }
    } cl{c, chunks, fchunks};
    if (K > 1) {
        sys_ck = live_chunks(c, N, moff, &foff, NM);
        sysmap.ck = sys_ck.as<int32_t>();
        sysmap.live = ilive;
    }
    // the batched preconditioner's kernels read the instance flags from the
    // context while this solve runs
    struct LiveScope {
        Ctx &c;
        LiveScope(Ctx &cc, const int8_t *l) : c(cc) { c.live = l; }
        ~LiveScope() {
            c.live = nullptr;
            c.live_host.clear();
            c.compact = false;
        }
    } live_scope(c, K > 1 ? ilive : nullptr);
    double *cs = pa.as<double>(), *sn = cs + (size_t)P * 32, *g = sn + (size_t)P * 32, *y = g + (size_t)P * 32,
           *h1 = y + (size_t)P * 32, *h2 = h1 + (size_t)P * 32, *nsq = h2 + (size_t)P * 32;
    double *sc = psc.as<double>();
    double *Vp = V.as<double>(), *Zp = Z.as<double>(), *PT = part.as<double>();
    MDS_CUDA(cudaMemsetAsync(pa.p, 0, pa.bytes, c.stream));
    MDS_CUDA(cudaMemsetAsync(psc.p, 0, psc.bytes, c.stream));
    unsigned eg = red_grid(N * NR);
    MDS_LAUNCH(c, KC_NONE, 16.0 * N * NR, (k_to_interleaved<NR>), eg, RED_BLOCK, 0, N, Bcol, c0, Bi.as<double>());
    if (o.x0_zero)  // the zero initial guess: X is output only
        MDS_CUDA(cudaMemsetAsync(Xi.p, 0, sizeof(double) * (size_t)(N * NR), c.stream));
    else
        MDS_LAUNCH(c, KC_NONE, 16.0 * N * NR, (k_to_interleaved<NR>), eg, RED_BLOCK, 0, N, Xcol, c0, Xi.as<double>());
    dim3 pgrid((unsigned)P, 1);
    // per-problem squared norms of a vector into nsq[p * 32]
    auto norms = [&](const double *w, const int8_t *mk) {
        MDS_LAUNCH(c, KC_NONE, 8.0 * N * NR, (k_bdot<NR>), (unsigned)(mk ? cl.nfine(nchf) : nchf), RED_BLOCK, 0, CHFp, nchf, Vp,
                   ldq, 0, w, PT, mk, mk ? cl.lfine() : nullptr);
        MDS_LAUNCH(c, KC_NONE, 0, k_breduce, dim3(P, 1), 32, 0, PT, nchf, 1, NR, IOF, ILF, P, nsq, 0, mk);
    };
    // upload the problem flags hact and the instance flags derived from them
    std::vector<int8_t> hbuf(P + K);
    auto upload_flags = [&](const std::vector<int8_t> &h) {
        for (int p = 0; p < P; p++) hbuf[p] = h[p];
        for (int k = 0; k < K; k++) {
            int8_t a = 0;
            for (int q = 0; q < NR; q++) a |= h[(size_t)k * NR + q];
            hbuf[P + k] = a;
        }
        std::memcpy(c.h_pin, hbuf.data(), (size_t)(P + K));
        MDS_CUDA(cudaMemcpyAsync(act.p, c.h_pin, (size_t)(P + K), cudaMemcpyHostToDevice, c.stream));
        if (K > 1) {
            const bool changed = c.live_host.size() != (size_t)K ||
                                 !std::equal(c.live_host.begin(), c.live_host.end(), hbuf.begin() + P);
            c.live_host.assign(hbuf.begin() + P, hbuf.end());
            int64_t r = 0;
            int nlive = 0;
            for (int k = 0; k < K; k++)
                if (hbuf[P + k]) {
                    r += (moff[k + 1] - moff[k]) + (foff[k + 1] - foff[k]);
                    nlive++;
                }
            sysmap.frac = N > 0 ? (double)r / (double)N : 1.0;
            // compacted launches once an instance has finished
            c.compact = nlive < K;
            if (changed) c.live_ver++;
            if (c.compact && changed) {
                std::vector<int64_t> t;
                sysmap.nch = live_ranges(c.live_host, moff, &foff, NM, t);
                upload_ranges(c, sys_rt, t, K);
                sysmap.rt = sys_rt.as<int64_t>();
                cl.build(c.live_host);
            }
            if (!c.compact) {
                sysmap.rt = nullptr;
                sysmap.nch = -1;
                cl.on = false;
            }
        }
    };
    std::vector<double> host(P * 8), bn(P);
    auto fetch = [&](const double *d, int stride, int slot) {
        MDS_CUDA(cudaMemcpyAsync(c.h_pin, d, sizeof(double) * (size_t)P * stride, cudaMemcpyDeviceToHost, c.stream));
        c.sync();
        const double *hp = static_cast<const double *>(c.h_pin);
        std::vector<double> v(P);
        for (int p = 0; p < P; p++) v[p] = hp[(size_t)p * stride + slot];
        return v;
    };
    MDS_REQUIRE((size_t)P * 32 * sizeof(double) <= Ctx::PIN_BYTES, MDS_ERR_INVALID,
                "too many batched problems (instances x columns > 4096)");
    c.live = nullptr;  // b and the first residual: every row
    norms(Bi.as<double>(), nullptr);
    {
        std::vector<double> b2 = fetch(nsq, 32, 0);
        for (int p = 0; p < P; p++) {
            bn[p] = std::sqrt(b2[p]);
            if (!std::isfinite(bn[p])) out[p].status = MDS_ERR_NONFINITE;
            if (bn[p] == 0.0) bn[p] = 1.0;
        }
    }
    std::vector<int> it(P, 0), rs(P, 0), done(P, 0);
    std::vector<double> est(P, 0.0);
    for (int p = 0; p < P; p++)
        if (out[p].status == MDS_ERR_NONFINITE) done[p] = 1;
    std::vector<int8_t> hact(P);
    std::vector<int32_t> hkd(P);
    // One lockstep Arnoldi step j of every problem: z_j = M v_j, w = A z_j,
    // the Gram-Schmidt passes (the second one masked to the flagged
    // problems), the Arnoldi / Givens update and the scaled v_{j+1}, and the
    // step's scalars copied to pinned host memory.  The kernels read the
    // problem and instance flags from device memory, so the sequence of
    // launches of step j does not change between restart cycles: it is
    // captured as a CUDA graph on its second use (the first one grows the
    // preconditioner's work vectors) and replayed.
    auto step_body = [&](int j) {
        double *vj = Vp + (size_t)j * ldq, *zj = Zp + (size_t)j * ldq, *w = Vp + (size_t)(j + 1) * ldq;
        M(vj, zj, NR);
        spmv_f64(c, A, zj, w, KC_SPMV, NR, sysmap);
        int nq = j + 1;
        const double sf = sysmap.frac;  // share of the rows of live instances
        double fl = 2.0 * (double)N * NR * nq * sf;
        // classical Gram-Schmidt for every problem; the second pass runs
        // for the problems whose first pass cancelled severely (the
        // others' chunks return at once)
        for (int pass = 0; pass < 2; pass++) {
            double *hh = pass == 0 ? h1 : h2;
            // first pass: the active problems' instances; second: the flagged problems'
            const int8_t *mk = pass == 0 ? act.as<int8_t>() : f2.as<int8_t>();
            int kd = pass == 0 ? KC_GS_DOT : KC_NONE, ka = pass == 0 ? KC_GS_AXPY : KC_NONE;
            MDS_LAUNCH_F(c, kd, 8.0 * N * NR * (nq + 1) * sf, fl, (k_bdot<NR>), (unsigned)((int64_t)cl.ncoarse(nch) * nq),
                         RED_BLOCK, 0, CHp, nch, Vp, ldq, nq, w, PT, mk, cl.lcoarse());
            MDS_LAUNCH(c, KC_NONE, 0, k_breduce, dim3(P, nq), 32, 0, PT, nch, nq, NR, IO, IL, P, hh, 0, mk);
            MDS_LAUNCH_F(c, ka, 8.0 * N * NR * (nq + 2) * sf, fl, (k_bmaxpy<NR, -1>), (unsigned)cl.nfine(nchf), RED_BLOCK, 0,
                         CHFp, Vp, ldq, nq, hh, w, PT, mk, (const int32_t *)nullptr, cl.lfine());
            MDS_LAUNCH(c, KC_NONE, 0, k_breduce, dim3(P, 1), 32, 0, PT, nchf, 1, NR, IOF, ILF, P, nsq, 0, mk);
            if (pass == 0)
                MDS_LAUNCH(c, KC_NONE, 0, k_bflag, grid_for(P, 128), 128, 0, P, nq, act.as<int8_t>(), h1, nsq,
                           o.reorth_eta2, f2.as<int8_t>(), h2);
        }
        MDS_LAUNCH(c, KC_NONE, 0, k_barnoldi, grid_for(P, 128), 128, 0, P, j, m, act.as<int8_t>(), H.as<double>(),
                   h1, h2, nsq, cs, sn, g, sc);
        MDS_LAUNCH(c, KC_NONE, 16.0 * N * NR + 4.0 * c.in_stage_rows * NR, k_bscale<NR>, (unsigned)cl.nfine(nchf),
                   RED_BLOCK, 0, CHFp, w, sc, 3,
                   act.as<int8_t>(), cl.lfine(), c.in_stage, c.in_stage_rows);
        MDS_CUDA(cudaMemcpyAsync(c.h_pin, sc, sizeof(double) * (size_t)P * 8, cudaMemcpyDeviceToHost, c.stream));
    };
    std::vector<std::unique_ptr<Graph>> graphs(m);
    bool graphs_ok = o.graphs != 0, warmed = false;
    auto run_step = [&](int j) {
        Graph *gj = nullptr;
        // graphs while every instance iterates; compacted direct launches
        // (grids sized to the live chunks) once some have finished
        if (graphs_ok && warmed && !c.compact) {
            auto &slot = graphs[j];
            if (!slot) {
                slot.reset(new Graph);
                slot->cap_share = sysmap.frac;
                if (!graph_capture(c, *slot, [&] { step_body(j); })) {
                    slot.reset();
                    graphs_ok = false;
                }
            }
            gj = slot.get();
        }
        if (gj) {
            gj->scale = gj->cap_share > 0.0 ? sysmap.frac / gj->cap_share : 1.0;
            graph_launch(c, *gj);
        } else {
            step_body(j);
        }
        warmed = true;
        c.sync();
        if (gj) graph_collect(c, *gj);
    };
    bool first_cycle = true;
    for (;;) {
        // V0 = B - A X for the problems not yet done
        const int8_t *mk = nullptr;
        if (!first_cycle && K > 1) {
            for (int p = 0; p < P; p++) hact[p] = done[p] ? 0 : 1;
            upload_flags(hact);
            c.live = ilive;
            mk = act.as<int8_t>();
        }
        spmv_sub_f64(c, A, Bi.as<double>(), Xi.as<double>(), Vp, NR, mk ? sysmap : LiveMap{});
        norms(Vp, mk);
        first_cycle = false;
        std::vector<double> r2 = fetch(nsq, 32, 0);
        bool any = false;
        for (int p = 0; p < P; p++) {
            if (done[p]) continue;
            est[p] = std::sqrt(r2[p]) / bn[p];
            if (!std::isfinite(est[p])) {
                out[p].status = MDS_ERR_NONFINITE;
                done[p] = 1;
            } else if (est[p] <= o.rtol) {
                out[p].status = MDS_OK;
                done[p] = 1;
            } else if (it[p] >= o.max_iters) {
                out[p].status = MDS_WARN_NOT_CONVERGED;
                done[p] = 1;
            } else {
                any = true;
            }
        }
        if (!any) break;
        for (int p = 0; p < P; p++) {
            hact[p] = done[p] ? 0 : 1;
            hkd[p] = 0;
        }
        upload_flags(hact);
        if (K > 1) c.live = ilive;
        MDS_LAUNCH(c, KC_NONE, 0, k_bcycle_start, grid_for(P, 128), 128, 0, P, nsq, m, g, sc);
        MDS_LAUNCH(c, KC_NONE, 16.0 * N * NR + 4.0 * c.in_stage_rows * NR, k_bscale<NR>, (unsigned)cl.nfine(nchf),
                   RED_BLOCK, 0, CHFp, Vp, sc, 1,
                   act.as<int8_t>(), cl.lfine(), c.in_stage, c.in_stage_rows);
        for (int j = 0; j < m; j++) {
            if (j > 0) upload_flags(hact);
            run_step(j);
            const double *hp = static_cast<const double *>(c.h_pin);
            bool live = false;
            for (int p = 0; p < P; p++) {
                if (!hact[p]) continue;
                it[p]++;
                hkd[p] = j + 1;
                est[p] = hp[p * 8 + 2] / bn[p];
                bool bad = hp[p * 8 + 4] == 2.0 || !std::isfinite(est[p]);
                if (bad) {
                    out[p].status = MDS_ERR_BREAKDOWN;
                    done[p] = 1;
                    hact[p] = 0;
                    hkd[p] = 0;  // keep x as it was at the cycle start
                } else if (est[p] <= o.rtol || it[p] >= o.max_iters || hp[p * 8 + 4] == 1.0) {
                    hact[p] = 0;
                }
                live = live || hact[p];
            }
            if (!live) break;
        }
        std::memcpy(c.h_pin, hkd.data(), sizeof(int32_t) * (size_t)P);
        MDS_CUDA(cudaMemcpyAsync(kd.p, c.h_pin, sizeof(int32_t) * (size_t)P, cudaMemcpyHostToDevice, c.stream));
        MDS_LAUNCH(c, KC_NONE, 0, k_bbacksolve, grid_for(P, 128), 128, 0, P, kd.as<int32_t>(), m, H.as<double>(), g, y);
        // every chunk: the problems that finished during this cycle are no
        // longer live but still take their update (qlim = their step count)
        MDS_LAUNCH(c, KC_NONE, 8.0 * N * NR * (m + 2), (k_bmaxpy<NR, 1>), nchf, RED_BLOCK, 0, CHFp, Zp, ldq, m, y,
                   Xi.as<double>(), nullptr, (const int8_t *)nullptr, kd.as<int32_t>(), (const int32_t *)nullptr);
        for (int p = 0; p < P; p++)
            if (hkd[p] > 0) rs[p]++;
    }
    // true residuals at exit (every row)
    c.live = nullptr;
    spmv_sub_f64(c, A, Bi.as<double>(), Xi.as<double>(), Vp, NR);
    norms(Vp, nullptr);
    std::vector<double> r2 = fetch(nsq, 32, 0);
    for (int p = 0; p < P; p++) {
        out[p].iterations = it[p];
        out[p].restarts = rs[p];
        out[p].relres_est = est[p];
        out[p].relres_true = std::sqrt(r2[p]) / bn[p];
    }
    MDS_LAUNCH(c, KC_NONE, 16.0 * N * NR, (k_from_interleaved<NR>), eg, RED_BLOCK, 0, N, Xi.as<double>(), c0, Xcol);
    c.sync();
}

void fgmres_batched(Ctx &c, const mds_csr &A, const BatchPrecFn &M, const std::vector<int64_t> &moff,
                    const std::vector<int64_t> &foff, const double *B, double *X, int nrhs, const mds_solve_opts &o,
                    std::vector<KrylovResult> &res) {
    const int K = (int)moff.size() - 1;
    res.assign((size_t)K * nrhs, KrylovResult());
    int c0 = 0;
    while (c0 < nrhs) {
        int left = nrhs - c0;
        int NR = left >= 8 ? 8 : left >= 4 ? 4 : left >= 2 ? 2 : 1;
        std::vector<KrylovResult> part((size_t)K * NR);
        switch (NR) {
            case 8: fgmres_group<8>(c, A, M, moff, foff, B, X, c0, o, part); break;
            case 4: fgmres_group<4>(c, A, M, moff, foff, B, X, c0, o, part); break;
            case 2: fgmres_group<2>(c, A, M, moff, foff, B, X, c0, o, part); break;
            default: fgmres_group<1>(c, A, M, moff, foff, B, X, c0, o, part); break;
        }
        for (int k = 0; k < K; k++)
            for (int cc = 0; cc < NR; cc++) res[(size_t)k * nrhs + c0 + cc] = part[(size_t)k * NR + cc];
        c0 += NR;
    }
}

}  // namespace mds
