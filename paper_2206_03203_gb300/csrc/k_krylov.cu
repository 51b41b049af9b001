// Krylov solvers in FP64: right-preconditioned flexible GMRES(m) with
// classical Gram-Schmidt applied twice (CGS2) and device-side Givens
// rotations, and preconditioned conjugate gradients.  Sec. 3.2 studies the
// right-preconditioned operator A B_L; Sec. 4 fixes x0 = 0 and a relative-
// residual stopping rule.  All reductions are two-stage with a fixed order,
// so results are run-to-run reproducible.
#include <cmath>
#include <functional>
#include <memory>
#include <mutex>

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

// partial[q][blk] = sum over this block's rows of V[q][i] w[i]; grid.y = q.
// One dot product per block row keeps registers low; w is re-read once per q
// and stays resident in L2, V is read once from HBM.
__global__ void __launch_bounds__(RED_BLOCK) k_mdot(int64_t n, const double *__restrict__ V, int64_t ldv, int nq,
                                                     const double *__restrict__ w, double *__restrict__ partial,
                                                     const double *__restrict__ run_flag) {
    if (run_flag && *run_flag == 0.0) return;
    __shared__ double ws[RED_BLOCK / 32];
    // rows of V are 16-byte aligned (ldv even); w is a row of V
    const double *v = (int)blockIdx.y < nq ? V + (int64_t)blockIdx.y * ldv : w;
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
    double s = s0 + s1;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < RED_BLOCK / 32; k++) t += ws[k];
        partial[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = t;
    }
}

// out[q] (+)= sum_b partial[q][b], one warp per q, fixed order
__global__ void k_reduce_rows(const double *__restrict__ partial, int nblk, int nq, double *__restrict__ out,
                              int accumulate, const double *__restrict__ run_flag) {
    if (run_flag && *run_flag == 0.0) return;
    int q = blockIdx.x;
    if (q >= nq) return;
    double s = 0.0;
    for (int b = threadIdx.x; b < nblk; b += 32) s += partial[(int64_t)q * nblk + b];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) out[q] = accumulate ? out[q] + s : s;
}

// out[q] (+)= sum over blocks of partial[blk][q] (stride QMAX); one warp per q,
// fixed order
__global__ void k_reduce_cols(const double *__restrict__ partial, int nblk, int nq, double *__restrict__ out,
                              int accumulate) {
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
    double s = *f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        o[i] = w[i] * s;
}

// scal[0] = beta = sqrt(normsq); g = (beta, 0, ...); scal[1] = 1/beta
__global__ void k_cycle_start(const double *__restrict__ normsq, double *__restrict__ g, int m,
                              double *__restrict__ scal) {
    double beta = sqrt(normsq[0]);
    scal[0] = beta;
    scal[1] = beta > 0.0 ? 1.0 / beta : 0.0;
    g[0] = beta;
    for (int q = 1; q <= m; q++) g[q] = 0.0;
}

// DGKS test after the first Gram-Schmidt pass: reorthogonalise when the
// projection removed more than half of ||w||^2 (||w_new|| < ||w|| / sqrt(2)).
// flag[0] = 1 to run the second pass; the second-pass coefficients start at 0.
__global__ void k_dgks(const double *__restrict__ nsq_before, const double *__restrict__ nsq_after,
                       double *__restrict__ flag, double *__restrict__ h2, int nq) {
    double run = (nsq_after[0] < 0.5 * nsq_before[0]) ? 1.0 : 0.0;
    flag[0] = run;
    for (int q = 0; q < nq; q++) h2[q] = 0.0;
}

// Arnoldi column j: H[0..j][j] = h1 + h2, H[j+1][j] = ||w|| (after the second
// pass when it ran); apply the previous rotations, form the new one, update
// g.  scal[2] = |g_{j+1}|, scal[3] = 1/H[j+1][j] (0 on breakdown), scal[4] =
// breakdown flag (1 lucky, 2 non-finite).
__global__ void k_arnoldi(int j, int m, double *__restrict__ H, const double *__restrict__ h,
                          const double *__restrict__ h2, const double *__restrict__ nsq1,
                          const double *__restrict__ nsq2, const double *__restrict__ flag, double *__restrict__ cs,
                          double *__restrict__ sn, double *__restrict__ g, double *__restrict__ scal) {
    bool two = flag[0] != 0.0;
    for (int q = 0; q <= j; q++) H[q * m + j] = two ? h[q] + h2[q] : h[q];
    double hn = sqrt(two ? nsq2[0] : nsq1[0]);
    H[(j + 1) * m + j] = hn;
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
    scal[2] = fabs(g[j + 1]);
    bool bad = !(hn > 0.0) || !isfinite(hn) || !isfinite(rr);
    scal[3] = bad ? 0.0 : 1.0 / hn;
    scal[4] = !isfinite(hn) || !isfinite(rr) ? 2.0 : (hn == 0.0 ? 1.0 : 0.0);
    scal[5] += two ? 1.0 : 0.0;
}

// upper-triangular solve H y = g (k columns)
__global__ void k_backsolve(int k, int m, const double *__restrict__ H, const double *__restrict__ g,
                            double *__restrict__ y) {
    for (int q = k - 1; q >= 0; q--) {
        double s = g[q];
        for (int p = q + 1; p < k; p++) s -= H[q * m + p] * y[p];
        y[q] = H[q * m + q] == 0.0 ? 0.0 : s / H[q * m + q];
    }
}

// PCG helpers
__global__ void k_pcg_p(int64_t n, const double *__restrict__ z, double *__restrict__ p, const double *__restrict__ sc,
                        int first) {
    double beta = first ? 0.0 : sc[0] / sc[1];  // rz_new / rz
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = first ? z[i] : z[i] + beta * p[i];
}

__global__ void __launch_bounds__(RED_BLOCK) k_pcg_xr(int64_t n, double *__restrict__ x, double *__restrict__ r,
                                                       const double *__restrict__ p, const double *__restrict__ q,
                                                       const double *__restrict__ sc, double *__restrict__ partial) {
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

__global__ void k_copy1(const double *__restrict__ a, double *__restrict__ b) { *b = *a; }

// ---------------------------------------------------------------- host side

struct Red {
    Buf partial;
    double *pp = nullptr;  // the partials buffer in use
    unsigned grid = 1;   // blocks of the single-vector reductions
    unsigned mgrid = 1;  // row blocks per basis vector in k_mdot
};

static unsigned mdot_grid(int64_t n) {
    int64_t g = (n + RED_BLOCK * 16 - 1) / (RED_BLOCK * 16);
    if (g < 1) g = 1;
    if (g > 1024) g = 1024;
    return (unsigned)g;
}

static void dot_dev(Ctx &c, Red &R, int64_t n, const double *a, const double *b, double *out) {
    MDS_LAUNCH(c, KC_NONE, 16.0 * n, k_dot, R.grid, RED_BLOCK, 0, n, a, b, R.pp);
    MDS_LAUNCH(c, KC_NONE, 0, k_reduce_cols, 1, 32, 0, R.pp, (int)R.grid, 1, out, 0);
}

static size_t round256(size_t doubles) { return (doubles + 31) / 32 * 32; }

// Workspace parts in order: reduction partials, V ((m+1) rows), Z (m rows),
// Hessenberg ((m+1) x m), small scalars (256).
size_t fgmres_workspace_doubles(int64_t n, int m) {
    const int64_t ld = (n + 63) / 64 * 64;
    unsigned g = red_grid(n) > mdot_grid(n) ? red_grid(n) : mdot_grid(n);
    return round256((size_t)g * QMAX) + round256((size_t)(m + 1) * ld) + round256((size_t)m * ld) +
           round256((size_t)(m + 1) * m) + 256;
}

FgmresWorkspace fgmres_workspace_carve(double *base, int64_t n, int m) {
    const int64_t ld = (n + 63) / 64 * 64;
    unsigned g = red_grid(n) > mdot_grid(n) ? red_grid(n) : mdot_grid(n);
    FgmresWorkspace w;
    w.partial = base;
    w.V = w.partial + round256((size_t)g * QMAX);
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
    R.mgrid = mdot_grid(n);
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
        R.partial = Buf(&c, sizeof(double) * (size_t)(R.grid > R.mgrid ? R.grid : R.mgrid) * QMAX);
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
    // cs, sn, g, y, h (first CGS pass), h + 32 (second pass), scalars, norms
    double *cs = d, *sn = d + 32, *g = d + 64, *y = d + 96, *h = d + 128, *h2 = d + 160, *scal = d + 192,
           *nsq = d + 224, *nsq2 = d + 225, *dflag = d + 226;
    // ||b||
    dot_dev(c, R, n, b, b, nsq);
    double bn = std::sqrt(c.read(nsq));
    if (!(bn < INFINITY)) {
        res.status = MDS_ERR_NONFINITE;
        return res;
    }
    if (bn == 0.0) bn = 1.0;
    // One Arnoldi step j: z_j = M v_j, w = A z_j, Gram-Schmidt, Givens, and
    // the step's scalars copied to pinned host memory.  Captured as a CUDA
    // graph on first use and replayed on later restart cycles.
    auto body = [&](int j) {
        double *vj = Vp + (size_t)j * ld, *zj = Zp + (size_t)j * ld, *w = Vp + (size_t)(j + 1) * ld;
        M(vj, zj);
        spmv_f64(c, A, zj, w, KC_SPMV);
        // classical Gram-Schmidt: h = V^T w (and ||w||^2), w -= V h, ||w||^2;
        // a second pass only when the DGKS test asks for it (device flag)
        int nq = j + 1;
        double fl = 2.0 * (double)n * nq;
        MDS_LAUNCH_F(c, KC_GS_DOT, 8.0 * n * (nq + 1), fl + 2.0 * n, k_mdot, dim3(R.mgrid, nq + 1), RED_BLOCK, 0, n,
                     Vp, ld, nq, w, R.pp, (const double *)nullptr);
        MDS_LAUNCH(c, KC_NONE, 0, k_reduce_rows, nq + 1, 32, 0, R.pp, (int)R.mgrid, nq + 1, h, 0,
                   (const double *)nullptr);
        MDS_LAUNCH_F(c, KC_GS_AXPY, 8.0 * n * (nq + 2), fl + 2.0 * n, (k_maxpy<-1, true>), R.grid, RED_BLOCK, 0, n,
                     Vp, ld, nq, h, w, R.pp, (const double *)nullptr);
        MDS_LAUNCH(c, KC_NONE, 0, k_reduce_cols, 1, 32, 0, R.pp, (int)R.grid, 1, nsq, 0);
        MDS_LAUNCH(c, KC_NONE, 0, k_dgks, 1, 1, 0, h + nq, nsq, dflag, h2, nq);
        MDS_LAUNCH_F(c, KC_GS_DOT, 8.0 * n * (nq + 1), fl, k_mdot, dim3(R.mgrid, nq), RED_BLOCK, 0, n, Vp, ld, nq, w,
                     R.pp, (const double *)dflag);
        MDS_LAUNCH(c, KC_NONE, 0, k_reduce_rows, nq, 32, 0, R.pp, (int)R.mgrid, nq, h2, 0,
                   (const double *)dflag);
        MDS_LAUNCH_F(c, KC_GS_AXPY, 8.0 * n * (nq + 2), fl + 2.0 * n, (k_maxpy<-1, true>), R.grid, RED_BLOCK, 0, n,
                     Vp, ld, nq, h2, w, R.pp, (const double *)dflag);
        MDS_LAUNCH(c, KC_NONE, 0, k_reduce_cols, 1, 32, 0, R.pp, (int)R.grid, 1, nsq2, 0);
        MDS_LAUNCH(c, KC_NONE, 0, k_arnoldi, 1, 1, 0, j, m, Hp, h, h2, nsq, nsq2, dflag, cs, sn, g, scal);
        MDS_LAUNCH(c, KC_NONE, 16.0 * n, k_scale, red_grid(n), RED_BLOCK, 0, n, w, scal + 3, w);
        MDS_CUDA(cudaMemcpyAsync(c.h_pin, scal, 5 * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    };
    std::vector<std::unique_ptr<Graph>> graphs(m);
    bool graphs_ok = o.graphs != 0;
    auto run_step = [&](int j) {
        Graph *gj = nullptr;
        if (graphs_ok) {
            if (!graphs[j]) {
                graphs[j].reset(new Graph);
                if (!graph_capture(c, *graphs[j], [&] { body(j); })) {
                    graphs[j].reset();
                    graphs_ok = false;
                }
            }
            gj = graphs[j].get();
        }
        if (gj)
            graph_launch(c, *gj);
        else
            body(j);
        c.sync();
        if (gj) graph_collect(c, *gj);
    };
    int it = 0, restarts = 0;
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
            double sv[5];
            std::memcpy(sv, c.h_pin, sizeof sv);
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

// ---------------------------------------------------------------- no-allocation workspace

// Static FGMRES workspace for mds_solve_noalloc: 8 MiB in every device that
// loads the library, enough for n <= MDS_NOALLOC_MAX_N and restart <= 30.
constexpr size_t NOALLOC_DOUBLES = (size_t)MDS_NOALLOC_SCRATCH_BYTES / sizeof(double);
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_DOUBLES];

size_t noalloc_scratch_doubles() { return NOALLOC_DOUBLES; }

// The symbol's device address, looked up once per device with that device
// current (the host-side name is only a stand-in, never a device address).
double *noalloc_scratch(Ctx &c) {
    static std::mutex mu;
    static double *addr[256] = {};
    std::lock_guard<std::mutex> lock(mu);
    MDS_REQUIRE(c.device >= 0 && c.device < 256, MDS_ERR_INVALID, "device index out of range");
    if (!addr[c.device]) {
        MDS_CUDA(cudaSetDevice(c.device));
        void *p = nullptr;
        MDS_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        addr[c.device] = static_cast<double *>(p);
    }
    return addr[c.device];
}

}  // namespace mds
