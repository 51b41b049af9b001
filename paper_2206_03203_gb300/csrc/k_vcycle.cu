// One aggregation-AMG V-cycle (Sec. 3.3: Q_mm and Q_ff of Algorithm 1), and
// the per-level storage it runs on.
//
// Per level, with L1 diagonal D1 and piecewise-constant P:
//   pre-smoothing from zero   x = S(0; b)            (L1-Jacobi or Chebyshev)
//   residual + restriction    b_c = P^T (b - A x)
//   coarse correction         x_c = V(b_c)           (dense inverse on the last level)
//   prolongation + smoothing  y = x + P x_c;  x = S(y; b)
// Storage per level: values in FP64, FP32, or BF16/FP16 with power-of-two
// row scales (a_ij = s_i q_ij, |q_ij| <= 1); matrix in CSR (G lanes per row)
// or SELL-C-sigma (one thread per row, slices of C rows stored column-major,
// rows sorted by length inside windows of sigma rows).
//
// Two kernel forms.  Memory-bound levels (FP32 and below, one L1-Jacobi
// sweep) form D1^-1 b and x + P x_c on the fly at every neighbour, so a level
// costs two matrix passes and the smoothed iterates are never stored.  FP64
// levels are bound by GB300's FP64 pipe, so there the iterates are stored
// once per row instead of being re-formed per nonzero; Chebyshev and
// multi-sweep smoothing also use the stored form.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <map>
#include <tuple>
#include <type_traits>

#include "internal.cuh"

namespace mds {

template <class XT, class VT> __device__ __forceinline__ XT cvt(VT v) { return (XT)v; }
template <> __device__ __forceinline__ float cvt<float, __nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <> __device__ __forceinline__ float cvt<float, __half>(__half v) { return __half2float(v); }

// Device view of one level's operator in its storage format.
template <class VT> struct LvlMat {
    int64_t n;
    const int32_t *rp, *ci;    // CSR
    const VT *v;               // CSR values or SELL values
    const int32_t *sp, *sl;    // SELL slice offsets and lengths
    const int32_t *sc;         // SELL columns
    const int32_t *perm;       // SELL stored row -> original row (NULL: identity)
    int C;                     // SELL slice height
    const float *rscale;       // row scales (NULL: unscaled)
};

// Matrix entries are streamed once per launch: load them evict-first so the
// L1/L2 capacity stays with the gathered vectors.
template <class T> __device__ __forceinline__ T ld_stream(const T *p) { return __ldcs(p); }
template <> __device__ __forceinline__ __nv_bfloat16 ld_stream(const __nv_bfloat16 *p) {
    unsigned short u = __ldcs(reinterpret_cast<const unsigned short *>(p));
    return __ushort_as_bfloat16(u);
}
template <> __device__ __forceinline__ __half ld_stream(const __half *p) {
    unsigned short u = __ldcs(reinterpret_cast<const unsigned short *>(p));
    return __ushort_as_half(u);
}

// NR right-hand sides are stored interleaved: entry (i, c) at i * NR + c, so
// one matrix entry multiplies NR contiguous vector entries (one vector load).
template <class XT, int NR> struct alignas(sizeof(XT) * NR >= 16 ? 16 : sizeof(XT) * NR) Vec {
    XT v[NR];
};
template <class XT, int NR> __device__ __forceinline__ Vec<XT, NR> ldv(const XT *p, int64_t j) {
    return reinterpret_cast<const Vec<XT, NR> *>(p)[j];
}
template <class XT, int NR> __device__ __forceinline__ void stv(XT *p, int64_t j, const Vec<XT, NR> &x) {
    reinterpret_cast<Vec<XT, NR> *>(p)[j] = x;
}

enum { VK_RESID0 = 0, VK_POST = 1, VK_RESID = 2, VK_SMOOTH = 3 };

// Neighbour values each kernel multiplies by a_ij (NR columns at once).
template <class XT, int NR, int K> struct Nb {
    const XT *dinv, *b, *xin, *xc;
    const int32_t *agg;
    __device__ __forceinline__ Vec<XT, NR> operator()(int32_t j) const {
        Vec<XT, NR> y;
        if (K == VK_RESID0 || K == VK_POST) {
            XT d = __ldg(dinv + j);
            Vec<XT, NR> bj = ldv<XT, NR>(b, j);
#pragma unroll
            for (int c = 0; c < NR; c++) y.v[c] = d * bj.v[c];
            if (K == VK_POST && agg) {
                int32_t a = __ldg(agg + j);
                if (a >= 0) {
                    Vec<XT, NR> xa = ldv<XT, NR>(xc, a);
#pragma unroll
                    for (int c = 0; c < NR; c++) y.v[c] += xa.v[c];
                }
            }
        } else {
            y = ldv<XT, NR>(xin, j);
        }
        return y;
    }
};

// Per-row sums over the nonzeros: CSR with G lanes per row (lane-partial
// sums), or SELL with one thread per row (G == 0).
template <int G, class VT, class XT, int NR, class F>
__device__ __forceinline__ void row_sum(const LvlMat<VT> &A, int64_t row, int lane, F f, XT (&s)[NR]) {
    if constexpr (G > 0) {
        int32_t p0 = A.rp[row], p1 = A.rp[row + 1];
#pragma unroll 4
        for (int32_t p = p0 + lane; p < p1; p += G) {
            XT a = cvt<XT>(ld_stream(A.v + p));
            Vec<XT, NR> y = f(ld_stream(A.ci + p));
#pragma unroll
            for (int c = 0; c < NR; c++) s[c] += a * y.v[c];
        }
    } else {
        int64_t sl = row / A.C;
        int r = (int)(row - sl * A.C);
        int32_t off = A.sp[sl], len = A.sl[sl];
        const VT *v = A.v + off + r;
        const int32_t *cc = A.sc + off + r;
#pragma unroll 8
        for (int32_t k = 0; k < len; k++) {
            XT a = cvt<XT>(ld_stream(v + k * A.C));
            Vec<XT, NR> y = f(ld_stream(cc + k * A.C));
#pragma unroll
            for (int c = 0; c < NR; c++) s[c] += a * y.v[c];
        }
    }
}

template <int G, class XT> __device__ __forceinline__ XT lane_reduce(XT s) {
    if constexpr (G > 1) {
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o, G);
    }
    return s;
}

template <int G> __device__ __forceinline__ void row_of(int64_t &row, int &lane) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if constexpr (G > 0) {
        row = t / G;
        lane = (int)(t % G);
    } else {
        row = t;
        lane = 0;
    }
}

// VK_RESID0: r = b - A (D1^-1 b)
// VK_POST:   x = y + D1^-1 (b - A y),  y = D1^-1 b + P x_c   (formed per neighbour)
// VK_RESID:  r = b - A x
// VK_SMOOTH: x = y + D1^-1 (b - A y)                       (y stored)
template <int G, class VT, class XT, int K, int NR>
__global__ void __launch_bounds__(256) k_level(LvlMat<VT> A, const XT *__restrict__ dinv, const XT *__restrict__ b,
                                               const XT *__restrict__ xin, const int32_t *__restrict__ agg,
                                               const XT *__restrict__ xc, XT *__restrict__ out) {
    int64_t row;
    int lane;
    row_of<G>(row, lane);
    XT s[NR];
#pragma unroll
    for (int c = 0; c < NR; c++) s[c] = 0;
    bool live = row < A.n;
    if (live) row_sum<G, VT, XT, NR>(A, row, lane, Nb<XT, NR, K>{dinv, b, xin, xc, agg}, s);
#pragma unroll
    for (int c = 0; c < NR; c++) s[c] = lane_reduce<G, XT>(s[c]);
    if (live && lane == 0) {
        int64_t o = (G == 0 && A.perm) ? A.perm[row] : row;
        XT sc = A.rscale ? (XT)A.rscale[o] : (XT)1;
        Vec<XT, NR> bo = ldv<XT, NR>(b, o), res;
        if (K == VK_RESID0 || K == VK_RESID) {
#pragma unroll
            for (int c = 0; c < NR; c++) res.v[c] = bo.v[c] - s[c] * sc;
        } else {
            XT d = dinv[o];
            Vec<XT, NR> y;
            if (K == VK_POST) {
#pragma unroll
                for (int c = 0; c < NR; c++) y.v[c] = d * bo.v[c];
                if (agg) {
                    int32_t a = agg[o];
                    if (a >= 0) {
                        Vec<XT, NR> xa = ldv<XT, NR>(xc, a);
#pragma unroll
                        for (int c = 0; c < NR; c++) y.v[c] += xa.v[c];
                    }
                }
            } else {
                y = ldv<XT, NR>(xin, o);
            }
#pragma unroll
            for (int c = 0; c < NR; c++) res.v[c] = y.v[c] + d * (bo.v[c] - s[c] * sc);
        }
        stv<XT, NR>(out, o, res);
    }
}

// ---- elementwise kernels (NR interleaved columns; row of entry e = e / NR)
template <class XT, int NR>
__global__ void k_vc_x0(int64_t n, const XT *__restrict__ dinv, const XT *__restrict__ b, XT *__restrict__ x) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * NR; e += (int64_t)gridDim.x * blockDim.x)
        x[e] = dinv[e / NR] * b[e];
}

// y_(i,c) += x_c(agg_i, c)
template <class XT, int NR>
__global__ void k_vc_prolong(int64_t n, const int32_t *__restrict__ agg, const XT *__restrict__ xc,
                             XT *__restrict__ y) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * NR; e += (int64_t)gridDim.x * blockDim.x) {
        int32_t a = agg[e / NR];
        if (a >= 0) y[e] += xc[(int64_t)a * NR + e % NR];
    }
}

// Chebyshev (Saad, Iterative Methods, Alg. 12.1 for D1^-1 A on [lo, hi]):
// first step d = (D1^-1 r) / theta, x = x0 + d; later steps
// d = c1 d + c2 D1^-1 r, x += d.
template <class XT, int NR>
__global__ void k_cheb_first(int64_t n, const XT *__restrict__ dinv, const XT *__restrict__ r,
                             const XT *__restrict__ x0, XT inv_theta, XT *__restrict__ d, XT *__restrict__ x) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * NR; e += (int64_t)gridDim.x * blockDim.x) {
        XT di = dinv[e / NR] * r[e] * inv_theta;
        d[e] = di;
        x[e] = x0 ? x0[e] + di : di;
    }
}

template <class XT, int NR>
__global__ void k_cheb_next(int64_t n, const XT *__restrict__ dinv, const XT *__restrict__ r, XT c1, XT c2,
                            XT *__restrict__ d, XT *__restrict__ x) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * NR; e += (int64_t)gridDim.x * blockDim.x) {
        XT di = c1 * d[e] + c2 * (dinv[e / NR] * r[e]);
        d[e] = di;
        x[e] += di;
    }
}

// b_c[I] = sum of r over the members of aggregate I (ascending), NR columns
template <class XT, int NR>
__global__ void k_vc_restrict(int64_t nc, const int32_t *__restrict__ off, const int32_t *__restrict__ mem,
                              const XT *__restrict__ r, XT *__restrict__ bc) {
    int64_t I = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nc) return;
    Vec<XT, NR> s;
#pragma unroll
    for (int c = 0; c < NR; c++) s.v[c] = 0;
    for (int32_t q = off[I]; q < off[I + 1]; q++) {
        Vec<XT, NR> x = ldv<XT, NR>(r, mem[q]);
#pragma unroll
        for (int c = 0; c < NR; c++) s.v[c] += x.v[c];
    }
    stv<XT, NR>(bc, I, s);
}

// Smoothed aggregation transfers (NR columns): b_c = R r and y += P x_c, one
// thread per output row, entries in CSR order.
template <class XT, int NR>
__global__ void k_sa_restrict(int64_t nc, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                              const XT *__restrict__ v, const XT *__restrict__ r, XT *__restrict__ bc) {
    int64_t I = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nc) return;
    Vec<XT, NR> s;
#pragma unroll
    for (int c = 0; c < NR; c++) s.v[c] = 0;
    for (int32_t p = rp[I]; p < rp[I + 1]; p++) {
        XT a = v[p];
        Vec<XT, NR> x = ldv<XT, NR>(r, ci[p]);
#pragma unroll
        for (int c = 0; c < NR; c++) s.v[c] += a * x.v[c];
    }
    stv<XT, NR>(bc, I, s);
}

template <class XT, int NR>
__global__ void k_sa_prolong(int64_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                             const XT *__restrict__ v, const XT *__restrict__ xc, XT *__restrict__ y) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    Vec<XT, NR> s = ldv<XT, NR>(y, i), t;
#pragma unroll
    for (int c = 0; c < NR; c++) t.v[c] = 0;
    for (int32_t p = rp[i]; p < rp[i + 1]; p++) {
        XT a = v[p];
        Vec<XT, NR> x = ldv<XT, NR>(xc, ci[p]);
#pragma unroll
        for (int c = 0; c < NR; c++) t.v[c] += a * x.v[c];
    }
#pragma unroll
    for (int c = 0; c < NR; c++) s.v[c] += t.v[c];
    stv<XT, NR>(y, i, s);
}

// ---------------------------------------------------------------- host dispatch

template <class VT> static LvlMat<VT> lvl_view(const Level &L) {
    LvlMat<VT> m{};
    m.n = L.A.nrow;
    m.rp = L.A.rowp();
    m.ci = L.A.cols();
    m.rscale = L.rscale.p ? L.rscale.as<float>() : nullptr;
    if (L.fmt == FMT_SELL) {
        m.v = L.sell_val.as<VT>();
        m.sp = L.sell_ptr.as<int32_t>();
        m.sl = L.sell_len.as<int32_t>();
        m.sc = L.sell_col.as<int32_t>();
        m.perm = L.sell_perm.p ? L.sell_perm.as<int32_t>() : nullptr;
        m.C = L.sell_c;
    } else {
        m.v = std::is_same<VT, double>::value ? (const VT *)L.A.vals() : L.vals_lp.as<VT>();
        m.C = 1;
    }
    return m;
}

template <class VT, class XT, int K, int NR>
static void launch_level(Ctx &c, const Level &L, const XT *dinv, const XT *b, const XT *xin, const int32_t *agg,
                         const XT *xc, XT *out, int64_t nc) {
    LvlMat<VT> m = lvl_view<VT>(L);
    int64_t n = L.A.nrow;
    double vb = L.fmt == FMT_SELL ? (sizeof(VT) + 4.0) * (double)L.sell_nnz : (sizeof(VT) + 4.0) * L.A.nnz;
    double xb = sizeof(XT) * (double)NR;
    double bytes = vb + (L.fmt == FMT_SELL ? 8.0 * L.sell_nslice : 4.0 * (n + 1)) + sizeof(XT) * n + 2.0 * xb * n +
                   (K == VK_POST && agg ? 4.0 * n + xb * (double)nc : 0.0) + (L.rscale.p ? 4.0 * n : 0.0) +
                   (K == VK_SMOOTH ? xb * (double)n : 0.0);
    double flops = NR * (2.0 * L.A.nnz + (K == VK_RESID0 ? n : K == VK_POST ? 5.0 * n : K == VK_SMOOTH ? 3.0 * n : 0.0));
    int cls = (K == VK_RESID0 || K == VK_RESID) ? KC_VC_RESID : KC_VC_POST;
    if (L.fmt == FMT_SELL) {
        int64_t rows = L.sell_nslice * L.sell_c;
        MDS_LAUNCH_F(c, cls, bytes, flops, (k_level<0, VT, XT, K, NR>), grid_for(rows, 256), 256, 0, m, dinv, b, xin,
                     agg, xc, out);
        return;
    }
    switch (L.G) {
        case 2:
            MDS_LAUNCH_F(c, cls, bytes, flops, (k_level<2, VT, XT, K, NR>), grid_for(n * 2, 256), 256, 0, m, dinv, b,
                         xin, agg, xc, out);
            break;
        case 4:
            MDS_LAUNCH_F(c, cls, bytes, flops, (k_level<4, VT, XT, K, NR>), grid_for(n * 4, 256), 256, 0, m, dinv, b,
                         xin, agg, xc, out);
            break;
        case 8:
            MDS_LAUNCH_F(c, cls, bytes, flops, (k_level<8, VT, XT, K, NR>), grid_for(n * 8, 256), 256, 0, m, dinv, b,
                         xin, agg, xc, out);
            break;
        case 16:
            MDS_LAUNCH_F(c, cls, bytes, flops, (k_level<16, VT, XT, K, NR>), grid_for(n * 16, 256), 256, 0, m, dinv, b,
                         xin, agg, xc, out);
            break;
        default:
            MDS_LAUNCH_F(c, cls, bytes, flops, (k_level<32, VT, XT, K, NR>), grid_for(n * 32, 256), 256, 0, m, dinv, b,
                         xin, agg, xc, out);
            break;
    }
}

template <class XT, int K, int NR>
static void level_op(Ctx &c, const Level &L, const XT *b, const XT *xin, const int32_t *agg, const XT *xc, XT *out,
                     int64_t nc) {
    const XT *dinv = L.dinv.as<XT>();
    if constexpr (std::is_same<XT, double>::value) {
        launch_level<double, XT, K, NR>(c, L, dinv, b, xin, agg, xc, out, nc);
    } else {
        switch (L.vt) {
            case VT_BF16: launch_level<__nv_bfloat16, XT, K, NR>(c, L, dinv, b, xin, agg, xc, out, nc); break;
            case VT_F16: launch_level<__half, XT, K, NR>(c, L, dinv, b, xin, agg, xc, out, nc); break;
            default: launch_level<float, XT, K, NR>(c, L, dinv, b, xin, agg, xc, out, nc); break;
        }
    }
}

static unsigned ew_grid(int64_t n) {
    unsigned g = grid_for(n, 256);
    return g > 4096 ? 4096 : g;
}

// x = S(x0; b): `sweeps` smoother applications starting from x0 (NULL = 0).
// x0 and x must differ; uses L.r (residual), L.t (copy) and L.d (Chebyshev
// direction) as scratch.
template <class XT, int NR>
static void smooth_stored(Ctx &c, const Hierarchy &h, const Level &L, const XT *b, const XT *x0, XT *x) {
    int64_t n = L.A.nrow;
    XT *r = L.r.as<XT>();
    const XT *dinv = L.dinv.as<XT>();
    const double lo = 0.3, hi = 1.0;
    const double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo), sigma = theta / delta, rho = 1.0 / sigma;
    const double rho1 = 1.0 / (2.0 * sigma - rho);
    const XT *cur = x0;
    for (int s = 0; s < h.sweeps; s++) {
        XT *dst = x;
        if (cur == x) {
            MDS_CUDA(cudaMemcpyAsync(L.t.p, x, sizeof(XT) * (size_t)n * NR, cudaMemcpyDeviceToDevice, c.stream));
            cur = L.t.as<XT>();
        }
        if (h.smoother == MDS_SMOOTHER_L1JACOBI) {
            if (!cur)
                MDS_LAUNCH(c, KC_NONE, 3.0 * sizeof(XT) * n * NR, (k_vc_x0<XT, NR>), ew_grid(n * NR), 256, 0, n, dinv,
                           b, dst);
            else
                level_op<XT, VK_SMOOTH, NR>(c, L, b, cur, nullptr, nullptr, dst, 0);
        } else {
            XT *d = L.d.as<XT>();
            if (cur) {
                level_op<XT, VK_RESID, NR>(c, L, b, cur, nullptr, nullptr, r, 0);
                MDS_LAUNCH(c, KC_NONE, 0, (k_cheb_first<XT, NR>), ew_grid(n * NR), 256, 0, n, dinv, r, cur,
                           (XT)(1.0 / theta), d, dst);
            } else {
                MDS_LAUNCH(c, KC_NONE, 0, (k_cheb_first<XT, NR>), ew_grid(n * NR), 256, 0, n, dinv, b,
                           (const XT *)nullptr, (XT)(1.0 / theta), d, dst);
            }
            level_op<XT, VK_RESID, NR>(c, L, b, dst, nullptr, nullptr, r, 0);
            MDS_LAUNCH(c, KC_NONE, 0, (k_cheb_next<XT, NR>), ew_grid(n * NR), 256, 0, n, dinv, r, (XT)(rho1 * rho),
                       (XT)(2.0 * rho1 / delta), d, dst);
        }
        cur = dst;
    }
}

template <class XT, int NR>
static void vcycle_level(Ctx &c, Hierarchy &h, int l, const XT *b, XT *x) {
    Level &L = h.lv[l];
    int last = (int)h.lv.size() - 1;
    if (l == last && h.dense) {
        dense_apply(c, h.Ainv.as<double>(), h.nd, NR, b, x);
        return;
    }
    int64_t n = L.A.nrow;
    XT *r = L.r.as<XT>();
    double rbytes = 4.0 * (L.nc + 1) + 4.0 * n + sizeof(XT) * NR * (double)(n + L.nc);
    bool fused = !std::is_same<XT, double>::value && h.smoother == MDS_SMOOTHER_L1JACOBI && h.sweeps == 1 &&
                 !L.smoothed;
    if (fused) {
        if (L.has_coarse) {
            Level &C = h.lv[l + 1];
            level_op<XT, VK_RESID0, NR>(c, L, b, nullptr, nullptr, nullptr, r, 0);
            MDS_LAUNCH(c, KC_VC_RESTRICT, rbytes, (k_vc_restrict<XT, NR>), grid_for(L.nc, 256), 256, 0, L.nc,
                       L.mem_off.as<int32_t>(), L.mem.as<int32_t>(), r, C.b.as<XT>());
            vcycle_level<XT, NR>(c, h, l + 1, C.b.as<XT>(), C.x.as<XT>());
            level_op<XT, VK_POST, NR>(c, L, b, nullptr, L.agg.as<int32_t>(), C.x.as<XT>(), x, L.nc);
        } else {
            level_op<XT, VK_POST, NR>(c, L, b, nullptr, nullptr, nullptr, x, 0);
        }
        return;
    }
    XT *y = L.y.as<XT>();
    smooth_stored<XT, NR>(c, h, L, b, nullptr, y);  // y = S(0; b)
    if (L.has_coarse) {
        Level &C = h.lv[l + 1];
        level_op<XT, VK_RESID, NR>(c, L, b, y, nullptr, nullptr, r, 0);
        if (L.smoothed) {
            const XT *rv = std::is_same<XT, double>::value ? (const XT *)L.R.vals() : L.Rv_lp.as<XT>();
            const XT *pv = std::is_same<XT, double>::value ? (const XT *)L.P.vals() : L.Pv_lp.as<XT>();
            double tb = (sizeof(XT) + 4.0) * L.R.nnz + 4.0 * (L.nc + 1) + sizeof(XT) * NR * (double)(n + L.nc);
            MDS_LAUNCH(c, KC_VC_RESTRICT, tb, (k_sa_restrict<XT, NR>), grid_for(L.nc, 256), 256, 0, L.nc, L.R.rowp(),
                       L.R.cols(), rv, r, C.b.as<XT>());
            vcycle_level<XT, NR>(c, h, l + 1, C.b.as<XT>(), C.x.as<XT>());
            MDS_LAUNCH(c, KC_NONE, tb + sizeof(XT) * NR * (double)n, (k_sa_prolong<XT, NR>), grid_for(n, 256), 256, 0,
                       n, L.P.rowp(), L.P.cols(), pv, C.x.as<XT>(), y);
        } else {
            MDS_LAUNCH(c, KC_VC_RESTRICT, rbytes, (k_vc_restrict<XT, NR>), grid_for(L.nc, 256), 256, 0, L.nc,
                       L.mem_off.as<int32_t>(), L.mem.as<int32_t>(), r, C.b.as<XT>());
            vcycle_level<XT, NR>(c, h, l + 1, C.b.as<XT>(), C.x.as<XT>());
            MDS_LAUNCH(c, KC_NONE, 3.0 * sizeof(XT) * n * NR, (k_vc_prolong<XT, NR>), ew_grid(n * NR), 256, 0, n,
                       L.agg.as<int32_t>(), C.x.as<XT>(), y);
        }
    }
    smooth_stored<XT, NR>(c, h, L, b, y, x);  // x = S(y; b)
}

// The level work vectors hold up to nr_cap interleaved columns.
void hierarchy_reserve(Ctx &c, Hierarchy &h, int nr) {
    if (nr <= h.nr_cap) return;
    size_t vb = h.prec == 64 ? sizeof(double) : sizeof(float);
    for (auto &L : h.lv) {
        size_t nb = vb * (size_t)(L.A.nrow > 0 ? L.A.nrow : 1) * (size_t)nr;
        L.b = Buf(&c, nb);
        L.x = Buf(&c, nb);
        L.r = Buf(&c, nb);
        L.y = Buf(&c, nb);
        L.t = Buf(&c, nb);
        if (h.smoother == MDS_SMOOTHER_CHEBYSHEV) L.d = Buf(&c, nb);
    }
    h.nr_cap = nr;
}

template <class XT>
static void vcycle_nr(Ctx &c, Hierarchy &h, const XT *b, XT *x, int nr) {
    switch (nr) {
        case 1: vcycle_level<XT, 1>(c, h, 0, b, x); break;
        case 2: vcycle_level<XT, 2>(c, h, 0, b, x); break;
        case 4: vcycle_level<XT, 4>(c, h, 0, b, x); break;
        case 8: vcycle_level<XT, 8>(c, h, 0, b, x); break;
        default: throw Error(MDS_ERR_INVALID, "V-cycle column count must be 1, 2, 4 or 8");
    }
}

void vcycle_apply(Ctx &c, Hierarchy &h, const void *b, void *x, int nr) {
    MDS_REQUIRE(nr <= h.nr_cap, MDS_ERR_INVALID, "V-cycle work vectors hold fewer columns");
    KTimer all(c, KC_VCYCLE, 0.0);
    if (h.prec == 64)
        vcycle_nr<double>(c, h, (const double *)b, (double *)x, nr);
    else
        vcycle_nr<float>(c, h, (const float *)b, (float *)x, nr);
}

// ---------------------------------------------------------------- level storage

// s_i = 2^ceil(log2 max_j |a_ij|) (1 for a zero row)
__global__ void k_row_scale(int64_t n, const int32_t *__restrict__ rp, const double *__restrict__ v,
                            float *__restrict__ s) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double mx = 0.0;
    for (int32_t p = rp[i]; p < rp[i + 1]; p++) mx = fmax(mx, fabs(v[p]));
    if (mx == 0.0) {
        s[i] = 1.0f;
        return;
    }
    int e = 0;
    double fr = frexp(mx, &e);
    if (fr == 0.5) e -= 1;
    s[i] = (float)ldexp(1.0, e);
}

template <class VT> __device__ __forceinline__ VT from_d(double a, double sc);
template <> __device__ __forceinline__ double from_d<double>(double a, double) { return a; }
template <> __device__ __forceinline__ float from_d<float>(double a, double) { return (float)a; }
template <> __device__ __forceinline__ __nv_bfloat16 from_d<__nv_bfloat16>(double a, double sc) {
    return __float2bfloat16_rn((float)(a / sc));
}
template <> __device__ __forceinline__ __half from_d<__half>(double a, double sc) {
    return __float2half_rn((float)(a / sc));
}

// CSR values in the storage type
template <class VT>
__global__ void k_csr_lowp(int64_t n, const int32_t *__restrict__ rp, const double *__restrict__ v,
                           const float *__restrict__ s, VT *__restrict__ o) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double sc = s ? (double)s[i] : 1.0;
    for (int32_t p = rp[i]; p < rp[i + 1]; p++) o[p] = from_d<VT>(v[p], sc);
}

// SELL: window sort of rows by decreasing length (stable), one thread per window
__global__ void k_sell_perm(int64_t n, const int32_t *__restrict__ rp, int sigma, int32_t *__restrict__ perm) {
    int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t a = w * sigma;
    if (a >= n) return;
    int64_t e = a + sigma < n ? a + sigma : n;
    for (int64_t i = a; i < e; i++) perm[i] = (int32_t)i;
    for (int64_t i = a + 1; i < e; i++) {
        int32_t x = perm[i];
        int32_t lx = rp[x + 1] - rp[x];
        int64_t q = i - 1;
        while (q >= a && (rp[perm[q] + 1] - rp[perm[q]]) < lx) {
            perm[q + 1] = perm[q];
            q--;
        }
        perm[q + 1] = x;
    }
}

__global__ void k_sell_len(int64_t n, int64_t nslice, int C, const int32_t *__restrict__ rp,
                           const int32_t *__restrict__ perm, int32_t *__restrict__ len, int32_t *__restrict__ cnt) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nslice) return;
    int32_t mx = 0;
    for (int r = 0; r < C; r++) {
        int64_t row = s * C + r;
        if (row >= n) break;
        int64_t o = perm ? perm[row] : row;
        int32_t l = rp[o + 1] - rp[o];
        mx = l > mx ? l : mx;
    }
    len[s] = mx;
    cnt[s] = mx * C;
}

template <class VT>
__global__ void k_sell_fill(int64_t n, int64_t nslice, int C, const int32_t *__restrict__ rp,
                            const int32_t *__restrict__ ci, const double *__restrict__ v, const float *__restrict__ s,
                            const int32_t *__restrict__ perm, const int32_t *__restrict__ sp,
                            const int32_t *__restrict__ sl, int32_t *__restrict__ sc, VT *__restrict__ sv) {
    int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= nslice * C) return;
    int64_t sli = row / C;
    int r = (int)(row - sli * C);
    int64_t o = row < n ? (perm ? perm[row] : row) : -1;
    int32_t a = o >= 0 ? rp[o] : 0, l = o >= 0 ? rp[o + 1] - rp[o] : 0;
    double scale = (o >= 0 && s) ? (double)s[o] : 1.0;
    for (int32_t k = 0; k < sl[sli]; k++) {
        int32_t p = sp[sli] + k * C + r;
        if (k < l) {
            sc[p] = ci[a + k];
            sv[p] = from_d<VT>(v[a + k], scale);
        } else {
            sc[p] = o >= 0 ? (int32_t)o : 0;  // padding: a valid column with a zero value
            sv[p] = from_d<VT>(0.0, 1.0);
        }
    }
}

template <class VT> static void build_sell(Ctx &c, Level &L, int C, int sigma) {
    int64_t n = L.A.nrow;
    L.sell_c = C;
    L.sell_nslice = (n + C - 1) / C;
    int64_t ns = L.sell_nslice;
    L.sell_perm.reset();
    if (sigma > 1) {
        L.sell_perm = Buf(&c, sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
        int64_t nw = (n + sigma - 1) / sigma;
        MDS_LAUNCH(c, KC_NONE, 0, k_sell_perm, grid_for(nw, 64), 64, 0, n, L.A.rowp(), sigma, L.sell_perm.as<int32_t>());
    }
    L.sell_len = Buf(&c, sizeof(int32_t) * (size_t)(ns + 1));
    L.sell_ptr = Buf(&c, sizeof(int32_t) * (size_t)(ns + 1));
    Buf cnt(&c, sizeof(int32_t) * (size_t)(ns + 1));
    const int32_t *perm = L.sell_perm.p ? L.sell_perm.as<int32_t>() : nullptr;
    MDS_LAUNCH(c, KC_NONE, 0, k_sell_len, grid_for(ns, 256), 256, 0, n, ns, C, L.A.rowp(), perm,
               L.sell_len.as<int32_t>(), cnt.as<int32_t>());
    L.sell_nnz = scan_counts(c, cnt.as<int32_t>(), L.sell_ptr.as<int32_t>(), ns);
    L.sell_col = Buf(&c, sizeof(int32_t) * (size_t)(L.sell_nnz > 0 ? L.sell_nnz : 1));
    L.sell_val = Buf(&c, sizeof(VT) * (size_t)(L.sell_nnz > 0 ? L.sell_nnz : 1));
    MDS_LAUNCH(c, KC_NONE, 0, k_sell_fill<VT>, grid_for(ns * C, 256), 256, 0, n, ns, C, L.A.rowp(), L.A.cols(),
               L.A.vals(), L.rscale.p ? L.rscale.as<float>() : nullptr, perm, L.sell_ptr.as<int32_t>(),
               L.sell_len.as<int32_t>(), L.sell_col.as<int32_t>(), L.sell_val.as<VT>());
    L.fmt = FMT_SELL;
}

static void build_sell_vt(Ctx &c, Level &L, int C, int sigma) {
    switch (L.vt) {
        case VT_F64: build_sell<double>(c, L, C, sigma); break;
        case VT_F32: build_sell<float>(c, L, C, sigma); break;
        case VT_BF16: build_sell<__nv_bfloat16>(c, L, C, sigma); break;
        case VT_F16: build_sell<__half>(c, L, C, sigma); break;
    }
}

static void drop_sell(Level &L) {
    L.sell_perm.reset();
    L.sell_len.reset();
    L.sell_ptr.reset();
    L.sell_col.reset();
    L.sell_val.reset();
    L.sell_nnz = 0;
    L.fmt = FMT_CSR;
}

static int default_g(const Level &L) {
    double avg = L.A.nrow ? (double)L.A.nnz / (double)L.A.nrow : 0.0;
    return avg <= 4.0 ? 2 : avg <= 10.0 ? 4 : avg <= 20.0 ? 8 : avg <= 40.0 ? 16 : 32;
}

// Time the stored-residual kernel on the level in its current storage (best
// of three after a warm-up launch).
template <class XT> static float time_level(Ctx &c, const Level &L) {
    cudaEvent_t e0, e1;
    MDS_CUDA(cudaEventCreate(&e0));
    MDS_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    for (int rep = 0; rep < 4; rep++) {
        MDS_CUDA(cudaEventRecord(e0, c.stream));
        level_op<XT, VK_RESID, 1>(c, L, L.b.as<XT>(), L.x.as<XT>(), nullptr, nullptr, L.r.as<XT>(), 0);
        MDS_CUDA(cudaEventRecord(e1, c.stream));
        MDS_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        MDS_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (rep > 0) best = std::min(best, ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return best;
}

// Autotuner: time CSR with G/2, G, 2G lanes per row and SELL-C-sigma for a
// few (C, sigma) pairs on this level, keep the fastest.  Choices are cached in
// the context by (rows, nonzeros, storage type).
template <class XT> static void autotune_level(Ctx &c, Level &L) {
    auto key = std::make_tuple(L.A.nrow, L.A.nnz, L.vt);
    auto it = c.tune_cache.find(key);
    if (it != c.tune_cache.end()) {
        const TuneChoice &t = it->second;
        if (t.fmt == FMT_SELL)
            build_sell_vt(c, L, t.C, t.sigma);
        else
            L.G = t.G;
        return;
    }
    // defined inputs for the timing runs
    size_t vb = sizeof(XT) * (size_t)L.A.nrow;
    MDS_CUDA(cudaMemsetAsync(L.b.p, 0, vb, c.stream));
    MDS_CUDA(cudaMemsetAsync(L.x.p, 0, vb, c.stream));
    TuneChoice best{FMT_CSR, default_g(L), 32, 1};
    float tbest = 1e30f;
    int g0 = default_g(L);
    for (int G : {g0 / 2, g0, g0 * 2}) {
        if (G < 2 || G > 32) continue;
        L.fmt = FMT_CSR;
        L.G = G;
        float t = time_level<XT>(c, L);
        if (t < tbest) {
            tbest = t;
            best = TuneChoice{FMT_CSR, G, 32, 1};
        }
    }
    const int cand[][2] = {{32, 1}, {32, 256}, {16, 1}};
    for (auto &cs : cand) {
        build_sell_vt(c, L, cs[0], cs[1]);
        float t = time_level<XT>(c, L);
        if (t < tbest) {
            tbest = t;
            best = TuneChoice{FMT_SELL, 0, cs[0], cs[1]};
        }
        drop_sell(L);
    }
    c.tune_cache[key] = best;
    L.G = best.fmt == FMT_CSR ? best.G : default_g(L);
    if (best.fmt == FMT_SELL) build_sell_vt(c, L, best.C, best.sigma);
}

void level_storage(Ctx &c, Hierarchy &h, const mds_setup_opts &o) {
    for (size_t l = 0; l < h.lv.size(); l++) {
        Level &L = h.lv[l];
        int64_t n = L.A.nrow;
        bool lowp = (o.precision == MDS_PREC_BF16 || o.precision == MDS_PREC_FP16) && (int)l >= o.lowp_from_level;
        L.vt = h.prec == 64 ? VT_F64 : !lowp ? VT_F32 : (o.precision == MDS_PREC_BF16 ? VT_BF16 : VT_F16);
        L.G = default_g(L);
        L.fmt = FMT_CSR;
        if (L.smoothed && h.prec != 64) {
            L.Pv_lp = Buf(&c, sizeof(float) * (size_t)(L.P.nnz > 0 ? L.P.nnz : 1));
            L.Rv_lp = Buf(&c, sizeof(float) * (size_t)(L.R.nnz > 0 ? L.R.nnz : 1));
            MDS_LAUNCH(c, KC_NONE, 0, k_csr_lowp<float>, grid_for(L.P.nrow, 256), 256, 0, L.P.nrow, L.P.rowp(),
                       L.P.vals(), (const float *)nullptr, L.Pv_lp.as<float>());
            MDS_LAUNCH(c, KC_NONE, 0, k_csr_lowp<float>, grid_for(L.R.nrow, 256), 256, 0, L.R.nrow, L.R.rowp(),
                       L.R.vals(), (const float *)nullptr, L.Rv_lp.as<float>());
        }
        if (l + 1 == h.lv.size() && h.dense) continue;  // applied through the dense inverse
        unsigned gr = grid_for(n, 256);
        if (L.vt == VT_BF16 || L.vt == VT_F16) {
            L.rscale = Buf(&c, sizeof(float) * (size_t)(n > 0 ? n : 1));
            MDS_LAUNCH(c, KC_NONE, 0, k_row_scale, gr, 256, 0, n, L.A.rowp(), L.A.vals(), L.rscale.as<float>());
        }
        const float *s = L.rscale.p ? L.rscale.as<float>() : nullptr;
        size_t nz = (size_t)(L.A.nnz > 0 ? L.A.nnz : 1);
        if (L.vt == VT_F32) {
            L.vals_lp = Buf(&c, 4 * nz);
            MDS_LAUNCH(c, KC_NONE, 0, k_csr_lowp<float>, gr, 256, 0, n, L.A.rowp(), L.A.vals(), s, L.vals_lp.as<float>());
        } else if (L.vt == VT_BF16) {
            L.vals_lp = Buf(&c, 2 * nz);
            MDS_LAUNCH(c, KC_NONE, 0, k_csr_lowp<__nv_bfloat16>, gr, 256, 0, n, L.A.rowp(), L.A.vals(), s,
                       L.vals_lp.as<__nv_bfloat16>());
        } else if (L.vt == VT_F16) {
            L.vals_lp = Buf(&c, 2 * nz);
            MDS_LAUNCH(c, KC_NONE, 0, k_csr_lowp<__half>, gr, 256, 0, n, L.A.rowp(), L.A.vals(), s,
                       L.vals_lp.as<__half>());
        }
        if (o.format == MDS_FORMAT_SELL) {
            build_sell_vt(c, L, o.sell_c, o.sell_sigma);
        } else if (o.format == MDS_FORMAT_AUTO && n >= 20000) {
            if (h.prec == 64)
                autotune_level<double>(c, L);
            else
                autotune_level<float>(c, L);
        }
    }
}

}  // namespace mds
