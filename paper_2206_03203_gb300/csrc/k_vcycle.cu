// One aggregation-AMG V-cycle (Sec. 3.3: Q_mm and Q_ff of Algorithm 1).
//
// Per level, with L1 diagonal D1 and piecewise-constant P:
//   pre-smooth from zero      x = D1^-1 b
//   residual + restriction    b_c = P^T (b - A x)
//   coarse correction         x_c = V(b_c)      (dense inverse on the last level)
//   prolongation + smoothing  x <- x + P x_c;  x <- x + D1^-1 (b - A x)
// The pre-smoothed x is never stored: the residual kernel forms D1^-1 b on
// the fly, and the post-smoothing kernel forms x + P x_c on the fly at every
// neighbour, so each level costs two passes over its matrix.
#include "internal.cuh"

namespace mds {

// r_i = b_i - sum_j a_ij (dinv_j b_j)
template <int G, class VT, class XT>
__global__ void __launch_bounds__(256) k_vc_resid0(int64_t n, const int32_t *__restrict__ rp,
                                                    const int32_t *__restrict__ ci, const VT *__restrict__ v,
                                                    const XT *__restrict__ dinv, const XT *__restrict__ b,
                                                    XT *__restrict__ r) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t row = t / G;
    int lane = (int)(t % G);
    XT s = 0;
    if (row < n) {
        int32_t p0 = rp[row], p1 = rp[row + 1];
        for (int32_t p = p0 + lane; p < p1; p += G) {
            int32_t j = ci[p];
            s += (XT)v[p] * (__ldg(dinv + j) * __ldg(b + j));
        }
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o, G);
    if (row < n && lane == 0) r[row] = b[row] - s;
}

// b_c[I] = sum of r over the members of aggregate I (ascending)
template <class XT>
__global__ void k_vc_restrict(int64_t nc, const int32_t *__restrict__ off, const int32_t *__restrict__ mem,
                              const XT *__restrict__ r, XT *__restrict__ bc) {
    int64_t I = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nc) return;
    XT s = 0;
    for (int32_t q = off[I]; q < off[I + 1]; q++) s += r[mem[q]];
    bc[I] = s;
}

// x_i = y_i + dinv_i (b_i - sum_j a_ij y_j),  y_j = dinv_j b_j + x_c[agg_j]
template <int G, class VT, class XT>
__global__ void __launch_bounds__(256) k_vc_post(int64_t n, const int32_t *__restrict__ rp,
                                                  const int32_t *__restrict__ ci, const VT *__restrict__ v,
                                                  const XT *__restrict__ dinv, const XT *__restrict__ b,
                                                  const int32_t *__restrict__ agg, const XT *__restrict__ xc,
                                                  XT *__restrict__ x) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t row = t / G;
    int lane = (int)(t % G);
    XT s = 0;
    if (row < n) {
        int32_t p0 = rp[row], p1 = rp[row + 1];
        for (int32_t p = p0 + lane; p < p1; p += G) {
            int32_t j = ci[p];
            XT y = __ldg(dinv + j) * __ldg(b + j);
            if (agg) {
                int32_t a = __ldg(agg + j);
                if (a >= 0) y += __ldg(xc + a);
            }
            s += (XT)v[p] * y;
        }
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o, G);
    if (row < n && lane == 0) {
        XT yi = dinv[row] * b[row];
        if (agg) {
            int32_t a = agg[row];
            if (a >= 0) yi += xc[a];
        }
        x[row] = yi + dinv[row] * (b[row] - s);
    }
}

template <class XT> struct VcKernels {
    template <int G>
    static void resid(Ctx &c, int64_t n, const Level &L, const XT *vals, const XT *b, XT *r) {
        double bytes = (sizeof(XT) + 4.0) * L.A.nnz + 4.0 * (n + 1) + 3.0 * sizeof(XT) * n;
        MDS_LAUNCH(c, KC_VC_RESID, bytes, (k_vc_resid0<G, XT, XT>), grid_for(n * G, 256),
                   256, 0, n, L.A.rowp(), L.A.cols(), vals, L.dinv.as<XT>(), b, r);
    }
    template <int G>
    static void post(Ctx &c, int64_t n, const Level &L, const XT *vals, const XT *b, const int32_t *agg,
                     const XT *xc, XT *x, int64_t nc) {
        double bytes = (sizeof(XT) + 4.0) * L.A.nnz + 4.0 * (n + 1) + 3.0 * sizeof(XT) * n +
                       (agg ? 4.0 * n + sizeof(XT) * (double)nc : 0.0);
        MDS_LAUNCH(c, KC_VC_POST, bytes, (k_vc_post<G, XT, XT>), grid_for(n * G, 256), 256, 0, n, L.A.rowp(),
                   L.A.cols(), vals, L.dinv.as<XT>(), b, agg, xc, x);
    }
};

template <class XT>
static int pick_g(const Level &L) {
    double avg = L.A.nrow ? (double)L.A.nnz / (double)L.A.nrow : 0.0;
    return avg <= 4.0 ? 2 : avg <= 10.0 ? 4 : avg <= 24.0 ? 8 : 32;
}

template <class XT>
static void level_resid(Ctx &c, const Level &L, const XT *vals, const XT *b, XT *r) {
    int64_t n = L.A.nrow;
    switch (pick_g<XT>(L)) {
        case 2: VcKernels<XT>::template resid<2>(c, n, L, vals, b, r); break;
        case 4: VcKernels<XT>::template resid<4>(c, n, L, vals, b, r); break;
        case 8: VcKernels<XT>::template resid<8>(c, n, L, vals, b, r); break;
        default: VcKernels<XT>::template resid<32>(c, n, L, vals, b, r); break;
    }
}

template <class XT>
static void level_post(Ctx &c, const Level &L, const XT *vals, const XT *b, const int32_t *agg, const XT *xc, XT *x,
                       int64_t nc) {
    int64_t n = L.A.nrow;
    switch (pick_g<XT>(L)) {
        case 2: VcKernels<XT>::template post<2>(c, n, L, vals, b, agg, xc, x, nc); break;
        case 4: VcKernels<XT>::template post<4>(c, n, L, vals, b, agg, xc, x, nc); break;
        case 8: VcKernels<XT>::template post<8>(c, n, L, vals, b, agg, xc, x, nc); break;
        default: VcKernels<XT>::template post<32>(c, n, L, vals, b, agg, xc, x, nc); break;
    }
}

static void gemv(Ctx &c, const double *M, int64_t n, const double *x, double *y) { dense_gemv_f64(c, M, n, x, y); }
static void gemv(Ctx &c, const double *M, int64_t n, const float *x, float *y) { dense_gemv_f32(c, M, n, x, y); }

template <class XT>
static void vcycle_level(Ctx &c, Hierarchy &h, int l, const XT *b, XT *x) {
    Level &L = h.lv[l];
    int last = (int)h.lv.size() - 1;
    if (l == last && h.dense) {
        gemv(c, h.Ainv.as<double>(), h.nd, b, x);
        return;
    }
    const XT *vals = h.prec == 64 ? (const XT *)L.A.vals() : (const XT *)L.vals_lp.p;
    if (L.has_coarse) {
        Level &C = h.lv[l + 1];
        XT *r = L.r.as<XT>();
        level_resid<XT>(c, L, vals, b, r);
        double rbytes = 4.0 * (L.nc + 1) + 4.0 * L.A.nrow + sizeof(XT) * (double)(L.A.nrow + L.nc);
        MDS_LAUNCH(c, KC_VC_RESTRICT, rbytes, k_vc_restrict<XT>, grid_for(L.nc, 256), 256, 0, L.nc,
                   L.mem_off.as<int32_t>(), L.mem.as<int32_t>(), r, C.b.as<XT>());
        vcycle_level<XT>(c, h, l + 1, C.b.as<XT>(), C.x.as<XT>());
        level_post<XT>(c, L, vals, b, L.agg.as<int32_t>(), C.x.as<XT>(), x, L.nc);
    } else {
        level_post<XT>(c, L, vals, b, (const int32_t *)nullptr, (const XT *)nullptr, x, 0);
    }
}

void vcycle_apply(Ctx &c, Hierarchy &h, const void *b, void *x) {
    KTimer all(c, KC_VCYCLE, 0.0);
    if (h.prec == 64)
        vcycle_level<double>(c, h, 0, (const double *)b, (double *)x);
    else
        vcycle_level<float>(c, h, 0, (const float *)b, (float *)x);
}

}  // namespace mds
