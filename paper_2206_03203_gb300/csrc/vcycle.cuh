// One aggregation-AMG V-cycle (Sec. 3.3: Q_mm and Q_ff of Algorithm 1):
// kernels and host-side level operations, included by the per-type
// translation units.
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
// Two kernel forms.  Memory-bound levels (FP32 and below, and FP64 levels
// small enough to be latency-bound, one L1-Jacobi sweep) form D1^-1 b and
// x + P x_c on the fly at every neighbour, so a level costs three launches
// (residual, restriction, post-smoothing) and the smoothed iterates are never
// stored.  Large FP64 levels are bound by
// GB300's FP64 pipe, so there the iterates are stored once per row instead of
// being re-formed per nonzero; Chebyshev and multi-sweep smoothing also use
// the stored form.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <map>
#include <tuple>
#include <type_traits>

#include "conv.cuh"
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
    int sigma;                 // SELL sorting window (a stored row's original row lies in its window)
    const float *rscale;       // row scales (NULL: unscaled)
    LiveMap lm;                // rows of finished batch instances are skipped
    double *out64;             // NULL, or the FP64 vector the rows are written to instead of out
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
// a level kernel's output row: in FP64 to out64 when given (the top level of
// an FP32 V-cycle writing the Krylov method's vector; the widening is exact,
// done by integer operations so that it leaves the FP64 unit free), else in
// the vector type to out
template <class XT> __device__ __forceinline__ double widen64(XT v) {
    if constexpr (std::is_same<XT, float>::value)
        return f2d_int(v);
    else
        return (double)v;
}
template <class XT, int NR>
__device__ __forceinline__ void st_out(XT *out, double *out64, int64_t j, const Vec<XT, NR> &x) {
    if (out64) {
        Vec<double, NR> w;
#pragma unroll
        for (int c = 0; c < NR; c++) w.v[c] = widen64<XT>(x.v[c]);
        stv<double, NR>(out64, j, w);
    } else {
        stv<XT, NR>(out, j, x);
    }
}

enum { VK_RESID0 = 0, VK_POST = 1, VK_RESID = 2, VK_SMOOTH = 3 };

// Explicitly rounded arithmetic of the level kernels: every storage (CSR,
// SELL, stencil planes), the fused and the stored-y forms and the coarse-tail
// kernel round each product, sum and difference at the same points whatever
// the compiler would contract, so that they agree bit for bit.  y_j = D1_j b_j
// [+ x_c] is two roundings (as when y is stored), the row sum one fused
// multiply-add per entry, x = y + D1 (b - s) a difference and a fused
// multiply-add.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

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
            for (int c = 0; c < NR; c++) y.v[c] = mul_rn(d, bj.v[c]);
            if (K == VK_POST && agg) {
                int32_t a = __ldg(agg + j);
                if (a >= 0) {
                    Vec<XT, NR> xa = ldv<XT, NR>(xc, a);
#pragma unroll
                    for (int c = 0; c < NR; c++) y.v[c] = add_rn(y.v[c], xa.v[c]);
                }
            }
        } else {
            y = ldv<XT, NR>(xin, j);
        }
        return y;
    }
    // the same with 1/D1_j and agg_j already loaded (fused forms)
    __device__ __forceinline__ Vec<XT, NR> with(int32_t j, XT d, int32_t a) const {
        Vec<XT, NR> y;
        Vec<XT, NR> bj = ldv<XT, NR>(b, j);
#pragma unroll
        for (int c = 0; c < NR; c++) y.v[c] = mul_rn(d, bj.v[c]);
        if (K == VK_POST && a >= 0) {
            Vec<XT, NR> xa = ldv<XT, NR>(xc, a);
#pragma unroll
            for (int c = 0; c < NR; c++) y.v[c] = add_rn(y.v[c], xa.v[c]);
        }
        return y;
    }
};

template <int G, class XT> __device__ __forceinline__ XT lane_reduce(XT s) {
    if constexpr (G > 1) {
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o, G);
    }
    return s;
}

template <int G> __device__ __forceinline__ void row_of(int64_t vb, int64_t &row, int &lane) {
    int64_t t = vb * blockDim.x + threadIdx.x;
    if constexpr (G > 0) {
        row = t / G;
        lane = (int)(t % G);
    } else {
        row = t;
        lane = 0;
    }
}

// Entries of each lane's share of a row loaded before the dependency wait.
constexpr int PREFETCH = 8;

// VK_RESID0: r = b - A (D1^-1 b)
// VK_POST:   x = y + D1^-1 (b - A y),  y = D1^-1 b + P x_c   (formed per neighbour)
// VK_RESID:  r = b - A x
// VK_SMOOTH: x = y + D1^-1 (b - A y)                       (y stored)
// Storage: CSR with G lanes per row (G = 1: one thread per row; lane-partial
// sums over entries lane, lane + G, ..., then a lane tree), or SELL with one
// thread per row (G = 0).  The level's matrix, row scales, 1/D1, aggregate
// map and SELL permutation do not change while a V-cycle runs, so each lane
// loads its first PREFETCH entries and its row constants before waiting for
// the previous kernel; only the vector gathers follow the wait.  (Kernels
// that write these arrays run in set-up, which launches without programmatic
// dependence.)  The prefetch (PF entries) pays off when the launch fits in
// about one wave of resident blocks; larger launches (PF = 0) keep registers
// low for occupancy instead.
template <int G, class VT, class XT, int K, int NR, int PF>
__device__ __forceinline__ void level_block(int64_t vb, const LvlMat<VT> &A, const XT *__restrict__ dinv,
                                            const XT *__restrict__ b, const XT *__restrict__ xin,
                                            const int32_t *__restrict__ agg, const XT *__restrict__ xc,
                                            XT *__restrict__ out) {
    {
        // this block's rows (whole sorting windows for permuted SELL)
        int64_t r0, r1;
        if constexpr (G > 0) {
            r0 = vb * (256 / G);
            r1 = r0 + 256 / G;
        } else {
            r0 = vb * 256;
            r1 = r0 + 256;
            if (A.perm) {
                r0 = r0 / A.sigma * A.sigma;
                r1 = (r1 + A.sigma - 1) / A.sigma * A.sigma;
            }
        }
        if (!block_rows_live(A.lm, r0, r1 < A.n ? r1 : A.n)) return;
    }
    int64_t row;
    int lane;
    row_of<G>(vb, row, lane);
    const bool live = row < A.n;
    // this lane's entries: index i0 + k * st for k < cnt
    const int32_t *cp = G > 0 ? A.ci : A.sc;
    int64_t i0 = 0;
    int st = 1, cnt = 0;
    if (live) {
        if constexpr (G > 0) {
            int32_t p0 = A.rp[row], p1 = A.rp[row + 1];
            i0 = p0 + lane;
            st = G;
            cnt = p1 > i0 ? (int)((p1 - i0 + G - 1) / G) : 0;
        } else {
            int64_t sl = row / A.C;
            int r = (int)(row - sl * A.C);
            i0 = (int64_t)A.sp[sl] + r;
            st = A.C;
            cnt = A.sl[sl];
        }
    }
    constexpr bool FUSED = K == VK_RESID0 || K == VK_POST;
    VT pa[PF > 0 ? PF : 1];
    int32_t pj[PF > 0 ? PF : 1];
    XT pd[FUSED && PF > 0 ? PF : 1];       // 1/D1 of the neighbours (fused forms)
    int32_t pg[K == VK_POST && PF > 0 ? PF : 1];  // their aggregates (post-smoothing)
#pragma unroll
    for (int k = 0; k < PF; k++)
        if (k < cnt) {
            pa[k] = ld_stream(A.v + i0 + (int64_t)k * st);
            pj[k] = ld_stream(cp + i0 + (int64_t)k * st);
        }
    if constexpr (FUSED && PF > 0) {
#pragma unroll
        for (int k = 0; k < PF; k++)
            if (k < cnt) {
                pd[k] = __ldg(dinv + pj[k]);
                if constexpr (K == VK_POST) pg[k] = agg ? __ldg(agg + pj[k]) : -1;
            }
    }
    int64_t o = row;
    XT sc = (XT)1, d = (XT)0;
    int32_t ag = -1;
    if (live && lane == 0) {
        if (G == 0 && A.perm) o = A.perm[row];
        if (A.rscale) sc = (XT)A.rscale[o];
        if (K == VK_POST || K == VK_SMOOTH) d = dinv[o];
        if (K == VK_POST && agg) ag = agg[o];
    }
    mds_pdl_wait();
    mds_pdl_trigger();
    // row terms that do not depend on the sum, loaded with the gathers
    Vec<XT, NR> bo, yo;
#pragma unroll
    for (int c = 0; c < NR; c++) bo.v[c] = yo.v[c] = (XT)0;
    if (live && lane == 0) {
        bo = ldv<XT, NR>(b, o);
        if (K == VK_SMOOTH) yo = ldv<XT, NR>(xin, o);
        if (K == VK_POST && ag >= 0) yo = ldv<XT, NR>(xc, ag);
    }
    Nb<XT, NR, K> f{dinv, b, xin, xc, agg};
    XT s[NR];
#pragma unroll
    for (int c = 0; c < NR; c++) s[c] = 0;
#pragma unroll
    for (int k = 0; k < PF; k++)
        if (k < cnt) {
            XT a = cvt<XT>(pa[k]);
            Vec<XT, NR> y;
            if constexpr (K == VK_POST)
                y = f.with(pj[k], pd[k], pg[k]);
            else if constexpr (K == VK_RESID0)
                y = f.with(pj[k], pd[k], -1);
            else
                y = f(pj[k]);
#pragma unroll
            for (int c = 0; c < NR; c++) s[c] = fma_rn(a, y.v[c], s[c]);
        }
#pragma unroll 4
    for (int k = PF; k < cnt; k++) {
        XT a = cvt<XT>(ld_stream(A.v + i0 + (int64_t)k * st));
        Vec<XT, NR> y = f(ld_stream(cp + i0 + (int64_t)k * st));
#pragma unroll
        for (int c = 0; c < NR; c++) s[c] = fma_rn(a, y.v[c], s[c]);
    }
#pragma unroll
    for (int c = 0; c < NR; c++) s[c] = lane_reduce<G, XT>(s[c]);
    if (live && lane == 0) {
        if (A.rscale) {
#pragma unroll
            for (int c = 0; c < NR; c++) s[c] = mul_rn(s[c], sc);
        }
        Vec<XT, NR> res;
        if (K == VK_RESID0 || K == VK_RESID) {
#pragma unroll
            for (int c = 0; c < NR; c++) res.v[c] = sub_rn(bo.v[c], s[c]);
        } else {
            Vec<XT, NR> y;
            if (K == VK_POST) {
#pragma unroll
                for (int c = 0; c < NR; c++) y.v[c] = mul_rn(d, bo.v[c]);
                if (ag >= 0) {
#pragma unroll
                    for (int c = 0; c < NR; c++) y.v[c] = add_rn(y.v[c], yo.v[c]);
                }
            } else {
                y = yo;
            }
#pragma unroll
            for (int c = 0; c < NR; c++) res.v[c] = fma_rn(d, sub_rn(bo.v[c], s[c]), y.v[c]);
        }
        st_out<XT, NR>(out, A.out64, o, res);
    }
}

// One launch covers `nvb` blocks of rows (virtual blocks): a grid of at most
// the resident blocks strides over them, so that the blocks of finished batch
// instances cost a flag check each instead of a block launch.
template <int G, class VT, class XT, int K, int NR, int PF>
__global__ void __launch_bounds__(256) k_level(LvlMat<VT> A, const XT *__restrict__ dinv, const XT *__restrict__ b,
                                               const XT *__restrict__ xin, const int32_t *__restrict__ agg,
                                               const XT *__restrict__ xc, XT *__restrict__ out, int64_t nvb) {
    constexpr int GC = G > 0 ? G : 1;  // blocks per 256-row chunk
    for (int64_t i = blockIdx.x; i < nvb; i += gridDim.x)
        level_block<G, VT, XT, K, NR, PF>(live_block(A.lm, i, GC), A, dinv, b, xin, agg, xc, out);
}

// ---- stencil storage (FMT_DIA): the finest level of S~ of a primal system on
// Cartesian instances.  Plane d holds every row's coefficient of its
// neighbour at offset o_d, ascending (3D: -s^2, -s, -1, 0, 1, s, s^2 with s
// the instance's cells per side; 2D: -s, -1, 0, 1, s), zero where the row has
// no such neighbour.  No column indices are stored or loaded, the planes and
// the neighbours' vector entries are read contiguously along each warp, and
// the row's products are added in ascending column order with the absent
// ones contributing exact zeros, so the result is the CSR one-thread-per-row
// result bit for bit.
template <class VT> struct DiaMat {
    int64_t n;
    int64_t stride;         // rows per plane (n padded to a multiple of 32)
    const VT *v;            // [D][stride]
    const int64_t *seg;     // instance row offsets [K + 1]
    const int32_t *side;    // cells per side [K]
    const int4 *ck;         // (first row, last row, cells per side, instance) of each 256-row chunk's
                            // instance; instance -1: the chunk holds rows of two instances
    int K;
    LiveMap lm;
    int *err;               // device error word (a bulk copy that never completed)
    double *out64;          // NULL, or the FP64 vector the rows are written to instead of out
};

// Resident blocks per SM asked of the compiler (measured on the finest level
// of a 256-instance batch): FP32 vectors of up to four columns, six for the
// residual forms (40 registers) and five for the post-smoothing form, which
// holds two gathers per neighbour; FP64 vectors of up to four columns, four;
// wider vectors, no bound.
template <class XT, int K, int NR> constexpr int dia_min_blocks() {
    return NR > 4 ? 1 : sizeof(XT) > 4 ? 4 : K == VK_POST ? 5 : 6;
}

template <class VT, class XT, int K, int NR, int D>
__device__ __forceinline__ void level_dia_block(int64_t vb, const DiaMat<VT> &A, const XT *__restrict__ dinv,
                                                const XT *__restrict__ b, const XT *__restrict__ xin,
                                                const int32_t *__restrict__ agg, const XT *__restrict__ xc,
                                                XT *__restrict__ out) {
    const int64_t r0 = vb * 256, r1 = r0 + 256 < A.n ? r0 + 256 : A.n;
    if (!block_rows_live(A.lm, r0, r1)) return;
    // level rows fit in 32 bits (column indices are 32-bit on every level)
    const int row = (int)r0 + (int)threadIdx.x;
    const bool live = row < A.n;
    // the bounds and grid side of the row's instance from its 256-row chunk
    // (one broadcast load); searched only in a chunk that holds rows of two
    // instances. Neighbour indices are clamped into the instance (an absent
    // neighbour has a zero coefficient), so no instance reads another's rows.
    int lo = 0, hi = 0, sd = 0;
    if (live) {
        const int4 t = __ldg(A.ck + (row >> LIVE_CHUNK_LOG2));
        lo = t.x;
        hi = t.y;
        sd = t.z;
        if (t.w < 0) {
            const int k = seg_find(A.seg, A.K, row);
            lo = (int)A.seg[k];
            hi = (int)A.seg[k + 1] - 1;
            sd = A.side[k];
        }
    }
    int off[D];
    if constexpr (D == 7) {
        off[0] = -sd * sd; off[1] = -sd; off[2] = -1; off[3] = 0; off[4] = 1; off[5] = sd; off[6] = sd * sd;
    } else {
        off[0] = -sd; off[1] = -1; off[2] = 0; off[3] = 1; off[4] = sd;
    }
    // constants of this launch (values, 1/D1, aggregates) before the wait
    constexpr bool FUSED = K == VK_RESID0 || K == VK_POST;
    VT pa[D];
    int32_t pj[D];
    XT pd[FUSED ? D : 1];
    int32_t pg[K == VK_POST ? D : 1];
#pragma unroll
    for (int d = 0; d < D; d++) {
        pa[d] = (VT)0;
        pj[d] = row;
        if (live) {
            pa[d] = ld_stream(A.v + (int64_t)d * A.stride + row);
            if (off[d] != 0 || d != D / 2) pj[d] = min(max(row + off[d], lo), hi);
        }
    }
    if constexpr (FUSED) {
#pragma unroll
        for (int d = 0; d < D; d++)
            if (live) {
                pd[d] = __ldg(dinv + pj[d]);
                if constexpr (K == VK_POST) pg[d] = agg ? __ldg(agg + pj[d]) : -1;
            }
    }
    XT dd = (XT)0;
    int32_t ag = -1;
    if (live) {
        if (K == VK_POST || K == VK_SMOOTH) dd = dinv[row];
        if (K == VK_POST && agg) ag = agg[row];
    }
    mds_pdl_wait();
    mds_pdl_trigger();
    if (!live) return;
    Nb<XT, NR, K> f{dinv, b, xin, xc, agg};
    Vec<XT, NR> bo = ldv<XT, NR>(b, row), yo;
#pragma unroll
    for (int c = 0; c < NR; c++) yo.v[c] = (XT)0;
    if (K == VK_SMOOTH) yo = ldv<XT, NR>(xin, row);
    if (K == VK_POST && ag >= 0) yo = ldv<XT, NR>(xc, ag);
    XT s[NR];
#pragma unroll
    for (int c = 0; c < NR; c++) s[c] = 0;
#pragma unroll
    for (int d = 0; d < D; d++) {
            XT a = cvt<XT>(pa[d]);
            Vec<XT, NR> y;
            if constexpr (K == VK_POST)
                y = f.with(pj[d], pd[d], pg[d]);
            else if constexpr (K == VK_RESID0)
                y = f.with(pj[d], pd[d], -1);
            else
                y = f(pj[d]);
#pragma unroll
            for (int c = 0; c < NR; c++) s[c] = fma_rn(a, y.v[c], s[c]);
        }
    Vec<XT, NR> res;
    if (K == VK_RESID0 || K == VK_RESID) {
#pragma unroll
        for (int c = 0; c < NR; c++) res.v[c] = sub_rn(bo.v[c], s[c]);
    } else {
        Vec<XT, NR> y;
        if (K == VK_POST) {
#pragma unroll
            for (int c = 0; c < NR; c++) y.v[c] = mul_rn(dd, bo.v[c]);
            if (ag >= 0) {
#pragma unroll
                for (int c = 0; c < NR; c++) y.v[c] = add_rn(y.v[c], yo.v[c]);
            }
        } else {
            y = yo;
        }
#pragma unroll
        for (int c = 0; c < NR; c++) res.v[c] = fma_rn(dd, sub_rn(bo.v[c], s[c]), y.v[c]);
    }
    st_out<XT, NR>(out, A.out64, row, res);
}

// grid-stride over the level's 256-row blocks (as k_level)
template <class VT, class XT, int K, int NR, int D>
__global__ void __launch_bounds__(256, dia_min_blocks<XT, K, NR>())
    k_level_dia(DiaMat<VT> A, const XT *__restrict__ dinv, const XT *__restrict__ b, const XT *__restrict__ xin,
                const int32_t *__restrict__ agg, const XT *__restrict__ xc, XT *__restrict__ out, int64_t nvb) {
    for (int64_t i = blockIdx.x; i < nvb; i += gridDim.x)
        level_dia_block<VT, XT, K, NR, D>(live_block(A.lm, i, 1), A, dinv, b, xin, agg, xc, out);
}

// ---- the stencil kernel with bulk-copy staging (MDS_FORMAT_STENCIL_BULK).
// Per 256-row block one thread issues asynchronous bulk copies
// (cp.async.bulk, completion counted in bytes on an mbarrier) of the block's
// D coefficient planes (constant during a solve: issued before the
// dependency wait) and of the window of the vector the neighbours' terms
// read, rows [r0 - s, r1 + s) of the block's instance (after the wait); the
// threads wait on the mbarrier, then read the planes and every neighbour
// inside the window from shared memory (the +-s^2 neighbours of 3D and rows
// outside the window from global memory).  The arithmetic is the direct
// kernel's, so the results are the same bit for bit (measured slower than
// the direct kernel on the finest level of the 256-instance batch: residual
// 262 vs 234 us, post-smoothing 396 vs 345 us; a double-buffered form that
// copies the next row block while computing on the current one, 294 and
// 401 us; the tuner keeps the faster).  The wait is bounded
// (about a second of clock): on expiry the block sets DERR_TIMEOUT, waits
// as long again for its copies and writes NaN to its rows, so the solve
// fails loudly instead of hanging.
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity, long long cycles) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > cycles) return false;
    return true;
}
// dst (shared) <- src (global), bytes a multiple of 16, both 16-byte aligned
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
// order the block's generic-proxy reads of shared memory before the next bulk writes to it
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

constexpr int DIA_WROWS = 512;  // staged window rows: the block's 256 and up to 128 on either side
constexpr long long DIA_WAIT_CYCLES = 2000000000LL;

template <class VT, class XT, int K, int NR, int D>
__global__ void __launch_bounds__(256, dia_min_blocks<XT, K, NR>())
    k_level_dia_bulk(DiaMat<VT> A, const XT *__restrict__ dinv, const XT *__restrict__ b, const XT *__restrict__ xin,
                     const int32_t *__restrict__ agg, const XT *__restrict__ xc, XT *__restrict__ out, int64_t nvb) {
    static_assert((NR * sizeof(XT)) % 16 == 0, "bulk-staged rows must be multiples of 16 bytes");
    constexpr bool FUSED = K == VK_RESID0 || K == VK_POST;
    __shared__ __align__(128) VT sp[D][256];
    __shared__ __align__(128) Vec<XT, NR> sw[DIA_WROWS];
    __shared__ __align__(8) uint64_t bar;
    const XT *gv = FUSED ? b : xin;  // the vector of the neighbours' terms
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    unsigned parity = 0;
    bool first = true;
    for (int64_t i = blockIdx.x; i < nvb; i += gridDim.x) {
        const int64_t vb = live_block(A.lm, i, 1);
        const int64_t r0 = vb * 256, r1 = r0 + 256 < A.n ? r0 + 256 : A.n;
        if (!block_rows_live(A.lm, r0, r1)) continue;  // the same for every thread of the block
        // the block's chunk (256-row blocks are the chunks of the table)
        const int4 tb = __ldg(A.ck + vb);
        int w0 = 0, w1 = 0;  // staged window [w0, w1): one instance, s <= 128
        if (tb.w >= 0 && tb.z >= 0 && tb.z <= (DIA_WROWS - 256) / 2 &&
            (reinterpret_cast<uintptr_t>(gv) & 15) == 0) {
            w0 = max((int)r0 - tb.z, tb.x);
            w1 = min((int)r1 + tb.z, tb.y + 1);
        }
        const unsigned pbytes = (unsigned)(((r1 - r0) * (int64_t)sizeof(VT) + 15) / 16 * 16);
        const unsigned wbytes = w1 > w0 ? (unsigned)((w1 - w0) * (int)sizeof(Vec<XT, NR>)) : 0u;
        if (threadIdx.x == 0) {
            fence_proxy_async_smem();
            mbar_expect_tx(&bar, (unsigned)D * pbytes + wbytes);
#pragma unroll
            for (int d = 0; d < D; d++) bulk_g2s(&sp[d][0], A.v + (int64_t)d * A.stride + r0, pbytes, &bar);
        }
        const int row = (int)r0 + (int)threadIdx.x;
        const bool live = row < A.n;
        int lo = tb.x, hi = tb.y, sd = tb.z;
        if (live && tb.w < 0) {
            const int k = seg_find(A.seg, A.K, row);
            lo = (int)A.seg[k];
            hi = (int)A.seg[k + 1] - 1;
            sd = A.side[k];
        }
        int off[D];
        if constexpr (D == 7) {
            off[0] = -sd * sd; off[1] = -sd; off[2] = -1; off[3] = 0; off[4] = 1; off[5] = sd; off[6] = sd * sd;
        } else {
            off[0] = -sd; off[1] = -1; off[2] = 0; off[3] = 1; off[4] = sd;
        }
        int32_t pj[D];
        XT pd[FUSED ? D : 1];
        int32_t pg[K == VK_POST ? D : 1];
#pragma unroll
        for (int d = 0; d < D; d++) {
            pj[d] = row;
            if (live && (off[d] != 0 || d != D / 2)) pj[d] = min(max(row + off[d], lo), hi);
        }
        if constexpr (FUSED) {
#pragma unroll
            for (int d = 0; d < D; d++)
                if (live) {
                    pd[d] = __ldg(dinv + pj[d]);
                    if constexpr (K == VK_POST) pg[d] = agg ? __ldg(agg + pj[d]) : -1;
                }
        }
        XT dd = (XT)0;
        int32_t ag = -1;
        if (live) {
            if (K == VK_POST || K == VK_SMOOTH) dd = dinv[row];
            if (K == VK_POST && agg) ag = agg[row];
        }
        if (first) {
            mds_pdl_wait();
            mds_pdl_trigger();
            first = false;
        }
        if (threadIdx.x == 0 && wbytes) bulk_g2s(&sw[0], gv + (int64_t)w0 * NR, wbytes, &bar);
        // a block-wide decision: every thread saw the copies complete, or none proceeds
        const bool done = __syncthreads_and(mbar_wait_bounded(&bar, parity, DIA_WAIT_CYCLES) ? 1 : 0) != 0;
        if (!done) {
            if (threadIdx.x == 0) atomicOr(A.err, DERR_TIMEOUT);
            mbar_wait_bounded(&bar, parity, DIA_WAIT_CYCLES);  // the copies still in flight
            if (live) {
                Vec<XT, NR> nan;
#pragma unroll
                for (int c = 0; c < NR; c++) nan.v[c] = (XT)NAN;
                st_out<XT, NR>(out, A.out64, row, nan);
            }
            return;
        }
        parity ^= 1u;
        auto gat = [&](int j) -> Vec<XT, NR> { return j >= w0 && j < w1 ? sw[j - w0] : ldv<XT, NR>(gv, j); };
        if (live) {
            Vec<XT, NR> bo = FUSED ? gat(row) : ldv<XT, NR>(b, row), yo;
#pragma unroll
            for (int c = 0; c < NR; c++) yo.v[c] = (XT)0;
            if (K == VK_SMOOTH) yo = gat(row);
            if (K == VK_POST && ag >= 0) yo = ldv<XT, NR>(xc, ag);
            XT s[NR];
#pragma unroll
            for (int c = 0; c < NR; c++) s[c] = 0;
#pragma unroll
            for (int d = 0; d < D; d++) {
                const XT a = cvt<XT>(sp[d][threadIdx.x]);
                Vec<XT, NR> y = gat(pj[d]);
                if constexpr (FUSED) {
#pragma unroll
                    for (int c = 0; c < NR; c++) y.v[c] = mul_rn(pd[d], y.v[c]);
                    if constexpr (K == VK_POST) {
                        if (pg[d] >= 0) {
                            const Vec<XT, NR> xa = ldv<XT, NR>(xc, pg[d]);
#pragma unroll
                            for (int c = 0; c < NR; c++) y.v[c] = add_rn(y.v[c], xa.v[c]);
                        }
                    }
                }
#pragma unroll
                for (int c = 0; c < NR; c++) s[c] = fma_rn(a, y.v[c], s[c]);
            }
            Vec<XT, NR> res;
            if (K == VK_RESID0 || K == VK_RESID) {
#pragma unroll
                for (int c = 0; c < NR; c++) res.v[c] = sub_rn(bo.v[c], s[c]);
            } else {
                Vec<XT, NR> y;
                if (K == VK_POST) {
#pragma unroll
                    for (int c = 0; c < NR; c++) y.v[c] = mul_rn(dd, bo.v[c]);
                    if (ag >= 0) {
#pragma unroll
                        for (int c = 0; c < NR; c++) y.v[c] = add_rn(y.v[c], yo.v[c]);
                    }
                } else {
                    y = yo;
                }
#pragma unroll
                for (int c = 0; c < NR; c++) res.v[c] = fma_rn(dd, sub_rn(bo.v[c], s[c]), y.v[c]);
            }
            st_out<XT, NR>(out, A.out64, row, res);
        }
        __syncthreads();  // the block's reads of sp and sw before the next block's copies
    }
}

// ---- elementwise kernels (NR interleaved columns; row of entry e = e / NR).
// 1/D1 and the aggregate map are fixed while solving: a thread's first entry
// of them is loaded before the dependency wait.
// One contiguous range of `per` rows per block, so that a block of finished
// batch instances' rows returns at once.
template <class XT, int NR>
__global__ void k_vc_x0(int64_t n, const XT *__restrict__ dinv, const XT *__restrict__ b, XT *__restrict__ x,
                        int64_t per, LiveMap lm) {
    const int64_t r0 = live_block(lm, blockIdx.x, 1) * per, r1 = r0 + per < n ? r0 + per : n;
    if (!block_rows_live(lm, r0, r1)) return;
    int64_t e = r0 * NR + threadIdx.x;
    const XT d0 = e < r1 * NR ? dinv[e / NR] : (XT)0;
    mds_pdl_wait();
    mds_pdl_trigger();
    if (e < r1 * NR) x[e] = mul_rn(d0, b[e]);
    for (e += blockDim.x; e < r1 * NR; e += blockDim.x) x[e] = mul_rn(dinv[e / NR], b[e]);
}

// y_(i,c) += x_c(agg_i, c)
template <class XT, int NR>
__global__ void k_vc_prolong(int64_t n, const int32_t *__restrict__ agg, const XT *__restrict__ xc,
                             XT *__restrict__ y, int64_t per, LiveMap lm) {
    const int64_t r0 = live_block(lm, blockIdx.x, 1) * per, r1 = r0 + per < n ? r0 + per : n;
    if (!block_rows_live(lm, r0, r1)) return;
    int64_t e = r0 * NR + threadIdx.x;
    const int32_t a0 = e < r1 * NR ? agg[e / NR] : -1;
    mds_pdl_wait();
    mds_pdl_trigger();
    if (a0 >= 0) y[e] = add_rn(y[e], xc[(int64_t)a0 * NR + e % NR]);
    for (e += blockDim.x; e < r1 * NR; e += blockDim.x) {
        int32_t a = agg[e / NR];
        if (a >= 0) y[e] = add_rn(y[e], xc[(int64_t)a * NR + e % NR]);
    }
}

// Chebyshev (Saad, Iterative Methods, Alg. 12.1 for D1^-1 A on [lo, hi]):
// first step d = (D1^-1 r) / theta, x = x0 + d; later steps
// d = c1 d + c2 D1^-1 r, x += d.
template <class XT, int NR>
__global__ void k_cheb_first(int64_t n, const XT *__restrict__ dinv, const XT *__restrict__ r,
                             const XT *__restrict__ x0, XT inv_theta, XT *__restrict__ d, XT *__restrict__ x) {
    mds_pdl_entry();
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * NR; e += (int64_t)gridDim.x * blockDim.x) {
        XT di = dinv[e / NR] * r[e] * inv_theta;
        d[e] = di;
        x[e] = x0 ? x0[e] + di : di;
    }
}

template <class XT, int NR>
__global__ void k_cheb_next(int64_t n, const XT *__restrict__ dinv, const XT *__restrict__ r, XT c1, XT c2,
                            XT *__restrict__ d, XT *__restrict__ x) {
    mds_pdl_entry();
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * NR; e += (int64_t)gridDim.x * blockDim.x) {
        XT di = c1 * d[e] + c2 * (dinv[e / NR] * r[e]);
        d[e] = di;
        x[e] += di;
    }
}

// b_c[I] = sum of r over the members of aggregate I (ascending), NR columns.
// The aggregate's member list is fixed while solving: its first entries are
// loaded before the dependency wait.
constexpr int RPRE = 8;
template <class XT, int NR>
__device__ __forceinline__ void restrict_block(int64_t vb, int64_t nc, const int32_t *__restrict__ off,
                                               const int32_t *__restrict__ mem, const XT *__restrict__ r,
                                               XT *__restrict__ bc, const LiveMap &lm) {
    {
        const int64_t r0 = vb * blockDim.x, r1 = r0 + blockDim.x < nc ? r0 + blockDim.x : nc;
        if (!block_rows_live(lm, r0, r1)) return;
    }
    int64_t I = vb * blockDim.x + threadIdx.x;
    int32_t q0 = 0, q1 = 0;
    if (I < nc) {
        q0 = off[I];
        q1 = off[I + 1];
    }
    int32_t pm[RPRE];
#pragma unroll
    for (int k = 0; k < RPRE; k++)
        if (q0 + k < q1) pm[k] = mem[q0 + k];
    mds_pdl_wait();
    mds_pdl_trigger();
    if (I >= nc) return;
    Vec<XT, NR> s;
#pragma unroll
    for (int c = 0; c < NR; c++) s.v[c] = 0;
#pragma unroll
    for (int k = 0; k < RPRE; k++)
        if (q0 + k < q1) {
            Vec<XT, NR> x = ldv<XT, NR>(r, pm[k]);
#pragma unroll
            for (int c = 0; c < NR; c++) s.v[c] += x.v[c];
        }
#pragma unroll 4
    for (int32_t q = q0 + RPRE; q < q1; q++) {
        Vec<XT, NR> x = ldv<XT, NR>(r, mem[q]);
#pragma unroll
        for (int c = 0; c < NR; c++) s.v[c] += x.v[c];
    }
    stv<XT, NR>(bc, I, s);
}

// grid-stride over the aggregates' 256-row blocks (as k_level)
template <class XT, int NR>
__global__ void __launch_bounds__(256) k_vc_restrict(int64_t nc, const int32_t *__restrict__ off,
                                                     const int32_t *__restrict__ mem, const XT *__restrict__ r,
                                                     XT *__restrict__ bc, LiveMap lm, int64_t nvb) {
    for (int64_t i = blockIdx.x; i < nvb; i += gridDim.x) restrict_block<XT, NR>(live_block(lm, i, 1), nc, off, mem, r, bc, lm);
}

// Smoothed aggregation transfers (NR columns): b_c = R r and y += P x_c, one
// thread per output row, entries in CSR order.
template <class XT, int NR>
__global__ void k_sa_restrict(int64_t nc, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                              const XT *__restrict__ v, const XT *__restrict__ r, XT *__restrict__ bc) {
    mds_pdl_entry();
    int64_t I = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nc) return;
    Vec<XT, NR> s;
#pragma unroll
    for (int c = 0; c < NR; c++) s.v[c] = 0;
    for (int32_t p = rp[I]; p < rp[I + 1]; p++) {
        XT a = v[p];
        Vec<XT, NR> x = ldv<XT, NR>(r, ci[p]);
#pragma unroll
        for (int c = 0; c < NR; c++) s.v[c] = fma_rn(a, x.v[c], s.v[c]);
    }
    stv<XT, NR>(bc, I, s);
}

template <class XT, int NR>
__global__ void k_sa_prolong(int64_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                             const XT *__restrict__ v, const XT *__restrict__ xc, XT *__restrict__ y) {
    mds_pdl_entry();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    Vec<XT, NR> s = ldv<XT, NR>(y, i), t;
#pragma unroll
    for (int c = 0; c < NR; c++) t.v[c] = 0;
    for (int32_t p = rp[i]; p < rp[i + 1]; p++) {
        XT a = v[p];
        Vec<XT, NR> x = ldv<XT, NR>(xc, ci[p]);
#pragma unroll
        for (int c = 0; c < NR; c++) t.v[c] = fma_rn(a, x.v[c], t.v[c]);
    }
#pragma unroll
    for (int c = 0; c < NR; c++) s.v[c] = add_rn(s.v[c], t.v[c]);
    stv<XT, NR>(y, i, s);
}

// ---------------------------------------------------------------- host dispatch

template <class VT> static LvlMat<VT> lvl_view(Ctx &c, const Level &L) {
    LvlMat<VT> m{};
    m.n = L.A.nrow;
    m.lm = level_live(c, L);
    m.sigma = L.sell_sigma > 0 ? L.sell_sigma : 1;
    m.rp = L.A.rowp();
    m.ci = L.A.cols();
    m.rscale = L.rscale.p ? L.rscale.as<float>() : nullptr;
    m.out64 = c.level_out64;
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

template <class VT, class XT, int K, int NR, int PF>
static void launch_level_pf(Ctx &c, const Level &L, const XT *dinv, const XT *b, const XT *xin, const int32_t *agg,
                         const XT *xc, XT *out, int64_t nc) {
    LvlMat<VT> m = lvl_view<VT>(c, L);
    int64_t n = L.A.nrow;
    double vb = L.fmt == FMT_SELL ? (sizeof(VT) + 4.0) * (double)L.sell_nnz : (sizeof(VT) + 4.0) * L.A.nnz;
    double xb = sizeof(XT) * (double)NR;
    double bytes = vb + (L.fmt == FMT_SELL ? 8.0 * L.sell_nslice : 4.0 * (n + 1)) + sizeof(XT) * n + 2.0 * xb * n +
                   (K == VK_POST && agg ? 4.0 * n + xb * (double)nc : 0.0) + (L.rscale.p ? 4.0 * n : 0.0) +
                   (K == VK_SMOOTH ? xb * (double)n : 0.0) +
                   (c.level_out64 ? (8.0 - sizeof(XT)) * NR * (double)n : 0.0);
    double flops = NR * (2.0 * L.A.nnz + (K == VK_RESID0 ? n : K == VK_POST ? 5.0 * n : K == VK_SMOOTH ? 3.0 * n : 0.0));
    int cls = !L.timed_level ? KC_NONE : (K == VK_RESID0 || K == VK_RESID) ? KC_VC_RESID : KC_VC_POST;
    if (L.fmt == FMT_DIA) {
        if constexpr (std::is_same<VT, float>::value || std::is_same<VT, double>::value) {
            DiaMat<VT> dm{n, L.dia_stride, L.dia_val.as<VT>(), L.dia_seg.as<int64_t>(), L.dia_side.as<int32_t>(),
                          L.dia_ck.as<int4>(), (int)(L.dia_side.bytes / sizeof(int32_t)), m.lm, c.d_err,
                          c.level_out64};
            // algorithmic bytes: the planes instead of values, columns and row pointers
            bytes = bytes - vb - 4.0 * (n + 1) + (double)L.dia_D * sizeof(VT) * n;
            if constexpr ((NR * sizeof(XT)) % 16 == 0) {
                if (L.dia_bulk) {
                    const int64_t nvb = live_blocks(m.lm, grid_for(n, 256), 1);
                    if (L.dia_D == 7)
                        MDS_LAUNCH_F(c, cls, bytes * m.lm.frac, flops * m.lm.frac, (k_level_dia_bulk<VT, XT, K, NR, 7>),
                                     stride_grid(c, k_level_dia_bulk<VT, XT, K, NR, 7>, 256, nvb), 256, 0, dm, dinv, b,
                                     xin, agg, xc, out, nvb);
                    else
                        MDS_LAUNCH_F(c, cls, bytes * m.lm.frac, flops * m.lm.frac, (k_level_dia_bulk<VT, XT, K, NR, 5>),
                                     stride_grid(c, k_level_dia_bulk<VT, XT, K, NR, 5>, 256, nvb), 256, 0, dm, dinv, b,
                                     xin, agg, xc, out, nvb);
                    return;
                }
            }
            if (L.dia_D == 7)
                MDS_LAUNCH_F(c, cls, bytes * m.lm.frac, flops * m.lm.frac, (k_level_dia<VT, XT, K, NR, 7>),
                             stride_grid(c, k_level_dia<VT, XT, K, NR, 7>, 256, live_blocks(m.lm, grid_for(n, 256), 1)),
                             256, 0, dm, dinv, b, xin, agg, xc, out, live_blocks(m.lm, grid_for(n, 256), 1));
            else
                MDS_LAUNCH_F(c, cls, bytes * m.lm.frac, flops * m.lm.frac, (k_level_dia<VT, XT, K, NR, 5>),
                             stride_grid(c, k_level_dia<VT, XT, K, NR, 5>, 256, live_blocks(m.lm, grid_for(n, 256), 1)),
                             256, 0, dm, dinv, b, xin, agg, xc, out, live_blocks(m.lm, grid_for(n, 256), 1));
            return;
        } else {
            throw Error(MDS_ERR_INVALID, "stencil storage holds FP32 or FP64 values only");
        }
    }
    bytes *= m.lm.frac;  // rows of finished batch instances are skipped
    flops *= m.lm.frac;
    if (L.fmt == FMT_SELL) {
        int64_t rows = L.sell_nslice * L.sell_c;
        const int64_t nvb = live_blocks(m.lm, grid_for(rows, 256), 1);
        MDS_LAUNCH_F(c, cls, bytes, flops, (k_level<0, VT, XT, K, NR, PF>),
                     stride_grid(c, k_level<0, VT, XT, K, NR, PF>, 256, nvb), 256, 0, m, dinv, b, xin, agg, xc, out,
                     nvb);
        return;
    }
    switch (L.G) {
        case 1:
            MDS_LAUNCH_F(c, cls, bytes, flops, (k_level<1, VT, XT, K, NR, PF>),
                         stride_grid(c, k_level<1, VT, XT, K, NR, PF>, 256, live_blocks(m.lm, grid_for(n, 256), 1)),
                         256, 0, m, dinv, b, xin, agg, xc, out, live_blocks(m.lm, grid_for(n, 256), 1));
            break;
        case 2:
            MDS_LAUNCH_F(c, cls, bytes, flops, (k_level<2, VT, XT, K, NR, PF>),
                         stride_grid(c, k_level<2, VT, XT, K, NR, PF>, 256, live_blocks(m.lm, grid_for(n * 2, 256), 2)),
                         256, 0, m, dinv, b, xin, agg, xc, out, live_blocks(m.lm, grid_for(n * 2, 256), 2));
            break;
        case 4:
            MDS_LAUNCH_F(c, cls, bytes, flops, (k_level<4, VT, XT, K, NR, PF>),
                         stride_grid(c, k_level<4, VT, XT, K, NR, PF>, 256, live_blocks(m.lm, grid_for(n * 4, 256), 4)),
                         256, 0, m, dinv, b, xin, agg, xc, out, live_blocks(m.lm, grid_for(n * 4, 256), 4));
            break;
        case 8:
            MDS_LAUNCH_F(c, cls, bytes, flops, (k_level<8, VT, XT, K, NR, PF>),
                         stride_grid(c, k_level<8, VT, XT, K, NR, PF>, 256, live_blocks(m.lm, grid_for(n * 8, 256), 8)),
                         256, 0, m, dinv, b, xin, agg, xc, out, live_blocks(m.lm, grid_for(n * 8, 256), 8));
            break;
        case 16:
            MDS_LAUNCH_F(c, cls, bytes, flops, (k_level<16, VT, XT, K, NR, PF>),
                         stride_grid(c, k_level<16, VT, XT, K, NR, PF>, 256, live_blocks(m.lm, grid_for(n * 16, 256), 16)),
                         256, 0, m, dinv, b, xin, agg, xc, out, live_blocks(m.lm, grid_for(n * 16, 256), 16));
            break;
        default:
            MDS_LAUNCH_F(c, cls, bytes, flops, (k_level<32, VT, XT, K, NR, PF>),
                         stride_grid(c, k_level<32, VT, XT, K, NR, PF>, 256, live_blocks(m.lm, grid_for(n * 32, 256), 32)),
                         256, 0, m, dinv, b, xin, agg, xc, out, live_blocks(m.lm, grid_for(n * 32, 256), 32));
            break;
    }
}

// Launches of at most this many 256-thread blocks use the prefetching form.
constexpr int64_t PREFETCH_MAX_BLOCKS = 1216;

template <class VT, class XT, int K, int NR>
static void launch_level(Ctx &c, const Level &L, const XT *dinv, const XT *b, const XT *xin, const int32_t *agg,
                         const XT *xc, XT *out, int64_t nc) {
    int64_t threads = L.fmt == FMT_SELL ? L.sell_nslice * L.sell_c : L.A.nrow * (int64_t)L.G;
    if ((threads + 255) / 256 <= PREFETCH_MAX_BLOCKS)
        launch_level_pf<VT, XT, K, NR, PREFETCH>(c, L, dinv, b, xin, agg, xc, out, nc);
    else
        launch_level_pf<VT, XT, K, NR, 0>(c, L, dinv, b, xin, agg, xc, out, nc);
}

// Level operations on FP32 vectors whose values are stored in VT = BF16 or
// FP16: defined here, instantiated in their own translation units
// (k_vcycle_bf16.cu, k_vcycle_f16.cu) so that the library compiles in
// parallel.
template <class VT, int K, int NR>
void level_op_lp(Ctx &c, const Level &L, const float *b, const float *xin, const int32_t *agg, const float *xc,
                 float *out, int64_t nc) {
    launch_level<VT, float, K, NR>(c, L, L.dinv.as<float>(), b, xin, agg, xc, out, nc);
}

#define MDS_LP_EACH(X, VT)                                                                            \
    X(VT, 0, 1) X(VT, 0, 2) X(VT, 0, 4) X(VT, 0, 8) X(VT, 1, 1) X(VT, 1, 2) X(VT, 1, 4) X(VT, 1, 8)   \
    X(VT, 2, 1) X(VT, 2, 2) X(VT, 2, 4) X(VT, 2, 8) X(VT, 3, 1) X(VT, 3, 2) X(VT, 3, 4) X(VT, 3, 8)
#define MDS_LP_DECL(VT, K, NR)                                                                             \
    extern template void level_op_lp<VT, K, NR>(Ctx &, const Level &, const float *, const float *,      \
                                                 const int32_t *, const float *, float *, int64_t);
#define MDS_LP_INST(VT, K, NR)                                                                                    \
    template void level_op_lp<VT, K, NR>(Ctx &, const Level &, const float *, const float *, const int32_t *,    \
                                          const float *, float *, int64_t);
#ifndef MDS_VCYCLE_LP_UNIT
MDS_LP_EACH(MDS_LP_DECL, __nv_bfloat16)
MDS_LP_EACH(MDS_LP_DECL, __half)
#endif

template <class XT, int K, int NR>
static void level_op(Ctx &c, const Level &L, const XT *b, const XT *xin, const int32_t *agg, const XT *xc, XT *out,
                     int64_t nc) {
    const XT *dinv = L.dinv.as<XT>();
    if constexpr (std::is_same<XT, double>::value) {
        launch_level<double, XT, K, NR>(c, L, dinv, b, xin, agg, xc, out, nc);
    } else {
        switch (L.vt) {
            case VT_BF16: level_op_lp<__nv_bfloat16, K, NR>(c, L, b, xin, agg, xc, out, nc); break;
            case VT_F16: level_op_lp<__half, K, NR>(c, L, b, xin, agg, xc, out, nc); break;
            default: launch_level<float, XT, K, NR>(c, L, dinv, b, xin, agg, xc, out, nc); break;
        }
    }
}


static unsigned ew_grid(int64_t n) {
    unsigned g = grid_for(n, 256);
    return g > 4096 ? 4096 : g;
}

// Elementwise level kernels: `ew_rows(n)` consecutive rows per block (at
// least 256, at most 8192 blocks), `ew_blocks(n)` blocks.
static int64_t ew_rows(int64_t n) {
    int64_t per = (n + 8191) / 8192;
    return per < 256 ? 256 : per;
}
static unsigned ew_blocks(int64_t n) { return (unsigned)((n + ew_rows(n) - 1) / ew_rows(n)); }
// the same for a launch over the live chunks of lm (256 rows per block)
static int64_t ew_rows(int64_t n, const LiveMap &lm) { return lm.rt ? 256 : ew_rows(n); }
static unsigned ew_blocks(int64_t n, const LiveMap &lm) {
    return lm.rt ? (unsigned)(lm.nch > 0 ? lm.nch : 1) : ew_blocks(n);
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
    const XT *cur = x0;
    for (int s = 0; s < h.sweeps; s++) {
        XT *dst = x;
        if (cur == x) {
            MDS_CUDA(cudaMemcpyAsync(L.t.p, x, sizeof(XT) * (size_t)n * NR, cudaMemcpyDeviceToDevice, c.stream));
            cur = L.t.as<XT>();
        }
        if (h.smoother == MDS_SMOOTHER_L1JACOBI) {
            if (!cur)
            {
                const LiveMap lm = level_live(c, L);
                MDS_LAUNCH(c, KC_NONE, 3.0 * sizeof(XT) * n * NR, (k_vc_x0<XT, NR>), ew_blocks(n, lm), 256, 0, n,
                           dinv, b, dst, ew_rows(n, lm), lm);
            }
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
            double rho_old = rho;
            for (int j = 2; j <= h.cheb_degree; j++) {
                const double rho_new = 1.0 / (2.0 * sigma - rho_old);
                level_op<XT, VK_RESID, NR>(c, L, b, dst, nullptr, nullptr, r, 0);
                MDS_LAUNCH(c, KC_NONE, 0, (k_cheb_next<XT, NR>), ew_grid(n * NR), 256, 0, n, dinv, r,
                           (XT)(rho_new * rho_old), (XT)(2.0 * rho_new / delta), d, dst);
                rho_old = rho_new;
            }
        }
        cur = dst;
    }
}

// ---------------------------------------------------------------- coarse tail
// The coarse end of the hierarchy (every level at most as many rows as the
// cluster has threads, fused L1-Jacobi form, values of the vector type) runs
// as one kernel on one thread block cluster: the phases of the down sweep
// (residual, restriction), the dense coarsest solve and the up sweep
// (prolongation + post-smoothing) are separated by cluster barriers instead
// of kernel boundaries.  The same arithmetic as the per-level kernels (G
// lanes per row); vectors written inside the kernel are read through L2
// (ld.global.cg).
constexpr int TAIL_MAX = 8;
constexpr int TAIL_THREADS = 512;  // a level takes at most one row per thread of the cluster

template <class XT> struct TailLevel {
    int64_t n, nc;
    const int32_t *rp, *ci;
    const XT *v;
    const float *rscale;
    const XT *dinv;
    XT *b, *x, *r;
    const int32_t *agg, *moff, *mem;  // agg == NULL: no coarser level
};
template <class XT> struct TailArgs {
    int nlev;        // levels lv[0 .. nlev-1]; lv[nlev] holds the coarsest b, x when dense
    int dense;
    int64_t nd;
    const double *M;  // dense inverse of the coarsest matrix
    TailLevel<XT> lv[TAIL_MAX + 1];
};

__device__ __forceinline__ void cluster_arrive() {
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Lanes per row for a level of n rows on T threads: the largest power of two
// up to 32 that still gives every row its lanes in one pass.
__device__ __forceinline__ int tail_lanes(int64_t n, int64_t T) {
    int G = 1;
    while (G < 32 && (int64_t)(2 * G) * n <= T) G *= 2;
    return G;
}

enum { TP_RES = 0, TP_RST = 1, TP_DENSE = 2, TP_POST = 3 };
constexpr int TPF = 8;  // entries of a row (or members, or dense columns) loaded ahead

// The constants one thread needs in a phase (matrix row share, 1/D1, the
// aggregate map, member lists, rows of the dense inverse), loaded between the
// barrier arrival that ends the previous phase and the wait that starts this
// one.
template <class XT> struct TailPre {
    int64_t i;          // row (or aggregate) of this thread, -1 = none
    int32_t p, p1;      // entry range [p, p1) with stride G
    XT v[TPF];
    XT dj[TPF];
    int32_t j[TPF];
    int32_t aj[TPF];
    XT di, sc;
    int32_t ai;
    double m[TPF];      // dense inverse row entries
};

template <class XT> __device__ __forceinline__ void tail_phase(const TailArgs<XT> &a, int ph, int &kind, int &li) {
    const int ndown = a.dense ? a.nlev : a.nlev - 1;
    if (ph < 2 * ndown) {
        kind = ph & 1 ? TP_RST : TP_RES;
        li = ph >> 1;
    } else if (a.dense && ph == 2 * ndown) {
        kind = TP_DENSE;
        li = a.nlev;
    } else {
        kind = TP_POST;
        li = a.nlev - 1 - (ph - 2 * ndown - (a.dense ? 1 : 0));
    }
}

template <class XT>
__device__ __forceinline__ void tail_prefetch(const TailArgs<XT> &a, int kind, int li, int64_t t0, int64_t T,
                                              TailPre<XT> &q) {
    q.i = -1;
    if (kind == TP_RES || kind == TP_POST) {
        const TailLevel<XT> &L = a.lv[li];
        const int G = tail_lanes(L.n, T);
        const int64_t i = t0 / G;
        if (i >= L.n) return;
        q.i = i;
        q.p = L.rp[i] + (int32_t)(t0 % G);
        q.p1 = L.rp[i + 1];
        const bool coarse = kind == TP_POST && L.agg;
#pragma unroll
        for (int k = 0; k < TPF; k++) {
            int32_t idx = q.p + k * G;
            if (idx < q.p1) {
                q.v[k] = L.v[idx];
                q.j[k] = L.ci[idx];
            }
        }
#pragma unroll
        for (int k = 0; k < TPF; k++) {
            if (q.p + k * G < q.p1) {
                q.dj[k] = L.dinv[q.j[k]];
                q.aj[k] = coarse ? L.agg[q.j[k]] : -1;
            }
        }
        q.sc = L.rscale ? (XT)L.rscale[i] : (XT)1;
        q.di = L.dinv[i];
        q.ai = coarse ? L.agg[i] : -1;
    } else if (kind == TP_RST) {
        const TailLevel<XT> &L = a.lv[li];
        if (t0 >= L.nc) return;
        q.i = t0;
        q.p = L.moff[t0];
        q.p1 = L.moff[t0 + 1];
#pragma unroll
        for (int k = 0; k < TPF; k++)
            if (q.p + k < q.p1) q.j[k] = L.mem[q.p + k];
    } else {  // dense: the first row of this warp
        const int64_t row = t0 >> 5;
        const int lane = (int)(t0 & 31);
        if (row >= a.nd) return;
        q.i = row;
#pragma unroll
        for (int k = 0; k < TPF; k++) {
            int64_t col = lane + 32 * (int64_t)k;
            q.m[k] = col < a.nd ? a.M[row * a.nd + col] : 0.0;
        }
    }
}

template <class XT, int NR>
__device__ __forceinline__ void tail_run(const TailArgs<XT> &a, int kind, int li, int64_t t0, int64_t T,
                                         const TailPre<XT> &q) {
    if (kind == TP_RES || kind == TP_POST) {
        const TailLevel<XT> &L = a.lv[li];
        const int G = tail_lanes(L.n, T);
        const XT *xc = kind == TP_POST && L.agg ? a.lv[li + 1].x : nullptr;
        XT s[NR];
#pragma unroll
        for (int c = 0; c < NR; c++) s[c] = 0;
        if (q.i >= 0) {
#pragma unroll
            for (int k = 0; k < TPF; k++) {
                if (q.p + k * G < q.p1) {
#pragma unroll
                    for (int c = 0; c < NR; c++) {
                        XT yj = mul_rn(q.dj[k], __ldcg(L.b + (int64_t)q.j[k] * NR + c));
                        if (kind == TP_POST && q.aj[k] >= 0) yj = add_rn(yj, __ldcg(xc + (int64_t)q.aj[k] * NR + c));
                        s[c] = fma_rn(q.v[k], yj, s[c]);
                    }
                }
            }
            for (int32_t idx = q.p + TPF * G; idx < q.p1; idx += G) {
                XT av = L.v[idx];
                int32_t j = L.ci[idx];
                XT dj = L.dinv[j];
                int32_t aj = xc ? L.agg[j] : -1;
#pragma unroll
                for (int c = 0; c < NR; c++) {
                    XT yj = mul_rn(dj, __ldcg(L.b + (int64_t)j * NR + c));
                    if (aj >= 0) yj = add_rn(yj, __ldcg(xc + (int64_t)aj * NR + c));
                    s[c] = fma_rn(av, yj, s[c]);
                }
            }
        }
#pragma unroll
        for (int c = 0; c < NR; c++)
            for (int o = G / 2; o > 0; o >>= 1) s[c] += __shfl_down_sync(0xffffffffu, s[c], o, G);
        if (q.i >= 0 && t0 % G == 0) {
            const int64_t i = q.i;
#pragma unroll
            for (int c = 0; c < NR; c++) {
                XT bi = __ldcg(L.b + i * NR + c);
                XT sv = L.rscale ? mul_rn(s[c], q.sc) : s[c];
                if (kind == TP_RES) {
                    __stcg(L.r + i * NR + c, sub_rn(bi, sv));
                } else {
                    XT yi = mul_rn(q.di, bi);
                    if (q.ai >= 0) yi = add_rn(yi, __ldcg(xc + (int64_t)q.ai * NR + c));
                    __stcg(L.x + i * NR + c, fma_rn(q.di, sub_rn(bi, sv), yi));
                }
            }
        }
    } else if (kind == TP_RST) {
        if (q.i < 0) return;
        const TailLevel<XT> &L = a.lv[li];
        XT *bc = a.lv[li + 1].b;
        XT s[NR];
#pragma unroll
        for (int c = 0; c < NR; c++) s[c] = 0;
#pragma unroll
        for (int k = 0; k < TPF; k++)
            if (q.p + k < q.p1)
#pragma unroll
                for (int c = 0; c < NR; c++) s[c] += __ldcg(L.r + (int64_t)q.j[k] * NR + c);
        for (int32_t idx = q.p + TPF; idx < q.p1; idx++) {
            int64_t m = L.mem[idx];
#pragma unroll
            for (int c = 0; c < NR; c++) s[c] += __ldcg(L.r + m * NR + c);
        }
#pragma unroll
        for (int c = 0; c < NR; c++) __stcg(bc + q.i * NR + c, s[c]);
    } else {  // dense x = M b, one warp per row
        const XT *bd = a.lv[a.nlev].b;
        XT *xd = a.lv[a.nlev].x;
        const int lane = (int)(t0 & 31);
        const int64_t nw = T >> 5;
        for (int64_t row = t0 >> 5; row < a.nd; row += nw) {
            const bool first = row == (t0 >> 5);
            double s[NR];
#pragma unroll
            for (int c = 0; c < NR; c++) s[c] = 0.0;
#pragma unroll
            for (int k = 0; k < TPF; k++) {
                int64_t col = lane + 32 * (int64_t)k;
                if (col < a.nd) {
                    double m = first ? q.m[k] : a.M[row * a.nd + col];
#pragma unroll
                    for (int c = 0; c < NR; c++) s[c] += m * (double)__ldcg(bd + col * NR + c);
                }
            }
            for (int64_t col = lane + 32 * TPF; col < a.nd; col += 32) {
                double m = a.M[row * a.nd + col];
#pragma unroll
                for (int c = 0; c < NR; c++) s[c] += m * (double)__ldcg(bd + col * NR + c);
            }
#pragma unroll
            for (int c = 0; c < NR; c++)
                for (int o = 16; o > 0; o >>= 1) s[c] += __shfl_down_sync(0xffffffffu, s[c], o);
            if (lane == 0)
#pragma unroll
                for (int c = 0; c < NR; c++) __stcg(xd + row * NR + c, (XT)s[c]);
        }
    }
}

// Phases: down sweep (residual, restriction per level), dense solve, up sweep
// (prolongation + post-smoothing per level).  Between phases: arrive at the
// cluster barrier (release), load the next phase's constants, wait (acquire).
template <class XT, int NR>
__global__ void __launch_bounds__(TAIL_THREADS) k_vcycle_tail(TailArgs<XT> a) {
    const int64_t T = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int ndown = a.dense ? a.nlev : a.nlev - 1;
    const int nph = 2 * ndown + (a.dense ? 1 : 0) + a.nlev;
    TailPre<XT> q;
    int kind, li;
    tail_phase(a, 0, kind, li);
    tail_prefetch(a, kind, li, t0, T, q);
    mds_pdl_wait();
    mds_pdl_trigger();
    for (int ph = 0; ph < nph; ph++) {
        tail_run<XT, NR>(a, kind, li, t0, T, q);
        if (ph + 1 < nph) {
            cluster_arrive();
            tail_phase(a, ph + 1, kind, li);
            tail_prefetch(a, kind, li, t0, T, q);
            cluster_wait();
        }
    }
}

// Cluster size of the tail kernel: 16 blocks when the device schedules such
// clusters, else 8 (the portable size).
template <class XT, int NR> static int tail_cluster(Ctx &c) {
    static int cl[64] = {};
    int &v = cl[c.device & 63];
    if (v) return v;
    v = 8;
    if (cudaFuncSetAttribute(k_vcycle_tail<XT, NR>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
        cudaSuccess) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(16);
        cfg.blockDim = dim3(TAIL_THREADS);
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 16;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, k_vcycle_tail<XT, NR>, &cfg) == cudaSuccess && n > 0) v = 16;
    }
    cudaGetLastError();
    return v;
}

// First level of the coarse tail (levels l0 .. last run in k_vcycle_tail), or
// -1 when the hierarchy has no eligible tail.
template <class XT> static int tail_start(const Hierarchy &h, int64_t max_rows) {
    const int last = (int)h.lv.size() - 1;
    const int top = h.dense ? last - 1 : last;  // smoothed levels
    if (h.smoother != MDS_SMOOTHER_L1JACOBI || h.sweeps != 1 || top < 0 || h.diagonal) return -1;
    const int want_vt = std::is_same<XT, double>::value ? VT_F64 : VT_F32;
    int l0 = -1;
    for (int l = top; l >= 0 && top - l + 1 <= TAIL_MAX; l--) {
        const Level &L = h.lv[l];
        if (L.A.nrow > max_rows || L.smoothed || L.vt != want_vt) break;
        l0 = l;
    }
    return l0;
}

// Launches the tail kernel; false (nothing launched, tail disabled for the
// hierarchy) when the device refuses the cluster launch.
template <class XT, int NR>
static bool vcycle_tail(Ctx &c, Hierarchy &h, int l0, const XT *b, XT *x) {
    const int last = (int)h.lv.size() - 1;
    const int top = h.dense ? last - 1 : last;
    TailArgs<XT> a{};
    a.nlev = top - l0 + 1;
    a.dense = h.dense ? 1 : 0;
    a.nd = h.nd;
    a.M = h.dense ? h.Ainv.as<double>() : nullptr;
    double bytes = 0.0;
    for (int k = 0; k <= a.nlev && l0 + k <= last; k++) {
        Level &L = h.lv[l0 + k];
        TailLevel<XT> &t = a.lv[k];
        t.n = L.A.nrow;
        t.b = k == 0 ? const_cast<XT *>(b) : L.b.as<XT>();
        t.x = k == 0 ? x : L.x.as<XT>();
        if (k == a.nlev) break;  // coarsest dense level: vectors only
        t.nc = L.has_coarse ? L.nc : 0;
        t.rp = L.A.rowp();
        t.ci = L.A.cols();
        t.v = std::is_same<XT, double>::value ? (const XT *)L.A.vals() : L.vals_lp.as<XT>();
        t.rscale = L.rscale.p ? L.rscale.as<float>() : nullptr;
        t.dinv = L.dinv.as<XT>();
        t.r = L.r.as<XT>();
        t.agg = L.has_coarse ? L.agg.as<int32_t>() : nullptr;
        t.moff = L.has_coarse ? L.mem_off.as<int32_t>() : nullptr;
        t.mem = L.has_coarse ? L.mem.as<int32_t>() : nullptr;
        bytes += 2.0 * (sizeof(XT) + 4.0) * L.A.nnz + 8.0 * (t.n + 1) + sizeof(XT) * NR * 8.0 * t.n;
    }
    if (a.dense) bytes += 8.0 * (double)h.nd * h.nd;
    const int cl = tail_cluster<XT, NR>(c);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cl);
    cfg.blockDim = dim3(TAIL_THREADS);
    cfg.stream = c.stream;
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cl;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[1].val.programmaticStreamSerializationAllowed = c.pdl && !c.setup_phase ? 1 : 0;
    cfg.attrs = at;
    cfg.numAttrs = 2;
    KTimer kt(c, KC_NONE, bytes);
    cudaError_t e = cudaLaunchKernelEx(&cfg, k_vcycle_tail<XT, NR>, a);
    if (e != cudaSuccess) {
        cudaGetLastError();
        h.use_tail = false;
        return false;
    }
    c.post_launch();
    return true;
}


// The level's last operation writes its rows to z64 in FP64 instead of x
// (for the duration of one level operation).
struct Out64Scope {
    Ctx &c;
    Out64Scope(Ctx &cc, double *p) : c(cc) { c.level_out64 = p; }
    ~Out64Scope() { c.level_out64 = nullptr; }
};

// One V-cycle from level l.  z64 (top level only): its last operation writes
// FP64 rows there instead of x where it is one level kernel; returns whether
// it did (false: x holds the result).
template <class XT, int NR>
static bool vcycle_level(Ctx &c, Hierarchy &h, int l, const XT *b, XT *x, double *z64 = nullptr) {
    Level &L = h.lv[l];
    int last = (int)h.lv.size() - 1;
    if (l == last && h.dense) {
        dense_apply(c, h.db, h.Ainv.as<double>(), NR, b, x, h.K > 1 ? c.live : nullptr);
        return false;
    }
    if (l == last && h.diagonal) {  // no couplings: exact x = b / a_ii
        const int64_t nd = L.A.nrow;
        const LiveMap lm = level_live(c, L);
        MDS_LAUNCH(c, KC_NONE, 3.0 * sizeof(XT) * nd * NR, (k_vc_x0<XT, NR>), ew_blocks(nd, lm), 256, 0, nd,
                   L.dinv.as<XT>(), b, x, ew_rows(nd, lm), lm);
        return false;
    }
    if (h.use_tail && l == tail_start<XT>(h, (int64_t)tail_cluster<XT, NR>(c) * TAIL_THREADS) &&
        vcycle_tail<XT, NR>(c, h, l, b, x))
        return false;
    int64_t n = L.A.nrow;
    XT *r = L.r.as<XT>();
    double rbytes = 4.0 * (L.nc + 1) + 4.0 * n + sizeof(XT) * NR * (double)(n + L.nc);
    // Fused form (y = D1^-1 b [+ P x_c] formed per neighbour, no stored
    // iterate): FP32 levels, and FP64 levels small enough to be bound by
    // latency rather than by the FP64 units (the fused form spends one to two
    // more FP64 operations per nonzero and saves two launches per level),
    // unless the level takes the stored form (chosen, or timed faster: on
    // levels with many entries per row the fused post-smoothing's gathers of
    // b, 1/D1, the aggregate and x_c per neighbour cost more than storing y)
    bool fused = h.smoother == MDS_SMOOTHER_L1JACOBI && h.sweeps == 1 && !L.smoothed &&
                 (!std::is_same<XT, double>::value || n <= FUSE_FP64_ROWS) && !L.stored;
    if (fused) {
        if (L.has_coarse) {
            Level &C = h.lv[l + 1];
            const LiveMap lmc = level_live(c, C);
            level_op<XT, VK_RESID0, NR>(c, L, b, nullptr, nullptr, nullptr, r, 0);
            MDS_LAUNCH(c, L.timed_level ? KC_VC_RESTRICT : KC_NONE, rbytes * level_live(c, L).frac,
                       (k_vc_restrict<XT, NR>), stride_grid(c, k_vc_restrict<XT, NR>, 256, live_blocks(lmc, grid_for(L.nc, 256), 1)),
                       256, 0, L.nc, L.mem_off.as<int32_t>(), L.mem.as<int32_t>(), r, C.b.as<XT>(), lmc,
                       live_blocks(lmc, grid_for(L.nc, 256), 1));
            vcycle_level<XT, NR>(c, h, l + 1, C.b.as<XT>(), C.x.as<XT>());
            Out64Scope o64(c, z64);
            level_op<XT, VK_POST, NR>(c, L, b, nullptr, L.agg.as<int32_t>(), C.x.as<XT>(), x, L.nc);
        } else {
            Out64Scope o64(c, z64);
            level_op<XT, VK_POST, NR>(c, L, b, nullptr, nullptr, nullptr, x, 0);
        }
        return z64 != nullptr;
    }
    XT *y = L.y.as<XT>();
    smooth_stored<XT, NR>(c, h, L, b, nullptr, y);  // y = S(0; b)
    if (L.has_coarse) {
        Level &C = h.lv[l + 1];
        if (L.smoothed) {
            level_op<XT, VK_RESID, NR>(c, L, b, y, nullptr, nullptr, r, 0);
            const XT *rv = std::is_same<XT, double>::value ? (const XT *)L.R.vals() : L.Rv_lp.as<XT>();
            const XT *pv = std::is_same<XT, double>::value ? (const XT *)L.P.vals() : L.Pv_lp.as<XT>();
            double tb = (sizeof(XT) + 4.0) * L.R.nnz + 4.0 * (L.nc + 1) + sizeof(XT) * NR * (double)(n + L.nc);
            MDS_LAUNCH(c, L.timed_level ? KC_VC_RESTRICT : KC_NONE, tb, (k_sa_restrict<XT, NR>), grid_for(L.nc, 256), 256, 0, L.nc, L.R.rowp(),
                       L.R.cols(), rv, r, C.b.as<XT>());
            vcycle_level<XT, NR>(c, h, l + 1, C.b.as<XT>(), C.x.as<XT>());
            MDS_LAUNCH(c, KC_NONE, tb + sizeof(XT) * NR * (double)n, (k_sa_prolong<XT, NR>), grid_for(n, 256), 256, 0,
                       n, L.P.rowp(), L.P.cols(), pv, C.x.as<XT>(), y);
        } else {
            const LiveMap lmc = level_live(c, C);
            level_op<XT, VK_RESID, NR>(c, L, b, y, nullptr, nullptr, r, 0);
            MDS_LAUNCH(c, L.timed_level ? KC_VC_RESTRICT : KC_NONE, rbytes * level_live(c, L).frac,
                       (k_vc_restrict<XT, NR>), stride_grid(c, k_vc_restrict<XT, NR>, 256, live_blocks(lmc, grid_for(L.nc, 256), 1)),
                       256, 0, L.nc, L.mem_off.as<int32_t>(), L.mem.as<int32_t>(), r, C.b.as<XT>(), lmc,
                       live_blocks(lmc, grid_for(L.nc, 256), 1));
            vcycle_level<XT, NR>(c, h, l + 1, C.b.as<XT>(), C.x.as<XT>());
            const LiveMap lml = level_live(c, L);
            MDS_LAUNCH(c, KC_NONE, 3.0 * sizeof(XT) * n * NR, (k_vc_prolong<XT, NR>), ew_blocks(n, lml), 256, 0, n,
                       L.agg.as<int32_t>(), C.x.as<XT>(), y, ew_rows(n, lml), lml);
        }
    }
    if (z64 && h.smoother == MDS_SMOOTHER_L1JACOBI && h.sweeps == 1) {
        // x = S(y; b) is one smoothing kernel
        Out64Scope o64(c, z64);
        level_op<XT, VK_SMOOTH, NR>(c, L, b, y, nullptr, nullptr, x, 0);
        return true;
    }
    smooth_stored<XT, NR>(c, h, L, b, y, x);  // x = S(y; b)
    return false;
}

template <class XT>
static bool vcycle_nr(Ctx &c, Hierarchy &h, const XT *b, XT *x, int nr, double *z64 = nullptr) {
    switch (nr) {
        case 1: return vcycle_level<XT, 1>(c, h, 0, b, x, z64);
        case 2: return vcycle_level<XT, 2>(c, h, 0, b, x, z64);
        case 4: return vcycle_level<XT, 4>(c, h, 0, b, x, z64);
        case 8: return vcycle_level<XT, 8>(c, h, 0, b, x, z64);
        default: throw Error(MDS_ERR_INVALID, "V-cycle column count must be 1, 2, 4 or 8");
    }
}

// xc == NULL: the stored-residual kernel; otherwise the pair of fused
// kernels the V-cycle runs on a level with a coarser one (the residual with
// y = D1^-1 b formed per neighbour, and the post-smoothing with y = D1^-1 b +
// P x_c formed per neighbour, x_c = xc), or with `stored` the four launches
// of the stored form in their place (y = D1^-1 b, the residual, y += P x_c,
// the smoothing from y).
template <class XT, int NR> static float time_level_nr(Ctx &c, const Level &L, const XT *xc, bool stored) {
    cudaEvent_t e0, e1;
    MDS_CUDA(cudaEventCreate(&e0));
    MDS_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    for (int rep = 0; rep < 4; rep++) {
        MDS_CUDA(cudaEventRecord(e0, c.stream));
        if (xc && stored) {
            const int64_t n = L.A.nrow;
            const LiveMap lm = level_live(c, L);
            XT *y = L.y.as<XT>();
            MDS_LAUNCH(c, KC_NONE, 0, (k_vc_x0<XT, NR>), ew_blocks(n, lm), 256, 0, n, L.dinv.as<XT>(), L.b.as<XT>(), y,
                       ew_rows(n, lm), lm);
            level_op<XT, VK_RESID, NR>(c, L, L.b.as<XT>(), y, nullptr, nullptr, L.r.as<XT>(), 0);
            MDS_LAUNCH(c, KC_NONE, 0, (k_vc_prolong<XT, NR>), ew_blocks(n, lm), 256, 0, n, L.agg.as<int32_t>(), xc, y,
                       ew_rows(n, lm), lm);
            level_op<XT, VK_SMOOTH, NR>(c, L, L.b.as<XT>(), y, nullptr, nullptr, L.x.as<XT>(), 0);
        } else if (xc) {
            level_op<XT, VK_RESID0, NR>(c, L, L.b.as<XT>(), nullptr, nullptr, nullptr, L.r.as<XT>(), 0);
            level_op<XT, VK_POST, NR>(c, L, L.b.as<XT>(), nullptr, L.agg.as<int32_t>(), xc, L.x.as<XT>(), L.nc);
        } else {
            level_op<XT, VK_RESID, NR>(c, L, L.b.as<XT>(), L.x.as<XT>(), nullptr, nullptr, L.r.as<XT>(), 0);
        }
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

// Time the level's kernels in its current storage with nr interleaved
// columns (best of three after a warm-up launch).
template <class XT> static float time_level(Ctx &c, const Level &L, int nr, const void *xc, bool stored) {
    const XT *x = (const XT *)xc;
    switch (nr) {
        case 8: return time_level_nr<XT, 8>(c, L, x, stored);
        case 4: return time_level_nr<XT, 4>(c, L, x, stored);
        case 2: return time_level_nr<XT, 2>(c, L, x, stored);
        default: return time_level_nr<XT, 1>(c, L, x, stored);
    }
}

}  // namespace mds
