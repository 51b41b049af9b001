// CSR SpMV kernel with G lanes per row (G in {2, 4, 8, 16, 32}).
#pragma once
#include <cstdint>

namespace mds {

template <class T> __device__ __forceinline__ double to_d(T v) { return (double)v; }

// MODE 0: y = A x;  MODE 1: y = r - A x.  Accumulation in FP64.  NR
// right-hand sides interleaved (entry (i, c) at i * NR + c): each matrix entry
// is read once for all NR columns.
template <int G, class VT, class XT, class OT, int MODE, int NR>
__global__ void __launch_bounds__(256) k_spmv_csr(int64_t nrow, const int32_t *__restrict__ rp,
                                                   const int32_t *__restrict__ ci, const VT *__restrict__ v,
                                                   const XT *__restrict__ x, const double *__restrict__ r,
                                                   OT *__restrict__ y, LiveMap lm) {
    // the block's rows: block b of the launch, or of its live chunks only
    const int64_t vb = live_block(lm, blockIdx.x, G);
    {
        const int64_t r0 = vb * (256 / G), r1 = r0 + 256 / G < nrow ? r0 + 256 / G : nrow;
        if (!block_rows_live(lm, r0, r1)) return;
    }
    mds_pdl_entry();
    int64_t t = vb * blockDim.x + threadIdx.x;
    int64_t row = t / G;
    int lane = (int)(t % G);
    double s[NR];
#pragma unroll
    for (int c = 0; c < NR; c++) s[c] = 0.0;
    if (row < nrow) {
        int32_t p0 = rp[row], p1 = rp[row + 1];
#pragma unroll 4
        for (int32_t p = p0 + lane; p < p1; p += G) {
            double a = to_d(__ldcs(v + p));
            int64_t j = __ldcs(ci + p);
#pragma unroll
            for (int c = 0; c < NR; c++) s[c] += a * to_d(__ldg(x + j * NR + c));
        }
    }
#pragma unroll
    for (int c = 0; c < NR; c++)
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) s[c] += __shfl_down_sync(0xffffffffu, s[c], o, G);
    if (row < nrow && lane == 0) {
#pragma unroll
        for (int c = 0; c < NR; c++) {
            if (MODE == 1)
                y[row * NR + c] = (OT)(r[row * NR + c] - s[c]);
            else
                y[row * NR + c] = (OT)s[c];
        }
    }
}

}  // namespace mds
