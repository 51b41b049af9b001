// Primitives: scan, fills, precision casts, CSR SpMV.
#include <algorithm>

#include "conv.cuh"
#include "internal.cuh"
#include "spmv.cuh"

namespace mds {

// ---------------------------------------------------------------- scan

constexpr int SCAN_BLOCK = 1024;

__global__ void k_scan_block(const int32_t *__restrict__ cnt, int64_t n, int32_t *__restrict__ out,
                             int64_t *__restrict__ bsum) {
    mds_pdl_entry();
    __shared__ int64_t wsum[32];
    int64_t i = (int64_t)blockIdx.x * SCAN_BLOCK + threadIdx.x;
    int64_t v = i < n ? (int64_t)cnt[i] : 0;
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t s = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t t = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o) s += t;
    }
    if (lane == 31) wsum[w] = s;
    __syncthreads();
    if (w == 0) {
        int64_t ws = wsum[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t t = __shfl_up_sync(0xffffffffu, ws, o);
            if (lane >= o) ws += t;
        }
        wsum[lane] = ws;
    }
    __syncthreads();
    int64_t incl = s + (w > 0 ? wsum[w - 1] : 0);
    if (i < n) out[i] = (int32_t)(incl - v);  // block-local exclusive
    if (threadIdx.x == SCAN_BLOCK - 1) bsum[blockIdx.x] = incl;
}

// exclusive scan of the block sums in place (one block, chunks of 1024)
__global__ void k_scan_bsums(int64_t *__restrict__ bsum, int64_t nb, int64_t *__restrict__ total) {
    mds_pdl_entry();
    __shared__ int64_t wsum[32];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int64_t base = 0; base < nb; base += SCAN_BLOCK) {
        int64_t i = base + threadIdx.x;
        int64_t v = i < nb ? bsum[i] : 0;
        int64_t s = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t t = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += t;
        }
        if (lane == 31) wsum[w] = s;
        __syncthreads();
        if (w == 0) {
            int64_t ws = wsum[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int64_t t = __shfl_up_sync(0xffffffffu, ws, o);
                if (lane >= o) ws += t;
            }
            wsum[lane] = ws;
        }
        __syncthreads();
        int64_t incl = s + (w > 0 ? wsum[w - 1] : 0);
        if (i < nb) bsum[i] = carry + incl - v;
        __syncthreads();
        if (threadIdx.x == SCAN_BLOCK - 1) carry += incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void k_scan_add(int32_t *__restrict__ out, int64_t n, const int64_t *__restrict__ bsum,
                           const int64_t *__restrict__ total) {
    mds_pdl_entry();
    int64_t i = (int64_t)blockIdx.x * SCAN_BLOCK + threadIdx.x;
    if (i < n) out[i] = (int32_t)((int64_t)out[i] + bsum[blockIdx.x]);
    if (i == n) out[n] = (int32_t)*total;
}

int64_t scan_counts(Ctx &c, const int32_t *cnt, int32_t *out, int64_t n) {
    int64_t nb = (n + SCAN_BLOCK - 1) / SCAN_BLOCK;
    if (nb < 1) nb = 1;
    Buf bs(&c, sizeof(int64_t) * (size_t)(nb + 1));
    int64_t *bsum = bs.as<int64_t>();
    int64_t *total = bsum + nb;
    MDS_LAUNCH(c, KC_NONE, 0, k_scan_block, (unsigned)nb, SCAN_BLOCK, 0, cnt, n, out, bsum);
    MDS_LAUNCH(c, KC_NONE, 0, k_scan_bsums, 1, SCAN_BLOCK, 0, bsum, nb, total);
    // one extra thread writes out[n]
    int64_t nb2 = (n + 1 + SCAN_BLOCK - 1) / SCAN_BLOCK;
    MDS_LAUNCH(c, KC_NONE, 0, k_scan_add, (unsigned)nb2, SCAN_BLOCK, 0, out, n, bsum, total);
    int64_t t = c.read(total);
    MDS_REQUIRE(t <= INT32_MAX, MDS_ERR_INVALID, "sparse matrix exceeds 2^31-1 nonzeros");
    return t;
}

// ---------------------------------------------------------------- fills, casts

template <class T>
__global__ void k_fill(T *__restrict__ p, T v, int64_t n) {
    mds_pdl_entry();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

void fill_i32(Ctx &c, int32_t *p, int32_t v, int64_t n) {
    if (n <= 0) return;
    MDS_LAUNCH(c, KC_NONE, 0, k_fill<int32_t>, grid_for(n, 256) > 4096 ? 4096 : grid_for(n, 256), 256, 0, p, v, n);
}

void fill_f64(Ctx &c, double *p, double v, int64_t n) {
    if (n <= 0) return;
    MDS_LAUNCH(c, KC_NONE, 0, k_fill<double>, grid_for(n, 256) > 4096 ? 4096 : grid_for(n, 256), 256, 0, p, v, n);
}

__global__ void k_scale(double *__restrict__ p, double a, int64_t n) {
    mds_pdl_entry();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = a * p[i];
}

int64_t live_ranges(const std::vector<int8_t> &live, const std::vector<int64_t> &a, const std::vector<int64_t> *b,
                    int64_t n1, std::vector<int64_t> &t) {
    std::vector<std::pair<int64_t, int64_t>> iv;
    auto add = [&](const std::vector<int64_t> &seg, int64_t base) {
        for (size_t k = 0; k + 1 < seg.size(); k++)
            if (k < live.size() && live[k] && seg[k + 1] > seg[k])
                iv.emplace_back((base + seg[k]) >> LIVE_CHUNK_LOG2,
                                ((base + seg[k + 1] - 1) >> LIVE_CHUNK_LOG2) + 1);
    };
    add(a, 0);
    if (b) add(*b, n1);
    std::sort(iv.begin(), iv.end());
    t.assign(1, 0);
    int64_t total = 0, lo = -1, hi = -1;
    auto flush = [&]() {
        if (hi > lo) {
            t.push_back(lo);
            t.push_back(total);
            total += hi - lo;
            t[0]++;
        }
    };
    for (auto &v : iv) {
        if (v.first <= hi) {
            hi = std::max(hi, v.second);
        } else {
            flush();
            lo = v.first;
            hi = v.second;
        }
    }
    flush();
    if (t[0] == 0) {  // nothing live: one empty range keeps the table well formed
        t.push_back(0);
        t.push_back(0);
        t[0] = 1;
    }
    return total;
}

void upload_ranges(Ctx &c, Buf &dev, const std::vector<int64_t> &t, int K) {
    const size_t cap = sizeof(int64_t) * (size_t)(2 * (2 * (size_t)K + 1) + 1);
    if (!dev.p || dev.bytes < cap) dev = Buf(&c, cap);
    MDS_REQUIRE(sizeof(int64_t) * t.size() <= dev.bytes, MDS_ERR_INVALID, "live chunk table overflow");
    MDS_CUDA(cudaMemcpyAsync(dev.p, t.data(), sizeof(int64_t) * t.size(), cudaMemcpyHostToDevice, c.stream));
}

Buf live_chunks(Ctx &c, int64_t rows, const std::vector<int64_t> &a, const std::vector<int64_t> *b, int64_t n1) {
    const int64_t nch = (rows + (1 << LIVE_CHUNK_LOG2) - 1) >> LIVE_CHUNK_LOG2;
    std::vector<int32_t> ck((size_t)(2 * (nch > 0 ? nch : 1)));
    for (int64_t q = 0; q < nch; q++) {
        ck[2 * q] = INT32_MAX;
        ck[2 * q + 1] = -1;
    }
    auto mark = [&](const std::vector<int64_t> &seg, int64_t base) {
        for (size_t k = 0; k + 1 < seg.size(); k++) {
            if (seg[k + 1] <= seg[k]) continue;
            const int64_t q0 = (base + seg[k]) >> LIVE_CHUNK_LOG2, q1 = (base + seg[k + 1] - 1) >> LIVE_CHUNK_LOG2;
            for (int64_t q = q0; q <= q1; q++) {
                ck[2 * q] = std::min(ck[2 * q], (int32_t)k);
                ck[2 * q + 1] = std::max(ck[2 * q + 1], (int32_t)k);
            }
        }
    };
    mark(a, 0);
    if (b) mark(*b, n1);
    for (int64_t q = 0; q < nch; q++)
        if (ck[2 * q + 1] < 0) ck[2 * q] = 0, ck[2 * q + 1] = -1;  // no rows: never live
    Buf d(&c, sizeof(int32_t) * ck.size());
    MDS_CUDA(cudaMemcpyAsync(d.p, ck.data(), sizeof(int32_t) * ck.size(), cudaMemcpyHostToDevice, c.stream));
    c.sync();  // the host table is released on return
    return d;
}

void scale_f64(Ctx &c, double *p, double a, int64_t n) {
    if (n <= 0) return;
    MDS_LAUNCH(c, KC_NONE, 2.0 * sizeof(double) * n, k_scale, grid_for(n, 256) > 4096 ? 4096 : grid_for(n, 256),
               256, 0, p, a, n);
}

// One contiguous range of `per` rows (nr entries each) per block, so that a
// block of finished instances' rows returns at once.
template <class A, class B>
__global__ void k_cast(const A *__restrict__ in, B *__restrict__ out, int64_t rows, int nr, int64_t per, LiveMap lm) {
    const int64_t r0 = live_block(lm, blockIdx.x, 1) * per, r1 = r0 + per < rows ? r0 + per : rows;
    if (!block_rows_live(lm, r0, r1)) return;
    mds_pdl_entry();
    for (int64_t i = r0 * nr + threadIdx.x; i < r1 * nr; i += blockDim.x) {
        // FP64 <-> FP32 by integer operations (the same results as the
        // hardware conversions; those issue on the FP64 unit)
        if constexpr (std::is_same<A, double>::value && std::is_same<B, float>::value)
            out[i] = d2f_int(in[i]);
        else if constexpr (std::is_same<A, float>::value && std::is_same<B, double>::value)
            out[i] = f2d_int(in[i]);
        else
            out[i] = (B)in[i];
    }
}

template <class A, class B> static void cast_rows(Ctx &c, const A *in, B *out, int64_t n, const LiveMap &lm, int nr) {
    if (n <= 0) return;
    const int64_t rows = n / nr;
    int64_t per = (rows + 8191) / 8192;  // at most 8192 blocks
    per = per < 256 ? 256 : per;
    unsigned g = (unsigned)((rows + per - 1) / per);
    if (lm.rt) {  // only the live chunks, one per block
        per = 256;
        g = (unsigned)(lm.nch > 0 ? lm.nch : 1);
    }
    MDS_LAUNCH(c, KC_NONE, (sizeof(A) + sizeof(B)) * (double)n, (k_cast<A, B>), g, 256, 0, in, out, rows, nr, per, lm);
}

void cast_f64_f32(Ctx &c, const double *in, float *out, int64_t n, const LiveMap &lm, int nr) {
    cast_rows<double, float>(c, in, out, n, lm, nr);
}

void cast_f32_f64(Ctx &c, const float *in, double *out, int64_t n, const LiveMap &lm, int nr) {
    cast_rows<float, double>(c, in, out, n, lm, nr);
}

// ---------------------------------------------------------------- SpMV

template <int G, class XT, class OT, int MODE, int NR>
static void spmv_launch(Ctx &c, const mds_csr &A, const XT *x, const double *r, OT *y, int kclass, const LiveMap &lm) {
    const int block = 256;
    double bytes = 12.0 * (double)A.nnz + 4.0 * (double)(A.nrow + 1) +
                   NR * (sizeof(XT) * (double)A.ncol + sizeof(OT) * (double)A.nrow + (MODE == 1 ? 8.0 * A.nrow : 0.0));
    const unsigned grid = (unsigned)live_blocks(lm, grid_for(A.nrow * G, block), G);
    MDS_LAUNCH_F(c, kclass, bytes * lm.frac, 2.0 * NR * A.nnz * lm.frac, (k_spmv_csr<G, double, XT, OT, MODE, NR>),
                 grid > 0 ? grid : 1, block, 0, A.nrow, A.row_ptr, A.col, A.val, x, r, y, lm);
}

template <int G, class XT, class OT, int MODE>
static void spmv_nr(Ctx &c, const mds_csr &A, const XT *x, const double *r, OT *y, int kclass, int nr,
                    const LiveMap &lm) {
    switch (nr) {
        case 1: spmv_launch<G, XT, OT, MODE, 1>(c, A, x, r, y, kclass, lm); break;
        case 2: spmv_launch<G, XT, OT, MODE, 2>(c, A, x, r, y, kclass, lm); break;
        case 4: spmv_launch<G, XT, OT, MODE, 4>(c, A, x, r, y, kclass, lm); break;
        case 8: spmv_launch<G, XT, OT, MODE, 8>(c, A, x, r, y, kclass, lm); break;
        default: throw Error(MDS_ERR_INVALID, "SpMV column count must be 1, 2, 4 or 8");
    }
}

template <class XT, class OT, int MODE>
static void spmv_dispatch(Ctx &c, const mds_csr &A, const XT *x, const double *r, OT *y, int kclass, int nr,
                          const LiveMap &lm) {
    if (A.nrow <= 0) return;
    // lanes per row: one thread per row for stencil-like rows (each thread
    // then has all of its row's loads in flight; measured 24 us vs 41 us with
    // four lanes on a 1.07M-row, 5-per-row FP64 operator), more for long rows
    double avg = A.nrow ? (double)A.nnz / (double)A.nrow : 0.0;
    if (avg <= 8.0)
        spmv_nr<1, XT, OT, MODE>(c, A, x, r, y, kclass, nr, lm);
    else if (avg <= 16.0)
        spmv_nr<2, XT, OT, MODE>(c, A, x, r, y, kclass, nr, lm);
    else if (avg <= 32.0)
        spmv_nr<4, XT, OT, MODE>(c, A, x, r, y, kclass, nr, lm);
    else if (avg <= 64.0)
        spmv_nr<8, XT, OT, MODE>(c, A, x, r, y, kclass, nr, lm);
    else
        spmv_nr<32, XT, OT, MODE>(c, A, x, r, y, kclass, nr, lm);
}

void spmv_f64(Ctx &c, const mds_csr &A, const double *x, double *y, int kclass, int nr, const LiveMap &lm) {
    spmv_dispatch<double, double, 0>(c, A, x, nullptr, y, kclass, nr, lm);
}

void spmv_sub_f64(Ctx &c, const mds_csr &A, const double *r, const double *x, double *out, int nr, const LiveMap &lm) {
    spmv_dispatch<double, double, 1>(c, A, x, r, out, KC_NONE, nr, lm);
}

void spmv_sub_f64_xf(Ctx &c, const mds_csr &A, const double *r, const float *x, float *out, int nr,
                     const LiveMap &lm) {
    spmv_dispatch<float, float, 1>(c, A, x, r, out, KC_NONE, nr, lm);
}

void spmv_sub_f64_to_f32(Ctx &c, const mds_csr &A, const double *r, const double *x, float *out, int nr,
                         const LiveMap &lm) {
    spmv_dispatch<double, float, 1>(c, A, x, r, out, KC_NONE, nr, lm);
}

}  // namespace mds
