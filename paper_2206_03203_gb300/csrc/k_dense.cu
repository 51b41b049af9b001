// Coarsest-level dense solve: FP64 Cholesky A = L L^T (blocked, right-looking)
// followed by the explicit inverse A^-1 = L^-T L^-1 (one warp per column), so
// that each V-cycle applies the coarsest solve as one parallel dense
// matrix-vector product instead of two sequential triangular solves.
//
// The coarsest level of a packed batch is block diagonal (one block per
// instance): every kernel works on K blocks at once (blockIdx.y = block), each
// block an n_b x n_b row-major matrix at its own offset; a single instance is
// the case K = 1.
#include "internal.cuh"

namespace mds {

constexpr int NB = 32;
constexpr int DTILE = 32;  // rows of a block applied by one thread block

__global__ void k_densify(const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                          const double *__restrict__ v, const DBlk *__restrict__ blk, double *__restrict__ D,
                          int *err) {
    mds_pdl_entry();
    const DBlk b = blk[blockIdx.y];
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= b.n) return;
    double *Db = D + b.off;
    for (int32_t p = rp[b.row + t]; p < rp[b.row + t + 1]; p++) {
        int64_t j = ci[p] - b.row;
        if (j < 0 || j >= b.n) {  // an entry coupling two instances
            atomicOr(err, DERR_CAPACITY);
            continue;
        }
        Db[t * b.n + j] = v[p];
    }
}

// factor the nb x nb diagonal tile at k0 in shared memory
__global__ void k_chol_diag(double *D, const DBlk *__restrict__ blk, int64_t k0, int *err) {
    mds_pdl_entry();
    const DBlk b = blk[blockIdx.y];
    if (k0 >= b.n) return;
    const int64_t n = b.n;
    const int nb = (int)((n - k0) < NB ? (n - k0) : NB);
    double *Db = D + b.off;
    __shared__ double T[NB][NB + 1];
    __shared__ int bad;
    int t = threadIdx.x;
    if (t == 0) bad = 0;
    for (int q = t; q < nb * nb; q += blockDim.x) {
        int i = q / nb, j = q % nb;
        T[i][j] = Db[(k0 + i) * n + k0 + j];
    }
    __syncthreads();
    for (int j = 0; j < nb; j++) {
        if (t == 0) {
            double s = T[j][j];
            if (!(s > 0.0)) {
                bad = 1;
                s = 1.0;
            }
            T[j][j] = sqrt(s);
        }
        __syncthreads();
        for (int i = j + 1 + t; i < nb; i += blockDim.x) T[i][j] /= T[j][j];
        __syncthreads();
        for (int q = t; q < nb * nb; q += blockDim.x) {
            int i = q / nb, k = q % nb;
            if (k > j && i >= k) T[i][k] -= T[i][j] * T[k][j];
        }
        __syncthreads();
    }
    for (int q = t; q < nb * nb; q += blockDim.x) {
        int i = q / nb, j = q % nb;
        if (i >= j) Db[(k0 + i) * n + k0 + j] = T[i][j];
    }
    if (t == 0 && bad) atomicOr(err, DERR_NOT_SPD);
}

// rows below the panel: L21 = A21 L11^-T, one thread per row
__global__ void k_chol_trsm(double *D, const DBlk *__restrict__ blk, int64_t k0) {
    mds_pdl_entry();
    const DBlk b = blk[blockIdx.y];
    if (k0 >= b.n) return;
    const int64_t n = b.n;
    const int nb = (int)((n - k0) < NB ? (n - k0) : NB);
    double *Db = D + b.off;
    __shared__ double L[NB][NB + 1];
    for (int q = threadIdx.x; q < nb * nb; q += blockDim.x) {
        int i = q / nb, j = q % nb;
        L[i][j] = Db[(k0 + i) * n + k0 + j];
    }
    __syncthreads();
    int64_t i = k0 + nb + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double x[NB];
    for (int j = 0; j < nb; j++) {
        double s = Db[i * n + k0 + j];
        for (int k = 0; k < j; k++) s -= x[k] * L[j][k];
        x[j] = s / L[j][j];
    }
    for (int j = 0; j < nb; j++) Db[i * n + k0 + j] = x[j];
}

// trailing update A22 -= L21 L21^T on the lower tiles
__global__ void k_chol_update(double *D, const DBlk *__restrict__ blk, int64_t k0) {
    mds_pdl_entry();
    const DBlk bk = blk[blockIdx.y];
    const int64_t n = bk.n;
    if (k0 + NB >= n) return;  // no trailing matrix
    const int nb = NB;
    const int64_t base = k0 + nb;
    const int64_t m = (n - base + NB - 1) / NB;
    int64_t b = blockIdx.x;
    if (b >= m * (m + 1) / 2) return;
    double *Db = D + bk.off;
    __shared__ double Li[NB][NB + 1], Lj[NB][NB + 1];
    // map b -> (bi, bj), bj <= bi
    int64_t bi = (int64_t)((sqrt(8.0 * (double)b + 1.0) - 1.0) / 2.0);
    while ((bi + 1) * (bi + 2) / 2 <= b) bi++;
    while (bi * (bi + 1) / 2 > b) bi--;
    int64_t bj = b - bi * (bi + 1) / 2;
    int64_t r0 = base + bi * NB, c0 = base + bj * NB;
    for (int q = threadIdx.x; q < NB * nb; q += blockDim.x) {
        int r = q / nb, k = q % nb;
        Li[r][k] = (r0 + r < n) ? Db[(r0 + r) * n + k0 + k] : 0.0;
        Lj[r][k] = (c0 + r < n) ? Db[(c0 + r) * n + k0 + k] : 0.0;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < NB * NB; q += blockDim.x) {
        int r = q / NB, s = q % NB;
        int64_t gi = r0 + r, gj = c0 + s;
        if (gi >= n || gj >= n || gj > gi) continue;
        double acc = 0.0;
        for (int k = 0; k < nb; k++) acc += Li[r][k] * Lj[s][k];
        Db[gi * n + gj] -= acc;
    }
}

__global__ void k_transpose_lower(const double *__restrict__ L, double *__restrict__ U, const DBlk *__restrict__ blk) {
    mds_pdl_entry();
    const DBlk b = blk[blockIdx.y];
    const int64_t n = b.n;
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n * n) return;
    int64_t i = q / n, j = q % n;
    U[b.off + j * n + i] = (i >= j) ? L[b.off + i * n + j] : 0.0;
}

// column j of A^-1: L y = e_j, then L^T x = y (x overwrites y); one warp per column
__global__ void k_chol_inverse(const double *__restrict__ Lall, const double *__restrict__ Uall,
                               const DBlk *__restrict__ blk, double *__restrict__ Xall) {
    mds_pdl_entry();
    extern __shared__ double ys[];
    const DBlk b = blk[blockIdx.y];
    const int64_t n = b.n;
    const double *L = Lall + b.off, *U = Uall + b.off;
    double *X = Xall + b.off;
    int wpb = blockDim.x / 32;
    int w = threadIdx.x / 32, lane = threadIdx.x % 32;
    int64_t j = (int64_t)blockIdx.x * wpb + w;
    if (j >= n) return;
    double *y = ys + (size_t)w * n;
    for (int64_t i = lane; i < n; i += 32) y[i] = 0.0;
    __syncwarp();
    for (int64_t i = j; i < n; i++) {
        double s = 0.0;
        for (int64_t k = j + lane; k < i; k += 32) s += L[i * n + k] * y[k];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) y[i] = ((i == j ? 1.0 : 0.0) - s) / L[i * n + i];
        __syncwarp();
    }
    for (int64_t i = n - 1; i >= 0; i--) {
        double s = 0.0;
        for (int64_t k = i + 1 + lane; k < n; k += 32) s += U[i * n + k] * y[k];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) y[i] = (y[i] - s) / L[i * n + i];
        __syncwarp();
    }
    for (int64_t i = lane; i < n; i += 32) X[j * n + i] = y[i];
}

// Columns j0 .. j0 + CW - 1 of A^-1 for one block (one thread block per
// CW-column tile, 256 threads): L Y = E, then L^T X = Y, by 32-row panels
// with the CW right-hand sides in shared memory (row stride CW + 1).  Each
// panel first takes the product of the finished panels (a group of CW
// lanes per 32 / (256 / CW) rows, one column per lane: FP64 products from
// shared memory, no reductions), then CW lanes solve the panel's 32 x 32
// triangle (right-looking, column per lane).  A^-1 is symmetric, so the
// backward pass stops at the 32-row panel holding j0 (half the products of
// a full one): the tile writes the entries of its columns from that panel
// down, and mirrors those of the later panels into the rows j0 .. j0 + CW - 1
// of the other tiles' columns.  CW = 16 keeps a block's shared memory at
// 136 n bytes, so that two or more blocks share an SM.
constexpr int INV_CW = 16;
template <int CW>
__global__ void __launch_bounds__(256) k_chol_inv_tiles(const double *__restrict__ Lall, const DBlk *__restrict__ blk,
                                                        const int2 *__restrict__ tiles, double *__restrict__ Xall) {
    constexpr int P = CW + 1;          // row stride of Y
    constexpr int RG = 32 * CW / 256;  // panel rows per lane group
    mds_pdl_entry();
    extern __shared__ double Y[];  // [n][P]
    __shared__ double T[32][33];   // the panel's diagonal block of L
    const int2 tl = tiles[blockIdx.x];
    const DBlk b = blk[tl.x];
    const int n = b.n, j0 = tl.y, tid = threadIdx.x, c = tid % CW, g = tid / CW;
    const double *L = Lall + b.off;
    double *X = Xall + b.off;
    for (int e = tid; e < n * CW; e += blockDim.x) {
        const int i = e / CW, cc = e % CW;
        Y[i * P + cc] = i == j0 + cc ? 1.0 : 0.0;
    }
    __syncthreads();
    // forward from the 32-row panel holding j0 (rows below j0 of Y are zero):
    // the panels, and so every rounding, are those of a 32-column tile
    const int jb = j0 / 32 * 32;
    for (int p0 = jb; p0 < n; p0 += 32) {
        const int pn = min(32, n - p0);
        if (p0 > jb) {
            double acc[RG];
#pragma unroll
            for (int q = 0; q < RG; q++) acc[q] = 0.0;
            for (int k = jb; k < p0; k++) {
                const double y = Y[k * P + c];
#pragma unroll
                for (int q = 0; q < RG; q++) {
                    const int r = g * RG + q;
                    if (r < pn) acc[q] += L[(int64_t)(p0 + r) * n + k] * y;
                }
            }
#pragma unroll
            for (int q = 0; q < RG; q++) {
                const int r = g * RG + q;
                if (r < pn) Y[(p0 + r) * P + c] -= acc[q];
            }
        }
        for (int e = tid; e < pn * pn; e += blockDim.x) {
            const int r = e / pn, q = e % pn;
            T[r][q] = q <= r ? L[(int64_t)(p0 + r) * n + p0 + q] : 0.0;
        }
        __syncthreads();
        if (tid < CW) {
            for (int i = 0; i < pn; i++) {
                const double yi = Y[(p0 + i) * P + c] / T[i][i];
                Y[(p0 + i) * P + c] = yi;
                for (int k = i + 1; k < pn; k++) Y[(p0 + k) * P + c] -= T[k][i] * yi;
            }
        }
        __syncthreads();
    }
    // backward over the rows from the panel holding j0 down (the same 32-row
    // grid as the forward pass, from the last panel up): A^-1 is symmetric,
    // so its entries above that panel are taken from the tiles owning their
    // columns (written below as mirrored rows)
    int last = jb;
    while (last + 32 < n) last += 32;
    const int top = jb;
    for (int s0 = last; s0 >= top; s0 -= 32) {
        const int a = max(s0, 0), e1 = min(s0 + 32, n), pn = e1 - a;
        if (pn <= 0) continue;
        if (e1 < n) {
            double acc[RG];
#pragma unroll
            for (int q = 0; q < RG; q++) acc[q] = 0.0;
            for (int k = e1; k < n; k++) {
                const double x = Y[k * P + c];
#pragma unroll
                for (int q = 0; q < RG; q++) {
                    const int r = g * RG + q;
                    if (r < pn) acc[q] += L[(int64_t)k * n + a + r] * x;
                }
            }
#pragma unroll
            for (int q = 0; q < RG; q++) {
                const int r = g * RG + q;
                if (r < pn) Y[(a + r) * P + c] -= acc[q];
            }
        }
        for (int e = tid; e < pn * pn; e += blockDim.x) {
            const int r = e / pn, q = e % pn;
            T[r][q] = q <= r ? L[(int64_t)(a + r) * n + a + q] : 0.0;
        }
        __syncthreads();
        if (tid < CW) {
            for (int i = pn - 1; i >= 0; i--) {
                const double xi = Y[(a + i) * P + c] / T[i][i];
                Y[(a + i) * P + c] = xi;
                for (int k = 0; k < i; k++) Y[(a + k) * P + c] -= T[i][k] * xi;
            }
        }
        __syncthreads();
    }
    // entry (i, j) of A^-1 goes to X[j n + i] for rows i >= jb, and, for
    // rows in the later panels (i >= jb + 32), also to X[i n + j]: every
    // entry is written once, by the tile whose column it is when i and j
    // share a 32-row panel or i lies below, by the mirror otherwise
    const int nc = min(CW, n - j0), nr = n - jb;
    for (int e = tid; e < nc * nr; e += blockDim.x) {
        const int cc = e / nr, i = jb + e % nr;
        X[(int64_t)(j0 + cc) * n + i] = Y[i * P + cc];
    }
    const int nm = max(nr - 32, 0);
    for (int e = tid; e < nc * nm; e += blockDim.x) {
        const int i = jb + 32 + e / nc, cc = e % nc;
        X[(int64_t)i * n + j0 + cc] = Y[i * P + cc];
    }
}

void dense_spd_inverse(Ctx &c, const mds_csr &A, const std::vector<int64_t> &seg, Buf &Ainv, DenseBlocks &db) {
    const int K = (int)seg.size() - 1;
    MDS_REQUIRE(K >= 1 && seg[0] == 0 && seg[K] == A.nrow, MDS_ERR_INVALID, "coarsest segments do not cover the level");
    std::vector<DBlk> hb(K);
    int64_t nmax = 0, tot = 0;
    for (int k = 0; k < K; k++) {
        int64_t n = seg[k + 1] - seg[k];
        MDS_REQUIRE(n >= 0 && n <= 8192, MDS_ERR_INVALID, "coarsest level size out of range for dense Cholesky");
        hb[k] = DBlk{seg[k], tot, (int32_t)n};
        tot += n * n;
        nmax = n > nmax ? n : nmax;
    }
    MDS_REQUIRE(nmax >= 1, MDS_ERR_INVALID, "empty coarsest level");
    db.K = K;
    db.nmax = nmax;
    db.nrow = A.nrow;
    db.total = tot;
    db.host = hb;
    db.blk = Buf(&c, sizeof(DBlk) * (size_t)K);
    MDS_CUDA(cudaMemcpyAsync(db.blk.p, hb.data(), sizeof(DBlk) * (size_t)K, cudaMemcpyHostToDevice, c.stream));
    {
        std::vector<int2> tl;
        for (int k = 0; k < K; k++)
            for (int32_t r = 0; r < hb[k].n; r += DTILE) tl.push_back(make_int2(k, r));
        db.ntiles = (int64_t)tl.size();
        db.tiles = Buf(&c, sizeof(int2) * tl.size());
        MDS_CUDA(cudaMemcpyAsync(db.tiles.p, tl.data(), sizeof(int2) * tl.size(), cudaMemcpyHostToDevice, c.stream));
        c.sync();
    }
    const DBlk *B = db.blk.as<DBlk>();
    Buf D(&c, sizeof(double) * (size_t)tot);
    MDS_CUDA(cudaMemsetAsync(D.p, 0, sizeof(double) * (size_t)tot, c.stream));
    c.clear_err();
    MDS_LAUNCH(c, KC_NONE, 0, k_densify, dim3(grid_for(nmax, 128), K), 128, 0, A.row_ptr, A.col, A.val, B,
               D.as<double>(), c.d_err);
    c.check_err("coarsest level (a coupling between two instances)");
    c.clear_err();
    for (int64_t k0 = 0; k0 < nmax; k0 += NB) {
        MDS_LAUNCH(c, KC_NONE, 0, k_chol_diag, dim3(1, K), 256, 0, D.as<double>(), B, k0, c.d_err);
        int64_t rest = nmax - k0 - NB;
        if (rest <= 0) break;
        MDS_LAUNCH(c, KC_NONE, 0, k_chol_trsm, dim3(grid_for(rest, 64), K), 64, 0, D.as<double>(), B, k0);
        int64_t m = (rest + NB - 1) / NB;
        MDS_LAUNCH(c, KC_NONE, 0, k_chol_update, dim3((unsigned)(m * (m + 1) / 2), K), 256, 0, D.as<double>(), B, k0);
    }
    c.check_err("coarsest Cholesky");
    Ainv = Buf(&c, sizeof(double) * (size_t)tot);
    const size_t tsmem = sizeof(double) * (size_t)nmax * (INV_CW + 1);
    if (tsmem <= 200 * 1024) {
        // INV_CW-column tiles of every block
        std::vector<int2> tl;
        for (int k = 0; k < K; k++)
            for (int32_t j = 0; j < hb[k].n; j += INV_CW) tl.push_back(make_int2(k, j));
        Buf tiles(&c, sizeof(int2) * tl.size());
        MDS_CUDA(cudaMemcpyAsync(tiles.p, tl.data(), sizeof(int2) * tl.size(), cudaMemcpyHostToDevice, c.stream));
        // with the kernel's static panel tile, even a dynamic size under
        // 48 KB can take the block past the default limit: always opt in
        MDS_CUDA(cudaFuncSetAttribute(k_chol_inv_tiles<INV_CW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)tsmem));
        MDS_LAUNCH(c, KC_NONE, 0, k_chol_inv_tiles<INV_CW>, (unsigned)tl.size(), 256, tsmem, D.as<double>(), B,
                   tiles.as<int2>(), Ainv.as<double>());
        c.sync();  // the host tile list is released on return
        return;
    }
    Buf U(&c, sizeof(double) * (size_t)tot);
    MDS_LAUNCH(c, KC_NONE, 0, k_transpose_lower, dim3(grid_for(nmax * nmax, 256), K), 256, 0, D.as<double>(),
               U.as<double>(), B);
    int wpb = 4;
    while (wpb > 1 && (size_t)wpb * nmax * sizeof(double) > 48 * 1024) wpb /= 2;
    size_t smem = (size_t)wpb * nmax * sizeof(double);
    if (smem > 48 * 1024)
        MDS_CUDA(cudaFuncSetAttribute(k_chol_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    MDS_LAUNCH(c, KC_NONE, 0, k_chol_inverse, dim3(grid_for(nmax, wpb), K), 32 * wpb, smem, D.as<double>(),
               U.as<double>(), B, Ainv.as<double>());
}

// The block holding row `row` of the coarsest level (blocks ascending by row).
__device__ __forceinline__ int dblk_of(const DBlk *blk, int K, int64_t row) {
    int lo = 0, hi = K - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (blk[mid].row <= row)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// y = M x for NR interleaved columns (entry (i, c) at i * NR + c), M the
// block-diagonal inverse; one warp per row, FP64 accumulation over the row of
// its block (k = lane, lane + 32, ...) then a lane tree.  M is fixed after
// set-up: each lane loads its first DPRE entries of the row before waiting
// for the kernel that produced x.
constexpr int DPRE = 16;
template <class XT, int NR>
__global__ void k_dense_apply(const double *__restrict__ Mall, const DBlk *__restrict__ blk, int K, int64_t nrow,
                              const XT *__restrict__ xall, XT *__restrict__ yall, const int8_t *__restrict__ on) {
    int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    int lane = threadIdx.x % 32;
    bool live = row < nrow;
    DBlk b{0, 0, 0};
    if (live) {
        const int k = K > 1 ? dblk_of(blk, K, row) : 0;
        b = blk[k];
        if (on && !on[k]) live = false;  // a finished instance of a batched solve
    }
    const int64_t n = b.n, i = row - b.row;
    const double *M = Mall + b.off + i * n;
    const XT *x = xall + b.row * NR;
    double pm[DPRE];
#pragma unroll
    for (int q = 0; q < DPRE; q++) {
        int64_t k = lane + 32 * (int64_t)q;
        pm[q] = live && k < n ? M[k] : 0.0;
    }
    mds_pdl_wait();
    mds_pdl_trigger();
    if (!live) return;
    double s[NR];
#pragma unroll
    for (int c = 0; c < NR; c++) s[c] = 0.0;
#pragma unroll
    for (int q = 0; q < DPRE; q++) {
        int64_t k = lane + 32 * (int64_t)q;
        if (k < n) {
#pragma unroll
            for (int c = 0; c < NR; c++) s[c] += pm[q] * (double)x[k * NR + c];
        }
    }
    for (int64_t k = lane + 32 * DPRE; k < n; k += 32) {
        double m = M[k];
#pragma unroll
        for (int c = 0; c < NR; c++) s[c] += m * (double)x[k * NR + c];
    }
#pragma unroll
    for (int c = 0; c < NR; c++)
        for (int o = 16; o > 0; o >>= 1) s[c] += __shfl_down_sync(0xffffffffu, s[c], o);
    if (lane == 0)
#pragma unroll
        for (int c = 0; c < NR; c++) yall[row * NR + c] = (XT)s[c];
}

// Sum of v[0..15] over the 32 lanes of a warp by halving exchanges: after
// the steps lanes 2u and 2u + 1 hold the total of value u = (lane >> 1) & 15
// (16 additions per lane instead of 5 per value).
__device__ __forceinline__ double warp_sum16(double (&v)[16]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int h = 8, m = 16; h >= 1; h >>= 1, m >>= 1) {
        const bool up = (lane & m) != 0;
#pragma unroll
        for (int i = 0; i < h; i++) {
            const double keep = up ? v[i + h] : v[i], send = up ? v[i] : v[i + h];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, m);
        }
    }
    return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

// y = M x on 32-row tiles: one thread block per tile (64 NR threads), the
// tile's block of x staged once in shared memory in FP64 (column-major, so a
// warp's reads are contiguous), each warp 16 / NR rows with the lanes
// striding over the columns of M; FP64 products and sums.
template <class XT, int NR>
__global__ void __launch_bounds__(64 * NR) k_dense_apply_tiles(const double *__restrict__ Mall,
                                                               const DBlk *__restrict__ blk,
                                                               const int2 *__restrict__ tiles,
                                                               const XT *__restrict__ xall, XT *__restrict__ yall,
                                                               const int8_t *__restrict__ on) {
    constexpr int RPW = 16 / NR;  // rows per warp
    extern __shared__ double xs[];  // [NR][n]
    const int2 t = tiles[blockIdx.x];
    if (on && !on[t.x]) return;  // a finished instance of a batched solve
    const DBlk b = blk[t.x];
    const int n = b.n, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int r0 = t.y + w * RPW;
    const double *M = Mall + b.off;
    // the first column stripe of the warp's rows (M is fixed after set-up)
    double m0[RPW];
#pragma unroll
    for (int r = 0; r < RPW; r++) m0[r] = r0 + r < n && lane < n ? M[(int64_t)(r0 + r) * n + lane] : 0.0;
    mds_pdl_wait();
    mds_pdl_trigger();
    const XT *x = xall + b.row * NR;
    for (int e = threadIdx.x; e < n * NR; e += blockDim.x) xs[(e % NR) * n + e / NR] = (double)x[e];
    __syncthreads();
    if (r0 >= n) return;  // a warp past the block's last row (after the barrier)
    double s[16];
#pragma unroll
    for (int v = 0; v < 16; v++) s[v] = 0.0;
    if (lane < n) {
#pragma unroll
        for (int r = 0; r < RPW; r++)
#pragma unroll
            for (int c = 0; c < NR; c++) s[r * NR + c] = m0[r] * xs[c * n + lane];
    }
    for (int k = lane + 32; k < n; k += 32) {
        double xv[NR];
#pragma unroll
        for (int c = 0; c < NR; c++) xv[c] = xs[c * n + k];
#pragma unroll
        for (int r = 0; r < RPW; r++) {
            const double mk = r0 + r < n ? M[(int64_t)(r0 + r) * n + k] : 0.0;
#pragma unroll
            for (int c = 0; c < NR; c++) s[r * NR + c] += mk * xv[c];
        }
    }
    const double tot = warp_sum16(s);
    const int u = (lane >> 1) & 15, r = u / NR, c = u % NR;
    if ((lane & 1) == 0 && r0 + r < n) yall[(b.row + r0 + r) * NR + c] = (XT)tot;
}

template <class XT>
static void dense_apply_t(Ctx &c, const DenseBlocks &db, const double *M, int nr, const XT *x, XT *y,
                          const int8_t *on) {
    const int64_t n = db.nrow;
    double bytes = 8.0 * (double)db.total + 2.0 * sizeof(XT) * n * nr;
    const DBlk *B = db.blk.as<DBlk>();
    const size_t smem = sizeof(double) * (size_t)db.nmax * (size_t)nr;
    // tiles when there are enough of them to fill the SMs (a batch's blocks);
    // a single small block keeps a warp per row (n warps instead of n / 32
    // thread blocks)
    if (db.ntiles >= (c.num_sms > 0 ? c.num_sms : 1) && smem <= 96 * 1024) {
        const int2 *T = db.tiles.as<int2>();
        const unsigned g = (unsigned)db.ntiles;
        switch (nr) {
#define MDS_DTILE_CASE(NRV)                                                                                        \
    case NRV:                                                                                                      \
        if (smem > 48 * 1024)                                                                                      \
            MDS_CUDA(cudaFuncSetAttribute(k_dense_apply_tiles<XT, NRV>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                          (int)smem));                                                             \
        MDS_LAUNCH(c, KC_NONE, bytes, (k_dense_apply_tiles<XT, NRV>), g, 64 * NRV, smem, M, B, T, x, y, on);     \
        return;
            MDS_DTILE_CASE(1)
            MDS_DTILE_CASE(2)
            MDS_DTILE_CASE(4)
            MDS_DTILE_CASE(8)
#undef MDS_DTILE_CASE
            default: throw Error(MDS_ERR_INVALID, "dense apply: column count must be 1, 2, 4 or 8");
        }
    }
    unsigned g = grid_for(n * 32, 256);
    switch (nr) {
        case 1: MDS_LAUNCH(c, KC_NONE, bytes, (k_dense_apply<XT, 1>), g, 256, 0, M, B, db.K, n, x, y, on); break;
        case 2: MDS_LAUNCH(c, KC_NONE, bytes, (k_dense_apply<XT, 2>), g, 256, 0, M, B, db.K, n, x, y, on); break;
        case 4: MDS_LAUNCH(c, KC_NONE, bytes, (k_dense_apply<XT, 4>), g, 256, 0, M, B, db.K, n, x, y, on); break;
        case 8: MDS_LAUNCH(c, KC_NONE, bytes, (k_dense_apply<XT, 8>), g, 256, 0, M, B, db.K, n, x, y, on); break;
        default: throw Error(MDS_ERR_INVALID, "dense apply: column count must be 1, 2, 4 or 8");
    }
}

void dense_apply(Ctx &c, const DenseBlocks &db, const double *M, int nr, const double *x, double *y,
                 const int8_t *on) {
    dense_apply_t<double>(c, db, M, nr, x, y, on);
}

void dense_apply(Ctx &c, const DenseBlocks &db, const double *M, int nr, const float *x, float *y, const int8_t *on) {
    dense_apply_t<float>(c, db, M, nr, x, y, on);
}

}  // namespace mds
