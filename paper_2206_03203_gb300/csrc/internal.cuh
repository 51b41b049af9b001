// Internal declarations of libmdsolve (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <map>
#include <atomic>
#include <memory>
#include <string>
#include <thread>
#include <tuple>
#include <utility>
#include <unordered_map>
#include <vector>

#include "mdsolve.h"

namespace mds {

// Programmatic dependent launch.  Every kernel of the library is launched
// with programmatic stream serialisation allowed and starts with this call:
// it waits until the previous kernel in the stream has completed and its
// writes are visible, then lets the next kernel's blocks be scheduled while
// this one runs.  The launch latency of each kernel thus overlaps the tail of
// its predecessor; the order of memory effects is that of plain stream order.
__device__ __forceinline__ void mds_pdl_wait() {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 900
    asm volatile("griddepcontrol.wait;" ::: "memory");
#endif
}
__device__ __forceinline__ void mds_pdl_trigger() {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 900
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
#endif
}
__device__ __forceinline__ void mds_pdl_entry() {
    mds_pdl_wait();
    mds_pdl_trigger();
}

struct Error {
    int code;
    std::string msg;
    Error(int c, std::string m) : code(c), msg(std::move(m)) {}
};

#define MDS_CUDA(call)                                                                   \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            throw ::mds::Error(e_ == cudaErrorMemoryAllocation ? MDS_ERR_OOM : MDS_ERR_CUDA, \
                               std::string(#call) + ": " + cudaGetErrorString(e_));      \
    } while (0)

#define MDS_REQUIRE(cond, code, msg)                        \
    do {                                                    \
        if (!(cond)) throw ::mds::Error((code), (msg));     \
    } while (0)

// Device error word bits set by kernels (never trap).
enum : int {
    DERR_DUP_FACE = 1,
    DERR_BAD_FRACTURE = 2,
    DERR_CAPACITY = 4,
    DERR_NOT_SPD = 8,
    DERR_ZERO_DIAG = 16,
    DERR_NONFINITE = 32,
    DERR_TIMEOUT = 64,  // an asynchronous copy did not complete within its time limit
};

// Kernel classes for event timing (match the C ABI's numbering).
enum : int {
    KC_NONE = -1,
    KC_SPMV = 0,
    KC_VC_RESID = 1,
    KC_VC_POST = 2,
    KC_GS_DOT = 3,
    KC_GS_AXPY = 4,
    KC_VCYCLE = 5,
    KC_VC_RESTRICT = 6,
};

// Storage of a V-cycle level: value type and sparse format.
enum : int { VT_F64 = 0, VT_F32 = 1, VT_BF16 = 2, VT_F16 = 3 };
enum : int { FMT_CSR = 0, FMT_SELL = 1, FMT_DIA = 2 };

struct TuneChoice {
    int fmt, G, C, sigma;
    int stored;  // the level runs the stored form (faster than the fused pair)
};

struct Ctx;

// Owned device allocation from the context's allocator (move-only).
struct Buf {
    Ctx *ctx = nullptr;
    void *p = nullptr;
    size_t bytes = 0;
    Buf() = default;
    Buf(Ctx *c, size_t n);
    ~Buf();
    Buf(const Buf &) = delete;
    Buf &operator=(const Buf &) = delete;
    Buf(Buf &&o) noexcept { *this = std::move(o); }
    Buf &operator=(Buf &&o) noexcept;
    void reset();
    template <class T> T *as() const { return static_cast<T *>(p); }
};

struct KTimerRec {
    cudaEvent_t e0, e1;
};

// FP64 levels up to this many rows run the fused L1-Jacobi forms (latency
// rather than the FP64 units bounds them); larger ones keep y stored.
constexpr int64_t FUSE_FP64_ROWS = 65536;

// Rows of a packed batch whose instance is still iterating.  The batched
// solve's kernels skip every thread block whose rows all belong to finished
// instances: the system is block diagonal, so no live row reads those rows.
// A row space (the rows of one block of the system, one level of a
// hierarchy, or the whole system: matrix rows, then fracture rows) is cut
// into chunks of 256 rows; ck[2 c] and ck[2 c + 1] are the least and the
// greatest instance owning a row of chunk c.  ck == NULL: every row is live.
constexpr int LIVE_CHUNK_LOG2 = 8;
//
// Once instances have finished, launches are also compacted: rt lists the
// 256-row chunks that hold a live row as merged ranges (rt[0] = R, then for
// range r its first chunk rt[1 + 2r] and the chunks of the ranges before it
// rt[2 + 2r]); a launch covers only those nch chunks and maps its block
// index through the table.  rt == NULL: every chunk, in order.
struct LiveMap {
    const int32_t *ck = nullptr;
    const int8_t *live = nullptr;
    double frac = 1.0;  // host side: share of the rows that are live (scales a launch's algorithmic work)
    const int64_t *rt = nullptr;
    int64_t nch = -1;   // host side: chunks of a compacted launch (-1: not compacted)
};

// The i-th chunk of a launch over the map's chunks.
__device__ __forceinline__ int64_t live_chunk(const LiveMap &m, int64_t i) {
    if (!m.rt) return i;
    int lo = 0, hi = (int)m.rt[0] - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (m.rt[2 + 2 * mid] <= i)
            lo = mid;
        else
            hi = mid - 1;
    }
    return m.rt[1 + 2 * lo] + (i - m.rt[2 + 2 * lo]);
}
// Blocks of a launch with g blocks per 256-row chunk: all of them, or only
// those of the live chunks.
inline int64_t live_blocks(const LiveMap &m, int64_t all, int g) { return m.nch >= 0 ? m.nch * g : all; }
// The block a launch's i-th block stands for (g blocks per chunk).
__device__ __forceinline__ int64_t live_block(const LiveMap &m, int64_t i, int g) {
    return m.rt ? live_chunk(m, i / g) * g + i % g : i;
}

__device__ __forceinline__ int seg_find(const int64_t *seg, int K, int64_t r) {
    int lo = 0, hi = K - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (seg[mid] <= r)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// Whether rows [r0, r1) hold a row of a live instance.  Every thread of a
// block gets the same answer from the same (broadcast) loads, so no barrier
// is needed.  The flags are written by host copies between solver steps,
// never by a kernel, so this may run before the programmatic dependency wait.
__device__ __forceinline__ bool block_rows_live(const LiveMap &m, int64_t r0, int64_t r1) {
    if (!m.ck || r0 >= r1) return true;
    const int64_t c0 = r0 >> LIVE_CHUNK_LOG2, c1 = (r1 - 1) >> LIVE_CHUNK_LOG2;
    int lo = __ldg(m.ck + 2 * c0), hi = __ldg(m.ck + 2 * c0 + 1);
    for (int64_t c = c0 + 1; c <= c1; c++) {
        lo = min(lo, __ldg(m.ck + 2 * c));
        hi = max(hi, __ldg(m.ck + 2 * c + 1));
    }
    for (int k = lo; k <= hi; k++)
        if (m.live[k]) return true;
    return false;
}

// One launch recorded while a CUDA graph is being captured: its accounting is
// replayed, and its events (when its class is timed) read, at every replay.
struct GraphRec {
    int cls;
    double bytes, flops;
    bool timed;
    cudaEvent_t e0, e1;
};

// A captured sequence of launches and its executable graph.
struct Graph {
    cudaGraphExec_t exec = nullptr;
    std::vector<GraphRec> recs;
    int64_t launches = 0;
    // share of a packed batch's rows live when captured: a replay scales the
    // recorded algorithmic work by (share at replay) / cap_share
    double cap_share = 1.0;
    double scale = 1.0;
    Graph() = default;
    Graph(const Graph &) = delete;
    Graph &operator=(const Graph &) = delete;
    ~Graph();
};

struct Ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    mds_allocator alloc{};
    bool custom_alloc = false;
    // the context's own stream-ordered pool (no custom allocator): freed
    // blocks stay mapped in it for the next set-up or solve, instead of going
    // back to the driver at the next synchronization; released by mds_destroy
    cudaMemPool_t pool = nullptr;
    int num_sms = 0;
    std::unordered_map<const void *, int> resident;  // kernel -> blocks of 256 threads the device holds at once
    std::string last_error;
    int *d_err = nullptr;      // device error word
    void *h_pin = nullptr;     // pinned host scratch (PIN_BYTES)
    static constexpr size_t PIN_BYTES = 1 << 20;
    bool timing[MDS_KCLASS_COUNT] = {};
    std::vector<KTimerRec> evs[MDS_KCLASS_COUNT];
    size_t ev_used[MDS_KCLASS_COUNT] = {};
    int64_t launches[MDS_KCLASS_COUNT] = {};
    double bytes[MDS_KCLASS_COUNT] = {};
    double flops[MDS_KCLASS_COUNT] = {};
    int64_t total_launches = 0;
    double graph_ms[MDS_KCLASS_COUNT] = {};
    // launches that were bracketed by events, and their algorithmic work
    int64_t tlaunches[MDS_KCLASS_COUNT] = {};
    double tbytes[MDS_KCLASS_COUNT] = {};
    double tflops[MDS_KCLASS_COUNT] = {};
    int sample_every = 1;          // FGMRES brackets every k-th restart cycle
    bool timing_suspended = false; // capture of the unbracketed graph variant
    Graph *capturing = nullptr;   // recording target while a stream capture is open
    void *owner = nullptr;        // the mds_ctx handle that holds this context
    // asynchronous solve (mds_solve_async): the host control loop of one
    // solve on a library thread; every other call on the context joins it first
    struct Async {
        std::thread th;
        bool pending = false;             // started and not yet collected by mds_solve_wait
        std::shared_ptr<std::atomic<int>> done;
        int status = 0;
        std::vector<mds_rhs_stats> stats;
    } async;
    int dependents = 0;           // live systems and preconditioners made on this context
    bool destroy_requested = false;
    cudaStream_t cap_stream = nullptr;
    // second stream for work that runs beside the main stream (the two
    // independent V-cycles of the block-diagonal preconditioner)
    cudaStream_t side_stream = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // instance flags of the batched solve in progress (NULL otherwise): the
    // kernels of a packed batch skip the rows of finished instances; their
    // host copy gives the launches' algorithmic work
    const int8_t *live = nullptr;
    std::vector<int8_t> live_host;
    // compacted launches (some instance has finished): live_ver counts the
    // changes of live_host, so that each row space rebuilds its chunk ranges
    // once per change
    bool compact = false;
    // set around one level operation: it writes its rows to this FP64 vector
    // instead of its own output (the top level of an FP32 V-cycle handing
    // its result to the FP64 Krylov method without a separate conversion)
    double *level_out64 = nullptr;
    // during a batched FGMRES with the mixed M_L: every new basis vector's
    // first in_stage_rows rows (the matrix block) are also written in FP32
    // to in_stage (the S~ V-cycle's input) by the scaling kernel that
    // produces it, so the preconditioner skips its input conversion; null
    // otherwise
    float *in_stage = nullptr;
    int64_t in_stage_rows = 0;
    int live_ver = 0;
    // device address of the static workspace of mds_solve_noalloc on this
    // context's device, resolved by mds_create
    double *noalloc_scratch = nullptr;
    void ensure_side_stream();
    bool pdl = true;              // launch with programmatic stream serialisation
    bool setup_phase = false;     // set-up writes level data: launch in plain stream order
    // autotuner choices by (rows, nonzeros, value type)
    std::map<std::tuple<int64_t, int64_t, int>, TuneChoice> tune_cache;

    void *raw_alloc(size_t n);
    void raw_free(void *p);
    void sync() { MDS_CUDA(cudaStreamSynchronize(stream)); }
    void post_launch() {
        if (capturing)
            capturing->launches++;
        else
            total_launches++;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) throw Error(MDS_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
    }
    // read device value (synchronises)
    template <class T> T read(const T *d) {
        MDS_CUDA(cudaMemcpyAsync(h_pin, d, sizeof(T), cudaMemcpyDeviceToHost, stream));
        sync();
        T v;
        std::memcpy(&v, h_pin, sizeof(T));
        return v;
    }
    void clear_err() { MDS_CUDA(cudaMemsetAsync(d_err, 0, sizeof(int), stream)); }
    // raise the matching status if a kernel set the device error word
    void check_err(const char *where);
};

// Capture the launches issued by f() into g (on an internal capture stream),
// then instantiate it.  Returns false, with nothing recorded and no work
// done, when the capture cannot be made.
template <class F> bool graph_capture(Ctx &c, Graph &g, F f);
// Launch a captured graph on the context stream and replay its accounting.
void graph_launch(Ctx &c, Graph &g);
// After the stream has been synchronised: add the timed launches of the last
// replay to the per-class event time.
void graph_collect(Ctx &c, Graph &g);

// Scope that brackets one launch with events when its class is being timed.
struct KTimer {
    Ctx &c;
    int cls;
    KTimerRec *rec = nullptr;
    int grec = -1;
    KTimer(Ctx &ctx, int k, double bytes, double flops = 0.0);
    ~KTimer();
};

// Launch on the context stream (programmatic dependent launch when enabled;
// every kernel begins with mds_pdl_entry()).
template <typename... KArgs, typename... Args>
inline void launch_kernel(Ctx &c, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = c.stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = c.pdl && !c.setup_phase ? 1 : 0;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
    if (e != cudaSuccess) throw Error(MDS_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
}

#define MDS_LAUNCH(ctx, cls, bytes, kern, grid, block, smem, ...)                  \
    do {                                                                           \
        ::mds::KTimer kt_((ctx), (cls), (double)(bytes));                          \
        ::mds::launch_kernel((ctx), kern, dim3(grid), dim3(block), (size_t)(smem), __VA_ARGS__); \
        (ctx).post_launch();                                                       \
    } while (0)

// as MDS_LAUNCH, also counting the launch's algorithmic floating-point operations
#define MDS_LAUNCH_F(ctx, cls, bytes, flops, kern, grid, block, smem, ...)         \
    do {                                                                           \
        ::mds::KTimer kt_((ctx), (cls), (double)(bytes), (double)(flops));         \
        ::mds::launch_kernel((ctx), kern, dim3(grid), dim3(block), (size_t)(smem), __VA_ARGS__); \
        (ctx).post_launch();                                                       \
    } while (0)

template <class F> bool graph_capture(Ctx &c, Graph &g, F f) {
    if (!c.cap_stream) MDS_CUDA(cudaStreamCreateWithFlags(&c.cap_stream, cudaStreamNonBlocking));
    cudaStream_t user = c.stream;
    MDS_CUDA(cudaStreamBeginCapture(c.cap_stream, cudaStreamCaptureModeThreadLocal));
    c.stream = c.cap_stream;
    c.capturing = &g;
    cudaGraph_t graph = nullptr;
    bool ok = true;
    try {
        f();
    } catch (...) {
        ok = false;
    }
    c.capturing = nullptr;
    c.stream = user;
    cudaError_t e = cudaStreamEndCapture(c.cap_stream, &graph);
    if (e != cudaSuccess || !ok || !graph) {
        cudaGetLastError();
        if (graph) cudaGraphDestroy(graph);
        g.recs.clear();
        g.launches = 0;
        return false;
    }
    e = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        cudaGetLastError();
        g.exec = nullptr;
        g.recs.clear();
        g.launches = 0;
        return false;
    }
    return true;
}

inline unsigned grid_for(int64_t n, int block) {
    int64_t g = (n + block - 1) / block;
    if (g < 1) g = 1;
    return (unsigned)g;
}

// Grid of a grid-stride launch over nvb blocks of work: at most as many
// blocks as the device holds at once, so that every block starts right away
// and none queues behind a long-running one (cached per kernel).
int resident_blocks(Ctx &c, const void *kern, int block);
template <class... KArgs> unsigned stride_grid(Ctx &c, void (*kern)(KArgs...), int block, int64_t nvb) {
    const int64_t cap = resident_blocks(c, (const void *)kern, block);
    int64_t g = nvb < cap ? nvb : cap;
    return (unsigned)(g < 1 ? 1 : g);
}

// Owned CSR (int32 row pointers and columns, FP64 values).
struct DCsr {
    int64_t nrow = 0, ncol = 0, nnz = 0;
    Buf rp, ci, v;
    int32_t *rowp() const { return rp.as<int32_t>(); }
    int32_t *cols() const { return ci.as<int32_t>(); }
    double *vals() const { return v.as<double>(); }
    mds_csr view() const { return mds_csr{nrow, ncol, nnz, rowp(), cols(), vals()}; }
};

inline DCsr csr_alloc(Ctx &c, int64_t nrow, int64_t ncol, int64_t nnz) {
    DCsr A;
    A.nrow = nrow;
    A.ncol = ncol;
    A.nnz = nnz;
    A.rp = Buf(&c, sizeof(int32_t) * (size_t)(nrow + 1));
    A.ci = Buf(&c, sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
    A.v = Buf(&c, sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
    return A;
}

// ---- primitives (k_prim.cu) ----
// out[0..n] = exclusive scan of cnt[0..n-1], out[n] = total; returns total.
int64_t scan_counts(Ctx &c, const int32_t *cnt, int32_t *out, int64_t n);
void fill_i32(Ctx &c, int32_t *p, int32_t v, int64_t n);
void fill_f64(Ctx &c, double *p, double v, int64_t n);
void scale_f64(Ctx &c, double *p, double a, int64_t n);  // p <- a p
// element casts of n = rows x nr interleaved entries; lm: rows to convert
void cast_f64_f32(Ctx &c, const double *in, float *out, int64_t n, const LiveMap &lm = {}, int nr = 1);
void cast_f32_f64(Ctx &c, const float *in, double *out, int64_t n, const LiveMap &lm = {}, int nr = 1);
// y = A x (FP64 CSR), nr in {1, 2, 4, 8} interleaved columns; lm: rows to
// compute (blocks of finished instances of a batch skipped)
void spmv_f64(Ctx &c, const mds_csr &A, const double *x, double *y, int kclass, int nr = 1, const LiveMap &lm = {});
// out = r - A x with out in FP64 or FP32
void spmv_sub_f64(Ctx &c, const mds_csr &A, const double *r, const double *x, double *out, int nr = 1,
                  const LiveMap &lm = {});
void spmv_sub_f64_xf(Ctx &c, const mds_csr &A, const double *r, const float *x, float *out, int nr = 1,
                     const LiveMap &lm = {});
void spmv_sub_f64_to_f32(Ctx &c, const mds_csr &A, const double *r, const double *x, float *out, int nr = 1,
                         const LiveMap &lm = {});

// ---- assembly (k_assemble.cu) ----
struct SystemData {
    int64_t n_m = 0, n_f = 0;
    int nrhs = 1;
    // packed instances: instance k owns matrix rows [moff[k], moff[k+1]) and
    // fracture rows n_m + [foff[k], foff[k+1])
    std::vector<int64_t> moff, foff;
    // Cartesian instances of the primal form: grid dimension and cells per
    // side of each instance (the matrix block, and S~, is then a 5- or
    // 7-point stencil per instance); stencil = false otherwise
    bool stencil = false;
    int dim = 0;
    std::vector<int32_t> side;
    DCsr full;
    DCsr blk[4];
    Buf b;  // [nrhs][N]
};
// flux: the paper's partition (all pressures; interface fluxes) instead of
// the primal [matrix; fracture] system
void assemble_instance(Ctx &c, const mds_instance &inst, SystemData &out, bool flux = false);
// pack several assembled instances into one block-diagonal system
void pack_instances(Ctx &c, std::vector<SystemData> &parts, SystemData &out);
// assemble K instances of the primal form straight into the packed system
void assemble_batch_primal(Ctx &c, const mds_instance *inst, int K, SystemData &out);
void split_blocks(Ctx &c, const mds_csr &full, int64_t n_m, DCsr blk[4]);
void merge_blocks(Ctx &c, const mds_csr blk[4], int64_t n_m, int64_t n_f, DCsr &full);

// ---- set-up (k_setup.cu) ----
DCsr schur_build(Ctx &c, const mds_csr &Amm, const mds_csr &Amf, const mds_csr &Afm,
                 const mds_csr &Aff, Buf &dk);

struct Level {
    DCsr A;           // FP64 master
    Buf agg;          // int32 [n], next-level aggregate or -1
    Buf roots;        // int8 [n]
    Buf mem_off;      // int32 [nc+1] members of each next-level aggregate
    Buf mem;          // int32 [#aggregated], ascending within an aggregate
    int64_t mem_count = 0;  // #aggregated vertices
    // the finest level of a large hierarchy: its V-cycle kernels are the ones
    // counted in the timed classes (coarse levels launch as KC_NONE)
    bool timed_level = false;
    bool stored = false;  // runs the stored form where the fused one would apply
    Buf l1;           // FP64 [n]
    Buf dinv;         // [n] 1/l1 in the vector precision
    bool has_coarse = false;
    int64_t nc = 0;
    bool smoothed = false;    // smoothed prolongator P (and R = P^T) instead of agg injection
    DCsr P, R;
    Buf Pv_lp, Rv_lp;         // their values in FP32 (FP32 and lower-precision hierarchies)
    // storage used by the V-cycle
    int vt = VT_F64;  // value type
    int fmt = FMT_CSR;
    int G = 4;        // CSR lanes per row
    Buf vals_lp;      // CSR values in vt (not for FP64)
    Buf rscale;       // float [n] power-of-two row scales (BF16/FP16)
    int sell_c = 32;
    int64_t sell_nslice = 0, sell_nnz = 0;
    Buf sell_ptr, sell_len, sell_col, sell_val, sell_perm;
    Buf b, x, r, y, d, t;  // work vectors in the vector precision
    Buf seg_d;             // int64 [K + 1] instance row offsets (packed batches)
    std::vector<int64_t> seg_h;  // the same on the host
    Buf ck;                // int32 [2 chunks] least / greatest instance of each 256-row chunk
    mutable Buf rt;        // int64 chunk ranges of the live instances (compacted launches)
    mutable int64_t rt_nch = 0;
    mutable int rt_ver = -1;
    // stencil storage (FMT_DIA): plane d holds each row's coefficient of the
    // neighbour at offset o_d (ascending), zero where the row has none
    int dia_D = 0;         // 5 (2D) or 7 (3D); 0: the level is no stencil
    int64_t dia_stride = 0;  // rows per plane (n padded to a multiple of 32)
    bool dia_bulk = false;   // stencil kernel staging each row block by bulk copies
    Buf dia_val;           // [dia_D][dia_stride] in the storage type
    Buf dia_seg;           // int64 [K + 1] instance row offsets
    Buf dia_side;          // int32 [K] cells per side
    Buf dia_ck;            // int32 [4 chunks]: (first row, last row, cells per side, instance) of the
                           // instance of each 256-row chunk; instance -1 for a chunk holding two
    int K = 1;             // instances (packed batches)
    int sell_sigma = 1;    // SELL sorting window (rows)
};

// Share of the rows [seg[k], seg[k+1]) of live instances (host flags).
inline double live_share(const std::vector<int8_t> &live, const std::vector<int64_t> &seg) {
    const int K = (int)seg.size() - 1;
    if (K < 1 || (int)live.size() < K || seg[K] <= 0) return 1.0;
    int64_t r = 0;
    for (int k = 0; k < K; k++)
        if (live[k]) r += seg[k + 1] - seg[k];
    return (double)r / (double)seg[K];
}

// Chunk ranges of the live instances of a row space (instance k owns the
// rows [a[k], a[k+1]) and, when b is given, also [n1 + b[k], n1 + b[k+1])),
// in the LiveMap::rt layout; returns the number of chunks.
int64_t live_ranges(const std::vector<int8_t> &live, const std::vector<int64_t> &a, const std::vector<int64_t> *b,
                    int64_t n1, std::vector<int64_t> &t);
// Upload t to dev (allocated for up to K ranges) on the context stream.
void upload_ranges(Ctx &c, Buf &dev, const std::vector<int64_t> &t, int K);

// The liveness map of one level (every row live outside a batched solve).
inline LiveMap level_live(Ctx &c, const Level &L) {
    LiveMap m;
    if (c.live && L.K > 1 && L.ck.p) {
        m.ck = L.ck.as<int32_t>();
        m.live = c.live;
        m.frac = live_share(c.live_host, L.seg_h);
        if (c.compact) {
            if (L.rt_ver != c.live_ver) {
                std::vector<int64_t> t;
                L.rt_nch = live_ranges(c.live_host, L.seg_h, nullptr, 0, t);
                upload_ranges(c, L.rt, t, L.K);
                L.rt_ver = c.live_ver;
            }
            m.rt = L.rt.as<int64_t>();
            m.nch = L.rt_nch;
        }
    }
    return m;
}

// The chunk table of a row space of `rows` rows whose instance k owns the
// rows [a[k], a[k+1]) and, when b is given, also [n1 + b[k], n1 + b[k+1]).
Buf live_chunks(Ctx &c, int64_t rows, const std::vector<int64_t> &a, const std::vector<int64_t> *b = nullptr,
                int64_t n1 = 0);

// One diagonal block of the coarsest level: its first row, the start of its
// n x n row-major matrices, its size.
struct DBlk {
    int64_t row, off;
    int32_t n;
};
struct DenseBlocks {
    int K = 0;
    int64_t nmax = 0, nrow = 0, total = 0;  // largest block, rows, sum of n_b^2
    std::vector<DBlk> host;
    Buf blk;              // DBlk [K]
    Buf tiles;            // int2 [ntiles]: (block, first row) of each 32-row tile of a block
    int64_t ntiles = 0;
};

struct Hierarchy {
    std::vector<Level> lv;
    // instances of a packed batch: per level, the row offsets [K + 1] of
    // each instance (every instance is coarsened as if alone); K = 1 for one
    int K = 1;
    std::vector<std::vector<int64_t>> seg;
    DenseBlocks db;   // the coarsest level's diagonal blocks (one per instance)
    bool dense = false;
    bool diagonal = false;  // last level has no couplings: x = b / a_ii
    int64_t nd = 0;
    Buf Ainv;         // FP64 inverse of each coarsest block (db)
    int prec = 64;    // vector precision: 64 or 32
    int smoother = 0;
    int sweeps = 1;
    int cheb_degree = 2;
    int form = 0;     // MDS_FORM_*
    int nr_cap = 0;   // columns the level work vectors hold
    int tune_nr = 1;  // columns the storage autotuner times with (those of the system's right-hand sides)
    bool use_tail = true;  // run the coarse end of the V-cycle as one cluster kernel
    // level 0 is a Cartesian stencil (the S~ of primal assembled systems):
    // grid dimension and cells per side of each instance (empty: unknown)
    int st_dim = 0;
    std::vector<int32_t> st_side;
};

// seg0: the instances' row offsets [K + 1] of a packed batch (NULL: one
// instance); every instance is coarsened as if alone (MIS-2 keys by the row's
// index within its instance, stop once every instance has at most n_coarse
// rows, block-diagonal coarsest solve).
void amg_setup(Ctx &c, const mds_csr &A, const mds_setup_opts &o, Hierarchy &h,
               const std::vector<int64_t> *seg0 = nullptr);
// bit 1: some row holds an off-diagonal entry (or no diagonal); bit 2: some
// diagonal entry is missing or not negative (synchronises)
int row_kinds(Ctx &c, const mds_csr &A);
// per-level value storage and format (k_vcycle.cu), run at the end of amg_setup
void level_storage(Ctx &c, Hierarchy &h, const mds_setup_opts &o);

// ---- dense (k_dense.cu) ----
// Cholesky of each diagonal block [seg[k], seg[k+1]) of the SPD matrix A
// (stored densely), then its inverse; fills the block table.
void dense_spd_inverse(Ctx &c, const mds_csr &A, const std::vector<int64_t> &seg, Buf &Ainv, DenseBlocks &db);
// y = M x for the block-diagonal inverse M, nr in {1, 2, 4, 8} interleaved
// columns; on (optional): per block, whether to compute it
void dense_apply(Ctx &c, const DenseBlocks &db, const double *M, int nr, const double *x, double *y,
                 const int8_t *on = nullptr);
void dense_apply(Ctx &c, const DenseBlocks &db, const double *M, int nr, const float *x, float *y,
                 const int8_t *on = nullptr);

// ---- V-cycle (k_vcycle.cu) ----
// x = V(b) on level 0 of h for nr in {1, 2, 4, 8} interleaved columns; b and
// x in the hierarchy's vector precision.
void vcycle_apply(Ctx &c, Hierarchy &h, const void *b, void *x, int nr = 1);
// An FP32 V-cycle (h.prec 32) whose top level writes its result to z64 (FP64,
// the same interleaved rows) instead of x where its last operation allows;
// returns false when x was written instead (the caller converts).
bool vcycle_apply_to64(Ctx &c, Hierarchy &h, const float *b, float *x, double *z64, int nr);
// grow the level work vectors to hold nr interleaved columns
void hierarchy_reserve(Ctx &c, Hierarchy &h, int nr);

// ---- Krylov (k_krylov.cu) ----
struct KrylovWork;
// z = M r on nr interleaved columns (api.cu)
void precond_apply(mds_precond p, const double *r, double *z, int nr);
}  // namespace mds

// Handle structs (opaque in the C ABI).
struct mds_ctx_s {
    mds::Ctx c;
};

struct mds_system_s {
    mds::Ctx *ctx = nullptr;
    int64_t n_m = 0, n_f = 0;
    int nrhs = 0;
    int n_inst = 1;
    mds_csr view[5]{};       // 0..3 blocks, 4 full
    mds::SystemData own;     // owned storage (blocks borrowed for from_csr)
    const double *b = nullptr;
};

struct mds_precond_s {
    mds::Ctx *ctx = nullptr;
    mds_system sys = nullptr;
    mds_setup_opts o{};
    mds::DCsr S;
    mds::Buf dk;
    mds::Hierarchy h[2];
    bool has_f = false;
    bool ff_negative = false;  // every a_ii of A_ff < 0 (flux block of the paper's partition)
    mds::Buf tf64;            // Algorithm 1 work vector (interleaved columns)
    int64_t tf_cap = 0;
};
