// The C ABI of libmdsolve (include/mdsolve.h): contexts, memory, systems,
// preconditioner set-up, Algorithm 1, solves and timing.
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstddef>
#include <cstdio>
#include <new>

#include "internal.cuh"
#include "krylov.cuh"

namespace mds {

// ---------------------------------------------------------------- memory

Buf::Buf(Ctx *c, size_t n) : ctx(c), bytes(n) {
    if (n == 0) n = 1;
    p = c->raw_alloc(n);
}

Buf::~Buf() { reset(); }

Buf &Buf::operator=(Buf &&o) noexcept {
    if (this != &o) {
        reset();
        ctx = o.ctx;
        p = o.p;
        bytes = o.bytes;
        o.p = nullptr;
        o.bytes = 0;
    }
    return *this;
}

void Buf::reset() {
    if (p && ctx) ctx->raw_free(p);
    p = nullptr;
    bytes = 0;
}

// The second stream and its fork / join events (block-diagonal
// preconditioner); created once per context.
void Ctx::ensure_side_stream() {
    if (side_stream) return;
    MDS_CUDA(cudaStreamCreateWithFlags(&side_stream, cudaStreamNonBlocking));
    MDS_CUDA(cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming));
    MDS_CUDA(cudaEventCreateWithFlags(&ev_join, cudaEventDisableTiming));
}

void *Ctx::raw_alloc(size_t n) {
    void *p = nullptr;
    if (custom_alloc) {
        p = alloc.alloc(n, alloc.user);
        if (!p) throw Error(MDS_ERR_OOM, "allocator returned NULL for " + std::to_string(n) + " bytes");
    } else {
        cudaError_t e = cudaMallocFromPoolAsync(&p, n, pool, stream);
        if (e != cudaSuccess) {
            cudaGetLastError();
            throw Error(MDS_ERR_OOM, "cudaMallocFromPoolAsync(" + std::to_string(n) + "): " + cudaGetErrorString(e));
        }
    }
    return p;
}

int resident_blocks(Ctx &c, const void *kern, int block) {
    auto it = c.resident.find(kern);
    if (it != c.resident.end()) return it->second;
    int per = 0;
    MDS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, block, 0));
    const int total = (per > 0 ? per : 1) * (c.num_sms > 0 ? c.num_sms : 1);
    c.resident[kern] = total;
    return total;
}

void Ctx::raw_free(void *p) {
    if (custom_alloc)
        alloc.free(p, alloc.user);
    else
        cudaFreeAsync(p, stream);
}

void Ctx::check_err(const char *where) {
    int e = read(d_err);
    if (!e) return;
    MDS_CUDA(cudaMemsetAsync(d_err, 0, sizeof(int), stream));
    std::string w(where);
    if (e & DERR_DUP_FACE) throw Error(MDS_ERR_INVALID, w + ": two fracture cells on one face");
    if (e & DERR_BAD_FRACTURE) throw Error(MDS_ERR_INVALID, w + ": fracture cell not on an interior face");
    if (e & DERR_CAPACITY) throw Error(MDS_ERR_CAPACITY, w + ": a row exceeded the kernel's row capacity");
    if (e & DERR_NOT_SPD) throw Error(MDS_ERR_NOT_SPD, w + ": non-positive pivot");
    if (e & DERR_ZERO_DIAG) throw Error(MDS_ERR_ZERO_DIAG, w + ": zero diagonal");
    if (e & DERR_TIMEOUT) throw Error(MDS_ERR_TIMEOUT, w + ": an asynchronous copy did not complete");
    throw Error(MDS_ERR_NONFINITE, w + ": non-finite value");
}

KTimer::KTimer(Ctx &ctx, int k, double b, double f) : c(ctx), cls(k) {
    if (k < 0 || k >= MDS_KCLASS_COUNT) return;
    if (c.capturing) {
        GraphRec r{k, b, f, c.timing[k] && !c.timing_suspended, nullptr, nullptr};
        if (r.timed) {
            MDS_CUDA(cudaEventCreate(&r.e0));
            MDS_CUDA(cudaEventCreate(&r.e1));
            // an external record becomes an event node of the graph, so the
            // event is written at every replay
            MDS_CUDA(cudaEventRecordWithFlags(r.e0, c.stream, cudaEventRecordExternal));
        }
        c.capturing->recs.push_back(r);
        grec = (int)c.capturing->recs.size() - 1;
        return;
    }
    c.launches[k]++;
    c.bytes[k] += b;
    c.flops[k] += f;
    if (!c.timing[k] || c.timing_suspended) return;
    c.tlaunches[k]++;
    c.tbytes[k] += b;
    c.tflops[k] += f;
    auto &v = c.evs[k];
    if (c.ev_used[k] == v.size()) {
        KTimerRec r;
        MDS_CUDA(cudaEventCreate(&r.e0));
        MDS_CUDA(cudaEventCreate(&r.e1));
        v.push_back(r);
    }
    rec = &v[c.ev_used[k]++];
    cudaEventRecord(rec->e0, c.stream);
}

KTimer::~KTimer() {
    if (rec) cudaEventRecord(rec->e1, c.stream);
    if (grec >= 0 && c.capturing && c.capturing->recs[grec].timed)
        cudaEventRecordWithFlags(c.capturing->recs[grec].e1, c.stream, cudaEventRecordExternal);
}

Graph::~Graph() {
    if (exec) cudaGraphExecDestroy(exec);
    for (auto &r : recs)
        if (r.timed) {
            cudaEventDestroy(r.e0);
            cudaEventDestroy(r.e1);
        }
}

void graph_launch(Ctx &c, Graph &g) {
    MDS_CUDA(cudaGraphLaunch(g.exec, c.stream));
    for (auto &r : g.recs) {
        c.launches[r.cls]++;
        c.bytes[r.cls] += r.bytes * g.scale;
        c.flops[r.cls] += r.flops * g.scale;
    }
    c.total_launches += g.launches;
}

void graph_collect(Ctx &c, Graph &g) {
    for (auto &r : g.recs)
        if (r.timed && c.timing[r.cls]) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, r.e0, r.e1) == cudaSuccess) {
                c.graph_ms[r.cls] += t;
                c.tlaunches[r.cls]++;
                c.tbytes[r.cls] += r.bytes * g.scale;
                c.tflops[r.cls] += r.flops * g.scale;
            }
        }
}

}  // namespace mds

using namespace mds;

#define API_BEGIN try {
#define API_END(ctxp)                                                     \
    }                                                                     \
    catch (const Error &e) {                                              \
        if (ctxp) (ctxp)->last_error = e.msg;                             \
        return e.code;                                                    \
    }                                                                     \
    catch (const std::bad_alloc &) {                                      \
        if (ctxp) (ctxp)->last_error = "host allocation failed";          \
        return MDS_ERR_OOM;                                               \
    }                                                                     \
    catch (...) {                                                         \
        if (ctxp) (ctxp)->last_error = "unexpected exception";            \
        return MDS_ERR_INVALID;                                           \
    }                                                                     \
    return MDS_OK;

namespace mds {
// Waits for the context's asynchronous solve, if one is running; its result
// stays for mds_solve_wait.
static void async_join(Ctx *c) {
    if (c && c->async.th.joinable()) c->async.th.join();
}
}  // namespace mds

extern "C" {

const char *mds_error_string(int s) {
    switch (s) {
        case MDS_OK: return "ok";
        case MDS_WARN_NOT_CONVERGED: return "not converged within max_iters";
        case MDS_ERR_INVALID: return "invalid argument";
        case MDS_ERR_CUDA: return "CUDA runtime error";
        case MDS_ERR_OOM: return "out of device memory";
        case MDS_ERR_NOT_SPD: return "coarsest matrix not positive definite";
        case MDS_ERR_BREAKDOWN: return "Krylov breakdown";
        case MDS_ERR_NONFINITE: return "non-finite value";
        case MDS_ERR_CAPACITY: return "row capacity exceeded";
        case MDS_ERR_TIMEOUT: return "iteration bound exceeded";
        case MDS_ERR_ZERO_DIAG: return "zero diagonal in A_ff";
        default: return "unknown status";
    }
}

const char *mds_last_error(mds_ctx ctx) { return ctx ? ctx->c.last_error.c_str() : "null context"; }

int mds_create(mds_ctx *out, int device, void *stream, const mds_allocator *alloc) {
    if (!out) return MDS_ERR_INVALID;
    *out = nullptr;
    mds_ctx h = new (std::nothrow) mds_ctx_s;
    if (!h) return MDS_ERR_OOM;
    Ctx *c = &h->c;
    try {
        int ndev = 0;
        MDS_CUDA(cudaGetDeviceCount(&ndev));
        MDS_REQUIRE(device >= 0 && device < ndev, MDS_ERR_INVALID, "no such CUDA device");
        MDS_CUDA(cudaSetDevice(device));
        c->device = device;
        c->owner = h;
        // MDS_PDL=0 launches without programmatic dependent launch (diagnosis)
        if (const char *e = std::getenv("MDS_PDL")) c->pdl = std::atoi(e) != 0;
        c->stream = (cudaStream_t)stream;
        if (alloc && alloc->alloc && alloc->free) {
            c->alloc = *alloc;
            c->custom_alloc = true;
        } else {
            cudaMemPoolProps pp{};
            pp.allocType = cudaMemAllocationTypePinned;
            pp.location.type = cudaMemLocationTypeDevice;
            pp.location.id = device;
            MDS_CUDA(cudaMemPoolCreate(&c->pool, &pp));
            uint64_t keep = UINT64_MAX;
            MDS_CUDA(cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &keep));
        }
        MDS_CUDA(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device));
        MDS_CUDA(cudaMalloc(&c->d_err, sizeof(int)));
        MDS_CUDA(cudaMemset(c->d_err, 0, sizeof(int)));
        MDS_CUDA(cudaMallocHost(&c->h_pin, Ctx::PIN_BYTES));
        // the static workspace of mds_solve_noalloc: resolving its address
        // loads the module holding it, here rather than inside a later solve
        c->noalloc_scratch = noalloc_scratch_lookup();
    } catch (const Error &e) {
        int code = e.code;
        if (c->d_err) cudaFree(c->d_err);
        if (c->h_pin) cudaFreeHost(c->h_pin);
        if (c->pool) cudaMemPoolDestroy(c->pool);
        delete h;
        return code;
    }
    *out = h;
    return MDS_OK;
}

static void ctx_release(mds_ctx ctx) {
    Ctx &c = ctx->c;
    cudaSetDevice(c.device);
    cudaStreamSynchronize(c.stream);
    for (int k = 0; k < MDS_KCLASS_COUNT; k++)
        for (auto &r : c.evs[k]) {
            cudaEventDestroy(r.e0);
            cudaEventDestroy(r.e1);
        }
    cudaFree(c.d_err);
    cudaFreeHost(c.h_pin);
    if (c.cap_stream) cudaStreamDestroy(c.cap_stream);
    if (c.side_stream) cudaStreamDestroy(c.side_stream);
    if (c.ev_fork) cudaEventDestroy(c.ev_fork);
    if (c.ev_join) cudaEventDestroy(c.ev_join);
    if (c.pool) {
        cudaStreamSynchronize(c.stream);
        cudaMemPoolDestroy(c.pool);
    }
    delete ctx;
}

// Systems and preconditioners keep their context alive: destroying a context
// that still has dependents only marks it, and the last dependent's destroy
// releases it.
static void ctx_drop_dependent(Ctx *c) {
    if (--c->dependents == 0 && c->destroy_requested) ctx_release(static_cast<mds_ctx>(c->owner));
}

int mds_destroy(mds_ctx ctx) {
    if (!ctx) return MDS_ERR_INVALID;
    async_join(&ctx->c);
    if (ctx->c.destroy_requested) return MDS_ERR_INVALID;
    if (ctx->c.dependents > 0) {
        ctx->c.destroy_requested = true;
        return MDS_OK;
    }
    ctx_release(ctx);
    return MDS_OK;
}

int mds_set_stream(mds_ctx ctx, void *stream) {
    if (!ctx) return MDS_ERR_INVALID;
    async_join(&ctx->c);
    ctx->c.stream = (cudaStream_t)stream;
    return MDS_OK;
}

static int assemble_any(mds_ctx ctx, const mds_instance *inst, int n_inst, mds_system *out, bool flux) {
    if (!ctx || !inst || !out || n_inst < 1) return MDS_ERR_INVALID;
    async_join(&ctx->c);
    Ctx *c = &ctx->c;
    *out = nullptr;
    API_BEGIN
    MDS_CUDA(cudaSetDevice(c->device));
    auto *s = new mds_system_s;
    try {
        s->ctx = c;
        if (n_inst == 1) {
            assemble_instance(*c, inst[0], s->own, flux);
        } else if (!flux) {
            assemble_batch_primal(*c, inst, n_inst, s->own);
        } else {
            std::vector<SystemData> parts(n_inst);
            for (int k = 0; k < n_inst; k++) assemble_instance(*c, inst[k], parts[k], flux);
            pack_instances(*c, parts, s->own);
        }
        s->n_m = s->own.n_m;
        s->n_f = s->own.n_f;
        s->nrhs = s->own.nrhs;
        s->n_inst = n_inst;
        for (int q = 0; q < 4; q++) s->view[q] = s->own.blk[q].view();
        s->view[4] = s->own.full.view();
        s->b = s->own.b.as<double>();
    } catch (...) {
        delete s;
        throw;
    }
    c->dependents++;
    *out = s;
    API_END(c)
}

int mds_assemble_batch(mds_ctx ctx, const mds_instance *inst, int n_inst, mds_system *out) {
    return assemble_any(ctx, inst, n_inst, out, false);
}

int mds_assemble(mds_ctx ctx, const mds_instance *inst, mds_system *out) {
    return assemble_any(ctx, inst, 1, out, false);
}

int mds_assemble_flux(mds_ctx ctx, const mds_instance *inst, mds_system *out) {
    return assemble_any(ctx, inst, 1, out, true);
}

int mds_system_instances(mds_system sys, int *n_inst, int64_t *m_off, int64_t *f_off) {
    if (!sys) return MDS_ERR_INVALID;
    if (n_inst) *n_inst = sys->n_inst;
    for (int k = 0; k <= sys->n_inst; k++) {
        if (m_off) m_off[k] = sys->own.moff.size() > (size_t)k ? sys->own.moff[k] : (k ? sys->n_m : 0);
        if (f_off) f_off[k] = sys->own.foff.size() > (size_t)k ? sys->own.foff[k] : (k ? sys->n_f : 0);
    }
    return MDS_OK;
}

static void check_csr(const mds_csr *A, int64_t nrow, int64_t ncol, const char *name) {
    MDS_REQUIRE(A && A->nrow == nrow && A->ncol == ncol && A->nnz >= 0, MDS_ERR_INVALID,
                std::string("block ") + name + " has the wrong shape");
    MDS_REQUIRE(A->row_ptr && (A->nnz == 0 || (A->col && A->val)), MDS_ERR_INVALID,
                std::string("block ") + name + " has null arrays");
}

int mds_system_from_csr(mds_ctx ctx, const mds_csr *Amm, const mds_csr *Amf, const mds_csr *Afm, const mds_csr *Aff,
                        const double *b, mds_system *out) {
    if (!ctx || !out || !Amm || !Aff) return MDS_ERR_INVALID;
    Ctx *c = &ctx->c;
    async_join(c);
    *out = nullptr;
    API_BEGIN
    MDS_CUDA(cudaSetDevice(c->device));
    int64_t nm = Amm->nrow, nf = Aff->nrow;
    check_csr(Amm, nm, nm, "A_mm");
    check_csr(Amf, nm, nf, "A_mf");
    check_csr(Afm, nf, nm, "A_fm");
    check_csr(Aff, nf, nf, "A_ff");
    MDS_REQUIRE(nm + nf < INT32_MAX, MDS_ERR_INVALID, "too many unknowns");
    auto *s = new mds_system_s;
    try {
        s->ctx = c;
        s->n_m = nm;
        s->n_f = nf;
        s->nrhs = 1;
        s->view[0] = *Amm;
        s->view[1] = *Amf;
        s->view[2] = *Afm;
        s->view[3] = *Aff;
        merge_blocks(*c, s->view, nm, nf, s->own.full);
        s->view[4] = s->own.full.view();
        s->own.moff = {0, nm};
        s->own.foff = {0, nf};
        s->own.b = Buf(c, sizeof(double) * (size_t)(nm + nf));
        if (b)
            MDS_CUDA(cudaMemcpyAsync(s->own.b.p, b, sizeof(double) * (size_t)(nm + nf), cudaMemcpyDeviceToDevice,
                                     c->stream));
        else
            fill_f64(*c, s->own.b.as<double>(), 0.0, nm + nf);
        s->b = s->own.b.as<double>();
        c->sync();
    } catch (...) {
        delete s;
        throw;
    }
    c->dependents++;
    *out = s;
    API_END(c)
}

int mds_system_destroy(mds_system sys) {
    if (!sys) return MDS_ERR_INVALID;
    Ctx *c = sys->ctx;
    async_join(c);
    cudaSetDevice(c->device);
    delete sys;
    ctx_drop_dependent(c);
    return MDS_OK;
}

int mds_system_info(mds_system sys, int64_t *n_m, int64_t *n_f, int *nrhs, int64_t nnz[5]) {
    if (!sys) return MDS_ERR_INVALID;
    if (n_m) *n_m = sys->n_m;
    if (n_f) *n_f = sys->n_f;
    if (nrhs) *nrhs = sys->nrhs;
    if (nnz)
        for (int q = 0; q < 5; q++) nnz[q] = sys->view[q].nnz;
    return MDS_OK;
}

int mds_system_view(mds_system sys, mds_csr blocks[5], const double **b) {
    if (!sys) return MDS_ERR_INVALID;
    if (blocks)
        for (int q = 0; q < 5; q++) blocks[q] = sys->view[q];
    if (b) *b = sys->b;
    return MDS_OK;
}

int mds_setup_opts_default(mds_setup_opts *o) {
    if (!o) return MDS_ERR_INVALID;
    o->theta = -1.0;  // automatic: 0.08, or 0.04 with smoothed prolongation (resolved by mds_setup)
    o->n_coarse = 512;
    o->max_levels = 25;
    o->stall_ratio = 0.9;
    o->seed = 0x220603203ULL;
    o->smoother = MDS_SMOOTHER_L1JACOBI;
    o->precision = MDS_PREC_FP64;
    o->lowp_from_level = 1;
    o->kind = MDS_BLOCK_LOWER;
    o->format = MDS_FORMAT_CSR;
    o->sell_c = 32;
    o->sell_sigma = 1;
    o->sweeps = 1;
    o->prolongation = MDS_PROLONG_PIECEWISE;
    o->coarse_tail = 0;
    o->cheb_degree = 2;
    o->level_form = MDS_FORM_AUTO;
    return MDS_OK;
}

int mds_setup(mds_ctx ctx, mds_system sys, const mds_setup_opts *opts, mds_precond *out) {
    if (!ctx || !sys || !out) return MDS_ERR_INVALID;
    Ctx *c = &ctx->c;
    async_join(c);
    *out = nullptr;
    API_BEGIN
    MDS_CUDA(cudaSetDevice(c->device));
    mds_setup_opts o;
    mds_setup_opts_default(&o);
    if (opts) o = *opts;
    MDS_REQUIRE(o.precision == MDS_PREC_FP64 || o.precision == MDS_PREC_FP32 || o.precision == MDS_PREC_BF16 ||
                    o.precision == MDS_PREC_FP16,
                MDS_ERR_INVALID, "unknown precision");
    MDS_REQUIRE(o.smoother == MDS_SMOOTHER_L1JACOBI || o.smoother == MDS_SMOOTHER_CHEBYSHEV, MDS_ERR_INVALID,
                "unknown smoother");
    MDS_REQUIRE(o.format >= MDS_FORMAT_AUTO && o.format <= MDS_FORMAT_STENCIL_BULK, MDS_ERR_INVALID, "unknown format");
    MDS_REQUIRE(o.level_form >= MDS_FORM_AUTO && o.level_form <= MDS_FORM_STORED, MDS_ERR_INVALID,
                "unknown level form");
    MDS_REQUIRE(o.sell_c == 8 || o.sell_c == 16 || o.sell_c == 32, MDS_ERR_INVALID, "sell_c must be 8, 16 or 32");
    MDS_REQUIRE(o.sell_sigma == 1 || (o.sell_sigma % o.sell_c == 0 && o.sell_sigma <= 1024), MDS_ERR_INVALID,
                "sell_sigma must be 1 or a multiple of sell_c up to 1024");
    MDS_REQUIRE(o.sweeps >= 1 && o.sweeps <= 8, MDS_ERR_INVALID, "sweeps must be 1..8");
    MDS_REQUIRE(o.cheb_degree >= 1 && o.cheb_degree <= 8, MDS_ERR_INVALID, "cheb_degree must be 1..8");
    MDS_REQUIRE(o.prolongation == MDS_PROLONG_PIECEWISE || o.prolongation == MDS_PROLONG_SMOOTHED, MDS_ERR_INVALID,
                "unknown prolongation");
    MDS_REQUIRE(o.kind >= 0 && o.kind <= 2, MDS_ERR_INVALID, "bad preconditioner kind");
    if (o.theta < 0.0) o.theta = o.prolongation == MDS_PROLONG_SMOOTHED ? 0.04 : 0.08;
    MDS_REQUIRE(o.theta >= 0.0 && o.n_coarse >= 1 && o.n_coarse <= 8192, MDS_ERR_INVALID, "bad AMG options");
    auto *p = new mds_precond_s;
    // set-up kernels write the level data that V-cycle kernels read before
    // their dependency wait: launch them in plain stream order, and finish
    // them before returning
    struct SetupPhase {
        Ctx *c;
        explicit SetupPhase(Ctx *cc) : c(cc) { c->setup_phase = true; }
        ~SetupPhase() { c->setup_phase = false; }
    } phase(c);
    try {
        p->ctx = c;
        p->sys = sys;
        p->o = o;
        p->S = schur_build(*c, sys->view[0], sys->view[1], sys->view[2], sys->view[3], p->dk);
        // the storage autotuner times with the column count of the system's
        // right-hand sides (interleaved in a multi-column solve)
        p->h[0].tune_nr = p->h[1].tune_nr = sys->nrhs;
        // a packed batch: every instance's blocks coarsened as if alone
        const bool packed = sys->n_inst > 1 && sys->own.moff.size() == (size_t)sys->n_inst + 1 &&
                            sys->own.foff.size() == (size_t)sys->n_inst + 1;
        // the S~ of a primal system assembled here is a Cartesian stencil on
        // its finest level (Eq. (7) restores the links cut by fractures)
        if (sys->own.stencil && !sys->own.side.empty()) {
            p->h[0].st_dim = sys->own.dim;
            p->h[0].st_side = sys->own.side;
        }
        amg_setup(*c, p->S.view(), o, p->h[0], packed ? &sys->own.moff : nullptr);
        p->has_f = sys->n_f > 0;
        if (p->has_f) {
            amg_setup(*c, sys->view[3], o, p->h[1], packed ? &sys->own.foff : nullptr);
            p->ff_negative = !(row_kinds(*c, sys->view[3]) & 2);
        }
        int64_t mx = sys->n_m > sys->n_f ? sys->n_m : sys->n_f;
        p->tf64 = Buf(c, sizeof(double) * (size_t)(mx > 0 ? mx : 1));
        p->tf_cap = mx;
        // B_D runs its two V-cycles on two streams: create the second one
        // now, so that applying the preconditioner creates nothing
        if (o.kind == MDS_BLOCK_DIAG && p->has_f) c->ensure_side_stream();
        c->sync();
    } catch (...) {
        delete p;
        throw;
    }
    c->dependents++;
    *out = p;
    API_END(c)
}

int mds_precond_destroy(mds_precond p) {
    if (!p) return MDS_ERR_INVALID;
    Ctx *c = p->ctx;
    async_join(c);
    cudaSetDevice(c->device);
    delete p;
    ctx_drop_dependent(c);
    return MDS_OK;
}

int mds_precond_info(mds_precond p, int block, int *nlevels, int64_t *level_n, int64_t *level_nnz, int *dense) {
    if (!p || block < 0 || block > 1) return MDS_ERR_INVALID;
    if (block == 1 && !p->has_f) {
        if (nlevels) *nlevels = 0;
        if (dense) *dense = 0;
        return MDS_OK;
    }
    const Hierarchy &h = p->h[block];
    if (nlevels) *nlevels = (int)h.lv.size();
    for (size_t l = 0; l < h.lv.size() && l < 32; l++) {
        if (level_n) level_n[l] = h.lv[l].A.nrow;
        if (level_nnz) level_nnz[l] = h.lv[l].A.nnz;
    }
    if (dense) *dense = h.dense ? 1 : (h.diagonal ? 2 : 0);
    return MDS_OK;
}

int mds_precond_level(mds_precond p, int block, int level, mds_csr *A, const int32_t **agg, const int8_t **roots) {
    if (!p || block < 0 || block > 1 || (block == 1 && !p->has_f)) return MDS_ERR_INVALID;
    const Hierarchy &h = p->h[block];
    if (level < 0 || level >= (int)h.lv.size()) return MDS_ERR_INVALID;
    const Level &L = h.lv[level];
    if (A) *A = L.A.view();
    if (agg) *agg = L.has_coarse ? L.agg.as<int32_t>() : nullptr;
    if (roots) *roots = L.roots.as<int8_t>();
    return MDS_OK;
}

int mds_precond_prolongator(mds_precond p, int block, int level, mds_csr *P) {
    if (!p || !P || block < 0 || block > 1 || (block == 1 && !p->has_f)) return MDS_ERR_INVALID;
    const Hierarchy &h = p->h[block];
    if (level < 0 || level >= (int)h.lv.size()) return MDS_ERR_INVALID;
    const Level &L = h.lv[level];
    *P = L.smoothed ? L.P.view() : mds_csr{L.A.nrow, L.nc, 0, nullptr, nullptr, nullptr};
    return MDS_OK;
}

int mds_precond_level_storage(mds_precond p, int block, int level, int *value_type, const void **values,
                              const float **row_scale, const void **dinv, int *format) {
    if (!p || block < 0 || block > 1 || (block == 1 && !p->has_f)) return MDS_ERR_INVALID;
    const Hierarchy &h = p->h[block];
    if (level < 0 || level >= (int)h.lv.size()) return MDS_ERR_INVALID;
    const Level &L = h.lv[level];
    static const int code[] = {MDS_PREC_FP64, MDS_PREC_FP32, MDS_PREC_BF16, MDS_PREC_FP16};
    const bool dense_last = level + 1 == (int)h.lv.size() && h.dense;
    if (value_type) *value_type = code[L.vt];
    if (values) *values = dense_last ? nullptr : L.vt == VT_F64 ? (const void *)L.A.vals() : L.vals_lp.p;
    if (row_scale) *row_scale = L.rscale.p ? L.rscale.as<float>() : nullptr;
    if (dinv) *dinv = L.dinv.p;
    if (format)
        *format = L.fmt == FMT_DIA    ? (L.dia_bulk ? MDS_FORMAT_STENCIL_BULK : MDS_FORMAT_STENCIL)
                  : L.fmt == FMT_SELL ? MDS_FORMAT_SELL
                                      : MDS_FORMAT_CSR;
    return MDS_OK;
}

}  // extern "C"

namespace mds {

// V-cycle on FP64 input/output regardless of the hierarchy's precision.
static void vcycle_f64(Ctx &c, Hierarchy &h, const double *b, double *x, int nr) {
    if (h.prec == 64) {
        vcycle_apply(c, h, b, x, nr);
        return;
    }
    int64_t n = h.lv[0].A.nrow * nr;
    const LiveMap lm = level_live(c, h.lv[0]);
    cast_f64_f32(c, b, h.lv[0].b.as<float>(), n, lm, nr);
    vcycle_apply(c, h, h.lv[0].b.p, h.lv[0].x.p, nr);
    cast_f32_f64(c, h.lv[0].x.as<float>(), x, n, lm, nr);
}

// Algorithm 1 (block lower), and the block-diagonal / block-upper variants,
// on nr interleaved columns (entry (i, c) at i nr + c).
void precond_apply(mds_precond p, const double *r, double *z, int nr) {
    Ctx &c = *p->ctx;
    mds_system s = p->sys;
    int64_t nm = s->n_m, nf = s->n_f;
    Hierarchy &HS = p->h[0];
    Hierarchy &HF = p->h[1];
    hierarchy_reserve(c, HS, nr);
    if (p->has_f) hierarchy_reserve(c, HF, nr);
    if ((int64_t)p->tf_cap < (nm > nf ? nm : nf) * nr) {
        int64_t mx = (nm > nf ? nm : nf) * nr;
        p->tf64 = Buf(&c, sizeof(double) * (size_t)(mx > 0 ? mx : 1));
        p->tf_cap = mx;
    }
    const mds_csr &Afm = s->view[2], &Amf = s->view[1];
    int kind = p->o.kind;
    const double *rm = r, *rf = r + nm * nr;
    double *zm = z, *zf = z + nm * nr;
    if (kind == MDS_BLOCK_UPPER && p->has_f) {
        // z_f = Q_ff r_f; r_m <- r_m - A_mf z_f; z_m = Q_mm r_m
        vcycle_f64(c, HF, rf, zf, nr);
        spmv_sub_f64(c, Amf, rm, zf, p->tf64.as<double>(), nr, level_live(c, HS.lv[0]));
        vcycle_f64(c, HS, p->tf64.as<double>(), zm, nr);
        return;
    }
    if (kind == MDS_BLOCK_DIAG && p->has_f) {
        // B_D: the two V-cycles are independent.  Q_ff runs on the side
        // stream while Q_mm runs on the main stream (fork and join by events,
        // which a CUDA graph capture turns into parallel branches).
        c.ensure_side_stream();  // created by mds_setup for this kind
        MDS_CUDA(cudaEventRecord(c.ev_fork, c.stream));
        MDS_CUDA(cudaStreamWaitEvent(c.side_stream, c.ev_fork, 0));
        cudaStream_t main = c.stream;
        c.stream = c.side_stream;
        try {
            vcycle_f64(c, HF, rf, zf, nr);
            if (p->ff_negative) scale_f64(c, zf, -1.0, nf * nr);
            MDS_CUDA(cudaEventRecord(c.ev_join, c.stream));
        } catch (...) {
            c.stream = main;
            throw;
        }
        c.stream = main;
        vcycle_f64(c, HS, rm, zm, nr);
        MDS_CUDA(cudaStreamWaitEvent(c.stream, c.ev_join, 0));
        return;
    }
    // step 1: z_m = Q_mm r_m  (in a batched solve only the live instances' rows)
    const LiveMap lmm = level_live(c, HS.lv[0]);
    if (HS.prec == 64) {
        vcycle_apply(c, HS, rm, zm, nr);
    } else {
        // the input in FP32: already written by the batched FGMRES's scaling
        // kernel when it stages into this buffer, else converted here
        if (c.in_stage != HS.lv[0].b.as<float>()) cast_f64_f32(c, rm, HS.lv[0].b.as<float>(), nm * nr, lmm, nr);
        // the top level's last kernel writes z_m in FP64 (else x, converted)
        if (!vcycle_apply_to64(c, HS, HS.lv[0].b.as<float>(), HS.lv[0].x.as<float>(), zm, nr))
            cast_f32_f64(c, HS.lv[0].x.as<float>(), zm, nm * nr, lmm, nr);
    }
    if (!p->has_f) return;
    // step 2: r_f <- r_f - A_fm z_m (block lower only); step 3: z_f = Q_ff r_f
    const LiveMap lmf = level_live(c, HF.lv[0]);
    if (HF.prec == 64) {
        if (kind == MDS_BLOCK_LOWER) {
            spmv_sub_f64(c, Afm, rf, zm, p->tf64.as<double>(), nr, lmf);
            vcycle_apply(c, HF, p->tf64.as<double>(), zf, nr);
        } else {
            vcycle_apply(c, HF, rf, zf, nr);
        }
        if (kind == MDS_BLOCK_DIAG && p->ff_negative) scale_f64(c, zf, -1.0, nf * nr);
    } else {
        float *bf = HF.lv[0].b.as<float>();
        // r_f - A_fm z_m with z_m read in FP64: the same values as the
        // V-cycle's FP32 x (exactly widened), so the same products
        if (kind == MDS_BLOCK_LOWER)
            spmv_sub_f64_to_f32(c, Afm, rf, zm, bf, nr, lmf);
        else
            cast_f64_f32(c, rf, bf, nf * nr, lmf, nr);
        if (!vcycle_apply_to64(c, HF, bf, HF.lv[0].x.as<float>(), zf, nr))
            cast_f32_f64(c, HF.lv[0].x.as<float>(), zf, nf * nr, lmf, nr);
        if (kind == MDS_BLOCK_DIAG && p->ff_negative) scale_f64(c, zf, -1.0, nf * nr);
    }
}

// The device address of page-locked host memory mapped into the device's
// address space (NULL for any other pointer).
template <class T> static T *mapped_host_ptr(T *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost && a.devicePointer ? static_cast<T *>(a.devicePointer) : nullptr;
}

static bool is_device_ptr(const void *p) {
    if (!p) return true;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace mds

extern "C" {

int mds_precond_apply(mds_ctx ctx, mds_precond p, const double *r, double *z) {
    if (!ctx || !p || !r || !z) return MDS_ERR_INVALID;
    Ctx *c = &ctx->c;
    async_join(c);
    API_BEGIN
    precond_apply(p, r, z, 1);
    API_END(c)
}

int mds_vcycle(mds_ctx ctx, mds_precond p, int block, const double *b, double *x) {
    if (!ctx || !p || !b || !x || block < 0 || block > 1 || (block == 1 && !p->has_f)) return MDS_ERR_INVALID;
    Ctx *c = &ctx->c;
    async_join(c);
    API_BEGIN
    vcycle_f64(*c, p->h[block], b, x, 1);
    API_END(c)
}

int mds_spmv(mds_ctx ctx, mds_system sys, const double *x, double *y) {
    if (!ctx || !sys || !x || !y) return MDS_ERR_INVALID;
    Ctx *c = &ctx->c;
    async_join(c);
    API_BEGIN
    spmv_f64(*c, sys->view[4], x, y, KC_SPMV);
    API_END(c)
}

int mds_solve_opts_default(mds_solve_opts *o) {
    if (!o) return MDS_ERR_INVALID;
    o->krylov = MDS_KRYLOV_FGMRES;
    o->restart = 30;
    o->rtol = 1e-8;
    o->max_iters = 1000;
    o->use_precond = 1;
    o->graphs = 1;
    o->batched = 1;
    o->reorth_eta2 = 1e-8;
    o->x0_zero = 0;
    return MDS_OK;
}

}  // extern "C"

static int solve_impl(mds_ctx ctx, mds_system sys, mds_precond prec, const double *b, double *x, int nrhs,
                      const mds_solve_opts *opts, mds_rhs_stats *stats) {
    Ctx *c = &ctx->c;
    int worst = MDS_OK;
    API_BEGIN
    MDS_CUDA(cudaSetDevice(c->device));
    mds_solve_opts o;
    mds_solve_opts_default(&o);
    if (opts) o = *opts;
    MDS_REQUIRE(o.rtol > 0.0 && o.max_iters >= 0 && o.restart >= 1 && o.reorth_eta2 >= 0.0, MDS_ERR_INVALID,
                "bad solve options");
    MDS_REQUIRE(o.krylov == MDS_KRYLOV_FGMRES || o.krylov == MDS_KRYLOV_PCG || o.krylov == MDS_KRYLOV_MINRES,
                MDS_ERR_INVALID, "unknown Krylov method");
    MDS_REQUIRE(!o.use_precond || (prec && prec->sys == sys), MDS_ERR_INVALID, "preconditioner of another system");
    MDS_REQUIRE(b || nrhs <= sys->nrhs, MDS_ERR_INVALID, "more right-hand sides than assembled");
    int64_t n = sys->n_m + sys->n_f;
    const double *B = b ? b : sys->b;
    bool bdev = is_device_ptr(B), xdev = is_device_ptr(x);
    Buf bst, xst;
    const double *Bd = B;
    double *Xd = x;
    size_t bytes = sizeof(double) * (size_t)n * (size_t)nrhs;
    bool batched = sys->n_inst > 1 || (nrhs > 1 && o.batched);
    // A batched FGMRES reads x once (its initial guess, not at all when
    // x0_zero) and writes it once at the end: page-locked host memory that
    // the device can address is then read and written in place by those two
    // kernels instead of through a device copy.
    if (!xdev && batched && o.krylov == MDS_KRYLOV_FGMRES) {
        if (double *mapped = mapped_host_ptr(x)) {
            Xd = mapped;
            xdev = true;
        }
    }
    if (!bdev) {
        bst = Buf(c, bytes);
        MDS_CUDA(cudaMemcpyAsync(bst.p, B, bytes, cudaMemcpyHostToDevice, c->stream));
        Bd = bst.as<double>();
    }
    if (!xdev) {
        xst = Buf(c, bytes);
        if (!o.x0_zero) MDS_CUDA(cudaMemcpyAsync(xst.p, x, bytes, cudaMemcpyHostToDevice, c->stream));
        Xd = xst.as<double>();
    }
    if (o.x0_zero && !batched) MDS_CUDA(cudaMemsetAsync(Xd, 0, bytes, c->stream));
    if (batched) {
        MDS_REQUIRE(o.krylov == MDS_KRYLOV_FGMRES, MDS_ERR_INVALID, "batched solves run FGMRES");
        BatchPrecFn BM;
        if (o.use_precond)
            BM = [prec](const double *r, double *z, int nr) { precond_apply(prec, r, z, nr); };
        else
            BM = [c, n](const double *r, double *z, int nr) {
                MDS_CUDA(cudaMemcpyAsync(z, r, sizeof(double) * (size_t)n * nr, cudaMemcpyDeviceToDevice, c->stream));
            };
        std::vector<int64_t> moff = sys->own.moff, foff = sys->own.foff;
        if (moff.size() < 2) {
            moff = {0, sys->n_m};
            foff = {0, sys->n_f};
        }
        std::vector<KrylovResult> res;
        // the mixed M_L's S~ V-cycle input is staged in FP32 by the scaling
        // kernel that writes each basis vector (its work vectors sized for
        // the widest column group first, so the buffer stays in place)
        struct StageScope {
            Ctx &c;
            ~StageScope() {
                c.in_stage = nullptr;
                c.in_stage_rows = 0;
            }
        } stage_scope{*c};
        if (o.use_precond && prec && prec->o.kind == MDS_BLOCK_LOWER && prec->h[0].prec == 32 && sys->n_m > 0) {
            const int nr0 = nrhs >= 8 ? 8 : nrhs >= 4 ? 4 : nrhs >= 2 ? 2 : 1;
            hierarchy_reserve(*c, prec->h[0], nr0);
            c->in_stage = prec->h[0].lv[0].b.as<float>();
            c->in_stage_rows = sys->n_m;
        }
        fgmres_batched(*c, sys->view[4], BM, moff, foff, Bd, Xd, nrhs, o, res);
        for (size_t q = 0; q < res.size(); q++) {
            const KrylovResult &r = res[q];
            if (stats) {
                stats[q].iterations = r.iterations;
                stats[q].restarts = r.restarts;
                stats[q].status = r.status;
                stats[q].relres_est = r.relres_est;
                stats[q].relres_true = r.relres_true;
            }
            if (r.status < 0) {
                if (worst >= 0) worst = r.status;
            } else if (r.status > worst && worst >= 0) {
                worst = r.status;
            }
        }
    }
    PrecFn M;
    if (o.use_precond) {
        M = [prec](const double *r, double *z) { precond_apply(prec, r, z, 1); };
    } else {
        M = [c, n](const double *r, double *z) {
            MDS_CUDA(cudaMemcpyAsync(z, r, sizeof(double) * (size_t)n, cudaMemcpyDeviceToDevice, c->stream));
        };
    }
    for (int k = 0; k < (batched ? 0 : nrhs); k++) {
        const double *bk = Bd + (size_t)k * n;
        double *xk = Xd + (size_t)k * n;
        KrylovResult r = o.krylov == MDS_KRYLOV_PCG      ? pcg(*c, sys->view[4], M, bk, xk, n, o)
                         : o.krylov == MDS_KRYLOV_MINRES ? minres(*c, sys->view[4], M, bk, xk, n, o)
                                                         : fgmres(*c, sys->view[4], M, bk, xk, n, o);
        if (stats) {
            stats[k].iterations = r.iterations;
            stats[k].restarts = r.restarts;
            stats[k].status = r.status;
            stats[k].relres_est = r.relres_est;
            stats[k].relres_true = r.relres_true;
        }
        if (r.status < 0) {
            if (worst >= 0) worst = r.status;
        } else if (r.status > worst && worst >= 0) {
            worst = r.status;
        }
    }
    if (!xdev) MDS_CUDA(cudaMemcpyAsync(x, Xd, bytes, cudaMemcpyDeviceToHost, c->stream));
    c->sync();
    if (worst < 0) c->last_error = "a right-hand side failed; see its stats";
    return worst;
    API_END(c)
}

extern "C" {

int mds_solve(mds_ctx ctx, mds_system sys, mds_precond prec, const double *b, double *x, int nrhs,
              const mds_solve_opts *opts, mds_rhs_stats *stats) {
    if (!ctx || !sys || !x || nrhs < 1) return MDS_ERR_INVALID;
    async_join(&ctx->c);
    return solve_impl(ctx, sys, prec, b, x, nrhs, opts, stats);
}

int mds_solve_async(mds_ctx ctx, mds_system sys, mds_precond prec, const double *b, double *x, int nrhs,
                    const mds_solve_opts *opts) {
    if (!ctx || !sys || !x || nrhs < 1) return MDS_ERR_INVALID;
    Ctx *c = &ctx->c;
    async_join(c);
    auto &A = c->async;
    if (A.pending) {
        c->last_error = "the previous asynchronous solve was not collected by mds_solve_wait";
        return MDS_ERR_INVALID;
    }
    mds_solve_opts o;
    mds_solve_opts_default(&o);
    if (opts) o = *opts;
    API_BEGIN
    A.stats.assign((size_t)nrhs * (size_t)sys->n_inst, mds_rhs_stats{});
    A.status = MDS_OK;
    A.done = std::make_shared<std::atomic<int>>(0);
    auto done = A.done;
    A.th = std::thread([ctx, sys, prec, b, x, nrhs, o, done] {
        Ctx *cc = &ctx->c;
        cudaSetDevice(cc->device);
        cc->async.status = solve_impl(ctx, sys, prec, b, x, nrhs, &o, cc->async.stats.data());
        done->store(1);
    });
    A.pending = true;
    API_END(c)
}

int mds_solve_done(mds_ctx ctx) {
    if (!ctx || !ctx->c.async.pending) return MDS_ERR_INVALID;
    return ctx->c.async.done->load();
}

int mds_solve_wait(mds_ctx ctx, mds_rhs_stats *stats, int count) {
    if (!ctx) return MDS_ERR_INVALID;
    Ctx *c = &ctx->c;
    async_join(c);
    auto &A = c->async;
    if (!A.pending) {
        c->last_error = "no asynchronous solve to wait for";
        return MDS_ERR_INVALID;
    }
    A.pending = false;
    if (stats)
        for (int q = 0; q < count && q < (int)A.stats.size(); q++) stats[q] = A.stats[q];
    return A.status;
}

int mds_tune(mds_ctx ctx, mds_system sys, const mds_setup_opts *base, const mds_solve_opts *sopts, const double *b,
             mds_tune_candidate *cands, int n_cands, int *best) {
    if (!ctx || !sys || !cands || n_cands < 1 || !best) return MDS_ERR_INVALID;
    Ctx *c = &ctx->c;
    async_join(c);
    *best = -1;
    mds_setup_opts o0;
    mds_setup_opts_default(&o0);
    if (base) o0 = *base;
    mds_solve_opts so;
    mds_solve_opts_default(&so);
    if (sopts) so = *sopts;
    so.use_precond = 1;
    const int64_t n = sys->n_m + sys->n_f;
    API_BEGIN
    MDS_CUDA(cudaSetDevice(c->device));
    Buf xb(c, sizeof(double) * (size_t)(n > 0 ? n : 1));  // trial solution (the context's allocator)
    double *x = xb.as<double>();
    using clk = std::chrono::steady_clock;
    double tbest = 0.0;
    for (int q = 0; q < n_cands; q++) {
        mds_tune_candidate &k = cands[q];
        mds_setup_opts o = o0;
        o.smoother = k.smoother;
        o.sweeps = k.sweeps;
        o.cheb_degree = k.cheb_degree;
        o.precision = k.precision;
        if (k.n_coarse > 0) o.n_coarse = k.n_coarse;
        k.iterations = 0;
        k.setup_ms = k.solve_ms = 0.0;
        mds_precond p = nullptr;
        cudaStreamSynchronize(c->stream);
        auto t0 = clk::now();
        k.status = mds_setup(ctx, sys, &o, &p);
        auto t1 = clk::now();
        k.setup_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
        if (k.status < 0) continue;
        mds_rhs_stats st{};
        cudaMemsetAsync(x, 0, sizeof(double) * (size_t)n, c->stream);
        cudaStreamSynchronize(c->stream);
        t0 = clk::now();
        int code = mds_solve(ctx, sys, p, b, x, 1, &so, &st);
        t1 = clk::now();
        k.solve_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
        k.status = code < 0 ? code : st.status;
        k.iterations = st.iterations;
        mds_precond_destroy(p);
        double t = k.setup_ms + k.solve_ms;
        if (k.status == MDS_OK && (*best < 0 || t < tbest)) {
            *best = q;
            tbest = t;
        }
    }
    if (*best < 0) {
        c->last_error = "mds_tune: no candidate converged";
        return MDS_WARN_NOT_CONVERGED;
    }
    API_END(c)
}

int mds_solve_noalloc(mds_ctx ctx, mds_system sys, mds_precond prec, const double *b, double *x,
                      const mds_solve_opts *opts, mds_rhs_stats *stats) {
    if (!ctx || !sys || !x) return MDS_ERR_INVALID;
    Ctx *c = &ctx->c;
    async_join(c);
    API_BEGIN
    MDS_CUDA(cudaSetDevice(c->device));
    mds_solve_opts o;
    mds_solve_opts_default(&o);
    if (opts) o = *opts;
    o.graphs = 0;  // graph instantiation may allocate
    int64_t n = sys->n_m + sys->n_f;
    MDS_REQUIRE(o.krylov == MDS_KRYLOV_FGMRES, MDS_ERR_INVALID, "mds_solve_noalloc runs FGMRES only");
    MDS_REQUIRE(sys->n_inst == 1, MDS_ERR_INVALID,
                "mds_solve_noalloc solves one instance; a packed batch needs mds_solve");
    MDS_REQUIRE(n <= MDS_NOALLOC_MAX_N, MDS_ERR_INVALID,
                "mds_solve_noalloc: n_m + n_f = " + std::to_string(n) + " exceeds MDS_NOALLOC_MAX_N = " +
                    std::to_string(MDS_NOALLOC_MAX_N));
    MDS_REQUIRE(o.restart >= 1 && o.restart <= 30, MDS_ERR_INVALID, "mds_solve_noalloc: restart must be 1..30");
    MDS_REQUIRE(o.rtol > 0.0 && o.max_iters >= 0, MDS_ERR_INVALID, "bad solve options");
    MDS_REQUIRE(!o.use_precond || (prec && prec->sys == sys), MDS_ERR_INVALID, "preconditioner of another system");
    const double *B = b ? b : sys->b;
    MDS_REQUIRE(is_device_ptr(B) && is_device_ptr(x), MDS_ERR_INVALID,
                "mds_solve_noalloc needs device pointers for b and x");
    if (o.x0_zero) MDS_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * (size_t)n, c->stream));
    size_t need = fgmres_workspace_doubles(n, o.restart);
    MDS_REQUIRE(need <= noalloc_scratch_doubles(), MDS_ERR_INVALID, "mds_solve_noalloc: workspace exceeds the array");
    FgmresWorkspace ws = fgmres_workspace_carve(noalloc_scratch(*c), n, o.restart);
    PrecFn M;
    if (o.use_precond)
        M = [prec](const double *r, double *z) { precond_apply(prec, r, z, 1); };
    else
        M = [c, n](const double *r, double *z) {
            MDS_CUDA(cudaMemcpyAsync(z, r, sizeof(double) * (size_t)n, cudaMemcpyDeviceToDevice, c->stream));
        };
    KrylovResult r = fgmres(*c, sys->view[4], M, B, x, n, o, &ws);
    c->sync();
    if (stats) {
        stats->iterations = r.iterations;
        stats->restarts = r.restarts;
        stats->status = r.status;
        stats->relres_est = r.relres_est;
        stats->relres_true = r.relres_true;
    }
    if (r.status < 0) c->last_error = "solve failed; see its stats";
    return r.status;
    API_END(c)
}

int mds_timing_enable(mds_ctx ctx, int k, int enable) {
    if (!ctx || k < 0 || k >= MDS_KCLASS_COUNT) return MDS_ERR_INVALID;
    async_join(&ctx->c);
    ctx->c.timing[k] = enable != 0;
    return MDS_OK;
}

int mds_timing_reset(mds_ctx ctx) {
    if (!ctx) return MDS_ERR_INVALID;
    Ctx &c = ctx->c;
    async_join(&c);
    cudaStreamSynchronize(c.stream);
    for (int k = 0; k < MDS_KCLASS_COUNT; k++) {
        c.ev_used[k] = 0;
        c.launches[k] = 0;
        c.bytes[k] = 0.0;
        c.flops[k] = 0.0;
        c.graph_ms[k] = 0.0;
        c.tlaunches[k] = 0;
        c.tbytes[k] = 0.0;
        c.tflops[k] = 0.0;
    }
    c.total_launches = 0;
    return MDS_OK;
}

int mds_timing_sample_every(mds_ctx ctx, int every) {
    if (!ctx || every < 1) return MDS_ERR_INVALID;
    async_join(&ctx->c);
    ctx->c.sample_every = every;
    return MDS_OK;
}

static double event_ms(Ctx *c, int k) {
    double tot = 0.0;
    for (size_t q = 0; q < c->ev_used[k]; q++) {
        float t = 0.f;
        MDS_CUDA(cudaEventElapsedTime(&t, c->evs[k][q].e0, c->evs[k][q].e1));
        tot += t;
    }
    return tot + c->graph_ms[k];
}

int mds_timing_sampled(mds_ctx ctx, int k, int64_t *launches, double *ms, double *bytes, double *flops) {
    if (!ctx || k < 0 || k >= MDS_KCLASS_COUNT) return MDS_ERR_INVALID;
    Ctx *c = &ctx->c;
    async_join(c);
    API_BEGIN
    c->sync();
    if (launches) *launches = c->tlaunches[k];
    if (ms) *ms = event_ms(c, k);
    if (bytes) *bytes = c->tbytes[k];
    if (flops) *flops = c->tflops[k];
    API_END(c)
}

int mds_timing_query(mds_ctx ctx, int k, int64_t *launches, double *ms, double *bytes, double *flops) {
    if (!ctx || k < 0 || k >= MDS_KCLASS_COUNT) return MDS_ERR_INVALID;
    Ctx *c = &ctx->c;
    async_join(c);
    API_BEGIN
    c->sync();
    if (launches) *launches = c->launches[k];
    if (ms) *ms = event_ms(c, k);
    if (bytes) *bytes = c->bytes[k];
    if (flops) *flops = c->flops[k];
    API_END(c)
}

int mds_memcpy(mds_ctx ctx, void *dst, const void *src, size_t bytes) {
    if (!ctx || (!dst && bytes) || (!src && bytes)) return MDS_ERR_INVALID;
    Ctx *c = &ctx->c;
    async_join(c);
    API_BEGIN
    if (bytes) MDS_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, c->stream));
    c->sync();
    API_END(c)
}

int mds_launch_count(mds_ctx ctx, int64_t *launches) {
    if (!ctx || !launches) return MDS_ERR_INVALID;
    async_join(&ctx->c);
    *launches = ctx->c.total_launches;
    return MDS_OK;
}

}  // extern "C"
