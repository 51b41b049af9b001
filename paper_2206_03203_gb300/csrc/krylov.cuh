// Krylov solver interfaces (internal).
#pragma once
#include <functional>
#include <vector>

#include "internal.cuh"

namespace mds {

using PrecFn = std::function<void(const double *r, double *z)>;
// z = M r on nr interleaved columns
using BatchPrecFn = std::function<void(const double *r, double *z, int nr)>;

struct KrylovResult {
    int iterations = 0;
    int restarts = 0;
    int status = MDS_OK;
    double relres_est = 0.0;
    double relres_true = 0.0;
};

// Caller-provided FGMRES workspace (device pointers, 256-byte aligned).
struct FgmresWorkspace {
    double *partial, *V, *Z, *H, *small;
};
// Doubles the workspace of an FGMRES(m) solve of size n occupies, with each
// part rounded up to 256 bytes, and its carving from one base pointer.
size_t fgmres_workspace_doubles(int64_t n, int m);
FgmresWorkspace fgmres_workspace_carve(double *base, int64_t n, int m);

// ws == nullptr: the workspace is allocated from the context.
KrylovResult fgmres(Ctx &c, const mds_csr &A, const PrecFn &M, const double *b, double *x, int64_t n,
                    const mds_solve_opts &o, const FgmresWorkspace *ws = nullptr);

// The library's static no-allocation workspace (see mds_solve_noalloc): its
// device address as resolved for the context at creation, the lookup itself
// (on the current device), and its size in doubles.
double *noalloc_scratch(Ctx &c);
double *noalloc_scratch_lookup();
size_t noalloc_scratch_doubles();
// K instances (row segments [moff_k, moff_k+1) and [NM + foff_k, NM +
// foff_k+1)) x nrhs columns (column-major [nrhs][N] in B and X) solved as
// independent FGMRES problems in lockstep; res[k * nrhs + c].
void fgmres_batched(Ctx &c, const mds_csr &A, const BatchPrecFn &M, const std::vector<int64_t> &moff,
                    const std::vector<int64_t> &foff, const double *B, double *X, int nrhs, const mds_solve_opts &o,
                    std::vector<KrylovResult> &res);
KrylovResult pcg(Ctx &c, const mds_csr &A, const PrecFn &M, const double *b, double *x, int64_t n,
                 const mds_solve_opts &o);
// preconditioned MINRES (symmetric A, SPD preconditioner)
KrylovResult minres(Ctx &c, const mds_csr &A, const PrecFn &M, const double *b, double *x, int64_t n,
                    const mds_solve_opts &o);

}  // namespace mds
