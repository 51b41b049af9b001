// Krylov solver interfaces (internal).
#pragma once
#include <functional>

#include "internal.cuh"

namespace mds {

using PrecFn = std::function<void(const double *r, double *z)>;

struct KrylovResult {
    int iterations = 0;
    int restarts = 0;
    int status = MDS_OK;
    double relres_est = 0.0;
    double relres_true = 0.0;
};

KrylovResult fgmres(Ctx &c, const mds_csr &A, const PrecFn &M, const double *b, double *x, int64_t n,
                    const mds_solve_opts &o);
KrylovResult pcg(Ctx &c, const mds_csr &A, const PrecFn &M, const double *b, double *x, int64_t n,
                 const mds_solve_opts &o);

}  // namespace mds
