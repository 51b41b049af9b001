// V-cycle kernels and level operations instantiated for double vectors (one
// translation unit per vector type, compiled in parallel).
#include "vcycle.cuh"

namespace mds {

void vcycle_run_f64(Ctx &c, Hierarchy &h, const double *b, double *x, int nr) { vcycle_nr<double>(c, h, b, x, nr); }

float time_level_f64(Ctx &c, const Level &L, int nr, const void *xc, bool stored) {
    return time_level<double>(c, L, nr, xc, stored);
}

}  // namespace mds
