// V-cycle kernels and level operations instantiated for float vectors (one
// translation unit per vector type, compiled in parallel).
#include "vcycle.cuh"

namespace mds {

void vcycle_run_f32(Ctx &c, Hierarchy &h, const float *b, float *x, int nr) { vcycle_nr<float>(c, h, b, x, nr); }

bool vcycle_run_f32_to64(Ctx &c, Hierarchy &h, const float *b, float *x, double *z64, int nr) {
    return vcycle_nr<float>(c, h, b, x, nr, z64);
}

float time_level_f32(Ctx &c, const Level &L, int nr, const void *xc, bool stored) {
    return time_level<float>(c, L, nr, xc, stored);
}

}  // namespace mds
