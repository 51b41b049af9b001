// V-cycle level operations on FP32 vectors with F16 stored values
// (row-scaled coarse levels), instantiated in their own translation unit.
#define MDS_VCYCLE_LP_UNIT
#include "vcycle.cuh"

namespace mds {

MDS_LP_EACH(MDS_LP_INST, __half)

}  // namespace mds
