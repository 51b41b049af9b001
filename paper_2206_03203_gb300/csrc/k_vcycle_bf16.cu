// V-cycle level operations on FP32 vectors with BF16 stored values
// (row-scaled coarse levels), instantiated in their own translation unit.
#define MDS_VCYCLE_LP_UNIT
#include "vcycle.cuh"

namespace mds {

MDS_LP_EACH(MDS_LP_INST, __nv_bfloat16)

}  // namespace mds
