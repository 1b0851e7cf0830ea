// Co-operative search kernels for G = 8, 16, 32 lanes per decode.
#include "coop_kernel.cuh"

namespace rcpsp {

RCPSP_COOP_ENTRY_POINTS(wide, false, 8, 16, 32)

}  // namespace rcpsp
