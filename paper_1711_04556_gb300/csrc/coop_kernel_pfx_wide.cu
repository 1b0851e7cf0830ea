// Co-operative search kernels with prefix reuse for G = 8, 16, 32 lanes per decode.
#include "coop_kernel.cuh"

namespace rcpsp {

RCPSP_COOP_ENTRY_POINTS(pfx_wide, true, 8, 16, 32)

}  // namespace rcpsp
