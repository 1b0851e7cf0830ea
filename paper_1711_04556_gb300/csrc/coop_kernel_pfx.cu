// Co-operative search kernels with prefix reuse for G = 1, 2, 4 lanes per decode.
#include "coop_kernel.cuh"

namespace rcpsp {

RCPSP_COOP_ENTRY_POINTS(pfx_narrow, true, 1, 2, 4)

}  // namespace rcpsp
