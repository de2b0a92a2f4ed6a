// Instantiations of the persistent batched kernel (and the warp-mode sweep kernel) for d = 1.
#include "te_kernels.cuh"

namespace te {
TE_BATCHED_PTR_FN(batched_ptr_d1, 1, 1)
TE_SWEEP_WARP_PTR_FN(sweep_warp_ptr_d1, 1)
}  // namespace te
