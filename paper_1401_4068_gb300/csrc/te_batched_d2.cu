// Instantiations of the persistent batched kernel (and the warp-mode sweep kernel) for d = 2.
#include "te_kernels.cuh"

namespace te {
TE_BATCHED_PTR_FN(batched_ptr_d2, 2, 2)
TE_SWEEP_WARP_PTR_FN(sweep_warp_ptr_d2, 2)
}  // namespace te
