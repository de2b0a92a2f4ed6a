// Instantiations of the persistent batched kernel for mixed embedding dimensions d = 1..5.
#include "te_kernels.cuh"

namespace te {
TE_BATCHED_PTR_FN(batched_ptr_mix, 1, 5)
}  // namespace te
