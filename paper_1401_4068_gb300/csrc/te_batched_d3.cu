// Instantiations of the persistent batched kernel for embedding dimension d = 3.
#include "te_kernels.cuh"

namespace te {
TE_BATCHED_PTR_FN(batched_ptr_d3, 3, 3)
}  // namespace te
