// Instantiations of the persistent batched kernel for embedding dimension d = 8.
#include "te_kernels.cuh"

namespace te {
TE_BATCHED_PTR_FN_WIDE(batched_ptr_d8, 8)
}  // namespace te
