// Instantiations of the persistent batched kernel for embedding dimension d = 5.
#include "te_kernels.cuh"

namespace te {
TE_BATCHED_PTR_FN(batched_ptr_d5, 5, 5)
}  // namespace te
