// Instantiations of the persistent batched kernel for embedding dimension d = 4.
#include "te_kernels.cuh"

namespace te {
TE_BATCHED_PTR_FN(batched_ptr_d4, 4, 4)
}  // namespace te
