// Instantiations of the persistent batched kernel for embedding dimension d = 1.
#include "te_kernels.cuh"

namespace te {
TE_BATCHED_PTR_FN(batched_ptr_d1, 1, 1)
}  // namespace te
