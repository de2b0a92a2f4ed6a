// Instantiations of the persistent batched kernel for embedding dimension d = 2.
#include "te_kernels.cuh"

namespace te {
TE_BATCHED_PTR_FN(batched_ptr_d2, 2, 2)
}  // namespace te
