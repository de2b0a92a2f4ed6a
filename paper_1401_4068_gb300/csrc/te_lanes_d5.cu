// Instantiations of the lane kernel (te_lanes.cuh) for d = 5, k <= 4, every delay class.
#include "te_lanes.cuh"

namespace te {

const void* lane_ptr_d5(int ks, int tc) { return lane_kernel_select<5>(ks, tc); }

}  // namespace te
