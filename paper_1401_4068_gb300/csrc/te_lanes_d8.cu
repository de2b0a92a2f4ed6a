// Instantiations of the lane kernel (te_lanes.cuh) for d = 8, k <= 4, every delay class.
#include "te_lanes.cuh"

namespace te {

const void* lane_ptr_d8(int ks, int tc) { return lane_kernel_select<8>(ks, tc); }

}  // namespace te
