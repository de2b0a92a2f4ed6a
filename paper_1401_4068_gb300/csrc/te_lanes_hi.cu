// Instantiations of the lane kernel (te_lanes.cuh) for d = 5 .. 8, k <= 4.
#include "te_lanes.cuh"

namespace te {

const void* lane_ptr_hi(int d, int ks) {
    if (ks != 5) return nullptr;
    switch (d) {
        case 5: return (const void*)lane_kernel<5, 5>;
        case 6: return (const void*)lane_kernel<6, 5>;
        case 7: return (const void*)lane_kernel<7, 5>;
        case 8: return (const void*)lane_kernel<8, 5>;
        default: return nullptr;
    }
}

}  // namespace te
