// Instantiations of the bundle kernel (te_bundle.cuh): one per embedding dimension and kind
// (resident / tiled bundles), k <= 4.
#include "te_bundle.cuh"

namespace te {

const void* bundle_kernel_ptr(int d, int ks, bool tiled) {
    if (ks != 5) return nullptr;
#define TE_BUNDLE_CASE(DD)                                                                        \
    case DD:                                                                                      \
        return tiled ? (const void*)bundle_kernel<DD, kBundleQ, 5, kBundleMax, true>              \
                     : (const void*)bundle_kernel<DD, kBundleQ, 5, kBundleMax, false>;
    switch (d) {
        TE_BUNDLE_CASE(1)
        TE_BUNDLE_CASE(2)
        TE_BUNDLE_CASE(3)
        TE_BUNDLE_CASE(4)
        TE_BUNDLE_CASE(5)
        default: return nullptr;
    }
#undef TE_BUNDLE_CASE
}

cudaError_t launch_bundle(int d, int ks, bool tiled, const BatchArgs& a, int grid, size_t smem, cudaStream_t s) {
    const void* fn = bundle_kernel_ptr(d, ks, tiled);
    if (!fn) return cudaErrorInvalidDeviceFunction;
    void* args[] = {const_cast<BatchArgs*>(&a)};
    return cudaLaunchKernel(fn, dim3(grid), dim3(kBundleThreads), args, smem, s);
}

}  // namespace te
