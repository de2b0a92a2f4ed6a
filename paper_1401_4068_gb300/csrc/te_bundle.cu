// Instantiations of the bundle kernel (te_bundle.cuh): one per embedding dimension, k <= 4.
#include "te_bundle.cuh"

namespace te {

const void* bundle_kernel_ptr(int d, int ks) {
    if (ks != 5) return nullptr;
    switch (d) {
        case 1: return (const void*)bundle_kernel<1, kBundleQ, 5, kBundleMax>;
        case 2: return (const void*)bundle_kernel<2, kBundleQ, 5, kBundleMax>;
        case 3: return (const void*)bundle_kernel<3, kBundleQ, 5, kBundleMax>;
        case 4: return (const void*)bundle_kernel<4, kBundleQ, 5, kBundleMax>;
        case 5: return (const void*)bundle_kernel<5, kBundleQ, 5, kBundleMax>;
        default: return nullptr;
    }
}

cudaError_t launch_bundle(int d, int ks, const BatchArgs& a, int grid, size_t smem, cudaStream_t s) {
    const void* fn = bundle_kernel_ptr(d, ks);
    if (!fn) return cudaErrorInvalidDeviceFunction;
    void* args[] = {const_cast<BatchArgs*>(&a)};
    return cudaLaunchKernel(fn, dim3(grid), dim3(kBundleThreads), args, smem, s);
}

}  // namespace te
