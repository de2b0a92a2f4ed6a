// Sort pre-pass of the sweep mode: for every (series, window start, window) group, the points
// i = r * W + w sorted by their target coordinate y_r(t_start + w - 1) (coordinate 1 of the joint
// space, shared by the original and all surrogates of the group), ties by point index. One CTA per
// group runs a bitonic sort of (key, index) pairs in shared memory, padded to a power of two with
// (+inf, INT_MAX).
#include "te_internal.h"

namespace te {

namespace {

constexpr int kSortThreads = 1024;

__global__ void __launch_bounds__(kSortThreads) sort_groups_kernel(const SortGroup* __restrict__ groups,
                                                                   int32_t* __restrict__ out_idx,
                                                                   float* __restrict__ out_key) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const SortGroup G = groups[blockIdx.x];
    const int N = G.N;
    int P = 1;
    while (P < N) P <<= 1;
    float* k = reinterpret_cast<float*>(smraw);
    int32_t* ix = reinterpret_cast<int32_t*>(k + P);
    for (int p = threadIdx.x; p < P; p += blockDim.x) {
        if (p < N) {
            const int r = p / G.W;
            const int w = p - r * G.W;
            k[p] = __ldg(G.tgt + (size_t)r * G.T + G.t_start + w - 1);
            ix[p] = p;
        } else {
            k[p] = __int_as_float(0x7f800000);
            ix[p] = 0x7fffffff;
        }
    }
    __syncthreads();
    for (int size = 2; size <= P; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = threadIdx.x; t < (P >> 1); t += blockDim.x) {
                const int i = 2 * t - (t & (stride - 1));
                const int j = i + stride;
                const bool up = (i & size) == 0;
                const float ki = k[i], kj = k[j];
                const int ii = ix[i], ij = ix[j];
                const bool greater = ki > kj || (ki == kj && ii > ij);
                if (greater == up) {
                    k[i] = kj;
                    k[j] = ki;
                    ix[i] = ij;
                    ix[j] = ii;
                }
            }
            __syncthreads();
        }
    }
    for (int p = threadIdx.x; p < N; p += blockDim.x) {
        out_idx[G.off + p] = ix[p];
        out_key[G.off + p] = k[p];
    }
}

int pow2_at_least(int n) {
    int P = 1;
    while (P < n) P <<= 1;
    return P;
}

}  // namespace

cudaError_t prepare_sort_kernel(int nmax) {
    const int bytes = pow2_at_least(nmax) * 8;
    return cudaFuncSetAttribute(sort_groups_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

cudaError_t launch_sort_groups(const SortGroup* groups, int n_groups, int nmax, int32_t* idx, float* key,
                               cudaStream_t s) {
    const int bytes = pow2_at_least(nmax) * 8;
    sort_groups_kernel<<<n_groups, kSortThreads, bytes, s>>>(groups, idx, key);
    return cudaGetLastError();
}

}  // namespace te
