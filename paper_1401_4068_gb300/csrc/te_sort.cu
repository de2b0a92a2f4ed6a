// Sort pre-pass of the sweep mode: for every (series, window start, window) group, the points
// i = r * W + w sorted by their target coordinate y_r(t_start + w - 1) (coordinate 1 of the joint
// space, shared by the original and all surrogates of the group), ties by point index, so the order
// is unique. One CTA per group:
//   N <= kSortRun: a bitonic sort of (key, index) pairs in shared memory, padded to a power of two
//                  with (+inf, INT_MAX);
//   larger N:      runs of kSortRun points sorted that way, then merge passes that double the run
//                  length, each thread merging its share of the output after a merge-path search
//                  for its starting split (ping-pong between the output and a scratch buffer, the
//                  first run buffer chosen so that the last pass writes the output).
#include "te_internal.h"

namespace te {

namespace {

constexpr int kSortThreads = 1024;
constexpr int kSortRun = 8192;  // points per shared-memory run (64 KB of (key, index) pairs)

__device__ __forceinline__ float group_key(const SortGroup& G, int p) {
    const int r = p / G.W;
    const int w = p - r * G.W;
    return __ldg(G.tgt + (size_t)r * G.T + G.t_start + w - 1);
}

// (key, index) order
__device__ __forceinline__ bool before(float ka, int ia, float kb, int ib) {
    return ka < kb || (ka == kb && ia < ib);
}

// points base .. base + n - 1 of the group into shared memory (padded to P), bitonic sort
__device__ void sort_run(const SortGroup& G, int base, int n, int P, float* k, int32_t* ix) {
    for (int p = threadIdx.x; p < P; p += blockDim.x) {
        if (p < n) {
            k[p] = group_key(G, base + p);
            ix[p] = base + p;
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
                const bool greater = before(kj, ij, ki, ii);
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
}

// merge sorted A (la) and B (lb) into out; every thread produces a contiguous share of the output
__device__ void merge_pair(const float* ak, const int32_t* ai, int la, const float* bk, const int32_t* bi, int lb,
                           float* ok, int32_t* oi) {
    const int total = la + lb;
    const int per = (total + blockDim.x - 1) / blockDim.x;
    const int o0 = threadIdx.x * per;
    if (o0 >= total) return;
    const int o1 = min(total, o0 + per);
    // first split i (elements of A among the first o0 outputs): A[i] is not before B[o0 - i - 1]
    int lo = max(0, o0 - lb), hi = min(o0, la);
    while (lo < hi) {
        const int i = (lo + hi) >> 1;
        const int j = o0 - i;
        if (j > 0 && i < la && before(ak[i], ai[i], bk[j - 1], bi[j - 1])) lo = i + 1;
        else hi = i;
    }
    int i = lo, j = o0 - lo;
    for (int o = o0; o < o1; ++o) {
        const bool take_a = j >= lb || (i < la && before(ak[i], ai[i], bk[j], bi[j]));
        if (take_a) {
            ok[o] = ak[i];
            oi[o] = ai[i];
            ++i;
        } else {
            ok[o] = bk[j];
            oi[o] = bi[j];
            ++j;
        }
    }
}

__global__ void __launch_bounds__(kSortThreads) sort_groups_kernel(const SortGroup* __restrict__ groups,
                                                                   int32_t* __restrict__ out_idx,
                                                                   float* __restrict__ out_key,
                                                                   int32_t* __restrict__ tmp_idx,
                                                                   float* __restrict__ tmp_key) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const SortGroup G = groups[blockIdx.x];
    const int N = G.N;
    float* k = reinterpret_cast<float*>(smraw);
    int32_t* ix = reinterpret_cast<int32_t*>(k + kSortRun);
    if (N <= kSortRun) {
        int P = 1;
        while (P < N) P <<= 1;
        sort_run(G, 0, N, P, k, ix);
        for (int p = threadIdx.x; p < N; p += blockDim.x) {
            out_idx[G.off + p] = ix[p];
            out_key[G.off + p] = k[p];
        }
        return;
    }
    int passes = 0;
    for (int L = kSortRun; L < N; L <<= 1) ++passes;
    float* sk = ((passes & 1) ? tmp_key : out_key) + G.off;
    int32_t* si = ((passes & 1) ? tmp_idx : out_idx) + G.off;
    float* dk = ((passes & 1) ? out_key : tmp_key) + G.off;
    int32_t* di = ((passes & 1) ? out_idx : tmp_idx) + G.off;
    for (int base = 0; base < N; base += kSortRun) {
        const int n = min(kSortRun, N - base);
        sort_run(G, base, n, kSortRun, k, ix);
        for (int p = threadIdx.x; p < n; p += blockDim.x) {
            sk[base + p] = k[p];
            si[base + p] = ix[p];
        }
        __syncthreads();  // shared memory is reused by the next run
    }
    for (int L = kSortRun; L < N; L <<= 1) {
        for (int b = 0; b < N; b += 2 * L) {
            const int la = min(L, N - b);
            const int lb = max(0, min(L, N - b - L));
            merge_pair(sk + b, si + b, la, sk + b + la, si + b + la, lb, dk + b, di + b);
        }
        __syncthreads();  // this pass's output is the next pass's input
        float* tk = sk;
        sk = dk;
        dk = tk;
        int32_t* ti = si;
        si = di;
        di = ti;
    }
}

}  // namespace

bool sort_needs_scratch(int nmax) { return nmax > kSortRun; }

cudaError_t prepare_sort_kernel(int /*nmax*/) {
    return cudaFuncSetAttribute(sort_groups_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSortRun * 8);
}

cudaError_t launch_sort_groups(const SortGroup* groups, int n_groups, int /*nmax*/, int32_t* idx, float* key,
                               int32_t* tmp_idx, float* tmp_key, cudaStream_t s) {
    sort_groups_kernel<<<n_groups, kSortThreads, kSortRun * 8, s>>>(groups, idx, key, tmp_idx, tmp_key);
    return cudaGetLastError();
}

}  // namespace te
