// Sort pre-pass of the sweep mode: for every (series, window start, window) group, the points
// i = r * W + w ordered by their target coordinates, which the original and all surrogates of the
// group share. One CTA per group sorts (64-bit key, point index) pairs, ties by index, so the
// order is unique: runs of kSortRun pairs bitonic-sorted in shared memory, then merge passes that
// double the run length through global memory (each thread merges its share of the output after a
// merge-path search for its starting split).
//   S == 1: key = y_{t'-1} (coordinate 1 of the joint space).
//   S > 1 (strips): first sorted by the second key y_{t'-k2lag} and cut into strips of G.L
//           consecutive ranks (the last one shorter), then sorted by (strip, y_{t'-1}); strip s is
//           written at positions s * G.L .. (the last strip padded to a multiple of four with
//           (index -1, key +inf)), and the lowest and highest second key of its points are
//           recorded.
// Keys are FP32 values mapped to unsigned integers that order like the floats.
#include "te_internal.h"

namespace te {

namespace {

typedef unsigned long long u64k;

constexpr int kSortThreads = 1024;
constexpr int kSortRun = 4096;  // pairs per shared-memory run (48 KB)

__device__ __forceinline__ unsigned ord_bits(float f) {
    const unsigned b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float from_ord(unsigned o) {
    return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
}

// target value y_{t' - lag} of point p of the group (lag 1: y_{t'-1}, 0: y_t)
__device__ __forceinline__ float group_coord(const SortGroup& G, int p, int lag) {
    const int r = p / G.W;
    const int w = p - r * G.W;
    return __ldg(G.tgt + (size_t)r * G.T + G.t_start + w - lag);
}

__device__ __forceinline__ bool before(u64k ka, int ia, u64k kb, int ib) {
    return ka < kb || (ka == kb && ia < ib);
}

__device__ void bitonic(u64k* k, int32_t* ix, int P) {
    __syncthreads();
    for (int size = 2; size <= P; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = threadIdx.x; t < (P >> 1); t += blockDim.x) {
                const int i = 2 * t - (t & (stride - 1));
                const int j = i + stride;
                const bool up = (i & size) == 0;
                const u64k ki = k[i], kj = k[j];
                const int ii = ix[i], ij = ix[j];
                if (before(kj, ij, ki, ii) == up) {
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
__device__ void merge_pair(const u64k* ak, const int32_t* ai, int la, const u64k* bk, const int32_t* bi, int lb,
                           u64k* ok, int32_t* oi) {
    const int total = la + lb;
    const int per = (total + blockDim.x - 1) / blockDim.x;
    const int o0 = threadIdx.x * per;
    if (o0 >= total) return;
    const int o1 = min(total, o0 + per);
    int lo = max(0, o0 - lb), hi = min(o0, la);
    while (lo < hi) {  // first split i: A[i] is not before B[o0 - i - 1]
        const int i = (lo + hi) >> 1;
        const int j = o0 - i;
        if (j > 0 && i < la && before(ak[i], ai[i], bk[j - 1], bi[j - 1])) lo = i + 1;
        else hi = i;
    }
    int i = lo, j = o0 - lo;
    for (int o = o0; o < o1; ++o) {
        if (j >= lb || (i < la && before(ak[i], ai[i], bk[j], bi[j]))) {
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

// Sort the n pairs load(p) = (key, index), p = 0 .. n-1, into (ak, ai); (bk, bi) is scratch.
// load may read (ak, ai) itself: every run is read whole before it is written back in place.
template <class Load>
__device__ void sort_pairs(int n, Load load, u64k* ak, int32_t* ai, u64k* bk, int32_t* bi, u64k* sk, int32_t* si) {
    int passes = 0;
    for (int L = kSortRun; L < n; L <<= 1) ++passes;
    // runs go where the last merge pass (or none) leaves the result in (ak, ai)
    u64k* rk = (passes & 1) ? bk : ak;
    int32_t* ri = (passes & 1) ? bi : ai;
    for (int base = 0; base < n; base += kSortRun) {
        const int m = min(kSortRun, n - base);
        int P = 1;
        while (P < m) P <<= 1;
        __syncthreads();
        for (int p = threadIdx.x; p < P; p += blockDim.x) {
            if (p < m) {
                u64k k;
                int i;
                load(base + p, k, i);
                sk[p] = k;
                si[p] = i;
            } else {
                sk[p] = ~0ull;
                si[p] = 0x7fffffff;
            }
        }
        bitonic(sk, si, P);
        for (int p = threadIdx.x; p < m; p += blockDim.x) {
            rk[base + p] = sk[p];
            ri[base + p] = si[p];
        }
    }
    __syncthreads();
    u64k* srk = rk;
    int32_t* sri = ri;
    u64k* dk = (passes & 1) ? ak : bk;
    int32_t* di = (passes & 1) ? ai : bi;
    for (int L = kSortRun; L < n; L <<= 1) {
        for (int b = 0; b < n; b += 2 * L) {
            const int la = min(L, n - b);
            const int lb = max(0, min(L, n - b - L));
            merge_pair(srk + b, sri + b, la, srk + b + la, sri + b + la, lb, dk + b, di + b);
        }
        __syncthreads();
        u64k* tk = srk;
        srk = dk;
        dk = tk;
        int32_t* ti = sri;
        sri = di;
        di = ti;
    }
}

__global__ void __launch_bounds__(kSortThreads) sort_groups_kernel(const SortGroup* __restrict__ groups,
                                                                   int32_t* __restrict__ out_idx,
                                                                   float* __restrict__ out_key, u64k* k64a,
                                                                   int32_t* ia, u64k* k64b, int32_t* ib,
                                                                   int32_t* __restrict__ strip_pos,
                                                                   float* __restrict__ strip_k2) {
    extern __shared__ __align__(16) unsigned char smraw[];
    u64k* sk = reinterpret_cast<u64k*>(smraw);
    int32_t* si = reinterpret_cast<int32_t*>(sk + kSortRun);
    __shared__ int s_pos[kMaxStrips + 1];
    const SortGroup G = groups[blockIdx.x];
    const int N = G.N;
    u64k* ak = k64a + G.off;
    int32_t* ai = ia + G.off;
    u64k* bk = k64b + G.off;
    int32_t* bi = ib + G.off;
    if (G.S <= 1) {
        sort_pairs(N, [&](int p, u64k& k, int& i) { k = ord_bits(group_coord(G, p, 1)); i = p; }, ak, ai, bk, bi, sk,
                   si);
        for (int p = threadIdx.x; p < N; p += blockDim.x) {
            out_idx[G.off + p] = ai[p];
            out_key[G.off + p] = from_ord((unsigned)ak[p]);
        }
        return;
    }
    const int S = G.S;
    const int L = G.L;
    // 1. by the second key: strip s holds the points of rank s L .. min((s + 1) L, N) - 1
    sort_pairs(N, [&](int p, u64k& k, int& i) { k = ord_bits(group_coord(G, p, G.k2lag)); i = p; }, ak, ai, bk,
               bi, sk, si);
    if (threadIdx.x == 0) {
        int pos = 0;
        for (int s = 0; s < S; ++s) {
            const int a = s * L, b = min((s + 1) * L, N);
            s_pos[s] = pos;
            strip_k2[2 * G.strip_off + 2 * s] = from_ord((unsigned)ak[a]);
            strip_k2[2 * G.strip_off + 2 * s + 1] = from_ord((unsigned)ak[b - 1]);
            pos += (b - a + 3) & ~3;
        }
        s_pos[S] = pos;
        for (int s = 0; s <= S; ++s) strip_pos[G.strip_off + s] = s_pos[s];
    }
    __syncthreads();
    // 2. by (strip, y_{t'-1}), read in place from step 1's result
    sort_pairs(
        N,
        [&](int p, u64k& k, int& i) {
            i = ai[p];
            const unsigned s = (unsigned)(p / L);
            k = ((u64k)s << 32) | ord_bits(group_coord(G, i, 1));
        },
        ak, ai, bk, bi, sk, si);
    // 3. scatter into the padded strip layout
    for (int p = threadIdx.x; p < G.npad; p += blockDim.x) {
        out_idx[G.off + p] = -1;
        out_key[G.off + p] = __int_as_float(0x7f800000);
    }
    __syncthreads();
    for (int p = threadIdx.x; p < N; p += blockDim.x) {
        const int s = (int)(ak[p] >> 32);
        const int dst = s_pos[s] + (p - s * L);
        out_idx[G.off + dst] = ai[p];
        out_key[G.off + dst] = from_ord((unsigned)ak[p]);
    }
}

}  // namespace

cudaError_t prepare_sort_kernel(int /*nmax*/) {
    return cudaFuncSetAttribute(sort_groups_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSortRun * 12);
}

cudaError_t launch_sort_groups(const SortGroup* groups, int n_groups, int32_t* idx, float* key, u64k* k64a,
                               int32_t* ia, u64k* k64b, int32_t* ib, int32_t* strip_pos, float* strip_k2,
                               cudaStream_t s) {
    sort_groups_kernel<<<n_groups, kSortThreads, kSortRun * 12, s>>>(groups, idx, key, k64a, ia, k64b, ib,
                                                                      strip_pos, strip_k2);
    return cudaGetLastError();
}

}  // namespace te
