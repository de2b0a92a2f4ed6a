// Single-instance kernels behind te_embed, te_knn_maxnorm and te_range_count.
//
// te_embed:        Eq. 6 / Eq. 7 delay embedding, source at t-u, points pooled as in Eq. 10.
// te_knn_maxnorm:  brute-force max-norm kNN (Implementation section, "Core algorithm").
// te_range_count:  strict range counts in the marginal spaces of Eq. 9.
//
// The joint dimensions of the supported embeddings (D = 1 + 2d, d = 1..5) run the same
// register-blocked tile loops as the batched kernel; any other D <= 32 runs a plain
// per-reference loop over zero-padded coordinates (padding is exact: |0 - 0| = 0 never
// raises a maximum).
#include "te_device.cuh"

namespace te {

namespace {

constexpr int kUnitThreads = 128;
constexpr int kUnitQ = 4;
constexpr int kUnitTile = 256;  // references per shared-memory tile (multiple of 4)

// ------------------------------------------------------------------------------- embed
__global__ void embed_kernel(const float* __restrict__ src, const float* __restrict__ tgt, int R,
                             int T, int d, int tau, int u, int t_start, int W,
                             const int32_t* __restrict__ perm, float* __restrict__ points, int ld,
                             int32_t* flags) {
    const int N = R * W;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int r = i / W;
    const int t = t_start + (i - r * W);
    int rs = r;
    if (perm) {
        rs = perm[r];
        if ((unsigned)rs >= (unsigned)R) {
            atomicOr(flags, kFlagBadPerm);
            rs = 0;
        }
    }
    const float* y = tgt + (size_t)r * T;
    const float* x = src + (size_t)rs * T;
    points[i] = y[t];
    for (int m = 0; m < d; ++m) points[(size_t)(1 + m) * ld + i] = y[t - 1 - m * tau];
    for (int m = 0; m < d; ++m) points[(size_t)(1 + d + m) * ld + i] = x[t - u - m * tau];
}

// stage references base .. base+kUnitTile-1 of an SoA point array into a shared-memory tile
// (groups of four points, te_device.cuh), +inf past N
template <int D>
__device__ __forceinline__ void stage_soa(const float* __restrict__ pts, int ld, int N, int base,
                                          float* s) {
    for (int p = threadIdx.x; p < kUnitTile; p += blockDim.x) {
        const bool ok = base + p < N;
#pragma unroll
        for (int c = 0; c < D; ++c) s[tile_index<D>(c, p)] = ok ? pts[(size_t)c * ld + base + p] : f_inf();
    }
}

// ------------------------------------------------------------------------------- kNN, exact D
template <int D, int KS>
__global__ void __launch_bounds__(kUnitThreads) knn_exact_kernel(const float* __restrict__ pts, int N,
                                                                 int ld, int k, float* __restrict__ eps) {
    __shared__ __align__(16) float s[D * kUnitTile];
    u64 qq[kUnitQ][D];
    float t[kUnitQ][KS];
    const int i0 = blockIdx.x * (kUnitThreads * kUnitQ) + threadIdx.x;
#pragma unroll
    for (int q = 0; q < kUnitQ; ++q) {
        const int i = i0 + q * kUnitThreads;
#pragma unroll
        for (int c = 0; c < D; ++c) qq[q][c] = dup2(i < N ? pts[(size_t)c * ld + i] : 0.0f);
#pragma unroll
        for (int m = 0; m < KS; ++m) t[q][m] = f_inf();
    }
    for (int base = 0; base < N; base += kUnitTile) {
        __syncthreads();
        stage_soa<D>(pts, ld, N, base, s);
        __syncthreads();
        const int nv = min(kUnitTile, N - base);
        knn_tile<D, kUnitQ, KS>(s, (nv + 3) >> 2, qq, t);
    }
#pragma unroll
    for (int q = 0; q < kUnitQ; ++q) {
        const int i = i0 + q * kUnitThreads;
        const float e = topk_select(t[q], k);
        if (i < N) eps[i] = e;
    }
}

// ------------------------------------------------------------------------------- kNN, generic
// Any D <= DP (zero padded), optional neighbour indices with (distance, index) ordering.
template <int DP, int KS, bool IDX>
__global__ void __launch_bounds__(kUnitThreads) knn_generic_kernel(const float* __restrict__ pts, int N,
                                                                   int D, int ld, int k,
                                                                   float* __restrict__ eps,
                                                                   int32_t* __restrict__ nn) {
    __shared__ __align__(16) float s[DP * kUnitTile];
    const int i = blockIdx.x * kUnitThreads + threadIdx.x;
    float qc[DP];
#pragma unroll
    for (int c = 0; c < DP; ++c) qc[c] = (i < N && c < D) ? pts[(size_t)c * ld + i] : 0.0f;
    float t[KS];
    int id[KS];
#pragma unroll
    for (int m = 0; m < KS; ++m) {
        t[m] = f_inf();
        id[m] = 0x7fffffff;
    }
    for (int base = 0; base < N; base += kUnitTile) {
        __syncthreads();
        for (int p = threadIdx.x; p < kUnitTile; p += blockDim.x) {
            const bool ok = base + p < N;
#pragma unroll
            for (int c = 0; c < DP; ++c)
                s[c * kUnitTile + p] = ok ? (c < D ? pts[(size_t)c * ld + base + p] : 0.0f) : f_inf();
        }
        __syncthreads();
        const int nv = min(kUnitTile, N - base);
#pragma unroll 1
        for (int j = 0; j < nv; ++j) {
            float m = fabsf(qc[0] - s[j]);
#pragma unroll
            for (int c = 1; c < DP; ++c) m = fmaxf(m, fabsf(qc[c] - s[c * kUnitTile + j]));
            if (!IDX) {
                topk_push(t, m);
            } else {
                const int jj = base + j;
                // lexicographic (distance, index) insertion into the ascending list
                if (m < t[KS - 1] || (m == t[KS - 1] && jj < id[KS - 1])) {
#pragma unroll
                    for (int sl = KS - 1; sl >= 0; --sl) {
                        const bool before_prev =
                            sl > 0 && (m < t[sl - 1] || (m == t[sl - 1] && jj < id[sl - 1]));
                        const bool before_cur = m < t[sl] || (m == t[sl] && jj < id[sl]);
                        if (before_prev) {
                            t[sl] = t[sl - 1];
                            id[sl] = id[sl - 1];
                        } else if (before_cur) {
                            t[sl] = m;
                            id[sl] = jj;
                        }
                    }
                }
            }
        }
    }
    if (i >= N) return;
    eps[i] = topk_select(t, k);
    if (IDX) {
        // the k+1 smallest (distance, index) pairs include i itself unless more than k other
        // points lie at distance 0 with a lower index; drop i, else drop the last one
        int w = 0;
        bool dropped = false;
#pragma unroll
        for (int sl = 0; sl < KS; ++sl) {
            if (sl > k) break;
            if (!dropped && id[sl] == i) {
                dropped = true;
                continue;
            }
            if (w < k) nn[(size_t)i * k + w] = id[sl];
            ++w;
        }
    }
}

// ------------------------------------------------------------------------------- counts, exact
template <int DY, int DX>
__global__ void __launch_bounds__(kUnitThreads) count_exact_kernel(const float* __restrict__ pts, int N,
                                                                   int ld, const float* __restrict__ eps,
                                                                   int32_t* __restrict__ counts) {
    constexpr int D = 1 + DY + DX;
    __shared__ __align__(16) float s[D * kUnitTile];
    u64 qq[kUnitQ][D];
    float e[kUnitQ];
    float cz[kUnitQ], cyz[kUnitQ], cxz[kUnitQ];
    const int i0 = blockIdx.x * (kUnitThreads * kUnitQ) + threadIdx.x;
#pragma unroll
    for (int q = 0; q < kUnitQ; ++q) {
        const int i = i0 + q * kUnitThreads;
#pragma unroll
        for (int c = 0; c < D; ++c) qq[q][c] = dup2(i < N ? pts[(size_t)c * ld + i] : 0.0f);
        e[q] = i < N ? eps[i] : 0.0f;
        cz[q] = cyz[q] = cxz[q] = 0.0f;
    }
    for (int base = 0; base < N; base += kUnitTile) {
        __syncthreads();
        stage_soa<D>(pts, ld, N, base, s);
        __syncthreads();
        const int nv = min(kUnitTile, N - base);
        count_tile<DY, DX, kUnitQ>(s, (nv + 3) >> 2, qq, e, cz, cyz, cxz);
    }
#pragma unroll
    for (int q = 0; q < kUnitQ; ++q) {
        const int i = i0 + q * kUnitThreads;
        if (i < N) {
            const int self = e[q] > 0.0f ? 1 : 0;  // the point itself lies at distance 0
            counts[i] = (int)cz[q] - self;
            counts[(size_t)N + i] = (int)cyz[q] - self;
            counts[(size_t)2 * N + i] = (int)cxz[q] - self;
        }
    }
}

// ------------------------------------------------------------------------------- counts, generic
template <int DP>
__global__ void __launch_bounds__(kUnitThreads) count_generic_kernel(const float* __restrict__ pts, int N,
                                                                     int dy, int dx, int ld,
                                                                     const float* __restrict__ eps,
                                                                     int32_t* __restrict__ counts) {
    __shared__ __align__(16) float s[DP * kUnitTile];
    const int D = 1 + dy + dx;
    const int i = blockIdx.x * kUnitThreads + threadIdx.x;
    float qc[DP];
#pragma unroll
    for (int c = 0; c < DP; ++c) qc[c] = (i < N && c < D) ? pts[(size_t)c * ld + i] : 0.0f;
    const float e = i < N ? eps[i] : 0.0f;
    int cz = 0, cyz = 0, cxz = 0;
    for (int base = 0; base < N; base += kUnitTile) {
        __syncthreads();
        for (int p = threadIdx.x; p < kUnitTile; p += blockDim.x) {
            const bool ok = base + p < N;
#pragma unroll
            for (int c = 0; c < DP; ++c)
                s[c * kUnitTile + p] = (ok && c < D) ? pts[(size_t)c * ld + base + p] : 0.0f;
        }
        __syncthreads();
        const int nv = min(kUnitTile, N - base);
#pragma unroll 1
        for (int j = 0; j < nv; ++j) {
            const float a = fabsf(qc[0] - s[j]);
            float b = 0.0f, x = 0.0f;
#pragma unroll
            for (int c = 1; c < DP; ++c) {
                const float v = fabsf(qc[c] - s[c * kUnitTile + j]);
                if (c <= dy) b = fmaxf(b, v);
                else x = fmaxf(x, v);  // source group and zero padding (|0-0| = 0)
            }
            cz += (b < e) ? 1 : 0;
            cyz += (fmaxf(a, b) < e) ? 1 : 0;
            cxz += (fmaxf(b, x) < e) ? 1 : 0;
        }
    }
    if (i < N) {
        const int self = e > 0.0f ? 1 : 0;
        counts[i] = cz - self;
        counts[(size_t)N + i] = cyz - self;
        counts[(size_t)2 * N + i] = cxz - self;
    }
}

template <int KS>
cudaError_t knn_dispatch(const float* pts, int N, int D, int ld, int k, float* eps, int32_t* nn,
                         cudaStream_t st) {
    const dim3 blk(kUnitThreads);
    if (!nn) {
        const dim3 grd((N + kUnitThreads * kUnitQ - 1) / (kUnitThreads * kUnitQ));
        switch (D) {
            case 3: knn_exact_kernel<3, KS><<<grd, blk, 0, st>>>(pts, N, ld, k, eps); return cudaGetLastError();
            case 5: knn_exact_kernel<5, KS><<<grd, blk, 0, st>>>(pts, N, ld, k, eps); return cudaGetLastError();
            case 7: knn_exact_kernel<7, KS><<<grd, blk, 0, st>>>(pts, N, ld, k, eps); return cudaGetLastError();
            case 9: knn_exact_kernel<9, KS><<<grd, blk, 0, st>>>(pts, N, ld, k, eps); return cudaGetLastError();
            case 11: knn_exact_kernel<11, KS><<<grd, blk, 0, st>>>(pts, N, ld, k, eps); return cudaGetLastError();
            default: break;
        }
    }
    const dim3 grd((N + kUnitThreads - 1) / kUnitThreads);
    if (D <= 4) {
        if (nn) knn_generic_kernel<4, KS, true><<<grd, blk, 0, st>>>(pts, N, D, ld, k, eps, nn);
        else knn_generic_kernel<4, KS, false><<<grd, blk, 0, st>>>(pts, N, D, ld, k, eps, nn);
    } else if (D <= 8) {
        if (nn) knn_generic_kernel<8, KS, true><<<grd, blk, 0, st>>>(pts, N, D, ld, k, eps, nn);
        else knn_generic_kernel<8, KS, false><<<grd, blk, 0, st>>>(pts, N, D, ld, k, eps, nn);
    } else if (D <= 16) {
        if (nn) knn_generic_kernel<16, KS, true><<<grd, blk, 0, st>>>(pts, N, D, ld, k, eps, nn);
        else knn_generic_kernel<16, KS, false><<<grd, blk, 0, st>>>(pts, N, D, ld, k, eps, nn);
    } else {
        if (nn) knn_generic_kernel<32, KS, true><<<grd, blk, 0, st>>>(pts, N, D, ld, k, eps, nn);
        else knn_generic_kernel<32, KS, false><<<grd, blk, 0, st>>>(pts, N, D, ld, k, eps, nn);
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_embed(const float* src, const float* tgt, int R, int T, int d, int tau, int u,
                         int t_start, int W, const int32_t* perm, float* points, int ld,
                         int32_t* flags, cudaStream_t s) {
    const int N = R * W;
    embed_kernel<<<(N + 255) / 256, 256, 0, s>>>(src, tgt, R, T, d, tau, u, t_start, W, perm, points,
                                                  ld, flags);
    return cudaGetLastError();
}

cudaError_t launch_knn(const float* pts, int N, int D, int ld, int k, float* eps, int32_t* nn,
                       int /*sm_count*/, cudaStream_t s) {
    if (k <= 4) return knn_dispatch<5>(pts, N, D, ld, k, eps, nn, s);
    if (k <= 8) return knn_dispatch<9>(pts, N, D, ld, k, eps, nn, s);
    return knn_dispatch<17>(pts, N, D, ld, k, eps, nn, s);
}

cudaError_t launch_count(const float* pts, int N, int dy, int dx, int ld, const float* eps,
                         int32_t* counts, int /*sm_count*/, cudaStream_t s) {
    const dim3 blk(kUnitThreads);
    if (dy == dx && dy >= 1 && dy <= 5) {
        const dim3 grd((N + kUnitThreads * kUnitQ - 1) / (kUnitThreads * kUnitQ));
        switch (dy) {
            case 1: count_exact_kernel<1, 1><<<grd, blk, 0, s>>>(pts, N, ld, eps, counts); break;
            case 2: count_exact_kernel<2, 2><<<grd, blk, 0, s>>>(pts, N, ld, eps, counts); break;
            case 3: count_exact_kernel<3, 3><<<grd, blk, 0, s>>>(pts, N, ld, eps, counts); break;
            case 4: count_exact_kernel<4, 4><<<grd, blk, 0, s>>>(pts, N, ld, eps, counts); break;
            default: count_exact_kernel<5, 5><<<grd, blk, 0, s>>>(pts, N, ld, eps, counts); break;
        }
        return cudaGetLastError();
    }
    const int D = 1 + dy + dx;
    const dim3 grd((N + kUnitThreads - 1) / kUnitThreads);
    if (D <= 4) count_generic_kernel<4><<<grd, blk, 0, s>>>(pts, N, dy, dx, ld, eps, counts);
    else if (D <= 8) count_generic_kernel<8><<<grd, blk, 0, s>>>(pts, N, dy, dx, ld, eps, counts);
    else if (D <= 16) count_generic_kernel<16><<<grd, blk, 0, s>>>(pts, N, dy, dx, ld, eps, counts);
    else count_generic_kernel<32><<<grd, blk, 0, s>>>(pts, N, dy, dx, ld, eps, counts);
    return cudaGetLastError();
}

}  // namespace te
