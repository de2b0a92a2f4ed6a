// Persistent batched kernel: every (instance, query tile) of a batch of estimates in one
// launch. An instance is one time point of one channel pair with one repetition pairing
// (original or a trial-shuffled surrogate, Fig. 3); its TE is Eq. 9 / Eq. 10.
//
// One CTA takes a work item from a device queue (atomic ticket, no waits), then:
//   1. gathers its queries' joint coordinates straight from the series (Eq. 6 / 7 with the
//      source at t-u and the surrogate's repetition pairing) into registers;
//   2. pass 1: streams the instance's points through shared memory in tiles (groups of four
//      points, see te_device.cuh) and keeps, per query, the k+1 smallest max-norm distances
//      (self included), so
//      eps = the k-th neighbour distance among the other points;
//   3. pass 2: streams the same tiles again (they stay resident when the whole instance fits)
//      and counts points strictly inside eps in the three marginal spaces;
//   4. maps the counts to digamma terms through a (hi, lo) float table, sums them per thread
//      in compensated FP32, per CTA in FP64, and writes one partial sum per work item.
// A separate finalisation kernel adds the partials of each instance (FP64, fixed order).
#pragma once

#include "te_device.cuh"

namespace te {

template <int d>
__device__ __forceinline__ void stage_tile(const InstDesc& I, int base, int nv, float* sm, int32_t* flags) {
    constexpr int D = 1 + 2 * d;
    const int nfill = (nv + 3) & ~3;
    for (int p = threadIdx.x; p < nfill; p += blockDim.x) {
        float v[D];
        if (p < nv) {
            gather_point<d>(I, base + p, v, flags);
        } else {
#pragma unroll
            for (int c = 0; c < D; ++c) v[c] = f_inf();
        }
#pragma unroll
        for (int c = 0; c < D; ++c) sm[tile_index<D>(c, p)] = v[c];
    }
}

template <int d, int Q, int KS>
__device__ __forceinline__ void process_item(const BatchArgs& a, const InstDesc& I, int q0, int it,
                                             float* sm, double* sred) {
    constexpr int D = 1 + 2 * d;
    const int N = I.N;
    const int T = blockDim.x;
    const int ldt = (a.smem_floats / D) & ~3;  // references per tile
    const int ntile = (N + ldt - 1) / ldt;

    // queries of this thread: q0 + threadIdx.x + q * T, each coordinate duplicated (q, q)
    u64 qq[Q][D];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int i = q0 + threadIdx.x + q * T;
        float p[D];
        if (i < N) {
            gather_point<d>(I, i, p, a.flags);
        } else {
#pragma unroll
            for (int c = 0; c < D; ++c) p[c] = 0.0f;
        }
#pragma unroll
        for (int c = 0; c < D; ++c) qq[q][c] = dup2(p[c]);
    }
    // warps whose first query is past N have nothing to compute (warp-uniform)
    const bool warp_active = q0 + (int)(threadIdx.x & ~31u) < N;

    // ---- pass 1: k-th neighbour distance in the joint space
    float t[Q][KS];
#pragma unroll
    for (int q = 0; q < Q; ++q)
#pragma unroll
        for (int m = 0; m < KS; ++m) t[q][m] = f_inf();
    for (int tile = 0; tile < ntile; ++tile) {
        const int base = tile * ldt;
        const int nv = min(ldt, N - base);
        __syncthreads();
        stage_tile<d>(I, base, nv, sm, a.flags);
        __syncthreads();
        if (warp_active) knn_tile<D, Q, KS>(sm, (nv + 3) >> 2, qq, t);
    }
    float e[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) e[q] = topk_select(t[q], a.k);

    // ---- pass 2: strict counts in the marginal spaces
    float cz[Q], cyz[Q], cxz[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) cz[q] = cyz[q] = cxz[q] = 0.0f;
    for (int tile = 0; tile < ntile; ++tile) {
        const int base = tile * ldt;
        const int nv = min(ldt, N - base);
        if (ntile > 1) {  // a single tile is still resident from pass 1
            __syncthreads();
            stage_tile<d>(I, base, nv, sm, a.flags);
            __syncthreads();
        }
        if (warp_active) count_tile<d, d, Q>(sm, (nv + 3) >> 2, qq, e, cz, cyz, cxz);
    }

    // ---- digamma terms of Eq. 9, compensated FP32 per thread
    FF acc{0.0f, 0.0f};
    float acc_abs = 0.0f;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int i = q0 + threadIdx.x + q * T;
        if (i < N) {
            const int self = e[q] > 0.0f ? 1 : 0;  // the point itself was counted at distance 0
            const int nz = (int)cz[q] - self, nyz = (int)cyz[q] - self, nxz = (int)cxz[q] - self;
            if (a.counts_out) {
                int32_t* co = a.counts_out + 3 * I.pt_off;
                co[i] = nz;
                co[N + i] = nyz;
                co[2 * N + i] = nxz;
            }
            if (a.eps_out) a.eps_out[I.pt_off + i] = e[q];
            const float2 p1 = __ldg(a.psi + nz + 1);
            const float2 p2 = __ldg(a.psi + nyz + 1);
            const float2 p3 = __ldg(a.psi + nxz + 1);
            acc = ff_add(acc, p1.x, p1.y);
            acc = ff_add(acc, -p2.x, -p2.y);
            acc = ff_add(acc, -p3.x, -p3.y);
            acc_abs += fabsf(p1.x) + fabsf(p2.x) + fabsf(p3.x);
        }
    }
    // ---- per-item partial in FP64, fixed reduction order
    double v = (double)acc.hi + (double)acc.lo;
    double w = (double)acc_abs;
    block_sum2(v, w, sred);
    if (threadIdx.x == 0) {
        a.partial[it] = v;
        a.partial_abs[it] = w;
    }
}

}  // namespace te
