// Device building blocks of the max-norm kNN search, the marginal range counts and the
// digamma sum (Wollstadt et al. 2014, Eq. 9 / Eq. 10; brute-force infinity-norm search of the
// Implementation section).
//
// Exactness: every distance is max_c |fl32(q_c - r_c)| with IEEE round-to-nearest subtraction
// (built without fast-math, FMA contraction or flush-to-zero); min/max/abs are exact, so eps
// and the counts equal the values of any sequential FP32 evaluation.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "te_internal.h"

namespace te {

__device__ __forceinline__ float f_inf() { return __int_as_float(0x7f800000); }

template <int E>
__device__ __forceinline__ float comp(const float4& v) {
    return E == 0 ? v.x : (E == 1 ? v.y : (E == 2 ? v.z : v.w));
}

// ---------------------------------------------------------------------------------------
// Top-(k+1) of all N distances, self included. The point's distance to itself is 0, the
// smallest possible value, so the (k+1)-th smallest over all j equals the k-th smallest over
// j != i for any data (duplicates included). KS slots hold the KS smallest values seen, in
// ascending order; an insertion is a min/max merge network.
// ---------------------------------------------------------------------------------------
template <int KS>
__device__ __forceinline__ void topk_push(float (&t)[KS], float x) {
    if (x < t[KS - 1]) {
#pragma unroll
        for (int s = KS - 1; s > 0; --s) t[s] = fmaxf(t[s - 1], fminf(t[s], x));
        t[0] = fminf(t[0], x);
    }
}

// slot k of the ascending list (k is a runtime value < KS), written as the maximum of slots
// 0..k so that the list stays in registers (a select on s == k is compiled as a dynamic index)
template <int KS>
__device__ __forceinline__ float topk_select(const float (&t)[KS], int k) {
    float e = t[0];
#pragma unroll
    for (int s = 1; s < KS; ++s) e = fmaxf(e, s <= k ? t[s] : t[0]);
    return e;
}

// ---------------------------------------------------------------------------------------
// Pass 1 over one staged reference tile: smem holds coordinate c of reference j at
// s[c * ldt + j] (structure of arrays, +inf past the last valid reference). Every thread
// streams the whole tile against its Q register-resident queries; four references are
// read per float4 broadcast load.
// ---------------------------------------------------------------------------------------
template <int D, int Q, int KS>
__device__ __forceinline__ void knn_tile(const float* __restrict__ s, int ldt, int n4,
                                         const float (&qc)[Q][D], float (&t)[Q][KS]) {
#pragma unroll 1
    for (int j = 0; j < n4; ++j) {
        float4 r[D];
#pragma unroll
        for (int c = 0; c < D; ++c) r[c] = *reinterpret_cast<const float4*>(s + c * ldt + 4 * j);
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            float m0 = fabsf(qc[q][0] - r[0].x);
            float m1 = fabsf(qc[q][0] - r[0].y);
            float m2 = fabsf(qc[q][0] - r[0].z);
            float m3 = fabsf(qc[q][0] - r[0].w);
#pragma unroll
            for (int c = 1; c < D; ++c) {
                m0 = fmaxf(m0, fabsf(qc[q][c] - r[c].x));
                m1 = fmaxf(m1, fabsf(qc[q][c] - r[c].y));
                m2 = fmaxf(m2, fabsf(qc[q][c] - r[c].z));
                m3 = fmaxf(m3, fabsf(qc[q][c] - r[c].w));
            }
            topk_push(t[q], m0);
            topk_push(t[q], m1);
            topk_push(t[q], m2);
            topk_push(t[q], m3);
        }
    }
}

// ---------------------------------------------------------------------------------------
// Pass 2 over one staged tile: grouped maxima a = |dy_t|, b = max |dy-|, x = max |dx-| and
// the three strict counts of Eq. 9: n_z (b < e), n_yz (max(a,b) < e), n_xz (max(b,x) < e).
// The query itself is included here (a = b = x = 0) and removed by the caller.
// ---------------------------------------------------------------------------------------
template <int DY, int DX, int Q, int E>
__device__ __forceinline__ void count_one(const float (&q)[1 + DY + DX], const float4 (&r)[1 + DY + DX],
                                          float e, int& cz, int& cyz, int& cxz) {
    const float a = fabsf(q[0] - comp<E>(r[0]));
    float b = 0.0f;
#pragma unroll
    for (int c = 1; c <= DY; ++c) b = (c == 1) ? fabsf(q[c] - comp<E>(r[c])) : fmaxf(b, fabsf(q[c] - comp<E>(r[c])));
    float x = 0.0f;
#pragma unroll
    for (int c = DY + 1; c <= DY + DX; ++c)
        x = (c == DY + 1) ? fabsf(q[c] - comp<E>(r[c])) : fmaxf(x, fabsf(q[c] - comp<E>(r[c])));
    cz += (b < e) ? 1 : 0;
    cyz += (fmaxf(a, b) < e) ? 1 : 0;
    cxz += (fmaxf(b, x) < e) ? 1 : 0;
}

template <int DY, int DX, int Q>
__device__ __forceinline__ void count_tile(const float* __restrict__ s, int ldt, int n4,
                                           const float (&qc)[Q][1 + DY + DX], const float (&e)[Q],
                                           int (&cz)[Q], int (&cyz)[Q], int (&cxz)[Q]) {
    constexpr int D = 1 + DY + DX;
#pragma unroll 1
    for (int j = 0; j < n4; ++j) {
        float4 r[D];
#pragma unroll
        for (int c = 0; c < D; ++c) r[c] = *reinterpret_cast<const float4*>(s + c * ldt + 4 * j);
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            count_one<DY, DX, Q, 0>(qc[q], r, e[q], cz[q], cyz[q], cxz[q]);
            count_one<DY, DX, Q, 1>(qc[q], r, e[q], cz[q], cyz[q], cxz[q]);
            count_one<DY, DX, Q, 2>(qc[q], r, e[q], cz[q], cyz[q], cxz[q]);
            count_one<DY, DX, Q, 3>(qc[q], r, e[q], cz[q], cyz[q], cxz[q]);
        }
    }
}

// ---------------------------------------------------------------------------------------
// Eq. 6 / 7 / 10 fused into the loads: coordinates of point i of an instance, read straight
// from the trial x sample series (target past at t'-1, source past at t'-u).
// ---------------------------------------------------------------------------------------
template <int d>
__device__ __forceinline__ void gather_point(const InstDesc& I, int i, float (&p)[1 + 2 * d],
                                             int32_t* flags) {
    const int r = i / I.W;
    const int t = I.t_start + (i - r * I.W);
    int rs = r;
    if (I.perm) {
        rs = __ldg(I.perm + r);
        if ((unsigned)rs >= (unsigned)I.R) {
            atomicOr(flags, kFlagBadPerm);
            rs = 0;
        }
    }
    const float* y = I.tgt + (size_t)r * I.T;
    const float* x = I.src + (size_t)rs * I.T;
    p[0] = __ldg(y + t);
#pragma unroll
    for (int m = 0; m < d; ++m) p[1 + m] = __ldg(y + t - 1 - m * I.tau);
#pragma unroll
    for (int m = 0; m < d; ++m) p[1 + d + m] = __ldg(x + t - I.u - m * I.tau);
}

// ---------------------------------------------------------------------------------------
// Compensated FP32 accumulation (float-float: TwoSum of the high parts, low parts added,
// renormalised with FastTwoSum). Intrinsics keep the compiler from reassociating.
// ---------------------------------------------------------------------------------------
struct FF {
    float hi, lo;
};

__device__ __forceinline__ FF ff_add(FF a, float bh, float bl) {
    const float s = __fadd_rn(a.hi, bh);
    const float bb = __fsub_rn(s, a.hi);
    const float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(bh, bb));
    float lo = __fadd_rn(__fadd_rn(a.lo, bl), err);
    const float hi = __fadd_rn(s, lo);
    lo = __fsub_rn(lo, __fsub_rn(hi, s));
    return FF{hi, lo};
}

// Block-wide sum of two doubles in a fixed order (deterministic). smem: 2 * 32 doubles.
// Returns the totals in thread 0.
__device__ __forceinline__ void block_sum2(double& v, double& w, double* sred) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v += __shfl_down_sync(0xffffffffu, v, o);
        w += __shfl_down_sync(0xffffffffu, w, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        sred[warp] = v;
        sred[32 + warp] = w;
    }
    __syncthreads();
    if (warp == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        v = lane < nw ? sred[lane] : 0.0;
        w = lane < nw ? sred[32 + lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            v += __shfl_down_sync(0xffffffffu, v, o);
            w += __shfl_down_sync(0xffffffffu, w, o);
        }
    }
}

}  // namespace te
