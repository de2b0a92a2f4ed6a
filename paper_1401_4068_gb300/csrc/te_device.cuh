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

// four candidates: one test of their minimum against the last slot guards the four insertions
// (once the list has filled, most groups of four change nothing)
template <int KS>
__device__ __forceinline__ void topk_push4(float (&t)[KS], float m0, float m1, float m2, float m3) {
    if (fminf(fminf(m0, m1), fminf(m2, m3)) < t[KS - 1]) {
        const float v[4] = {m0, m1, m2, m3};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
#pragma unroll
            for (int s = KS - 1; s > 0; --s) t[s] = fmaxf(t[s - 1], fminf(t[s], v[e]));
            t[0] = fminf(t[0], v[e]);
        }
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
// Packed FP32 forms of sm_100-family GPUs, written as inline PTX:
//   sub.rn.f32x2   two IEEE round-to-nearest subtractions in one instruction (each lane of the
//                  pair is exactly fl32(a - b));
//   max.abs.f32    with three inputs: max(|a|, |b|, |c|), two new coordinates per instruction;
//   set.lt.f32.f32 1.0f if a < b else 0.0f.
// A query coordinate is kept duplicated in a 64-bit register pair (q, q) so that one packed
// subtraction covers two references.
// ---------------------------------------------------------------------------------------
typedef unsigned long long u64;

__device__ __forceinline__ u64 dup2(float q) {
    u64 r;
    asm("mov.b64 %0, {%1, %1};" : "=l"(r) : "f"(q));
    return r;
}
__device__ __forceinline__ u64 sub2(u64 a, u64 b) {
    u64 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ void split2(u64 v, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ float absmax3(float a, float b, float c) {
    float d;
    asm("max.abs.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}
__device__ __forceinline__ float set_lt(float a, float b) {
    float d;
    asm("set.lt.f32.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b));
    return d;
}
__device__ __forceinline__ float abs_set_lt(float a, float b) {
    float d;
    asm("{.reg .f32 t; abs.f32 t, %1; set.lt.f32.f32 %0, t, %2;}" : "=f"(d) : "f"(a), "f"(b));
    return d;
}

// max |v[c]| over c = C0 .. C1 (inclusive, C1 >= C0), three inputs per instruction
template <int C0, int C1, int N>
__device__ __forceinline__ float absmax_range(const float (&v)[N]) {
    constexpr int n = C1 - C0 + 1;
    float m = absmax3(v[C0], v[n >= 2 ? C0 + 1 : C0], v[n >= 3 ? C0 + 2 : (n >= 2 ? C0 + 1 : C0)]);
#pragma unroll
    for (int c = C0 + 3; c <= C1; c += 2) m = absmax3(m, v[c], v[c + 1 <= C1 ? c + 1 : c]);
    return m;
}

// the D coordinate differences of one query against four references, unpacked per reference
template <int D>
__device__ __forceinline__ void diff4(const u64 (&qq)[D], const ulonglong2 (&r)[D], float (&dx)[D],
                                      float (&dy)[D], float (&dz)[D], float (&dw)[D]) {
#pragma unroll
    for (int c = 0; c < D; ++c) {
        split2(sub2(qq[c], r[c].x), dx[c], dy[c]);
        split2(sub2(qq[c], r[c].y), dz[c], dw[c]);
    }
}

// ---------------------------------------------------------------------------------------
// Shared-memory tiles hold points in groups of four: group g (points 4g .. 4g+3) stores its
// D coordinates x 4 points contiguously, coordinate c of point p at
//   s[((p >> 2) * D + c) * 4 + (p & 3)],
// so one 128-bit broadcast load reads coordinate c of a whole group at the constant offset 16c
// bytes from the group's base (one address per group instead of one per coordinate).
// ---------------------------------------------------------------------------------------
template <int D>
__device__ __forceinline__ int tile_index(int c, int p) {
    return ((p >> 2) * D + c) * 4 + (p & 3);
}

template <int D>
__device__ __forceinline__ void load_refs4(const float* __restrict__ s, int j, ulonglong2 (&r)[D]) {
    const float* g = s + j * (4 * D);
#pragma unroll
    for (int c = 0; c < D; ++c) r[c] = *reinterpret_cast<const ulonglong2*>(g + 4 * c);
}

// smallest / largest key (coordinate 1) of group j of a tile (groups are in key order in the sweep)
template <int D>
__device__ __forceinline__ float group_key_lo(const float* __restrict__ s, int j) {
    return s[(j * D + 1) * 4];
}
template <int D>
__device__ __forceinline__ float group_key_hi(const float* __restrict__ s, int j) {
    return s[(j * D + 1) * 4 + 3];
}

// Pass-1 step for four references against the thread's Q queries. For D >= 5 every distance
// is computed before the first (branching) top-k insertion, which leaves the scheduler more
// independent work across the branches; for D = 3 the interleaved order measures faster.
template <int D, int Q, int KS>
__device__ __forceinline__ void knn_step4(const u64 (&qq)[Q][D], const ulonglong2 (&r)[D], float (&t)[Q][KS]) {
    if constexpr (D <= 3) {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            float dx[D], dy[D], dz[D], dw[D];
            diff4<D>(qq[q], r, dx, dy, dz, dw);
            topk_push4(t[q], absmax_range<0, D - 1>(dx), absmax_range<0, D - 1>(dy), absmax_range<0, D - 1>(dz),
                       absmax_range<0, D - 1>(dw));
        }
    } else {
        float m[Q][4];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            float dx[D], dy[D], dz[D], dw[D];
            diff4<D>(qq[q], r, dx, dy, dz, dw);
            m[q][0] = absmax_range<0, D - 1>(dx);
            m[q][1] = absmax_range<0, D - 1>(dy);
            m[q][2] = absmax_range<0, D - 1>(dz);
            m[q][3] = absmax_range<0, D - 1>(dw);
        }
#pragma unroll
        for (int q = 0; q < Q; ++q) topk_push4(t[q], m[q][0], m[q][1], m[q][2], m[q][3]);
    }
}

// ---------------------------------------------------------------------------------------
// Pass 1 over one staged reference tile (grouped layout above, +inf past the last valid
// reference). Every thread streams the whole tile against its Q register-resident queries;
// four references are read per 128-bit broadcast load.
// ---------------------------------------------------------------------------------------
template <int D, int Q, int KS>
__device__ __forceinline__ void knn_tile(const float* __restrict__ s, int n4, const u64 (&qq)[Q][D],
                                         float (&t)[Q][KS]) {
#pragma unroll 1
    for (int j = 0; j < n4; ++j) {
        ulonglong2 r[D];
        load_refs4<D>(s, j, r);
        knn_step4<D, Q, KS>(qq, r, t);
    }
}

// ---------------------------------------------------------------------------------------
// Pass 2 over one staged tile: grouped maxima a = |dy_t|, b = max |dy-|, x = max |dx-| and
// the three strict counts of Eq. 9: n_z (b < e), n_yz (max(a,b) < e, i.e. a < e and b < e),
// n_xz (max(b,x) < e, i.e. b < e and x < e). Indicators are 1.0f / 0.0f; the products of two
// indicators and the sums stay exact in FP32 (counts < 2^24). The query itself is included
// here (a = b = x = 0) and removed by the caller. Requires DY >= 1 and DX >= 1.
// ---------------------------------------------------------------------------------------
template <int DY, int DX>
__device__ __forceinline__ void count_one(const float (&d)[1 + DY + DX], float e, float& cz, float& cyz,
                                          float& cxz) {
    // a group of one coordinate needs no maximum: compare |d| directly
    float sb, sx;
    if constexpr (DY == 1) sb = abs_set_lt(d[1], e);
    else sb = set_lt(absmax_range<1, DY>(d), e);
    if constexpr (DX == 1) sx = abs_set_lt(d[DY + 1], e);
    else sx = set_lt(absmax_range<DY + 1, DY + DX>(d), e);
    const float sa = abs_set_lt(d[0], e);
    cz += sb;
    cyz = fmaf(sa, sb, cyz);
    cxz = fmaf(sx, sb, cxz);
}

template <int DY, int DX, int Q>
__device__ __forceinline__ void count_tile(const float* __restrict__ s, int n4, const u64 (&qq)[Q][1 + DY + DX],
                                           const float (&e)[Q], float (&cz)[Q], float (&cyz)[Q],
                                           float (&cxz)[Q]) {
    constexpr int D = 1 + DY + DX;
#pragma unroll 1
    for (int j = 0; j < n4; ++j) {
        ulonglong2 r[D];
        load_refs4<D>(s, j, r);
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            float dx[D], dy[D], dz[D], dw[D];
            diff4<D>(qq[q], r, dx, dy, dz, dw);
            count_one<DY, DX>(dx, e[q], cz[q], cyz[q], cxz[q]);
            count_one<DY, DX>(dy, e[q], cz[q], cyz[q], cxz[q]);
            count_one<DY, DX>(dz, e[q], cz[q], cyz[q], cxz[q]);
            count_one<DY, DX>(dw, e[q], cz[q], cyz[q], cxz[q]);
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
