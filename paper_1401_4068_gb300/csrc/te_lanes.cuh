// One estimate per lane: the estimates of one (target series, repetitions, window start, window,
// d, tau) group share every target coordinate of their joint points (y_t and y- of Eq. 6 /
// Eq. 10) and differ only in the source part x-: a trial-shuffled surrogate (Fig. 3) pairs
// target repetition r with another source repetition, a scanned delay (Eq. 5) takes the source
// at another t-u. Here a warp takes ONE query point and 32 such estimates, one per lane: the
// target part of every (query, reference) distance is the same in all lanes, so it is computed
// once per reference (32 references per warp instruction, one per lane) and the decision to skip
// a reference is warp-uniform:
//   pass 1: dT = max |dy_t|, |dy-| of a reference is a lower bound of its joint distance in every
//           estimate; with thr = the largest current (k+1)-th smallest distance over the 32
//           lanes, a reference with dT >= thr cannot enter any lane's top-k list and is skipped
//           before any source coordinate is read;
//   pass 2: b = max |dy-| bounds all three counts of Eq. 9 from below (n_z: b < eps, n_yz:
//           max(|dy_t|, b) < eps, n_xz: max(b, |dx-|) < eps), so a reference with b >= the
//           largest eps over the lanes is skipped.
// Only the references that pass are evaluated per lane: their source coordinates are gathered
// from the lane's own source row (the permutation of the lane's estimate) and joined with the
// shared dT or b. Every lane sees exactly the FP32 differences of the unshared search (max is
// exact), so eps and the counts are identical to it and to the brute-force definition.
//
// References are visited in the group's sorted order (key y_{t'-1}, see te_sweep.cuh): the
// query's own 32-position chunk first, then chunks to the right and to the left while their keys
// lie inside the window (key_q - thr, key_q + thr) with bounds rounded outward; pass 2 visits the
// chunks of the window of the largest eps, a subset of those pass 1 visited.
#pragma once

#include "te_sweep.cuh"

namespace te {

// max over lanes of a non-negative float (or +inf): the order of non-negative IEEE floats is the
// order of their bit patterns as unsigned integers
__device__ __forceinline__ float lanes_max(float v) {
    return __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(v)));
}

__device__ __forceinline__ u64 pack2(float lo, float hi) {
    u64 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}

// Source coordinates x_{t-u}, x_{t-u-tau}, ... of point (r, t) for the lane's estimate (delay u),
// read from the block's member-minor array (LaneXBlock) as packed pairs for sub.rn.f32x2 (an odd d
// repeats its last coordinate: max is unchanged); one 128-byte line per coordinate for the warp.
template <int d>
__device__ __forceinline__ void lane_source(const float* __restrict__ xl, int ncols, int tau32, int r, int c,
                                            u64 (&x2)[(d + 1) / 2]) {
    const float* xp = xl + ((size_t)r * ncols + c) * 32;
    float x[d];
#pragma unroll
    for (int k = 0; k < d; ++k) x[k] = __ldg(xp - k * tau32);
#pragma unroll
    for (int c2 = 0; c2 < (d + 1) / 2; ++c2) x2[c2] = pack2(x[2 * c2], x[2 * c2 + 1 < d ? 2 * c2 + 1 : 2 * c2]);
}

// max(a, |q_c - x_c| over the d source coordinates), a >= 0
template <int d>
__device__ __forceinline__ float lane_join(float a, const u64 (&q2)[(d + 1) / 2], const u64 (&x2)[(d + 1) / 2]) {
    constexpr int P = (d + 1) / 2;
    float v[2 * P + 1];
    v[0] = a;
#pragma unroll
    for (int c2 = 0; c2 < P; ++c2) split2(sub2(q2[c2], x2[c2]), v[1 + 2 * c2], v[2 + 2 * c2]);
    return absmax_range<0, 2 * P>(v);
}

// Sorted target part of a lane group's points (written by lane_stage_kernel): DA2 rows of NP
// float2, row c2 holding coordinates (2 c2, 2 c2 + 1) of the joint point (y_t, y_{t'-1},
// y_{t'-1-tau}, ...), the last pair of an even d completed with coordinate 1 again; positions N ..
// NP-1 hold +inf. rw[p] = r << 16 | w of the point at sorted position p (N <= 65536, so r, w <
// 65536).
template <int d>
__device__ __forceinline__ void lane_target(const float2* __restrict__ tp, int NP, int j, u64 (&r2)[(d + 2) / 2]) {
#pragma unroll
    for (int c2 = 0; c2 < (d + 2) / 2; ++c2) {
        const float2 v = __ldg(tp + (size_t)c2 * NP + j);
        r2[c2] = pack2(v.x, v.y);
    }
}

template <int d, int KS>
__device__ __forceinline__ void lane_query(const BatchArgs& a, const LaneGroup& G, const float* __restrict__ xl,
                                           int ncols, int cu, bool mv, unsigned nv, int p, FF& acc, float& acc_abs,
                                           const int64_t pt_off) {
    constexpr int DA2 = (d + 2) / 2;  // pairs of target coordinates (1 + d of them)
    constexpr int P = (d + 1) / 2;    // pairs of source coordinates
    const int lane = threadIdx.x & 31;
    const int N = G.N, NP = (G.N + 31) & ~31;
    const float2* tp = a.tpart + G.tp_off;
    const int32_t* rwp = a.lane_rw + G.sort_off;
    const float* skey = a.sorted_key + G.sort_off;

    // the query (uniform): target coordinates, its repetition and sample; the lane's source part
    u64 tq[DA2];
    lane_target<d>(tp, NP, p, tq);
    const uint32_t rwq = (uint32_t)__ldg(rwp + p);
    // column of the source sample x_{t-u} of a point at window offset w: cu + w (cu = t_start - u - t0)
    const int tau32 = G.tau * 32;
    u64 xq[P];
    lane_source<d>(xl, ncols, tau32, (int)(rwq >> 16), cu + (int)(rwq & 0xffffu), xq);
    float keyq, tmp;
    split2(tq[0], tmp, keyq);

    pass1_begin(a);
    unsigned long long visited = 0, passed = 0;
    float t[KS];
#pragma unroll
    for (int s = 0; s < KS; ++s) t[s] = f_inf();
    float thr = f_inf();
    const int cb = p & ~31;
    int cl = cb, cr = cb;
    // one chunk of 32 sorted positions (one reference per lane)
    auto chunk1 = [&](int c) {
        const int j = c + lane;
        u64 r2[DA2];
        lane_target<d>(tp, NP, j, r2);
        float v[2 * DA2];
#pragma unroll
        for (int c2 = 0; c2 < DA2; ++c2) split2(sub2(tq[c2], r2[c2]), v[2 * c2], v[2 * c2 + 1]);
        const float dT = absmax_range<0, 2 * DA2 - 1>(v);
        unsigned ball = __ballot_sync(0xffffffffu, dT < thr);
        visited += (unsigned long long)min(32, N - c);
        if (ball) {
            const int rw = __ldg(rwp + min(j, N - 1));
            passed += __popc(ball);
            while (ball) {  // two passing references per round for independent loads
                const int j0 = __ffs(ball) - 1;
                ball &= ball - 1;
                const bool two = ball != 0;
                const int j1 = two ? __ffs(ball) - 1 : j0;
                if (two) ball &= ball - 1;
                const float dT0 = __shfl_sync(0xffffffffu, dT, j0);
                const float dT1 = __shfl_sync(0xffffffffu, dT, j1);
                const uint32_t rw0 = (uint32_t)__shfl_sync(0xffffffffu, rw, j0);
                const uint32_t rw1 = (uint32_t)__shfl_sync(0xffffffffu, rw, j1);
                u64 x0[P], x1[P];
                lane_source<d>(xl, ncols, tau32, (int)(rw0 >> 16), cu + (int)(rw0 & 0xffffu), x0);
                lane_source<d>(xl, ncols, tau32, (int)(rw1 >> 16), cu + (int)(rw1 & 0xffffu), x1);
                const float d0 = lane_join<d>(dT0, xq, x0);
                const float d1 = two ? lane_join<d>(dT1, xq, x1) : f_inf();
                topk_push(t, d0);
                topk_push(t, d1);
            }
        }
        thr = lanes_max(mv ? t[KS - 1] : 0.0f);
    };
    chunk1(cb);
    for (int c = cb + 32; c < N; c += 32) {  // right
        if (!(__ldg(skey + c) < __fadd_ru(keyq, thr))) break;
        chunk1(c);
        cr = c;
    }
    for (int c = cb - 32; c >= 0; c -= 32) {  // left
        if (!(__ldg(skey + c + 31) > __fsub_rd(keyq, thr))) break;
        chunk1(c);
        cl = c;
    }
    const float e = topk_select(t, a.k);
    const float emax = lanes_max(mv ? e : 0.0f);
    pass1_end(a, visited * nv);
    const unsigned long long visited1 = visited, passed1 = passed;
    visited = passed = 0;

    // ---- pass 2: chunks of the window of the largest eps
    const float lb = __fsub_rd(keyq, emax), rb = __fadd_ru(keyq, emax);
    float cz = 0.0f, cyz = 0.0f, cxz = 0.0f;
    for (int c = cl; c <= cr; c += 32) {
        if (!(__ldg(skey + min(c + 31, N - 1)) > lb)) continue;
        if (!(__ldg(skey + c) < rb)) break;
        const int j = c + lane;
        u64 r2[DA2];
        lane_target<d>(tp, NP, j, r2);
        float v[2 * DA2];
#pragma unroll
        for (int c2 = 0; c2 < DA2; ++c2) split2(sub2(tq[c2], r2[c2]), v[2 * c2], v[2 * c2 + 1]);
        const float b = absmax_range<1, 2 * DA2 - 1>(v);   // y- (and the repeated coordinate 1)
        const float ayz = fmaxf(fabsf(v[0]), b);           // (y_t, y-)
        unsigned ball = __ballot_sync(0xffffffffu, b < emax);
        visited += (unsigned long long)min(32, N - c);
        if (ball) {
            const int rw = __ldg(rwp + min(j, N - 1));
            passed += __popc(ball);
            while (ball) {
                const int j0 = __ffs(ball) - 1;
                ball &= ball - 1;
                const bool two = ball != 0;
                const int j1 = two ? __ffs(ball) - 1 : j0;
                if (two) ball &= ball - 1;
                // a round with one reference left pairs it with +inf (counted nowhere)
                const float b0 = __shfl_sync(0xffffffffu, b, j0), y0 = __shfl_sync(0xffffffffu, ayz, j0);
                float b1 = __shfl_sync(0xffffffffu, b, j1), y1 = __shfl_sync(0xffffffffu, ayz, j1);
                if (!two) b1 = y1 = f_inf();
                const uint32_t rw0 = (uint32_t)__shfl_sync(0xffffffffu, rw, j0);
                const uint32_t rw1 = (uint32_t)__shfl_sync(0xffffffffu, rw, j1);
                u64 x0[P], x1[P];
                lane_source<d>(xl, ncols, tau32, (int)(rw0 >> 16), cu + (int)(rw0 & 0xffffu), x0);
                lane_source<d>(xl, ncols, tau32, (int)(rw1 >> 16), cu + (int)(rw1 & 0xffffu), x1);
                const float x0m = lane_join<d>(b0, xq, x0);  // max(b, |dx-|)
                const float x1m = lane_join<d>(b1, xq, x1);
                cz += set_lt(b0, e) + set_lt(b1, e);
                cyz += set_lt(y0, e) + set_lt(y1, e);
                cxz += set_lt(x0m, e) + set_lt(x1m, e);
            }
        }
    }
    pass2_end(a);

    // ---- digamma terms of Eq. 9 for the lane's estimate (compensated FP32); the query itself was
    // counted (all its differences are 0 < eps) when eps > 0
    const int self = e > 0.0f ? 1 : 0;
    const int nz = (int)cz - self, nyz = (int)cyz - self, nxz = (int)cxz - self;
    if (mv) {
        const int i = __ldg(a.sorted_idx + G.sort_off + p);
        if (a.counts_out) {
            int32_t* co = a.counts_out + 3 * pt_off;
            co[i] = nz;
            co[N + i] = nyz;
            co[2 * N + i] = nxz;
        }
        if (a.eps_out) a.eps_out[pt_off + i] = e;
        const float2 p1 = __ldg(a.psi + nz + 1);
        const float2 p2 = __ldg(a.psi + nyz + 1);
        const float2 p3 = __ldg(a.psi + nxz + 1);
        acc = ff_add(acc, p1.x, p1.y);
        acc = ff_add(acc, -p2.x, -p2.y);
        acc = ff_add(acc, -p3.x, -p3.y);
        acc_abs += fabsf(p1.x) + fabsf(p2.x) + fabsf(p3.x);
    }
    if (a.exec && lane == 0) {
        // pairs decided per estimate (every visited reference, for each valid lane), their 2 D
        // algorithmic operations, and the operations not executed: the target part (2 (1 + d)
        // ops) runs once per reference for all lanes, the source part (2 d) only for references
        // that passed the shared test
        constexpr int D = 1 + 2 * d;
        const unsigned long long pairs = (visited1 + visited) * nv;
        const unsigned long long alg = pairs * 2ull * D;
        const unsigned long long run = (visited1 + visited) * 2ull * (1 + d) + (passed1 + passed) * nv * 2ull * d;
        work_add(0, pairs);
        work_add(1, alg);
        work_add(2, alg > run ? alg - run : 0ull);
    }
}

// The lane kernel: persistent CTAs of kLaneThreads take work items (group, block of 32 estimates,
// block of kLaneQB sorted query positions) from the queue; warp w takes positions q0 + w, q0 + w
// + kLaneWarps, ... (a fixed assignment, so the partial sums are deterministic), and the CTA adds
// its warps' per-lane sums in warp order into one partial per estimate and query block.
template <int d, int KS>
__global__ void __launch_bounds__(kLaneThreads, d <= 5 ? 4 : 3) lane_kernel(const BatchArgs a) {
    __shared__ double s_v[kLaneWarps][32], s_w[kLaneWarps][32];
    __shared__ int s_item;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    work_reset();
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = atomicAdd(a.queue, 1);
        __syncthreads();
        const int ticket = s_item;
        if (ticket >= a.n_items) break;
        const LaneItem it = a.litems[a.item_base + ticket];
        const LaneGroup G = a.lgroups[it.group];
        const int mi = it.mblock * 32 + lane;
        const bool mv = mi < G.n_mem;
        const InstDesc& J = a.insts[__ldg(a.lane_members + G.mem_off + min(mi, G.n_mem - 1))];
        const LaneXBlock& XB = a.lane_xb[it.xblk];
        const int ncols = XB.ncols;
        const float* xl = a.lane_x + XB.off + lane;
        const int cu = G.t_start - J.u - XB.t0;
        const int64_t pt_off = J.pt_off;
        const unsigned nv = (unsigned)min(32, G.n_mem - it.mblock * 32);
        FF acc{0.0f, 0.0f};
        float acc_abs = 0.0f;
        const int qend = min(it.q0 + kLaneQB, G.N);
        for (int p = it.q0 + warp; p < qend; p += kLaneWarps)
            lane_query<d, KS>(a, G, xl, ncols, cu, mv, nv, p, acc, acc_abs, pt_off);
        s_v[warp][lane] = (double)acc.hi + (double)acc.lo;
        s_w[warp][lane] = (double)acc_abs;
        __syncthreads();
        if (warp == 0 && mv) {
            double v = 0.0, w = 0.0;
#pragma unroll
            for (int k = 0; k < kLaneWarps; ++k) {
                v += s_v[k][lane];
                w += s_w[k][lane];
            }
            const int qb = it.q0 / kLaneQB;
            a.partial[J.part_begin + qb] = v;
            a.partial_abs[J.part_begin + qb] = w;
        }
    }
    work_flush(a);
}

}  // namespace te
