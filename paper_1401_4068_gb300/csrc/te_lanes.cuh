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
// chunks of the window of the largest eps. A group of 4096 points or more is cut into strips by
// a second target coordinate (SortGroup): the sweeps then also skip whole strips whose second-key
// range misses the window.
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

// Source coordinates x_{t-u}, x_{t-u-tau}, ... of one point for the lane's estimate, read from the
// block's member-minor array (LaneXBlock) at xp (the point's column) as packed pairs for
// sub.rn.f32x2 (an odd d repeats its last coordinate: max is unchanged); one 128-byte line per
// coordinate for the warp.
template <int d>
__device__ __forceinline__ void lane_source(const float* __restrict__ xp, int tau32, u64 (&x2)[(d + 1) / 2]) {
    float x[d];
#pragma unroll
    for (int k = 0; k < d; ++k) x[k] = __ldg(xp - k * tau32);
#pragma unroll
    for (int c2 = 0; c2 < (d + 1) / 2; ++c2) x2[c2] = pack2(x[2 * c2], x[2 * c2 + 1 < d ? 2 * c2 + 1 : 2 * c2]);
}

// offset (floats, relative to the lane's column base) of point rw = r << 16 | w in a member-minor
// array of ncols32 = 32 * columns floats per repetition
__device__ __forceinline__ int lane_xoff(uint32_t rw, int ncols32) {
    return (int)(rw >> 16) * ncols32 + (int)(rw & 0xffffu) * 32;
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

// Sorted target part of a lane group (written by lane_stage_kernel), chunk-major: chunk ch (sorted
// positions 32 ch .. 32 ch + 31) holds DA2 = (d + 2) / 2 rows of 32 float2, row c2 the coordinates
// (2 c2, 2 c2 + 1) of the joint point (y_t, y_{t'-1}, y_{t'-1-tau}, ...), the last pair of an even
// d completed with coordinate 1 again; positions past N hold +inf. So a chunk's loads are one
// pointer plus constant offsets, and the key y_{t'-1} of its first and last position are .y of its
// row-0 entries 0 and 31. rw[32 ch + l] = r << 16 | w of the point at sorted position 32 ch + l
// (0 past N), ckey[ch] the key of the chunk's first position (+inf past N).
template <int d>
__device__ __forceinline__ void lane_load(const float2* __restrict__ cp, const int32_t* __restrict__ rwp,
                                          float2 (&r)[(d + 2) / 2], int32_t& rw) {
#pragma unroll
    for (int c2 = 0; c2 < (d + 2) / 2; ++c2) r[c2] = __ldg(cp + c2 * 32);
    rw = __ldg(rwp);
}

template <int d>
__device__ __forceinline__ void lane_diff(const float2 (&r)[(d + 2) / 2], const u64 (&tq)[(d + 2) / 2],
                                          float (&v)[2 * ((d + 2) / 2)]) {
#pragma unroll
    for (int c2 = 0; c2 < (d + 2) / 2; ++c2) split2(sub2(tq[c2], pack2(r[c2].x, r[c2].y)), v[2 * c2], v[2 * c2 + 1]);
}

// Passing references evaluated per round of a lane sweep (their loads in flight together), chosen
// by measurement on GB300: an explicitly written pair (0) from d = 3 on (C3 shapes, d = 3: 42.4 ms
// against 44.6 ms with 4 per round; the Lorenz delay scan, d = 4: 625 ms against 849 ms with a
// generic pair loop; C5 shapes, d = 5: 307.7 ms against 310.3 ms generic and 431 ms with 4), 4 per
// round for d = 2.
template <int d>
__host__ __device__ constexpr int lane_round() { return d <= 2 ? 4 : 0; }

// insertion into the ascending top-KS list without a branch (a value >= t[KS - 1] leaves the
// list unchanged through the min/max network)
template <int KS>
__device__ __forceinline__ void lane_topk_push(float (&t)[KS], float x) {
#pragma unroll
    for (int s = KS - 1; s > 0; --s) t[s] = fmaxf(t[s - 1], fminf(t[s], x));
    t[0] = fminf(t[0], x);
}

// insertion of two values at once: with lo <= hi the pair in order, slot s of the merged list is
// the smallest of t[s], max(lo, t[s - 1]) and max(hi, t[s - 2]) (a min/max network of depth 3)
template <int KS>
__device__ __forceinline__ void lane_topk_push2(float (&t)[KS], float x0, float x1) {
    const float lo = fminf(x0, x1), hi = fmaxf(x0, x1);
    float m[KS];
    m[0] = fminf(t[0], lo);
    if constexpr (KS > 1) m[1] = fminf(fminf(t[1], fmaxf(lo, t[0])), hi);
#pragma unroll
    for (int s = 2; s < KS; ++s) m[s] = fminf(fminf(t[s], fmaxf(lo, t[s - 1])), fmaxf(hi, t[s - 2]));
#pragma unroll
    for (int s = 0; s < KS; ++s) t[s] = m[s];
}

// pass 1: push the joint distances of the references in `ball` (their dT and source offsets xo
// live in the lanes named by the bits) into the lane's top-k list
template <int d, int KS, int RB>
__device__ __forceinline__ void lane_push_refs(unsigned ball, float dT, int xo, const float* __restrict__ xlq, int tau32,
                                               const u64 (&xq)[(d + 1) / 2], float (&t)[KS]) {
    constexpr int P = (d + 1) / 2;
    if constexpr (RB == 0) {
        while (ball) {
            const int j0 = __ffs(ball) - 1;
            ball &= ball - 1;
            const bool two = ball != 0;
            const int j1 = two ? __ffs(ball) - 1 : j0;
            if (two) ball &= ball - 1;
            const float dT0 = __shfl_sync(0xffffffffu, dT, j0);
            const float dT1 = __shfl_sync(0xffffffffu, dT, j1);
            const int xo0 = __shfl_sync(0xffffffffu, xo, j0);
            const int xo1 = __shfl_sync(0xffffffffu, xo, j1);
            u64 x0[P], x1[P];
            lane_source<d>(xlq + xo0, tau32, x0);
            lane_source<d>(xlq + xo1, tau32, x1);
            const float d0 = lane_join<d>(dT0, xq, x0);
            const float d1 = two ? lane_join<d>(dT1, xq, x1) : f_inf();
            lane_topk_push2(t, d0, d1);
        }
    } else {
        while (ball) {
            int jr[RB];
            bool ok[RB];
#pragma unroll
            for (int b = 0; b < RB; ++b) {
                ok[b] = ball != 0;
                jr[b] = ok[b] ? __ffs(ball) - 1 : jr[0];
                ball &= ball - 1;
            }
            u64 xr[RB][P];
            float dr[RB];
#pragma unroll
            for (int b = 0; b < RB; ++b) {
                dr[b] = __shfl_sync(0xffffffffu, dT, jr[b]);
                lane_source<d>(xlq + __shfl_sync(0xffffffffu, xo, jr[b]), tau32, xr[b]);
            }
#pragma unroll
            for (int b = 0; b < RB; ++b)  // a missing reference pushes +inf (no change)
                lane_topk_push(t, ok[b] ? lane_join<d>(dr[b], xq, xr[b]) : f_inf());
        }
    }
}

// pass 2: count the references in `ball` (b = max |dy-| and |dy_t| in the lanes named by the bits)
// against the lane's eps e
template <int d, int RB>
__device__ __forceinline__ void lane_count_refs(unsigned ball, float bv, float ay, int xo, const float* __restrict__ xlq,
                                                int tau32, const u64 (&xq)[(d + 1) / 2], float e, float& cz,
                                                float& cyz, float& cxz) {
    constexpr int P = (d + 1) / 2;
    if constexpr (RB == 0) {
        const float ayz = fmaxf(ay, bv);  // (y_t, y-)
        while (ball) {
            const int j0 = __ffs(ball) - 1;
            ball &= ball - 1;
            const bool two = ball != 0;
            const int j1 = two ? __ffs(ball) - 1 : j0;
            if (two) ball &= ball - 1;
            // a round with one reference left pairs it with +inf (counted nowhere)
            const float b0 = __shfl_sync(0xffffffffu, bv, j0), y0 = __shfl_sync(0xffffffffu, ayz, j0);
            float b1 = __shfl_sync(0xffffffffu, bv, j1), y1 = __shfl_sync(0xffffffffu, ayz, j1);
            if (!two) b1 = y1 = f_inf();
            const int xo0 = __shfl_sync(0xffffffffu, xo, j0);
            const int xo1 = __shfl_sync(0xffffffffu, xo, j1);
            u64 x0[P], x1[P];
            lane_source<d>(xlq + xo0, tau32, x0);
            lane_source<d>(xlq + xo1, tau32, x1);
            const float x0m = lane_join<d>(b0, xq, x0);  // max(b, |dx-|)
            const float x1m = lane_join<d>(b1, xq, x1);
            cz += set_lt(b0, e) + set_lt(b1, e);
            cyz += set_lt(y0, e) + set_lt(y1, e);
            cxz += set_lt(x0m, e) + set_lt(x1m, e);
        }
    } else {
        while (ball) {
            int jr[RB];
            bool ok[RB];
#pragma unroll
            for (int b = 0; b < RB; ++b) {
                ok[b] = ball != 0;
                jr[b] = ok[b] ? __ffs(ball) - 1 : jr[0];
                ball &= ball - 1;
            }
            u64 xr[RB][P];
            float br[RB], yr[RB];
#pragma unroll
            for (int b = 0; b < RB; ++b) {
                // a missing reference gets b = +inf (counted nowhere)
                br[b] = ok[b] ? __shfl_sync(0xffffffffu, bv, jr[b]) : f_inf();
                yr[b] = __shfl_sync(0xffffffffu, ay, jr[b]);
                lane_source<d>(xlq + __shfl_sync(0xffffffffu, xo, jr[b]), tau32, xr[b]);
            }
#pragma unroll
            for (int b = 0; b < RB; ++b) {
                cz += set_lt(br[b], e);
                cyz += set_lt(fmaxf(yr[b], br[b]), e);
                cxz += set_lt(lane_join<d>(br[b], xq, xr[b]), e);  // max(b, |dx-|)
            }
        }
    }
}

template <int d, int KS, int TAU>
__device__ __forceinline__ void lane_query(const BatchArgs& a, const LaneGroup& G, const float* __restrict__ xlq,
                                           int ncols32, bool mv, unsigned nv, int p, FF& acc, float& acc_abs,
                                           const int64_t pt_off) {
    constexpr int DA2 = (d + 2) / 2;  // pairs of target coordinates (1 + d of them)
    constexpr int P = (d + 1) / 2;    // pairs of source coordinates
    constexpr int CH = DA2 * 32;      // float2 per chunk
    const int lane = threadIdx.x & 31;
    const int N = G.N, nch = (G.N + 31) >> 5;
    const int S = G.strips;
    const float2* tpb = a.tpart + G.tp_off;  // uniform base; tpb + lane: this lane's column
    const float2* tpl = tpb + lane;
    const int32_t* rwl = a.lane_rw + G.rw_off + lane;
    // strip tables read through the group descriptor in shared memory where used (no pointers
    // held in registers through the sweeps)
    auto spos = [&](int s) { return __ldg(a.strip_pos + G.strip_off + s); };
    auto sk2 = [&](int i) { return __ldg(a.strip_k2 + 2 * G.strip_off + i); };
    // the embedding delay in floats of the member-minor arrays: a constant for TAU = 1, 2, 3 (the
    // source coordinates of a point are then at immediate offsets), read at run time for TAU = 0
    const int tau32 = TAU > 0 ? TAU * 32 : G.tau * 32;

    // the query (uniform): target coordinates, key and second key; the lane's source part
    const int pc = p >> 5;
    u64 tq[DA2];
#pragma unroll
    for (int c2 = 0; c2 < DA2; ++c2) {
        const float2 q = __ldg(tpb + pc * CH + c2 * 32 + (p & 31));
        tq[c2] = pack2(q.x, q.y);
    }
    float keyq, k2q, tmp;
    split2(tq[0], tmp, keyq);
    split2(tq[1], k2q, tmp);  // coordinate 2, y_{t'-1-tau}: the strips' second key (d >= 2)
    u64 xq[P];
    lane_source<d>(xlq + lane_xoff((uint32_t)__ldg(a.lane_rw + G.rw_off + p), ncols32), tau32, xq);

    // With strips (S > 1; strip s = chunks 32 s .. 32 s + 31, sorted by y_{t'-1} inside, strips in
    // order of the second key): where a key window starts in strip s. Lane l holds the first key
    // of the strip's chunk l; the window starts at the last chunk whose first key is <= lb.
    auto strip_start = [&](int s, float lb, float& fk, int& ce) {
        const int cs = s << 5;
        ce = min(nch, (spos(s + 1) + 31) >> 5);
        fk = cs + lane < ce ? __ldg(a.lane_ckey + G.ck_off + lane + cs) : f_inf();
        return cs + max(0, __popc(__ballot_sync(0xffffffffu, fk <= lb)) - 1);
    };

    pass1_begin(a);
    unsigned vis = 0, pas = 0;  // references visited / passed (both passes)
    float t[KS];
#pragma unroll
    for (int s = 0; s < KS; ++s) t[s] = f_inf();
    float thr = f_inf();
    // one chunk (a reference per lane; its data r, rw already loaded): the target-part distance dT,
    // then every reference with dT < thr for all lanes
    auto scan1 = [&](const float2 (&r)[DA2], int32_t rwv, int ch) {
        float v[2 * DA2];
        lane_diff<d>(r, tq, v);
        const float dT = absmax_range<0, 2 * DA2 - 1>(v);
        unsigned ball = __ballot_sync(0xffffffffu, dT < thr);
        vis += min(32, N - (ch << 5));
        if (ball) {
            const int xo = lane_xoff((uint32_t)rwv, ncols32);
            pas += __popc(ball);
            lane_push_refs<d, KS, lane_round<d>()>(ball, dT, xo, xlq, tau32, xq, t);
            thr = lanes_max(mv ? t[KS - 1] : 0.0f);  // the lists change only here
        }
    };
    // The sweeps load chunk ch + 1 (or ch - 1) before processing chunk ch, so its latency overlaps
    // the work on ch; the window test reads the key of a chunk's first (right) or last (left)
    // position from its loaded row 0. A prefetched chunk past the window is not used.
    float2 cur[DA2], nxt[DA2];
    int32_t rwc, rwn;
    // own strip (the whole group without strips): outward from the query's chunk
    int cs0 = 0, ce0 = nch;
    if (S > 1) {
        cs0 = pc & ~31;
        ce0 = min(nch, (spos((pc >> 5) + 1) + 31) >> 5);
    }
    int chl = pc, chr = pc;
    lane_load<d>(tpl + pc * CH, rwl + (pc << 5), cur, rwc);
    if (pc + 1 < ce0) lane_load<d>(tpl + (pc + 1) * CH, rwl + ((pc + 1) << 5), nxt, rwn);
    scan1(cur, rwc, pc);
    for (int ch = pc + 1; ch < ce0; ++ch) {  // right: stop at the first chunk starting outside
#pragma unroll
        for (int c2 = 0; c2 < DA2; ++c2) cur[c2] = nxt[c2];
        rwc = rwn;
        if (!(__shfl_sync(0xffffffffu, cur[0].y, 0) < __fadd_ru(keyq, thr))) break;
        if (ch + 1 < ce0) lane_load<d>(tpl + (ch + 1) * CH, rwl + ((ch + 1) << 5), nxt, rwn);
        scan1(cur, rwc, ch);
        chr = ch;
    }
    if (pc > cs0) lane_load<d>(tpl + (pc - 1) * CH, rwl + ((pc - 1) << 5), nxt, rwn);
    for (int ch = pc - 1; ch >= cs0; --ch) {  // left: stop at the first chunk ending outside
#pragma unroll
        for (int c2 = 0; c2 < DA2; ++c2) cur[c2] = nxt[c2];
        rwc = rwn;
        if (!(__shfl_sync(0xffffffffu, cur[0].y, 31) > __fsub_rd(keyq, thr))) break;
        if (ch > cs0) lane_load<d>(tpl + (ch - 1) * CH, rwl + ((ch - 1) << 5), nxt, rwn);
        scan1(cur, rwc, ch);
        chl = ch;
    }
    // the other strips nearest first in the second key, while their second-key range meets the
    // window; in each, the chunks of the key window (both keys are coordinates of y-, so a
    // reference outside either window has dT >= thr and could not enter any list)
    if (S > 1) {
        const int s0 = pc >> 5;
        bool up = s0 + 1 < S, down = s0 > 0;
        for (int step = 1; up || down; ++step) {
#pragma unroll
            for (int side = 0; side < 2; ++side) {
                const int s = side == 0 ? s0 + step : s0 - step;
                if (side == 0 ? (!up || s >= S) : (!down || s < 0)) {
                    if (side == 0) up = false;
                    else down = false;
                    continue;
                }
                if (side == 0 && !(sk2(2 * s) < __fadd_ru(k2q, thr))) {
                    up = false;
                    continue;
                }
                if (side == 1 && !(sk2(2 * s + 1) > __fsub_rd(k2q, thr))) {
                    down = false;
                    continue;
                }
                float fk;
                int ce;
                const int c0 = strip_start(s, __fsub_rd(keyq, thr), fk, ce);
                lane_load<d>(tpl + c0 * CH, rwl + (c0 << 5), nxt, rwn);
                for (int ch = c0; ch < ce; ++ch) {
#pragma unroll
                    for (int c2 = 0; c2 < DA2; ++c2) cur[c2] = nxt[c2];
                    rwc = rwn;
                    if (!(__shfl_sync(0xffffffffu, fk, ch - (s << 5)) < __fadd_ru(keyq, thr))) break;
                    if (ch + 1 < ce) lane_load<d>(tpl + (ch + 1) * CH, rwl + ((ch + 1) << 5), nxt, rwn);
                    scan1(cur, rwc, ch);
                }
            }
        }
    }
    const float e = topk_select(t, a.k);
    const float emax = lanes_max(mv ? e : 0.0f);
    pass1_end(a, (unsigned long long)vis * nv);

    // ---- pass 2: the chunks of the window of the largest eps (without strips inside those pass 1
    // visited; with strips, in every strip whose second-key range meets the window)
    const float lb = __fsub_rd(keyq, emax), rb = __fadd_ru(keyq, emax);
    float cz = 0.0f, cyz = 0.0f, cxz = 0.0f;
    auto scan2 = [&](const float2 (&r)[DA2], int32_t rwv, int ch) {
        float v[2 * DA2];
        lane_diff<d>(r, tq, v);
        const float bv = absmax_range<1, 2 * DA2 - 1>(v);  // y- (and the repeated coordinate 1)
        const float ayz = fabsf(v[0]);                     // y_t (joined with b per reference)
        unsigned ball = __ballot_sync(0xffffffffu, bv < emax);
        vis += min(32, N - (ch << 5));
        if (ball) {
            const int xo = lane_xoff((uint32_t)rwv, ncols32);
            pas += __popc(ball);
            lane_count_refs<d, lane_round<d>()>(ball, bv, ayz, xo, xlq, tau32, xq, e, cz, cyz, cxz);
        }
    };
    if (S > 1) {
        const float lb2 = __fsub_rd(k2q, emax), rb2 = __fadd_ru(k2q, emax);
        for (int s = 0; s < S; ++s) {
            if (!(sk2(2 * s + 1) > lb2)) continue;  // strip entirely below the window
            if (!(sk2(2 * s) < rb2)) break;         // this and every later strip above it
            float fk;
            int ce;
            const int c0 = strip_start(s, lb, fk, ce);
            lane_load<d>(tpl + c0 * CH, rwl + (c0 << 5), nxt, rwn);
            for (int ch = c0; ch < ce; ++ch) {
#pragma unroll
                for (int c2 = 0; c2 < DA2; ++c2) cur[c2] = nxt[c2];
                rwc = rwn;
                if (!(__shfl_sync(0xffffffffu, fk, ch - (s << 5)) < rb)) break;
                if (ch + 1 < ce) lane_load<d>(tpl + (ch + 1) * CH, rwl + ((ch + 1) << 5), nxt, rwn);
                scan2(cur, rwc, ch);
            }
        }
    } else {
        lane_load<d>(tpl + chl * CH, rwl + (chl << 5), nxt, rwn);
        for (int ch = chl; ch <= chr; ++ch) {
#pragma unroll
            for (int c2 = 0; c2 < DA2; ++c2) cur[c2] = nxt[c2];
            rwc = rwn;
            if (!(__shfl_sync(0xffffffffu, cur[0].y, 0) < rb)) break;
            if (ch < chr) lane_load<d>(tpl + (ch + 1) * CH, rwl + ((ch + 1) << 5), nxt, rwn);
            if (!(__shfl_sync(0xffffffffu, cur[0].y, 31) > lb)) continue;  // padding (+inf) never skips
            scan2(cur, rwc, ch);
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
        const unsigned long long pairs = (unsigned long long)vis * nv;
        const unsigned long long alg = pairs * 2ull * D;
        const unsigned long long run = (unsigned long long)vis * 2ull * (1 + d) + (unsigned long long)pas * nv * 2ull * d;
        work_add(0, pairs);
        work_add(1, alg);
        work_add(2, alg > run ? alg - run : 0ull);
    }
}

// The lane kernel: persistent CTAs of kLaneThreads take work items (group, block of 32 estimates,
// block of kLaneQB sorted query positions) from the queue; warp w takes positions q0 + w, q0 + w
// + kLaneWarps, ... (a fixed assignment, so the partial sums are deterministic), and the CTA adds
// its warps' per-lane sums in warp order into one partial per estimate and query block.
template <int d, int KS, int TAU>
__global__ void __launch_bounds__(kLaneThreads, d <= 5 ? 4 : 3) lane_kernel(const BatchArgs a) {
    __shared__ double s_v[kLaneWarps][32], s_w[kLaneWarps][32];
    __shared__ int s_item;
    __shared__ LaneGroup s_group;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    work_reset();
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = atomicAdd(a.queue, 1);
        __syncthreads();
        const int ticket = s_item;
        if (ticket >= a.n_items) break;
        const LaneItem it = a.litems[a.item_base + ticket];
        // the item's group descriptor stays in shared memory (read where used, not held in
        // registers through the sweeps)
        if (threadIdx.x == 0) s_group = a.lgroups[it.group];
        __syncthreads();
        const LaneGroup& G = s_group;
        const int mi = it.mblock * 32 + lane;
        const bool mv = mi < G.n_mem;
        const InstDesc& J = a.insts[__ldg(a.lane_members + G.mem_off + min(mi, G.n_mem - 1))];
        const LaneXBlock& XB = a.lane_xb[it.xblk];
        // this lane's column base: the sample x_{t-u} of a point at window offset w is column
        // t_start - u - t0 + w of repetition r (lane_xoff)
        const float* xlq = a.lane_x + XB.off + lane + (size_t)(G.t_start - J.u - XB.t0) * 32;
        const int ncols32 = XB.ncols * 32;
        const int64_t pt_off = J.pt_off;
        const unsigned nv = (unsigned)min(32, G.n_mem - it.mblock * 32);
        FF acc{0.0f, 0.0f};
        float acc_abs = 0.0f;
        const int qend = min(it.q0 + kLaneQB, G.N);
        for (int p = it.q0 + warp; p < qend; p += kLaneWarps)
            lane_query<d, KS, TAU>(a, G, xlq, ncols32, mv, nv, p, acc, acc_abs, pt_off);
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

// The instantiation for embedding dimension d, k <= 4 (ks = 5) and delay class tc (1, 2, 3: that
// tau compiled in; 0: any tau read at run time).
template <int d>
const void* lane_kernel_select(int ks, int tc) {
    if (ks != 5) return nullptr;
    switch (tc) {
        case 1: return (const void*)lane_kernel<d, 5, 1>;
        case 2: return (const void*)lane_kernel<d, 5, 2>;
        case 3: return (const void*)lane_kernel<d, 5, 3>;
        default: return (const void*)lane_kernel<d, 5, 0>;
    }
}

}  // namespace te
