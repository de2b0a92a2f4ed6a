// Sweep mode of the batched kernel: the same exact estimator as process_item (Eq. 9 / Eq. 10),
// with the reference points of an instance visited in the order of their target coordinate
// y_{t'-1} (coordinate 1, a coordinate of the y- group) so that references that cannot matter
// are never evaluated.
//
// Why it is exact: for a query q with current radius r (its (k+1)-th smallest distance so far in
// pass 1, its final eps in pass 2) and a reference j, every distance the estimator uses to decide
// (the joint distance of pass 1, b = max over y- of pass 2, and hence max(a, b) and max(b, x))
// is at least fl(|key_q - key_j|). With bounds rounded outward,
//   key_j <= fsub_rd(key_q, r)  or  key_j >= fadd_ru(key_q, r)   =>   fl(|key_q - key_j|) >= r,
// so such a reference can neither enter the top-k list (strict < r) nor be counted (strict < eps).
// Queries of a warp are a contiguous block of the sorted order; a warp first evaluates its own
// block (tight radii early), then sweeps right and left and stops on each side at the first
// group of four references entirely outside its window. Radii only shrink during pass 1, so a
// window computed earlier is a superset of the current one.
#pragma once

#include "te_batched.cuh"

namespace te {

__device__ __forceinline__ float warp_min(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// CTA-wide min of a and max of b (every thread gets both); sb: 64 floats of shared memory
// Work counters of the sweep, per warp in shared memory (lane 0 only): [0] (query, reference)
// pair evaluations, [1] their 2 D FP32 operations, [2] operations target-part sharing saved,
// [3] pass-1 pair evaluations, [4] the warp's cycles in pass 1, [5] its cycles in pass 2 (digamma
// terms included). A pass's cycles are added as -clock64() at its start and clock64() at its end
// (sums exact modulo 2^64, so no register stays live across a pass). The persistent kernels add
// the slots to BatchArgs::exec once, when the CTA leaves its work loop, so a warp block costs no
// global atomics.
__device__ __forceinline__ unsigned long long* work_slot() {
    __shared__ unsigned long long s_work[32][6];
    return s_work[threadIdx.x >> 5];
}
__device__ __forceinline__ void work_add(int i, unsigned long long v) { work_slot()[i] += v; }
__device__ __forceinline__ void work_reset() {
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int i = 0; i < 6; ++i) work_slot()[i] = 0;
}
__device__ __forceinline__ void work_flush(const BatchArgs& a) {
    if (a.exec && (threadIdx.x & 31) == 0) {
        const unsigned long long* w = work_slot();
#pragma unroll
        for (int i = 0; i < 6; ++i)
            if (w[i]) atomicAdd(a.exec + i, w[i]);
    }
}
__device__ __forceinline__ void pass1_begin(const BatchArgs& a) {
    if (a.exec && (threadIdx.x & 31) == 0) work_add(4, 0ull - (unsigned long long)clock64());
}
__device__ __forceinline__ void pass1_end(const BatchArgs& a, unsigned long long pairs1) {
    if (a.exec && (threadIdx.x & 31) == 0) {
        const unsigned long long c = (unsigned long long)clock64();
        work_add(4, c);
        work_add(5, 0ull - c);
        work_add(3, pairs1);
    }
}
__device__ __forceinline__ void pass2_end(const BatchArgs& a) {
    if (a.exec && (threadIdx.x & 31) == 0) work_add(5, (unsigned long long)clock64());
}

__device__ __forceinline__ void block_minmax(float& a, float& b, float* sb) {
    a = warp_min(a);
    b = warp_max(b);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) {
        sb[warp] = a;
        sb[32 + warp] = b;
    }
    __syncthreads();
    a = sb[0];
    b = sb[32];
    for (int w = 1; w < nw; ++w) {
        a = fminf(a, sb[w]);
        b = fmaxf(b, sb[32 + w]);
    }
}

template <int d>
__device__ __forceinline__ void stage_tile_sorted(const InstDesc& I, const int32_t* __restrict__ sidx, int base,
                                                  int nv, float* sm, int32_t* flags) {
    constexpr int D = 1 + 2 * d;
    const int nfill = (nv + 3) & ~3;
    for (int p = threadIdx.x; p < nfill; p += blockDim.x) {
        float v[D];
        const int i = p < nv ? __ldg(sidx + base + p) : -1;  // -1: strip padding
        if (i >= 0) {
            gather_point<d>(I, i, v, flags);
        } else {
#pragma unroll
            for (int c = 0; c < D; ++c) v[c] = f_inf();
        }
#pragma unroll
        for (int c = 0; c < D; ++c) sm[tile_index<D>(c, p)] = v[c];
    }
}

// window of the warp around its queries' keys for radii r (outward rounded, invalid slots ignored)
template <int Q>
__device__ __forceinline__ void warp_window(const float (&qkey)[Q], const bool (&qv)[Q], const float (&r)[Q],
                                            float& lb, float& rb) {
    lb = f_inf();
    rb = -f_inf();
#pragma unroll
    for (int q = 0; q < Q; ++q)
        if (qv[q]) {
            lb = fminf(lb, __fsub_rd(qkey[q], r[q]));
            rb = fmaxf(rb, __fadd_ru(qkey[q], r[q]));
        }
    lb = warp_min(lb);
    rb = warp_max(rb);
}

template <int Q, int KS>
__device__ __forceinline__ void current_radii(const float (&t)[Q][KS], float (&r)[Q]) {
#pragma unroll
    for (int q = 0; q < Q; ++q) r[q] = t[q][KS - 1];
}

// one group of four references (group j of the staged tile) against the warp's queries, pass 1
template <int D, int Q, int KS>
__device__ __forceinline__ void knn_group(const float* __restrict__ s, int j, const u64 (&qq)[Q][D],
                                          float (&t)[Q][KS]) {
    ulonglong2 r[D];
    load_refs4<D>(s, j, r);
    knn_step4<D, Q, KS>(qq, r, t);
}

// pass 1 over groups [g0, g1) of the staged tile: dir 0 evaluates all of them (the warp's own
// block), dir +1 ascends and stops at the first group whose smallest key is right of the
// window, dir -1 descends and stops at the first group whose largest key is left of it.
// Returns the number of groups evaluated; sets `done` when it stopped at a window edge.
template <int D, int Q, int KS>
__device__ __forceinline__ int knn_range(const float* __restrict__ s, int g0, int g1, int dir,
                                         const u64 (&qq)[Q][D], const float (&qkey)[Q], const bool (&qv)[Q],
                                         float (&t)[Q][KS], bool& done) {
    float r[Q], lb, rb;
    current_radii(t, r);
    warp_window(qkey, qv, r, lb, rb);
    int n = 0;
#pragma unroll 1
    for (int jj = g0; jj < g1; ++jj) {
        const int j = dir < 0 ? g1 - 1 - (jj - g0) : jj;
        if (dir > 0 && group_key_lo<D>(s, j) >= rb) {
            done = true;
            break;
        }
        if (dir < 0 && group_key_hi<D>(s, j) <= lb) {
            done = true;
            break;
        }
        knn_group<D, Q, KS>(s, j, qq, t);
        if ((++n & 3) == 0 && dir != 0) {
            current_radii(t, r);
            warp_window(qkey, qv, r, lb, rb);
        }
    }
    return n;
}

// pass 2 over groups [g0, g1) ascending, skipping groups left of the window [lb, rb] and
// stopping at the first group right of it
template <int DY, int DX, int Q>
__device__ __forceinline__ int count_range(const float* __restrict__ s, int g0, int g1, float lb, float rb,
                                           const u64 (&qq)[Q][1 + DY + DX], const float (&e)[Q], float (&cz)[Q],
                                           float (&cyz)[Q], float (&cxz)[Q]) {
    constexpr int D = 1 + DY + DX;
    int n = 0;
#pragma unroll 1
    for (int j = g0; j < g1; ++j) {
        if (group_key_lo<D>(s, j) >= rb) break;
        if (group_key_hi<D>(s, j) <= lb) continue;
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
        ++n;
    }
    return n;
}

// first sorted position whose key is > x (keys ascending, n of them)
__device__ __forceinline__ int first_greater(const float* __restrict__ key, int n, float x) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(key + mid) > x) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}
// first sorted position whose key is >= x
__device__ __forceinline__ int first_not_less(const float* __restrict__ key, int n, float x) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(key + mid) >= x) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

template <int d, int Q, int KS>
__device__ __forceinline__ void process_item_sweep(const BatchArgs& a, const InstDesc& I, int q0, int it, float* sm,
                                                   double* sred, float* sb) {
    pass1_begin(a);
    constexpr int D = 1 + 2 * d;
    const int N = I.N;
    const int T = blockDim.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int32_t* sidx = a.sorted_idx + I.sort_off;
    const float* skey = a.sorted_key + I.sort_off;
    // one tile when the instance fits, else tiles of whole CTA query blocks (a CTA's queries then
    // lie in one tile)
    const int block = T * Q;
    int ldt = (N + 3) & ~3;
    if (ldt * D > a.smem_floats) ldt = ((a.smem_floats / D) / block) * block;
    const int ntile = (N + ldt - 1) / ldt;
    const int ctile = q0 / ldt;

    // queries: warp-contiguous runs of the sorted order
    const int wbase = q0 + warp * 32 * Q;
    u64 qq[Q][D];
    float qkey[Q];
    int qidx[Q];
    bool qv[Q];
    int nvalid = 0;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int pos = wbase + q * 32 + lane;
        qv[q] = pos < N;
        float p[D];
        if (qv[q]) {
            qidx[q] = __ldg(sidx + pos);
            gather_point<d>(I, qidx[q], p, a.flags);
        } else {
            qidx[q] = -1;
#pragma unroll
            for (int c = 0; c < D; ++c) p[c] = 0.0f;
        }
        qkey[q] = p[1];
#pragma unroll
        for (int c = 0; c < D; ++c) qq[q][c] = dup2(p[c]);
        nvalid += __popc(__ballot_sync(0xffffffffu, qv[q]));
    }
    const bool warp_active = wbase < N;
    unsigned long long groups_done = 0;

    int staged = -1;
    auto stage = [&](int ti) {
        if (staged == ti) return;
        const int base = ti * ldt;
        __syncthreads();
        stage_tile_sorted<d>(I, sidx, base, min(ldt, N - base), sm, a.flags);
        __syncthreads();
        staged = ti;
    };
    auto ngroups = [&](int ti) { return (min(ldt, N - ti * ldt) + 3) >> 2; };

    // ---- pass 1: own block, then right, then left
    float t[Q][KS];
#pragma unroll
    for (int q = 0; q < Q; ++q)
#pragma unroll
        for (int m = 0; m < KS; ++m) t[q][m] = f_inf();
    bool rdone = false, ldone = false;
    stage(ctile);
    if (warp_active) {
        const int g_own0 = (wbase - ctile * ldt) >> 2;
        const int g_own1 = min(ngroups(ctile), (min(wbase + 32 * Q, N) - ctile * ldt + 3) >> 2);
        groups_done += knn_range<D, Q, KS>(sm, g_own0, g_own1, 0, qq, qkey, qv, t, rdone);
        rdone = false;
        groups_done += knn_range<D, Q, KS>(sm, g_own1, ngroups(ctile), +1, qq, qkey, qv, t, rdone);
        groups_done += knn_range<D, Q, KS>(sm, 0, g_own0, -1, qq, qkey, qv, t, ldone);
    }
    for (int ti = ctile + 1; ti < ntile; ++ti) {  // right tiles
        float r[Q], lb, rb;
        current_radii(t, r);
        warp_window(qkey, qv, r, lb, rb);
        float blb = f_inf(), brb = (warp_active && !rdone) ? rb : -f_inf();
        block_minmax(blb, brb, sb);
        if (!(__ldg(skey + ti * ldt) < brb)) break;
        stage(ti);
        if (warp_active && !rdone)
            groups_done += knn_range<D, Q, KS>(sm, 0, ngroups(ti), +1, qq, qkey, qv, t, rdone);
    }
    for (int ti = ctile - 1; ti >= 0; --ti) {  // left tiles
        float r[Q], lb, rb;
        current_radii(t, r);
        warp_window(qkey, qv, r, lb, rb);
        float blb = (warp_active && !ldone) ? lb : f_inf(), brb = -f_inf();
        block_minmax(blb, brb, sb);
        if (!(__ldg(skey + (ti + 1) * ldt - 1) > blb)) break;
        stage(ti);
        if (warp_active && !ldone)
            groups_done += knn_range<D, Q, KS>(sm, 0, ngroups(ti), -1, qq, qkey, qv, t, ldone);
    }
    float e[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) e[q] = topk_select(t[q], a.k);
    pass1_end(a, groups_done * 4ull * (unsigned long long)nvalid);

    // ---- pass 2: only the key window (key_q - eps, key_q + eps) of the CTA's queries
    float cz[Q], cyz[Q], cxz[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) cz[q] = cyz[q] = cxz[q] = 0.0f;
    float lb, rb;
    warp_window(qkey, qv, e, lb, rb);
    float blb = warp_active ? lb : f_inf(), brb = warp_active ? rb : -f_inf();
    block_minmax(blb, brb, sb);
    const int plo = first_greater(skey, N, blb);
    const int phi = first_not_less(skey, N, brb);
    if (plo < phi) {
        for (int ti = plo / ldt; ti <= (phi - 1) / ldt; ++ti) {
            stage(ti);
            if (warp_active)
                groups_done += count_range<d, d, Q>(sm, 0, ngroups(ti), lb, rb, qq, e, cz, cyz, cxz);
        }
    }

    // ---- digamma terms of Eq. 9 (compensated FP32 per thread), outputs at the original index
    FF acc{0.0f, 0.0f};
    float acc_abs = 0.0f;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        if (qv[q]) {
            const int i = qidx[q];
            const int self = e[q] > 0.0f ? 1 : 0;
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
    pass2_end(a);
    if (a.exec && warp_active && lane == 0) {
        const unsigned long long pairs = groups_done * 4ull * (unsigned long long)nvalid;
        work_add(0, pairs);
        work_add(1, pairs * 2ull * D);
    }
    double v = (double)acc.hi + (double)acc.lo;
    double w = (double)acc_abs;
    block_sum2(v, w, sred);
    if (threadIdx.x == 0) {
        a.partial[it] = v;
        a.partial_abs[it] = w;
    }
}

// first position p in [0, n) of a staged tile whose key (coordinate 1) is > x (keys ascending)
template <int D>
__device__ __forceinline__ int smem_first_greater(const float* __restrict__ s, int n, float x) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (s[tile_index<D>(1, mid)] > x) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

// One warp's block of 32*Q consecutive sorted queries of an instance staged whole in shared
// memory: pass 1 (own block, then right, then left), pass 2 over the key window, digamma terms;
// the block's partial sum is written to part. No CTA-wide barrier.
template <int d, int Q, int KS>
__device__ __forceinline__ void sweep_warp_block(const BatchArgs& a, const InstDesc& I, const float* sm, int wb,
                                                 int part) {
    pass1_begin(a);
    constexpr int D = 1 + 2 * d;
    const int N = I.N;
    const int lane = threadIdx.x & 31;
    const int32_t* sidx = a.sorted_idx + I.sort_off;
    const int wbase = wb * 32 * Q;
    u64 qq[Q][D];
    float qkey[Q];
    int qidx[Q];
    bool qv[Q];
    int nvalid = 0;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int pos = wbase + q * 32 + lane;
        qv[q] = pos < N;
        qidx[q] = qv[q] ? __ldg(sidx + pos) : -1;
        // the staged tile holds the sorted points: read the query's coordinates from it
#pragma unroll
        for (int c = 0; c < D; ++c) qq[q][c] = dup2(qv[q] ? sm[tile_index<D>(c, pos)] : 0.0f);
        qkey[q] = qv[q] ? sm[tile_index<D>(1, pos)] : 0.0f;
        nvalid += __popc(__ballot_sync(0xffffffffu, qv[q]));
    }
    const int ng = (N + 3) >> 2;
    unsigned long long groups_done = 0;
    float t[Q][KS];
#pragma unroll
    for (int q = 0; q < Q; ++q)
#pragma unroll
        for (int m = 0; m < KS; ++m) t[q][m] = f_inf();
    bool done = false;
    const int g_own0 = wbase >> 2;
    const int g_own1 = min(ng, (min(wbase + 32 * Q, N) + 3) >> 2);
    groups_done += knn_range<D, Q, KS>(sm, g_own0, g_own1, 0, qq, qkey, qv, t, done);
    groups_done += knn_range<D, Q, KS>(sm, g_own1, ng, +1, qq, qkey, qv, t, done);
    groups_done += knn_range<D, Q, KS>(sm, 0, g_own0, -1, qq, qkey, qv, t, done);
    float e[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) e[q] = topk_select(t[q], a.k);
    pass1_end(a, groups_done * 4ull * (unsigned long long)nvalid);

    float cz[Q], cyz[Q], cxz[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) cz[q] = cyz[q] = cxz[q] = 0.0f;
    float lb, rb;
    warp_window(qkey, qv, e, lb, rb);
    const int g_lo = smem_first_greater<D>(sm, N, lb) >> 2;
    groups_done += count_range<d, d, Q>(sm, g_lo, ng, lb, rb, qq, e, cz, cyz, cxz);

    FF acc{0.0f, 0.0f};
    float acc_abs = 0.0f;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        if (qv[q]) {
            const int i = qidx[q];
            const int self = e[q] > 0.0f ? 1 : 0;
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
    double v = (double)acc.hi + (double)acc.lo;
    double w = (double)acc_abs;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v += __shfl_down_sync(0xffffffffu, v, o);
        w += __shfl_down_sync(0xffffffffu, w, o);
    }
    pass2_end(a);
    if (lane == 0) {
        a.partial[part] = v;
        a.partial_abs[part] = w;
        if (a.exec) {
            const unsigned long long pairs = groups_done * 4ull * (unsigned long long)nvalid;
            work_add(0, pairs);
            work_add(1, pairs * 2ull * D);
        }
    }
}

// process_item_sweep for an estimate whose sort group is cut into strips (SortGroup): the CTA's
// query block (a divisor of kStripPoints, so it lies in one strip) first sweeps its own strip,
// staged whole, outward from each warp's queries, then the other strips nearest first in the
// second key (coordinate K2: y_{t'-1-tau} for d >= 2, y_t for d = 1) while their key range meets
// the CTA's window, each staged over the CTA's y_{t'-1} window; pass 2 stages the y_{t'-1} window
// of every strip (d >= 2: of those meeting the second-key window). Skips are exact as in
// sweep_warp_block_strips. A tile holds at least one strip (the plan).
template <int d, int Q, int KS>
__device__ __forceinline__ void process_item_sweep_strips(const BatchArgs& a, const InstDesc& I, int q0, int it,
                                                          float* sm, double* sred, float* sbnd) {
    pass1_begin(a);
    constexpr int D = 1 + 2 * d;
    constexpr int K2 = d >= 2 ? 2 : 0;
    const int N = I.N;
    const int npos = I.npad;
    const int S = I.strips;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int32_t* sidx = a.sorted_idx + I.sort_off;
    const float* skey = a.sorted_key + I.sort_off;
    const int32_t* spos = a.strip_pos + I.strip_off;
    const float* sk2 = a.strip_k2 + 2 * I.strip_off;
    const int wbase = q0 + warp * 32 * Q;
    u64 qq[Q][D];
    float qkey[Q], qk2[Q];
    int qidx[Q];
    bool qv[Q];
    int nvalid = 0;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int pos = wbase + q * 32 + lane;
        qidx[q] = pos < npos ? __ldg(sidx + pos) : -1;
        qv[q] = qidx[q] >= 0;
        float p[D];
        if (qv[q]) {
            gather_point<d>(I, qidx[q], p, a.flags);
        } else {
#pragma unroll
            for (int c = 0; c < D; ++c) p[c] = 0.0f;
        }
        qkey[q] = p[1];
        qk2[q] = p[K2];
#pragma unroll
        for (int c = 0; c < D; ++c) qq[q][c] = dup2(p[c]);
        nvalid += __popc(__ballot_sync(0xffffffffu, qv[q]));
    }
    const bool warp_active = nvalid > 0;
    unsigned long long groups_done = 0;

    int st_base = -1, st_n = 0;
    auto stage = [&](int base, int n) {  // sorted positions base .. base + n - 1 as one tile
        if (st_base == base && st_n == n) return;
        __syncthreads();
        stage_tile_sorted<d>(I, sidx, base, n, sm, a.flags);
        __syncthreads();
        st_base = base;
        st_n = n;
    };

    float t[Q][KS];
#pragma unroll
    for (int q = 0; q < Q; ++q)
#pragma unroll
        for (int m = 0; m < KS; ++m) t[q][m] = f_inf();
    const int s0 = q0 / kStripPoints;
    {
        const int ps = __ldg(spos + s0), pe = __ldg(spos + s0 + 1);
        stage(ps, pe - ps);
        if (warp_active) {
            const int ng = (pe - ps + 3) >> 2;
            const int g_own0 = (wbase - ps) >> 2;
            const int g_own1 = min(ng, (min(wbase + 32 * Q, pe) - ps + 3) >> 2);
            bool done = false;
            groups_done += knn_range<D, Q, KS>(sm, g_own0, g_own1, 0, qq, qkey, qv, t, done);
            done = false;
            groups_done += knn_range<D, Q, KS>(sm, g_own1, ng, +1, qq, qkey, qv, t, done);
            done = false;
            groups_done += knn_range<D, Q, KS>(sm, 0, g_own0, -1, qq, qkey, qv, t, done);
        }
    }
    bool up = s0 + 1 < S, down = s0 > 0;
    for (int step = 1; up || down; ++step) {
        for (int side = 0; side < 2; ++side) {
            const int s = side == 0 ? s0 + step : s0 - step;
            if (side == 0 ? (!up || s >= S) : (!down || s < 0)) {
                if (side == 0) up = false;
                else down = false;
                continue;
            }
            float r[Q], lb, rb, lb2, rb2;
            current_radii(t, r);
            warp_window(qkey, qv, r, lb, rb);
            warp_window(qk2, qv, r, lb2, rb2);
            float blb2 = lb2, brb2 = rb2;
            block_minmax(blb2, brb2, sbnd);
            if (side == 0 && !(__ldg(sk2 + 2 * s) < brb2)) {
                up = false;
                continue;
            }
            if (side == 1 && !(__ldg(sk2 + 2 * s + 1) > blb2)) {
                down = false;
                continue;
            }
            float blb = lb, brb = rb;
            block_minmax(blb, brb, sbnd);
            const int ps = __ldg(spos + s), len = __ldg(spos + s + 1) - ps;
            const int plo = ps + first_greater(skey + ps, len, blb);
            const int phi = ps + first_not_less(skey + ps, len, brb);
            if (plo >= phi) continue;
            stage(plo, phi - plo);
            if (warp_active) {
                const int ng = (phi - plo + 3) >> 2;
                int g = 0;
                while (g < ng && group_key_hi<D>(sm, g) <= lb) ++g;
                bool done = false;
                groups_done += knn_range<D, Q, KS>(sm, g, ng, +1, qq, qkey, qv, t, done);
            }
        }
    }
    float e[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) e[q] = topk_select(t[q], a.k);
    pass1_end(a, groups_done * 4ull * (unsigned long long)nvalid);

    float cz[Q], cyz[Q], cxz[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) cz[q] = cyz[q] = cxz[q] = 0.0f;
    float lb, rb, lb2, rb2;
    warp_window(qkey, qv, e, lb, rb);
    warp_window(qk2, qv, e, lb2, rb2);
    float blb = lb, brb = rb, blb2 = lb2, brb2 = rb2;
    block_minmax(blb, brb, sbnd);
    block_minmax(blb2, brb2, sbnd);
    for (int s = 0; s < S; ++s) {
        if constexpr (K2 != 0) {
            if (!(__ldg(sk2 + 2 * s + 1) > blb2)) continue;
            if (!(__ldg(sk2 + 2 * s) < brb2)) break;
        }
        const int ps = __ldg(spos + s), len = __ldg(spos + s + 1) - ps;
        const int plo = ps + first_greater(skey + ps, len, blb);
        const int phi = ps + first_not_less(skey + ps, len, brb);
        if (plo >= phi) continue;
        stage(plo, phi - plo);
        if (warp_active) {
            const int ng = (phi - plo + 3) >> 2;
            int g = 0;
            while (g < ng && group_key_hi<D>(sm, g) <= lb) ++g;
            groups_done += count_range<d, d, Q>(sm, g, ng, lb, rb, qq, e, cz, cyz, cxz);
        }
    }

    FF acc{0.0f, 0.0f};
    float acc_abs = 0.0f;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        if (qv[q]) {
            const int i = qidx[q];
            const int self = e[q] > 0.0f ? 1 : 0;
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
    pass2_end(a);
    if (a.exec && warp_active && lane == 0) {
        const unsigned long long pairs = groups_done * 4ull * (unsigned long long)nvalid;
        work_add(0, pairs);
        work_add(1, pairs * 2ull * D);
    }
    double v = (double)acc.hi + (double)acc.lo;
    double w = (double)acc_abs;
    block_sum2(v, w, sred);
    if (threadIdx.x == 0) {
        a.partial[it] = v;
        a.partial_abs[it] = w;
    }
}

// first group g in [g0, g1) of a staged tile with group_key_hi(g) > x (keys ascending in range)
template <int D>
__device__ __forceinline__ int smem_first_group_above(const float* __restrict__ s, int g0, int g1, float x) {
    int lo = g0, hi = g1;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (group_key_hi<D>(s, mid) > x) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

// sweep_warp_block for a group cut into strips (SortGroup). Two target coordinates bound the
// distances: key1 = y_{t'-1} (coordinate 1) and key2 (coordinate K2 = 2, y_{t'-1-tau}, for d >= 2;
// K2 = 0, y_t, for d = 1). fl(|Δkey1|) bounds from below the joint distance and b = max over y-
// (hence max(a, b) and max(b, x)); fl(|Δkey2|) bounds the joint distance, and for d >= 2 also b.
// A reference is skipped when one of them is >= r for every query of the warp, decided per strip
// from its key2 range and inside a strip from its key1 order, bounds rounded outward. Pass 1: the
// warp's own positions, its own strip(s) outward from them, then the other strips nearest first
// in key2, each entered at the warp's middle key1 and swept both ways. Pass 2: the key1 window of
// every strip (for d >= 2 only the strips whose key2 range meets the key2 window). Strip padding
// (index -1, +inf coordinates) is neither a query nor ever inside a radius.
template <int d, int Q, int KS>
__device__ __forceinline__ void sweep_warp_block_strips(const BatchArgs& a, const InstDesc& I, const float* sm,
                                                        int wb, int part) {
    pass1_begin(a);
    constexpr int D = 1 + 2 * d;
    constexpr int K2 = d >= 2 ? 2 : 0;  // coordinate of the second key
    const int N = I.N;
    const int npos = I.npad;
    const int S = I.strips;
    const int lane = threadIdx.x & 31;
    const int32_t* sidx = a.sorted_idx + I.sort_off;
    const int32_t* spos = a.strip_pos + I.strip_off;
    const float* sk2 = a.strip_k2 + 2 * I.strip_off;
    const int wbase = wb * 32 * Q;
    u64 qq[Q][D];
    float qkey[Q], qk2[Q];
    int qidx[Q];
    bool qv[Q];
    int nvalid = 0;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int pos = wbase + q * 32 + lane;
        qidx[q] = pos < npos ? __ldg(sidx + pos) : -1;
        qv[q] = qidx[q] >= 0;
#pragma unroll
        for (int c = 0; c < D; ++c) qq[q][c] = dup2(qv[q] ? sm[tile_index<D>(c, pos)] : 0.0f);
        qkey[q] = qv[q] ? sm[tile_index<D>(1, pos)] : 0.0f;
        qk2[q] = qv[q] ? sm[tile_index<D>(K2, pos)] : 0.0f;
        nvalid += __popc(__ballot_sync(0xffffffffu, qv[q]));
    }
    unsigned long long groups_done = 0;
    if (nvalid == 0) {  // a warp block of strip padding only
        if (lane == 0) {
            a.partial[part] = 0.0;
            a.partial_abs[part] = 0.0;
        }
        pass1_end(a, 0);
        pass2_end(a);
        return;
    }
    // median-ish entry key: the middle valid query key of the warp
    float kmin = f_inf(), kmax = -f_inf();
#pragma unroll
    for (int q = 0; q < Q; ++q)
        if (qv[q]) {
            kmin = fminf(kmin, qkey[q]);
            kmax = fmaxf(kmax, qkey[q]);
        }
    kmin = warp_min(kmin);
    kmax = warp_max(kmax);
    const float kmid = 0.5f * kmin + 0.5f * kmax;
    // the strips holding the warp's positions
    int s_lo = 0;
    while (s_lo + 1 < S && __ldg(spos + s_lo + 1) <= wbase) ++s_lo;
    int s_hi = s_lo;
    const int wend = min(wbase + 32 * Q, npos);
    while (s_hi + 1 < S && __ldg(spos + s_hi + 1) < wend) ++s_hi;
    const int g_own0 = wbase >> 2, g_own1 = (wend + 3) >> 2;

    // ---- pass 1
    float t[Q][KS];
#pragma unroll
    for (int q = 0; q < Q; ++q)
#pragma unroll
        for (int m = 0; m < KS; ++m) t[q][m] = f_inf();
    bool done = false;
    groups_done += knn_range<D, Q, KS>(sm, g_own0, g_own1, 0, qq, qkey, qv, t, done);
    for (int s = s_lo; s <= s_hi; ++s) {  // own strip(s), outward from the own positions
        const int gs = __ldg(spos + s) >> 2, ge = __ldg(spos + s + 1) >> 2;
        done = false;
        groups_done += knn_range<D, Q, KS>(sm, max(gs, g_own1), ge, +1, qq, qkey, qv, t, done);
        done = false;
        groups_done += knn_range<D, Q, KS>(sm, gs, min(ge, g_own0), -1, qq, qkey, qv, t, done);
    }
    // other strips, nearest first in key2, while their key2 range meets the window
    bool up = s_hi + 1 < S, down = s_lo > 0;
    for (int step = 1; up || down; ++step) {
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            const int s = side == 0 ? s_hi + step : s_lo - step;
            if (side == 0 ? (!up || s >= S) : (!down || s < 0)) {
                if (side == 0) up = false;
                else down = false;
                continue;
            }
            float r[Q], lb2, rb2;
            current_radii(t, r);
            warp_window(qk2, qv, r, lb2, rb2);
            if (side == 0 && !(__ldg(sk2 + 2 * s) < rb2)) {
                up = false;
                continue;
            }
            if (side == 1 && !(__ldg(sk2 + 2 * s + 1) > lb2)) {
                down = false;
                continue;
            }
            const int gs = __ldg(spos + s) >> 2, ge = __ldg(spos + s + 1) >> 2;
            const int gm = smem_first_group_above<D>(sm, gs, ge, kmid);
            done = false;
            groups_done += knn_range<D, Q, KS>(sm, gm, ge, +1, qq, qkey, qv, t, done);
            done = false;
            groups_done += knn_range<D, Q, KS>(sm, gs, gm, -1, qq, qkey, qv, t, done);
        }
    }
    float e[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) e[q] = topk_select(t[q], a.k);
    pass1_end(a, groups_done * 4ull * (unsigned long long)nvalid);

    // ---- pass 2: the key1 window of every strip (d >= 2: whose key2 range meets the window; the
    // counts of n_z and n_xz do not involve y_t, so for d = 1 no strip is skipped)
    float cz[Q], cyz[Q], cxz[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) cz[q] = cyz[q] = cxz[q] = 0.0f;
    float lb, rb, lb2, rb2;
    warp_window(qkey, qv, e, lb, rb);
    warp_window(qk2, qv, e, lb2, rb2);
    for (int s = 0; s < S; ++s) {
        if constexpr (K2 != 0) {
            if (!(__ldg(sk2 + 2 * s + 1) > lb2)) continue;
            if (!(__ldg(sk2 + 2 * s) < rb2)) break;
        }
        const int gs = __ldg(spos + s) >> 2, ge = __ldg(spos + s + 1) >> 2;
        const int g_lo = smem_first_group_above<D>(sm, gs, ge, lb);
        groups_done += count_range<d, d, Q>(sm, g_lo, ge, lb, rb, qq, e, cz, cyz, cxz);
    }

    FF acc{0.0f, 0.0f};
    float acc_abs = 0.0f;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        if (qv[q]) {
            const int i = qidx[q];
            const int self = e[q] > 0.0f ? 1 : 0;
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
    double v = (double)acc.hi + (double)acc.lo;
    double w = (double)acc_abs;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v += __shfl_down_sync(0xffffffffu, v, o);
        w += __shfl_down_sync(0xffffffffu, w, o);
    }
    pass2_end(a);
    if (lane == 0) {
        a.partial[part] = v;
        a.partial_abs[part] = w;
        if (a.exec) {
            const unsigned long long pairs = groups_done * 4ull * (unsigned long long)nvalid;
            work_add(0, pairs);
            work_add(1, pairs * 2ull * D);
        }
    }
}

// A whole instance that fits shared memory: staged once in sorted order, then every warp takes
// blocks of 32*Q queries from a CTA-local counter until none is left (work balances across the
// warps; the only barriers are at the start and the end of the instance).
template <int d, int Q, int KS>
__device__ __forceinline__ void process_instance_sweep_warps(const BatchArgs& a, const InstDesc& I, int wb0,
                                                             float* sm, int* s_wblock) {
    constexpr int D = 1 + 2 * d;
    const int npos = I.npad;  // sorted positions (N, or N plus strip padding)
    const int32_t* sidx = a.sorted_idx + I.sort_off;
    stage_tile_sorted<d>(I, sidx, 0, npos, sm, a.flags);
    if (threadIdx.x == 0) *s_wblock = wb0;
    __syncthreads();
    const int wb1 = min((npos + 32 * Q - 1) / (32 * Q), wb0 + I.wb_chunk);  // this item's warp blocks
    for (;;) {
        int wb = 0;
        if ((threadIdx.x & 31) == 0) wb = atomicAdd(s_wblock, 1);
        wb = __shfl_sync(0xffffffffu, wb, 0);
        if (wb >= wb1) break;
        if (I.strips > 1)
            sweep_warp_block_strips<d, Q, KS>(a, I, sm, wb, I.part_begin + wb);
        else
            sweep_warp_block<d, Q, KS>(a, I, sm, wb, I.part_begin + wb);
    }
    __syncthreads();  // the staged instance stays until every warp is done with it
    (void)D;
}

}  // namespace te
