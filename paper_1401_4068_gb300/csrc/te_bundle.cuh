// Target-part sharing: the estimates of one (series, window start, window, d, tau) share every
// target coordinate of their joint points (y_t and y- of Eq. 6 / Eq. 10); they differ only in the
// source part x-, which comes from a permuted repetition (a surrogate, Fig. 3) or another
// interaction delay u (the scan of Eq. 5). A bundle of up to M such estimates is staged once in
// shared memory in the order of its sort group (target part once, then each member's source
// part), and every warp evaluates a block of 32*Q sorted queries against all members at once:
//   pass 1: the target-part distance max(|dy_t|, |dy-|) of a (query, reference) pair is computed
//           once and joined with each member's |dx-| to give that member's joint distance;
//   pass 2: a = |dy_t| and b = max |dy-| are computed once and compared with each member's eps.
// Every member's distances are exactly the ones the unshared search computes (the same FP32
// subtractions, max is exact), so eps and the counts are identical. The key windows of the sorted
// sweep (see te_sweep.cuh) use the largest radius over the members, a superset of each member's.
#pragma once

#include "te_sweep.cuh"

namespace te {

// max(a, |c_0|, ..., |c_{n-1}|) for a >= 0, three inputs per instruction
template <int n>
__device__ __forceinline__ float absmax_join(float a, const float (&c)[n]) {
    float v[n + 1];
    v[0] = a;
#pragma unroll
    for (int i = 0; i < n; ++i) v[i + 1] = c[i];
    return absmax_range<0, n>(v);
}

// Stage sorted positions base .. base + nv - 1 of a bundle, in the grouped tile layout of
// te_device.cuh: first a tile of the target part (1 + d coordinates: y_t, y_{t'-1}, ...), then
// one tile per member of its source part (d coordinates), member m's at the float offset
// cap * (1 + d + m * d) (cap: points per tile, a multiple of 4); +inf past the last point (a
// padded reference is never inside any radius).
template <int d, int M>
__device__ __forceinline__ void stage_bundle(const BatchArgs& a, const InstDesc& L, const int32_t* mem, int nb,
                                             const int32_t* __restrict__ sidx, int base, int nv, int cap,
                                             float* sm) {
    constexpr int DA = 1 + d;
    const int N = nv;
    const int nfill = (N + 3) & ~3;
    for (int p = threadIdx.x; p < nfill; p += blockDim.x) {
        const int i = p < N ? __ldg(sidx + base + p) : -1;  // -1: strip padding
        if (i >= 0) {
            const int r = i / L.W;
            const int t = L.t_start + (i - r * L.W);
            const float* y = L.tgt + (size_t)r * L.T;
            sm[tile_index<DA>(0, p)] = __ldg(y + t);
#pragma unroll
            for (int c = 0; c < d; ++c) sm[tile_index<DA>(1 + c, p)] = __ldg(y + t - 1 - c * L.tau);
        } else {
#pragma unroll
            for (int c = 0; c < DA; ++c) sm[tile_index<DA>(c, p)] = f_inf();
        }
    }
#pragma unroll 1
    for (int m = 0; m < nb; ++m) {
        const InstDesc& J = a.insts[mem[m]];
        const int32_t* perm = J.perm;
        const float* src = J.src;
        const int u = J.u, R = J.R;
        float* col = sm + cap * (DA + m * d);
        for (int p = threadIdx.x; p < nfill; p += blockDim.x) {
            const int i = p < N ? __ldg(sidx + base + p) : -1;
            if (i >= 0) {
                const int r = i / L.W;
                const int t = L.t_start + (i - r * L.W);
                int rs = r;
                if (perm) {
                    rs = __ldg(perm + r);
                    if ((unsigned)rs >= (unsigned)R) {
                        atomicOr(a.flags, kFlagBadPerm);
                        rs = 0;
                    }
                }
                const float* x = src + (size_t)rs * L.T;
#pragma unroll
                for (int c = 0; c < d; ++c) col[tile_index<d>(c, p)] = __ldg(x + t - u - c * L.tau);
            } else {
#pragma unroll
                for (int c = 0; c < d; ++c) col[tile_index<d>(c, p)] = f_inf();
            }
        }
    }
}

// Members m >= nb of a ragged bundle repeat member nb - 1 (the same staged columns and query
// coordinates), so every loop over the members is branch-free; their results are discarded.
template <int Q, int KS, int M>
__device__ __forceinline__ void bundle_radii(const float (&t)[M][Q][KS], float (&r)[Q]) {
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        r[q] = t[0][q][KS - 1];
#pragma unroll
        for (int m = 1; m < M; ++m) r[q] = fmaxf(r[q], t[m][q][KS - 1]);
    }
}

// pass 1 for one group of four references: the target part once, then every member's joint
// distances, all of them before the first (branching) top-k insertion
template <int d, int Q, int KS, int M>
__device__ __forceinline__ void bknn_group(const float* __restrict__ s, const int (&coff)[M], int j,
                                           const u64 (&qa)[Q][1 + d], const u64 (&qc)[M][Q][d],
                                           float (&t)[M][Q][KS]) {
    constexpr int DA = 1 + d;
    ulonglong2 ra[DA];
    load_refs4<DA>(s, j, ra);
    float ma[Q][4];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        float dx[DA], dy[DA], dz[DA], dw[DA];
        diff4<DA>(qa[q], ra, dx, dy, dz, dw);
        ma[q][0] = absmax_range<0, DA - 1>(dx);
        ma[q][1] = absmax_range<0, DA - 1>(dy);
        ma[q][2] = absmax_range<0, DA - 1>(dz);
        ma[q][3] = absmax_range<0, DA - 1>(dw);
    }
    float mm[M][Q][4];
#pragma unroll
    for (int m = 0; m < M; ++m) {
        ulonglong2 rc[d];
        load_refs4<d>(s + coff[m], j, rc);
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            float cx[d], cy[d], cz[d], cw[d];
            diff4<d>(qc[m][q], rc, cx, cy, cz, cw);
            mm[m][q][0] = absmax_join<d>(ma[q][0], cx);
            mm[m][q][1] = absmax_join<d>(ma[q][1], cy);
            mm[m][q][2] = absmax_join<d>(ma[q][2], cz);
            mm[m][q][3] = absmax_join<d>(ma[q][3], cw);
        }
        if constexpr (d >= 4) {  // wide members: insert before the next member's loads (registers)
#pragma unroll
            for (int q = 0; q < Q; ++q)
#pragma unroll
                for (int e = 0; e < 4; ++e) topk_push(t[m][q], mm[m][q][e]);
        }
    }
    if constexpr (d < 4) {
#pragma unroll
        for (int m = 0; m < M; ++m)
#pragma unroll
            for (int q = 0; q < Q; ++q)
#pragma unroll
                for (int e = 0; e < 4; ++e) topk_push(t[m][q], mm[m][q][e]);
    }
}

// pass 1 over groups [g0, g1) in direction dir (as knn_range in te_sweep.cuh)
template <int d, int Q, int KS, int M>
__device__ __forceinline__ int bknn_range(const float* __restrict__ s, const int (&coff)[M], int g0, int g1,
                                          int dir, const u64 (&qa)[Q][1 + d], const u64 (&qc)[M][Q][d],
                                          const float (&qkey)[Q], const bool (&qv)[Q], float (&t)[M][Q][KS],
                                          bool& done) {
    float r[Q], lb, rb;
    bundle_radii<Q, KS, M>(t, r);
    warp_window(qkey, qv, r, lb, rb);
    int n = 0;
#pragma unroll 1
    for (int jj = g0; jj < g1; ++jj) {
        const int j = dir < 0 ? g1 - 1 - (jj - g0) : jj;
        if (dir > 0 && group_key_lo<1 + d>(s, j) >= rb) {
            done = true;
            break;
        }
        if (dir < 0 && group_key_hi<1 + d>(s, j) <= lb) {
            done = true;
            break;
        }
        bknn_group<d, Q, KS, M>(s, coff, j, qa, qc, t);
        if ((++n & 3) == 0 && dir != 0) {
            bundle_radii<Q, KS, M>(t, r);
            warp_window(qkey, qv, r, lb, rb);
        }
    }
    return n;
}

// pass 2 over groups [g0, g1) ascending inside the key window [lb, rb]
template <int d, int Q, int M>
__device__ __forceinline__ int bcount_range(const float* __restrict__ s, const int (&coff)[M], int g0, int g1,
                                            float lb, float rb, const u64 (&qa)[Q][1 + d], const u64 (&qc)[M][Q][d],
                                            const float (&e)[M][Q], float (&cz)[M][Q], float (&cyz)[M][Q],
                                            float (&cxz)[M][Q]) {
    constexpr int DA = 1 + d;
    int n = 0;
#pragma unroll 1
    for (int j = g0; j < g1; ++j) {
        if (group_key_lo<DA>(s, j) >= rb) break;
        if (group_key_hi<DA>(s, j) <= lb) continue;
        ulonglong2 ra[DA];
        load_refs4<DA>(s, j, ra);
        // a: signed dy_t (compared through |.|), b: max |dy-| (or the signed single coordinate)
        float va[Q][4], vb[Q][4];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            float dd[4][DA];
            diff4<DA>(qa[q], ra, dd[0], dd[1], dd[2], dd[3]);
#pragma unroll
            for (int x = 0; x < 4; ++x) {
                va[q][x] = dd[x][0];
                if constexpr (d == 1) vb[q][x] = dd[x][1];
                else vb[q][x] = absmax_range<1, d>(dd[x]);
            }
        }
#pragma unroll
        for (int m = 0; m < M; ++m) {
            ulonglong2 rc[d];
            load_refs4<d>(s + coff[m], j, rc);
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                float cc[4][d];
                diff4<d>(qc[m][q], rc, cc[0], cc[1], cc[2], cc[3]);
                const float em = e[m][q];
#pragma unroll
                for (int x = 0; x < 4; ++x) {
                    float sb, sx;
                    if constexpr (d == 1) {
                        sb = abs_set_lt(vb[q][x], em);
                        sx = abs_set_lt(cc[x][0], em);
                    } else {
                        sb = set_lt(vb[q][x], em);
                        sx = set_lt(absmax_range<0, d - 1>(cc[x]), em);
                    }
                    const float sa = abs_set_lt(va[q][x], em);
                    cz[m][q] += sb;
                    cyz[m][q] = fmaf(sa, sb, cyz[m][q]);
                    cxz[m][q] = fmaf(sx, sb, cxz[m][q]);
                }
            }
        }
        ++n;
    }
    return n;
}

// One warp's block of 32*Q sorted queries against all nb members of a staged bundle; writes one
// partial sum per member (its part wb) and the members' optional per-point outputs.
template <int d, int Q, int KS, int M>
__device__ __forceinline__ void bundle_warp_block(const BatchArgs& a, const InstDesc& L, const int32_t* mem, int nb,
                                                  const float* sm, int wb) {
    pass1_begin(a);
    constexpr int DA = 1 + d;
    constexpr int D = 1 + 2 * d;
    constexpr int K2 = d >= 2 ? 2 : 0;  // coordinate of the second key (strips)
    const int N = L.N;
    const int npos = L.npad;  // sorted positions (N, or N plus the last strip's padding)
    const int S = L.strips;
    const int lane = threadIdx.x & 31;
    const int32_t* sidx = a.sorted_idx + L.sort_off;
    const int wbase = wb * 32 * Q;
    const int ng = (npos + 3) >> 2;
    int coff[M];  // offset of member m's source tile (ragged bundles repeat the last member)
#pragma unroll
    for (int m = 0; m < M; ++m) coff[m] = ng * 4 * (DA + min(m, nb - 1) * d);
    u64 qa[Q][DA];
    u64 qc[M][Q][d];
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
        for (int c = 0; c < DA; ++c) qa[q][c] = dup2(qv[q] ? sm[tile_index<DA>(c, pos)] : 0.0f);
#pragma unroll
        for (int m = 0; m < M; ++m)
#pragma unroll
            for (int c = 0; c < d; ++c)
                qc[m][q][c] = dup2(qv[q] ? sm[coff[m] + tile_index<d>(c, pos)] : 0.0f);
        qkey[q] = qv[q] ? sm[tile_index<DA>(1, pos)] : 0.0f;
        qk2[q] = qv[q] ? sm[tile_index<DA>(K2, pos)] : 0.0f;
        nvalid += __popc(__ballot_sync(0xffffffffu, qv[q]));
    }
    unsigned long long groups_done = 0;
    if (nvalid == 0) {  // strip padding only
        if (lane == 0)
            for (int m = 0; m < nb; ++m) {
                const InstDesc& J = a.insts[mem[m]];
                a.partial[J.part_begin + wb] = 0.0;
                a.partial_abs[J.part_begin + wb] = 0.0;
            }
        pass1_end(a, 0);
        pass2_end(a);
        return;
    }
    const int32_t* spos = a.strip_pos + L.strip_off;
    const float* sk2 = a.strip_k2 + 2 * L.strip_off;

    // ---- pass 1: own block, then right, then left (radii: largest over the members); over
    // strips: own strip(s) outward, then the other strips nearest first in the second key (as
    // sweep_warp_block_strips in te_sweep.cuh)
    float t[M][Q][KS];
#pragma unroll
    for (int m = 0; m < M; ++m)
#pragma unroll
        for (int q = 0; q < Q; ++q)
#pragma unroll
            for (int s = 0; s < KS; ++s) t[m][q][s] = f_inf();
    const int wend = min(wbase + 32 * Q, npos);
    const int g_own0 = wbase >> 2;
    const int g_own1 = min(ng, (wend + 3) >> 2);
    bool done = false;
    groups_done += bknn_range<d, Q, KS, M>(sm, coff, g_own0, g_own1, 0, qa, qc, qkey, qv, t, done);
    // a resident bundle reaches the 4096 points of a striped group only for d <= 2 (the 200 KB
    // budget holds 3,938 points of d = 3): the strip code is compiled for those alone
    if (d > 2 || S <= 1) {
        groups_done += bknn_range<d, Q, KS, M>(sm, coff, g_own1, ng, +1, qa, qc, qkey, qv, t, done);
        groups_done += bknn_range<d, Q, KS, M>(sm, coff, 0, g_own0, -1, qa, qc, qkey, qv, t, done);
    } else if constexpr (d <= 2) {
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
        int s_lo = 0;
        while (s_lo + 1 < S && __ldg(spos + s_lo + 1) <= wbase) ++s_lo;
        int s_hi = s_lo;
        while (s_hi + 1 < S && __ldg(spos + s_hi + 1) < wend) ++s_hi;
        for (int s = s_lo; s <= s_hi; ++s) {
            const int gs = __ldg(spos + s) >> 2, ge = __ldg(spos + s + 1) >> 2;
            done = false;
            groups_done += bknn_range<d, Q, KS, M>(sm, coff, max(gs, g_own1), ge, +1, qa, qc, qkey, qv, t, done);
            done = false;
            groups_done += bknn_range<d, Q, KS, M>(sm, coff, gs, min(ge, g_own0), -1, qa, qc, qkey, qv, t, done);
        }
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
                bundle_radii<Q, KS, M>(t, r);
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
                const int gm = smem_first_group_above<DA>(sm, gs, ge, kmid);
                done = false;
                groups_done += bknn_range<d, Q, KS, M>(sm, coff, gm, ge, +1, qa, qc, qkey, qv, t, done);
                done = false;
                groups_done += bknn_range<d, Q, KS, M>(sm, coff, gs, gm, -1, qa, qc, qkey, qv, t, done);
            }
        }
    }
    float e[M][Q], emax[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        emax[q] = 0.0f;
#pragma unroll
        for (int m = 0; m < M; ++m) {
            e[m][q] = topk_select(t[m][q], a.k);
            emax[q] = fmaxf(emax[q], e[m][q]);
        }
    }
    pass1_end(a, groups_done * 4ull * (unsigned long long)nvalid * (unsigned long long)nb);

    // ---- pass 2: the key window of the largest eps
    float cz[M][Q], cyz[M][Q], cxz[M][Q];
#pragma unroll
    for (int m = 0; m < M; ++m)
#pragma unroll
        for (int q = 0; q < Q; ++q) cz[m][q] = cyz[m][q] = cxz[m][q] = 0.0f;
    float lb, rb;
    warp_window(qkey, qv, emax, lb, rb);
    if (d > 2 || S <= 1) {
        const int g_lo = smem_first_greater<DA>(sm, N, lb) >> 2;
        groups_done += bcount_range<d, Q, M>(sm, coff, g_lo, ng, lb, rb, qa, qc, e, cz, cyz, cxz);
    } else if constexpr (d <= 2) {
        float lb2, rb2;
        warp_window(qk2, qv, emax, lb2, rb2);
        for (int s = 0; s < S; ++s) {
            if constexpr (K2 != 0) {  // y_t (d = 1) bounds neither n_z nor n_xz: no strip is skipped
                if (!(__ldg(sk2 + 2 * s + 1) > lb2)) continue;
                if (!(__ldg(sk2 + 2 * s) < rb2)) break;
            }
            const int gs = __ldg(spos + s) >> 2, ge = __ldg(spos + s + 1) >> 2;
            const int g_lo = smem_first_group_above<DA>(sm, gs, ge, lb);
            groups_done += bcount_range<d, Q, M>(sm, coff, g_lo, ge, lb, rb, qa, qc, e, cz, cyz, cxz);
        }
    }

    // ---- per member: digamma terms of Eq. 9 (compensated FP32), outputs at the original index
#pragma unroll
    for (int m = 0; m < M; ++m) {
        if (m < nb) {
            const InstDesc& J = a.insts[mem[m]];
            const int64_t pt_off = J.pt_off;
            FF acc{0.0f, 0.0f};
            float acc_abs = 0.0f;
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                if (qv[q]) {
                    const int i = qidx[q];
                    const int self = e[m][q] > 0.0f ? 1 : 0;
                    const int nz = (int)cz[m][q] - self, nyz = (int)cyz[m][q] - self, nxz = (int)cxz[m][q] - self;
                    if (a.counts_out) {
                        int32_t* co = a.counts_out + 3 * pt_off;
                        co[i] = nz;
                        co[N + i] = nyz;
                        co[2 * N + i] = nxz;
                    }
                    if (a.eps_out) a.eps_out[pt_off + i] = e[m][q];
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
            if (lane == 0) {
                a.partial[J.part_begin + wb] = v;
                a.partial_abs[J.part_begin + wb] = w;
            }
        }
    }
    pass2_end(a);
    if (a.exec && lane == 0) {
        // pairs per member; 2 D algorithmic operations per pair; executed: the target part's
        // 2 (1 + d) once and 2 d per member slot (M slots, padding included)
        const unsigned long long g4 = groups_done * 4ull * (unsigned long long)nvalid;
        const unsigned long long alg = g4 * (unsigned long long)nb * 2ull * D;
        const unsigned long long run = g4 * (2ull * DA + (unsigned long long)M * 2ull * d);
        work_add(0, g4 * (unsigned long long)nb);
        work_add(1, alg);
        work_add(2, alg > run ? alg - run : 0ull);
    }
}

// A bundle too large to stage whole: a CTA takes a block of blockDim.x * Q consecutive sorted
// queries (one work item; `item` is its index within the bundle) and stages tiles of `cap` points
// (a multiple of the query block, so the block lies in one tile) around it, as process_item_sweep
// does for one estimate: the own tile first, then tiles to the right and to the left while any
// warp's key window reaches them, then pass 2 over the tiles of the CTA's key window. Windows use
// the largest radius over the members; the partial sums are per CTA block and member.
template <int d, int Q, int KS, int M>
__device__ __forceinline__ void bundle_item_tiled(const BatchArgs& a, const InstDesc& L, const int32_t* mem, int nb,
                                                  int q0, int item, float* sm, double* sred, float* sbnd) {
    pass1_begin(a);
    constexpr int DA = 1 + d;
    constexpr int D = 1 + 2 * d;
    const int N = L.N;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int32_t* sidx = a.sorted_idx + L.sort_off;
    const float* skey = a.sorted_key + L.sort_off;
    const int block = blockDim.x * Q;
    const int cap = ((a.smem_floats / (DA + M * d)) / block) * block;  // points per tile
    const int ntile = (N + cap - 1) / cap;
    const int ctile = q0 / cap;
    int coff[M];
#pragma unroll
    for (int m = 0; m < M; ++m) coff[m] = cap * (DA + min(m, nb - 1) * d);

    // queries: warp-contiguous runs of the sorted order, gathered from the series (Eq. 6 / 7)
    const int wbase = q0 + warp * 32 * Q;
    u64 qa[Q][DA];
    u64 qc[M][Q][d];
    float qkey[Q];
    int qidx[Q];
    bool qv[Q];
    int nvalid = 0;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int pos = wbase + q * 32 + lane;
        qv[q] = pos < N;
        qidx[q] = qv[q] ? __ldg(sidx + pos) : 0;
        const int r = qidx[q] / L.W;
        const int tt = L.t_start + (qidx[q] - r * L.W);
        const float* y = L.tgt + (size_t)r * L.T;
        qa[q][0] = dup2(qv[q] ? __ldg(y + tt) : 0.0f);
#pragma unroll
        for (int c = 0; c < d; ++c) qa[q][1 + c] = dup2(qv[q] ? __ldg(y + tt - 1 - c * L.tau) : 0.0f);
        qkey[q] = qv[q] ? __ldg(y + tt - 1) : 0.0f;
#pragma unroll
        for (int m = 0; m < M; ++m) {
            const InstDesc& J = a.insts[mem[min(m, nb - 1)]];
            int rs = r;
            if (J.perm && qv[q]) {
                rs = __ldg(J.perm + r);
                if ((unsigned)rs >= (unsigned)J.R) {
                    atomicOr(a.flags, kFlagBadPerm);
                    rs = 0;
                }
            }
            const float* x = J.src + (size_t)rs * L.T;
#pragma unroll
            for (int c = 0; c < d; ++c) qc[m][q][c] = dup2(qv[q] ? __ldg(x + tt - J.u - c * L.tau) : 0.0f);
        }
        nvalid += __popc(__ballot_sync(0xffffffffu, qv[q]));
        if (!qv[q]) qidx[q] = -1;
    }
    const bool warp_active = wbase < N;
    unsigned long long groups_done = 0;

    int staged = -1;
    auto stage = [&](int ti) {
        if (staged == ti) return;
        const int base = ti * cap;
        __syncthreads();
        stage_bundle<d, M>(a, L, mem, nb, sidx, base, min(cap, N - base), cap, sm);
        __syncthreads();
        staged = ti;
    };
    auto ngroups = [&](int ti) { return (min(cap, N - ti * cap) + 3) >> 2; };

    // ---- pass 1: own block, then right, then left
    float t[M][Q][KS];
#pragma unroll
    for (int m = 0; m < M; ++m)
#pragma unroll
        for (int q = 0; q < Q; ++q)
#pragma unroll
            for (int s = 0; s < KS; ++s) t[m][q][s] = f_inf();
    bool rdone = false, ldone = false;
    stage(ctile);
    if (warp_active) {
        const int g_own0 = (wbase - ctile * cap) >> 2;
        const int g_own1 = min(ngroups(ctile), (min(wbase + 32 * Q, N) - ctile * cap + 3) >> 2);
        groups_done += bknn_range<d, Q, KS, M>(sm, coff, g_own0, g_own1, 0, qa, qc, qkey, qv, t, rdone);
        rdone = false;
        groups_done += bknn_range<d, Q, KS, M>(sm, coff, g_own1, ngroups(ctile), +1, qa, qc, qkey, qv, t, rdone);
        groups_done += bknn_range<d, Q, KS, M>(sm, coff, 0, g_own0, -1, qa, qc, qkey, qv, t, ldone);
    }
    for (int ti = ctile + 1; ti < ntile; ++ti) {  // right tiles
        float r[Q], lb, rb;
        bundle_radii<Q, KS, M>(t, r);
        warp_window(qkey, qv, r, lb, rb);
        float blb = f_inf(), brb = (warp_active && !rdone) ? rb : -f_inf();
        block_minmax(blb, brb, sbnd);
        if (!(__ldg(skey + ti * cap) < brb)) break;
        stage(ti);
        if (warp_active && !rdone)
            groups_done += bknn_range<d, Q, KS, M>(sm, coff, 0, ngroups(ti), +1, qa, qc, qkey, qv, t, rdone);
    }
    for (int ti = ctile - 1; ti >= 0; --ti) {  // left tiles
        float r[Q], lb, rb;
        bundle_radii<Q, KS, M>(t, r);
        warp_window(qkey, qv, r, lb, rb);
        float blb = (warp_active && !ldone) ? lb : f_inf(), brb = -f_inf();
        block_minmax(blb, brb, sbnd);
        if (!(__ldg(skey + (ti + 1) * cap - 1) > blb)) break;
        stage(ti);
        if (warp_active && !ldone)
            groups_done += bknn_range<d, Q, KS, M>(sm, coff, 0, ngroups(ti), -1, qa, qc, qkey, qv, t, ldone);
    }
    float e[M][Q], emax[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        emax[q] = 0.0f;
#pragma unroll
        for (int m = 0; m < M; ++m) {
            e[m][q] = topk_select(t[m][q], a.k);
            emax[q] = fmaxf(emax[q], e[m][q]);
        }
    }
    pass1_end(a, groups_done * 4ull * (unsigned long long)nvalid * (unsigned long long)nb);

    // ---- pass 2: the tiles of the CTA's key window (largest eps over the members)
    float cz[M][Q], cyz[M][Q], cxz[M][Q];
#pragma unroll
    for (int m = 0; m < M; ++m)
#pragma unroll
        for (int q = 0; q < Q; ++q) cz[m][q] = cyz[m][q] = cxz[m][q] = 0.0f;
    float lb, rb;
    warp_window(qkey, qv, emax, lb, rb);
    float blb = warp_active ? lb : f_inf(), brb = warp_active ? rb : -f_inf();
    block_minmax(blb, brb, sbnd);
    const int plo = first_greater(skey, N, blb);
    const int phi = first_not_less(skey, N, brb);
    if (plo < phi) {
        for (int ti = plo / cap; ti <= (phi - 1) / cap; ++ti) {
            stage(ti);
            if (warp_active)
                groups_done += bcount_range<d, Q, M>(sm, coff, 0, ngroups(ti), lb, rb, qa, qc, e, cz, cyz, cxz);
        }
    }

    // ---- per member: digamma terms of Eq. 9, FP64 partial per CTA block
#pragma unroll 1
    for (int m = 0; m < nb; ++m) {
        const InstDesc& J = a.insts[mem[m]];
        const int64_t pt_off = J.pt_off;
        FF acc{0.0f, 0.0f};
        float acc_abs = 0.0f;
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            float em = e[0][q], cm = cz[0][q], cym = cyz[0][q], cxm = cxz[0][q];
#pragma unroll
            for (int mm = 1; mm < M; ++mm)
                if (mm == m) {
                    em = e[mm][q];
                    cm = cz[mm][q];
                    cym = cyz[mm][q];
                    cxm = cxz[mm][q];
                }
            if (qv[q]) {
                const int i = qidx[q];
                const int self = em > 0.0f ? 1 : 0;
                const int nz = (int)cm - self, nyz = (int)cym - self, nxz = (int)cxm - self;
                if (a.counts_out) {
                    int32_t* co = a.counts_out + 3 * pt_off;
                    co[i] = nz;
                    co[N + i] = nyz;
                    co[2 * N + i] = nxz;
                }
                if (a.eps_out) a.eps_out[pt_off + i] = em;
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
        __syncthreads();  // sred of the previous member is read
        block_sum2(v, w, sred);
        if (threadIdx.x == 0) {
            a.partial[J.part_begin + item] = v;
            a.partial_abs[J.part_begin + item] = w;
        }
    }
    pass2_end(a);
    if (a.exec && warp_active && lane == 0) {
        const unsigned long long g4 = groups_done * 4ull * (unsigned long long)nvalid;
        const unsigned long long alg = g4 * (unsigned long long)nb * 2ull * D;
        const unsigned long long run = g4 * (2ull * DA + (unsigned long long)M * 2ull * d);
        work_add(0, g4 * (unsigned long long)nb);
        work_add(1, alg);
        work_add(2, alg > run ? alg - run : 0ull);
    }
}

// bundle_item_tiled for a bundle whose sort group is cut into strips (SortGroup; strips start at
// multiples of kStripPoints, so the CTA's query block lies in one strip, and a strip fits one tile).
// Pass 1: the own strip staged whole and swept outward from each warp's queries, then the other
// strips nearest first in the second key (coordinate K2: y_{t'-1-tau} for d >= 2, y_t for d = 1)
// while their key range meets the CTA's window, each staged over the CTA's y_{t'-1} window.
// Pass 2: the y_{t'-1} window of every strip (for d >= 2 only those meeting the second-key
// window: y_t bounds neither n_z nor n_xz). Skips are exact as in sweep_warp_block_strips.
template <int d, int Q, int KS, int M>
__device__ __forceinline__ void bundle_item_tiled_strips(const BatchArgs& a, const InstDesc& L, const int32_t* mem,
                                                         int nb, int q0, int item, float* sm, double* sred,
                                                         float* sbnd) {
    pass1_begin(a);
    constexpr int DA = 1 + d;
    constexpr int D = 1 + 2 * d;
    constexpr int K2 = d >= 2 ? 2 : 0;
    const int N = L.N;
    const int npos = L.npad;
    const int S = L.strips;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int32_t* sidx = a.sorted_idx + L.sort_off;
    const float* skey = a.sorted_key + L.sort_off;
    const int32_t* spos = a.strip_pos + L.strip_off;
    const float* sk2 = a.strip_k2 + 2 * L.strip_off;
    const int block = blockDim.x * Q;
    const int cap = ((a.smem_floats / (DA + M * d)) / block) * block;  // >= kStripPoints (the plan)
    int coff[M];
#pragma unroll
    for (int m = 0; m < M; ++m) coff[m] = cap * (DA + min(m, nb - 1) * d);

    const int wbase = q0 + warp * 32 * Q;
    u64 qa[Q][DA];
    u64 qc[M][Q][d];
    float qkey[Q], qk2[Q];
    int qidx[Q];
    bool qv[Q];
    int nvalid = 0;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int pos = wbase + q * 32 + lane;
        qidx[q] = pos < npos ? __ldg(sidx + pos) : -1;
        qv[q] = qidx[q] >= 0;
        const int ii = qv[q] ? qidx[q] : 0;
        const int r = ii / L.W;
        const int tt = L.t_start + (ii - r * L.W);
        const float* y = L.tgt + (size_t)r * L.T;
        float pa[DA];
        pa[0] = qv[q] ? __ldg(y + tt) : 0.0f;
#pragma unroll
        for (int c = 0; c < d; ++c) pa[1 + c] = qv[q] ? __ldg(y + tt - 1 - c * L.tau) : 0.0f;
#pragma unroll
        for (int c = 0; c < DA; ++c) qa[q][c] = dup2(pa[c]);
        qkey[q] = pa[1];
        qk2[q] = pa[K2];
#pragma unroll
        for (int m = 0; m < M; ++m) {
            const InstDesc& J = a.insts[mem[min(m, nb - 1)]];
            int rs = r;
            if (J.perm && qv[q]) {
                rs = __ldg(J.perm + r);
                if ((unsigned)rs >= (unsigned)J.R) {
                    atomicOr(a.flags, kFlagBadPerm);
                    rs = 0;
                }
            }
            const float* x = J.src + (size_t)rs * L.T;
#pragma unroll
            for (int c = 0; c < d; ++c) qc[m][q][c] = dup2(qv[q] ? __ldg(x + tt - J.u - c * L.tau) : 0.0f);
        }
        nvalid += __popc(__ballot_sync(0xffffffffu, qv[q]));
    }
    const bool warp_active = nvalid > 0;
    unsigned long long groups_done = 0;

    int st_base = -1, st_n = 0;
    auto stage = [&](int base, int n) {  // sorted positions base .. base + n - 1 as one tile
        if (st_base == base && st_n == n) return;
        __syncthreads();
        stage_bundle<d, M>(a, L, mem, nb, sidx, base, n, cap, sm);
        __syncthreads();
        st_base = base;
        st_n = n;
    };

    float t[M][Q][KS];
#pragma unroll
    for (int m = 0; m < M; ++m)
#pragma unroll
        for (int q = 0; q < Q; ++q)
#pragma unroll
            for (int s = 0; s < KS; ++s) t[m][q][s] = f_inf();

    // ---- pass 1, own strip: staged whole, each warp outward from its queries
    const int s0 = q0 / kStripPoints;
    {
        const int ps = __ldg(spos + s0), pe = __ldg(spos + s0 + 1);
        stage(ps, pe - ps);
        if (warp_active) {
            const int ng = (pe - ps + 3) >> 2;
            const int g_own0 = (wbase - ps) >> 2;
            const int g_own1 = min(ng, (min(wbase + 32 * Q, pe) - ps + 3) >> 2);
            bool done = false;
            groups_done += bknn_range<d, Q, KS, M>(sm, coff, g_own0, g_own1, 0, qa, qc, qkey, qv, t, done);
            done = false;
            groups_done += bknn_range<d, Q, KS, M>(sm, coff, g_own1, ng, +1, qa, qc, qkey, qv, t, done);
            done = false;
            groups_done += bknn_range<d, Q, KS, M>(sm, coff, 0, g_own0, -1, qa, qc, qkey, qv, t, done);
        }
    }
    // ---- pass 1, other strips nearest first in the second key
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
            bundle_radii<Q, KS, M>(t, r);
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
                while (g < ng && group_key_hi<DA>(sm, g) <= lb) ++g;
                bool done = false;
                groups_done += bknn_range<d, Q, KS, M>(sm, coff, g, ng, +1, qa, qc, qkey, qv, t, done);
            }
        }
    }
    float e[M][Q], emax[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        emax[q] = 0.0f;
#pragma unroll
        for (int m = 0; m < M; ++m) {
            e[m][q] = topk_select(t[m][q], a.k);
            emax[q] = fmaxf(emax[q], e[m][q]);
        }
    }
    pass1_end(a, groups_done * 4ull * (unsigned long long)nvalid * (unsigned long long)nb);

    // ---- pass 2
    float cz[M][Q], cyz[M][Q], cxz[M][Q];
#pragma unroll
    for (int m = 0; m < M; ++m)
#pragma unroll
        for (int q = 0; q < Q; ++q) cz[m][q] = cyz[m][q] = cxz[m][q] = 0.0f;
    float lb, rb, lb2, rb2;
    warp_window(qkey, qv, emax, lb, rb);
    warp_window(qk2, qv, emax, lb2, rb2);
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
            while (g < ng && group_key_hi<DA>(sm, g) <= lb) ++g;
            groups_done += bcount_range<d, Q, M>(sm, coff, g, ng, lb, rb, qa, qc, e, cz, cyz, cxz);
        }
    }

    // ---- per member: digamma terms of Eq. 9, FP64 partial per CTA block
#pragma unroll 1
    for (int m = 0; m < nb; ++m) {
        const InstDesc& J = a.insts[mem[m]];
        const int64_t pt_off = J.pt_off;
        FF acc{0.0f, 0.0f};
        float acc_abs = 0.0f;
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            float em = e[0][q], cm = cz[0][q], cym = cyz[0][q], cxm = cxz[0][q];
#pragma unroll
            for (int mm = 1; mm < M; ++mm)
                if (mm == m) {
                    em = e[mm][q];
                    cm = cz[mm][q];
                    cym = cyz[mm][q];
                    cxm = cxz[mm][q];
                }
            if (qv[q]) {
                const int i = qidx[q];
                const int self = em > 0.0f ? 1 : 0;
                const int nz = (int)cm - self, nyz = (int)cym - self, nxz = (int)cxm - self;
                if (a.counts_out) {
                    int32_t* co = a.counts_out + 3 * pt_off;
                    co[i] = nz;
                    co[N + i] = nyz;
                    co[2 * N + i] = nxz;
                }
                if (a.eps_out) a.eps_out[pt_off + i] = em;
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
        __syncthreads();  // sred of the previous member is read
        block_sum2(v, w, sred);
        if (threadIdx.x == 0) {
            a.partial[J.part_begin + item] = v;
            a.partial_abs[J.part_begin + item] = w;
        }
    }
    pass2_end(a);
    if (a.exec && warp_active && lane == 0) {
        const unsigned long long g4 = groups_done * 4ull * (unsigned long long)nvalid;
        const unsigned long long alg = g4 * (unsigned long long)nb * 2ull * D;
        const unsigned long long run = g4 * (2ull * DA + (unsigned long long)M * 2ull * d);
        work_add(0, g4 * (unsigned long long)nb);
        work_add(1, alg);
        work_add(2, alg > run ? alg - run : 0ull);
    }
}

// The bundle kernel: a CTA takes a bundle (its leader's work item) from the queue, stages it,
// and its warps take 32*Q-query blocks from a CTA-local counter; TILED: bundles too large to stage
// whole, one CTA query block per work item (a separate instantiation, so that the resident path
// keeps the registers it needs without the tiled path's). Three CTAs per SM for d <= 3
// (a C3-sized bundle, 1200 points x 13 columns, takes 62 KB of shared memory), two above.
template <int d, int Q, int KS, int M, bool TILED>
__global__ void __launch_bounds__(kBundleThreads, d <= 3 ? 3 : 2) bundle_kernel(const BatchArgs a) {
    extern __shared__ __align__(16) float sm[];
    __shared__ double sred[64];
    __shared__ float sbnd[64];
    __shared__ int s_item;
    __shared__ int s_wblock;
    work_reset();
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = atomicAdd(a.queue, 1);
        __syncthreads();
        const int ticket = s_item;
        if (ticket >= a.n_items) break;
        const WorkItem w = a.items[a.item_base + ticket];
        const InstDesc L = a.insts[w.inst];
        const int32_t* mem = a.members + L.bundle_off;
        const int nb = L.bundle_n;
        if constexpr (TILED) {  // too large to stage whole: CTA tiles around a block of queries
            const int item = w.q0 / (int)(blockDim.x * Q);
            if (L.strips > 1)
                bundle_item_tiled_strips<d, Q, KS, M>(a, L, mem, nb, w.q0, item, sm, sred, sbnd);
            else
                bundle_item_tiled<d, Q, KS, M>(a, L, mem, nb, w.q0, item, sm, sred, sbnd);
            continue;
        } else {
            (void)sred;
            (void)sbnd;
        }
        stage_bundle<d, M>(a, L, mem, nb, a.sorted_idx + L.sort_off, 0, L.npad, (L.npad + 3) & ~3, sm);
        if (threadIdx.x == 0) s_wblock = w.q0;
        __syncthreads();
        const int wb1 = min((L.npad + 32 * Q - 1) / (32 * Q), w.q0 + L.wb_chunk);
        for (;;) {
            int wb = 0;
            if ((threadIdx.x & 31) == 0) wb = atomicAdd(&s_wblock, 1);
            wb = __shfl_sync(0xffffffffu, wb, 0);
            if (wb >= wb1) break;
            bundle_warp_block<d, Q, KS, M>(a, L, mem, nb, sm, wb);
        }
    }
    work_flush(a);
}

}  // namespace te
