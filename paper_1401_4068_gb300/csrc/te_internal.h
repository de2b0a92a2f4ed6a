// Internal declarations shared by the library's translation units (host + device).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "te_gb300.h"

namespace te {

// Device-side descriptor of one estimate: where its points come from (Eq. 6/7/10) and where
// its work items and per-point outputs live.
struct InstDesc {
    const float* src;      // source series [R][T]
    const float* tgt;      // target series [R][T]
    const int32_t* perm;   // source repetition paired with target repetition r, or nullptr
    int32_t R, T, W, t_start;
    int32_t tau, u, d, N;  // N = R * W points, joint dimension 1 + 2d
    int64_t pt_off;        // offset of this instance's points in concatenated eps/counts outputs
    int64_t sort_off;      // offset of its group's sorted order in the sweep arrays (sweep mode)
    int32_t item_begin;    // its work items are item_begin .. item_begin + n_items - 1
    int32_t n_items;
    int32_t part_begin;    // its partial sums are part_begin .. part_begin + n_parts - 1
    int32_t n_parts;
    int32_t warp_mode;     // 1: the instance is staged whole and warps take 32*Q-query blocks
    int32_t wb_chunk;      // warp mode: warp blocks per work item (an item's q0 is its first block)
    int32_t bundle_n;      // bundle leader: members that share its target part (0: not a leader)
    int32_t bundle_off;    // bundle leader: its members' instance indices start at members[bundle_off]
    int32_t strips;        // sweep: strips of its sort group (1: one key order, see SortGroup)
    int32_t npad;          // sweep: sorted positions of its group (N plus strip padding)
    int64_t strip_off;     // strips > 1: its group's strip table at strip_pos / strip_k2
};

// Points of one (series, window start, window) group: the estimates of a group (original and
// surrogates) share the target coordinates, so they share one order of the points sorted by the
// target coordinate y_{t'-1} (coordinate 1 of the joint space). With S > 1 strips the points are
// first ordered by a second target coordinate y_{t'-k2lag} and cut into strips of L consecutive
// ranks (the last one shorter, padded to a multiple of four positions with index -1 and key
// +inf), each sorted by y_{t'-1}; strip s holds positions strip_pos[s] = s * L .. strip_pos[s+1]-1
// and its second-key values lie in [strip_k2[2s], strip_k2[2s+1]]. L = kStripPoints (groups of
// 4 L points or more), so no warp block or 256-query CTA block spans two strips and a strip fits
// a tile of the tiled paths.
// The second key is y_{t'-1-tau} (coordinate 2, in y-) for d >= 2 and y_t (coordinate 0, not in
// y-) for d = 1.
struct SortGroup {
    const float* tgt;
    int32_t R, T, W, t_start, N;
    int32_t S;             // strips (1: one key order)
    int32_t npad;          // sorted positions (N when S == 1)
    int32_t k2lag;         // S > 1: the second key is y_{t' - k2lag}
    int32_t L;             // S > 1: points per strip (the last strip holds the rest)
    int32_t reserved;      // keeps the 64-bit fields aligned
    int64_t off;           // offset of the group's sorted index / key arrays (npad entries)
    int64_t strip_off;     // S > 1: strip_pos[strip_off .. strip_off + S], strip_k2[2 strip_off ..
                           // 2 strip_off + 2 S - 1]
};

constexpr int kStripPoints = 1024;  // points per strip (a multiple of 256 and of 32 Q)
constexpr int kMaxStrips = 64;

// Largest point count the sweep mode sorts (one CTA per group; runs in shared memory, merges
// through global memory above 8192 points).
constexpr int kSweepMaxN = 65536;

// One unit of work of the persistent kernel: queries q0 .. q0 + threads*qpt - 1 of an instance.
struct WorkItem {
    int32_t inst;
    int32_t q0;
};

// Largest CTA of the persistent batched kernel (its __launch_bounds__).
constexpr int kBatchedMaxThreads = 512;
// CTA of the warp-mode sweep kernel (d <= 2, every estimate resident in shared memory).
constexpr int kSweepWarpThreads = 1024;

// One estimate per lane (te_lanes.cuh): a group of estimates that share one target part (target
// series, repetitions, window start, window, d, tau) and one sorted order. Its members are
// members[mem_off .. mem_off + n_mem - 1] (instance indices), processed in blocks of 32 (one per
// lane); its sorted target part is tpart[tp_off ..] ((d + 2) / 2 float2 per position, chunk-major
// in chunks of 32 positions, N rounded up to 32) and the (repetition, sample) of each sorted
// position lane_rw[rw_off ..] (N rounded up to 32 entries).
struct LaneGroup {
    const float* tgt;
    int64_t sort_off;      // the group's sorted order (sorted_idx)
    int64_t tp_off;        // its sorted target part
    int64_t rw_off;        // its (repetition, sample) table
    int64_t ck_off;        // the key of each chunk's first position (lane_ckey)
    int64_t strip_off;     // strips > 1: its strip table (strip_pos / strip_k2, see SortGroup)
    int32_t R, T, W, t_start, N, d, tau;
    int32_t mem_off, n_mem;
    int32_t strips, npad;  // the sort group's strips and sorted positions (with strip padding)
    int32_t reserved;
};

// Source part of a block of 32 estimates, member-minor (written by lane_x_kernel): for repetition
// r, sample t = t0 + c and lane l, X[off + (r * ncols + c) * 32 + l] = src_l[perm_l[r]][t] (the lane's
// source repetition paired with target repetition r; perm nullptr: the identity). One coalesced
// 128-byte line then holds one source coordinate of one point for all 32 estimates (lanes past a
// ragged group's last estimate repeat it). Blocks with
// the same source series and pairings (the same surrogates at every analysis time point) share one
// array; the columns cover every sample their groups read.
struct LaneXBlock {
    int64_t off;
    int32_t R, T, t0, ncols;
    const float* src[32];
    const int32_t* perm[32];
};

// Work item of the lane kernel: sorted query positions q0 .. q0 + kLaneQB - 1 of group `group`
// against its estimates mblock * 32 .. mblock * 32 + 31, whose source parts are X block xblk.
struct LaneItem {
    int32_t group, mblock, q0, xblk;
};

constexpr int kLaneWarps = 8;
constexpr int kLaneThreads = 32 * kLaneWarps;
constexpr int kLaneQB = 256;         // sorted query positions per work item (one partial sum each)
constexpr int kLaneMinMembers = 8;   // smallest group the lane kernel takes (sharing mode 3)
// sharing mode 1 (default): the lane kernel for groups of at least kLaneAutoMembers estimates
// with d >= kLaneAutoMinD, where it measured faster than bundles or the unshared kernel (C5- and
// C3-shaped surrogate tests and the Lorenz delay scan: yes; the 16-estimate 17-D benchmark chunk:
// no)
constexpr int kLaneAutoMembers = 32, kLaneAutoMinD = 3;
constexpr int kLaneMinD = 2, kLaneMaxD = 8;

// Bits of the device flag word.
enum : int32_t { kFlagBadPerm = 1 };

struct BatchArgs {
    const InstDesc* insts;
    const WorkItem* items;
    int32_t n_items;         // items item_base .. item_base + n_items - 1 are this launch's
    int32_t item_base;
    int32_t* queue;          // work-queue head, zeroed before every launch
    int32_t* flags;          // device flag word (kFlag*)
    const float2* psi;       // psi(n) as (hi, lo) float pair, n = 0 .. psi_n-1 (entry 0 unused)
    int32_t k;
    int32_t smem_floats;     // floats of dynamic shared memory (reference tile capacity * D)
    double* partial;         // per-part sum of the Eq. 9 digamma terms (InstDesc part ranges)
    double* partial_abs;     // per-part sum of |terms| (for the error bound)
    int32_t* counts_out;     // nullable: per instance [3][N] at 3 * pt_off
    float* eps_out;          // nullable: per instance [N] at pt_off
    const int32_t* sorted_idx;  // sweep mode: per group, point indices in ascending key order
    const float* sorted_key;    // sweep mode: the keys in that order
    unsigned long long* exec;   // sweep mode: [0] evaluated (query, reference) pairs, [1] their
                                // 2 D FP32 ops, [2] ops not executed thanks to target-part sharing
    const int32_t* members;     // bundle kernel: member instance indices (leader first)
    const int32_t* strip_pos;   // sweep with strips: per group S + 1 sorted positions
    const float* strip_k2;      // sweep with strips: per group S (lowest, highest) y_t
    const LaneGroup* lgroups;   // lane kernel: groups, work items, sorted target parts, (r, w)
    const LaneItem* litems;
    const float2* tpart;
    const int32_t* lane_rw;
    const int32_t* lane_members;
    const LaneXBlock* lane_xb;
    const float* lane_x;
    const float* lane_ckey;
};

// ---- launchers (te_unit.cu) ----
cudaError_t launch_embed(const float* src, const float* tgt, int R, int T, int d, int tau, int u,
                         int t_start, int W, const int32_t* perm, float* points, int ld,
                         int32_t* flags, cudaStream_t s);
cudaError_t launch_knn(const float* pts, int N, int D, int ld, int k, float* eps, int32_t* nn,
                       int sm_count, cudaStream_t s);
cudaError_t launch_count(const float* pts, int N, int dy, int dx, int ld, const float* eps,
                         int32_t* counts, int sm_count, cudaStream_t s);

// ---- launchers (te_batched_*.cu, te_finalize.cu) ----
// Variant of the persistent kernel: d in [dlo, dhi] (dlo == dhi: specialised, d = 1..8; else
// dhi <= 5), ks = k-slots, qpt = queries per thread (1 for d >= 6).
struct BatchedVariant {
    int dlo, dhi, ks, qpt;
    bool sweep;      // sorted-sweep search instead of the exhaustive one
    bool warp_only;  // sweep_warp_kernel: every estimate staged whole, d = dlo = dhi <= 2, ks = 5
};
// Sort pre-pass: sorted index / key arrays (npad per group) and the strip tables; scratch: two
// (64-bit key, index) buffers of N entries per group at the group's offset.
cudaError_t launch_sort_groups(const SortGroup* groups, int n_groups, int32_t* idx, float* key,
                               unsigned long long* k64a, int32_t* ia, unsigned long long* k64b, int32_t* ib,
                               int32_t* strip_pos, float* strip_k2, cudaStream_t s);
cudaError_t prepare_sort_kernel(int nmax);
const void* batched_kernel_ptr(const BatchedVariant& v);
const void* batched_ptr_d1(int ks, int q, bool sweep);
const void* batched_ptr_d2(int ks, int q, bool sweep);
const void* batched_ptr_d3(int ks, int q, bool sweep);
const void* batched_ptr_d4(int ks, int q, bool sweep);
const void* batched_ptr_d5(int ks, int q, bool sweep);
const void* batched_ptr_d6(int ks, int q, bool sweep);
const void* batched_ptr_d7(int ks, int q, bool sweep);
const void* batched_ptr_d8(int ks, int q, bool sweep);
const void* batched_ptr_mix(int ks, int q, bool sweep);
const void* sweep_warp_ptr_d1(int ks, int q);
const void* sweep_warp_ptr_d2(int ks, int q);
cudaError_t launch_batched(const BatchedVariant& v, const BatchArgs& a, int grid, int threads,
                           size_t smem, cudaStream_t s);

// ---- the bundle kernel (te_bundle.cu): estimates sharing one target part, sorted sweep ----
constexpr int kBundleMax = 3;       // members per bundle
constexpr int kBundleQ = 1;         // queries per thread
constexpr int kBundleThreads = 256;
const void* bundle_kernel_ptr(int d, int ks, bool tiled);
cudaError_t launch_bundle(int d, int ks, bool tiled, const BatchArgs& a, int grid, size_t smem, cudaStream_t s);
// ---- the lane kernel (te_lanes*.cu): one estimate per lane, d = kLaneMinD .. kLaneMaxD, k <= 4, ----
// ---- one instantiation per delay class (tau = 1, 2, 3 compiled in; class 0: any tau) ----
constexpr int kLaneTauClasses = 4;
constexpr int kLaneSlots = (kLaneMaxD - kLaneMinD + 1) * kLaneTauClasses;  // (d, delay class) pairs
inline int lane_tau_class(int tau) { return tau >= 1 && tau < kLaneTauClasses ? tau : 0; }
const void* lane_kernel_ptr(int d, int ks, int tc);
const void* lane_ptr_d2(int ks, int tc);
const void* lane_ptr_d3(int ks, int tc);
const void* lane_ptr_d4(int ks, int tc);
const void* lane_ptr_d5(int ks, int tc);
const void* lane_ptr_d6(int ks, int tc);
const void* lane_ptr_d7(int ks, int tc);
const void* lane_ptr_d8(int ks, int tc);
cudaError_t launch_lanes(int d, int ks, int tc, const BatchArgs& a, int grid, cudaStream_t s);
cudaError_t launch_lane_stage(const LaneGroup* groups, int n_groups, int max_np, const int32_t* sorted_idx,
                              float2* tpart, int32_t* lane_rw, float* lane_ckey, const LaneXBlock* xblocks,
                              int n_xblocks, int64_t max_x, float* lane_x, int32_t* flags, cudaStream_t s);
cudaError_t launch_finalize_te(const InstDesc* insts, int n_inst, const double* partial,
                               const double* partial_abs, double psi_k, double err_coef,
                               double* te, double* err, cudaStream_t s);
cudaError_t launch_delay_argmax(const double* te, int n_u, int n_t, int u_lo, int32_t* u_best, cudaStream_t s);
cudaError_t launch_finalize_groups(const double* te_all, int n_groups, int S, double* te_orig,
                                   double* te_surr, double* p, cudaStream_t s);

}  // namespace te
