// Host side of the C ABI declared in te_gb300.h: argument validation, the batch plan
// (instance table, cost-ordered work items, launch shape), device workspace, the digamma
// table, CUDA-graph capture/replay and the measurement hooks. All arithmetic of the method
// runs in the kernels of te_unit.cu / te_batched_*.cu / te_finalize.cu.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <tuple>
#include <string>
#include <vector>

#include "te_internal.h"

#define TE_EXPORT extern "C" __attribute__((visibility("default")))

namespace {

using te::BatchArgs;
using te::BatchedVariant;
using te::InstDesc;
using te::WorkItem;

constexpr int kMaxN = 65536;          // largest point count of one estimate
constexpr int kMaxK = 16;
constexpr int kMaxD = 32;             // te_knn_maxnorm / te_range_count
constexpr int kMaxEmbedDim = 15;      // te_embed: D = 1 + 2d <= 31
constexpr int kMaxBatchedD = 8;       // te_estimate / te_surrogate_test / te_delay_scan
constexpr int kMaxMixedD = 5;         // largest d of a batch that mixes embedding dimensions
constexpr int kMaxBundleD = 5;        // target-part sharing
constexpr int kSmemCapBytes = 64 * 1024;  // reference tile budget of the batched kernel
constexpr int kSweepSmemMaxBytes = 160 * 1024;  // sweep mode: room for whole query blocks per tile
constexpr int64_t kResidentMaxBytes = 200 * 1024;  // sweep mode: whole instances in shared memory
// device word array: [0] batched-kernel queue, [1] flags, [2..3] bundle-kernel queues, one lane-kernel
// queue per (d, delay class) slot, then one queue per instance for per-instance launches
constexpr int kWordLaneQueue = 4;
constexpr int64_t kLaneXMaxBytes = (int64_t)16 << 30;  // member-minor source arrays of the lane kernel
constexpr int kWordPerInstance = kWordLaneQueue + te::kLaneSlots;

thread_local std::string g_create_error;  // per host thread: concurrent te_create calls do not race

// digamma at positive integers in FP64: -gamma + H_{n-1} below 16, the asymptotic expansion
// ln n - 1/(2n) - sum_k B_2k / (2k n^2k) (six terms, error < 1e-16) from 16 on
double digamma_int(int n) {
    if (n < 16) {
        double s = -0.57721566490153286060651209;
        for (int m = 1; m < n; ++m) s += 1.0 / m;
        return s;
    }
    const double x = n, r2 = 1.0 / (x * x);
    const double series =
        r2 * (1.0 / 12 - r2 * (1.0 / 120 - r2 * (1.0 / 252 - r2 * (1.0 / 240 - r2 * (1.0 / 132 - r2 * (691.0 / 32760))))));
    return std::log(x) - 0.5 / x - series;
}

template <class T>
struct DevBuf {
    T* p = nullptr;
    size_t n = 0;
    cudaError_t ensure(size_t want, bool* grew = nullptr) {
        if (want <= n) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
        size_t cap = std::max<size_t>(want, 64);
        cudaError_t e = cudaMalloc(&p, cap * sizeof(T));
        if (e != cudaSuccess) {
            p = nullptr;
            return e;
        }
        n = cap;
        if (grew) *grew = true;
        return cudaSuccess;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
};

template <class T>
struct HostBuf {  // pinned staging for asynchronous uploads
    T* p = nullptr;
    size_t n = 0;
    cudaError_t ensure(size_t want) {
        if (want <= n) return cudaSuccess;
        if (p) cudaFreeHost(p);
        p = nullptr;
        n = 0;
        size_t cap = std::max<size_t>(want, 64);
        cudaError_t e = cudaMallocHost(&p, cap * sizeof(T));
        if (e != cudaSuccess) {
            p = nullptr;
            return e;
        }
        n = cap;
        return cudaSuccess;
    }
    void release() {
        if (p) cudaFreeHost(p);
        p = nullptr;
        n = 0;
    }
};

struct Plan {
    std::vector<InstDesc> insts;  // caller order
    std::vector<WorkItem> items;  // cost order, items of an instance contiguous
    std::vector<te::SortGroup> groups;  // sweep mode: one sorted order per (series, start, window)
    int64_t sorted_total = 0;
    int64_t strip_total = 0;        // strip table entries (S + 1 per striped group)
    int nmax = 0;
    int n_parts = 0;                // partial sums (per CTA query block or per warp block)
    uint64_t exhaustive_pairs = 0;  // pair evaluations of the exhaustive search (both passes)
    uint64_t exhaustive_ops = 0;
    BatchedVariant var{};
    int threads = 0, grid = 0, smem_floats = 0;
    size_t smem = 0;
    double err_coef = 0;
    int64_t n_points = 0;
    // bundle kernel (target-part sharing): its work items, member lists, d and launch shape
    std::vector<WorkItem> bitems;  // resident bundles' items first (n_bres), then tiled bundles'
    std::vector<int32_t> members;
    int bd = 0, bgrid = 0, tgrid = 0, n_bundled = 0, n_bres = 0;
    size_t bsmem = 0, tsmem = 0;   // dynamic shared memory of the resident / tiled bundle launches
    // lane kernel (one estimate per lane): groups, their members, work items ordered by d
    // and delay class (items of slot s = (d - kLaneMinD) * kLaneTauClasses + class:
    // litems[lane_begin[s] .. lane_begin[s + 1] - 1]) and the grid per slot
    std::vector<te::LaneGroup> lgroups;
    std::vector<te::LaneItem> litems;
    std::vector<int32_t> lmembers;
    int64_t tp_total = 0;          // float2 entries of the sorted target parts
    int64_t rw_total = 0;          // entries of the (repetition, sample) tables
    int64_t ck_total = 0;          // entries of the chunk first-key tables
    std::vector<te::LaneXBlock> xblocks;
    int64_t x_total = 0, x_max = 0;  // floats of all / the largest member-minor source array
    int lane_max_np = 0;
    int lane_begin[te::kLaneSlots + 1] = {0};
    int lane_grid[te::kLaneSlots] = {0};
    int n_lane = 0;                // estimates on the lane kernel
    uint64_t table_hash = 0;  // of the device tables (instances, items, bundles): part of the graph key
};

struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// 64-bit hash of a byte range, eight bytes per step (FNV-style multiply with an extra shift mix)
uint64_t fnv(uint64_t h, const void* data, size_t n) {
    const unsigned char* c = static_cast<const unsigned char*>(data);
    size_t i = 0;
    for (; i + 8 <= n; i += 8) {
        uint64_t w;
        std::memcpy(&w, c + i, 8);
        h = (h ^ w) * 1099511628211ull;
        h ^= h >> 29;
    }
    for (; i < n; ++i) h = (h ^ c[i]) * 1099511628211ull;
    return h;
}

}  // namespace

struct te_handle {
    int device = 0;
    int sm_count = 0;
    std::string err;
    cudaStream_t cap_stream = nullptr;  // private stream used only for graph capture
    cudaEvent_t upload_done = nullptr;  // guards reuse of the pinned staging buffer
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    bool profiling = false, ev_recorded = false;
    int last_launches = 0;
    int cfg_threads = 0, cfg_qpt = 0;
    std::map<std::string, std::pair<int, int>> tuned;  // batch signature -> (threads, qpt)
    int tune_gen = 0;                                   // bumped whenever `tuned` changes
    bool per_instance = false;  // one launch per instance instead of one persistent launch
    int search_mode = 1;        // 1: sorted sweep where it applies, 0: exhaustive search
    int sharing = 1;            // 1: lanes and bundles, 2: bundles only, 0: no target-part sharing
    bool last_sweep = false;
    uint64_t last_pairs = 0, last_ops = 0;
    int last_bundled = 0;
    int last_paths[3] = {0, 0, 0};  // estimates on the lane kernel, in bundles, unshared

    DevBuf<InstDesc> d_insts;
    DevBuf<WorkItem> d_items;
    DevBuf<int32_t> d_words;  // [0] queue head, [1] flags
    DevBuf<double> d_partial, d_partial_abs, d_te_all, d_surr_ws, d_p_ws;
    DevBuf<float2> d_psi;
    DevBuf<te::SortGroup> d_groups;
    DevBuf<int32_t> d_sidx, d_sia, d_sib, d_strip_pos;
    DevBuf<float> d_skey, d_strip_k2;
    DevBuf<unsigned long long> d_sk64a, d_sk64b;
    DevBuf<unsigned long long> d_exec;
    DevBuf<WorkItem> d_bitems;
    DevBuf<int32_t> d_members;
    DevBuf<te::LaneGroup> d_lgroups;
    DevBuf<te::LaneItem> d_litems;
    DevBuf<int32_t> d_lmembers, d_lrw;
    DevBuf<float2> d_tpart;
    DevBuf<te::LaneXBlock> d_lxb;
    DevBuf<float> d_lx, d_lck;
    HostBuf<unsigned char> h_stage;
    int workspace_gen = 0;

    // the last plan and the exact inputs it was built from: an identical call reuses it
    std::vector<te_series> pc_series;
    std::vector<te_instance> pc_inst;
    std::vector<int> pc_cfg;
    bool pc_valid = false;
    Plan plan;

    uint64_t graph_key = 0;
    int graph_gen = -1;
    cudaGraphExec_t graph_exec = nullptr;
    int graph_launches = 0;

    te_status fail(te_status s, const char* fmt, ...) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        err = buf;
        return s;
    }
    te_status cuda_fail(cudaError_t e, const char* what) {
        return fail(TE_ECUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
    }
    void drop_graph() {
        if (graph_exec) cudaGraphExecDestroy(graph_exec);
        graph_exec = nullptr;
        graph_key = 0;
        graph_gen = -1;
    }
};

namespace {

te_status ensure_psi(te_handle* h) {
    if (h->d_psi.n >= (size_t)kMaxN + 2) return TE_OK;
    bool grew = false;
    cudaError_t e = h->d_psi.ensure((size_t)kMaxN + 2, &grew);
    if (e != cudaSuccess) return h->fail(TE_ENOMEM, "digamma table: %s", cudaGetErrorString(e));
    std::vector<float2> tab((size_t)kMaxN + 2);
    tab[0] = make_float2(0.f, 0.f);
    for (int n = 1; n < kMaxN + 2; ++n) {
        const double v = digamma_int(n);
        const float hi = (float)v;
        const float lo = (float)(v - (double)hi);
        tab[n] = make_float2(hi, lo);
    }
    e = cudaMemcpy(h->d_psi.p, tab.data(), tab.size() * sizeof(float2), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return h->cuda_fail(e, "digamma table upload");
    ++h->workspace_gen;
    return TE_OK;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// sample-index range of one estimate: target past reaches t_start-1-(d-1)tau, source past
// t_start-u-(d-1)tau, the window ends at t_start+W-1
bool embed_in_range(int T, int d, int tau, int u, int t_start, int W) {
    if (t_start < 0 || W < 1) return false;
    if ((int64_t)t_start + W - 1 > (int64_t)T - 1) return false;
    if ((int64_t)t_start - 1 - (int64_t)(d - 1) * tau < 0) return false;
    if ((int64_t)t_start - u - (int64_t)(d - 1) * tau < 0) return false;
    return true;
}

te_status validate_series(te_handle* h, const te_series* series, int n_series) {
    if (!series || n_series < 1) return h->fail(TE_EINVAL, "series: null or n_series < 1");
    for (int s = 0; s < n_series; ++s) {
        const te_series& S = series[s];
        if (!S.src || !S.tgt) return h->fail(TE_EINVAL, "series %d: null src/tgt", s);
        if (S.R < 1 || S.T < 1) return h->fail(TE_EINVAL, "series %d: R=%d T=%d", s, S.R, S.T);
        if (S.d < 1 || S.d > kMaxBatchedD)
            return h->fail(TE_ENOTIMPL, "series %d: d=%d outside 1..%d", s, S.d, kMaxBatchedD);
        if (S.tau < 1 || S.u < 0) return h->fail(TE_EINVAL, "series %d: tau=%d u=%d", s, S.tau, S.u);
        if (S.S < 0 || (S.S > 0 && !S.perms))
            return h->fail(TE_EINVAL, "series %d: S=%d with perms=%p", s, S.S, (const void*)S.perms);
        if ((int64_t)S.R * S.T > ((int64_t)1 << 40)) return h->fail(TE_EINVAL, "series %d too large", s);
    }
    return TE_OK;
}

// choose CTA size and queries per thread for a batch: 4 queries per thread (2 when d = 5 or
// k > 4, where 4 would not fit the register budget), and for a uniform point count the CTA size
// with the fewest padded query slots, ties to the smallest CTA of at least 128 threads (several
// CTAs per SM hide the per-item barriers)
// Signature of a batch for the autotuner's cache: embedding dimensions, top-k slots and the
// point count (exact when uniform, else the power-of-two bucket of the largest).
std::string shape_signature(const std::vector<InstDesc>& insts, int ks) {
    int dlo = 99, dhi = 0, nmax = 0;
    bool uniform = true;
    for (const auto& I : insts) {
        dlo = std::min(dlo, I.d);
        dhi = std::max(dhi, I.d);
        nmax = std::max(nmax, I.N);
        uniform &= I.N == insts[0].N;
    }
    int bucket = 1;
    while (bucket < nmax) bucket <<= 1;
    char buf[96];
    snprintf(buf, sizeof buf, "d%d-%d_ks%d_%s%d", dlo, dhi, ks, uniform ? "N" : "Nmax", uniform ? nmax : bucket);
    return buf;
}

void choose_shape(te_handle* h, const std::vector<InstDesc>& insts, int ks, int* threads, int* qpt) {
    int dmax = 1;
    for (const auto& I : insts) dmax = std::max(dmax, I.d);
    // the sweep prefers 2 (narrower key windows per warp, no register spills); d >= 6 runs one
    // query per thread
    int q = (ks == 5 && dmax <= 4 && h->search_mode == 0) ? 4 : 2;
    if (h->cfg_qpt) q = ks == 5 ? h->cfg_qpt : 2;
    if (q == 1) q = 2;  // d <= 5 has no one-query variant
    if (dmax > 5) q = 1;
    *qpt = q;
    if (h->cfg_threads) {
        *threads = h->cfg_threads;
        return;
    }
    if (!h->cfg_qpt) {
        auto it = h->tuned.find(shape_signature(insts, ks));
        if (it != h->tuned.end()) {
            *threads = it->second.first;
            *qpt = it->second.second;
            return;
        }
    }
    bool uniform = true;
    for (const auto& I : insts) uniform &= (I.N == insts[0].N);
    if (!uniform) {
        *threads = 256;
        return;
    }
    const int N = insts[0].N;
    int best_t = 0;
    int64_t best_slots = INT64_MAX;
    for (int t = 64; t <= te::kBatchedMaxThreads; t += 32) {
        const int64_t per = (int64_t)t * q;
        const int64_t slots = ((N + per - 1) / per) * per;
        const bool better = slots < best_slots ||
                            (slots == best_slots && best_t < 128 && t >= 128);
        if (better) {
            best_slots = slots;
            best_t = t;
        }
    }
    *threads = best_t;
}

te_status build_plan(te_handle* h, const te_series* series, int n_series, const te_instance* inst,
                     int n_inst, int k, Plan* P) {
    P->insts.resize(n_inst);
    int dlo = 99, dhi = 0, nmax = 0, dmaxN = 0;
    int64_t off = 0;
    for (int i = 0; i < n_inst; ++i) {
        const te_instance& in = inst[i];
        if (in.series < 0 || in.series >= n_series)
            return h->fail(TE_EINVAL, "instance %d: series %d out of range", i, in.series);
        const te_series& S = series[in.series];
        if (in.window < 1) return h->fail(TE_EINVAL, "instance %d: window %d", i, in.window);
        if (in.perm < -1 || in.perm >= S.S)
            return h->fail(TE_EINVAL, "instance %d: perm %d outside -1..%d", i, in.perm, S.S - 1);
        const int64_t N = (int64_t)S.R * in.window;
        if (N > kMaxN) return h->fail(TE_ENOTIMPL, "instance %d: N=%lld > %d", i, (long long)N, kMaxN);
        if (N < k + 1) return h->fail(TE_EINVAL, "instance %d: N=%lld < k+1=%d", i, (long long)N, k + 1);
        if (!embed_in_range(S.T, S.d, S.tau, S.u, in.t_start, in.window))
            return h->fail(TE_ERANGE, "instance %d: t_start=%d window=%d d=%d tau=%d u=%d outside 0..%d", i,
                           in.t_start, in.window, S.d, S.tau, S.u, S.T - 1);
        InstDesc& I = P->insts[i];
        I.src = S.src;
        I.tgt = S.tgt;
        I.perm = in.perm >= 0 ? S.perms + (size_t)in.perm * S.R : nullptr;
        I.R = S.R;
        I.T = S.T;
        I.W = in.window;
        I.t_start = in.t_start;
        I.tau = S.tau;
        I.u = S.u;
        I.d = S.d;
        I.N = (int)N;
        I.pt_off = off;
        off += N;
        dlo = std::min(dlo, S.d);
        dhi = std::max(dhi, S.d);
        nmax = std::max(nmax, (int)N);
        dmaxN = std::max(dmaxN, (int)(((N + 3) & ~3) * (1 + 2 * S.d)));
    }
    P->n_points = off;
    if (dlo != dhi && dhi > kMaxMixedD)
        return h->fail(TE_ENOTIMPL, "a batch that mixes embedding dimensions must have d <= %d (got %d..%d)",
                       kMaxMixedD, dlo, dhi);
    const int ks = k <= 4 ? 5 : 17;
    int threads, qpt;
    choose_shape(h, P->insts, ks, &threads, &qpt);
    // CTAs above kBatchedMaxThreads exist only for the warp-mode sweep kernel, decided once the
    // items are known: the items of tiled estimates are cut for the clamped size
    const int asked_threads = threads;
    threads = std::min(threads, te::kBatchedMaxThreads);
    P->var = BatchedVariant{dlo == dhi ? dlo : 1, dlo == dhi ? dhi : 5, ks, qpt};
    P->threads = threads;
    // work items: instances in descending cost (N^2 D), items of one instance contiguous
    std::vector<int> order(n_inst);
    for (int i = 0; i < n_inst; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        const InstDesc &A = P->insts[a], &B = P->insts[b];
        return (double)A.N * A.N * (1 + 2 * A.d) > (double)B.N * B.N * (1 + 2 * B.d);
    });
    const int per = threads * qpt;
    P->smem_floats = std::min(kSmemCapBytes / 4, dmaxN);
    P->smem_floats = std::max(P->smem_floats, 4 * 11);
    P->nmax = nmax;
    // sweep mode: every instance must either fit one tile or leave room for a whole CTA query
    // block per tile (its queries then lie in one tile)
    bool sweep = h->search_mode == 1 && nmax <= te::kSweepMaxN;
    if (sweep) {
        // every instance resident in shared memory (up to kResidentMaxBytes) when it fits there,
        // which lets warps balance the work; otherwise tiles of whole CTA query blocks
        if ((int64_t)dmaxN * (int64_t)sizeof(float) <= kResidentMaxBytes) {
            P->smem_floats = std::max(P->smem_floats, dmaxN);
        } else {
            int need = P->smem_floats;
            for (const auto& I : P->insts) {
                const int D = 1 + 2 * I.d;
                if ((int64_t)((I.N + 3) & ~3) * D > P->smem_floats) need = std::max(need, per * D);
            }
            if (need * (int)sizeof(float) > kSweepSmemMaxBytes) sweep = false;
            else P->smem_floats = need;
        }
    }
    P->var.sweep = sweep;
    P->smem = (size_t)P->smem_floats * sizeof(float);
    for (const auto& I : P->insts) {
        P->exhaustive_pairs += 2ull * (uint64_t)I.N * (uint64_t)I.N;
        P->exhaustive_ops += 2ull * (uint64_t)I.N * (uint64_t)I.N * 2ull * (uint64_t)(1 + 2 * I.d);
    }
    // work items (cost order, an instance's items contiguous) and partial-sum ranges: an instance
    // that the sweep keeps whole in shared memory is one item whose warps each produce one part
    // per block of 32 * qpt queries; any other instance has one part per CTA query block
    P->items.clear();
    // warp mode splits an instance into several items when the batch alone would not give every
    // SM a few items (each item stages the instance and takes a share of its warp blocks)
    const int want_items = 4 * h->sm_count;
    int max_parts = 1;
    int n_parts = 0;
    // one estimate per lane: groups of at least kLaneMinMembers estimates with one target part
    // (target series, repetitions, window start, window, d, tau) and d in kLaneMinD .. kLaneMaxD;
    // each member has one partial sum per block of kLaneQB sorted query positions. Blocks of 32
    // members read their source part from member-minor arrays (LaneXBlock), shared by blocks with
    // the same source series and pairings; past kLaneXMaxBytes of such arrays no lanes are used.
    std::vector<char> laned(n_inst, 0);
    if (sweep && (h->sharing == 1 || h->sharing == 3) && !h->per_instance && ks == 5) {
        const bool all_lanes = h->sharing == 3;
        typedef std::tuple<const float*, int, int, int, int, int, int> TK;
        std::map<TK, std::vector<int>> by_target;
        std::vector<TK> korder;
        for (int i = 0; i < n_inst; ++i) {
            const InstDesc& I = P->insts[i];
            if (I.d < te::kLaneMinD || I.d > te::kLaneMaxD) continue;
            const TK key = std::make_tuple(I.tgt, I.T, I.R, I.t_start, I.W, I.d, I.tau);
            auto f = by_target.find(key);
            if (f == by_target.end()) {
                korder.push_back(key);
                f = by_target.emplace(key, std::vector<int>()).first;
            }
            f->second.push_back(i);
        }
        // X blocks: one per distinct (R, T, the 32 lanes' source series and pairings), columns the
        // union of the samples its groups read
        std::vector<te::LaneXBlock> xb;
        std::map<std::vector<uintptr_t>, int> xsig;
        std::vector<std::vector<int>> cand;     // member lists of the lane groups
        std::vector<std::vector<int>> cand_xb;  // their blocks' X block
        for (const auto& key : korder) {
            const std::vector<int>& v = by_target[key];
            if ((int)v.size() < (all_lanes ? te::kLaneMinMembers : te::kLaneAutoMembers)) continue;
            if (!all_lanes && P->insts[v[0]].d < te::kLaneAutoMinD) continue;
            std::vector<int> blocks;
            for (size_t b = 0; b * 32 < v.size(); ++b) {
                std::vector<uintptr_t> sig;
                const InstDesc& I0 = P->insts[v[0]];
                sig.push_back((uintptr_t)I0.R);
                sig.push_back((uintptr_t)I0.T);
                int cmin = INT32_MAX, cmax = INT32_MIN;
                for (int l = 0; l < 32; ++l) {
                    const InstDesc& I = P->insts[v[std::min(v.size() - 1, b * 32 + (size_t)l)]];
                    sig.push_back((uintptr_t)I.src);
                    sig.push_back((uintptr_t)I.perm);
                    cmin = std::min(cmin, I.t_start - I.u - (I.d - 1) * I.tau);
                    cmax = std::max(cmax, I.t_start + I.W - 1 - I.u);
                }
                auto f = xsig.find(sig);
                if (f == xsig.end()) {
                    te::LaneXBlock X{};
                    X.R = I0.R;
                    X.T = I0.T;
                    X.t0 = cmin;
                    X.ncols = cmax - cmin + 1;
                    for (int l = 0; l < 32; ++l) {
                        const InstDesc& I = P->insts[v[std::min(v.size() - 1, b * 32 + (size_t)l)]];
                        X.src[l] = I.src;
                        X.perm[l] = I.perm;
                    }
                    f = xsig.emplace(sig, (int)xb.size()).first;
                    xb.push_back(X);
                } else {
                    te::LaneXBlock& X = xb[f->second];
                    const int hi = std::max(X.t0 + X.ncols - 1, cmax);
                    X.t0 = std::min(X.t0, cmin);
                    X.ncols = hi - X.t0 + 1;
                }
                blocks.push_back(f->second);
            }
            cand.push_back(v);
            cand_xb.push_back(blocks);
        }
        int64_t xtotal = 0, xmax = 0;
        for (auto& X : xb) {
            X.off = xtotal;
            const int64_t n = (int64_t)X.R * X.ncols * 32;
            xtotal += n;
            xmax = std::max(xmax, n);
        }
        // the kernel indexes one array with 32-bit offsets
        if (xtotal * (int64_t)sizeof(float) > kLaneXMaxBytes || xmax >= ((int64_t)1 << 31)) cand.clear();
        for (size_t g = 0; g < cand.size(); ++g) {
            const std::vector<int>& v = cand[g];
            const InstDesc& I0 = P->insts[v[0]];
            te::LaneGroup G{};
            G.tgt = I0.tgt;
            G.R = I0.R;
            G.T = I0.T;
            G.W = I0.W;
            G.t_start = I0.t_start;
            G.N = I0.N;
            G.d = I0.d;
            G.tau = I0.tau;
            G.mem_off = (int)P->lmembers.size();
            G.n_mem = (int)v.size();
            const int NP = (I0.N + 31) & ~31;
            G.tp_off = P->tp_total;
            P->tp_total += (int64_t)((I0.d + 2) / 2) * NP;
            G.rw_off = P->rw_total;
            P->rw_total += NP;
            G.ck_off = P->ck_total;
            P->ck_total += NP / 32;
            P->lane_max_np = std::max(P->lane_max_np, NP);
            const int nqb = (I0.N + te::kLaneQB - 1) / te::kLaneQB;
            for (int i : v) {
                InstDesc& I = P->insts[i];
                P->lmembers.push_back(i);
                laned[i] = 1;
                I.item_begin = 0;
                I.n_items = 0;
                I.warp_mode = 0;
                I.part_begin = n_parts;
                I.n_parts = nqb;
                n_parts += nqb;
                max_parts = std::max(max_parts, nqb);
            }
            P->lgroups.push_back(G);
            P->n_lane += (int)v.size();
        }
        if (!cand.empty()) {
            P->xblocks = xb;
            P->x_total = xtotal;
            P->x_max = xmax;
        }
        for (int slot = 0; slot < te::kLaneSlots; ++slot) {
            const int d = te::kLaneMinD + slot / te::kLaneTauClasses, tc = slot % te::kLaneTauClasses;
            P->lane_begin[slot] = (int)P->litems.size();
            for (int g = 0; g < (int)P->lgroups.size(); ++g) {
                const te::LaneGroup& G = P->lgroups[g];
                if (G.d != d || te::lane_tau_class(G.tau) != tc) continue;
                for (int mb = 0; mb * 32 < G.n_mem; ++mb)
                    for (int q0 = 0; q0 < G.N; q0 += te::kLaneQB)
                        P->litems.push_back(te::LaneItem{g, mb, q0, cand_xb[g][mb]});
            }
        }
        P->lane_begin[te::kLaneSlots] = (int)P->litems.size();
    }
    // target-part sharing: estimates with one target part (target series, repetitions, window
    // start, window, d, tau) form bundles of up to kBundleMax (no bundle of one), processed by the
    // bundle kernel; one embedding dimension per batch. A bundle that fits kResidentMaxBytes is
    // staged whole (warps take 32-query blocks); a larger one runs CTA tiles around blocks of
    // kBundleThreads queries (tile budget: three CTAs per SM for d <= 3, two above), but only when
    // its estimates would not be resident on their own either (a resident unshared estimate beats
    // a tiled bundle: the AR(1) scan measured 317 ms unshared vs 450 ms tiled-bundled)
    std::vector<char> bundled(n_inst, 0);
    std::vector<int> tiled_leaders;  // leaders of bundles too large to stage whole
    if (sweep && h->sharing && !h->per_instance && ks == 5) {
        std::map<std::tuple<const float*, int, int, int, int, int, int>, std::vector<int>> by_target;
        for (int i = 0; i < n_inst; ++i) {
            const InstDesc& I = P->insts[i];
            if (laned[i]) continue;
            by_target[std::make_tuple(I.tgt, I.T, I.R, I.t_start, I.W, I.d, I.tau)].push_back(i);
        }
        auto resident_bytes = [](const InstDesc& I) {
            return (int64_t)((I.N + 3) & ~3) * (1 + I.d + te::kBundleMax * I.d) * 4;
        };
        auto shares = [&](const InstDesc& I) {  // a bundle of I's group is staged whole or helps tiled
            return resident_bytes(I) <= kResidentMaxBytes ||
                   (int64_t)((I.N + 3) & ~3) * (1 + 2 * I.d) * 4 > kResidentMaxBytes;
        };
        int64_t shareable[kMaxBatchedD + 1] = {0};  // estimates in groups of >= 2 that share, per d
        for (const auto& kv : by_target)
            if (kv.second.size() >= 2 && shares(P->insts[kv.second[0]]))
                shareable[P->insts[kv.second[0]].d] += (int64_t)kv.second.size();
        for (int d = 1; d <= kMaxBundleD; ++d)
            if (shareable[d] > (P->bd ? shareable[P->bd] : 0)) P->bd = d;
        int n_bundles = 0;  // resident ones, for their work split
        for (const auto& kv : by_target) {
            const InstDesc& I0 = P->insts[kv.second[0]];
            if (kv.second.size() < 2 || I0.d != P->bd || !shares(I0)) continue;
            if (resident_bytes(I0) <= kResidentMaxBytes) {
                P->bsmem = std::max(P->bsmem, (size_t)resident_bytes(I0));
                n_bundles += (int)((kv.second.size() + te::kBundleMax - 1) / te::kBundleMax);
            }
        }
        const int per_b = 32 * te::kBundleQ;
        for (const auto& kv : by_target) {
            const std::vector<int>& v = kv.second;
            const InstDesc& I0 = P->insts[v[0]];
            if (v.size() < 2 || I0.d != P->bd || !shares(I0)) continue;
            const bool resident = resident_bytes(I0) <= kResidentMaxBytes;
            int nparts_b = 0, chunk = 0;
            if (resident) {
                const int nwb = (I0.N + per_b - 1) / per_b;
                const int split = std::max(1, std::min(nwb, (want_items + n_bundles - 1) / std::max(1, n_bundles)));
                chunk = (nwb + split - 1) / split;
                nparts_b = nwb;
            } else {  // tiles of at least one strip (kStripPoints) of the bundle
                const int cols = 1 + I0.d + te::kBundleMax * I0.d;
                const int budget = I0.d <= 3 ? 72 * 1024 : 110 * 1024;
                const int blockq = te::kBundleThreads * te::kBundleQ;
                const int cap = std::max(te::kStripPoints, (budget / (cols * 4)) / blockq * blockq);
                P->tsmem = std::max(P->tsmem, (size_t)cap * cols * 4);
            }
            size_t pos = 0;
            while (pos < v.size()) {
                size_t nb = std::min<size_t>(te::kBundleMax, v.size() - pos);
                if (v.size() - pos - nb == 1) nb -= 1;  // leave two for the last bundle, not one
                InstDesc& L = P->insts[v[pos]];
                L.bundle_n = (int)nb;
                L.bundle_off = (int)P->members.size();
                L.wb_chunk = chunk;
                for (size_t m = 0; m < nb; ++m) {
                    const int i = v[pos + m];
                    InstDesc& I = P->insts[i];
                    P->members.push_back(i);
                    bundled[i] = 1;
                    I.warp_mode = resident ? 1 : 0;
                    I.item_begin = 0;
                    I.n_items = 0;
                    if (resident) {
                        I.part_begin = n_parts;
                        I.n_parts = nparts_b;
                        n_parts += nparts_b;
                        max_parts = std::max(max_parts, nparts_b);
                    }
                }
                if (resident) {
                    for (int c = 0; c * chunk < nparts_b; ++c) P->bitems.push_back(WorkItem{v[pos], c * chunk});
                } else {
                    tiled_leaders.push_back(v[pos]);  // parts and items once the sort groups are known
                }
                pos += nb;
                ++P->n_bundled;
            }
        }
        P->n_bres = (int)P->bitems.size();
    }
    // warp mode of every unshared estimate: staged whole when it fits shared memory
    for (int i = 0; i < n_inst; ++i) {
        InstDesc& I = P->insts[i];
        I.strips = 1;
        I.npad = I.N;
        I.strip_off = 0;
        if (bundled[i] || laned[i]) continue;
        const bool fits = (int64_t)((I.N + 3) & ~3) * (1 + 2 * I.d) <= P->smem_floats;
        I.warp_mode = (sweep && fits) ? 1 : 0;
    }
    // sort groups: one per (target series, repetitions, window start, window); a group whose every
    // estimate takes a strip-aware path and agrees on the second key is cut into strips
    if (sweep) {
        std::map<std::tuple<const float*, int, int, int, int>, std::vector<int>> gmem;
        std::vector<std::tuple<const float*, int, int, int, int>> gorder;
        for (int i = 0; i < n_inst; ++i) {
            const InstDesc& I = P->insts[i];
            auto key = std::make_tuple(I.tgt, I.T, I.R, I.t_start, I.W);
            auto f = gmem.find(key);
            if (f == gmem.end()) {
                gorder.push_back(key);
                f = gmem.emplace(key, std::vector<int>()).first;
            }
            f->second.push_back(i);
        }
        int64_t strip_total = 0;
        for (const auto& key : gorder) {
            const std::vector<int>& v = gmem[key];
            const InstDesc& I0 = P->insts[v[0]];
            const int N = I0.N;
            const int k2lag = I0.d >= 2 ? 1 + I0.tau : 0;
            // estimates that can take strips: staged whole (alone or bundled), tiled bundles, and
            // tiled estimates whose CTA block divides a strip; all agreeing on the second key
            bool ok = true;
            for (int i : v) {
                const InstDesc& I = P->insts[i];
                const int lag = I.d >= 2 ? 1 + I.tau : 0;
                const bool resident_alone = !bundled[i] && I.warp_mode == 1;
                const bool resident_bundle = bundled[i] && I.warp_mode == 1 && I.d <= 2;
                const bool tiled_bundle = bundled[i] && I.warp_mode == 0;
                const bool tiled_alone = !bundled[i] && I.warp_mode == 0 && te::kStripPoints % per == 0 &&
                                         (int64_t)te::kStripPoints * (1 + 2 * I.d) * 4 <= kSweepSmemMaxBytes;
                // the lane kernel sweeps strips too (its estimates have d >= 2: the second key is in y-)
                if (lag != k2lag || !(laned[i] || resident_alone || resident_bundle || tiled_bundle || tiled_alone))
                    ok = false;
            }
            // strips of kStripPoints, for groups of 4 strips or more (shorter strips were measured
            // slower: a C3 group of 1200 points in 4 strips took 66.7 ms instead of 46.9 ms; the
            // own strip then yields poor first radii)
            const int L = te::kStripPoints;
            int S = (ok && N >= 4 * L) ? std::min(te::kMaxStrips, (N + L - 1) / L) : 1;
            const int npad = S > 1 ? ((N + 3) & ~3) : N;
            te::SortGroup G{I0.tgt, I0.R, I0.T, I0.W, I0.t_start, N, S, npad, k2lag, S > 1 ? L : 0, 0,
                            P->sorted_total, S > 1 ? strip_total : 0};
            P->groups.push_back(G);
            for (int i : v) {
                InstDesc& I = P->insts[i];
                I.sort_off = P->sorted_total;
                I.strips = S;
                I.npad = npad;
                I.strip_off = G.strip_off;
                // a tiled estimate over strips stages a whole strip per tile
                if (S > 1 && !bundled[i] && !laned[i] && I.warp_mode == 0)
                    P->smem_floats = std::max(P->smem_floats, te::kStripPoints * (1 + 2 * I.d));
            }
            P->sorted_total += npad;
            if (S > 1) strip_total += S + 1;
        }
        P->strip_total = strip_total;
        for (auto& G : P->lgroups) {
            const InstDesc& I = P->insts[P->lmembers[G.mem_off]];
            G.sort_off = I.sort_off;
            G.strips = I.strips;
            G.npad = I.npad;
            G.strip_off = I.strip_off;
        }
    }
    // tiled bundles: one work item per block of kBundleThreads * kBundleQ sorted positions
    {
        const int blockq = te::kBundleThreads * te::kBundleQ;
        for (int leader : tiled_leaders) {
            const InstDesc& L = P->insts[leader];
            const int nparts_b = (L.npad + blockq - 1) / blockq;
            for (int m = 0; m < L.bundle_n; ++m) {
                InstDesc& I = P->insts[P->members[L.bundle_off + m]];
                I.part_begin = n_parts;
                I.n_parts = nparts_b;
                n_parts += nparts_b;
                max_parts = std::max(max_parts, nparts_b);
            }
            for (int c = 0; c < nparts_b; ++c) P->bitems.push_back(WorkItem{leader, c * blockq});
        }
    }
    // work items of the unshared estimates (cost order, an estimate's items contiguous) and their
    // partial-sum ranges: a staged-whole estimate is cut into items of warp blocks (32 * qpt
    // sorted positions), any other into CTA query blocks
    for (int i : order) {
        if (bundled[i] || laned[i]) continue;
        InstDesc& I = P->insts[i];
        I.item_begin = (int)P->items.size();
        I.part_begin = n_parts;
        if (I.warp_mode) {
            const int nwb = (I.npad + 32 * qpt - 1) / (32 * qpt);
            const int split = std::max(1, std::min(nwb, (want_items + n_inst - 1) / n_inst));
            I.wb_chunk = (nwb + split - 1) / split;
            I.n_items = (nwb + I.wb_chunk - 1) / I.wb_chunk;
            I.n_parts = nwb;
            for (int m = 0; m < I.n_items; ++m) P->items.push_back(WorkItem{i, m * I.wb_chunk});
        } else {
            I.n_items = (I.npad + per - 1) / per;
            I.n_parts = I.n_items;
            for (int m = 0; m < I.n_items; ++m) P->items.push_back(WorkItem{i, m * per});
        }
        n_parts += I.n_parts;
        max_parts = std::max(max_parts, I.n_parts);
    }
    P->n_parts = n_parts;
    P->smem = (size_t)P->smem_floats * sizeof(float);
    // every unshared estimate staged whole with one d <= 2: the warp-mode sweep kernel (1024-thread
    // CTAs unless a shape was set or tuned for this signature)
    bool all_warp = !P->items.empty();
    for (int i = 0; i < n_inst; ++i)
        if (!bundled[i] && !laned[i] && !P->insts[i].warp_mode) all_warp = false;
    if (sweep && !h->per_instance && all_warp && dlo == dhi && dlo <= 2 && ks == 5) {
        P->var.warp_only = true;
        const bool shaped = h->cfg_threads || h->tuned.find(shape_signature(P->insts, ks)) != h->tuned.end();
        threads = shaped ? asked_threads : te::kSweepWarpThreads;
    }
    P->threads = threads;
    // bound on the summation error relative to sum |terms| (see te_estimate in the header):
    // 3*qpt float-float additions per thread (<= 2^-46 each), table rounding (2^-47), FP64
    // reductions over threads and items
    // (a lane of the lane kernel adds 3 terms per query for kLaneQB / kLaneWarps queries)
    const int ff_terms = std::max(3 * qpt, P->n_lane ? 3 * (te::kLaneQB / te::kLaneWarps) : 0);
    P->err_coef = ff_terms * 0x1p-46 + 0x1p-47 + (threads + max_parts + 64) * 0x1p-52;
    const void* fn = te::batched_kernel_ptr(P->var);
    if (!fn) return h->fail(TE_ENOTIMPL, "no kernel variant for d=%d..%d ks=%d qpt=%d", dlo, dhi, ks, qpt);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P->smem);
    if (e != cudaSuccess) return h->cuda_fail(e, "cudaFuncSetAttribute");
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, P->smem);
    if (e != cudaSuccess) return h->cuda_fail(e, "occupancy query");
    if (per_sm < 1) return h->fail(TE_ENOTIMPL, "batched kernel does not fit: threads=%d smem=%zu", threads, P->smem);
    P->grid = (int)std::min<int64_t>((int64_t)per_sm * h->sm_count, (int64_t)P->items.size());
    for (int tiled = 0; tiled < 2; ++tiled) {
        const int64_t n = tiled ? (int64_t)P->bitems.size() - P->n_bres : (int64_t)P->n_bres;
        if (n <= 0) continue;
        const size_t smem = tiled ? P->tsmem : P->bsmem;
        const void* bf = te::bundle_kernel_ptr(P->bd, ks, tiled != 0);
        if (!bf) return h->fail(TE_ENOTIMPL, "no bundle kernel for d=%d ks=%d", P->bd, ks);
        if ((e = cudaFuncSetAttribute(bf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
            return h->cuda_fail(e, "cudaFuncSetAttribute (bundle)");
        int bper = 0;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bper, bf, te::kBundleThreads, smem)) != cudaSuccess)
            return h->cuda_fail(e, "occupancy query (bundle)");
        if (bper < 1) return h->fail(TE_ENOTIMPL, "bundle kernel does not fit: smem=%zu", smem);
        (tiled ? P->tgrid : P->bgrid) = (int)std::min<int64_t>((int64_t)bper * h->sm_count, n);
    }
    for (int slot = 0; slot < te::kLaneSlots; ++slot) {
        const int d = te::kLaneMinD + slot / te::kLaneTauClasses, tc = slot % te::kLaneTauClasses;
        const int n = P->lane_begin[slot + 1] - P->lane_begin[slot];
        if (n <= 0) continue;
        const void* lf = te::lane_kernel_ptr(d, ks, tc);
        if (!lf) return h->fail(TE_ENOTIMPL, "no lane kernel for d=%d ks=%d delay class %d", d, ks, tc);
        int lper = 0;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&lper, lf, te::kLaneThreads, 0)) != cudaSuccess)
            return h->cuda_fail(e, "occupancy query (lanes)");
        if (lper < 1) return h->fail(TE_ENOTIMPL, "lane kernel does not fit");
        P->lane_grid[slot] = (int)std::min<int64_t>((int64_t)lper * h->sm_count, n);
    }
    uint64_t th = 1469598103934665603ull;
    th = fnv(th, P->insts.data(), P->insts.size() * sizeof(InstDesc));
    th = fnv(th, P->items.data(), P->items.size() * sizeof(WorkItem));
    th = fnv(th, P->bitems.data(), P->bitems.size() * sizeof(WorkItem));
    th = fnv(th, P->members.data(), P->members.size() * sizeof(int32_t));
    th = fnv(th, P->lgroups.data(), P->lgroups.size() * sizeof(te::LaneGroup));
    th = fnv(th, P->litems.data(), P->litems.size() * sizeof(te::LaneItem));
    th = fnv(th, P->lmembers.data(), P->lmembers.size() * sizeof(int32_t));
    th = fnv(th, P->xblocks.data(), P->xblocks.size() * sizeof(te::LaneXBlock));
    P->table_hash = th;
    (void)nmax;
    return TE_OK;
}

// The handle's plan for this batch: reused when the series array, the instances, k and every
// setting that shapes a plan equal those of the previous call byte for byte, else rebuilt.
te_status cached_plan(te_handle* h, const te_series* series, int n_series, const te_instance* inst, int n_inst,
                      int k, Plan** out) {
    std::vector<int> cfg = {k, h->search_mode, h->sharing, h->per_instance ? 1 : 0, h->cfg_threads,
                            h->cfg_qpt, h->tune_gen, h->sm_count};
    const bool hit = h->pc_valid && h->pc_cfg == cfg && (int)h->pc_series.size() == n_series &&
                     (int)h->pc_inst.size() == n_inst &&
                     std::memcmp(h->pc_series.data(), series, sizeof(te_series) * (size_t)n_series) == 0 &&
                     std::memcmp(h->pc_inst.data(), inst, sizeof(te_instance) * (size_t)n_inst) == 0;
    if (!hit) {
        h->pc_valid = false;
        h->plan = Plan();
        te_status st = build_plan(h, series, n_series, inst, n_inst, k, &h->plan);
        if (st != TE_OK) return st;
        h->pc_series.assign(series, series + n_series);
        h->pc_inst.assign(inst, inst + n_inst);
        h->pc_cfg = cfg;
        h->pc_valid = true;
    }
    *out = &h->plan;
    return TE_OK;
}

// Upload the plan's tables (pinned staging -> device on `stream`).
te_status upload_tables(te_handle* h, const Plan& P, cudaStream_t stream) {
    const size_t bi = P.insts.size() * sizeof(InstDesc), bt = P.items.size() * sizeof(WorkItem);
    const size_t bg = P.groups.size() * sizeof(te::SortGroup);
    const size_t bb = P.bitems.size() * sizeof(WorkItem), bm = P.members.size() * sizeof(int32_t);
    const size_t blg = P.lgroups.size() * sizeof(te::LaneGroup), bli = P.litems.size() * sizeof(te::LaneItem);
    const size_t blm = P.lmembers.size() * sizeof(int32_t), blx = P.xblocks.size() * sizeof(te::LaneXBlock);
    const size_t ol = bi + bt + bg + bb + bm;  // lane tables follow (8-byte aligned: every size above is)
    cudaError_t e;
    if ((e = cudaEventSynchronize(h->upload_done)) != cudaSuccess) return h->cuda_fail(e, "staging reuse");
    if ((e = h->h_stage.ensure(ol + blg + bli + blm + blx + 64)) != cudaSuccess)
        return h->fail(TE_ENOMEM, "pinned staging");
    unsigned char* hs = h->h_stage.p;
    std::memcpy(hs, P.insts.data(), bi);
    if (bt) std::memcpy(hs + bi, P.items.data(), bt);
    if (bg) std::memcpy(hs + bi + bt, P.groups.data(), bg);
    if (bb) std::memcpy(hs + bi + bt + bg, P.bitems.data(), bb);
    if (bm) std::memcpy(hs + bi + bt + bg + bb, P.members.data(), bm);
    const size_t olg = (ol + 7) & ~(size_t)7, oli = olg + blg, olm = oli + bli, olx = (olm + blm + 7) & ~(size_t)7;
    if (blg) std::memcpy(hs + olg, P.lgroups.data(), blg);
    if (bli) std::memcpy(hs + oli, P.litems.data(), bli);
    if (blm) std::memcpy(hs + olm, P.lmembers.data(), blm);
    if (blx) std::memcpy(hs + olx, P.xblocks.data(), blx);
    if ((blg && (e = cudaMemcpyAsync(h->d_lgroups.p, hs + olg, blg, cudaMemcpyHostToDevice, stream)) != cudaSuccess) ||
        (bli && (e = cudaMemcpyAsync(h->d_litems.p, hs + oli, bli, cudaMemcpyHostToDevice, stream)) != cudaSuccess) ||
        (blm && (e = cudaMemcpyAsync(h->d_lmembers.p, hs + olm, blm, cudaMemcpyHostToDevice, stream)) != cudaSuccess) ||
        (blx && (e = cudaMemcpyAsync(h->d_lxb.p, hs + olx, blx, cudaMemcpyHostToDevice, stream)) != cudaSuccess))
        return h->cuda_fail(e, "lane table upload");
    if ((e = cudaMemcpyAsync(h->d_insts.p, hs, bi, cudaMemcpyHostToDevice, stream)) != cudaSuccess ||
        (bt && (e = cudaMemcpyAsync(h->d_items.p, hs + bi, bt, cudaMemcpyHostToDevice, stream)) != cudaSuccess) ||
        (bg && (e = cudaMemcpyAsync(h->d_groups.p, hs + bi + bt, bg, cudaMemcpyHostToDevice, stream)) !=
                   cudaSuccess) ||
        (bb && (e = cudaMemcpyAsync(h->d_bitems.p, hs + bi + bt + bg, bb, cudaMemcpyHostToDevice, stream)) !=
                   cudaSuccess) ||
        (bm && (e = cudaMemcpyAsync(h->d_members.p, hs + bi + bt + bg + bb, bm, cudaMemcpyHostToDevice, stream)) !=
                   cudaSuccess) ||
        (e = cudaEventRecord(h->upload_done, stream)) != cudaSuccess)
        return h->cuda_fail(e, "table upload");
    return TE_OK;
}

// sweep mode: workspace for the sorted orders and the work counters, the sort kernel's limit
te_status prepare_sweep(te_handle* h, const Plan& P, bool* grew) {
    if (!P.var.sweep) return TE_OK;
    cudaError_t e;
    if ((e = h->d_groups.ensure(P.groups.size(), grew)) != cudaSuccess ||
        (e = h->d_sidx.ensure((size_t)P.sorted_total, grew)) != cudaSuccess ||
        (e = h->d_skey.ensure((size_t)P.sorted_total, grew)) != cudaSuccess ||
        (e = h->d_exec.ensure(6, grew)) != cudaSuccess ||
        (e = h->d_bitems.ensure(P.bitems.size(), grew)) != cudaSuccess ||
        (e = h->d_members.ensure(P.members.size(), grew)) != cudaSuccess)
        return h->fail(TE_ENOMEM, "sweep workspace: %s", cudaGetErrorString(e));
    if ((e = h->d_sia.ensure((size_t)P.sorted_total, grew)) != cudaSuccess ||
        (e = h->d_sib.ensure((size_t)P.sorted_total, grew)) != cudaSuccess ||
        (e = h->d_sk64a.ensure((size_t)P.sorted_total, grew)) != cudaSuccess ||
        (e = h->d_sk64b.ensure((size_t)P.sorted_total, grew)) != cudaSuccess ||
        (e = h->d_strip_pos.ensure((size_t)std::max<int64_t>(1, P.strip_total), grew)) != cudaSuccess ||
        (e = h->d_strip_k2.ensure((size_t)std::max<int64_t>(2, 2 * P.strip_total), grew)) != cudaSuccess)
        return h->fail(TE_ENOMEM, "sort scratch: %s", cudaGetErrorString(e));
    if ((e = te::prepare_sort_kernel(P.nmax)) != cudaSuccess) return h->cuda_fail(e, "sort kernel attribute");
    if (!P.lgroups.empty()) {
        if ((e = h->d_lgroups.ensure(P.lgroups.size(), grew)) != cudaSuccess ||
            (e = h->d_litems.ensure(P.litems.size(), grew)) != cudaSuccess ||
            (e = h->d_lmembers.ensure(P.lmembers.size(), grew)) != cudaSuccess ||
            (e = h->d_tpart.ensure((size_t)P.tp_total, grew)) != cudaSuccess ||
            (e = h->d_lrw.ensure((size_t)P.rw_total, grew)) != cudaSuccess ||
            (e = h->d_lxb.ensure(P.xblocks.size(), grew)) != cudaSuccess ||
            (e = h->d_lx.ensure((size_t)P.x_total, grew)) != cudaSuccess ||
            (e = h->d_lck.ensure((size_t)P.ck_total, grew)) != cudaSuccess)
            return h->fail(TE_ENOMEM, "lane workspace: %s", cudaGetErrorString(e));
    }
    return TE_OK;
}

// the sweep's pre-pass (work counters cleared, groups sorted) on `s`
cudaError_t launch_sweep_prepass(te_handle* h, const Plan& P, cudaStream_t s) {
    if (!P.var.sweep) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(h->d_exec.p, 0, 6 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    return te::launch_sort_groups(h->d_groups.p, (int)P.groups.size(), h->d_sidx.p, h->d_skey.p, h->d_sk64a.p,
                                  h->d_sia.p, h->d_sk64b.p, h->d_sib.p, h->d_strip_pos.p, h->d_strip_k2.p, s);
}

BatchArgs batch_args(te_handle* h, const Plan& P, int k, int32_t* counts, float* eps) {
    BatchArgs a{};
    a.insts = h->d_insts.p;
    a.items = h->d_items.p;
    a.n_items = (int)P.items.size();
    a.item_base = 0;
    a.queue = h->d_words.p;
    a.flags = h->d_words.p + 1;
    a.psi = h->d_psi.p;
    a.k = k;
    a.smem_floats = P.smem_floats;
    a.partial = h->d_partial.p;
    a.partial_abs = h->d_partial_abs.p;
    a.counts_out = counts;
    a.eps_out = eps;
    if (P.var.sweep) {
        a.sorted_idx = h->d_sidx.p;
        a.sorted_key = h->d_skey.p;
        a.exec = h->d_exec.p;
        a.members = h->d_members.p;
        a.strip_pos = h->d_strip_pos.p;
        a.strip_k2 = h->d_strip_k2.p;
        if (!P.lgroups.empty()) {
            a.lgroups = h->d_lgroups.p;
            a.litems = h->d_litems.p;
            a.tpart = h->d_tpart.p;
            a.lane_rw = h->d_lrw.p;
            a.lane_members = h->d_lmembers.p;
            a.lane_xb = h->d_lxb.p;
            a.lane_x = h->d_lx.p;
            a.lane_ckey = h->d_lck.p;
        }
    }
    return a;
}

// The unbatched baseline: the same kernel and tables, but one launch per instance (its grid is
// that instance's work items, its queue counter its own), launched directly without a graph.
te_status run_per_instance(te_handle* h, const Plan& P, int n_inst, int k, double* te_dst, double* err,
                           int32_t* counts, float* eps, int n_groups, int S, double* te_orig,
                           double* te_surr, double* p, cudaStream_t stream) {
    te_status st = upload_tables(h, P, stream);
    if (st != TE_OK) return st;
    h->drop_graph();
    cudaError_t e = cudaMemsetAsync(h->d_words.p + kWordPerInstance, 0, (size_t)n_inst * sizeof(int32_t), stream);
    if (e != cudaSuccess) return h->cuda_fail(e, "clear queues");
    const BatchArgs a = batch_args(h, P, k, counts, eps);
    int launches = 0;
    if (P.var.sweep) {
        if ((e = launch_sweep_prepass(h, P, stream)) != cudaSuccess) return h->cuda_fail(e, "sort pre-pass");
        ++launches;
    }
    for (int i = 0; i < n_inst; ++i) {
        const InstDesc& I = P.insts[i];
        BatchArgs ai = a;
        ai.item_base = I.item_begin;
        ai.n_items = I.n_items;
        ai.queue = h->d_words.p + kWordPerInstance + i;
        if (h->profiling && i == 0 && (e = cudaEventRecord(h->ev0, stream)) != cudaSuccess)
            return h->cuda_fail(e, "event");
        if ((e = te::launch_batched(P.var, ai, std::min(I.n_items, P.grid), P.threads, P.smem, stream)) !=
            cudaSuccess)
            return h->cuda_fail(e, "per-instance launch");
        ++launches;
    }
    if (h->profiling && (e = cudaEventRecord(h->ev1, stream)) != cudaSuccess) return h->cuda_fail(e, "event");
    if ((e = te::launch_finalize_te(h->d_insts.p, n_inst, h->d_partial.p, h->d_partial_abs.p, digamma_int(k),
                                    P.err_coef, te_dst, err, stream)) != cudaSuccess)
        return h->cuda_fail(e, "finalize");
    ++launches;
    if (n_groups > 0) {
        if ((e = te::launch_finalize_groups(h->d_te_all.p, n_groups, S, te_orig, te_surr, p, stream)) !=
            cudaSuccess)
            return h->cuda_fail(e, "finalize groups");
        ++launches;
    }
    h->last_launches = launches;
    h->ev_recorded = h->profiling;
    return TE_OK;
}

// upload the plan's tables and run (or replay) the captured graph
te_status run_batched(te_handle* h, const Plan& P, const te_series* series, int n_series,
                      const te_instance* inst, int n_inst, int k, double* te_out, double* err,
                      int32_t* counts, float* eps, int n_groups, int S, double* te_orig,
                      double* te_surr, double* p, cudaStream_t stream) {
    te_status st = ensure_psi(h);
    if (st != TE_OK) return st;
    bool grew = false;
    cudaError_t e;
    if ((e = h->d_insts.ensure(P.insts.size(), &grew)) != cudaSuccess ||
        (e = h->d_items.ensure(P.items.size(), &grew)) != cudaSuccess ||
        (e = h->d_words.ensure(kWordPerInstance + (size_t)n_inst, &grew)) != cudaSuccess ||
        (e = h->d_partial.ensure((size_t)P.n_parts, &grew)) != cudaSuccess ||
        (e = h->d_partial_abs.ensure((size_t)P.n_parts, &grew)) != cudaSuccess ||
        (n_groups > 0 && (e = h->d_te_all.ensure((size_t)n_inst, &grew)) != cudaSuccess))
        return h->fail(TE_ENOMEM, "workspace: %s", cudaGetErrorString(e));
    if ((st = prepare_sweep(h, P, &grew)) != TE_OK) return st;
    h->last_sweep = P.var.sweep;
    h->last_pairs = P.exhaustive_pairs;
    h->last_ops = P.exhaustive_ops;
    h->last_bundled = P.n_bundled;
    {
        int nb = 0;
        for (const auto& I : P.insts) nb += I.bundle_n;
        h->last_paths[0] = P.n_lane;
        h->last_paths[1] = nb;
        h->last_paths[2] = n_inst - P.n_lane - nb;
    }
    if (grew) {
        ++h->workspace_gen;
        // a fresh flag word must start cleared
        if ((e = cudaMemsetAsync(h->d_words.p, 0, 2 * sizeof(int32_t), stream)) != cudaSuccess)
            return h->cuda_fail(e, "clear flags");
    }
    double* te_dst = n_groups > 0 ? h->d_te_all.p : te_out;

    // signature of everything the captured graph bakes in
    uint64_t key = P.table_hash;
    const void* outs[] = {te_out, err, counts, eps, te_orig, te_surr, p};
    key = fnv(key, outs, sizeof outs);
    const int cfg[] = {k, P.threads, P.grid, P.smem_floats, P.var.dlo, P.var.dhi, P.var.ks, P.var.qpt,
                       P.var.warp_only ? 1 : 0,
                       n_groups, S, h->profiling ? 1 : 0, n_inst, P.var.sweep ? 1 : 0, P.bd, P.bgrid,
                       (int)P.bsmem, P.tgrid, (int)P.tsmem, P.n_bres, P.n_lane, P.lane_max_np};
    key = fnv(key, cfg, sizeof cfg);
    key = fnv(key, P.lane_grid, sizeof P.lane_grid);
    const bool replay = !h->per_instance && h->graph_exec && h->graph_key == key &&
                        h->graph_gen == h->workspace_gen;
    if (h->per_instance) return run_per_instance(h, P, n_inst, k, te_dst, err, counts, eps, n_groups, S,
                                                 te_orig, te_surr, p, stream);

    if (!replay) {
        h->drop_graph();
        te_status ust = upload_tables(h, P, stream);
        if (ust != TE_OK) return ust;
        const BatchArgs a = batch_args(h, P, k, counts, eps);
        const double psi_k = digamma_int(k);

        cudaGraph_t g = nullptr;
        if ((e = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
            return h->cuda_fail(e, "begin capture");
        cudaError_t ce = cudaMemsetAsync(h->d_words.p, 0, sizeof(int32_t), h->cap_stream);
        if (ce == cudaSuccess && !P.bitems.empty())
            ce = cudaMemsetAsync(h->d_words.p + 2, 0, 2 * sizeof(int32_t), h->cap_stream);
        int launches = 0;
        if (ce == cudaSuccess && P.var.sweep) {
            ce = launch_sweep_prepass(h, P, h->cap_stream);
            ++launches;
        }
        if (ce == cudaSuccess && !P.lgroups.empty()) {
            ce = cudaMemsetAsync(h->d_words.p + kWordLaneQueue, 0, (kWordPerInstance - kWordLaneQueue) * sizeof(int32_t),
                                 h->cap_stream);
            if (ce == cudaSuccess)
                ce = te::launch_lane_stage(h->d_lgroups.p, (int)P.lgroups.size(), P.lane_max_np, h->d_sidx.p,
                                           h->d_tpart.p, h->d_lrw.p, h->d_lck.p, h->d_lxb.p, (int)P.xblocks.size(),
                                           P.x_max, h->d_lx.p, h->d_words.p + 1, h->cap_stream);
            ++launches;
        }
        // an event recorded during capture becomes a graph node only with cudaEventRecordExternal
        if (ce == cudaSuccess && h->profiling) ce = cudaEventRecordWithFlags(h->ev0, h->cap_stream, cudaEventRecordExternal);
        for (int slot = 0; slot < te::kLaneSlots && ce == cudaSuccess; ++slot) {
            const int n = P.lane_begin[slot + 1] - P.lane_begin[slot];
            if (n <= 0) continue;
            BatchArgs al = a;
            al.item_base = P.lane_begin[slot];
            al.n_items = n;
            al.queue = h->d_words.p + kWordLaneQueue + slot;
            ce = te::launch_lanes(te::kLaneMinD + slot / te::kLaneTauClasses, P.var.ks, slot % te::kLaneTauClasses, al,
                                  P.lane_grid[slot], h->cap_stream);
            ++launches;
        }
        for (int tiled = 0; tiled < 2 && ce == cudaSuccess; ++tiled) {
            const int n = tiled ? (int)P.bitems.size() - P.n_bres : P.n_bres;
            if (n <= 0) continue;
            BatchArgs ab = a;
            ab.items = h->d_bitems.p;
            ab.item_base = tiled ? P.n_bres : 0;
            ab.n_items = n;
            ab.queue = h->d_words.p + 2 + tiled;
            ab.smem_floats = (int)((tiled ? P.tsmem : P.bsmem) / sizeof(float));
            ce = te::launch_bundle(P.bd, P.var.ks, tiled != 0, ab, tiled ? P.tgrid : P.bgrid,
                                   tiled ? P.tsmem : P.bsmem, h->cap_stream);
            ++launches;
        }
        if (ce == cudaSuccess && !P.items.empty()) {
            ce = te::launch_batched(P.var, a, P.grid, P.threads, P.smem, h->cap_stream);
            ++launches;
        }
        if (ce == cudaSuccess && h->profiling) ce = cudaEventRecordWithFlags(h->ev1, h->cap_stream, cudaEventRecordExternal);
        if (ce == cudaSuccess) {
            ce = te::launch_finalize_te(h->d_insts.p, n_inst, h->d_partial.p, h->d_partial_abs.p, psi_k,
                                        P.err_coef, te_dst, err, h->cap_stream);
            ++launches;
        }
        if (ce == cudaSuccess && n_groups > 0) {
            ce = te::launch_finalize_groups(h->d_te_all.p, n_groups, S, te_orig, te_surr, p, h->cap_stream);
            ++launches;
        }
        e = cudaStreamEndCapture(h->cap_stream, &g);
        if (ce != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return h->cuda_fail(ce, "kernel launch (capture)");
        }
        if (e != cudaSuccess) return h->cuda_fail(e, "end capture");
        e = cudaGraphInstantiate(&h->graph_exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            h->graph_exec = nullptr;
            return h->cuda_fail(e, "graph instantiate");
        }
        h->graph_key = key;
        h->graph_gen = h->workspace_gen;
        h->graph_launches = launches;
    }
    if ((e = cudaGraphLaunch(h->graph_exec, stream)) != cudaSuccess) return h->cuda_fail(e, "graph launch");
    h->last_launches = h->graph_launches;
    h->ev_recorded = h->profiling;
    (void)series;
    (void)n_series;
    (void)inst;
    return TE_OK;
}

}  // namespace

// =========================================================================================
// exported C ABI
// =========================================================================================

TE_EXPORT te_status te_create(te_handle** out, int32_t device) {
    if (!out) {
        g_create_error = "te_create: out is NULL";
        return TE_EINVAL;
    }
    *out = nullptr;
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess) {
        g_create_error = std::string("cudaGetDeviceCount: ") + cudaGetErrorString(e);
        return TE_ECUDA;
    }
    if (device < 0 || device >= n) {
        g_create_error = "te_create: device index out of range";
        return TE_EINVAL;
    }
    DeviceGuard g(device);
    if (!g.ok) {
        g_create_error = "te_create: cudaSetDevice failed";
        return TE_ECUDA;
    }
    te_handle* h = new te_handle();
    h->device = device;
    cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, device);
    if ((e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&h->upload_done, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreate(&h->ev0)) != cudaSuccess || (e = cudaEventCreate(&h->ev1)) != cudaSuccess) {
        g_create_error = std::string("te_create: ") + cudaGetErrorString(e);
        delete h;
        return TE_ECUDA;
    }
    *out = h;
    return TE_OK;
}

TE_EXPORT void te_destroy(te_handle* h) {
    if (!h) return;
    DeviceGuard g(h->device);
    cudaStreamSynchronize(h->cap_stream);
    if (h->upload_done) cudaEventSynchronize(h->upload_done);
    h->drop_graph();
    h->d_insts.release();
    h->d_items.release();
    h->d_words.release();
    h->d_partial.release();
    h->d_partial_abs.release();
    h->d_te_all.release();
    h->d_surr_ws.release();
    h->d_p_ws.release();
    h->d_psi.release();
    h->d_groups.release();
    h->d_sidx.release();
    h->d_skey.release();
    h->d_sia.release();
    h->d_sib.release();
    h->d_sk64a.release();
    h->d_sk64b.release();
    h->d_strip_pos.release();
    h->d_strip_k2.release();
    h->d_exec.release();
    h->d_bitems.release();
    h->d_members.release();
    h->d_lgroups.release();
    h->d_litems.release();
    h->d_lmembers.release();
    h->d_lrw.release();
    h->d_tpart.release();
    h->d_lxb.release();
    h->d_lx.release();
    h->d_lck.release();
    h->h_stage.release();
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
    if (h->upload_done) cudaEventDestroy(h->upload_done);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    delete h;
}

TE_EXPORT const char* te_last_error(const te_handle* h) {
    return h ? h->err.c_str() : g_create_error.c_str();
}

TE_EXPORT te_status te_sync_status(te_handle* h, void* stream) {
    if (!h) return TE_EINVAL;
    h->err.clear();
    DeviceGuard g(h->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return h->cuda_fail(e, "stream synchronize");
    if (!h->d_words.p) return TE_OK;
    int32_t w[2] = {0, 0};
    if ((e = cudaMemcpyAsync(w, h->d_words.p, sizeof w, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return h->cuda_fail(e, "read flags");
    if (w[1]) {
        cudaMemsetAsync(h->d_words.p + 1, 0, sizeof(int32_t), st);
        cudaStreamSynchronize(st);
        if (w[1] & te::kFlagBadPerm)
            return h->fail(TE_EINVAL, "a permutation entry was outside 0..R-1 (clamped to 0)");
    }
    return TE_OK;
}

TE_EXPORT te_status te_embed(te_handle* h, const float* src, const float* tgt, int32_t R, int32_t T,
                             const te_params* p, const int32_t* src_perm, float* points, int32_t ld,
                             void* stream) {
    if (!h) return TE_EINVAL;
    h->err.clear();
    if (!src || !tgt || !p || !points) return h->fail(TE_EINVAL, "te_embed: null pointer");
    if (R < 1 || T < 1) return h->fail(TE_EINVAL, "te_embed: R=%d T=%d", R, T);
    if (p->d < 1 || p->d > kMaxEmbedDim) return h->fail(TE_EINVAL, "te_embed: d=%d outside 1..%d", p->d, kMaxEmbedDim);
    if (p->tau < 1 || p->u < 0 || p->window < 1)
        return h->fail(TE_EINVAL, "te_embed: tau=%d u=%d window=%d", p->tau, p->u, p->window);
    const int64_t N = (int64_t)R * p->window;
    if (N > INT32_MAX / 2) return h->fail(TE_EINVAL, "te_embed: N too large");
    if (ld < N || (ld & 3) || !aligned16(points))
        return h->fail(TE_EINVAL, "te_embed: ld=%d must be >= N=%lld, a multiple of 4, points 16-byte aligned", ld,
                       (long long)N);
    if (!embed_in_range(T, p->d, p->tau, p->u, p->t_start, p->window))
        return h->fail(TE_ERANGE, "te_embed: t_start=%d window=%d reaches outside 0..%d", p->t_start, p->window, T - 1);
    DeviceGuard g(h->device);
    bool grew = false;
    cudaError_t e = h->d_words.ensure(2, &grew);
    if (e != cudaSuccess) return h->fail(TE_ENOMEM, "flags: %s", cudaGetErrorString(e));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (grew) {
        ++h->workspace_gen;
        cudaMemsetAsync(h->d_words.p, 0, 2 * sizeof(int32_t), st);
    }
    e = te::launch_embed(src, tgt, R, T, p->d, p->tau, p->u, p->t_start, p->window, src_perm, points, ld,
                         h->d_words.p + 1, st);
    h->last_launches = 1;
    return e == cudaSuccess ? TE_OK : h->cuda_fail(e, "te_embed launch");
}

TE_EXPORT te_status te_knn_maxnorm(te_handle* h, const float* points, int32_t N, int32_t D, int32_t ld,
                                   int32_t k, float* eps, int32_t* nn, void* stream) {
    if (!h) return TE_EINVAL;
    h->err.clear();
    if (!points || !eps) return h->fail(TE_EINVAL, "te_knn_maxnorm: null pointer");
    if (D < 1 || D > kMaxD) return h->fail(TE_EINVAL, "te_knn_maxnorm: D=%d outside 1..%d", D, kMaxD);
    if (k < 1 || k > kMaxK) return h->fail(TE_EINVAL, "te_knn_maxnorm: k=%d outside 1..%d", k, kMaxK);
    if (N < k + 1) return h->fail(TE_EINVAL, "te_knn_maxnorm: N=%d < k+1", N);
    if (ld < N || (ld & 3) || !aligned16(points))
        return h->fail(TE_EINVAL, "te_knn_maxnorm: ld=%d must be >= N, a multiple of 4, points 16-byte aligned", ld);
    DeviceGuard g(h->device);
    cudaError_t e = te::launch_knn(points, N, D, ld, k, eps, nn, h->sm_count, static_cast<cudaStream_t>(stream));
    h->last_launches = 1;
    return e == cudaSuccess ? TE_OK : h->cuda_fail(e, "te_knn_maxnorm launch");
}

TE_EXPORT te_status te_range_count(te_handle* h, const float* points, int32_t N, int32_t d_y, int32_t d_x,
                                   int32_t ld, const float* eps, int32_t* counts, void* stream) {
    if (!h) return TE_EINVAL;
    h->err.clear();
    if (!points || !eps || !counts) return h->fail(TE_EINVAL, "te_range_count: null pointer");
    if (d_y < 0 || d_x < 0 || 1 + d_y + d_x > kMaxD)
        return h->fail(TE_EINVAL, "te_range_count: d_y=%d d_x=%d", d_y, d_x);
    if (N < 1) return h->fail(TE_EINVAL, "te_range_count: N=%d", N);
    if (ld < N || (ld & 3) || !aligned16(points))
        return h->fail(TE_EINVAL, "te_range_count: ld=%d must be >= N, a multiple of 4, points 16-byte aligned", ld);
    DeviceGuard g(h->device);
    cudaError_t e = te::launch_count(points, N, d_y, d_x, ld, eps, counts, h->sm_count,
                                     static_cast<cudaStream_t>(stream));
    h->last_launches = 1;
    return e == cudaSuccess ? TE_OK : h->cuda_fail(e, "te_range_count launch");
}

TE_EXPORT te_status te_estimate(te_handle* h, const te_series* series, int32_t n_series,
                                const te_instance* inst, int32_t n_inst, int32_t k, double* te,
                                double* err_bound, int32_t* counts, float* eps, void* stream) {
    if (!h) return TE_EINVAL;
    h->err.clear();
    if (k < 1 || k > kMaxK) return h->fail(TE_EINVAL, "te_estimate: k=%d outside 1..%d", k, kMaxK);
    if (n_inst < 0 || (n_inst > 0 && (!inst || !te))) return h->fail(TE_EINVAL, "te_estimate: null instances/te");
    te_status st = validate_series(h, series, n_series);
    if (st != TE_OK) return st;
    if (n_inst == 0) {
        h->last_launches = 0;
        return TE_OK;
    }
    DeviceGuard g(h->device);
    Plan* P = nullptr;
    if ((st = cached_plan(h, series, n_series, inst, n_inst, k, &P)) != TE_OK) return st;
    return run_batched(h, *P, series, n_series, inst, n_inst, k, te, err_bound, counts, eps, 0, 0, nullptr,
                       nullptr, nullptr, static_cast<cudaStream_t>(stream));
}

TE_EXPORT te_status te_surrogate_test(te_handle* h, const te_series* series, int32_t n_series,
                                      const int32_t* t_starts, int32_t n_t, int32_t window, int32_t S,
                                      int32_t k, double* te_orig, double* te_surr, double* p, void* stream) {
    if (!h) return TE_EINVAL;
    h->err.clear();
    if (k < 1 || k > kMaxK) return h->fail(TE_EINVAL, "te_surrogate_test: k=%d outside 1..%d", k, kMaxK);
    if (n_t < 0 || S < 0 || window < 1 || (n_t > 0 && !t_starts))
        return h->fail(TE_EINVAL, "te_surrogate_test: n_t=%d S=%d window=%d", n_t, S, window);
    if (!te_orig || !p || (S > 0 && !te_surr)) return h->fail(TE_EINVAL, "te_surrogate_test: null output");
    te_status st = validate_series(h, series, n_series);
    if (st != TE_OK) return st;
    for (int s = 0; s < n_series; ++s)
        if (series[s].S < S) return h->fail(TE_EINVAL, "series %d has %d permutations < S=%d", s, series[s].S, S);
    const int64_t n_inst64 = (int64_t)n_series * n_t * (S + 1);
    if (n_inst64 > INT32_MAX / 4) return h->fail(TE_ENOTIMPL, "te_surrogate_test: too many estimates");
    if (n_inst64 == 0) {
        h->last_launches = 0;
        return TE_OK;
    }
    std::vector<te_instance> inst;
    inst.reserve((size_t)n_inst64);
    for (int s = 0; s < n_series; ++s)
        for (int j = 0; j < n_t; ++j)
            for (int m = -1; m < S; ++m) inst.push_back(te_instance{s, t_starts[j], window, m});
    DeviceGuard g(h->device);
    Plan* P = nullptr;
    if ((st = cached_plan(h, series, n_series, inst.data(), (int)inst.size(), k, &P)) != TE_OK) return st;
    return run_batched(h, *P, series, n_series, inst.data(), (int)inst.size(), k, nullptr, nullptr, nullptr,
                       nullptr, n_series * n_t, S, te_orig, te_surr, p, static_cast<cudaStream_t>(stream));
}

namespace {

bool load_tune_cache(te_handle* h, const char* path) {
    FILE* f = fopen(path, "r");
    if (!f) return false;
    char line[512], key[128];
    int t = 0, q = 0;
    while (fgets(line, sizeof line, f)) {
        if (sscanf(line, " \"%127[^\"]\": {\"threads\": %d, \"qpt\": %d", key, &t, &q) == 3 && t >= 64 &&
            t <= te::kSweepWarpThreads && t % 32 == 0 && (q == 1 || q == 2 || q == 4))
            h->tuned[key] = {t, q}, ++h->tune_gen;
    }
    fclose(f);
    return true;
}

bool save_tune_cache(te_handle* h, const char* path, const std::map<std::string, float>& ms) {
    std::string tmp = std::string(path) + ".tmp";
    FILE* f = fopen(tmp.c_str(), "w");
    if (!f) return false;
    fprintf(f, "{\n");
    size_t n = 0;
    for (const auto& kv : h->tuned) {
        auto it = ms.find(kv.first);
        fprintf(f, " \"%s\": {\"threads\": %d, \"qpt\": %d, \"ms\": %.4f}%s\n", kv.first.c_str(), kv.second.first,
                kv.second.second, it == ms.end() ? -1.0 : (double)it->second, ++n < h->tuned.size() ? "," : "");
    }
    fprintf(f, "}\n");
    fclose(f);
    return rename(tmp.c_str(), path) == 0;
}

}  // namespace

TE_EXPORT te_status te_autotune(te_handle* h, const te_series* series, int32_t n_series, const te_instance* inst,
                                int32_t n_inst, int32_t k, const char* cache_path, int32_t* threads_out,
                                int32_t* qpt_out, void* stream) {
    if (!h) return TE_EINVAL;
    h->err.clear();
    if (k < 1 || k > kMaxK) return h->fail(TE_EINVAL, "te_autotune: k=%d outside 1..%d", k, kMaxK);
    if (n_inst < 1 || !inst) return h->fail(TE_EINVAL, "te_autotune: no instances");
    te_status st = validate_series(h, series, n_series);
    if (st != TE_OK) return st;
    DeviceGuard g(h->device);
    cudaStream_t strm = static_cast<cudaStream_t>(stream);
    const int save_t = h->cfg_threads, save_q = h->cfg_qpt;
    const bool save_prof = h->profiling;
    const int save_share = h->sharing;
    auto restore = [&]() {
        h->cfg_threads = save_t;
        h->cfg_qpt = save_q;
        h->profiling = save_prof;
        h->sharing = save_share;
    };
    h->sharing = 0;  // the shapes tuned are those of the batched kernel
    h->cfg_threads = h->cfg_qpt = 0;
    Plan P;
    if ((st = build_plan(h, series, n_series, inst, n_inst, k, &P)) != TE_OK) {
        restore();
        return st;
    }
    const int ks = P.var.ks;
    const std::string sig = shape_signature(P.insts, ks);
    if (cache_path && cache_path[0]) load_tune_cache(h, cache_path);
    std::map<std::string, float> best_ms;
    auto found = h->tuned.find(sig);
    if (found == h->tuned.end()) {
        // a cost-stratified subset of about eight waves of the default plan's work items
        std::vector<int> order(n_inst);
        for (int i = 0; i < n_inst; ++i) order[i] = i;
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
            const InstDesc &A = P.insts[a], &B = P.insts[b];
            return (double)A.N * A.N * (1 + 2 * A.d) > (double)B.N * B.N * (1 + 2 * B.d);
        });
        const int64_t want_items = 8LL * P.grid;
        const int stride = (int)std::max<int64_t>(1, (int64_t)P.items.size() / std::max<int64_t>(1, want_items));
        std::vector<te_instance> sub;
        for (int i = 0; i < n_inst; i += stride) sub.push_back(inst[order[i]]);
        int dmax = 1;
        for (const auto& I : P.insts) dmax = std::max(dmax, I.d);
        std::vector<int> qs = dmax > 5 ? std::vector<int>{1}
                              : (ks == 5 && dmax <= 4) ? std::vector<int>{4, 2} : std::vector<int>{2};
        bool uniform = true;
        for (const auto& I : P.insts) uniform &= I.N == P.insts[0].N;
        bool grew = false;
        cudaError_t e = h->d_te_all.ensure(sub.size(), &grew);
        if (e != cudaSuccess) {
            restore();
            return h->fail(TE_ENOMEM, "te_autotune: %s", cudaGetErrorString(e));
        }
        if (grew) ++h->workspace_gen;
        float best = 1e30f;
        int bt = 0, bq = 0;
        h->profiling = true;
        for (int q : qs) {
            int64_t min_slots = INT64_MAX;
            const int tmax = P.var.warp_only ? te::kSweepWarpThreads : te::kBatchedMaxThreads;
            if (uniform)
                for (int t = 64; t <= tmax; t += 32) {
                    const int64_t per = (int64_t)t * q;
                    min_slots = std::min(min_slots, ((P.insts[0].N + per - 1) / per) * per);
                }
            for (int t = 64; t <= tmax; t += 32) {
                if (uniform) {
                    const int64_t per = (int64_t)t * q;
                    if (((P.insts[0].N + per - 1) / per) * per > min_slots + min_slots / 8) continue;
                } else if (t % 64) {
                    continue;
                }
                h->cfg_threads = t;
                h->cfg_qpt = q;
                Plan S;
                if (build_plan(h, series, n_series, sub.data(), (int)sub.size(), k, &S) != TE_OK) continue;
                float med = 0;
                std::vector<float> v;
                for (int rep = 0; rep < 4; ++rep) {
                    if (run_batched(h, S, series, n_series, sub.data(), (int)sub.size(), k, h->d_te_all.p, nullptr,
                                    nullptr, nullptr, 0, 0, nullptr, nullptr, nullptr, strm) != TE_OK)
                        break;
                    float ms = 0;
                    if (cudaEventSynchronize(h->ev1) != cudaSuccess ||
                        cudaEventElapsedTime(&ms, h->ev0, h->ev1) != cudaSuccess)
                        break;
                    if (rep > 0) v.push_back(ms);  // the first run captures the graph
                }
                if (v.size() == 3) {
                    std::sort(v.begin(), v.end());
                    med = v[1];
                    if (med < best) {
                        best = med;
                        bt = t;
                        bq = q;
                    }
                }
            }
        }
        restore();
        h->err.clear();
        if (!bt) return h->fail(TE_ECUDA, "te_autotune: no candidate ran");
        h->tuned[sig] = {bt, bq};
        ++h->tune_gen;
        best_ms[sig] = best;
        if (cache_path && cache_path[0] && !save_tune_cache(h, cache_path, best_ms))
            return h->fail(TE_EINVAL, "te_autotune: cannot write %s", cache_path);
        found = h->tuned.find(sig);
    }
    restore();
    if (threads_out) *threads_out = found->second.first;
    if (qpt_out) *qpt_out = found->second.second;
    return TE_OK;
}

TE_EXPORT te_status te_delay_scan(te_handle* h, const te_series* series, const int32_t* t_starts, int32_t n_t,
                                  int32_t window, int32_t u_lo, int32_t u_hi, int32_t S, int32_t k, double* te,
                                  double* p, int32_t* u_best, void* stream) {
    if (!h) return TE_EINVAL;
    h->err.clear();
    if (k < 1 || k > kMaxK) return h->fail(TE_EINVAL, "te_delay_scan: k=%d outside 1..%d", k, kMaxK);
    if (!series || !t_starts || n_t < 1 || window < 1 || S < 0 || !te || !u_best)
        return h->fail(TE_EINVAL, "te_delay_scan: null output, n_t=%d, window=%d or S=%d", n_t, window, S);
    if (u_lo < 0 || u_hi < u_lo) return h->fail(TE_EINVAL, "te_delay_scan: u range %d..%d", u_lo, u_hi);
    te_status st = validate_series(h, series, 1);
    if (st != TE_OK) return st;
    if (series->S < S) return h->fail(TE_EINVAL, "te_delay_scan: series has %d permutations < S=%d", series->S, S);
    const int n_u = u_hi - u_lo + 1;
    const int64_t n_inst64 = (int64_t)n_u * n_t * (S + 1);
    if (n_inst64 > INT32_MAX / 4) return h->fail(TE_ENOTIMPL, "te_delay_scan: too many estimates");
    // one series descriptor per scanned delay (same data), estimates grouped per (u, t)
    std::vector<te_series> ser((size_t)n_u, *series);
    for (int iu = 0; iu < n_u; ++iu) ser[iu].u = u_lo + iu;
    std::vector<te_instance> inst;
    inst.reserve((size_t)n_inst64);
    for (int iu = 0; iu < n_u; ++iu)
        for (int j = 0; j < n_t; ++j)
            for (int m = -1; m < S; ++m) inst.push_back(te_instance{iu, t_starts[j], window, m});
    DeviceGuard g(h->device);
    Plan* P = nullptr;
    if ((st = cached_plan(h, ser.data(), n_u, inst.data(), (int)inst.size(), k, &P)) != TE_OK) return st;
    const int n_groups = n_u * n_t;
    bool grew = false;
    cudaError_t e;
    if ((S > 0 && (e = h->d_surr_ws.ensure((size_t)n_groups * S, &grew)) != cudaSuccess) ||
        (!p && (e = h->d_p_ws.ensure((size_t)n_groups, &grew)) != cudaSuccess))
        return h->fail(TE_ENOMEM, "te_delay_scan workspace: %s", cudaGetErrorString(e));
    if (grew) ++h->workspace_gen;
    cudaStream_t strm = static_cast<cudaStream_t>(stream);
    st = run_batched(h, *P, ser.data(), n_u, inst.data(), (int)inst.size(), k, nullptr, nullptr, nullptr, nullptr,
                     n_groups, S, te, S > 0 ? h->d_surr_ws.p : nullptr, p ? p : h->d_p_ws.p, strm);
    if (st != TE_OK) return st;
    if ((e = te::launch_delay_argmax(te, n_u, n_t, u_lo, u_best, strm)) != cudaSuccess)
        return h->cuda_fail(e, "delay argmax");
    h->last_launches += 1;
    return TE_OK;
}

TE_EXPORT te_status te_set_profiling(te_handle* h, int32_t enable) {
    if (!h) return TE_EINVAL;
    h->profiling = enable != 0;
    return TE_OK;
}

TE_EXPORT te_status te_last_kernel_ms(te_handle* h, float* ms) {
    if (!h || !ms) return TE_EINVAL;
    h->err.clear();
    if (!h->ev_recorded) return h->fail(TE_EINVAL, "no profiled batched launch yet");
    DeviceGuard g(h->device);
    cudaError_t e = cudaEventSynchronize(h->ev1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, h->ev0, h->ev1);
    return e == cudaSuccess ? TE_OK : h->cuda_fail(e, "kernel timing");
}

TE_EXPORT int32_t te_last_launch_count(const te_handle* h) { return h ? h->last_launches : 0; }

TE_EXPORT te_status te_set_search(te_handle* h, int32_t mode) {
    if (!h) return TE_EINVAL;
    if (mode != 0 && mode != 1) return h->fail(TE_EINVAL, "te_set_search: mode %d is not 0 or 1", mode);
    h->search_mode = mode;
    return TE_OK;
}

TE_EXPORT te_status te_last_work(te_handle* h, uint64_t* pairs, uint64_t* ops, int32_t* swept) {
    if (!h) return TE_EINVAL;
    h->err.clear();
    uint64_t pr = h->last_pairs, op = h->last_ops;
    if (h->last_sweep && h->d_exec.p) {
        DeviceGuard g(h->device);
        unsigned long long v[2] = {0, 0};
        cudaError_t e = cudaMemcpy(v, h->d_exec.p, sizeof v, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return h->cuda_fail(e, "read work counters");
        pr = v[0];
        op = v[1];
    }
    if (pairs) *pairs = pr;
    if (ops) *ops = op;
    if (swept) *swept = h->last_sweep ? 1 : 0;
    return TE_OK;
}

TE_EXPORT te_status te_set_sharing(te_handle* h, int32_t enable) {
    if (!h) return TE_EINVAL;
    h->err.clear();
    if (enable < 0 || enable > 3) return h->fail(TE_EINVAL, "te_set_sharing: %d is not 0, 1, 2 or 3", enable);
    h->sharing = enable;
    return TE_OK;
}

TE_EXPORT te_status te_last_paths(te_handle* h, int32_t* paths) {
    if (!h || !paths) return TE_EINVAL;
    for (int i = 0; i < 3; ++i) paths[i] = h->last_paths[i];
    return TE_OK;
}

TE_EXPORT te_status te_last_alu_ops(te_handle* h, uint64_t* ops, int32_t* bundles) {
    if (!h || !ops) return TE_EINVAL;
    h->err.clear();
    uint64_t op = h->last_ops;
    if (h->last_sweep && h->d_exec.p) {
        DeviceGuard g(h->device);
        unsigned long long v[3] = {0, 0, 0};
        cudaError_t e = cudaMemcpy(v, h->d_exec.p, sizeof v, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return h->cuda_fail(e, "read work counters");
        op = v[1] - v[2];
    }
    *ops = op;
    if (bundles) *bundles = h->last_bundled;
    return TE_OK;
}

TE_EXPORT te_status te_last_pass_work(te_handle* h, uint64_t* pairs, uint64_t* cycles) {
    if (!h || !pairs || !cycles) return TE_EINVAL;
    h->err.clear();
    // exhaustive search: N^2 pairs per pass, no cycle accounting
    pairs[0] = pairs[1] = h->last_pairs / 2;
    cycles[0] = cycles[1] = 0;
    if (h->last_sweep && h->d_exec.p) {
        DeviceGuard g(h->device);
        unsigned long long v[6] = {0, 0, 0, 0, 0, 0};
        cudaError_t e = cudaMemcpy(v, h->d_exec.p, sizeof v, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return h->cuda_fail(e, "read work counters");
        pairs[0] = v[3];
        pairs[1] = v[0] - v[3];
        cycles[0] = v[4];
        cycles[1] = v[5];
    }
    return TE_OK;
}

TE_EXPORT te_status te_set_batching(te_handle* h, int32_t per_instance) {
    if (!h) return TE_EINVAL;
    h->per_instance = per_instance != 0;
    return TE_OK;
}

TE_EXPORT te_status te_set_launch_config(te_handle* h, int32_t threads, int32_t qpt) {
    if (!h) return TE_EINVAL;
    h->err.clear();
    if (threads != 0 && (threads < 64 || threads > te::kSweepWarpThreads || threads % 32))
        return h->fail(TE_EINVAL, "threads=%d: multiple of 32 in 64..%d or 0", threads, te::kSweepWarpThreads);
    if (qpt != 0 && qpt != 1 && qpt != 2 && qpt != 4) return h->fail(TE_EINVAL, "qpt=%d: 1, 2, 4 or 0", qpt);
    h->cfg_threads = threads;
    h->cfg_qpt = qpt;
    return TE_OK;
}
