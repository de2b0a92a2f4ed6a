/* te_gb300.h - C ABI of the GB300 (sm_103a) ensemble transfer-entropy hot path.
 *
 * The library estimates TE_SPO(X -> Y, t, u) with the ensemble KSG estimator of Wollstadt et
 * al. (PLoS ONE 2014): for every analysis time point and every trial-shuffled surrogate it
 * builds the delay-embedded joint space (y_t, y-, x-) (Eq. 6, Eq. 7, Eq. 10), finds every
 * point's k-th nearest neighbour distance under the maximum norm, counts neighbours strictly
 * inside that radius in the three marginal spaces and averages the digamma sum of Eq. 9.
 * All arithmetic runs in the library's CUDA kernels; no call falls back to the CPU.
 *
 * Conventions shared by every call
 *  - Data pointers (series, perms, points, eps, counts, results) are caller-owned DEVICE
 *    pointers on the handle's device, e.g. torch tensors' data_ptr(). Descriptor arrays
 *    (te_series, te_instance, t_starts, te_params) are HOST memory, read during the call.
 *  - `stream` is a cudaStream_t passed as void* (NULL: the legacy default stream). Every call
 *    is asynchronous on it: results are valid after the stream has been synchronised.
 *  - Arguments are validated on the host before anything is launched; an invalid call
 *    returns TE_EINVAL or TE_ERANGE, launches nothing and leaves outputs untouched.
 *  - Series are trials x samples, float32, row-major: x[r * T + t] (repetition r, time t).
 *  - Coordinates must be finite. Distances are FP32 (|fl32(p - q)|, round to nearest, no
 *    flush to zero); neighbour counts are exact integers; TE is returned in FP64 nats.
 *  - Point layout (te_embed output, te_knn_maxnorm / te_range_count input) is structure of
 *    arrays: coordinate c of point i at points[c * ld + i], ld >= N, ld a multiple of 4 and
 *    the base pointer 16-byte aligned. Joint coordinate order: [ y_t | y- (d_y) | x- (d_x) ].
 *    Points are repetitions concatenated in order: i = r * W + w for window sample w.
 *  - A handle may be used by one host thread at a time.
 *  - Errors: TE_ECUDA reports a CUDA runtime error, te_last_error() the message.
 */
#ifndef TE_GB300_H
#define TE_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TE_ABI_VERSION 1

typedef enum te_status {
    TE_OK = 0,
    TE_EINVAL = 1,   /* bad argument: null pointer, size, alignment, k, permutation index    */
    TE_ERANGE = 2,   /* embedding reaches before sample 0 or past sample T-1                   */
    TE_ENOMEM = 3,   /* device workspace could not be allocated                                */
    TE_ECUDA = 4,    /* CUDA runtime error (launch or previous asynchronous fault)             */
    TE_ETIMEOUT = 5, /* reserved: a bounded device wait ran out (no kernel waits today)        */
    TE_ENOTIMPL = 6  /* size outside what this build supports (see each call's limits)         */
} te_status;

/* Embedding parameters of one estimate (paper notation):
 *   d       embedding dimension of target and source past states (Eq. 6 / Eq. 7): 1 <= d <= 8
 *           for te_estimate / te_surrogate_test, 1 <= d <= 15 for te_embed
 *   tau     embedding delay in samples (Eq. 6), tau >= 1
 *   u       assumed interaction delay: the source state is taken at t - u (Eq. 3), u >= 0
 *   k       number of nearest neighbours in the joint space (Eq. 9), 1 <= k <= 16
 *   t_start first sample of the analysis window, window = its length W >= 1 (Eq. 10) */
typedef struct te_params {
    int32_t d, tau, u, k, t_start, window;
} te_params;

/* One source/target pair of trial ensembles.
 *   src, tgt  device float32 [R][T]; perms device int32 [S][R] (NULL when S == 0).
 *   Surrogate s pairs target repetition r with source repetition perms[s * R + r]; this is
 *   the repetition shuffling of Fig. 3 (TE depends only on the pairing). Entries must lie in
 *   0 .. R-1: the kernels clamp an entry outside that range to 0 and raise a device flag that
 *   te_sync_status() reports as TE_EINVAL. */
typedef struct te_series {
    const float* src;
    const float* tgt;
    int32_t R, T, d, tau, u, S;
    const int32_t* perms;
} te_series;

/* One estimate: series index, analysis window [t_start, t_start + window), pairing
 * (perm = -1: original repetitions, perm = s >= 0: surrogate s of that series). */
typedef struct te_instance {
    int32_t series, t_start, window, perm;
} te_instance;

typedef struct te_handle te_handle;

/* Create a handle bound to CUDA device `device` (made current during every call). The handle
 * owns the device workspace (instance tables, work queue, per-item partial sums, the digamma
 * table), cached plans and CUDA graphs; memory grows on demand and is freed by te_destroy.
 * Returns TE_EINVAL for a null `out` or a bad device index, TE_ECUDA if the device cannot be
 * used. */
te_status te_create(te_handle** out, int32_t device);

/* Free everything the handle owns. Waits for the handle's internal work; NULL is a no-op. */
void te_destroy(te_handle* h);

/* Message of the last failed call on this handle ("" after success). Valid until the next
 * call on the handle. A NULL handle returns the message of the calling thread's last failed
 * te_create. */
const char* te_last_error(const te_handle* h);

/* Synchronise `stream` and report device-side flags raised since the previous check
 * (currently: an out-of-range permutation entry -> TE_EINVAL). Clears the flags. */
te_status te_sync_status(te_handle* h, void* stream);

/* te_embed - delay embedding of one estimate's point set (Eq. 6, Eq. 7, source state at t-u
 * as in the State space reconstruction paragraph, pooling of Eq. 10).
 * Point i = r * W + w (t' = t_start + w) gets the D = 1 + 2d coordinates
 *   [ y_r(t'), y_r(t'-1), y_r(t'-1-tau), ..., y_r(t'-1-(d-1)tau),
 *     x_s(t'-u), x_s(t'-u-tau), ..., x_s(t'-u-(d-1)tau) ],   s = src_perm ? src_perm[r] : r.
 *   src, tgt  device [R][T]; src_perm device int32 [R] or NULL (identity).
 *   points    device output [D][ld], N = R * window, ld >= N, ld % 4 == 0, 16-byte aligned.
 *   p->k is not used. TE_ERANGE if a touched sample lies outside 0 .. T-1. */
te_status te_embed(te_handle* h, const float* src, const float* tgt, int32_t R, int32_t T,
                   const te_params* p, const int32_t* src_perm, float* points, int32_t ld,
                   void* stream);

/* te_knn_maxnorm - k-th nearest-neighbour distance of every point in the joint space under
 * the maximum norm, the point itself excluded (kNNS of the Implementation section, "Core
 * algorithm": brute-force infinity-norm search; the radii of Eq. 9).
 *   points  device [D][ld] (layout above), 1 <= D <= 32, N >= k + 1, 1 <= k <= 16.
 *   eps     device float32 [N] output: eps[i] = k-th smallest of max_c |fl32(p_ic - p_jc)|,
 *           j != i (exact: equal to the FP32 value a sequential search computes).
 *   nn      device int32 [N][k] output or NULL: the k nearest indices in (distance, index)
 *           order, ties to the lower index. */
te_status te_knn_maxnorm(te_handle* h, const float* points, int32_t N, int32_t D, int32_t ld,
                         int32_t k, float* eps, int32_t* nn, void* stream);

/* te_range_count - neighbour counts strictly inside eps[i] in the three marginal spaces of
 * Eq. 9 (range search of the Implementation section), the point itself excluded:
 *   counts[0*N + i] = n_z  : #{ j != i : max over y- coords          < eps[i] }
 *   counts[1*N + i] = n_yz : #{ j != i : max over (y_t, y-) coords   < eps[i] }
 *   counts[2*N + i] = n_xz : #{ j != i : max over (y-, x-) coords    < eps[i] }
 *   points  device [D][ld], D = 1 + d_y + d_x <= 32, d_y >= 0, d_x >= 0, N >= 1.
 *   eps     device float32 [N] (typically te_knn_maxnorm's output).
 *   counts  device int32 [3][N] output. */
te_status te_range_count(te_handle* h, const float* points, int32_t N, int32_t d_y, int32_t d_x,
                         int32_t ld, const float* eps, int32_t* counts, void* stream);

/* te_estimate - TE of many estimates in one batched launch (Eq. 9 / Eq. 10 for each instance):
 * embedding, kNN search, range counts and the digamma sum of every instance run in one
 * persistent kernel that takes (instance, query tile) work items from a device queue, followed
 * by one finalisation kernel; the pair of launches is captured once per argument signature in
 * a CUDA graph and replayed. Instances may mix R, d, W and series.
 *   series   host array [n_series]; inst host array [n_inst], N_i = R * window >= k + 1.
 *   te       device float64 [n_inst] output: psi(k) + mean_i(psi(n_z+1) - psi(n_yz+1)
 *            - psi(n_xz+1)). Per-point digamma terms are summed in compensated FP32
 *            (float-float), per-item partials and the mean in FP64.
 *   err_bound device float64 [n_inst] or NULL: a bound on |te - exact-arithmetic value of
 *            the same counts| from that summation.
 *   counts   device int32 or NULL: per instance its [3][N_i] block, blocks concatenated in
 *            instance order.   eps: device float32 or NULL: per instance [N_i], concatenated.
 * Limits: N_i <= 65536, 1 <= d <= 8, k <= 16; a batch that mixes embedding dimensions has
 * d <= 5 (TE_ENOTIMPL beyond). */
te_status te_estimate(te_handle* h, const te_series* series, int32_t n_series,
                      const te_instance* inst, int32_t n_inst, int32_t k, double* te,
                      double* err_bound, int32_t* counts, float* eps, void* stream);

/* te_surrogate_test - the surrogate test of the paper ("TE calculation and statistical testing
 * against surrogate data", Fig. 2 steps 2-6): for every series and every analysis start
 * t_starts[j], the original estimate and S surrogates (perms[0 .. S-1] of the series), all in
 * one batched launch as te_estimate, then p = #{s : TE_s >= TE_0} / S.
 *   te_orig device float64 [n_series][n_t]; te_surr device float64 [n_series][n_t][S];
 *   p       device float64 [n_series][n_t] (NaN when S == 0). Every series needs S <= its S. */
te_status te_surrogate_test(te_handle* h, const te_series* series, int32_t n_series,
                            const int32_t* t_starts, int32_t n_t, int32_t window, int32_t S,
                            int32_t k, double* te_orig, double* te_surr, double* p, void* stream);

/* Measurement hooks (no effect on results).
 * te_set_profiling(h, 1) makes te_estimate / te_surrogate_test record CUDA events around the
 * persistent kernel on the call's stream; te_last_kernel_ms() synchronises on the stop event
 * and returns that kernel's duration. te_last_launch_count() returns how many kernels the
 * last call launched (graph replays count their kernel nodes). */
te_status te_set_profiling(te_handle* h, int32_t enable);
te_status te_last_kernel_ms(te_handle* h, float* ms);
int32_t te_last_launch_count(const te_handle* h);

/* Launch-configuration control for the batched kernel (used by the autotuner and tests).
 * threads: CTA size (multiple of 32, 64..1024; above 512 only the warp-mode sweep kernel of d <= 2
 * uses it, other batches run with 512) or 0 for the built-in choice; qpt: queries per thread
 * (1, 2 or 4; d >= 6 always runs 1, d <= 5 runs 2 when 1 is asked) or 0 for automatic. Takes
 * effect on the next te_estimate / te_surrogate_test / te_delay_scan call. */
te_status te_set_launch_config(te_handle* h, int32_t threads, int32_t qpt);

/* te_delay_scan - delay reconstruction (Eq. 5, "Reconstruction of information transfer delays"):
 * TE_SPO(X -> Y, t, u) for every scanned delay u = u_lo .. u_hi (the series' own u is not used)
 * and every analysis start t_starts[j], each with S surrogates (perms[0 .. S-1]), all estimates
 * in one batched launch as te_surrogate_test; the reconstructed delay of start j is the u of
 * largest original TE (ties to the smaller u).
 *   te      device float64 [n_u][n_t] original TE, n_u = u_hi - u_lo + 1
 *   p       device float64 [n_u][n_t] p-values, or NULL (NaN values when S == 0)
 *   u_best  device int32 [n_t]
 * Every (u, t) must satisfy the embedding range of te_estimate (TE_ERANGE otherwise). */
te_status te_delay_scan(te_handle* h, const te_series* series, const int32_t* t_starts, int32_t n_t,
                        int32_t window, int32_t u_lo, int32_t u_hi, int32_t S, int32_t k, double* te,
                        double* p, int32_t* u_best, void* stream);

/* te_autotune - choose the batched kernel's launch shape (CTA size, queries per thread) for a
 * batch by measurement. The paper fixes 512 threads per block (Implementation, "Low-level
 * implementation details"); here candidates are timed on a cost-stratified subset of the batch
 * (about eight waves of work items; candidates whose padded query slots exceed the minimum by more
 * than 1/8 are skipped) and the fastest is kept in the handle for every later batch with the same
 * signature (embedding dimensions, k, point count). Results do not depend on the shape.
 *   inst        the batch as for te_estimate (or the instances te_surrogate_test would build).
 *   cache_path  nullable: a JSON file read before tuning (a cached signature skips the timing)
 *               and rewritten with the handle's entries after tuning.
 *   threads_out, qpt_out  nullable: the shape now in effect for this signature.
 * Synchronises the stream. Launch-config overrides (te_set_launch_config) take precedence. */
te_status te_autotune(te_handle* h, const te_series* series, int32_t n_series, const te_instance* inst,
                      int32_t n_inst, int32_t k, const char* cache_path, int32_t* threads_out,
                      int32_t* qpt_out, void* stream);

/* Search mode of te_estimate / te_surrogate_test / te_delay_scan (results are identical):
 *   1 (default): sorted sweep. The points of every (series, window start, window) group are sorted
 *      by the target coordinate y_{t'-1} (shared by the original and all surrogates of the group)
 *      and each warp visits only references whose key lies inside the window its queries' radii
 *      allow: every distance the estimator compares is at least fl(|key_q - key_j|), and the window
 *      bounds are rounded outward, so no reference that could enter a top-k list or a count is
 *      skipped. Applies to every point count (up to the 65536 limit of an estimate).
 *   0: exhaustive search over all N^2 pairs (the paper's brute force, Implementation section). */
te_status te_set_search(te_handle* h, int32_t mode);

/* Work of the last te_estimate / te_surrogate_test / te_delay_scan call: (query, reference)
 * pair evaluations over both passes and the FP32 operations they cost (2 D per pair), counted on
 * the device by the sweep (synchronises the device) or N^2 per pass for the exhaustive search;
 * `swept` (nullable) is 1 when the sweep ran. */
te_status te_last_work(te_handle* h, uint64_t* pairs, uint64_t* ops, int32_t* swept);

/* Target-part sharing in the sorted sweep (results are identical in every mode): estimates whose
 * joint points share the target part y_t, y- (same target series, repetitions, window start,
 * window, d and tau; they differ only in the source part x-: the original and its trial-shuffled
 * surrogates of Fig. 3, and every scanned delay u of Eq. 5) compute the target part of each
 * distance and count once for several estimates. The paper computes each surrogate separately;
 * this is exact because max is exact: each estimate sees the same FP32 differences the unshared
 * search computes.
 *   enable = 1 (default): groups of at least 32 such estimates with d = 3..8 run one estimate per
 *     lane (a warp takes one query point for 32 estimates; a reference whose target-part distance
 *     already reaches every lane's current radius is skipped for all 32 before any source
 *     coordinate is read); other groups of two or more with d <= 5 run in bundles of up to 3
 *     staged together in shared memory (one embedding dimension per batch, the most frequent
 *     among them). The lane kernel measured faster than bundles for those groups only.
 *   enable = 3: the lane kernel for every group of at least 8 estimates with d = 2..8, bundles
 *     for the other groups.
 *   enable = 2: bundles only (no lane kernel).
 *   enable = 0: no sharing.
 * Sharing applies with k <= 4; every other estimate runs unshared. TE_EINVAL for other values. */
te_status te_set_sharing(te_handle* h, int32_t enable);

/* FP32 operations the kernels of the last te_estimate / te_surrogate_test / te_delay_scan call
 * executed: te_last_work's ops minus those target-part sharing saved (the same as te_last_work's
 * ops without sharing). `bundles` (nullable): the number of bundles formed. The sweep's counters
 * are read from the device (synchronises the device). */
te_status te_last_alu_ops(te_handle* h, uint64_t* ops, int32_t* bundles);

/* How the last te_estimate / te_surrogate_test / te_delay_scan call ran its estimates (a delay
 * scan counts every (delay, estimate) pair): paths[0] = on the lane kernel (one estimate per
 * lane), paths[1] = in bundles of up to 3, paths[2] = unshared. `paths` has three entries. */
te_status te_last_paths(te_handle* h, int32_t* paths);

/* The work of the last te_estimate / te_surrogate_test / te_delay_scan call split by pass:
 * pairs[0], pairs[1] = (query, reference) pair evaluations of pass 1 (the k-th neighbour search,
 * Eq. 9's eps) and of pass 2 (the three range counts), summed over estimates (pairs[0] +
 * pairs[1] = te_last_work's pairs); cycles[0], cycles[1] = SM clock cycles the warps spent in
 * each pass, summed over warps (pass 2 includes the digamma terms), measured on the device by
 * the sweep: their ratio splits the kernel time between the passes. Exhaustive search: N^2
 * pairs per pass and cycles 0 (not measured). Both arrays have two entries and must be
 * non-NULL; synchronises the device. */
te_status te_last_pass_work(te_handle* h, uint64_t* pairs, uint64_t* cycles);

/* Batching mode of te_estimate / te_surrogate_test. per_instance = 0 (default): one persistent
 * launch for the whole batch, captured in a CUDA graph. per_instance = 1: the unshared persistent
 * kernel and tables, launched once per instance with a grid of that instance's work items and no
 * graph, the way an unbatched implementation runs one search space per launch (the comparison of
 * the Implementation section's "several chunks per launch" design). Per instance, target parts
 * are not shared (no lane kernel, no bundles); an estimate that fits shared memory is staged whole
 * as in one launch. Counts and eps are bit-identical in both modes; TE is bit-identical to a
 * batched launch without sharing (te_set_sharing(h, 0)) and otherwise agrees within the two
 * err_bound values. */
te_status te_set_batching(te_handle* h, int32_t per_instance);

/* te_surrogate_test_static - te_surrogate_test for one series, for callers that cannot allocate
 * GPU memory. The paper has no counterpart: this exists for embedding the library where
 * cudaMalloc is not allowed (a host process whose device memory is owned by another runtime or
 * pool, a fixed memory budget, code that must not cause the implicit synchronisation an
 * allocation can bring). It needs no handle and allocates nothing on the device or the host.
 * Its scratch (work-queue head, per-item partial sums, per-estimate TE, digamma table) is one
 * fixed static device array of about 2.6 MiB that every GPU using it holds until the process
 * exits.
 *   Runs on the calling thread's current device. The first call on a device sets it up (looks
 *   up the array's device address, fills the digamma table and waits for that on `stream`, sets
 *   kernel attributes). With the CUDA driver's lazy module loading, that first call is also when
 *   the driver maps the array and its kernels on the device, which allocates device memory and
 *   may synchronise: make the first call on each device where that is acceptable (at start-up),
 *   and before any stream capture; later calls allocate nothing. Calls reuse the array; the queue head is cleared on each
 *   call and every other value is rewritten before it is read. Calls whose GPU work overlaps
 *   (other streams or host threads) race on the array and must be serialised by the caller.
 *   Limits: k <= 4, d = 1..5, N = R * window <= 8192, n_t <= 256, n_t * (S + 1) <= 65536
 *   estimates; beyond them TE_ENOTIMPL and a message. Out-of-range permutation entries are
 *   read as repetition 0 (no flag is reported).
 *   Outputs as te_surrogate_test with n_series = 1: te_orig [n_t], te_surr [n_t][S], p [n_t].
 *   msg (nullable, msg_len bytes) receives the reason of a failed call. */
te_status te_surrogate_test_static(const te_series* series, const int32_t* t_starts, int32_t n_t,
                                   int32_t window, int32_t S, int32_t k, double* te_orig,
                                   double* te_surr, double* p, void* stream, char* msg,
                                   int32_t msg_len);

#ifdef __cplusplus
}
#endif
#endif /* TE_GB300_H */
