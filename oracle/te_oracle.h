/* Ensemble transfer-entropy oracle: plain, slow, brute-force KSG estimator on the CPU.
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the benchmark's CPU-baseline
 * leg call this code. The library's compute path never includes, links or calls it, and this
 * file shares no code with it.
 *
 * Point layout here is array-of-structures: points[i * D + c], i = r * W + w (repetitions
 * concatenated in order, each contributing its W window samples in time order).
 * Return codes: 0 ok, 1 invalid argument, 2 embedding reaches outside the recorded samples,
 * 3 out of memory.
 */
#ifndef TE_ORACLE_H
#define TE_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct oracle_series {
    const float* src;    /* [R][T] source X                         */
    const float* tgt;    /* [R][T] target Y                         */
    int32_t R, T, d, tau, u, S;
    const int32_t* perms; /* [S][R] or NULL                         */
} oracle_series;

typedef struct oracle_instance {
    int32_t series, t_start, window, perm; /* perm -1: original pairing */
} oracle_instance;

/* Eq. 6/7 delay embedding + Eq. 10 point set. dy, dx: target / source embedding dimensions. */
int oracle_embed(const float* src, const float* tgt, int R, int T, int dy, int dx, int tau, int u,
                 int t_start, int W, const int32_t* perm, float* points);

/* k-th nearest neighbour distance (max-norm, self excluded) by a full sort of the N-1
 * distances; nn (nullable) receives the k nearest indices, ties by lower index. */
int oracle_knn(const float* points, int N, int D, int k, float* eps, int32_t* nn);

/* Strict range counts in the marginal spaces y-, (y_t, y-), (y-, x-): counts[3][N]. */
int oracle_range_count(const float* points, int N, int dy, int dx, const float* eps,
                       int32_t* counts);

/* eps and counts ([3][n_idx]: n_z, n_yz, n_xz) of the query points idx[0..n_idx-1] only, by the
 * same per-point definitions as oracle_knn / oracle_range_count; host threads split the points. */
int oracle_points_at(const float* points, int N, int dy, int dx, int k, const int32_t* idx, int n_idx,
                     int n_threads, float* eps, int32_t* counts);

/* Digamma at a positive integer, FP64, from psi(1) = -gamma and psi(n+1) = psi(n) + 1/n. */
double oracle_digamma(int n);

/* TE of one point set (Eq. 9 / Eq. 10). eps, counts nullable outputs. */
int oracle_te_points(const float* points, int N, int dy, int dx, int k, double* te, float* eps,
                     int32_t* counts);

/* TE of many instances, host threads split the instances. counts/eps (nullable) are written
 * concatenated in instance order: counts block of instance i is [3][N_i], eps block [N_i]. */
int oracle_te_batch(const oracle_series* series, int n_series, const oracle_instance* inst,
                    int n_inst, int k, int n_threads, double* te, int32_t* counts, float* eps);

/* p-value: share of surrogate values >= the original value. */
double oracle_pvalue(double te_orig, const double* te_surr, int S);

#ifdef __cplusplus
}
#endif
#endif
