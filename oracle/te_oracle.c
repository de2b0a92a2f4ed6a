/* Ensemble transfer-entropy oracle: plain, slow, brute-force KSG estimator on the CPU.
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the benchmark's CPU-baseline
 * leg call this code. The library's compute path never includes, links or calls it.
 *
 * What each function follows (Wollstadt et al., "Efficient transfer entropy analysis of
 * non-stationary neural time series", PLoS ONE 2014):
 *   oracle_embed       Eq. 6 / Eq. 7 (target past state at t-1 with dimension d and delay tau),
 *                      the same construction for the source at t-u ("State space
 *                      reconstruction" paragraph), and Eq. 10 (points pooled over repetitions r
 *                      and the samples t' of the analysis window).
 *   oracle_knn         kNN search in the highest-dimensional space (y_t, y-, x-) under the
 *                      infinity (maximum) norm ("Core algorithm" paragraph of the GPU
 *                      implementation section; distances define the radii of Eq. 9).
 *   oracle_range_count range search in the three marginal spaces of Eq. 9: y-, (y_t, y-),
 *                      (y-, x-), inside the kNN radius.
 *   oracle_digamma     the digamma function of Eq. 9 at integer arguments.
 *   oracle_te_points   Eq. 9 / Eq. 10: psi(k) + < psi(n_y- + 1) - psi(n_yt,y- + 1)
 *                      - psi(n_y-,x- + 1) > averaged over all points.
 *   oracle_pvalue      the surrogate test ("TE calculation and statistical testing against
 *                      surrogate data"): share of surrogate TE values equal to or larger than
 *                      the original TE.
 *
 * Readings where the paper is silent (the design notes list them all):
 *   - distances are computed in FP32 (the paper's data are single precision): the
 *     coordinate difference is rounded to float, its absolute value taken, the maximum kept;
 *   - range counts are strict (distance < eps), as in the KSG type-1 estimator the paper
 *     names; the query point itself is excluded from both the kNN search and the counts;
 *   - ties in neighbour identity go to the lower index (eps and counts do not depend on it);
 *   - window W means the W consecutive samples t_start .. t_start+W-1;
 *   - source past: x_{t-u}, x_{t-u-tau}, ..., x_{t-u-(dx-1)tau};
 *   - a surrogate pairs target repetition r with source repetition perm[r];
 *   - p = #{s : TE_s >= TE_0} / S, no +1 correction.
 *
 * Pins: tests/test_oracle_*.py check every function here against values that do not come
 * from this file (hand-worked examples, exhaustive enumeration, library digamma, the closed
 * form of Gaussian processes, exact invariants).
 */
#include "te_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_EULER_GAMMA 0.57721566490153286060651209008240243

/* ------------------------------------------------------------------------------------------
 * Eq. 6 / 7 / 10: the point set of one estimate
 * ---------------------------------------------------------------------------------------- */
int oracle_embed(const float* src, const float* tgt, int R, int T, int dy, int dx, int tau, int u,
                 int t_start, int W, const int32_t* perm, float* points)
{
    if (!src || !tgt || !points || R < 1 || T < 1 || dy < 0 || dx < 0 || tau < 1 || u < 0 ||
        W < 1 || t_start < 0)
        return 1;
    const int D = 1 + dy + dx;
    /* every sample index touched must lie in 0 .. T-1 */
    if (t_start + W - 1 > T - 1) return 2;
    if (dy > 0 && t_start - 1 - (dy - 1) * tau < 0) return 2;
    if (dx > 0 && t_start - u - (dx - 1) * tau < 0) return 2;
    for (int r = 0; r < R; ++r) {
        const int rs = perm ? perm[r] : r; /* source repetition paired with target r */
        if (rs < 0 || rs >= R) return 1;
        const float* y = tgt + (size_t)r * T;
        const float* x = src + (size_t)rs * T;
        for (int w = 0; w < W; ++w) {
            const int t = t_start + w;
            float* p = points + ((size_t)r * W + w) * D;
            p[0] = y[t];                                      /* y_t               */
            for (int m = 0; m < dy; ++m) p[1 + m] = y[t - 1 - m * tau];      /* Eq. 7 */
            for (int m = 0; m < dx; ++m) p[1 + dy + m] = x[t - u - m * tau]; /* at t-u */
        }
    }
    return 0;
}

/* max-norm distance between points a and b restricted to coordinates c0 .. c1-1 (FP32);
 * an empty coordinate set has distance 0 */
static float maxnorm(const float* a, const float* b, int c0, int c1)
{
    float m = 0.0f;
    for (int c = c0; c < c1; ++c) {
        float v = fabsf(a[c] - b[c]);
        if (v > m) m = v;
    }
    return m;
}

typedef struct {
    float dist;
    int32_t j;
} nb_t;

static int cmp_nb(const void* pa, const void* pb)
{
    const nb_t* a = (const nb_t*)pa;
    const nb_t* b = (const nb_t*)pb;
    if (a->dist < b->dist) return -1;
    if (a->dist > b->dist) return 1;
    return (a->j > b->j) - (a->j < b->j);
}

/* ------------------------------------------------------------------------------------------
 * kNN in the joint space: eps_i = k-th smallest of { dist(i, j) : j != i }
 * (a: scratch for the N-1 distances of point i)
 * ---------------------------------------------------------------------------------------- */
static void knn_point(const float* points, int N, int D, int k, int i, nb_t* a, float* eps_i, int32_t* nn_i)
{
    int n = 0;
    for (int j = 0; j < N; ++j) {
        if (j == i) continue;
        a[n].dist = maxnorm(points + (size_t)i * D, points + (size_t)j * D, 0, D);
        a[n].j = j;
        ++n;
    }
    qsort(a, (size_t)n, sizeof(nb_t), cmp_nb);
    *eps_i = a[k - 1].dist;
    if (nn_i)
        for (int m = 0; m < k; ++m) nn_i[m] = a[m].j;
}

int oracle_knn(const float* points, int N, int D, int k, float* eps, int32_t* nn)
{
    if (!points || !eps || D < 1 || k < 1 || N < k + 1) return 1;
    nb_t* a = (nb_t*)malloc((size_t)(N - 1) * sizeof(nb_t));
    if (!a) return 3;
    for (int i = 0; i < N; ++i) knn_point(points, N, D, k, i, a, eps + i, nn ? nn + (size_t)i * k : NULL);
    free(a);
    return 0;
}

/* ------------------------------------------------------------------------------------------
 * Range counts of Eq. 9: coordinates are [ y_t | y- (dy) | x- (dx) ]
 *   n_z  : points with max-norm distance < eps in the y- space       (coords 1 .. dy)
 *   n_yz : points with max-norm distance < eps in the (y_t, y-) space (coords 0 .. dy)
 *   n_xz : points with max-norm distance < eps in the (y-, x-) space  (coords 1 .. dy+dx)
 * ---------------------------------------------------------------------------------------- */
static void count_point(const float* points, int N, int dy, int dx, int i, float e, int32_t* nz_i,
                        int32_t* nyz_i, int32_t* nxz_i)
{
    const int D = 1 + dy + dx;
    const float* pi = points + (size_t)i * D;
    int32_t nz = 0, nyz = 0, nxz = 0;
    for (int j = 0; j < N; ++j) {
        if (j == i) continue;
        const float* pj = points + (size_t)j * D;
        if (maxnorm(pi, pj, 1, 1 + dy) < e) ++nz;
        if (maxnorm(pi, pj, 0, 1 + dy) < e) ++nyz;
        if (maxnorm(pi, pj, 1, D) < e) ++nxz;
    }
    *nz_i = nz;
    *nyz_i = nyz;
    *nxz_i = nxz;
}

int oracle_range_count(const float* points, int N, int dy, int dx, const float* eps,
                       int32_t* counts)
{
    if (!points || !eps || !counts || N < 1 || dy < 0 || dx < 0) return 1;
    for (int i = 0; i < N; ++i)
        count_point(points, N, dy, dx, i, eps[i], counts + i, counts + (size_t)N + i, counts + (size_t)2 * N + i);
    return 0;
}

/* eps and the three counts of selected query points only (the same per-point definitions as
 * oracle_knn / oracle_range_count), host threads split the points: for checking outputs of
 * point sets too large to evaluate whole. counts is [3][n_idx]. */
typedef struct {
    const float* points;
    int N, dy, dx, k, n_idx, tid, nthreads, rc;
    const int32_t* idx;
    float* eps;
    int32_t* counts;
} at_job;

static void* at_worker(void* arg)
{
    at_job* jb = (at_job*)arg;
    const int D = 1 + jb->dy + jb->dx;
    nb_t* a = (nb_t*)malloc((size_t)(jb->N - 1) * sizeof(nb_t));
    if (!a) {
        jb->rc = 3;
        return NULL;
    }
    for (int q = jb->tid; q < jb->n_idx; q += jb->nthreads) {
        const int i = jb->idx[q];
        knn_point(jb->points, jb->N, D, jb->k, i, a, jb->eps + q, NULL);
        count_point(jb->points, jb->N, jb->dy, jb->dx, i, jb->eps[q], jb->counts + q,
                    jb->counts + (size_t)jb->n_idx + q, jb->counts + (size_t)2 * jb->n_idx + q);
    }
    free(a);
    return NULL;
}

int oracle_points_at(const float* points, int N, int dy, int dx, int k, const int32_t* idx, int n_idx,
                     int n_threads, float* eps, int32_t* counts)
{
    if (!points || !idx || !eps || !counts || N < k + 1 || k < 1 || dy < 0 || dx < 0 || n_idx < 0) return 1;
    for (int q = 0; q < n_idx; ++q)
        if (idx[q] < 0 || idx[q] >= N) return 1;
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 256) n_threads = 256;
    pthread_t th[256];
    at_job jobs[256];
    for (int t = 0; t < n_threads; ++t) {
        jobs[t] = (at_job){points, N, dy, dx, k, n_idx, t, n_threads, 0, idx, eps, counts};
        pthread_create(&th[t], NULL, at_worker, &jobs[t]);
    }
    int rc = 0;
    for (int t = 0; t < n_threads; ++t) {
        pthread_join(th[t], NULL);
        if (jobs[t].rc) rc = jobs[t].rc;
    }
    return rc;
}

/* ------------------------------------------------------------------------------------------
 * digamma at positive integers
 * ---------------------------------------------------------------------------------------- */
static double* psi_table(int nmax)
{
    double* t = (double*)malloc((size_t)(nmax + 1) * sizeof(double));
    if (!t) return NULL;
    t[0] = 0.0; /* unused */
    t[1] = -ORACLE_EULER_GAMMA;
    for (int n = 1; n < nmax; ++n) t[n + 1] = t[n] + 1.0 / (double)n;
    return t;
}

double oracle_digamma(int n)
{
    if (n < 1) return NAN;
    double v = -ORACLE_EULER_GAMMA;
    for (int m = 1; m < n; ++m) v += 1.0 / (double)m;
    return v;
}

/* ------------------------------------------------------------------------------------------
 * Eq. 9 / Eq. 10
 * ---------------------------------------------------------------------------------------- */
int oracle_te_points(const float* points, int N, int dy, int dx, int k, double* te, float* eps,
                     int32_t* counts)
{
    if (!points || !te || k < 1 || N < k + 1 || dy < 0 || dx < 0) return 1;
    const int D = 1 + dy + dx;
    float* e = eps ? eps : (float*)malloc((size_t)N * sizeof(float));
    int32_t* c = counts ? counts : (int32_t*)malloc((size_t)3 * N * sizeof(int32_t));
    double* psi = psi_table(N + 1);
    int rc = (!e || !c || !psi) ? 3 : 0;
    if (!rc) rc = oracle_knn(points, N, D, k, e, NULL);
    if (!rc) rc = oracle_range_count(points, N, dy, dx, e, c);
    if (!rc) {
        double sum = 0.0;
        for (int i = 0; i < N; ++i)
            sum += psi[c[i] + 1] - psi[c[(size_t)N + i] + 1] - psi[c[(size_t)2 * N + i] + 1];
        *te = psi[k] + sum / (double)N;
    }
    if (!eps) free(e);
    if (!counts) free(c);
    free(psi);
    return rc;
}

/* ------------------------------------------------------------------------------------------
 * many instances, host threads over instances
 * ---------------------------------------------------------------------------------------- */
typedef struct {
    const oracle_series* series;
    int n_series;
    const oracle_instance* inst;
    int n_inst, k, tid, nthreads;
    double* te;
    int32_t* counts;
    float* eps;
    const int64_t* off; /* point offset of each instance */
    int rc;
} batch_job;

static void* batch_worker(void* arg)
{
    batch_job* jb = (batch_job*)arg;
    jb->rc = 0;
    for (int i = jb->tid; i < jb->n_inst; i += jb->nthreads) {
        const oracle_instance* in = &jb->inst[i];
        if (in->series < 0 || in->series >= jb->n_series) { jb->rc = 1; return NULL; }
        const oracle_series* s = &jb->series[in->series];
        const int N = s->R * in->window;
        const int D = 1 + 2 * s->d;
        const int32_t* perm = NULL;
        if (in->perm >= 0) {
            if (!s->perms || in->perm >= s->S) { jb->rc = 1; return NULL; }
            perm = s->perms + (size_t)in->perm * s->R;
        }
        float* pts = (float*)malloc((size_t)N * D * sizeof(float));
        if (!pts) { jb->rc = 3; return NULL; }
        int rc = oracle_embed(s->src, s->tgt, s->R, s->T, s->d, s->d, s->tau, s->u, in->t_start,
                              in->window, perm, pts);
        if (!rc)
            rc = oracle_te_points(pts, N, s->d, s->d, jb->k, &jb->te[i],
                                  jb->eps ? jb->eps + jb->off[i] : NULL,
                                  jb->counts ? jb->counts + 3 * jb->off[i] : NULL);
        free(pts);
        if (rc) { jb->rc = rc; return NULL; }
    }
    return NULL;
}

int oracle_te_batch(const oracle_series* series, int n_series, const oracle_instance* inst,
                    int n_inst, int k, int n_threads, double* te, int32_t* counts, float* eps)
{
    if (!series || !inst || !te || n_inst < 0 || n_series < 1) return 1;
    if (n_threads < 1) n_threads = 1;
    if (n_threads > n_inst) n_threads = n_inst > 0 ? n_inst : 1;
    int64_t* off = (int64_t*)malloc((size_t)(n_inst + 1) * sizeof(int64_t));
    if (!off) return 3;
    off[0] = 0;
    for (int i = 0; i < n_inst; ++i) {
        if (inst[i].series < 0 || inst[i].series >= n_series) { free(off); return 1; }
        off[i + 1] = off[i] + (int64_t)series[inst[i].series].R * inst[i].window;
    }
    batch_job* jobs = (batch_job*)calloc((size_t)n_threads, sizeof(batch_job));
    pthread_t* th = (pthread_t*)calloc((size_t)n_threads, sizeof(pthread_t));
    if (!jobs || !th) { free(off); free(jobs); free(th); return 3; }
    for (int t = 0; t < n_threads; ++t) {
        batch_job b = {series, n_series, inst, n_inst, k, t, n_threads, te, counts, eps, off, 0};
        jobs[t] = b;
    }
    for (int t = 1; t < n_threads; ++t) pthread_create(&th[t], NULL, batch_worker, &jobs[t]);
    batch_worker(&jobs[0]);
    int rc = jobs[0].rc;
    for (int t = 1; t < n_threads; ++t) {
        pthread_join(th[t], NULL);
        if (!rc) rc = jobs[t].rc;
    }
    free(jobs);
    free(th);
    free(off);
    return rc;
}

double oracle_pvalue(double te_orig, const double* te_surr, int S)
{
    if (S < 1 || !te_surr) return NAN;
    int n = 0;
    for (int s = 0; s < S; ++s)
        if (te_surr[s] >= te_orig) ++n;
    return (double)n / (double)S;
}
