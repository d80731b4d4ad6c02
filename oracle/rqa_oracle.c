/*
 * Plain-C oracle for averaged RQA -- TEST INFRASTRUCTURE, not product code.
 *
 * Used only by the tests, the smoke check and the benchmark's CPU baseline to
 * check and time the CUDA library; it shares no code with it.  Everything here
 * is the definition written out cell by cell, for series too long to
 * materialise in NumPy:
 *
 *   delay vectors  x_i = (y[i], y[i+tau], ..., y[i+(m-1)tau]), i < Ne,
 *                  Ne = N - (m-1)tau                          (Sect. 3.3)
 *   distance       d_ij = max_q |y[i+q tau] - y[j+q tau]|      (Eq. 1, max norm)
 *   recurrence     R_ij = [d_ij <= eps], upper triangle i < j  (Eq. 1-2, Sect. 4)
 *   lines          maximal runs of R along each diagonal j-i   (Eq. 4)
 *
 * All distance arithmetic is FP32 subtract / fabsf / compare, with no
 * contraction and no fast-math, so results are exact IEEE values.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_KMAX 128 /* thresholds per call (capacity of the per-thread arrays) */

static inline float orc_dist(const float *y, int64_t i, int64_t j, int m, int tau)
{
    float d = fabsf(y[i] - y[j]);
    for (int q = 1; q < m; ++q) {
        float v = fabsf(y[i + (int64_t)q * tau] - y[j + (int64_t)q * tau]);
        if (v > d) d = v;
    }
    return d;
}

/* All P = Ne(Ne-1)/2 distances, diagonal delta = 1..Ne-1 in order, then i. */
int orc_distances(const float *y, int64_t n, int m, int tau, float *out)
{
    int64_t ne = n - (int64_t)(m - 1) * tau;
    int64_t o = 0;
    for (int64_t dl = 1; dl < ne; ++dl)
        for (int64_t i = 0; i + dl < ne; ++i)
            out[o++] = orc_dist(y, i, i + dl, m, tau);
    return 0;
}

/*
 * For each threshold t_k: le[k] = #{d <= t_k}, lt[k] = #{d < t_k} over all
 * upper-triangle cells.  Used as the exactness certificate of a threshold:
 * t_k is the T_k-th smallest distance iff lt[k] < T_k <= le[k].
 */
int orc_count(const float *y, int64_t n, int m, int tau, const float *thr, int K,
              uint64_t *le, uint64_t *lt, int threads)
{
    if (K < 1 || K > ORC_KMAX) return -1;
    int64_t ne = n - (int64_t)(m - 1) * tau;
    for (int k = 0; k < K; ++k) { le[k] = 0; lt[k] = 0; }
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel
#endif
    {
        uint64_t ple[ORC_KMAX], plt[ORC_KMAX];
        for (int k = 0; k < K; ++k) { ple[k] = 0; plt[k] = 0; }
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 16)
#endif
        for (int64_t dl = 1; dl < ne; ++dl) {
            for (int64_t i = 0; i + dl < ne; ++i) {
                float d = orc_dist(y, i, i + dl, m, tau);
                for (int k = 0; k < K; ++k) {
                    ple[k] += (d <= thr[k]);
                    plt[k] += (d < thr[k]);
                }
            }
        }
#ifdef _OPENMP
#pragma omp critical
#endif
        for (int k = 0; k < K; ++k) { le[k] += ple[k]; lt[k] += plt[k]; }
    }
    return 0;
}

/*
 * Diagonal line statistics for each threshold eps_k (Eq. 4, Sect. 4):
 *   hist[k*(Ne-1) + l-1] = P_k(l), number of maximal diagonal runs of length l
 *                          (hist may be NULL),
 *   count[k]   = recurrent cells,
 *   stencil[k] = recurrent cells with a recurrent diagonal neighbour,
 *   lmax[k]    = longest run,
 *   short_hist[k*n_short + l-1] = P_k(l) for l <= n_short (may be NULL).
 * Each diagonal is scanned from i = 0 upwards with one open-run counter per
 * threshold.
 */
int orc_lines(const float *y, int64_t n, int m, int tau, const float *eps, int K,
              uint64_t *hist, uint64_t *count, uint64_t *stencil, uint32_t *lmax,
              uint64_t *short_hist, int n_short, int threads)
{
    if (K < 1 || K > ORC_KMAX) return -1;
    int64_t ne = n - (int64_t)(m - 1) * tau;
    int64_t nl = ne - 1;
    if (hist) memset(hist, 0, sizeof(uint64_t) * (size_t)K * (size_t)(nl > 0 ? nl : 0));
    if (short_hist) memset(short_hist, 0, sizeof(uint64_t) * (size_t)K * (size_t)n_short);
    for (int k = 0; k < K; ++k) { count[k] = 0; stencil[k] = 0; lmax[k] = 0; }
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel
#endif
    {
        uint64_t pc[ORC_KMAX], ps[ORC_KMAX];
        uint32_t pm[ORC_KMAX];
        int64_t run[ORC_KMAX];
        uint64_t *ph = NULL;
        uint64_t *psh = NULL;
        if (hist) ph = (uint64_t *)calloc((size_t)K * (size_t)nl, sizeof(uint64_t));
        if (short_hist) psh = (uint64_t *)calloc((size_t)K * (size_t)n_short, sizeof(uint64_t));
        for (int k = 0; k < K; ++k) { pc[k] = 0; ps[k] = 0; pm[k] = 0; }
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 16)
#endif
        for (int64_t dl = 1; dl < ne; ++dl) {
            int64_t len = ne - dl;
            for (int k = 0; k < K; ++k) run[k] = 0;
            int prev_rec[ORC_KMAX];
            for (int k = 0; k < K; ++k) prev_rec[k] = 0;
            float dn = (len > 0) ? orc_dist(y, 0, dl, m, tau) : 0.0f;
            for (int64_t i = 0; i <= len; ++i) {
                /* i == len is a virtual non-recurrent cell closing the last run. */
                float d = dn;
                dn = (i + 1 < len) ? orc_dist(y, i + 1, i + 1 + dl, m, tau) : 0.0f;
                for (int k = 0; k < K; ++k) {
                    int rec = (i < len) && (d <= eps[k]);
                    if (rec) {
                        pc[k]++;
                        int nb = prev_rec[k] || ((i + 1 < len) && (dn <= eps[k]));
                        if (nb) ps[k]++;
                        run[k]++;
                    } else if (run[k] > 0) {
                        int64_t l = run[k];
                        if (ph) ph[(size_t)k * nl + (size_t)(l - 1)]++;
                        if (psh && l <= n_short) psh[(size_t)k * n_short + (size_t)(l - 1)]++;
                        if ((uint32_t)l > pm[k]) pm[k] = (uint32_t)l;
                        run[k] = 0;
                    }
                    prev_rec[k] = rec;
                }
            }
        }
#ifdef _OPENMP
#pragma omp critical
#endif
        {
            for (int k = 0; k < K; ++k) {
                count[k] += pc[k];
                stencil[k] += ps[k];
                if (pm[k] > lmax[k]) lmax[k] = pm[k];
            }
            if (ph)
                for (size_t t = 0; t < (size_t)K * (size_t)nl; ++t) hist[t] += ph[t];
            if (psh)
                for (size_t t = 0; t < (size_t)K * (size_t)n_short; ++t) short_hist[t] += psh[t];
        }
        free(ph);
        free(psh);
    }
    return 0;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
