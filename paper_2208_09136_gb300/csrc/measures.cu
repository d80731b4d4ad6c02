// Average diagonal line length L and line-length entropy ENTR per target, and
// their averages over the targets.  Sect. 2 ends by noting that averaging over
// a range of recurrence rates applies to other RQA measures than DET; these
// are the two diagonal-line measures usually reported with it (Marwan et al.
// 2007, Phys. Rep. 438, Sect. 5.1), over lines of length >= lmin:
//   N_l  = sum_{l >= lmin} P(l),  L = sum_{l >= lmin} l P(l) / N_l,
//   ENTR = -sum_{l >= lmin} p(l) ln p(l),  p(l) = P(l) / N_l.
// The input is the full histogram the line pass wrote (upper triangle; both
// triangles hold the same lines, so the ratios equal the full-matrix ones).
// loi: the whole matrix with the line of identity, i.e. P(l) -> 2 P(l) plus
// one line of length Ne.
#include <cstdint>
#include "rqa_common.cuh"

namespace rqa {

constexpr int MT = 256;  // threads per (series, target)

// One CTA per (series s, target k): integer sums first (exact in any order),
// then the entropy terms in FP64 (a fixed reduction tree).
__global__ void __launch_bounds__(MT)
k_line_measures(const uint64_t *__restrict__ hist, const int64_t *__restrict__ hoff, int K,
                const int32_t *__restrict__ lmin, int n_lmin, double *L_out, double *E_out, bool loi)
{
    __shared__ unsigned long long red_n[MT / 32][LMIN_MAX], red_m[MT / 32][LMIN_MAX];
    __shared__ double red_e[MT / 32][LMIN_MAX];
    __shared__ unsigned long long tot_n[LMIN_MAX];
    const int s = blockIdx.x / K, k = blockIdx.x - s * K;
    const int64_t nl = (hoff[s + 1] - hoff[s]) / K;  // lengths 1..nl
    const uint64_t *row = hist + hoff[s] + (int64_t)k * nl;
    const int t = threadIdx.x, w = t >> 5, lane = t & 31;
    const unsigned long long mult = loi ? 2ull : 1ull;  // lines per upper-triangle line
    const int64_t ne = nl + 1;                           // the identity line's length

    unsigned long long n[LMIN_MAX], m[LMIN_MAX];
#pragma unroll
    for (int j = 0; j < LMIN_MAX; ++j) n[j] = m[j] = 0ull;
    for (int64_t l = 1 + t; l <= nl; l += MT) {
        const unsigned long long c = mult * row[l - 1];
        if (!c) continue;
#pragma unroll
        for (int j = 0; j < LMIN_MAX; ++j)
            if (j < n_lmin && l >= lmin[j]) {
                n[j] += c;
                m[j] += c * (unsigned long long)l;
            }
    }
    if (loi && t == 0)  // the line of identity: one line of length Ne
#pragma unroll
        for (int j = 0; j < LMIN_MAX; ++j)
            if (j < n_lmin && ne >= lmin[j]) {
                n[j] += 1ull;
                m[j] += (unsigned long long)ne;
            }
#pragma unroll
    for (int j = 0; j < LMIN_MAX; ++j) {
        for (int o = 16; o > 0; o >>= 1) {
            n[j] += __shfl_xor_sync(FULL, n[j], o);
            m[j] += __shfl_xor_sync(FULL, m[j], o);
        }
        if (lane == 0) {
            red_n[w][j] = n[j];
            red_m[w][j] = m[j];
        }
    }
    __syncthreads();
    if (t < n_lmin) {
        unsigned long long sn = 0, sm = 0;
        for (int q = 0; q < MT / 32; ++q) {
            sn += red_n[q][t];
            sm += red_m[q][t];
        }
        tot_n[t] = sn;
        if (L_out)
            L_out[((int64_t)s * K + k) * n_lmin + t] =
                sn ? (double)sm / (double)sn : __longlong_as_double(0x7ff8000000000000ll);
    }
    __syncthreads();
    if (!E_out) return;
    double e[LMIN_MAX];
#pragma unroll
    for (int j = 0; j < LMIN_MAX; ++j) e[j] = 0.0;
    for (int64_t l = 1 + t; l <= nl; l += MT) {
        const unsigned long long c = mult * row[l - 1];
        if (!c) continue;
#pragma unroll
        for (int j = 0; j < LMIN_MAX; ++j)
            if (j < n_lmin && l >= lmin[j]) {
                const double p = (double)c / (double)tot_n[j];
                e[j] -= p * log(p);
            }
    }
    if (loi && t == 0)
#pragma unroll
        for (int j = 0; j < LMIN_MAX; ++j)
            if (j < n_lmin && ne >= lmin[j]) {
                const double p = 1.0 / (double)tot_n[j];
                e[j] -= p * log(p);
            }
#pragma unroll
    for (int j = 0; j < LMIN_MAX; ++j) {
        for (int o = 16; o > 0; o >>= 1) e[j] += __shfl_xor_sync(FULL, e[j], o);
        if (lane == 0) red_e[w][j] = e[j];
    }
    __syncthreads();
    if (t < n_lmin) {
        double se = 0.0;
        for (int q = 0; q < MT / 32; ++q) se += red_e[q][t];
        E_out[((int64_t)s * K + k) * n_lmin + t] = se;
    }
}

// Averages over the K targets of one series: FP64 sum in k order, then / K
// (the reduction of Eq. avgDET).
__global__ void k_measure_avg(const double *v, int K, int n_lmin, double *avg)
{
    const int s = blockIdx.x, j = threadIdx.x;
    if (j >= n_lmin) return;
    double acc = 0.0;
    for (int k = 0; k < K; ++k) acc = acc + v[((int64_t)s * K + k) * n_lmin + j];
    avg[(int64_t)s * n_lmin + j] = acc / (double)K;
}

cudaError_t launch_line_measures(const uint64_t *hist, const int64_t *hoff_dev, int S, int K,
                                 const int32_t *lmin_dev, int n_lmin, double *L_out,
                                 double *E_out, double *L_avg, double *E_avg, bool loi,
                                 cudaStream_t st)
{
    if (!hist || !hoff_dev || !lmin_dev || S < 1 || K < 1 || K > KMAX || n_lmin < 1 ||
        n_lmin > LMIN_MAX || (L_avg && !L_out) || (E_avg && !E_out))
        return cudaErrorInvalidValue;
    k_line_measures<<<S * K, MT, 0, st>>>(hist, hoff_dev, K, lmin_dev, n_lmin, L_out, E_out, loi);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (L_avg) k_measure_avg<<<S, 32, 0, st>>>(L_out, K, n_lmin, L_avg);
    if (E_avg) k_measure_avg<<<S, 32, 0, st>>>(E_out, K, n_lmin, E_avg);
    return cudaGetLastError();
}

}  // namespace rqa

namespace rqa {

// Laminarity and trapping time from a vertical-line histogram V_k(l)
// (Marwan et al. 2007, Sect. 5.1; Sect. 2 of the paper extends the RR
// averaging to such measures):
//   LAM = sum_{l >= vmin} l V(l) / sum_{l >= 1} l V(l)   (the denominator is
//         every recurrent cell: each lies on exactly one vertical line)
//   TT  = sum_{l >= vmin} l V(l) / sum_{l >= vmin} V(l)  (NaN: no such line)
// FP64 ratios of exact integer sums; one CTA per (series, target).
__global__ void __launch_bounds__(MT)
k_lam_tt(const uint64_t *__restrict__ hist, const int64_t *__restrict__ hoff, int K,
         const int32_t *__restrict__ vmin, int n_vmin, double *lam_out, double *tt_out)
{
    __shared__ unsigned long long red[MT / 32][2 * LMIN_MAX + 1];
    const int s = blockIdx.x / K, k = blockIdx.x - s * K;
    const int64_t nl = (hoff[s + 1] - hoff[s]) / K;
    const uint64_t *row = hist + hoff[s] + (int64_t)k * nl;
    const int t = threadIdx.x, w = t >> 5, lane = t & 31;
    unsigned long long n[LMIN_MAX], m[LMIN_MAX], all = 0ull;
#pragma unroll
    for (int j = 0; j < LMIN_MAX; ++j) n[j] = m[j] = 0ull;
    for (int64_t l = 1 + t; l <= nl; l += MT) {
        const unsigned long long c = row[l - 1];
        if (!c) continue;
        all += c * (unsigned long long)l;
#pragma unroll
        for (int j = 0; j < LMIN_MAX; ++j)
            if (j < n_vmin && l >= vmin[j]) {
                n[j] += c;
                m[j] += c * (unsigned long long)l;
            }
    }
    for (int o = 16; o > 0; o >>= 1) all += __shfl_xor_sync(FULL, all, o);
#pragma unroll
    for (int j = 0; j < LMIN_MAX; ++j)
        for (int o = 16; o > 0; o >>= 1) {
            n[j] += __shfl_xor_sync(FULL, n[j], o);
            m[j] += __shfl_xor_sync(FULL, m[j], o);
        }
    if (lane == 0) {
#pragma unroll
        for (int j = 0; j < LMIN_MAX; ++j) {
            red[w][j] = n[j];
            red[w][LMIN_MAX + j] = m[j];
        }
        red[w][2 * LMIN_MAX] = all;
    }
    __syncthreads();
    if (t < n_vmin) {
        unsigned long long sn = 0, sm = 0, sa = 0;
        for (int q = 0; q < MT / 32; ++q) {
            sn += red[q][t];
            sm += red[q][LMIN_MAX + t];
            sa += red[q][2 * LMIN_MAX];
        }
        const double nan = __longlong_as_double(0x7ff8000000000000ll);
        const int64_t o = ((int64_t)s * K + k) * n_vmin + t;
        if (lam_out) lam_out[o] = sa ? (double)sm / (double)sa : nan;
        if (tt_out) tt_out[o] = sn ? (double)sm / (double)sn : nan;
    }
}

cudaError_t launch_lam_tt(const uint64_t *hist, const int64_t *hoff_dev, int S, int K,
                          const int32_t *vmin_dev, int n_vmin, double *lam_out, double *tt_out,
                          double *lam_avg, double *tt_avg, cudaStream_t st)
{
    if (!hist || !hoff_dev || !vmin_dev || S < 1 || K < 1 || K > KMAX || n_vmin < 1 ||
        n_vmin > LMIN_MAX || (lam_avg && !lam_out) || (tt_avg && !tt_out))
        return cudaErrorInvalidValue;
    k_lam_tt<<<S * K, MT, 0, st>>>(hist, hoff_dev, K, vmin_dev, n_vmin, lam_out, tt_out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (lam_avg) k_measure_avg<<<S, 32, 0, st>>>(lam_out, K, n_vmin, lam_avg);
    if (tt_avg) k_measure_avg<<<S, 32, 0, st>>>(tt_out, K, n_vmin, tt_avg);
    return cudaGetLastError();
}

}  // namespace rqa
