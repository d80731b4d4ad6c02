// Per-series finalisation after the line pass: DET_k for each lmin and its
// average over the targets (Eq. 4, Eq. avgDET), and the short line lengths
// copied into the caller's full histogram with the stencil counts.
#include <cstdint>
#include "rqa_common.cuh"

namespace rqa {

// DET_k(lmin) = (C_k - sum_{l < lmin} l P_k(l)) / C_k  (Eq. 4), an FP64 ratio of
// exact integers, and the average over k in order (Eq. avgDET).  loi: the
// whole matrix with the line of identity, (2 num + Ne [Ne >= lmin]) / (2 C + Ne).
__global__ void k_finalize_det(LineBufs lb, const SeriesDev *series, int K, const int32_t *lmin,
                               int n_lmin, double *det, double *det_avg, bool loi)
{
    __shared__ double dk[KMAX * LMIN_MAX];
    const int s = blockIdx.x;
    const int t = threadIdx.x;
    if (t < K) {
        const int64_t o = (int64_t)s * K + t;
        const uint64_t C = lb.count[o];
        const uint64_t *h = lb.hshort + o * LSH;
        for (int j = 0; j < n_lmin; ++j) {
            uint64_t shortmass = 0;
            for (int l = 1; l < lmin[j]; ++l) shortmass += (uint64_t)l * h[l - 1];
            uint64_t num = C - shortmass, den = C;
            if (loi) {
                const uint64_t ne = (uint64_t)series[s].ne;
                num = 2 * num + (ne >= (uint64_t)lmin[j] ? ne : 0);
                den = 2 * den + ne;
            }
            const double v = (double)num / (double)den;
            dk[t * LMIN_MAX + j] = v;
            if (det) det[o * n_lmin + j] = v;
        }
    }
    __syncthreads();
    if (t < n_lmin) {
        double acc = 0.0;
        for (int k = 0; k < K; ++k) acc = acc + dk[k * LMIN_MAX + t];
        det_avg[(int64_t)s * n_lmin + t] = acc / (double)K;
    }
}

cudaError_t launch_finalize_det(const LineBufs &lb, const SeriesDev *series, int S, int K,
                                const int32_t *lmin_dev, int n_lmin, double *det,
                                double *det_avg, bool loi, cudaStream_t st)
{
    if (K < 1 || K > KMAX) return cudaErrorInvalidValue;
    k_finalize_det<<<S, 128, 0, st>>>(lb, series, K, lmin_dev, n_lmin, det, det_avg, loi);  // a thread per target
    return cudaGetLastError();
}

// Short lengths into the caller's full histogram; stencil count C_k - P_k(1).
__global__ void k_finalize_hist(LineBufs lb, const SeriesDev *series, int K, uint64_t *stencil)
{
    const int s = blockIdx.x;
    const int ne = series[s].ne;
    const int row = ne - 1 + (lb.loi ? 1 : 0);  // lengths per target (vertical, identity: Ne)
    const int nl = min(LSH, row);
    for (int x = threadIdx.x; x < K * LSH; x += blockDim.x) {
        const int k = x / LSH, l = x - k * LSH + 1;
        const uint64_t v = lb.hshort[((int64_t)s * K + k) * LSH + (l - 1)];
        if (lb.hist && l <= nl) lb.hist[lb.hist_off[s] + (int64_t)k * row + (l - 1)] = v;
    }
    if (stencil && threadIdx.x < K) {
        const int64_t o = (int64_t)s * K + threadIdx.x;
        stencil[o] = lb.count[o] - lb.hshort[o * LSH];
    }
}

cudaError_t launch_finalize_hist(const LineBufs &lb, const SeriesDev *series, int S, int K,
                                 uint64_t *stencil, cudaStream_t st)
{
    k_finalize_hist<<<S, 256, 0, st>>>(lb, series, K, stencil);
    return cudaGetLastError();
}

}  // namespace rqa
