// The paper's approximate threshold search (given in its source as a
// comment, Sect. 2): each series mapped onto [0, 1], RR evaluated at a fixed
// grid of thresholds, and for each target the grid threshold whose RR is the
// closest.  Kept for comparison with the exact selection of select.cu.
//
// Grid, in the series' own units and FP32 with correctly rounded operations
// so that any implementation reproduces it: thr_i = i * ((max - min) / n),
// i = 1..n.  A cell is recurrent at thr_i iff d <= thr_i (upper triangle).
#include <cstdint>
#include "rqa_common.cuh"

namespace rqa {

constexpr int GT = 256;  // threads of the grid kernels

// Per series: min and max of the values, then the grid.
__global__ void __launch_bounds__(GT)
k_grid_thr(const float *__restrict__ y, const SeriesDev *__restrict__ series, int n_thr, float *thr)
{
    __shared__ float smin[GT / 32], smax[GT / 32];
    const int s = blockIdx.x;
    const SeriesDev sd = series[s];
    float lo = 3.4e38f, hi = -3.4e38f;
    for (int i = threadIdx.x; i < sd.n; i += GT) {
        const float v = y[sd.off + i];
        lo = fminf(lo, v);
        hi = fmaxf(hi, v);
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = fminf(lo, __shfl_xor_sync(FULL, lo, o));
        hi = fmaxf(hi, __shfl_xor_sync(FULL, hi, o));
    }
    if ((threadIdx.x & 31) == 0) {
        smin[threadIdx.x >> 5] = lo;
        smax[threadIdx.x >> 5] = hi;
    }
    __syncthreads();
    lo = smin[0];
    hi = smax[0];
    for (int w = 1; w < GT / 32; ++w) {
        lo = fminf(lo, smin[w]);
        hi = fmaxf(hi, smax[w]);
    }
    const float scale = __fdiv_rn(__fsub_rn(hi, lo), (float)n_thr);
    for (int i = threadIdx.x; i < n_thr; i += GT)
        thr[(int64_t)s * n_thr + i] = __fmul_rn((float)(i + 1), scale);
}

// Counting pass: for every cell the number of grid thresholds below its
// distance, r = #{i : thr_i < d} in 0..n (a binary search over the grid keys
// in shared memory), histogrammed per series: bin r holds the cells first
// recurrent at thr_{r+1}.  Persistent CTAs over the band items of the exact
// selection.
template <int M, int TAU>
__global__ void __launch_bounds__(GT)
k_count_grid(CellArgs a, const float *__restrict__ thr, int n_thr, uint64_t *hist)
{
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t *h = reinterpret_cast<uint32_t *>(smem);   // n_thr + 1 bins
    uint32_t *tk = h + n_thr + 1;                         // grid keys, padded to a power of two
    __shared__ int slot, next_band;
    const int lane = threadIdx.x & 31;
    int npow = 1;
    while (npow < n_thr) npow <<= 1;
    for (;;) {
        const int it = next_item(a.queue, a.n_items, &slot);
        if (it < 0) break;
        const Item item = a.items[it];
        const SeriesDev sd = a.series[item.s];
        for (int x = threadIdx.x; x <= n_thr; x += GT) h[x] = 0;
        for (int x = threadIdx.x; x < npow; x += GT)
            tk[x] = x < n_thr ? __float_as_uint(thr[(int64_t)item.s * n_thr + x]) : 0xffffffffu;
        if (threadIdx.x == 0) next_band = item.b_lo;
        __syncthreads();
        const float *ys = a.y + sd.off;
        for (;;) {
            int b = 0;
            if (lane == 0) b = atomicAdd(&next_band, 1);
            b = __shfl_sync(FULL, b, 0);
            if (b >= item.b_hi) break;
            int d_lo, d_hi;
            band_range(b, BAND, sd.ne, d_lo, d_hi);
            const int rows = sd.ne - d_lo;
            for (int i0 = 0; i0 < rows; i0 += 32) {
                const int i = i0 + lane;
                BandTile<M, TAU, BAND> tile;
                tile.load(ys, sd.n, i, d_lo, rows, sd.tau, sd.m);
#pragma unroll 4
                for (int j = 0; j < BAND; ++j) {
                    const int dl = d_lo + j;
                    const bool valid = i < sd.ne - dl;
                    if (!(TAU > 0 || valid)) continue;
                    const uint32_t key = __float_as_uint(tile.dist(ys, j, i, dl, sd.tau, sd.m));
                    int r = 0;  // grid keys below key (non-negative floats order as their bits)
                    for (int step = npow >> 1; step > 0; step >>= 1)
                        if (tk[r + step - 1] < key) r += step;
                    if (r < npow && r < n_thr && tk[r] < key) ++r;
                    if (valid) atomicAdd(&h[min(r, n_thr)], 1u);
                }
            }
        }
        __syncthreads();
        uint64_t *gh = hist + (int64_t)item.s * (n_thr + 1);
        for (int x = threadIdx.x; x <= n_thr; x += GT)
            if (h[x]) atomicAdd(reinterpret_cast<unsigned long long *>(gh + x), (unsigned long long)h[x]);
        __syncthreads();
    }
}

// Per series: grid counts C_j = #{d <= thr_j} (prefix sums of the bins) and,
// for each target, the first j minimising |C_j den - rr_num P| (exact).
__global__ void __launch_bounds__(GT)
k_select_grid(const uint64_t *hist, const float *thr, const SeriesDev *series, int n_thr,
              const int32_t *rr_num, int rr_den, int K, float *eps_out, double *rr_out,
              uint64_t *count_out)
{
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t *c = reinterpret_cast<uint64_t *>(smem);  // n_thr prefix counts
    const int s = blockIdx.x;
    const uint64_t *h = hist + (int64_t)s * (n_thr + 1);
    if (threadIdx.x == 0) {
        uint64_t acc = 0;
        for (int j = 0; j < n_thr; ++j) {
            acc += h[j];
            c[j] = acc;
        }
    }
    __syncthreads();
    const uint64_t P = series[s].P;
    for (int k = threadIdx.x; k < K; k += GT) {
        const unsigned __int128 target = (unsigned __int128)(uint64_t)rr_num[k] * P;
        int best = 0;
        unsigned __int128 best_err = ~(unsigned __int128)0;
        for (int j = 0; j < n_thr; ++j) {
            const unsigned __int128 v = (unsigned __int128)c[j] * (unsigned)rr_den;
            const unsigned __int128 err = v > target ? v - target : target - v;
            if (err < best_err) {
                best_err = err;
                best = j;
            }
        }
        const int64_t o = (int64_t)s * K + k;
        eps_out[o] = thr[(int64_t)s * n_thr + best];
        if (rr_out) rr_out[o] = (double)c[best] / (double)P;
        if (count_out) count_out[o] = c[best];
    }
}

cudaError_t launch_grid_select(const CellArgs &a, int S, int n_thr, float *thr, uint64_t *hist,
                               const int32_t *rr_num_dev, int rr_den, int K, float *eps_out,
                               double *rr_out, uint64_t *count_out, int grid, int embed,
                               cudaStream_t st)
{
    if (!a.y || !a.series || !a.items || !a.queue || a.n_items < 1 || a.band != BAND || S < 1 ||
        n_thr < 1 || n_thr > 1024 || !thr || !hist || !rr_num_dev || K < 1 || K > KMAX || !eps_out ||
        grid < 1)
        return cudaErrorInvalidValue;
    k_grid_thr<<<S, GT, 0, st>>>(a.y, a.series, n_thr, thr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int smem = (n_thr + 1 + 1024) * 4;
    void (*kern)(CellArgs, const float *, int, uint64_t *);
    switch (embed) {
    case E_M1T1: kern = k_count_grid<1, 1>; break;
    case E_M3T1: kern = k_count_grid<3, 1>; break;
    case E_M3T3: kern = k_count_grid<3, 3>; break;
    case E_M1: kern = k_count_grid<1, 0>; break;
    case E_M2: kern = k_count_grid<2, 0>; break;
    case E_M3: kern = k_count_grid<3, 0>; break;
    case E_M4: kern = k_count_grid<4, 0>; break;
    default: kern = k_count_grid<0, 0>; break;
    }
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess)
        return e;
    grid = persistent_cap(reinterpret_cast<const void *>(kern), smem, grid, GT);
    kern<<<grid, GT, smem, st>>>(a, thr, n_thr, hist);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_select_grid<<<S, GT, n_thr * 8, st>>>(hist, thr, a.series, n_thr, rr_num_dev, rr_den, K, eps_out,
                                            rr_out, count_out);
    return cudaGetLastError();
}

}  // namespace rqa
