// The learned threshold bracket: distance sketch, a small FP32 network with
// its forward and backward passes, the pinball loss, Adam, and the step that
// turns predicted intervals into the coarse buckets the first counting round
// splits at once.  None of it affects a result, only how many counting
// passes the exact selection needs.
//
// The network is three dense layers on at most a few thousand rows, so the
// contractions are hand-tiled FP32 FFMA (64 x 64 output tiles, 4 x 4 per
// thread); at this size the tensor cores would not change the step time.
#include <cstdint>
#include "rqa_common.cuh"
#include <algorithm>
#include "rqa_learn_internal.h"

namespace rqa {

// ------------------------------------------------------------ SplitMix64
__device__ __forceinline__ uint64_t sm64_mix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
constexpr uint64_t SM64_GAMMA = 0x9E3779B97F4A7C15ull;
constexpr uint64_t SERIES_MULT = 0xD1B54A32D192ED03ull;

// ------------------------------------------------------------ sketch
// One CTA per series: 4096 random pairs, their distances sorted in shared
// memory (bitonic network on the bit patterns), 128 quantiles, their logs.
__global__ void __launch_bounds__(THREADS)
k_sketch(const float *__restrict__ y, const SeriesDev *series, int s_base, uint64_t seed,
         float *feats, float *centre, float *qdist)
{
    __shared__ uint32_t keys[SKETCH_PAIRS];
    __shared__ float fl[SKETCH_BINS];
    const int s = s_base + blockIdx.x;
    const SeriesDev sd = series[s];
    const float *ys = y + sd.off;
    const uint64_t ks = sm64_mix(seed ^ ((uint64_t)(s + 1) * SERIES_MULT));
    for (int p = threadIdx.x; p < SKETCH_PAIRS; p += THREADS) {
        const uint64_t a = sm64_mix(ks + (uint64_t)(2 * p + 1) * SM64_GAMMA);
        const uint64_t b = sm64_mix(ks + (uint64_t)(2 * p + 2) * SM64_GAMMA);
        const int i = (int)(a % (uint64_t)sd.ne);
        int j = (int)(b % (uint64_t)(sd.ne - 1));
        if (j >= i) ++j;
        float d = fabsf(ys[i] - ys[j]);
        for (int q = 1; q < sd.m; ++q)
            d = fmaxf(d, fabsf(ys[i + q * sd.tau] - ys[j + q * sd.tau]));
        keys[p] = __float_as_uint(d);
    }
    __syncthreads();
    // bitonic sort, ascending
    for (int size = 2; size <= SKETCH_PAIRS; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = threadIdx.x; t < SKETCH_PAIRS / 2; t += THREADS) {
                const int lo = 2 * t - (t & (stride - 1));
                const int hi = lo + stride;
                const bool up = (lo & size) == 0;
                const uint32_t x = keys[lo], z = keys[hi];
                if ((x > z) == up) {
                    keys[lo] = z;
                    keys[hi] = x;
                }
            }
            __syncthreads();
        }
    }
    const int t = threadIdx.x;
    if (t < SKETCH_BINS) {
        const float q = __uint_as_float(keys[32 * t + 16]);
        if (qdist) qdist[(int64_t)s * SKETCH_BINS + t] = q;
        fl[t] = logf(fmaxf(q, 1.17549435e-38f));  // ln(max(q, 2^-126))
    }
    __syncthreads();
    const float c = fl[SKETCH_BINS / 2];
    float *f = feats + (int64_t)s * FEATURES;
    if (t < SKETCH_BINS) f[t] = fl[t] - c;
    if (t == 0) {
        f[128] = log10f((float)sd.n);
        f[129] = (float)sd.m;
        f[130] = (float)sd.tau;
        if (centre) centre[s] = c;
    }
}

cudaError_t launch_sketch(const float *y, const SeriesDev *series, int s_base, int S,
                          uint64_t seed, float *feats, float *centre, float *qdist, cudaStream_t st)
{
    if (!y || !series || !feats || S < 1) return cudaErrorInvalidValue;
    k_sketch<<<S, THREADS, 0, st>>>(y, series, s_base, seed, feats, centre, qdist);
    return cudaGetLastError();
}

// ------------------------------------------------------------ GEMM
// C[M x N] = op(A) op(B) (+ bias[N]) (ReLU) (* [mask > 0]), row-major.
// op(A) is A [M x K] or, TA, A stored [K x M]; op(B) is B [K x N] or, TB,
// B stored [N x K].
constexpr int GT = 64, GK = 16;

template <bool TA, bool TB>
__global__ void __launch_bounds__(256)
k_gemm(const float *__restrict__ A, const float *__restrict__ B, float *__restrict__ C, int M,
       int N, int K, const float *__restrict__ bias, bool relu, const float *__restrict__ mask)
{
    __shared__ float As[GK][GT + 1];
    __shared__ float Bs[GK][GT + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int m0 = blockIdx.y * GT, n0 = blockIdx.x * GT;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += GK) {
        for (int e = threadIdx.x; e < GK * GT; e += 256) {
            const int kk = e / GT, mm = e % GT;
            const int gm = m0 + mm, gk = k0 + kk;
            float va = 0.f;
            if (gm < M && gk < K) va = TA ? A[(int64_t)gk * M + gm] : A[(int64_t)gm * K + gk];
            As[kk][mm] = va;
            const int gn = n0 + mm;
            float vb = 0.f;
            if (gn < N && gk < K) vb = TB ? B[(int64_t)gn * K + gk] : B[(int64_t)gk * N + gn];
            Bs[kk][mm] = vb;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) a[r] = As[kk][ty + 16 * r];
#pragma unroll
            for (int q = 0; q < 4; ++q) b[q] = Bs[kk][tx + 16 * q];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[r][q] = fmaf(a[r], b[q], acc[r][q]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int gm = m0 + ty + 16 * r;
        if (gm >= M) continue;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int gn = n0 + tx + 16 * q;
            if (gn >= N) continue;
            float v = acc[r][q];
            if (bias) v += bias[gn];
            if (relu) v = fmaxf(v, 0.f);
            if (mask && !(mask[(int64_t)gm * N + gn] > 0.f)) v = 0.f;
            C[(int64_t)gm * N + gn] = v;
        }
    }
}

static cudaError_t gemm(bool ta, bool tb, const float *A, const float *B, float *C, int M, int N,
                        int K, const float *bias, bool relu, const float *mask, cudaStream_t st)
{
    dim3 grid((N + GT - 1) / GT, (M + GT - 1) / GT);
    if (!ta && !tb) k_gemm<false, false><<<grid, 256, 0, st>>>(A, B, C, M, N, K, bias, relu, mask);
    else if (!ta && tb) k_gemm<false, true><<<grid, 256, 0, st>>>(A, B, C, M, N, K, bias, relu, mask);
    else if (ta && !tb) k_gemm<true, false><<<grid, 256, 0, st>>>(A, B, C, M, N, K, bias, relu, mask);
    else k_gemm<true, true><<<grid, 256, 0, st>>>(A, B, C, M, N, K, bias, relu, mask);
    return cudaGetLastError();
}

// Column sums of G [M x N] into out[N].
__global__ void k_colsum(const float *__restrict__ G, int M, int N, float *out)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float acc = 0.f;
    for (int m = 0; m < M; ++m) acc += G[(int64_t)m * N + n];
    out[n] = acc;
}

// Mean pinball loss of Y [B x 2K] against T [B x K] and its gradient.
__global__ void k_pinball(const float *__restrict__ Y, const float *__restrict__ T, int B, int K,
                          float tau_lo, float tau_hi, float *dY, float *loss)
{
    const int64_t n = (int64_t)B * 2 * K;
    const float inv = 1.f / (float)n;
    float part = 0.f;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = e / (2 * K);
        const int o = (int)(e % (2 * K));
        const float tau = (o & 1) ? tau_hi : tau_lo;
        const float r = T[b * K + (o >> 1)] - Y[e];
        part += (r >= 0.f) ? tau * r : (tau - 1.f) * r;
        dY[e] = ((r >= 0.f) ? -tau : 1.f - tau) * inv;
    }
    if (loss) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(FULL, part, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(loss, part * inv);
    }
}

__global__ void k_adam(float *p, const float *__restrict__ g, float *m, float *v, int64_t n,
                       float lr, float b1, float b2, float eps, float c1, float c2)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const float ge = g[e];
        const float me = b1 * m[e] + (1.f - b1) * ge;
        const float ve = b2 * v[e] + (1.f - b2) * ge * ge;
        m[e] = me;
        v[e] = ve;
        p[e] -= lr * (me / c1) / (sqrtf(ve / c2) + eps);
    }
}

// Parameter blocks inside the flat vector.
struct MlpView {
    const float *W1, *b1, *W2, *b2, *W3, *b3;
};
__host__ __device__ inline MlpView mlp_view(const float *p)
{
    MlpView v;
    v.W1 = p;
    v.b1 = v.W1 + HIDDEN * FEATURES;
    v.W2 = v.b1 + HIDDEN;
    v.b2 = v.W2 + HIDDEN * HIDDEN;
    v.W3 = v.b2 + HIDDEN;
    v.b3 = v.W3 + MLP_OUT * HIDDEN;
    return v;
}

cudaError_t mlp_forward(const float *params, const float *X, int B, float *Y, float *acts,
                        cudaStream_t st)
{
    const MlpView v = mlp_view(params);
    float *H1 = acts, *H2 = acts + (int64_t)B * HIDDEN;
    cudaError_t e;
    if ((e = gemm(false, true, X, v.W1, H1, B, HIDDEN, FEATURES, v.b1, true, nullptr, st))) return e;
    if ((e = gemm(false, true, H1, v.W2, H2, B, HIDDEN, HIDDEN, v.b2, true, nullptr, st))) return e;
    return gemm(false, true, H2, v.W3, Y, B, MLP_OUT, HIDDEN, v.b3, false, nullptr, st);
}

cudaError_t mlp_backward(const float *params, const float *X, const float *acts, const float *Y,
                         const float *T, int B, float tau_lo, float tau_hi, float *grads,
                         float *loss, float *scratch, cudaStream_t st)
{
    const MlpView v = mlp_view(params);
    const float *H1 = acts, *H2 = acts + (int64_t)B * HIDDEN;
    float *gW1 = grads, *gb1 = gW1 + HIDDEN * FEATURES, *gW2 = gb1 + HIDDEN,
          *gb2 = gW2 + HIDDEN * HIDDEN, *gW3 = gb2 + HIDDEN, *gb3 = gW3 + MLP_OUT * HIDDEN;
    float *dY = scratch, *dZ2 = dY + (int64_t)B * MLP_OUT, *dZ1 = dZ2 + (int64_t)B * HIDDEN;
    cudaError_t e;
    if (loss && (e = cudaMemsetAsync(loss, 0, sizeof(float), st))) return e;
    const int64_t n = (int64_t)B * MLP_OUT;
    k_pinball<<<(int)std::min<int64_t>((n + 255) / 256, 1024), 256, 0, st>>>(
        Y, T, B, MLP_OUT / 2, tau_lo, tau_hi, dY, loss);
    if ((e = cudaGetLastError())) return e;
    // layer 3
    if ((e = gemm(true, false, dY, H2, gW3, MLP_OUT, HIDDEN, B, nullptr, false, nullptr, st))) return e;
    k_colsum<<<1, 64, 0, st>>>(dY, B, MLP_OUT, gb3);
    if ((e = gemm(false, false, dY, v.W3, dZ2, B, HIDDEN, MLP_OUT, nullptr, false, H2, st))) return e;
    // layer 2
    if ((e = gemm(true, false, dZ2, H1, gW2, HIDDEN, HIDDEN, B, nullptr, false, nullptr, st))) return e;
    k_colsum<<<1, HIDDEN, 0, st>>>(dZ2, B, HIDDEN, gb2);
    if ((e = gemm(false, false, dZ2, v.W2, dZ1, B, HIDDEN, HIDDEN, nullptr, false, H1, st))) return e;
    // layer 1
    if ((e = gemm(true, false, dZ1, X, gW1, HIDDEN, FEATURES, B, nullptr, false, nullptr, st))) return e;
    k_colsum<<<1, HIDDEN, 0, st>>>(dZ1, B, HIDDEN, gb1);
    return cudaGetLastError();
}

cudaError_t adam_step(float *p, const float *g, float *m, float *v, int64_t n, int t, float lr,
                      float b1, float b2, float eps, cudaStream_t st)
{
    const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
    k_adam<<<(int)std::min<int64_t>((n + 255) / 256, 2048), 256, 0, st>>>(p, g, m, v, n, lr, b1, b2,
                                                                          eps, c1, c2);
    return cudaGetLastError();
}

// ------------------------------------------------------------ training data
// Labels of the network: T[s][k] = ln(max(eps[s][k], 2^-126)) - c[s], the
// thresholds in the centred log scale of the sketch features.
__global__ void k_log_labels(const float *__restrict__ eps, const float *__restrict__ centre, int S,
                             int K, float *__restrict__ T)
{
    const int64_t n = (int64_t)S * K;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x)
        T[e] = logf(fmaxf(eps[e], 0x1p-126f)) - centre[e / K];
}

cudaError_t launch_log_labels(const float *eps, const float *centre, int S, int K, float *T,
                              cudaStream_t st)
{
    const int64_t n = (int64_t)S * K;
    k_log_labels<<<(int)std::min<int64_t>((n + 255) / 256, 1024), 256, 0, st>>>(eps, centre, S, K, T);
    return cudaGetLastError();
}

// Validation of a bracket network over B rows: the summed pinball loss of the
// 2K outputs (lower ends at tau_lo, upper at tau_hi), the targets inside
// [lo - margin, hi + margin] and the summed width hi - lo + 2 margin.
__global__ void k_bracket_eval(const float *__restrict__ Y, const float *__restrict__ T, int B,
                               int K, float tau_lo, float tau_hi, float margin, double *loss_sum,
                               unsigned long long *inside, double *width_sum)
{
    double l = 0.0, w = 0.0;
    unsigned long long in = 0;
    const int64_t n = (int64_t)B * K;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = e / K;
        const int k = (int)(e % K);
        const float t = T[e];
        const float lo = Y[b * 2 * K + 2 * k], hi = Y[b * 2 * K + 2 * k + 1];
        const float rl = t - lo, rh = t - hi;
        l += (double)((rl >= 0.f) ? tau_lo * rl : (tau_lo - 1.f) * rl);
        l += (double)((rh >= 0.f) ? tau_hi * rh : (tau_hi - 1.f) * rh);
        in += (t >= lo - margin && t <= hi + margin) ? 1ull : 0ull;
        w += (double)((hi + margin) - (lo - margin));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        l += __shfl_xor_sync(FULL, l, o);
        w += __shfl_xor_sync(FULL, w, o);
        in += __shfl_xor_sync(FULL, in, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(loss_sum, l);
        atomicAdd(width_sum, w);
        atomicAdd(inside, in);
    }
}

cudaError_t launch_bracket_eval(const float *Y, const float *T, int B, int K, float tau_lo,
                                float tau_hi, float margin, double *loss_sum,
                                unsigned long long *inside, double *width_sum, cudaStream_t st)
{
    cudaError_t e;
    if ((e = cudaMemsetAsync(loss_sum, 0, sizeof(double), st))) return e;
    if ((e = cudaMemsetAsync(width_sum, 0, sizeof(double), st))) return e;
    if ((e = cudaMemsetAsync(inside, 0, sizeof(unsigned long long), st))) return e;
    const int64_t n = (int64_t)B * K;
    k_bracket_eval<<<(int)std::min<int64_t>((n + 255) / 256, 512), 256, 0, st>>>(
        Y, T, B, K, tau_lo, tau_hi, margin, loss_sum, inside, width_sum);
    return cudaGetLastError();
}

// dst row r = src row idx[r], rows of `width` floats (a minibatch gather).
__global__ void k_gather_rows(const float *__restrict__ src, const int64_t *__restrict__ idx, int n,
                              int width, float *__restrict__ dst)
{
    const int64_t total = (int64_t)n * width;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / width;
        dst[e] = src[idx[r] * width + (e - r * width)];
    }
}

cudaError_t launch_gather_rows(const float *src, const int64_t *idx, int n, int width, float *dst,
                               cudaStream_t st)
{
    const int64_t total = (int64_t)n * width;
    k_gather_rows<<<(int)std::min<int64_t>((total + 255) / 256, 2048), 256, 0, st>>>(src, idx, n, width, dst);
    return cudaGetLastError();
}

// ------------------------------------------------------------ bracket
// Coarse buckets to split in the first counting round.  Per target the
// interval runs from the bucket of exp(c + lo - margin) to that of
// exp(c + hi + margin).  If all of them fit in NSUB_MAX buckets, every bucket
// from the lowest to the highest end is split (and up to two below); else the
// buckets nearest each target's middle bucket first, then the narrowest gaps
// between split buckets.  Keys between the first and the last split bucket
// are counted either way (unsplit buckets at coarse resolution).
__global__ void k_bracket(const float *__restrict__ Yb, const float *__restrict__ centre,
                          float margin, int K, const uint8_t *__restrict__ dom, int8_t *tab_sub,
                          int32_t *n_sub, uint32_t *range)
{
    __shared__ uint16_t lo_b[KMAX], hi_b[KMAX], mid_b[KMAX];
    __shared__ int8_t tb[NCOARSE];
    const int s = blockIdx.x;
    if (!dom[s]) {  // outside the network's domain: the full selection takes it
        int8_t *tab = tab_sub + (int64_t)s * NCOARSE;
        for (int x = threadIdx.x; x < NCOARSE; x += blockDim.x) tab[x] = -1;
        if (threadIdx.x == 0) {
            n_sub[s] = 0;
            range[2 * s] = 0xffffffffu;
            range[2 * s + 1] = 0u;
        }
        return;
    }
    for (int x = threadIdx.x; x < NCOARSE; x += blockDim.x) tb[x] = -1;
    if (threadIdx.x < K) {
        const float c = centre[s];
        float lo = Yb[(int64_t)s * MLP_OUT + 2 * threadIdx.x] - margin;
        float hi = Yb[(int64_t)s * MLP_OUT + 2 * threadIdx.x + 1] + margin;
        if (!(lo <= hi)) {  // crossed or NaN ends: a narrow interval around their mean
            float mm = 0.5f * (lo + hi);
            if (!(mm == mm)) mm = 0.f;
            lo = mm - margin;
            hi = mm + margin;
        }
        auto bucket = [](float ln_v) {
            const float v = expf(fminf(fmaxf(ln_v, -87.f), 88.f));
            return (uint16_t)(__float_as_uint(v) >> COARSE_SHIFT);
        };
        lo_b[threadIdx.x] = bucket(c + lo);
        hi_b[threadIdx.x] = bucket(c + hi);
        mid_b[threadIdx.x] = bucket(c + 0.5f * (lo + hi));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int lo_all = NCOARSE, hi_all = -1;
        for (int k = 0; k < K; ++k) {
            lo_all = min(lo_all, (int)lo_b[k]);
            hi_all = max(hi_all, (int)hi_b[k]);
        }
        const int span = hi_all - lo_all + 1;
        if (span <= NSUB_MAX) {
            // every bucket from the lowest to the highest interval end: a
            // threshold between two targets' intervals is found too; up to
            // two more buckets below (they hold few keys)
            const int a = max(0, lo_all - min(2, NSUB_MAX - span));
            for (int b = a; b <= hi_all; ++b) tb[b] = 0;
        } else {
            // rings around each target's most likely bucket, inside its
            // interval, all targets alike, until the split budget is spent
            int used = 0;
            for (int r = 0; used < NSUB_MAX; ++r) {
                bool any = false;
                for (int k = 0; k < K; ++k) {
                    for (int side = -1; side <= 1; side += 2) {
                        if (r == 0 && side > 0) continue;
                        const int b = (int)mid_b[k] + side * r;
                        if (b < (int)lo_b[k] || b > (int)hi_b[k]) continue;
                        any = true;
                        if (tb[b] != 0 && used < NSUB_MAX) {
                            tb[b] = 0;
                            ++used;
                        }
                    }
                }
                if (!any) break;
            }
            // the rest of the budget closes the narrowest gaps between them
            int first = 0, last = NCOARSE - 1;
            while (first < NCOARSE && tb[first] != 0) ++first;
            while (last > first && tb[last] != 0) --last;
            for (;;) {
                int best_a = -1, best_n = NCOARSE;
                for (int b = first; b <= last; ++b) {
                    if (tb[b] == 0) continue;
                    int e = b;
                    while (tb[e] != 0) ++e;  // tb[last] is marked: ends inside
                    if (e - b < best_n) {
                        best_n = e - b;
                        best_a = b;
                    }
                    b = e;
                }
                if (best_a < 0 || used + best_n > NSUB_MAX) break;
                for (int b = best_a; b < best_a + best_n; ++b) tb[b] = 0;
                used += best_n;
            }
        }
        int g = 0;  // marked buckets numbered in ascending order
        int first = -1, last = -1;
        for (int b = 0; b < NCOARSE; ++b) {
            if (tb[b] != 0) continue;
            if (g < NSUB_MAX) {
                tb[b] = (int8_t)(g++);
                if (first < 0) first = b;
                last = b;
            } else {
                tb[b] = -1;
            }
        }
        n_sub[s] = g;
        // keys the bracket round counts: from its first to its last split bucket
        range[2 * s] = first < 0 ? 0xffffffffu : (uint32_t)first << COARSE_SHIFT;
        range[2 * s + 1] = first < 0 ? 0u : (((uint32_t)last + 1u) << COARSE_SHIFT) - 1u;
    }
    __syncthreads();
    int8_t *tab = tab_sub + (int64_t)s * NCOARSE;
    for (int x = threadIdx.x; x < NCOARSE; x += blockDim.x) tab[x] = tb[x];
}

cudaError_t launch_bracket(const float *Y, const float *centre, float margin, int S, int K,
                           const uint8_t *dom, int8_t *tab_sub, int32_t *n_sub, uint32_t *range,
                           cudaStream_t st)
{
    if (!dom) return cudaErrorInvalidValue;
    k_bracket<<<S, 256, 0, st>>>(Y, centre, margin, K, dom, tab_sub, n_sub, range);
    return cudaGetLastError();
}

// Hits and misses of a bracketed selection: a target hit when its key
// prefix was fixed by the split round (level 2 right after it); series
// outside the network's domain (dom[s] == 0) are not counted.
__global__ void k_bracket_stats(const uint8_t *level, const uint8_t *dom, int S, int K,
                                unsigned long long *hm)
{
    unsigned long long h = 0, m = 0;
    const int64_t n = (int64_t)S * K;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        if (!dom[e / K]) continue;
        if (level[e] == 2) ++h;
        else ++m;
    }
    atomicAdd(hm, h);
    atomicAdd(hm + 1, m);
}

cudaError_t launch_bracket_stats(const uint8_t *level, const uint8_t *dom, int S, int K,
                                 unsigned long long *hm, cudaStream_t st)
{
    if (!dom || S < 1 || K < 1) return cudaErrorInvalidValue;
    const int64_t n = (int64_t)S * K;
    k_bracket_stats<<<(int)std::min<int64_t>((n + 255) / 256, 256), 256, 0, st>>>(level, dom, S, K, hm);
    return cudaGetLastError();
}

}  // namespace rqa
