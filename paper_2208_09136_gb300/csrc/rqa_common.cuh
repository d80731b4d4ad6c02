// Device helpers shared by the cell kernels: distances on the fly and the
// persistent work loop.
#pragma once
#include <cstdint>
#include "rqa_internal.h"

namespace rqa {

constexpr unsigned FULL = 0xffffffffu;

// Record the first device-side error; later ones are dropped.
__device__ __forceinline__ void set_status(int *status, int code)
{
    atomicCAS(status, 0, code);
}

// Add 1 to the shared word at shared-space address a when x <= y
// (unsigned), as one compare and one predicated reduction: no branch, so a
// warp whose lanes disagree does not split, and no predicate turned into an
// integer and back.  a is not touched when x > y; a caller folds a further
// condition into x (x = ~0u when it fails, with y < ~0u).
__device__ __forceinline__ void red_shared_if_le(uint32_t a, uint32_t x, uint32_t y)
{
    asm volatile("{\n\t.reg .pred q;\n\tsetp.le.u32 q, %1, %2;\n\t@q red.shared.add.u32 [%0], 1;\n\t}"
                 :: "r"(a), "r"(x), "r"(y) : "memory");
}

// Add 1 to the shared word at shared-space address a: one reduction, no
// predicate.  A cell that counts nowhere adds to a per-lane scratch word
// instead, so no branch region is needed around the reduction.
__device__ __forceinline__ void red_shared(uint32_t a)
{
    asm volatile("red.shared.add.u32 [%0], 1;" :: "r"(a) : "memory");
}

// max(a, b, c) in one instruction (three-input FP32 max of sm_100 and later);
// exact, like two two-input maxima.
__device__ __forceinline__ float fmax3(float a, float b, float c)
{
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// Maximum norm of the M per-coordinate differences a[q] - b[q] (Sect. 2):
// absolute values folded into the maxima, three at a time.
template <int M>
__device__ __forceinline__ float maxnorm(const float (&diff)[M])
{
    float d = fabsf(diff[0]);
    int q = 1;
#pragma unroll
    for (; q + 1 < M; q += 2) d = fmax3(d, fabsf(diff[q]), fabsf(diff[q + 1]));
#pragma unroll
    for (; q < M; ++q) d = fmaxf(d, fabsf(diff[q]));
    return d;
}

// Distances of one lane's cells in a band: row i (lane), diagonals
// d_lo .. d_lo+D-1.  Maximum-norm distance (Sect. 2) with FP32 subtract, abs
// and max only, so every value is exact and equal to a CPU evaluation.
//
// Compile-time embedding (M >= 1, TAU >= 1): the row vector
// x_i = (y[i], y[i+TAU], ...) and the column window y[i+d_lo .. i+d_lo+D-1+
// (M-1)TAU] are loaded into registers once per 32-row block, so the D cells of
// the lane need no further memory traffic.
template <int M, int TAU, int D>
struct BandTile {
    float a[M];
    float w[D + (M - 1) * TAU];
    __device__ __forceinline__ void load(const float *__restrict__ ys, int n, int i, int d_lo,
                                         int rows, int, int)
    {
        if (i < rows) {
#pragma unroll
            for (int q = 0; q < M; ++q) a[q] = __ldg(ys + i + q * TAU);
        }
#pragma unroll
        for (int x = 0; x < D + (M - 1) * TAU; ++x) {
            const int idx = i + d_lo + x;
            w[x] = (i < rows && idx < n) ? __ldg(ys + idx) : 0.f;
        }
    }
    // every lane's row and window inside the series (an interior row block)
    __device__ __forceinline__ void load_fast(const float *__restrict__ ys, int i, int d_lo, int)
    {
#pragma unroll
        for (int q = 0; q < M; ++q) a[q] = __ldg(ys + i + q * TAU);
#pragma unroll
        for (int x = 0; x < D + (M - 1) * TAU; ++x) w[x] = __ldg(ys + i + d_lo + x);
    }
    // the same window from shared memory: rb holds y[i0..], cb y[i0 + d_lo + jc..]
    // (row i = i0 + lane)
    __device__ __forceinline__ void load_smem(const float *rb, const float *cb, int lane)
    {
#pragma unroll
        for (int q = 0; q < M; ++q) a[q] = rb[lane + q * TAU];
#pragma unroll
        for (int x = 0; x < D + (M - 1) * TAU; ++x) w[x] = cb[lane + x];
    }
    // vertical pass: row i, columns c_lo .. c_lo+D-1 (the same window for
    // every lane); zeros outside the series
    __device__ __forceinline__ void load_vert(const float *__restrict__ ys, int n, int ne, int i,
                                              int c_lo, int)
    {
#pragma unroll
        for (int q = 0; q < M; ++q) a[q] = i < ne ? __ldg(ys + i + q * TAU) : 0.f;
#pragma unroll
        for (int x = 0; x < D + (M - 1) * TAU; ++x)
            w[x] = c_lo + x < n ? __ldg(ys + c_lo + x) : 0.f;
    }
    __device__ __forceinline__ void load_vert_fast(const float *__restrict__ ys, int i, int c_lo, int)
    {
#pragma unroll
        for (int q = 0; q < M; ++q) a[q] = __ldg(ys + i + q * TAU);
#pragma unroll
        for (int x = 0; x < D + (M - 1) * TAU; ++x) w[x] = __ldg(ys + c_lo + x);
    }
    // cell (i, i + d_lo + j), or (i, c_lo + j) after load_vert; only called
    // for cells inside the matrix
    __device__ __forceinline__ float dist(const float *__restrict__, int j, int, int, int,
                                          int) const
    {
        float diff[M];
#pragma unroll
        for (int q = 0; q < M; ++q) diff[q] = a[q] - w[j + q * TAU];
        return maxnorm<M>(diff);
    }
};

// Compile-time M, run-time tau: the row vector in registers, columns read per cell.
template <int M, int D>
struct BandTile<M, 0, D> {
    float a[M];
    __device__ __forceinline__ void load(const float *__restrict__ ys, int, int i, int,
                                         int rows, int tau, int)
    {
        if (i < rows) {
#pragma unroll
            for (int q = 0; q < M; ++q) a[q] = __ldg(ys + i + q * tau);
        }
    }
    __device__ __forceinline__ void load_fast(const float *__restrict__ ys, int i, int, int tau)
    {
#pragma unroll
        for (int q = 0; q < M; ++q) a[q] = __ldg(ys + i + q * tau);
    }
    __device__ __forceinline__ void load_vert(const float *__restrict__ ys, int, int ne, int i, int,
                                              int tau)
    {
        if (i < ne) {
#pragma unroll
            for (int q = 0; q < M; ++q) a[q] = __ldg(ys + i + q * tau);
        }
    }
    __device__ __forceinline__ void load_vert_fast(const float *__restrict__ ys, int i, int, int tau)
    {
        load_fast(ys, i, 0, tau);
    }
    __device__ __forceinline__ float dist(const float *__restrict__ ys, int, int i, int dl,
                                          int tau, int) const
    {
        const int j = i + dl;
        float diff[M];
#pragma unroll
        for (int q = 0; q < M; ++q) diff[q] = a[q] - __ldg(ys + j + q * tau);
        return maxnorm<M>(diff);
    }
};

// Generic embedding: everything read per cell.
template <int D>
struct BandTile<0, 0, D> {
    __device__ __forceinline__ void load(const float *, int, int, int, int, int, int) {}
    __device__ __forceinline__ void load_fast(const float *, int, int, int) {}
    __device__ __forceinline__ void load_vert(const float *, int, int, int, int, int) {}
    __device__ __forceinline__ void load_vert_fast(const float *, int, int, int) {}
    __device__ __forceinline__ float dist(const float *__restrict__ ys, int, int i, int dl,
                                          int tau, int m) const
    {
        const int j = i + dl;
        float d = fabsf(__ldg(ys + i) - __ldg(ys + j));
        for (int q = 1; q < m; ++q)
            d = fmaxf(d, fabsf(__ldg(ys + i + q * tau) - __ldg(ys + j + q * tau)));
        return d;
    }
};

// Embedding variants with their own kernel instantiation.
enum Embed : int { E_GENERIC = 0, E_M1 = 1, E_M2 = 2, E_M3 = 3, E_M4 = 4,
                   E_M1T1 = 11, E_M3T1 = 31, E_M3T3 = 33 };

// Host: CTAs of `kern` (THREADS threads, `smem` dynamic bytes) resident per
// SM, and the SM count of the current device; both cached per host thread.
inline int resident_per_sm(const void *kern, int smem, int threads = THREADS)
{
    struct Entry { const void *k; int s, v; };
    static thread_local Entry cache[64];
    static thread_local int n = 0;
    for (int i = 0; i < n; ++i)
        if (cache[i].k == kern && cache[i].s == smem) return cache[i].v;
    int v = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kern, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        v = 1;
    }
    v = v < 1 ? 1 : v;
    if (n < 64) cache[n++] = Entry{kern, smem, v};
    return v;
}

inline int sm_count_current()
{
    static thread_local int cache[64] = {};
    int d = 0;
    cudaGetDevice(&d);
    if (d >= 0 && d < 64 && cache[d]) return cache[d];
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, d);
    if (d >= 0 && d < 64) cache[d] = v;
    return v;
}

// A persistent grid: at most the CTAs that can be resident at once.
inline int persistent_cap(const void *kern, int smem, int grid, int threads = THREADS)
{
    const int cap = sm_count_current() * resident_per_sm(kern, smem, threads);
    return grid < cap ? grid : (cap > 0 ? cap : 1);
}

// Threads per CTA of a counting round: rounds whose shared histogram allows
// only two CTAs per SM run twice as many warps per CTA.
__host__ __device__ constexpr int count_threads(int round) { return (round == 1 || round == 2) ? 512 : THREADS; }

// Fetch the next work item for this CTA (one atomic per CTA), -1 when done.
__device__ __forceinline__ int next_item(unsigned int *queue, int n_items, int *sh_slot)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned t = atomicAdd(queue, 1u);
        *sh_slot = (t < (unsigned)n_items) ? (int)t : -1;
    }
    __syncthreads();
    return *sh_slot;
}

// Diagonals of band b: [d_lo, d_hi), d_hi <= Ne.
__device__ __forceinline__ void band_range(int b, int band, int ne, int &d_lo, int &d_hi)
{
    d_lo = 1 + b * band;
    d_hi = min(d_lo + band, ne);
}

}  // namespace rqa
