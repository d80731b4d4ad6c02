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

// Row vector x_i = (y[i], y[i+tau], ..., y[i+(m-1)tau]) held in registers for
// a compile-time embedding dimension M (M == 0: generic, re-read per cell).
template <int M>
struct RowVec {
    float a[M];
    __device__ __forceinline__ void load(const float *__restrict__ ys, int i, int tau, int)
    {
#pragma unroll
        for (int q = 0; q < M; ++q) a[q] = __ldg(ys + i + q * tau);
    }
    // Maximum-norm distance to x_j (Sect. 2): FP32 subtract, abs and max only,
    // so the result is exact and identical to a CPU evaluation.
    __device__ __forceinline__ float dist(const float *__restrict__ ys, int i, int j, int tau,
                                          int) const
    {
        float d = fabsf(a[0] - __ldg(ys + j));
#pragma unroll
        for (int q = 1; q < M; ++q) d = fmaxf(d, fabsf(a[q] - __ldg(ys + j + q * tau)));
        return d;
    }
};

template <>
struct RowVec<0> {
    __device__ __forceinline__ void load(const float *, int, int, int) {}
    __device__ __forceinline__ float dist(const float *__restrict__ ys, int i, int j, int tau,
                                          int m) const
    {
        float d = fabsf(__ldg(ys + i) - __ldg(ys + j));
        for (int q = 1; q < m; ++q)
            d = fmaxf(d, fabsf(__ldg(ys + i + q * tau) - __ldg(ys + j + q * tau)));
        return d;
    }
};

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
