// Internal declarations of the learned bracket (learn.cu).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include "rqa_internal.h"

namespace rqa {

constexpr int SKETCH_PAIRS = 4096;
constexpr int SKETCH_BINS = 128;
constexpr int FEATURES = 131;
constexpr int HIDDEN = 256;
constexpr int MLP_OUT = 40;   // 2 x 20 interval ends
constexpr int MLP_K = 20;     // targets RR = 1..20 % the network predicts
constexpr int64_t MLP_PARAMS = (int64_t)HIDDEN * FEATURES + HIDDEN + (int64_t)HIDDEN * HIDDEN +
                               HIDDEN + (int64_t)MLP_OUT * HIDDEN + MLP_OUT;

// series s_base .. s_base+S-1 of the batch (their rows of feats/centre/qdist)
cudaError_t launch_sketch(const float *y, const SeriesDev *series, int s_base, int S,
                          uint64_t seed, float *feats, float *centre, float *qdist, cudaStream_t st);
// acts: B x 2*HIDDEN (H1 then H2 blocks)
cudaError_t mlp_forward(const float *params, const float *X, int B, float *Y, float *acts,
                        cudaStream_t st);
// scratch: B x (MLP_OUT + 2*HIDDEN) floats
cudaError_t mlp_backward(const float *params, const float *X, const float *acts, const float *Y,
                         const float *T, int B, float tau_lo, float tau_hi, float *grads,
                         float *loss, float *scratch, cudaStream_t st);
cudaError_t adam_step(float *p, const float *g, float *m, float *v, int64_t n, int t, float lr,
                      float b1, float b2, float eps, cudaStream_t st);
cudaError_t launch_log_labels(const float *eps, const float *centre, int S, int K, float *T,
                              cudaStream_t st);
cudaError_t launch_bracket_eval(const float *Y, const float *T, int B, int K, float tau_lo,
                                float tau_hi, float margin, double *loss_sum,
                                unsigned long long *inside, double *width_sum, cudaStream_t st);
cudaError_t launch_gather_rows(const float *src, const int64_t *idx, int n, int width, float *dst,
                               cudaStream_t st);
// also writes range[2s], range[2s+1]: the keys of the split buckets' span.
// dom[s] == 0: series s is not bracketed (no split bucket, empty range).
cudaError_t launch_bracket(const float *Y, const float *centre, float margin, int S, int K,
                           const uint8_t *dom, int8_t *tab_sub, int32_t *n_sub, uint32_t *range,
                           cudaStream_t st);
// hits / misses over the S x K levels of the series with dom[s] != 0
cudaError_t launch_bracket_stats(const uint8_t *level, const uint8_t *dom, int S, int K,
                                 unsigned long long *hm, cudaStream_t st);

}  // namespace rqa
