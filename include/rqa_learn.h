/*
 * rqa_learn.h -- the learned threshold bracket of librqa.
 *
 * The paper selects thresholds by their recurrence rate (Sect. 2) but says
 * nothing about how to find them fast; it has no learned component.  This
 * part of the library predicts, per series, an interval [lo_k, hi_k] that
 * probably holds eps_k, so the exact selection (rqa.h) can count the keys of
 * those intervals at a finer resolution in its first pass and skip its middle
 * pass.  The prediction never changes a result: a threshold outside its
 * interval is found by the full selection instead (see rqa_bracket_stats).
 *
 * Model: a sketch of each series (4096 random pairs of embedded vectors,
 * their maximum-norm distances sorted, 128 quantiles sorted[32b+16], natural
 * logarithms centred on the median quantile c) plus log10 N, m and tau gives
 * RQA_FEATURES = 131 inputs; three FP32 linear layers 131 -> 256 -> 256 -> 40
 * with ReLU between them give, for the K = 20 targets RR = 1..20 %, the lower
 * (output 2k) and upper (output 2k+1) ends of ln(eps_k) - c.  The pairs come
 * from SplitMix64 used as a counter-based generator:
 *   key_s = mix(seed ^ ((s + 1) * 0xD1B54A32D192ED03)),
 *   u_t   = mix(key_s + (t + 1) * 0x9E3779B97F4A7C15),
 *   pair p: i = u_{2p} mod Ne, j' = u_{2p+1} mod (Ne - 1), j = j' + [j' >= i],
 * with mix() the SplitMix64 output function (Steele, Lea & Flood 2014).
 *
 * Parameters are one FP32 vector: W1 [256][131], b1 [256], W2 [256][256],
 * b2 [256], W3 [40][256], b3 [40] (RQA_MLP_PARAMS values).  All pointers are
 * device memory of the context's device unless stated; calls are
 * asynchronous on the context's stream like those of rqa.h.
 */
#ifndef RQA_LEARN_H
#define RQA_LEARN_H

#include "rqa.h"

#ifdef __cplusplus
extern "C" {
#endif

#define RQA_MLP_HIDDEN 256
#define RQA_MLP_OUT 40
#define RQA_MLP_PARAMS (256 * 131 + 256 + 256 * 256 + 256 + 40 * 256 + 40)
#define RQA_MLP_ACTS 512 /* per-row activations kept for the backward pass */

/* Sketch features of every series of the batch.
 *   feats   S x RQA_FEATURES FP32 (row s: 128 centred log quantiles, log10 N, m, tau)
 *   centre  S FP32, the centre c (may be NULL)
 *   qdist   S x RQA_SKETCH_BINS FP32 quantile distances (may be NULL) */
int rqa_sketch(rqa_ctx *ctx, const rqa_batch *batch, uint64_t seed, float *feats,
               float *centre, float *qdist);

/* Network forward pass for B rows.  X: B x 131, Y: B x 40.  acts: 512 B
 * floats receiving the hidden activations for rqa_mlp_backward: layer 1
 * (B x 256, row-major) followed by layer 2 (B x 256); may be NULL. */
int rqa_mlp_forward(rqa_ctx *ctx, const float *params, const float *X, int32_t B, float *Y,
                    float *acts);

/* Gradient of the mean pinball loss over the B x 40 outputs: output 2k is
 * scored at quantile tau_lo against T[b][k], output 2k+1 at tau_hi.
 *   X, acts, Y  from rqa_mlp_forward;  T: B x 20 targets
 *   grads       RQA_MLP_PARAMS FP32, overwritten
 *   loss        one FP32, overwritten with the mean loss (may be NULL) */
int rqa_mlp_backward(rqa_ctx *ctx, const float *params, const float *X, const float *acts,
                     const float *Y, const float *T, int32_t B, float tau_lo, float tau_hi,
                     float *grads, float *loss);

/* One Adam step (Kingma & Ba 2015) over n parameters; t counts from 1. */
int rqa_adam_step(rqa_ctx *ctx, float *params, const float *grads, float *m, float *v,
                  int64_t n, int32_t t, float lr, float beta1, float beta2, float eps);

/* Training data and validation of the network, on the device:
 *   rqa_log_labels    T[s][k] = ln(max(eps[s][k], 2^-126)) - centre[s]
 *                     (eps, T: S x K; centre: S), the targets of the network
 *                     in the centred log scale of rqa_sketch's features.
 *   rqa_bracket_eval  over B rows of outputs Y (B x 2K, the ends lo_k, hi_k)
 *                     and targets T (B x K): loss_sum = summed pinball loss of
 *                     the 2BK outputs (lower ends at tau_lo, upper at tau_hi;
 *                     divide by 2BK for the mean of rqa_mlp_backward),
 *                     inside = targets with lo - margin <= T <= hi + margin,
 *                     width_sum = summed (hi + margin) - (lo - margin); the
 *                     three outputs are device scalars (double, uint64, double).
 *   rqa_gather_rows   dst row r = src row idx[r] (rows of `width` floats, idx
 *                     device int64, n rows): a minibatch gather. */
int rqa_log_labels(rqa_ctx *ctx, const float *eps, const float *centre, int32_t S, int32_t K,
                   float *T);
int rqa_bracket_eval(rqa_ctx *ctx, const float *Y, const float *T, int32_t B, int32_t K,
                     float tau_lo, float tau_hi, float margin, double *loss_sum,
                     uint64_t *inside, double *width_sum);
int rqa_gather_rows(rqa_ctx *ctx, const float *src, const int64_t *idx, int32_t n, int32_t width,
                    float *dst);

/* Install a trained network in the context (params copied, device pointer)
 * and the widening margin added to both ends of every interval (in ln units).
 * params == NULL removes the model.  With a model, RQA_SELECT_AUTO uses the
 * bracket when a call asks for RR = 1..20 % (rr_num 1..20, rr_den 100), for
 * the series whose embedding lies in the model's domain (below). */
int rqa_set_bracket_model(rqa_ctx *ctx, const float *params, float margin);

/* The embeddings (m[i], tau[i]), i < n, the installed network was trained on
 * (host arrays, copied).  With RQA_SELECT_AUTO only series with one of these
 * embeddings are bracketed; the others take the full selection, and a call
 * none of whose series qualifies runs no sketch or network at all.  n = 0
 * (the default) puts no restriction; RQA_SELECT_BRACKET ignores the domain.
 * At most 64 pairs; RQA_ERR_INVALID_ARG for m or tau < 1. */
int rqa_set_bracket_domain(rqa_ctx *ctx, const int32_t *m, const int32_t *tau, int32_t n);

/* Targets of the context's last bracketed selection whose interval held the
 * threshold (hits) and those that needed the full selection (misses), over
 * the series that were bracketed; host pointers, synchronises the stream. */
int rqa_bracket_stats(rqa_ctx *ctx, uint64_t *hits, uint64_t *misses);

#ifdef __cplusplus
}
#endif
#endif /* RQA_LEARN_H */
