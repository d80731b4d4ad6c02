/*
 * rqa.h -- C ABI of the GB300 (sm_103a) library for averaged recurrence
 * quantification analysis: exact recurrence-rate-preselected thresholds and
 * determinism, computed over never-materialised recurrence matrices.
 *
 * Definitions (Pánis, Adámek & Marwan, "Averaged recurrence quantification
 * analysis"):
 *   series       y[0..N-1], FP32, delay embedded with dimension m and delay
 *                tau (Sect. 3.3): x_i = (y[i], y[i+tau], ..., y[i+(m-1)tau]),
 *                i < Ne = N - (m-1) tau.
 *   distance     d_ij = max_q |y[i+q tau] - y[j+q tau]|, maximum norm (Sect. 2).
 *   recurrence   R_ij = [d_ij <= eps] (Eq. 1-2; see below for the boundary).
 *   upper        only pairs i < j are used (Sect. 4); P = Ne(Ne-1)/2 pairs.
 *   RR target    rr_num/rr_den of the P pairs (Eq. 3; Sect. 2 fixes RR first).
 *   eps_k        the T_k-th smallest distance, T_k = ceil(rr_num_k * P / rr_den).
 *                Cells with d <= eps_k are recurrent, so #{d < eps_k} < T_k
 *                <= #{d <= eps_k}.  (Eq. 2 has H(0) = 0; the inclusive test is
 *                Eq. 1 taken at the next float above eps_k.)
 *   lines        maximal runs of recurrent cells along a diagonal j - i = const;
 *                P_k(l) = number of such runs of length l (Eq. 4).
 *   DET_k(lmin)  sum_{l >= lmin} l P_k(l) / #{d <= eps_k}   (Eq. 4), FP64 ratio
 *                of exact integer counts.
 *   DET average  (1/K) sum_k DET_k, summed in k order   (Eq. avgDET, Sect. 2).
 *
 * Conventions for every entry point:
 *   - Pointers documented "device" must be device memory of cfg.device;
 *     "host" pointers are read before the call returns.  The caller owns every
 *     input and output buffer; the context owns its scratch memory.
 *   - Work is enqueued on the context's stream (cfg.stream) and is
 *     asynchronous: outputs are valid after the stream is synchronised.
 *     Errors found on the host return at once; errors found by the kernels
 *     (non-finite input, unsorted thresholds, capacity, time-outs) are
 *     reported by rqa_status().
 *   - A context is not thread safe; use one per host thread.
 *   - K (number of thresholds per series) is 1 .. RQA_K_MAX, so a call can
 *     average over RR = 1..99 % (Sect. 2 considers RR* up to 99).  The line
 *     pass handles up to 20 thresholds per sweep over the cells; a call with
 *     larger K makes ceil(K / 20) sweeps (same results, proportionally
 *     slower line pass).
 *   - The line pass (rqa_det_avg, rqa_line_hist, rqa_vline_hist) counts
 *     series with Ne < 2^26 (6.7e7 vectors, 2.2e15 cells); longer ones are
 *     RQA_ERR_CAPACITY.  Every call takes series with Ne <= 3 * 2^30 / 32
 *     (1.0e8 vectors, 5e15 cells), else RQA_ERR_CAPACITY.
 *   - A series must have Ne >= 2 (P >= 1), otherwise RQA_ERR_TOO_SHORT.
 */
#ifndef RQA_H
#define RQA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RQA_ABI_VERSION 3
#define RQA_K_MAX 127         /* thresholds per series and call */
#define RQA_M_MAX 16          /* embedding dimension */
#define RQA_LMIN_MAX 8        /* entries of the lmin list of rqa_det_avg */
#define RQA_SKETCH_PAIRS 4096 /* random pairs of the distance sketch */
#define RQA_SKETCH_BINS 128   /* quantiles kept from the sketch */
#define RQA_FEATURES 131      /* sketch bins + log10 N, m, tau */

/* Return codes. */
enum {
    RQA_OK = 0,
    RQA_ERR_INVALID_ARG = 1, /* NULL pointer, K or m or tau out of range, bad rr */
    RQA_ERR_TOO_SHORT = 2,   /* a series has fewer than two embedded vectors */
    RQA_ERR_NONFINITE = 3,   /* device: a series holds NaN or +-Inf */
    RQA_ERR_CUDA = 4,        /* a CUDA runtime call failed (no device, launch) */
    RQA_ERR_OOM = 5,         /* scratch allocation failed */
    RQA_ERR_TIMEOUT = 6,     /* device: a bounded wait gave up */
    RQA_ERR_CAPACITY = 7,    /* output buffer too small / size limit exceeded */
    RQA_ERR_UNSORTED = 8,    /* device: thresholds of a series not ascending */
    RQA_ERR_NO_MODEL = 9,    /* bracket selection requested without a model */
    RQA_ERR_INTERNAL = 10    /* device: inconsistent counts (a library bug) */
};

/* Work schedule: one persistent launch per phase over the whole batch, or one
 * launch sequence per series (the plain per-series form). */
enum { RQA_SCHED_BATCHED = 0, RQA_SCHED_PER_SERIES = 1 };

/* Threshold selection: full radix select over FP32 bit patterns (3 counting
 * passes), or the learned bracket (2 passes when the bracket holds, radix
 * fallback per threshold when it misses).  AUTO = bracket if a model is set. */
enum { RQA_SELECT_AUTO = 0, RQA_SELECT_RADIX = 1, RQA_SELECT_BRACKET = 2 };

typedef struct rqa_ctx rqa_ctx;

typedef struct {
    int device;        /* CUDA device ordinal */
    void *stream;      /* cudaStream_t owned by the caller; NULL = default stream */
    int schedule;      /* RQA_SCHED_* */
    int select;        /* RQA_SELECT_* */
    int tile;          /* line pass: diagonals whose cells a lane computes from
                          one register window of the series: 0 = default (16,
                          or the rqa_autotune choice), else 8, 16 or 32 (8 and
                          32 only for (m, tau) = (1, any), (3, 1), (3, 3);
                          otherwise 16 is used) */
    int blocks_per_sm; /* persistent CTAs per SM: 0 = as many as each kernel
                          can keep resident, else at most this many */
    int flags;         /* RQA_FLAG_* */
    int reserved[3];   /* must be zero */
} rqa_config;

/* rqa_det_avg records its launch sequence in a CUDA graph and replays it when
 * the next call has the same arguments (batch layout and contents pointers,
 * targets, outputs) -- only on a caller-owned stream, not on the legacy
 * default stream.  This flag turns that off. */
#define RQA_FLAG_NO_GRAPHS 1

/* Count the line of identity, as Eq. 3 and Eq. 4 are printed: RR over the
 * whole Ne x Ne matrix (both triangles and the Ne always-recurrent diagonal
 * cells), so a target needs 2 C + Ne >= ceil(rr_num Ne^2 / rr_den) and the
 * upper-triangle target is T_k = ceil((ceil(rr_num Ne^2 / rr_den) - Ne) / 2);
 * DET_k(lmin) = (2 sum_{l>=lmin} l P_k(l) + Ne [Ne >= lmin]) / (2 C_k + Ne),
 * and rqa_line_measures adds the identity line (length Ne) to twice the
 * upper-triangle histogram.  A target that the identity line reaches alone
 * (T_k <= 0) is RQA_ERR_INVALID_ARG.  Counts, histograms and L_max stay those
 * of the upper triangle.  Without the flag the line of identity is left out
 * everywhere (counts over the P = Ne(Ne-1)/2 pairs i < j). */
#define RQA_FLAG_LOI 2

/* A batch of S series stored back to back in one device buffer. */
typedef struct {
    const float *y;          /* device, offsets[S] FP32 values, caller-owned */
    const int64_t *offsets;  /* host, S+1 ascending, offsets[0] = 0 */
    const int32_t *m;        /* host, S embedding dimensions, 1..RQA_M_MAX */
    const int32_t *tau;      /* host, S delays, >= 1 */
    int32_t n_series;        /* S >= 1 */
} rqa_batch;

/* ---- lifetime ------------------------------------------------------------ */

/* Create a context on cfg->device.  cfg may be NULL (device 0, default
 * stream, batched, auto select).  Returns RQA_ERR_CUDA if the device cannot be
 * used.  *out is NULL on failure. */
int rqa_create(rqa_ctx **out, const rqa_config *cfg);

/* Release the context and its scratch (synchronises its stream first). */
void rqa_destroy(rqa_ctx *ctx);

/* Synchronise the context's stream and return the first error any kernel
 * recorded since the last call (then clear it), or a pending CUDA error. */
int rqa_status(rqa_ctx *ctx);

/* Static description of a return code. */
const char *rqa_error_string(int code);

int rqa_abi_version(void);

/* Number of SMs of the context's device and the schedule parameters in use
 * (line-pass register window, blocks per SM as configured: 0 = resident limit);
 * any pointer may be NULL. */
int rqa_device_info(rqa_ctx *ctx, int *sm_count, int *tile, int *blocks_per_sm);

/* Per-phase device times of the context's last hot-path call, in ms, when
 * timing is on (rqa_set_timing): [0] finiteness check, [1] coarse counting
 * round + selection, [2] middle round, [3] final round, [4] line pass,
 * [5] finalisation.  Synchronises the stream.  n >= 6.  Batched schedule
 * only (per-series calls report zeros). */
int rqa_set_timing(rqa_ctx *ctx, int enable);
int rqa_phase_times(rqa_ctx *ctx, float *ms, int n);

/* Number of kernels this context has launched since it was created (graph
 * replays count the kernels of the graph). */
uint64_t rqa_kernel_launches(rqa_ctx *ctx);

/* Graph replays of rqa_det_avg since the context was created. */
uint64_t rqa_graph_replays(rqa_ctx *ctx);

/* Schedule knobs of the line pass.  Every setting gives the same results;
 * only the time differs. */
typedef struct {
    int tile;       /* diagonals per register window of the cell phase: 8, 16 or 32
                       (0 = the default, 16; 8 and 32 only for the embeddings
                       that cfg.tile lists) */
    int unit_bands; /* bands of 32 diagonals per work unit a warp takes from the
                       queue (0 = planned from the batch: about eight units per
                       resident warp, 1..64 otherwise; capped so a unit stays
                       under 2^33 cells) */
    int line_ctas;  /* persistent CTAs of the line pass per SM (0 = as many as
                       fit, else 1..8) */
    int stage;      /* 1: the diagonal pass brings each interior row block's
                       series values into shared memory with 1-D bulk copies
                       (cp.async.bulk, completion on an mbarrier, the next
                       block's copy in flight while the current one computes);
                       0: every lane reads its window through L1.  Only for
                       m = 3 with tau = 3 or 1 and windows of 16 or 32
                       diagonals; ignored elsewhere.  A copy whose barrier does
                       not complete within a bounded wait sets RQA_ERR_TIMEOUT
                       and the block is read directly. */
    float ms;       /* rqa_autotune: the line-pass time of the chosen knobs on
                       the probe, in ms (output only) */
} rqa_tuning;

/* Line-pass tuning: times the line pass over (a prefix of, at most ~2*10^10
 * cells of) the batch with the thresholds of rr_num/rr_den, first over the
 * register windows, then the unit size (half, planned, twice), the CTAs per
 * SM (all that fit, or six) and the staging of series windows (off, on where
 * the variant exists), each step keeping the fastest; stores the choice
 * in the context and returns it in *out (host, may be NULL).  A context
 * created with cfg.tile != 0 keeps that window.  Synchronises the stream. */
int rqa_autotune(rqa_ctx *ctx, const rqa_batch *batch, const int32_t *rr_num, int32_t rr_den,
                 int32_t K, rqa_tuning *out);

/* Set (e.g. from a cache of earlier rqa_autotune results) or read the
 * context's line-pass knobs; RQA_ERR_INVALID_ARG for values out of range. */
int rqa_set_tuning(rqa_ctx *ctx, const rqa_tuning *t);
int rqa_get_tuning(rqa_ctx *ctx, rqa_tuning *t);

/* ---- host helpers (no GPU needed) -------------------------------------- */

/* T_k = ceil(rr_num[k] * P / rr_den) in exact integer arithmetic (Eq. 3
 * inverted).  rr_num[k] in 1..rr_den-1, P >= 1.  Host pointers. */
int rqa_target_counts(uint64_t P, const int32_t *rr_num, int32_t rr_den, int32_t K,
                      uint64_t *T_out);

/* The same with the line of identity counted (RQA_FLAG_LOI; Eq. 3 over the
 * whole Ne x Ne matrix): T_k = ceil((ceil(rr_num Ne^2 / rr_den) - Ne) / 2),
 * the upper-triangle cells that reach the rate.  RQA_ERR_INVALID_ARG when the
 * identity line alone reaches a rate (T_k <= 0), for Ne < 2 or Ne > 2^32.
 * Host pointers. */
int rqa_target_counts_loi(uint64_t Ne, const int32_t *rr_num, int32_t rr_den, int32_t K,
                          uint64_t *T_out);

/* ---- the hot path -------------------------------------------------------- */

/*
 * Exact thresholds for K recurrence-rate targets per series (Sect. 2: the
 * recurrence rate is chosen first and eps is the value that yields it; Eq. 3).
 *   rr_num     host, K numerators, strictly ascending, each in 1..rr_den-1
 *   rr_den     denominator (100 for RR in per cent)
 *   eps_out    device, S*K FP32, row s = series s: eps_k is the T_k-th smallest
 *              upper-triangle distance (non-decreasing in k)
 *   count_le   device, S*K uint64: #{d <= eps_k} (may be NULL)
 *   count_lt   device, S*K uint64: #{d < eps_k}  (may be NULL)
 */
int rqa_eps_for_rr(rqa_ctx *ctx, const rqa_batch *batch, const int32_t *rr_num,
                   int32_t rr_den, int32_t K, float *eps_out, uint64_t *count_le,
                   uint64_t *count_lt);

/* Optional line outputs of rqa_det_avg (any member may be NULL). */
typedef struct {
    uint64_t *hist;               /* device, packed as in rqa_line_hist */
    const int64_t *hist_offsets;  /* host, S+1, as in rqa_line_hist */
    uint32_t *lmax;               /* device, S*K longest line */
    uint64_t *count;              /* device, S*K recurrent cells C_k */
    uint64_t *stencil;            /* device, S*K cells with a recurrent diagonal neighbour */
} rqa_line_outputs;

/*
 * Determinism for each threshold and its average over the thresholds
 * (Eq. 4 and Eq. avgDET) -- the whole hot path in one call when eps == NULL:
 * threshold selection, then one pass over every cell that yields the counts,
 * the line-length histogram and DET for all K thresholds at once.
 *   eps        device, S*K FP32 thresholds, ascending within each series; or
 *              NULL to select them first from rr_num/rr_den as rqa_eps_for_rr
 *              does
 *   rr_num     host, K numerators (read only when eps == NULL)
 *   lmin       host, n_lmin (1..RQA_LMIN_MAX) minimal line lengths, each in
 *              1..65 (paper: 2); DET_k(lmin) is NaN when C_k = 0
 *   det_out    device, S*K*n_lmin FP64, [s][k][j] = DET_k(lmin[j]) (may be NULL)
 *   det_avg    device, S*n_lmin FP64, [s][j] = (1/K) sum_k DET_k(lmin[j])
 *   eps_used   device, S*K FP32 copy of the thresholds used (may be NULL)
 *   lines      optional line outputs of the same pass (may be NULL)
 */
int rqa_det_avg(rqa_ctx *ctx, const rqa_batch *batch, const int32_t *rr_num,
                int32_t rr_den, const float *eps, int32_t K, const int32_t *lmin,
                int32_t n_lmin, double *det_out, double *det_avg, float *eps_used,
                const rqa_line_outputs *lines);

/*
 * Full diagonal line-length histogram of the upper triangle (Eq. 4, Sect. 4).
 *   eps          device, S*K FP32, ascending within each series
 *   hist         device uint64, packed per series: series s occupies
 *                hist[hist_offsets[s] .. hist_offsets[s+1]) laid out as
 *                [k][l-1], l = 1..Ne_s-1, i.e. K*(Ne_s-1) entries; overwritten.
 *                May be NULL (then hist_offsets is ignored).
 *   hist_offsets host, S+1; hist_offsets[s+1]-hist_offsets[s] must equal
 *                K*(Ne_s-1), else RQA_ERR_CAPACITY.
 *   lmax         device, S*K uint32, longest line (may be NULL)
 *   count        device, S*K uint64, recurrent cells C_k (may be NULL)
 *   stencil      device, S*K uint64, recurrent cells with a recurrent diagonal
 *                neighbour = C_k - P_k(1) (may be NULL)
 */
int rqa_line_hist(rqa_ctx *ctx, const rqa_batch *batch, const float *eps, int32_t K,
                  uint64_t *hist, const int64_t *hist_offsets, uint32_t *lmax,
                  uint64_t *count, uint64_t *stencil);

/*
 * Other diagonal-line measures from the same histograms, averaged over the
 * targets like DET (Sect. 2 ends by noting that the averaging applies to
 * other RQA measures; these are the two usually reported next to DET):
 *   N_l  = sum_{l >= lmin} P_k(l)                 lines of length >= lmin
 *   L    = sum_{l >= lmin} l P_k(l) / N_l         average line length, FP64
 *                                                 ratio of exact integers; NaN
 *                                                 when N_l = 0
 *   ENTR = -sum_{l >= lmin} p ln p, p = P_k(l)/N_l  line-length entropy, FP64,
 *                                                 natural log; 0 when N_l = 0
 *   hist, hist_offsets  a full histogram as written by rqa_line_hist or
 *                rqa_det_avg (device; host offsets, checked like theirs)
 *   lmin         host, n_lmin (1..RQA_LMIN_MAX) minimal lengths, each >= 1
 *   L_out, entr_out   device, S*K*n_lmin FP64, [s][k][j] (may be NULL)
 *   L_avg, entr_avg   device, S*n_lmin FP64: the mean over k, summed in k
 *                order then divided by K (may be NULL; computed in context
 *                scratch when the per-target array is NULL)
 * Asynchronous on the context's stream; the histogram must be complete when
 * the stream reaches this call.
 */
int rqa_line_measures(rqa_ctx *ctx, const rqa_batch *batch, int32_t K, const uint64_t *hist,
                      const int64_t *hist_offsets, const int32_t *lmin, int32_t n_lmin,
                      double *L_out, double *entr_out, double *L_avg, double *entr_avg);

/*
 * Vertical lines of the whole Ne x Ne recurrence matrix (both triangles), the
 * input of laminarity and trapping time: V_k(l) = number of maximal runs of
 * length l of recurrent cells along a column (Sect. 2 extends the averaging
 * to other RQA measures; definitions as usual in RQA).  The cell (j, j) ends
 * a run, unless the context has RQA_FLAG_LOI, where it is recurrent.
 *   eps          device, S*K FP32, ascending within each series
 *   vhist        device uint64, packed per series as [k][l-1], l = 1..Ne-1
 *                (l = 1..Ne with RQA_FLAG_LOI); overwritten; may be NULL
 *   vhist_offsets host, S+1: vhist_offsets[s+1]-vhist_offsets[s] must be
 *                K*(Ne_s-1) (K*Ne_s with RQA_FLAG_LOI), else RQA_ERR_CAPACITY
 *   vmax         device, S*K uint32, longest vertical line (may be NULL)
 *   vmass        device, S*K uint64, sum of l V_k(l): every recurrent cell of
 *                the matrix, 2 C_k (+ Ne with RQA_FLAG_LOI) (may be NULL)
 * One sweep over every cell of the matrix per group of at most 20 targets
 * (2P + Ne cells: about twice the diagonal line pass).
 */
int rqa_vline_hist(rqa_ctx *ctx, const rqa_batch *batch, const float *eps, int32_t K,
                   uint64_t *vhist, const int64_t *vhist_offsets, uint32_t *vmax, uint64_t *vmass);

/*
 * Laminarity and trapping time from vertical-line histograms, per target and
 * averaged over the targets (mean in k order, like DET):
 *   LAM = sum_{l >= vmin} l V_k(l) / sum_{l >= 1} l V_k(l)
 *   TT  = sum_{l >= vmin} l V_k(l) / sum_{l >= vmin} V_k(l)   (NaN: no line)
 * FP64 ratios of exact integer sums.
 *   vhist, vhist_offsets  as written by rqa_vline_hist (same context flags)
 *   vmin         host, n_vmin (1..RQA_LMIN_MAX) minimal lengths, each >= 1
 *   lam_out, tt_out   device, S*K*n_vmin FP64 (may be NULL)
 *   lam_avg, tt_avg   device, S*n_vmin FP64 (may be NULL)
 */
int rqa_lam_tt(rqa_ctx *ctx, const rqa_batch *batch, int32_t K, const uint64_t *vhist,
               const int64_t *vhist_offsets, const int32_t *vmin, int32_t n_vmin, double *lam_out,
               double *tt_out, double *lam_avg, double *tt_avg);

/*
 * The paper's approximate threshold search, for comparison with the exact
 * selection (its source describes it in a comment to Sect. 2): every series
 * mapped onto [0, 1] and RR evaluated at n_thr fixed thresholds; for each
 * target the threshold whose RR is the closest.  Grid, in the series' own
 * units (FP32, correctly rounded): thr_i = i * ((max y - min y) / n_thr),
 * i = 1..n_thr.  Upper triangle, recurrent iff d <= thr (RQA_FLAG_LOI is not
 * applied here).  Ties in |RR - target| go to the lower threshold.
 *   rr_num, rr_den, K  as in rqa_eps_for_rr;  n_thr 1..1024 (the paper: 400)
 *   eps_out    device, S*K FP32, the chosen grid thresholds
 *   rr_out     device, S*K FP64, their recurrence rates #{d <= eps}/P (may be NULL)
 *   count_out  device, S*K uint64, #{d <= eps} (may be NULL)
 * The thresholds may then go to rqa_det_avg (its eps argument) for DET.
 */
int rqa_eps_approx(rqa_ctx *ctx, const rqa_batch *batch, const int32_t *rr_num, int32_t rr_den,
                   int32_t K, int32_t n_thr, float *eps_out, double *rr_out, uint64_t *count_out);

/* ---- selection without allocation ---------------------------------------
 *
 * The paper has no counterpart to this entry point; it exists for callers
 * that cannot allocate device memory at the time they need thresholds, for
 * example an application whose own allocator owns the whole device, or a
 * latency-bound host thread that cannot afford the device-wide
 * synchronisation of cudaMalloc/cudaFree.  It computes the same thresholds
 * and counts as rqa_eps_for_rr (bit for bit), for at most
 * RQA_NOALLOC_MAX_SERIES series, without a context and without allocating:
 * its histograms, tables, work items and counters live in one fixed device
 * array of RQA_NOALLOC_SCRATCH_BYTES inside the library, which every device
 * that loads the library keeps until the process exits.
 *   - Runs on the current CUDA device and the given stream (NULL = default).
 *   - The first call on a device looks up that array's device address
 *     (cudaGetSymbolAddress) and the SM count; make that first call before
 *     any stream capture.
 *   - All calls on a device share the array and each call overwrites it;
 *     calls whose work overlaps on the GPU (other streams, other host
 *     threads) race and give wrong results.  Order them on one stream.
 *   - batch->y, eps_out, count_le, count_lt: device, as in rqa_eps_for_rr;
 *     count_le / count_lt may be NULL.
 *   - status_out: device int (may be NULL) that receives the device-side
 *     status of the call (RQA_OK, RQA_ERR_NONFINITE, ...) when it completes.
 *   - K is at most RQA_NOALLOC_K_MAX here (RQA_ERR_INVALID_ARG above).
 *   - Series have Ne <= RQA_NOALLOC_NE_MAX vectors here: each work item
 *     (consecutive diagonals of one series, at most 1024 per series) covers
 *     at most 2^30 cells so the 32-bit shared counts stay exact; a longer
 *     series is RQA_ERR_CAPACITY.
 *   - batch->y, eps_out and the non-NULL count_le, count_lt, status_out must
 *     be memory the current device can address (its device memory or managed
 *     memory), else RQA_ERR_INVALID_ARG.
 *   - Returns RQA_ERR_CAPACITY for more than RQA_NOALLOC_MAX_SERIES series,
 *     and the argument errors of rqa_eps_for_rr; nothing is enqueued then.
 */
#define RQA_NOALLOC_MAX_SERIES 4
#define RQA_NOALLOC_K_MAX 31
#define RQA_NOALLOC_NE_MAX 1048576 /* 2^20 vectors per series */
#define RQA_NOALLOC_SCRATCH_BYTES 1310720 /* 1.25 MiB */
int rqa_eps_for_rr_noalloc(const rqa_batch *batch, const int32_t *rr_num, int32_t rr_den,
                           int32_t K, float *eps_out, uint64_t *count_le, uint64_t *count_lt,
                           int *status_out, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* RQA_H */
