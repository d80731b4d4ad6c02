// Internal declarations shared by the host API and the kernels of librqa.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace rqa {

// FP32 distances are non-negative, so their bit patterns ("keys") order like
// the values and use only bits 30..0.  Exact selection splits a key into an
// 11-bit coarse digit (bits 30..20), a 10-bit middle digit (19..10) and a
// 10-bit low digit (9..0).
constexpr int KMAX = 127;        // targets per series and call
constexpr int LINE_KMAX = 20;    // targets per line-pass sweep (per-lane run state in registers)
constexpr int LINE_BAND = 32;    // diagonals (columns) per warp band of the line pass: one per lane
constexpr int MID_GROUPS = 48;   // middle-round groups per launch (4 KB of shared bins each)
constexpr int COARSE_SHIFT = 20;
constexpr int NCOARSE = 1 << 11;   // 2048 coarse buckets
constexpr int NFINE = 1 << 10;     // 1024 bins per middle / low digit group
constexpr int NHASH_BITS = 12;     // final round: hashed table of the targets' 21-bit prefixes
constexpr int NHASH = 1 << NHASH_BITS;
constexpr int NSUB_MAX = 24;       // bracket-subdivided coarse buckets per series
constexpr int LSH = 64;            // line lengths 1..LSH counted in shared memory
constexpr int LMIN_MAX = 8;        // entries of an lmin list
constexpr int THREADS = 256;       // threads per CTA of the cell kernels
constexpr int BAND = 32;           // diagonals per warp band of the counting rounds
constexpr int ITEM_MIN_BANDS = 4 * 16 * 16 / BAND;  // bands of a work item (1024 diagonals) at least
constexpr int LINE_TILE_DEFAULT = 16;  // diagonals per register window of the line pass's cell phase
constexpr int LINE_NE_MAX = (1 << 26) - 1;  // vectors per series the line pass counts exactly
// vectors per series the counting rounds take: a work item holds under 2^30
// cells plus one band (BAND x Ne), so its 32-bit shared bins cannot overflow
constexpr int64_t COUNT_NE_MAX = ((int64_t)3 << 30) / BAND;
constexpr int WARPS = THREADS / 32;

// Counting rounds of the selection.
enum Round : int {
    R_COARSE = 0,      // coarse digit of every key
    R_COARSE_SUB = 1,  // coarse digit, bracket buckets already split by middle digit
    R_MID = 2,         // middle digit of keys whose coarse digit holds a target
    R_FINAL = 3        // low digit of keys whose 21-bit prefix holds a target
};

struct SeriesDev {
    int64_t off;      // first value of the series in the batch buffer
    int32_t n;        // N
    int32_t ne;       // Ne = N - (m-1) tau
    int32_t m, tau;
    uint64_t P;       // Ne (Ne - 1) / 2
    int32_t nbands;   // ceil((Ne - 1) / band)
    int32_t pad;
};

struct Item {         // bands [b_lo, b_hi) of series s: one CTA's unit of work
    int32_t s, b_lo, b_hi, pad;
};

// Device buffers of the selection state; [s*K + k] unless stated.
struct SelBufs {
    const uint64_t *T;     // target counts
    uint32_t *prefix;      // key bits fixed so far
    uint8_t *level;        // 1: coarse digit known, 2: 21-bit prefix known
    uint64_t *rank;        // rank of the target within its current key interval
    uint64_t *below;       // keys below the current key interval
    int8_t *tab_sub;       // [s][NCOARSE] bracket split buckets -> group, -1
    int8_t *tab_mid;       // [s][NCOARSE] coarse bucket -> middle group, -1
    int8_t *tab_fin1;      // [s][NCOARSE] coarse bucket -> final super group, -1
    int8_t *tab_fin2;      // [s][fin2_stride] = [s][targets][NFINE] (super group, middle digit) -> group
    int64_t fin2_stride;   // entries of tab_fin2 per series (>= K * NFINE)
    uint32_t *tab_hash;    // [s][NHASH] prefix | group << 21 at slot (prefix * mul) >> 20,
                           // 0x1fffff empty; may be null (two-level tables only)
    uint32_t *hash_mul;    // [s]: the slot multiplier, 0 = no collision-free one (or no table)
    int32_t *n_sub, *n_mid, *n_fin;   // [s]
    uint32_t *range;       // [s][2]: keys the next filtered round can count, inclusive
    uint8_t *redo;         // [s]: 1 = the plain coarse round runs for this series
    uint64_t *hist;        // [s][hstride]: NCOARSE coarse bins then fine bins
    int64_t hstride;
};

struct CellArgs {
    const float *y;
    const SeriesDev *series;
    // CTA-level work (counting rounds): items of bands
    const Item *items;
    int32_t n_items;
    int32_t band;
    int32_t g0, gn;          // middle round: the groups [g0, g0 + gn) this launch counts
    // warp-level work (line pass): units of `chunk` consecutive bands of the
    // series order[0..n_pos)
    const int32_t *order;    // series, largest first
    const int64_t *uprefix;  // n_pos + 1 prefix of unit counts along order
    int32_t n_pos;
    int32_t chunk;           // bands per unit
    int32_t line_tile;       // diagonals per register window of the line pass (8, 16 or 32)
    int32_t line_ctas;       // persistent CTAs of the line pass per SM (0: as many as fit)
    int32_t line_stage;      // line pass: stage the series windows by bulk copies (where supported)
    int64_t y_len;           // values in the batch buffer y (bulk copies stay below it)
    int64_t n_units;
    unsigned int *queue;   // ticket counter (64-bit aligned), zeroed before launch
    int *status;
};

// Kernels (launch wrappers return cudaGetLastError()).
cudaError_t launch_check_finite(const float *y, int64_t n, int *status, cudaStream_t st);
// embed: the Embed code of the batch (rqa_common.cuh), picks the distance kernel variant.
cudaError_t launch_count(int round, const CellArgs &a, const SelBufs &sb, int K, int grid,
                         int embed, cudaStream_t st);
cudaError_t launch_select(int round, const SelBufs &sb, const SeriesDev *series, int s_begin,
                          int n_series, int K, float *eps_out, uint64_t *le_out,
                          uint64_t *lt_out, int *status, cudaStream_t st);

struct LineBufs {
    const float *eps;      // [s*kstride + k], ascending per series
    uint64_t *count;       // [s*kstride + k]
    uint32_t *lmax;        // [s*kstride + k]
    uint64_t *hshort;      // [s][kstride][LSH]: P_k(l) for l = 1..LSH
    uint64_t *hist;        // caller's full histogram or nullptr
    const int64_t *hist_off;  // device [S+1] offsets into hist (nullptr if no hist)
    int32_t k0;            // line pass: first target of this launch's group
    int32_t kstride;       // targets per series in all arrays above (the call's K)
    int32_t loi;           // vertical pass: the cells (j, j) are recurrent
};
cudaError_t launch_lines(const CellArgs &a, const LineBufs &lb, int K, int grid, int embed,
                         cudaStream_t st);
// Vertical lines of the whole matrix: the same warp pass over bands of
// LINE_BAND columns (every row of each), reusing the diagonal pass's work plan.
cudaError_t launch_vlines(const CellArgs &a, const LineBufs &lb, int K, int grid, int embed,
                          cudaStream_t st);
bool lines_tile_ok(int embed, int tile);
// The diagonal pass of this embedding and window has a staged variant.
bool lines_stage_ok(int embed, int tile);
cudaError_t launch_finalize_det(const LineBufs &lb, const SeriesDev *series, int S, int K,
                                const int32_t *lmin_dev, int n_lmin, double *det,
                                double *det_avg, bool loi, cudaStream_t st);
cudaError_t launch_line_measures(const uint64_t *hist, const int64_t *hoff_dev, int S, int K,
                                 const int32_t *lmin_dev, int n_lmin, double *L_out,
                                 double *E_out, double *L_avg, double *E_avg, bool loi,
                                 cudaStream_t st);
cudaError_t launch_grid_select(const CellArgs &a, int S, int n_thr, float *thr, uint64_t *hist,
                               const int32_t *rr_num_dev, int rr_den, int K, float *eps_out,
                               double *rr_out, uint64_t *count_out, int grid, int embed,
                               cudaStream_t st);
cudaError_t launch_lam_tt(const uint64_t *hist, const int64_t *hoff_dev, int S, int K,
                          const int32_t *vmin_dev, int n_vmin, double *lam_out, double *tt_out,
                          double *lam_avg, double *tt_avg, cudaStream_t st);
cudaError_t launch_finalize_hist(const LineBufs &lb, const SeriesDev *series, int S, int K,
                                 uint64_t *stencil, cudaStream_t st);

// Largest dynamic shared memory a count round needs for K thresholds.
int count_smem_bytes(int round, int K);

}  // namespace rqa
