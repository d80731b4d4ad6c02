// The line pass kernel (template).  Diagonal lines of the never-materialised recurrence matrices for all K
// thresholds at once (Eq. 4; Sect. 4: upper triangle, cells computed on the
// fly, line lengths from the beginnings and ends of runs).
//
// A warp owns a band of LD = 32 consecutive diagonals and walks down it 32
// rows at a time.  Each 32 x 32 row block takes two phases:
//
//  cells  lane t holds row i0+t.  For every diagonal j of the band it computes
//         the distance of cell (i0+t, i0+t+d_lo+j) and its rank
//         r = #{k : eps_k < d} (one lookup in a bucket table of the
//         thresholds, or a 5-step search over them) and stores r as a byte of
//         row j of a 32 x 32 rank matrix in shared memory.
//  runs   lane j holds diagonal j.  It reads row j of the matrix (the ranks of
//         its 32 cells, two 16-byte loads) and gathers their five bit planes:
//         two words of four ranks are interleaved bit by bit, so one mask and
//         one multiply bring bit p of eight ranks into the top byte of a
//         product, and byte permutes put four such bytes together (the rows
//         are stored in the byte order this produces); then, for every
//         threshold k, rebuilds the 32-row recurrence word {t : r_t <= k} (the
//         borrow out of r - (k+1), two LOP3s).  A line ends at row t-1 where
//         row t-1 is recurrent and row t is not; copies of the word shifted
//         down by 1..4 rows (the rows above the block come from the state
//         carried from the previous block) tell whether that line is at least
//         2, 3 or 4 long, so lines of length >= 1, 2 and 3 are counted with
//         three popcounts per word.  Lines of length >= 4 are measured one by one
//         from the nearest non-recurrent row above their end, or from the
//         carried run length when the run started in an earlier block.
//
// All K thresholds share one distance evaluation per cell, and every lane
// works on its own diagonal in the run phase.  The run state carried from one
// row block to the next (per lane and threshold) is the top four bits of the
// previous word and the length of the run open at its last row.
//
// Outputs per (series, threshold): P_k(l) (lengths 1..3 from packed register
// tallies, less the lines measured one by one for length 3; 4..WSH in the
// warp's shared histogram; both flushed once per work
// unit; WSH+1..LSH in the series' global short histogram; longer lines to the
// caller's full histogram), L_max, and C_k = sum of l P_k(l), the recurrent
// cells.
//
// The vertical pass (VERT) is the same kernel over bands of 32 consecutive
// columns walked over every row of the matrix: the word of column c is the
// ballot over 32 consecutive rows, so its runs are vertical lines.
#pragma once
#include <cstdint>
#include <type_traits>
#include "rqa_common.cuh"

namespace rqa {

constexpr int LD = 32;        // diagonals (or columns) per band: one per lane in the run phase
constexpr int KT = LINE_KMAX; // thresholds per sweep: per-lane carry state and tallies in registers
constexpr int WSH = 44;       // lines of length 4..WSH counted in the warp's shared histogram
constexpr int HROW = WSH + 1; // rows 0..WSH of that histogram (row 0: lines longer than WSH)
constexpr int TMAX = 384;     // entries of the rank table
constexpr uint32_t CMASK = 0x0FFFFFFFu;  // carry state: length of the open run ...
constexpr uint32_t TOP4 = 0xF0000000u;   // ... and the top four rows of the previous word
constexpr int SETTLE = 60;    // row blocks between tally settles (10-bit fields, <= 17 per block)

static_assert(LSH > WSH, "lengths WSH+1..LSH go to the global short histogram");

// Per-warp shared memory, in 32-bit words:
//   lq    [KT][LD] 8 bytes each: when the word of threshold k of diagonal j
//         ends lines of length >= 4, their end mask and the run state carried
//         into the word (the run open above it in the low 28 bits); they are
//         measured after the threshold loop (the word
//         itself is rebuilt there from the row block's planes).  The same
//         space first holds the row block's rank matrix, [LD][32] bytes (row
//         j: the ranks of diagonal j's 32 cells), read before any slot is
//         written.
//   pl    [LD][4] bit planes 0..3 of the ranks of the current row block (16-byte rows)
//   pl4   [LD]    bit plane 4 (both written by lane j for diagonal j, read back
//                 when the lines of length >= 4 are measured)
//   epsb  [32]    threshold keys of the current series (padding above every key)
//   tab   [TMAX]  rank table
//   hs    [HROW][32] line counts by length, one column (bank) per lane:
//         rows 1..3 from the tallies (row 3: every line of length >= 3),
//         rows 4..WSH one by one, row 0 the lines longer than WSH
constexpr int O_LQ = 0, O_PL = O_LQ + KT * LD * 2, O_PL4 = O_PL + LD * 4, O_EPS = O_PL4 + LD,
              O_TAB = O_EPS + 32, O_HS = O_TAB + TMAX, WARP_WORDS = (O_HS + HROW * 32 + 3) & ~3;

// Staged variant (diagonal pass, register windows): after hs, the series
// values of one interior row block as the bulk-copy engine brings them in
//   srow  [SR]  the rows' values y[i0 - 3 .. i0 + 32 + (m-1) tau + 3), 16-byte aligned
//   scol  [SC]  the columns' values from y[i0 + d_lo - 3 ..], 16-byte aligned
//   bar   one mbarrier (8 bytes) that counts the two copies' bytes
constexpr int SR = 44, SC = 72;
constexpr int O_STG = WARP_WORDS, O_BAR = O_STG + SR + SC, WARP_WORDS_ST = (O_BAR + 2 + 3) & ~3;
static_assert(O_STG % 4 == 0 && (O_STG + SR) % 4 == 0 && O_BAR % 2 == 0, "copy and barrier alignment");
constexpr uint32_t STAGE_SPIN = 1u << 20;  // polls of a staged block's barrier before giving up

// CTAs of 2 warps: eight fit per SM (shared memory and registers), sixteen warps
constexpr int LTHREADS = 64;
constexpr int LWARPS = LTHREADS / 32;
inline int lines_smem_bytes_impl(bool stage) { return LWARPS * (stage ? WARP_WORDS_ST : WARP_WORDS) * 4; }

// mbarrier and 1-D bulk copy (global -> this CTA's shared memory) in inline PTX.
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(bar), "r"(count) : "memory");
}
// the barrier's initialisation made visible to the copy engine (async proxy),
// and, before a copy overwrites a buffer, the generic-proxy reads of it ordered first
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// one arrival that also announces `bytes` of copies completing on the barrier
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(bar), "r"(bytes)
                 : "memory");
}
// dst and src 16-byte aligned, bytes a multiple of 16
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        :: "r"(dst), "l"(__cvta_generic_to_global(src)), "r"(bytes), "r"(bar) : "memory");
}
// true once the barrier's phase of the given parity has completed
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
    return ok != 0;
}

// Recurrence word of threshold k over the 32 rows: bit t = [r_t <= k], i.e.
// the borrow out of r_t - (k+1) rippled through the bit planes B[0..4] of the
// ranks.  k is a compile-time constant after unrolling, so every step is a
// two-input function of (plane, borrow) and the compiler fuses pairs of steps
// into single LOP3s.  Rank 31 (a cell outside the matrix) is recurrent for no
// k <= 30.
__device__ __forceinline__ uint32_t rank_le_word(const uint32_t (&B)[5], int k)
{
    const int c = k + 1;
    uint32_t lt = 0;
    bool on = false;
#pragma unroll
    for (int b = 0; b < 5; ++b) {
        const bool cb = (c >> b) & 1;
        if (!on) {
            if (cb) {
                lt = ~B[b];
                on = true;
            }
        } else {
            lt = cb ? (~B[b] | lt) : (~B[b] & lt);
        }
    }
    return lt;
}

// 3-input bitwise function with an 8-bit truth table (one LOP3 instruction):
// bit i of the table is the output for (a, b, c) = bits of (0xF0, 0xCC, 0xAA).
template <uint32_t LUT>
__device__ __forceinline__ uint32_t lop3(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t d;
    asm("lop3.b32 %0, %1, %2, %3, %4;" : "=r"(d) : "r"(a), "r"(b), "r"(c), "n"(LUT));
    return d;
}

// The same word for a threshold that differs between lanes: kbm[b] is all
// ones where bit b of k + 1 is set.  Each step is the borrow of one bit
// plane: (~r & c) | (~r & borrow) | (c & borrow), one LOP3.
__device__ __forceinline__ uint32_t rank_le_word_lane(uint32_t b0, uint32_t b1, uint32_t b2,
                                                      uint32_t b3, uint32_t b4,
                                                      const uint32_t (&kbm)[5])
{
    uint32_t w = lop3<0x0C>(b0, kbm[0], 0u);  // ~r0 & c0
    w = lop3<0x8E>(b1, kbm[1], w);
    w = lop3<0x8E>(b2, kbm[2], w);
    w = lop3<0x8E>(b3, kbm[3], w);
    return lop3<0x8E>(b4, kbm[4], w);
}

// Series s and bands [b_lo, b_hi) of work unit u: a unit is a.chunk
// consecutive bands of one series; units run over the series in a.order
// (largest first), band 0 (longest diagonals) first.  The vertical pass uses
// the same units over bands of columns; a series has ceil(Ne / LD) of them,
// at most one more than of diagonals, which its last unit takes on.
template <bool VERT>
__device__ __forceinline__ void unit_of(const CellArgs &a, int64_t u, int &s, int &b_lo,
                                        int &b_hi, const SeriesDev *series)
{
    int lo = 0, hi = a.n_pos;  // last pos with uprefix[pos] <= u
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (a.uprefix[mid] <= u) lo = mid;
        else hi = mid;
    }
    s = a.order[lo];
    b_lo = (int)(u - a.uprefix[lo]) * a.chunk;
    const int nbd = (series[s].ne - 1 + LD - 1) / LD;
    b_hi = min(b_lo + a.chunk, nbd);
    if (VERT && b_lo + a.chunk >= nbd) b_hi = (series[s].ne + LD - 1) / LD;
}

// Warp-centric: every warp pulls units from one global queue and keeps its
// own histogram in shared memory, flushed after each unit.  No CTA-wide
// barrier, so no warp waits for another.
// JC: diagonals whose cells a lane computes from one register window of the
// series (the cell phase walks the band's 32 diagonals in LD / JC windows).
// Transpose a 32 x 32 bit matrix held one row per lane: on return lane k
// holds column k (bit j of the result = bit k of lane j's word).  Five rounds
// of exchanging off-diagonal blocks with the lane s apart.
__device__ __forceinline__ uint32_t transpose32(uint32_t x, int lane)
{
    constexpr uint32_t MASKS[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
    for (int r = 0; r < 5; ++r) {
        const int sh = 16 >> r;
        const uint32_t m = MASKS[r];
        const uint32_t y = __shfl_xor_sync(FULL, x, sh);
        x = (lane & sh) ? ((x & ~m) | ((y & ~m) >> sh)) : ((x & m) | ((y & m) << sh));
    }
    return x;
}

// STAGE: the interior row blocks' series values come into shared memory by
// bulk copies (one per segment, issued by lane 0 for the next row block while
// the current one computes) instead of per-lane loads through L1.
// FK: a full sweep, K = KT thresholds known at compile time (the per-threshold
// code then runs without a test of k against K); the argument is ignored.
template <int M, int TAU, int JC, bool VERT, bool STAGE = false, bool FK = false>
__global__ void __launch_bounds__(LTHREADS, 8) k_lines(CellArgs a, LineBufs lb, int K_arg)
{
    const int K = FK ? KT : K_arg;
    static_assert(LD % JC == 0 && JC % 4 == 0, "windows of whole plane-4 groups");
    static_assert(!STAGE || (TAU > 0 && !VERT && ((32 + (M - 1) * TAU + 6) & ~3) <= SR &&
                             ((31 + LD + (M - 1) * TAU + 6) & ~3) <= SC),
                  "staging: register windows of the diagonal pass that fit the buffers");
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t *ws = reinterpret_cast<uint32_t *>(smem) + warp * (STAGE ? WARP_WORDS_ST : WARP_WORDS);
    uint32_t *pl = ws + O_PL, *pl4 = ws + O_PL4, *epsb = ws + O_EPS, *tab = ws + O_TAB;
    uint32_t *hs = ws + O_HS + lane;  // this lane's column: [l * 32], threshold kk (below)
    uint2 *lqa = reinterpret_cast<uint2 *>(ws + O_LQ);  // [k * LD + j]
    unsigned char *rkm = reinterpret_cast<unsigned char *>(ws + O_LQ);  // rank matrix, row j
    uint2 *lq = lqa + lane;                               // slots of this lane's diagonal
    const bool klane = lane < K;
    // byte of row `lane` in a row of the rank matrix: rows 8h + 2u and 8h + 2u + 1
    // sit four bytes apart (bytes 8h + u and 8h + u + 4), the order the plane
    // gather of the run phase reads them in
    const int rcol = (lane & ~7) | ((lane & 7) >> 1) | ((lane & 1) << 2);
    // Lines of length >= 4: lane k < K measures those of threshold k; the
    // 32 - K lanes left over help the top thresholds (the ones with the most
    // lines), lane L >= K taking threshold L - (32 - K) on the odd diagonals
    // while that threshold's own lane keeps the even ones.  kk: the threshold
    // a lane measures (-1: none); its histogram column is its own.
    const int kpart = lane - (32 - K);  // lane >= K: the threshold it helps (< 0: none)
    const int kk = klane ? lane : kpart;
    const uint32_t dsel = klane ? (lane >= 2 * K - 32 ? 0x55555555u : FULL)
                                : (kpart >= 0 ? 0xAAAAAAAAu : 0u);
    // the bits of kk + 1 as masks, for rebuilding the recurrence words of threshold kk
    uint32_t kbm[5];
#pragma unroll
    for (int b = 0; b < 5; ++b) kbm[b] = (((kk + 1) >> b) & 1) ? FULL : 0u;

    for (int l = 0; l < HROW; ++l) hs[l * 32] = 0;

    // staging state (warp-uniform): the buffers hold at most one row block
    float *const srow = reinterpret_cast<float *>(ws + O_STG), *const scol = srow + SR;
    const uint32_t sbar = static_cast<uint32_t>(__cvta_generic_to_shared(ws + O_BAR));
    bool son = STAGE && (reinterpret_cast<uintptr_t>(a.y) & 15u) == 0;  // copies allowed
    bool sinf = false;      // a copy issued and not yet waited for
    uint32_t sph = 0;       // parity of the barrier phase that copy completes
    int srs = 0, scs = 0;   // offsets of y[i0] in srow and of y[i0 + d_lo] in scol
    if (STAGE && lane == 0) {
        mbar_init(sbar, 1);
        fence_proxy_async_smem();
    }
    __syncwarp();
    uint64_t lmass = 0;  // cells on lines of threshold kk longer than WSH (this unit, this lane)
    uint32_t lmx = 0;    // the longest of them

    int cur = -1;
    bool bad = false;
    SeriesDev sd{};
    int tshift = 0, tbm1 = 0, tnb = 0;
    uint32_t tmul = 0;  // 2^(32 - tshift)
    bool use_tab = false;
    uint32_t tal[KT];   // per threshold: ends of lines >= 1, >= 2, >= 3 minus those >= 4
                        // (10-bit fields at bits 0, 10, 20)
#pragma unroll
    for (int k = 0; k < KT; ++k) tal[k] = 0;
    int nrb = 0;        // row blocks since the last settle

    // tallies -> column k, rows 1..3: P(1) = f1 - f2, P(2) = f2 - f3, P(3) = f3
    auto settle = [&]() {
        uint32_t g1 = 0, g2 = 0, g3 = 0;  // lane k: the sums of threshold k
#pragma unroll
        for (int k = 0; k < KT; ++k) {
            if (k < K) {
                const uint32_t f1 = __reduce_add_sync(FULL, tal[k] & 1023u);
                const uint32_t f2 = __reduce_add_sync(FULL, (tal[k] >> 10) & 1023u);
                const uint32_t f3 = __reduce_add_sync(FULL, tal[k] >> 20);
                if (lane == k) {
                    g1 = f1;
                    g2 = f2;
                    g3 = f3;
                }
            }
            tal[k] = 0;
        }
        if (klane) {
            hs[1 * 32] += g1 - g2;
            hs[2 * 32] += g2 - g3;
            hs[3 * 32] += g3;
        }
        nrb = 0;
        __syncwarp();
    };

    // A lane's column to the short histogram of threshold kk (both lanes of a
    // helped threshold add theirs).  Row 3 of column k holds every line of
    // length >= 3; those of length >= 4 are counted again one by one (rows
    // 4..WSH and row 0, in the columns of threshold k's lane and its helper),
    // so P_k(3) is row 3 less them.  C_k is the line mass, sum over l of
    // l * P_k(l) (every recurrent cell lies on exactly one line of its
    // diagonal), and L_max the longest line.
    auto flush = [&]() {
        if (cur < 0) return;
        settle();
        const int64_t o = (int64_t)cur * lb.kstride + lb.k0 + (kk < 0 ? 0 : kk);
        uint64_t *gs = lb.hshort + o * LSH;
        uint64_t cnt = lmass;
        uint32_t lm = lmx;
        uint32_t longer = hs[0];  // this column's lines of length >= 4
        hs[0] = 0;
        auto put = [&](int l, uint32_t v) {
            if (v) {
                atomicAdd(reinterpret_cast<unsigned long long *>(gs + (l - 1)), (unsigned long long)v);
                cnt += (uint64_t)l * v;
                lm = max(lm, (uint32_t)l);
            }
        };
        if (kk >= 0) {
#pragma unroll 1
            for (int l = 4; l <= WSH; ++l) {  // row l: one bank per lane
                const uint32_t v = hs[l * 32];
                if (v) {
                    hs[l * 32] = 0;
                    longer += v;
                    put(l, v);
                }
            }
        }
        // lane k: the lines of length >= 4 its helper counted
        const uint32_t helped = __shfl_sync(FULL, longer, min(lane + 32 - K, 31));
        if (klane) {
            if (lane >= 2 * K - 32) longer += helped;
            put(1, hs[1 * 32]);
            put(2, hs[2 * 32]);
            put(3, hs[3 * 32] - longer);
            hs[1 * 32] = 0;
            hs[2 * 32] = 0;
            hs[3 * 32] = 0;
        }
        if (kk >= 0) {
            if (cnt) atomicAdd(reinterpret_cast<unsigned long long *>(lb.count + o),
                               (unsigned long long)cnt);
            if (lm) atomicMax(lb.lmax + o, lm);
        }
        lmass = 0;
        lmx = 0;
        __syncwarp();
    };

    for (;;) {
        int64_t u = 0;
        if (lane == 0) u = (int64_t)atomicAdd(reinterpret_cast<unsigned long long *>(a.queue), 1ull);
        u = __shfl_sync(FULL, u, 0);
        if (u >= a.n_units) break;
        int s, ub_lo, ub_hi;
        unit_of<VERT>(a, u, s, ub_lo, ub_hi, a.series);
        if (s != cur) {
            flush();
            cur = s;
            sd = a.series[s];
            uint32_t v = 0xffffffffu;   // padding: above every key
            bool ok = true;
            if (klane) {
                v = __float_as_uint(lb.eps[(int64_t)s * lb.kstride + lb.k0 + lane]);
                if (v == 0x80000000u) v = 0u;                           // -0 == +0
                if ((v & 0x80000000u) || v > 0x7f800000u) ok = false;  // negative or NaN
            }
            const uint32_t prev = __shfl_up_sync(FULL, v, 1);
            if (klane && lane > 0 && prev > v) ok = false;              // not ascending
            bad = !__all_sync(FULL, ok);
            epsb[lane] = v;
            if (bad && lane == 0) set_status(a.status, 8 /*UNSORTED*/);
            // rank table: the widest buckets that still separate every pair
            // of distinct thresholds
            tshift = 22;
            for (; tshift > 0; --tshift) {
                const bool clash = klane && lane > 0 && prev != v && (prev >> tshift) == (v >> tshift);
                if (!__any_sync(FULL, clash)) break;
            }
            const uint32_t vmin = __shfl_sync(FULL, v, 0), vmax = __shfl_sync(FULL, v, K - 1);
            const int tbase = (int)(vmin >> tshift);
            tbm1 = tbase - 1;
            tnb = (int)(vmax >> tshift) - tbase + 1;
            tmul = tshift > 0 ? 1u << (32 - tshift) : 0u;
            use_tab = !bad && tshift > 0 && tnb + 2 <= TMAX;
            __syncwarp();
            if (use_tab) {
                // entry: rank of a key up to the bucket's threshold (bits 0-4),
                // rank of a key above it (bits 5-9), the threshold's offset
                // inside the bucket in the top tshift bits
                for (int q = lane; q < tnb + 2; q += 32) {
                    uint32_t e;
                    if (q == 0) {
                        e = 0u;                    // below every threshold's bucket
                    } else if (q == tnb + 1) {
                        e = (uint32_t)K | ((uint32_t)K << 5);  // above: all K thresholds are smaller
                    } else {
                        uint32_t rlo = 0, cnt = 0, off = 0;
                        for (int k = 0; k < K; ++k) {
                            const uint32_t ek = epsb[k];
                            const int eb = (int)(ek >> tshift) - tbase;
                            if (eb < q - 1) ++rlo;
                            else if (eb == q - 1) { ++cnt; off = ek * tmul; }
                        }
                        e = rlo | ((rlo + cnt) << 5) | off;
                    }
                    tab[q] = e;
                }
            }
            __syncwarp();
        }
        if (bad) continue;

        const float *ys = a.y + sd.off;
        // the full histogram row of threshold k (lane-independent base)
        const int64_t hrow = sd.ne - 1 + (VERT && lb.loi ? 1 : 0);
        uint64_t *const hbase =
            lb.hist ? lb.hist + lb.hist_off[s] + (int64_t)lb.k0 * hrow : nullptr;
        uint64_t *const gshort = lb.hshort + ((int64_t)s * lb.kstride + lb.k0) * LSH;

        // Staging of interior row block i0 of the band at d_lo: the values of
        // its rows, y[i0 .. i0 + 32 + (m-1) tau), and of its columns,
        // y[i0 + d_lo .. i0 + d_lo + 31 + LD + (m-1) tau), both widened to
        // 16-byte boundaries; only when the widened segments stay inside the
        // batch buffer (else the block reads global memory).  The caller has
        // finished reading the buffers.
        auto stage_issue = [&](int i0, int d_lo) -> bool {
            const int64_t gr = sd.off + i0, gc = gr + d_lo;
            const int64_t ar = gr & ~(int64_t)3, ac = gc & ~(int64_t)3;
            const int64_t er = (gr + 32 + (M - 1) * TAU + 3) & ~(int64_t)3;
            const int64_t ec = (gc + 31 + LD + (M - 1) * TAU + 3) & ~(int64_t)3;
            if (er > a.y_len || ec > a.y_len) return false;
            srs = (int)(gr - ar);
            scs = (int)(gc - ac);
            __syncwarp();  // every lane's reads of the buffers done
            if (lane == 0) {
                const uint32_t br = (uint32_t)(er - ar) * 4u, bc = (uint32_t)(ec - ac) * 4u;
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(sbar, br + bc);
                bulk_g2s(static_cast<uint32_t>(__cvta_generic_to_shared(srow)), a.y + ar, br, sbar);
                bulk_g2s(static_cast<uint32_t>(__cvta_generic_to_shared(scol)), a.y + ac, bc, sbar);
            }
            sinf = true;
            return true;
        };
        // wait (bounded) for the staged block; on a time-out the block reads
        // global memory, staging stops and the status records RQA_ERR_TIMEOUT
        auto stage_wait = [&]() -> bool {
            bool ok = false;
            for (uint32_t it = 0; it < STAGE_SPIN && !ok; ++it) ok = mbar_try_wait(sbar, sph);
            if (__all_sync(FULL, ok)) {
                sph ^= 1u;
                sinf = false;
                return true;
            }
            son = false;
            if (lane == 0) set_status(a.status, 6 /*TIMEOUT*/);
            return false;
        };

        // a line of threshold kk longer than WSH (rare): its length into the
        // series' short histogram or the caller's full one
        auto emit_rare = [&](uint32_t len) {
            lmx = max(lmx, len);
            lmass += len;
            hs[0] += 1u;  // row 0 of the lane's column: lines longer than WSH
            if (len <= (uint32_t)LSH)
                atomicAdd(reinterpret_cast<unsigned long long *>(gshort + (int64_t)kk * LSH + (len - 1)),
                          1ull);
            else if (hbase)
                atomicAdd(reinterpret_cast<unsigned long long *>(hbase + (int64_t)kk * hrow + (len - 1)),
                          1ull);
        };

        // Lines of length >= 4.  Lane j's mask has bit k when slot [k][j]
        // holds the word of threshold k of diagonal j; a bit transpose hands
        // lane k the diagonals of its threshold, so every lane adds to its own
        // histogram column.  In a slot, a line ends at row t - 1 for each bit t
        // of the end mask; its first row follows the nearest non-recurrent row
        // above, or it continues the run open above the word (bit 0: a line
        // ending at the previous word's last row).
        //
        // The loop is warp-uniform (its condition is a vote) and takes at most
        // one line per lane per turn with predicated steps and a predicated
        // shared reduction, so no lane's data steers the warp's control flow;
        // only a line longer than WSH branches.
        auto long_lines = [&](uint32_t mask) {
            if (!__any_sync(FULL, mask != 0u)) return;
            __syncwarp();  // every lane's slots written before other lanes read them
            // lane k: diagonals j with lines of threshold k; then the share of the
            // lane's own threshold kk (all, the even or the odd diagonals)
            uint32_t diag = transpose32(mask, lane);
            diag = __shfl_sync(FULL, diag, kk < 0 ? 0 : kk) & dsel;
            uint32_t x = 0, wq = 0, cq = 0;           // the slot being read
            const uint32_t hcol = static_cast<uint32_t>(__cvta_generic_to_shared(hs));
            while (__any_sync(FULL, (x | diag) != 0u)) {
                if (x == 0u && diag != 0u) {  // the next diagonal's slot
                    const int j = __ffs(diag) - 1;
                    diag &= diag - 1u;
                    const uint2 q = lqa[kk * LD + j];
                    x = q.x;
                    cq = q.y & CMASK;
                    const uint4 b4 = *reinterpret_cast<const uint4 *>(pl + j * 4);
                    wq = rank_le_word_lane(b4.x, b4.y, b4.z, b4.w, pl4[j], kbm);
                }
                // the lowest end bit t of the slot (lowb = 2^t; 0 when the lane
                // has no line left); the line ends at row t - 1 and starts below
                // the nearest non-recurrent row above it, or continues the run
                // open above the word when rows 0 .. t - 1 are all recurrent
                // (then clz(zb) = 32): len = t - 32 + clz(zb) + [zb == 0] * cq
                const bool has = x != 0u;
                const uint32_t lowb = x & (0u - x);
                x ^= lowb;
                const uint32_t zb = ~wq & (lowb - 1u);
                const uint32_t cz = __clz(zb);
                const uint32_t len = cz - (uint32_t)__clz(lowb) - 1u + (cz >> 5) * cq;
                red_shared_if_le(hcol + min(len, (uint32_t)WSH) * 128u, has ? len : ~0u, (uint32_t)WSH);
                if (has && len > (uint32_t)WSH) emit_rare(len);
            }
            __syncwarp();  // slots are rewritten by the next block
        };

        // the unit's bands; the rank method is fixed per unit (branch hoisted)
        auto bands = [&](auto use_table) {
            constexpr bool TABLE = decltype(use_table)::value;
            auto rank_of = [&](uint32_t key) -> uint32_t {
                if (TABLE) {
                    const uint64_t pk = (uint64_t)key * tmul;
                    // bucket - (tbase - 1) clamped to [0, tnb + 1]: max(min(a + b, c), 0)
                    const int q = __viaddmin_s32_relu((int)(uint32_t)(pk >> 32), -tbm1, tnb + 1);
                    const uint32_t e = tab[q];
                    return ((uint32_t)pk > e) ? (e >> 5) : e;  // bits 0-4: the rank
                }
                uint32_t rk = 0;
                rk += (epsb[rk + 15] < key) ? 16u : 0u;
                rk += (epsb[rk + 7] < key) ? 8u : 0u;
                rk += (epsb[rk + 3] < key) ? 4u : 0u;
                rk += (epsb[rk + 1] < key) ? 2u : 0u;
                rk += (epsb[rk] < key) ? 1u : 0u;
                return rk;
            };
            for (int b = ub_lo; b < ub_hi; ++b) {
                const int d_lo = 1 + b * LD;                 // diagonal pass: first diagonal
                const int c_lo = b * LD;                     // vertical pass: first column
                const int rows = VERT ? sd.ne : sd.ne - d_lo;  // rows of the band's longest line
                uint32_t st[KT];
#pragma unroll
                for (int k = 0; k < KT; ++k) st[k] = 0;
                bool staged = false;  // the next interior row block is in the buffers

                // cell phase of the 32 rows i0..i0+31: bit planes of the ranks
                // of every diagonal into pl / pl4.  INTERIOR: every cell of the
                // block inside the triangle (no bounds checks).
                // STAGE: `next` says that row block i0 + 32 is interior too;
                // its copy is issued once this block's windows are in registers.
                auto cell_phase = [&](int i0, auto interior, bool next) {
                    constexpr bool INTERIOR = decltype(interior)::value;
                    const int i = i0 + lane;
                    bool from_smem = false;
                    if (STAGE && INTERIOR && staged) {
                        from_smem = stage_wait();
                        staged = false;
                    }
#pragma unroll 1
                    for (int jc = 0; jc < LD; jc += JC) {
                        BandTile<M, TAU, JC> tile;
                        if constexpr (STAGE) {
                            if (INTERIOR && from_smem) tile.load_smem(srow + srs, scol + scs + jc, lane);
                            else if (INTERIOR) tile.load_fast(ys, i, d_lo + jc, sd.tau);
                            else tile.load(ys, sd.n, i, d_lo + jc, rows, sd.tau, sd.m);
                            if (INTERIOR && next && son && jc + JC == LD) staged = stage_issue(i0 + 32, d_lo);
                        } else if (VERT) {
                            if (INTERIOR) tile.load_vert_fast(ys, i, c_lo + jc, sd.tau);
                            else tile.load_vert(ys, sd.n, sd.ne, i, c_lo + jc, sd.tau);
                        } else {
                            if (INTERIOR) tile.load_fast(ys, i, d_lo + jc, sd.tau);
                            else tile.load(ys, sd.n, i, d_lo + jc, rows, sd.tau, sd.m);
                        }
#pragma unroll
                        for (int j = 0; j < JC; ++j) {
                            const int col = c_lo + jc + j;   // vertical pass: column
                            // diagonal pass: cell (i, i + dl); vertical: (i, col)
                            const int dl = VERT ? col - i : d_lo + jc + j;
                            const bool valid =
                                VERT ? (INTERIOR || (i < sd.ne && col < sd.ne)) && (lb.loi || dl != 0)
                                     : INTERIOR || i < sd.ne - dl;
                            uint32_t r = 31;  // outside the matrix: recurrent for no k
                            // register windows read no memory per cell, so cells
                            // outside the triangle are computed and discarded
                            if (TAU > 0 || valid) {
                                const uint32_t key =
                                    __float_as_uint(tile.dist(ys, j, i, dl, sd.tau, sd.m));
                                const uint32_t rk = rank_of(key);
                                r = valid ? rk : 31u;
                            }
                            rkm[(jc + j) * 32 + rcol] = (unsigned char)r;
                        }
                    }
                };

                // run phase of the same 32 rows: lane j takes diagonal j
                auto run_phase = [&]() {
                    __syncwarp();
                    const uint4 ra = *reinterpret_cast<const uint4 *>(rkm + lane * 32);
                    const uint4 rb = *reinterpret_cast<const uint4 *>(rkm + lane * 32 + 16);
                    const uint32_t R[8] = {ra.x, ra.y, ra.z, ra.w, rb.x, rb.y, rb.z, rb.w};
                    // Words 2h and 2h + 1 hold rows 8h .. 8h + 7 (byte u of word
                    // 2h: row 8h + 2u, of word 2h + 1: row 8h + 2u + 1).  X[h]
                    // interleaves their even bits (bit p of byte u of word 2h
                    // at p + 8u, of word 2h + 1 at p + 1 + 8u), Xo[h] their odd
                    // bits one place lower.  For plane p the two bits of each
                    // byte pair are masked and one multiply by
                    // 2^24 + 2^18 + 2^12 + 2^6 (shifted down by the pair's bit
                    // position) moves the eight of them, rows in order, into
                    // bits 24..31 with no two partial products meeting (so no
                    // carry reaches the top byte); three byte permutes join the
                    // four top bytes into the plane.
                    uint32_t X[4], Xo[4];
#pragma unroll
                    for (int h = 0; h < 4; ++h) {
                        X[h] = (R[2 * h] & 0x55555555u) | ((R[2 * h + 1] << 1) & 0xAAAAAAAAu);
                        Xo[h] = ((R[2 * h] >> 1) & 0x55555555u) | (R[2 * h + 1] & 0xAAAAAAAAu);
                    }
                    uint32_t B[5];
#pragma unroll
                    for (int p = 0; p < 5; ++p) {
                        const int sh = p & ~1;
                        uint32_t v[4];
#pragma unroll
                        for (int h = 0; h < 4; ++h)
                            v[h] = ((p & 1 ? Xo[h] : X[h]) & (0x03030303u << sh)) * (0x01041040u >> sh);
                        const uint32_t lo = __byte_perm(v[0], v[1], 0x0073);
                        const uint32_t hi = __byte_perm(v[2], v[3], 0x7300);
                        B[p] = __byte_perm(lo, hi, 0x7610);
                    }
                    // this diagonal's planes, for rebuilding words of long lines
                    *reinterpret_cast<uint4 *>(pl + lane * 4) = make_uint4(B[0], B[1], B[2], B[3]);
                    pl4[lane] = B[4];
                    __syncwarp();  // rank rows read before slots overwrite them
                    uint32_t lmask = 0;  // thresholds whose word ends lines of length >= 4
#pragma unroll
                    for (int k = 0; k < KT; ++k) {
                        if (k < K) {
                            const uint32_t w = rank_le_word(B, k);
                            const uint32_t s0 = st[k];
                            // row t of p_n = row t - n (rows above the block: the
                            // previous word's top four rows, kept in the state)
                            const uint32_t p1 = __funnelshift_l(s0, w, 1);
                            const uint32_t p2 = __funnelshift_l(s0, w, 2);
                            const uint32_t p3 = __funnelshift_l(s0, w, 3);
                            const uint32_t p4 = __funnelshift_l(s0, w, 4);
                            // bit t: a line ends at row t - 1 (t = 0: the previous
                            // block's last row) and is at least 1, 2, 3, 4 long
                            const uint32_t e1 = p1 & ~w;
                            const uint32_t e2 = e1 & p2;
                            const uint32_t e3 = e2 & p3;
                            const uint32_t e4 = e3 & p4;
                            // every line counts towards lengths >= 1, 2, 3; those of
                            // length >= 4 are measured one by one after the loop
                            // (rare for noisy series) and taken off length 3 at the flush
                            tal[k] += __popc(e1) + (__popc(e2) << 10) + (__popc(e3) << 20);
                            if (e4) {  // the reader takes the run length from the state's low bits
                                lq[k * LD] = make_uint2(e4, s0);
                                lmask |= 1u << k;
                            }
                            // the new state: top rows of this word and the run open at
                            // its last row.  c = 32 only for an all-ones word, whose run
                            // continues the one open above: c + s0 has the old length
                            // + 32 in its low bits (the sum stays under 2^28), and its
                            // top bits are overwritten by the word's, all ones.
                            const uint32_t c = __clz(~w);
                            st[k] = (w & TOP4) | (s0 * (c >> 5) + c);
                        }
                    }
                    long_lines(lmask);
                };

                // the packed tallies take SETTLE row blocks before a field could overflow
                int i0 = 0;
                // interior row blocks: every cell of the block inside the matrix
                const int i_end = VERT ? (c_lo + LD <= sd.ne ? rows - 31 : 0) : rows - (LD - 1) - 31;
                if (STAGE && son && i_end > 0) staged = stage_issue(0, d_lo);
                for (; i0 < i_end; i0 += 32) {
                    cell_phase(i0, std::true_type{}, i0 + 32 < i_end);
                    run_phase();
                    if (++nrb == SETTLE) settle();
                }
                for (; i0 < rows; i0 += 32) {
                    cell_phase(i0, std::false_type{}, false);
                    run_phase();
                    if (++nrb == SETTLE) settle();
                }
                // lines that reach the end of a diagonal exactly at a block's last
                // row: a line of length c ending just above a word (end bit 0)
                uint32_t bmask = 0;
#pragma unroll
                for (int k = 0; k < KT; ++k) {
                    if (k < K) {
                        const uint32_t c = st[k] & CMASK;
                        tal[k] += c == 0 ? 0u : c == 1 ? 1u : c == 2 ? 0x401u : 0x100401u;
                        if (c >= 4) {
                            lq[k * LD] = make_uint2(1u, c);
                            bmask |= 1u << k;
                        }
                    }
                }
                long_lines(bmask);
            }
        };
        if (use_tab) bands(std::true_type{});
        else bands(std::false_type{});
        // flush after each unit: a warp's next unit is usually another series
        flush();
        cur = -1;
    }
    flush();
    // a copy left in flight by a time-out: wait for it (bounded) before the
    // CTA's shared memory is released
    if (STAGE && sinf) {
        bool ok = false;
        for (uint32_t it = 0; it < STAGE_SPIN && !ok; ++it) ok = mbar_try_wait(sbar, sph);
    }
}

}  // namespace rqa

namespace rqa {
using LinesKernel = void (*)(CellArgs, LineBufs, int);
// Instantiations, one group per translation unit (they compile in parallel).
// full: the diagonal pass's variant for a sweep of exactly LINE_KMAX thresholds
LinesKernel lines_kernel_m3t3(int tile, bool vert, bool full);
LinesKernel lines_kernel_m3t1(int tile, bool vert, bool full);
LinesKernel lines_kernel_m1t1(int tile, bool vert, bool full);
LinesKernel lines_kernel_generic(int m, bool vert);
LinesKernel lines_kernel_staged(int embed, int tile);  // nullptr where there is none
}  // namespace rqa
