// Diagonal lines of the never-materialised recurrence matrices for all K
// thresholds at once (Eq. 4; Sect. 4: upper triangle, cells computed on the
// fly, line lengths from the beginnings and ends of runs).
//
// A warp owns a band of D consecutive diagonals and walks down it 32 rows at
// a time.  For each diagonal of the band, lane t computes the distance of
// cell (i0+t, i0+t+delta) and its rank r = #{k : eps_k < d} (one lookup in
// a bucket table of the thresholds, or a 5-step search over them).  Five
// __ballot_sync calls publish the bit planes of r to the warp; lane k then
// rebuilds its own 32-cell recurrence word {t : r_t <= k} with a bit-sliced
// comparison, and reads its runs with __ffs/__clz/popc bit tricks.  The run
// still open at bit 31 is carried (per diagonal, in a register) into the next
// 32 rows.  So all K thresholds share one distance evaluation per cell, and
// the bitmask work per cell is spread over K lanes.
//
// Outputs per (series, threshold): P_k(l) (lengths up to WSH in a per-warp
// shared histogram flushed once per work unit, WSH+1..LSH in the series'
// global short histogram, longer lines straight to the caller's full
// histogram), L_max, and C_k = sum of l P_k(l), the recurrent cells.
#include <cstdint>
#include <type_traits>
#include "rqa_common.cuh"

namespace rqa {


// Lines of length 1..WSH are counted in the warp's shared histogram; lengths
// WSH+1..LSH go straight to the series' global short histogram and longer
// ones to the caller's full histogram (both rare).
constexpr int WSH = 48;
static_assert(WSH >= 30, "lines inside one 32-cell word must fit the warp histogram");

template <bool HIST>
struct LineSink {
    uint32_t *hs;           // this lane's column of the warp's shared histogram, [length][lane]
    uint64_t *hist;         // this series' full histogram row for lane k, or null
    uint64_t *gshort;       // this series' global short histogram row for lane k
    uint32_t lmax;          // longest line over WSH (shorter ones: read from hs at flush)
    uint32_t longmass;      // cells on lines over WSH (the rest: sum of l * hs[l] at flush)
    uint32_t cp;            // interior lines of length 1, 2, 3 counted by popcount,
                            // packed in 10-bit fields (bits 0, 10, 20)
    bool real;              // lane < K (the other lanes write a dummy row)
    // one line of length len; len == 0 means none (slot 0 is a scratch slot)
    __device__ __forceinline__ void emit(uint32_t len)
    {
        // own column, own bank: no conflicts; one shared atomic instead of a
        // load-add-store chain
        atomicAdd(&hs[(len <= (uint32_t)WSH ? len : 0u) * 32u], 1u);
        if (len > (uint32_t)WSH) {  // rare
            if (real) {
                if (len <= (uint32_t)LSH)
                    atomicAdd(reinterpret_cast<unsigned long long *>(gshort + (len - 1)), 1ull);
                else if (HIST)
                    atomicAdd(reinterpret_cast<unsigned long long *>(hist + (len - 1)), 1ull);
            }
            lmax = max(lmax, len);
            longmass += len;
        }
    }
    // a line strictly inside one 32-cell word: 4 <= len <= 30 < WSH
    __device__ __forceinline__ void emit_interior(uint32_t len) { atomicAdd(&hs[len * 32u], 1u); }
    // fold the popcount tallies into the histogram column
    __device__ __forceinline__ void settle()
    {
        hs[1 * 32] += cp & 1023u;
        hs[2 * 32] += (cp >> 10) & 1023u;
        hs[3 * 32] += cp >> 20;
        cp = 0;
    }
};

// Runs of one 32-cell word (bit t = row i0+t) joined with the open run c,
// without branches on the word's content: the run open from the previous
// word is extended by the word's low ones and closes at its first zero; the
// high ones stay open.  Lines strictly inside the word are bounded by zeros:
// those of length 1..3 are counted with popcounts of the run-start mask,
// longer ones are read one by one with __ffs.
// 3-input bitwise function with an 8-bit truth table (one LOP3 instruction):
// bit i of the table is the output for (a, b, c) = bits of (0xF0, 0xCC, 0xAA).
template <uint32_t LUT>
__device__ __forceinline__ uint32_t lop3(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t d;
    asm("lop3.b32 %0, %1, %2, %3, %4;" : "=r"(d) : "r"(a), "r"(b), "r"(c), "n"(LUT));
    return d;
}
constexpr uint32_t LUT_BORROW = 0x8E;      // (~a & b) | (~a & c) | (b & c)
constexpr uint32_t LUT_A_ANDNOT_B_AND_C = 0x20;  // a & ~b & c
constexpr uint32_t LUT_NOT_A_AND_B = 0x0C;  // ~a & b (c ignored)

__device__ __forceinline__ uint32_t shr_clamped(uint32_t a, uint32_t n)
{
    uint32_t d;  // PTX shr: shift amounts >= 32 give 0
    asm("shr.b32 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(n));
    return d;
}

template <class Sink>
__device__ __forceinline__ void runs_word(uint32_t w, uint32_t &c, Sink &sink)
{
    const uint32_t low = lop3<LUT_NOT_A_AND_B>(w, w + 1u, 0u);  // lowest zero of w (0 if none)
    const uint32_t below = low - 1u;             // the low ones; all ones for a full word
    const uint32_t t0 = __popc(below);           // count of low ones, 32 for a full word
    const uint32_t tl = __clz(~w);               // high ones (32 for a full word)
    const bool open = low == 0u;                 // the carried run crosses the whole word
    const uint32_t ct = c + t0;
    sink.emit(open ? 0u : ct);                   // the carried run closes at the first zero
    c = open ? ct : tl;                          // ... and the high ones stay open
    // interior: without the low ones and without the high ones
    const uint32_t mid = lop3<LUT_A_ANDNOT_B_AND_C>(w, below, shr_clamped(FULL, tl));
    const uint32_t st = mid & ~(mid << 1);       // first cell of each interior line
    const uint32_t s2 = st & (mid >> 1);         // ... of lines of length >= 2
    const uint32_t s3 = s2 & (mid >> 2);         // >= 3
    uint32_t x = s3 & (mid >> 3);                // >= 4
    const uint32_t n1 = __popc(st), n2 = __popc(s2), n3 = __popc(s3);
    // (n1 - n2) + (n2 - n3) 2^10 + (n3 - n4) 2^20 as multiply-adds: each field
    // grows by at most 15 per word (interior lines need a zero between them)
    sink.cp += n1 + n2 * 1023u + n3 * 0xFFC00u - (uint32_t)__popc(x) * 0x100000u;
    while (x) {
        const int p = __ffs(x) - 1;
        sink.emit_interior((uint32_t)(__ffs(~(mid >> p)) - 1));
        x &= x - 1;
    }
}

// Rank table: keys bucketed by key >> shift (1 <= shift <= 22), at most one
// distinct threshold value per bucket; entry = rank of a key up to that value
// (bits 0-4), rank of a key above it (bits 5-9), and the value's offset
// inside the bucket in the top `shift` bits.  One 32x32 -> 64-bit multiply of
// the key by 2^(32-shift) gives the bucket (high word) and the key's offset
// aligned with the entry's (low word): the low word is above the entry
// exactly when the key is above the bucket's threshold, whatever bits 0-9
// hold.
constexpr int TMAX = 384;

// Per-warp shared memory: the warp's own short-line histogram laid out
// [length 0..WSH][lane] (each lane owns one bank; length 0 is a scratch slot,
// lanes >= K own scratch columns), thresholds and rank table.
__host__ __device__ constexpr int warp_smem_words() { return (WSH + 1) * 32 + 32 + TMAX; }

// CTAs of 4 warps: seven fit per SM (registers and shared memory), 28 warps
constexpr int LTHREADS = 128;
constexpr int LWARPS = LTHREADS / 32;
int lines_smem_bytes(int) { return LWARPS * warp_smem_words() * 4; }

// Series s and bands [b_lo, b_hi) of work unit u: a unit is a.chunk
// consecutive bands of one series; units run over the series in a.order
// (largest first), band 0 (longest diagonals) first.  The vertical pass uses
// the same units over bands of columns; a series has ceil(Ne / D) of them,
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
    const int nbd = (series[s].ne - 1 + a.band_lines - 1) / a.band_lines;
    b_hi = min(b_lo + a.chunk, nbd);
    if (VERT && b_lo + a.chunk >= nbd) b_hi = (series[s].ne + a.band_lines - 1) / a.band_lines;
}

// Warp-centric: every warp pulls whole bands from one global queue and keeps
// its own histogram in shared memory, flushed when it moves to another series
// and at exit.  No CTA-wide barrier, so no warp waits for another.
// VERT: the vertical pass -- a band is D consecutive columns c, walked over
// every row i of the matrix (the cell (c, c) ends a line unless lb.loi), and
// the lines found are vertical ones.
template <int D, int M, int TAU, bool HIST, bool VERT = false>
__global__ void __launch_bounds__(LTHREADS, 7) k_lines(CellArgs a, LineBufs lb, int K)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t *hs = reinterpret_cast<uint32_t *>(smem) + warp * warp_smem_words();
    uint32_t *epsb = hs + (WSH + 1) * 32;
    uint32_t *tab = epsb + 32;
    const bool klane = lane < K;

    // bits of k+1 as masks, for the bit-sliced test r <= k (k = lane <= 30
    // for real thresholds; lane 31 would need a sixth bit and is scratch)
    uint32_t kb[5];
#pragma unroll
    for (int b = 0; b < 5; ++b) kb[b] = (((lane + 1) >> b) & 1) ? FULL : 0u;

    for (int x = lane; x < (WSH + 1) * 32; x += 32) hs[x] = 0;
    __syncwarp();

    int cur = -1;
    bool bad = false;
    SeriesDev sd{};
    LineSink<HIST> sink;
    sink.hs = hs + lane;
    sink.hist = nullptr;
    sink.gshort = nullptr;
    sink.lmax = 0;
    sink.longmass = 0;
    sink.cp = 0;
    sink.real = klane;
    int tshift = 0, tbase = 0, tbm1 = 0, tnb = 0;
    uint32_t tmul = 0;  // 2^(32 - tshift)
    bool use_tab = false;

    auto flush = [&]() {
        if (cur < 0) return;
        if (klane) sink.settle();
        __syncwarp();
        uint64_t *gs = lb.hshort + ((int64_t)cur * lb.kstride + lb.k0 + lane) * LSH;
        uint32_t lm = sink.lmax;
        // C_k is the line mass: sum over l of l * P_k(l) (every recurrent cell
        // lies on exactly one line of its diagonal)
        uint32_t cnt = sink.longmass;
#pragma unroll 1
        for (int l = 1; l <= WSH; ++l) {  // row l: one bank per lane
            const uint32_t v = hs[l * 32 + lane];
            if (klane && v) {
                atomicAdd(reinterpret_cast<unsigned long long *>(gs + (l - 1)), (unsigned long long)v);
                hs[l * 32 + lane] = 0;
                lm = max(lm, (uint32_t)l);
                cnt += (uint32_t)l * v;
            }
        }
        sink.lmax = lm;
        if (klane) {
            const int64_t o = (int64_t)cur * lb.kstride + lb.k0 + lane;
            if (cnt) atomicAdd(reinterpret_cast<unsigned long long *>(lb.count + o),
                               (unsigned long long)cnt);
            if (sink.lmax) atomicMax(lb.lmax + o, sink.lmax);
        }
        sink.lmax = 0;
        sink.longmass = 0;
        sink.cp = 0;
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
            tbase = (int)(vmin >> tshift);
            tbm1 = tbase - 1;
            tnb = (int)(vmax >> tshift) - tbase + 1;
            tmul = tshift > 0 ? 1u << (32 - tshift) : 0u;
            use_tab = !bad && tshift > 0 && tnb + 2 <= TMAX;
            __syncwarp();
            if (use_tab) {
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
            if (HIST && klane)
                // a vertical line may span a whole column (Ne cells) when the
                // identity cells are recurrent
                sink.hist = lb.hist + lb.hist_off[s] +
                            (int64_t)(lb.k0 + lane) * (sd.ne - 1 + (VERT && lb.loi ? 1 : 0));
            sink.gshort = lb.hshort + ((int64_t)s * lb.kstride + lb.k0 + (klane ? lane : 0)) * LSH;
            __syncwarp();
        }
        if (bad) continue;

        const float *ys = a.y + sd.off;
        // the unit's bands; the rank method is fixed per unit (branch hoisted)
        auto bands = [&](auto use_table) {
            constexpr bool TABLE = decltype(use_table)::value;
            for (int b = ub_lo; b < ub_hi; ++b) {
                int d_lo = 0, d_hi = 0;
                if (!VERT) band_range(b, D, sd.ne, d_lo, d_hi);
                const int c_lo = b * D;                      // vertical pass: first column
                const int rows = VERT ? sd.ne : sd.ne - d_lo;
                uint32_t carry[D];
#pragma unroll
                for (int j = 0; j < D; ++j) carry[j] = 0;
                // 32 rows of the band; INTERIOR: every cell inside the triangle
                auto row_block = [&](int i0, auto interior) {
                    constexpr bool INTERIOR = decltype(interior)::value;
                    const int i = i0 + lane;
                    BandTile<M, TAU, D> tile;
                    if (VERT) {
                        if (INTERIOR) tile.load_vert_fast(ys, i, c_lo, sd.tau);
                        else tile.load_vert(ys, sd.n, sd.ne, i, c_lo, sd.tau);
                    } else {
                        if (INTERIOR) tile.load_fast(ys, i, d_lo, sd.tau);
                        else tile.load(ys, sd.n, i, d_lo, rows, sd.tau, sd.m);
                    }
#pragma unroll
                    for (int j = 0; j < D; ++j) {
                        // diagonal pass: cell (i, i + dl); vertical: (i, c_lo + j)
                        const int dl = VERT ? c_lo + j - i : d_lo + j;
                        const bool valid =
                            VERT ? (INTERIOR || (i < sd.ne && c_lo + j < sd.ne)) && (lb.loi || dl != 0)
                                 : INTERIOR || i < sd.ne - dl;
                        uint32_t r = 31;  // outside the diagonal: recurrent for no k
                        // register windows read no memory per cell, so cells
                        // outside the triangle are computed and discarded
                        if (TAU > 0 || valid) {
                            const uint32_t key =
                                __float_as_uint(tile.dist(ys, j, i, dl, sd.tau, sd.m));
                            uint32_t rk;
                            if (TABLE) {
                                const uint64_t pk = (uint64_t)key * tmul;
                                const int q = min(max((int)(uint32_t)(pk >> 32) - tbm1, 0), tnb + 1);
                                const uint32_t e = tab[q];
                                rk = ((uint32_t)pk > e) ? (e >> 5) : e;  // bits 0-4: the rank
                            } else {
                                rk = 0;
                                rk += (epsb[rk + 15] < key) ? 16u : 0u;
                                rk += (epsb[rk + 7] < key) ? 8u : 0u;
                                rk += (epsb[rk + 3] < key) ? 4u : 0u;
                                rk += (epsb[rk + 1] < key) ? 2u : 0u;
                                rk += (epsb[rk] < key) ? 1u : 0u;
                            }
                            r = valid ? rk : 31u;
                        }
                        const uint32_t B0 = __ballot_sync(FULL, r & 1u);
                        const uint32_t B1 = __ballot_sync(FULL, r & 2u);
                        const uint32_t B2 = __ballot_sync(FULL, r & 4u);
                        const uint32_t B3 = __ballot_sync(FULL, r & 8u);
                        const uint32_t B4 = __ballot_sync(FULL, r & 16u);
                        // lane k's word {t : r_t <= k}: the borrow out of
                        // r - (k+1), rippled through the five bit planes; each
                        // step is the 3-input majority (~B_j, kb_j, borrow), one
                        // LOP3.  Lanes >= K run it on their scratch column.
                        uint32_t w = lop3<LUT_NOT_A_AND_B>(B0, kb[0], 0u);
                        w = lop3<LUT_BORROW>(B1, kb[1], w);
                        w = lop3<LUT_BORROW>(B2, kb[2], w);
                        w = lop3<LUT_BORROW>(B3, kb[3], w);
                        w = lop3<LUT_BORROW>(B4, kb[4], w);
                        runs_word(w, carry[j], sink);
                    }
                };
                // the packed tallies take 1023 / (15 D) row blocks before a
                // field could overflow
                constexpr int SETTLE = 1023 / (15 * D);
                int i0 = 0, nrb = 0;
                // interior row blocks: every lane's D cells inside the matrix
                const int i_end = VERT ? (c_lo + D <= sd.ne ? rows - 31 : 0) : rows - (D - 1) - 31;
                for (; i0 < i_end; i0 += 32) {
                    row_block(i0, std::true_type{});
                    if (++nrb == SETTLE) {
                        sink.settle();
                        nrb = 0;
                    }
                }
                for (; i0 < rows; i0 += 32) {
                    row_block(i0, std::false_type{});
                    if (++nrb == SETTLE) {
                        sink.settle();
                        nrb = 0;
                    }
                }
                sink.settle();
#pragma unroll
                for (int j = 0; j < D; ++j) sink.emit(carry[j]);  // lines reaching the diagonal's end
            }
        };
        if (use_tab) bands(std::true_type{});
        else bands(std::false_type{});
        // flush after each unit: a warp's next unit is usually another series
        flush();
        cur = -1;
    }
    flush();
}

template <int D, bool HIST>
static void (*lines_kernel_d(int embed))(CellArgs, LineBufs, int)
{
    switch (embed) {
    case E_M1T1: return k_lines<D, 1, 1, HIST>;
    case E_M3T1: return k_lines<D, 3, 1, HIST>;
    case E_M3T3: return k_lines<D, 3, 3, HIST>;
    default: return nullptr;
    }
}

template <bool HIST>
static cudaError_t launch_lines_h(const CellArgs &a, const LineBufs &lb, int K, int grid,
                                  int embed, cudaStream_t st)
{
    void (*kern)(CellArgs, LineBufs, int) = nullptr;
    switch (a.band_lines) {  // band width: specialised embeddings only, others use 4
    case 8: kern = lines_kernel_d<8, HIST>(embed); break;
    case 16: kern = lines_kernel_d<16, HIST>(embed); break;
    default: kern = lines_kernel_d<4, HIST>(embed); break;
    }
    if (!kern) {
        if (a.band_lines != DL_DEFAULT) return cudaErrorInvalidValue;
        switch (embed) {
        case E_M1: kern = k_lines<DL_DEFAULT, 1, 0, HIST>; break;
        case E_M2: kern = k_lines<DL_DEFAULT, 2, 0, HIST>; break;
        case E_M3: kern = k_lines<DL_DEFAULT, 3, 0, HIST>; break;
        case E_M4: kern = k_lines<DL_DEFAULT, 4, 0, HIST>; break;
        default: kern = k_lines<DL_DEFAULT, 0, 0, HIST>; break;
        }
    }
    const int smem = lines_smem_bytes(K);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    grid *= WARPS / LWARPS;  // the caller counts CTAs of WARPS warps
    grid = persistent_cap(reinterpret_cast<const void *>(kern), smem, grid, LTHREADS);
    kern<<<grid, LTHREADS, smem, st>>>(a, lb, K);
    return cudaGetLastError();
}

template <bool HIST>
static cudaError_t launch_vlines_h(const CellArgs &a, const LineBufs &lb, int K, int grid,
                                   int embed, cudaStream_t st)
{
    constexpr int D = DL_DEFAULT;
    void (*kern)(CellArgs, LineBufs, int) = nullptr;
    switch (embed) {
    case E_M1T1: kern = k_lines<D, 1, 1, HIST, true>; break;
    case E_M3T1: kern = k_lines<D, 3, 1, HIST, true>; break;
    case E_M3T3: kern = k_lines<D, 3, 3, HIST, true>; break;
    case E_M1: kern = k_lines<D, 1, 0, HIST, true>; break;
    case E_M2: kern = k_lines<D, 2, 0, HIST, true>; break;
    case E_M3: kern = k_lines<D, 3, 0, HIST, true>; break;
    case E_M4: kern = k_lines<D, 4, 0, HIST, true>; break;
    default: kern = k_lines<D, 0, 0, HIST, true>; break;
    }
    const int smem = lines_smem_bytes(K);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    grid *= WARPS / LWARPS;
    grid = persistent_cap(reinterpret_cast<const void *>(kern), smem, grid, LTHREADS);
    kern<<<grid, LTHREADS, smem, st>>>(a, lb, K);
    return cudaGetLastError();
}

cudaError_t launch_vlines(const CellArgs &a, const LineBufs &lb, int K, int grid, int embed,
                          cudaStream_t st)
{
    const bool hist = lb.hist != nullptr;
    if (a.band_lines != DL_DEFAULT || !a.y || !a.series || !a.order || !a.uprefix || !a.queue ||
        !a.status || !lb.eps || !lb.count || !lb.lmax || !lb.hshort || (hist && !lb.hist_off) ||
        K < 1 || K > LINE_KMAX || lb.k0 < 0 || lb.k0 + K > lb.kstride || grid < 1 || a.n_units < 1 ||
        a.n_pos < 1)
        return cudaErrorInvalidValue;
    return hist ? launch_vlines_h<true>(a, lb, K, grid, embed, st)
                : launch_vlines_h<false>(a, lb, K, grid, embed, st);
}

// Band widths the line pass supports for an embedding variant.
bool lines_band_ok(int embed, int band)
{
    if (band == DL_DEFAULT) return true;
    const bool special = embed == E_M1T1 || embed == E_M3T1 || embed == E_M3T3;
    return special && (band == 8 || band == 16);
}

cudaError_t launch_lines(const CellArgs &a, const LineBufs &lb, int K, int grid, int embed,
                         cudaStream_t st)
{
    const bool hist = lb.hist != nullptr;
    if (!lines_band_ok(embed, a.band_lines)) return cudaErrorInvalidValue;
    if (!a.y || !a.series || !a.order || !a.uprefix || !a.queue || !a.status || !lb.eps ||
        !lb.count || !lb.lmax || !lb.hshort || (hist && !lb.hist_off) || K < 1 || K > LINE_KMAX ||
        lb.k0 < 0 || lb.k0 + K > lb.kstride ||
        grid < 1 || a.n_units < 1 || a.n_pos < 1)
        return cudaErrorInvalidValue;
    return hist ? launch_lines_h<true>(a, lb, K, grid, embed, st)
                : launch_lines_h<false>(a, lb, K, grid, embed, st);
}

}  // namespace rqa
