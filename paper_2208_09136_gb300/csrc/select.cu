// Exact selection of the thresholds that give the chosen recurrence rates
// (Sect. 2: RR is fixed first and eps follows from it; Eq. 3).
//
// eps_k is the T_k-th smallest upper-triangle distance.  Distances are never
// stored: every counting round recomputes them over diagonal bands and
// histograms one digit of their FP32 bit pattern (the "key"; non-negative
// floats order like their bit patterns).  Rounds:
//   R_COARSE      bits 30..20 of every key                    -> 2048 bins
//   R_COARSE_SUB  as R_COARSE, but coarse buckets a learned bracket marks are
//                 split at once by bits 19..10 (skips R_MID for those targets)
//   R_MID         bits 19..10 of keys in a target's coarse bucket
//   R_FINAL       bits 9..0 of keys in a target's 21-bit prefix
// After each round a select kernel turns the histogram into (prefix, rank,
// below) per target.  After R_FINAL the key is complete: eps_k, and
// #{d < eps_k} = below, #{d <= eps_k} = below + (keys equal to eps_k).
#include <cstdint>
#include <type_traits>
#include "rqa_common.cuh"

namespace rqa {

// ------------------------------------------------------------ finiteness
__global__ void k_check_finite(const float *__restrict__ y, int64_t n, int *status)
{
    int bad = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        bad |= !isfinite(y[i]);
    if (__any_sync(FULL, bad) && (threadIdx.x & 31) == 0) set_status(status, 3 /*NONFINITE*/);
}

cudaError_t launch_check_finite(const float *y, int64_t n, int *status, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    k_check_finite<<<(int)blocks, 256, 0, st>>>(y, n, status);
    return cudaGetLastError();
}

// ------------------------------------------------------------ counting
int count_smem_bytes(int round, int K)
{
    switch (round) {
    case R_COARSE: return NCOARSE * 4;
    case R_COARSE_SUB: return (NCOARSE + NSUB_MAX * NFINE) * 4 + NCOARSE;
    case R_MID: return (K < MID_GROUPS ? K : MID_GROUPS) * NFINE * 4 + NCOARSE;
    default: {  // tables only (final-round keys are rare): the hash or the two levels
        const int two = NCOARSE + 1 + K * NFINE;
        return two > NHASH * 4 ? two : NHASH * 4;
    }
    }
}

__device__ __forceinline__ uint32_t smem_addr(const uint32_t *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Resident CTAs per SM the compiler must leave room for (0: no bound): the
// final round of the compile-time embeddings with tau > 1 fits four in 64
// registers without spills instead of three in 80; the others keep the
// compiler's own choice.
__host__ __device__ constexpr int count_min_ctas(int round, int tau)
{
    return round == R_FINAL && tau > 1 ? 4 : 0;
}

// One persistent launch over the work items; each CTA histograms the keys of
// its item's bands in shared memory and adds the non-zero bins to the
// series' 64-bit global histogram at the end of the item.
//
// R_COARSE counts every key.  The bracket round counts only the keys of its
// split range and keeps the keys below it as one register count; the middle
// and final rounds look each key up in their group tables (the final round's
// rare hits go straight to the global bins, so it needs no shared histogram).
template <int ROUND, int M, int TAU>
__global__ void __launch_bounds__(count_threads(ROUND), count_min_ctas(ROUND, TAU)) k_count(CellArgs a, SelBufs sb, int K)
{
    constexpr int NT = count_threads(ROUND);
    constexpr bool FILTERED = ROUND != R_COARSE;
    constexpr bool GLOBAL_BINS = ROUND == R_FINAL;  // final-round keys are rare: count in HBM
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int slot;
    __shared__ int nb_used_sh;
    __shared__ uint32_t hmul_sh;
    __shared__ int next_band;
    __shared__ uint32_t key_lo, key_hi;
    __shared__ unsigned long long below_sh;
    __shared__ uint32_t sink[32];  // lane x's reductions of cells that count nowhere (never read)
    const int nbins_max = (ROUND == R_COARSE) ? NCOARSE
                        : (ROUND == R_COARSE_SUB) ? NCOARSE + NSUB_MAX * NFINE
                        : (ROUND == R_MID) ? (K < MID_GROUPS ? K : MID_GROUPS) * NFINE : 0;
    uint32_t *h = reinterpret_cast<uint32_t *>(smem);
    int8_t *t1 = reinterpret_cast<int8_t *>(h + nbins_max);
    int8_t *t2 = t1 + NCOARSE;
    uint32_t *th = reinterpret_cast<uint32_t *>(smem);  // final round, hashed: instead of t1/t2
    const int lane = threadIdx.x & 31;

    for (int x = threadIdx.x; x < nbins_max; x += NT) h[x] = 0;

    for (;;) {
        const int it = next_item(a.queue, a.n_items, &slot);
        if (it < 0) break;
        const Item item = a.items[it];
        const SeriesDev sd = a.series[item.s];
        if (threadIdx.x == 0) {
            int nb;
            if (ROUND == R_COARSE) nb = sb.redo[item.s] ? NCOARSE : 0;
            else if (ROUND == R_COARSE_SUB) nb = sb.n_sub[item.s] ? NCOARSE + sb.n_sub[item.s] * NFINE : 0;
            else if (ROUND == R_MID) nb = max(0, min(sb.n_mid[item.s] - a.g0, a.gn)) * NFINE;
            else nb = sb.n_fin[item.s] * NFINE;
            nb_used_sh = nb;
            next_band = item.b_lo;
            key_lo = 0u;
            key_hi = 0xffffffffu;
            if (FILTERED) {
                key_lo = sb.range[2 * (int64_t)item.s];
                key_hi = sb.range[2 * (int64_t)item.s + 1];
            }
            below_sh = 0ull;
            hmul_sh = (ROUND == R_FINAL && sb.hash_mul) ? sb.hash_mul[item.s] : 0u;
        }
        __syncthreads();
        const int nb_used = nb_used_sh;
        const uint32_t hmul = hmul_sh;
        if (nb_used == 0) continue;  // no target of this series needs this round
        if (ROUND == R_FINAL && hmul) {
            const uint4 *src = reinterpret_cast<const uint4 *>(sb.tab_hash + (int64_t)item.s * NHASH);
            for (int x = threadIdx.x; x < NHASH / 4; x += NT) reinterpret_cast<uint4 *>(th)[x] = src[x];
            __syncthreads();
        } else if (ROUND != R_COARSE) {
            const int8_t *src = (ROUND == R_COARSE_SUB) ? sb.tab_sub
                              : (ROUND == R_MID) ? sb.tab_mid : sb.tab_fin1;
            src += (int64_t)item.s * NCOARSE;
            for (int x = threadIdx.x; x < NCOARSE; x += NT) t1[x] = src[x];
            if (ROUND == R_FINAL) {
                const int8_t *s2 = sb.tab_fin2 + (int64_t)item.s * sb.fin2_stride;
                for (int x = threadIdx.x; x < K * NFINE; x += NT) t2[1 + x] = s2[x];
                if (threadIdx.x == 0) t2[0] = -1;
            }
            __syncthreads();
        }

        const float *ys = a.y + sd.off;
        const uint32_t klo = key_lo, kspan = key_hi - key_lo;  // inside: key - klo <= kspan
        unsigned long long *gbins =
            reinterpret_cast<unsigned long long *>(sb.hist + (int64_t)item.s * sb.hstride + NCOARSE);
        uint32_t below = 0;  // bracket round: keys under its range
        // bracket round with every bucket from the first to the last split
        // one split (the usual case): split group g is bucket first + g, so
        // the bin is (key - klo) >> 10 past the coarse bins, no table
        const bool dense = ROUND == R_COARSE_SUB && ((kspan >> COARSE_SHIFT) + 1u) * NFINE + NCOARSE ==
                                                        (uint32_t)nb_used;
        const uint32_t hsub = static_cast<uint32_t>(__cvta_generic_to_shared(h + NCOARSE));
        const uint32_t sink_a = smem_addr(&sink[lane]);
        // the item's bands; FAST: dense bracket round, or final round with the
        // hashed prefix table
        auto item_bands = [&](auto fast) {
        constexpr bool FAST = decltype(fast)::value;
        for (;;) {
            // bands are handed to warps one at a time, so no warp idles while
            // another still has several bands of the item left
            int b = 0;
            if (lane == 0) b = atomicAdd(&next_band, 1);
            b = __shfl_sync(FULL, b, 0);
            if (b >= item.b_hi) break;
            int d_lo, d_hi;
            band_range(b, BAND, sd.ne, d_lo, d_hi);
            const int rows = sd.ne - d_lo;
            int last = -1;
            uint32_t run = 0;
            // plain coarse round: every key counts and neighbouring cells of
            // a lane often share a coarse bin, so equal bins are aggregated
            auto count_coarse = [&](uint32_t key) {
                const int bin = (int)(key >> COARSE_SHIFT);
                if (bin == last) {
                    ++run;
                } else {
                    if (run) atomicAdd(&h[last], run);
                    last = bin;
                    run = 1;
                }
            };
            // the BAND cells of a lane in one row block; valid = inside the
            // triangle.  The filtered rounds compute the bin of every cell
            // (keys of finite or NaN distances have bit 31 clear, so key >> 20
            // indexes the 2048-entry table).  The bracket round, where many
            // cells fall in the range, adds one for every cell with an
            // unconditional reduction (into the lane's sink word for a cell
            // outside the range); a conditional one would make the compiler
            // wrap each cell in a branch region.  The middle round, where few
            // cells count, uses a predicated reduction, and the final round
            // branches around its rare global atomics.
            auto row_block = [&](const BandTile<M, TAU, BAND> &tile, int i, bool interior) {
#pragma unroll
                for (int j = 0; j < BAND; ++j) {
                    const int dl = d_lo + j;
                    const bool valid = interior || i < sd.ne - dl;
                    const uint32_t key = __float_as_uint(tile.dist(ys, j, i, dl, sd.tau, sd.m));
                    const int c = (int)(key >> COARSE_SHIFT);
                    const int fine = (int)((key >> 10) & (NFINE - 1));
                    if (ROUND == R_COARSE) {
                        if (valid) count_coarse(key);
                    } else if (ROUND == R_COARSE_SUB && FAST) {
                        // keys under klo wrap to rel >= 2^31 (keys are < 2^31)
                        const uint32_t rel = key - klo;
                        below += valid ? rel >> 31 : 0u;
                        red_shared(valid && rel <= kspan ? hsub + ((rel >> 10) << 2) : sink_a);
                    } else if (ROUND == R_COARSE_SUB) {
                        below += (valid && key < klo) ? 1u : 0u;
                        const int g = t1[c];
                        const int bin = g < 0 ? c : NCOARSE + g * NFINE + fine;
                        red_shared(valid && key - klo <= kspan ? smem_addr(&h[bin]) : sink_a);
                    } else if (ROUND == R_MID) {
                        // groups outside this launch's window [g0, g0 + gn) wait for another
                        const uint32_t gw = (uint32_t)((int)t1[c] - a.g0);
                        red_shared_if_le(smem_addr(&h[min(gw, (uint32_t)(nbins_max / NFINE - 1)) * NFINE + fine]),
                                         valid ? gw : ~0u, (uint32_t)a.gn - 1u);
                    } else if (FAST) {
                        // one probe: the slot holds the only target prefix
                        // that can map there.  Empty slots hold group 0 with
                        // prefix 0x1fffff, which only a NaN key (already an
                        // error) can match, inside group 0's bins.
                        const uint32_t pfx = key >> 10;
                        const uint32_t e = th[(pfx * hmul) >> (32 - NHASH_BITS)];
                        if (valid && ((e ^ pfx) & 0x1FFFFFu) == 0u)  // rare
                            atomicAdd(gbins + (e >> 21) * NFINE + (key & (NFINE - 1)), 1ull);
                    } else {
                        // t2[0] is a -1 sentinel: no branch on the first lookup
                        const int g1 = t1[c];
                        const int g = t2[g1 < 0 ? 0 : 1 + g1 * NFINE + fine];
                        if (valid && g >= 0)  // rare: a key of a target's 21-bit prefix
                            atomicAdd(gbins + g * NFINE + (int)(key & (NFINE - 1)), 1ull);
                    }
                }
            };
            int i0 = 0;
            // interior row blocks: every lane's cells on all BAND diagonals exist
            for (; i0 + 32 <= rows - (BAND - 1); i0 += 32) {
                BandTile<M, TAU, BAND> tile;
                tile.load_fast(ys, i0 + lane, d_lo, sd.tau);
                row_block(tile, i0 + lane, true);
            }
            for (; i0 < rows; i0 += 32) {
                BandTile<M, TAU, BAND> tile;
                tile.load(ys, sd.n, i0 + lane, d_lo, rows, sd.tau, sd.m);
                row_block(tile, i0 + lane, false);
            }
            if (run) atomicAdd(&h[last], run);
        }
        };
        if ((ROUND == R_FINAL && hmul) || dense) item_bands(std::true_type{});
        else item_bands(std::false_type{});
        if (ROUND == R_COARSE_SUB) {
            // keys under the bracket: one count, kept in the coarse bucket
            // just below it (every bucket under it is empty in this round)
            unsigned long long bw = below;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) bw += __shfl_xor_sync(FULL, bw, o);
            if (lane == 0 && bw) atomicAdd(&below_sh, bw);
        }
        __syncthreads();
        if (ROUND == R_COARSE_SUB && threadIdx.x == 0 && below_sh) {
            const int cb = (int)(klo >> COARSE_SHIFT) - 1;  // >= 0 whenever keys lie below
            atomicAdd(reinterpret_cast<unsigned long long *>(sb.hist + (int64_t)item.s * sb.hstride + cb),
                      below_sh);
        }
        uint64_t *gh = sb.hist + (int64_t)item.s * sb.hstride + (ROUND >= R_MID ? NCOARSE : 0) +
                       (ROUND == R_MID ? (int64_t)a.g0 * NFINE : 0);
        for (int x = threadIdx.x; x < (GLOBAL_BINS ? 0 : nb_used); x += NT) {
            const uint32_t v = h[x];
            if (v) {
                atomicAdd(reinterpret_cast<unsigned long long *>(gh + x), (unsigned long long)v);
                h[x] = 0;
            }
        }
    }
}

template <int ROUND>
static cudaError_t launch_count_m(const CellArgs &a, const SelBufs &sb, int K, int grid,
                                  int embed, cudaStream_t st)
{
    const int smem = count_smem_bytes(ROUND, K);
    void (*kern)(CellArgs, SelBufs, int);
    switch (embed) {
    case E_M1T1: kern = k_count<ROUND, 1, 1>; break;
    case E_M3T1: kern = k_count<ROUND, 3, 1>; break;
    case E_M3T3: kern = k_count<ROUND, 3, 3>; break;
    case E_M1: kern = k_count<ROUND, 1, 0>; break;
    case E_M2: kern = k_count<ROUND, 2, 0>; break;
    case E_M3: kern = k_count<ROUND, 3, 0>; break;
    case E_M4: kern = k_count<ROUND, 4, 0>; break;
    default: kern = k_count<ROUND, 0, 0>; break;
    }
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    grid = persistent_cap(reinterpret_cast<const void *>(kern), smem, grid, count_threads(ROUND));
    kern<<<grid, count_threads(ROUND), smem, st>>>(a, sb, K);
    return cudaGetLastError();
}

cudaError_t launch_count(int round, const CellArgs &a, const SelBufs &sb, int K, int grid,
                         int embed, cudaStream_t st)
{
    if (!a.y || !a.series || !a.items || !a.queue || !a.status || !sb.hist || K < 1 || K > KMAX ||
        grid < 1 || a.n_items < 1 || a.band != BAND)
        return cudaErrorInvalidValue;
    if (round == R_MID && (a.g0 < 0 || a.gn < 1 || a.gn > MID_GROUPS)) return cudaErrorInvalidValue;
    switch (round) {
    case R_COARSE: return launch_count_m<R_COARSE>(a, sb, K, grid, embed, st);
    case R_COARSE_SUB: return launch_count_m<R_COARSE_SUB>(a, sb, K, grid, embed, st);
    case R_MID: return launch_count_m<R_MID>(a, sb, K, grid, embed, st);
    default: return launch_count_m<R_FINAL>(a, sb, K, grid, embed, st);
    }
}

// ------------------------------------------------------------ selection
// In-place inclusive scan of n 64-bit values in shared memory (n a multiple
// of THREADS).
__device__ void block_scan_u64(uint64_t *v, int n, uint64_t *warp_tot)
{
    const int per = n / THREADS;
    const int t = threadIdx.x;
    uint64_t s = 0;
    for (int x = 0; x < per; ++x) {
        s += v[t * per + x];
        v[t * per + x] = s;
    }
    uint64_t incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t u = __shfl_up_sync(FULL, incl, o);
        if ((t & 31) >= o) incl += u;
    }
    if ((t & 31) == 31) warp_tot[t >> 5] = incl;
    __syncthreads();
    uint64_t wpre = 0;
    for (int w = 0; w < (t >> 5); ++w) wpre += warp_tot[w];
    const uint64_t excl = wpre + incl - s;
    for (int x = 0; x < per; ++x) v[t * per + x] += excl;
    __syncthreads();
}

// Smallest index x with a[x] >= v (n if none).
__device__ __forceinline__ int lower_bound_u64(const uint64_t *a, int n, uint64_t v)
{
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Load the NFINE bins of fine group g of series s and scan them.
__device__ void load_scan_group(const uint64_t *gh_fine, int g, uint64_t *cum, uint64_t *wt)
{
    const uint64_t *src = gh_fine + (int64_t)g * NFINE;
    for (int x = threadIdx.x; x < NFINE; x += THREADS) cum[x] = src[x];
    __syncthreads();
    block_scan_u64(cum, NFINE, wt);
}

// One CTA per series.  ROUND is the counting round whose histogram is read.
template <int ROUND>
__global__ void __launch_bounds__(THREADS)
k_select(SelBufs sb, const SeriesDev *series, int s_begin, int K, float *eps_out,
         uint64_t *le_out, uint64_t *lt_out, int *status)
{
    __shared__ uint64_t cum[NCOARSE];
    __shared__ uint64_t wt[WARPS];
    __shared__ uint32_t pre[KMAX];
    __shared__ uint8_t lev[KMAX];
    __shared__ uint64_t rnk[KMAX], blw[KMAX];
    __shared__ int grp[KMAX];
    const int s = s_begin + blockIdx.x;
    const int t = threadIdx.x;
    const int64_t sk = (int64_t)s * K;
    const uint64_t *gh = sb.hist + (int64_t)s * sb.hstride;
    const uint64_t *gfine = gh + NCOARSE;
    (void)series;

    if (ROUND == R_COARSE && !sb.redo[s]) return;  // the bracket settled this series
    if (ROUND == R_COARSE || ROUND == R_COARSE_SUB) {
        __shared__ int hard;  // bracket round: some target outside the bracket
        if (t == 0) hard = 0;
        // bucket totals; a split bucket's keys sit in its fine group
        for (int x = t; x < NCOARSE; x += THREADS) cum[x] = gh[x];
        __syncthreads();
        if (ROUND == R_COARSE_SUB) {
            __shared__ int inv[NSUB_MAX];
            const int nsub = sb.n_sub[s];
            const int8_t *tab = sb.tab_sub + (int64_t)s * NCOARSE;
            if (t < NSUB_MAX) inv[t] = -1;
            __syncthreads();
            for (int c = t; c < NCOARSE; c += THREADS) {
                const int g = tab[c];
                if (g >= 0 && g < NSUB_MAX) inv[g] = c;
            }
            __syncthreads();
            for (int g = 0; g < nsub; ++g) {
                uint64_t part = 0;
                for (int x = t; x < NFINE; x += THREADS) part += gfine[(int64_t)g * NFINE + x];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(FULL, part, o);
                if ((t & 31) == 0) wt[t >> 5] = part;
                __syncthreads();
                if (t == 0 && inv[g] >= 0) {
                    uint64_t tot = 0;
                    for (int w = 0; w < WARPS; ++w) tot += wt[w];
                    cum[inv[g]] += tot;
                }
                __syncthreads();
            }
        }
        block_scan_u64(cum, NCOARSE, wt);
        // bracket round: only the bracket's buckets were counted (keys under it
        // lumped into the bucket just below, keys above it not at all)
        const int sub_lo = (int)(sb.range[2 * (int64_t)s] >> COARSE_SHIFT);
        const int sub_hi = (int)(sb.range[2 * (int64_t)s + 1] >> COARSE_SHIFT);
        if (t < K) {
            const uint64_t R = sb.T[sk + t];
            const int c = lower_bound_u64(cum, NCOARSE, R);
            if (ROUND == R_COARSE_SUB &&
                (sb.n_sub[s] == 0 || c >= NCOARSE || c < sub_lo || c > sub_hi)) {
                pre[t] = 0; lev[t] = 0; rnk[t] = R; blw[t] = 0;  // outside: full selection
                hard = 1;
            } else if (c >= NCOARSE || R == 0) {
                set_status(status, 10 /*INTERNAL*/);
                pre[t] = 0; lev[t] = 1; rnk[t] = 1; blw[t] = 0;
            } else {
                const uint64_t below = c ? cum[c - 1] : 0;
                pre[t] = (uint32_t)c;
                lev[t] = 1;
                rnk[t] = R - below;
                blw[t] = below;
            }
            grp[t] = -1;
        }
        __syncthreads();
        if (ROUND == R_COARSE_SUB) {
            const int8_t *tab = sb.tab_sub + (int64_t)s * NCOARSE;
            if (t < K) grp[t] = (lev[t] == 1) ? tab[pre[t]] : -1;
            __syncthreads();
            const int nsub = sb.n_sub[s];
            for (int g = 0; g < nsub; ++g) {
                bool any = false;
                for (int k = 0; k < K; ++k) any |= (grp[k] == g);
                if (!any) continue;
                load_scan_group(gfine, g, cum, wt);
                if (t < K && grp[t] == g) {
                    const int x = lower_bound_u64(cum, NFINE, rnk[t]);
                    if (x >= NFINE) {
                        set_status(status, 10);
                    } else {
                        const uint64_t below = x ? cum[x - 1] : 0;
                        pre[t] = (pre[t] << 10) | (uint32_t)x;
                        lev[t] = 2;
                        rnk[t] -= below;
                        blw[t] += below;
                    }
                }
                __syncthreads();
            }
        }
        if (ROUND == R_COARSE_SUB) {
            if (t == 0) sb.redo[s] = (uint8_t)hard;
            if (hard) {  // the plain rounds redo this series; levels kept for the statistics
                if (t < K) sb.level[sk + t] = lev[t];
                return;
            }
        }
        // middle-round table: coarse bucket -> group, for targets at level 1
        int8_t *tm = sb.tab_mid + (int64_t)s * NCOARSE;
        for (int x = t; x < NCOARSE; x += THREADS) tm[x] = -1;
        __syncthreads();
        if (t == 0) {
            int g = 0;
            uint32_t lo = 0xffffffffu, hi = 0u;
            for (int k = 0; k < K; ++k) {
                if (lev[k] != 1) continue;
                if (tm[pre[k]] < 0) tm[pre[k]] = (int8_t)g++;
                lo = min(lo, pre[k] << COARSE_SHIFT);
                hi = max(hi, ((pre[k] + 1u) << COARSE_SHIFT) - 1u);
            }
            sb.n_mid[s] = g;
            sb.range[2 * (int64_t)s] = lo;
            sb.range[2 * (int64_t)s + 1] = hi;
        }
        if (t < K) {
            sb.prefix[sk + t] = pre[t];
            sb.level[sk + t] = lev[t];
            sb.rank[sk + t] = rnk[t];
            sb.below[sk + t] = blw[t];
        }
        return;
    }

    // R_MID and R_FINAL: state from global memory
    if (t < K) {
        pre[t] = sb.prefix[sk + t];
        lev[t] = sb.level[sk + t];
        rnk[t] = sb.rank[sk + t];
        blw[t] = sb.below[sk + t];
    }
    __syncthreads();

    if (ROUND == R_MID) {
        const int8_t *tm = sb.tab_mid + (int64_t)s * NCOARSE;
        if (t < K) grp[t] = (lev[t] == 1) ? tm[pre[t]] : -1;
        __syncthreads();
        const int nmid = sb.n_mid[s];
        for (int g = 0; g < nmid; ++g) {
            load_scan_group(gfine, g, cum, wt);
            if (t < K && grp[t] == g) {
                const int x = lower_bound_u64(cum, NFINE, rnk[t]);
                if (x >= NFINE) {
                    set_status(status, 10);
                } else {
                    const uint64_t below = x ? cum[x - 1] : 0;
                    pre[t] = (pre[t] << 10) | (uint32_t)x;
                    lev[t] = 2;
                    rnk[t] -= below;
                    blw[t] += below;
                }
            }
            __syncthreads();
        }
        // final-round tables for all targets (every target is at level 2 now)
        int8_t *f1 = sb.tab_fin1 + (int64_t)s * NCOARSE;
        int8_t *f2 = sb.tab_fin2 + (int64_t)s * sb.fin2_stride;
        uint32_t *fh = sb.tab_hash ? sb.tab_hash + (int64_t)s * NHASH : nullptr;
        for (int x = t; x < NCOARSE; x += THREADS) f1[x] = -1;
        for (int x = t; x < K * NFINE; x += THREADS) f2[x] = -1;
        for (int x = t; fh && x < NHASH; x += THREADS) fh[x] = 0x1fffffu;  // group 0, no finite key
        __syncthreads();
        if (t == 0) {
            int g1 = 0, g = 0;
            uint32_t lo = 0xffffffffu, hi = 0u;
            for (int k = 0; k < K; ++k) {
                const uint32_t c = pre[k] >> 10, mid = pre[k] & (NFINE - 1);
                if (f1[c] < 0) f1[c] = (int8_t)g1++;
                int8_t *e = f2 + f1[c] * NFINE + mid;
                if (*e < 0) *e = (int8_t)g++;
                lo = min(lo, pre[k] << 10);
                hi = max(hi, ((pre[k] + 1u) << 10) - 1u);
            }
            sb.n_fin[s] = g;
            sb.range[2 * (int64_t)s] = lo;
            sb.range[2 * (int64_t)s + 1] = hi;
            // hashed table of the distinct prefixes (group order): the first
            // odd multiplier of a fixed sequence that puts them in distinct
            // slots; none among 64 (never seen) keeps the two-level tables
            if (fh) {
                uint32_t pg[KMAX];
                for (int k = 0; k < K; ++k) {
                    const int gk = f2[f1[pre[k] >> 10] * NFINE + (pre[k] & (NFINE - 1))];
                    pg[gk] = pre[k];
                }
                uint32_t mul = 0;
                for (int a = 0; a < 64 && !mul; ++a) {
                    const uint32_t m = (0x9E3779B1u + 0x6A09E668u * (uint32_t)a) | 1u;
                    bool ok = true;
                    for (int i = 1; i < g && ok; ++i)
                        for (int j = 0; j < i && ok; ++j)
                            ok = ((pg[i] * m) >> (32 - NHASH_BITS)) != ((pg[j] * m) >> (32 - NHASH_BITS));
                    if (ok) mul = m;
                }
                if (mul)
                    for (int i = 0; i < g; ++i) fh[(pg[i] * mul) >> (32 - NHASH_BITS)] = pg[i] | ((uint32_t)i << 21);
                sb.hash_mul[s] = mul;
            }
        }
        if (t < K) {
            sb.prefix[sk + t] = pre[t];
            sb.level[sk + t] = lev[t];
            sb.rank[sk + t] = rnk[t];
            sb.below[sk + t] = blw[t];
        }
        return;
    }

    // R_FINAL: the low digit completes the key
    {
        const int8_t *f1 = sb.tab_fin1 + (int64_t)s * NCOARSE;
        const int8_t *f2 = sb.tab_fin2 + (int64_t)s * sb.fin2_stride;
        if (t < K) {
            const int g1 = f1[pre[t] >> 10];
            grp[t] = (g1 < 0) ? -1 : f2[g1 * NFINE + (pre[t] & (NFINE - 1))];
            if (grp[t] < 0) set_status(status, 10);
        }
        __syncthreads();
        const int nfin = sb.n_fin[s];
        for (int g = 0; g < nfin; ++g) {
            load_scan_group(gfine, g, cum, wt);
            if (t < K && grp[t] == g) {
                const int x = lower_bound_u64(cum, NFINE, rnk[t]);
                if (x >= NFINE) {
                    set_status(status, 10);
                } else {
                    const uint64_t lt = blw[t] + (x ? cum[x - 1] : 0);
                    const uint64_t le = blw[t] + cum[x];
                    const uint32_t key = (pre[t] << 10) | (uint32_t)x;
                    eps_out[sk + t] = __uint_as_float(key);
                    if (le_out) le_out[sk + t] = le;
                    if (lt_out) lt_out[sk + t] = lt;
                }
            }
            __syncthreads();
        }
    }
}

cudaError_t launch_select(int round, const SelBufs &sb, const SeriesDev *series, int s_begin,
                          int n_series, int K, float *eps_out, uint64_t *le_out,
                          uint64_t *lt_out, int *status, cudaStream_t st)
{
    if (n_series <= 0) return cudaSuccess;
    switch (round) {
    case R_COARSE:
        k_select<R_COARSE><<<n_series, THREADS, 0, st>>>(sb, series, s_begin, K, eps_out, le_out,
                                                          lt_out, status);
        break;
    case R_COARSE_SUB:
        k_select<R_COARSE_SUB><<<n_series, THREADS, 0, st>>>(sb, series, s_begin, K, eps_out,
                                                              le_out, lt_out, status);
        break;
    case R_MID:
        k_select<R_MID><<<n_series, THREADS, 0, st>>>(sb, series, s_begin, K, eps_out, le_out,
                                                       lt_out, status);
        break;
    default:
        k_select<R_FINAL><<<n_series, THREADS, 0, st>>>(sb, series, s_begin, K, eps_out, le_out,
                                                         lt_out, status);
        break;
    }
    return cudaGetLastError();
}

}  // namespace rqa
