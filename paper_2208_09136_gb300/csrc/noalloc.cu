// rqa_eps_for_rr_noalloc: exact threshold selection for a few series with
// every piece of scratch memory taken from one fixed array in this file.
//
// Some callers cannot allocate device memory when they need a result: an
// application that has handed the whole device to its own allocator, or a
// latency-bound host thread for which the device-wide synchronisation of
// cudaMalloc/cudaFree is not acceptable.  This entry point runs the same
// counting and selection kernels as rqa_eps_for_rr but keeps their
// histograms, tables, work items and counters in g_scratch below, which
// exists from the moment the library is loaded on a device until the process
// exits.  Inputs and outputs are the caller's.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "rqa.h"
#include "rqa_common.cuh"

namespace rqa {
namespace {

constexpr int NA_MAX_S = RQA_NOALLOC_MAX_SERIES;
constexpr int NA_MAX_ITEMS_PER_SERIES = 1024;
// Cells of one work item at most: the counting kernels histogram an item in
// 32-bit shared bins, so an item of more cells could wrap a bin that holds
// most of its keys (a constant or heavily quantised series).
constexpr uint64_t NA_ITEM_CELLS_MAX = (uint64_t)1 << 30;
constexpr int NA_KMAX = RQA_NOALLOC_K_MAX;  // targets per call here (one middle-round launch)
static_assert(NA_KMAX < MID_GROUPS && NA_KMAX >= NSUB_MAX, "fixed-scratch layout assumptions");

// Layout of the fixed scratch array (byte offsets, 256-aligned blocks).
constexpr size_t al(size_t x) { return (x + 255) & ~size_t(255); }
constexpr int64_t NA_HSTRIDE = NCOARSE + (int64_t)NA_KMAX * NFINE;  // NA_KMAX >= NSUB_MAX
constexpr size_t O_STATUS = 0;
constexpr size_t O_QUEUE = O_STATUS + 256;
constexpr size_t O_SERIES = O_QUEUE + 256;
constexpr size_t O_T = O_SERIES + al(sizeof(SeriesDev) * NA_MAX_S);
constexpr size_t O_ITEMS = O_T + al(sizeof(uint64_t) * NA_MAX_S * NA_KMAX);
constexpr size_t O_PREFIX = O_ITEMS + al(sizeof(Item) * NA_MAX_S * NA_MAX_ITEMS_PER_SERIES);
constexpr size_t O_LEVEL = O_PREFIX + al(sizeof(uint32_t) * NA_MAX_S * NA_KMAX);
constexpr size_t O_RANK = O_LEVEL + al(sizeof(uint8_t) * NA_MAX_S * NA_KMAX);
constexpr size_t O_BELOW = O_RANK + al(sizeof(uint64_t) * NA_MAX_S * NA_KMAX);
constexpr size_t O_TSUB = O_BELOW + al(sizeof(uint64_t) * NA_MAX_S * NA_KMAX);
constexpr size_t O_TMID = O_TSUB + al((size_t)NA_MAX_S * NCOARSE);
constexpr size_t O_TFIN1 = O_TMID + al((size_t)NA_MAX_S * NCOARSE);
constexpr size_t O_TFIN2 = O_TFIN1 + al((size_t)NA_MAX_S * NCOARSE);
constexpr size_t O_NGROUPS = O_TFIN2 + al((size_t)NA_MAX_S * NA_KMAX * NFINE);
constexpr size_t O_RANGE = O_NGROUPS + al(sizeof(int32_t) * 3 * NA_MAX_S);
constexpr size_t O_REDO = O_RANGE + al(sizeof(uint32_t) * 2 * NA_MAX_S);
constexpr size_t O_HIST = O_REDO + 256;
constexpr size_t NA_BYTES = O_HIST + al(sizeof(uint64_t) * NA_HSTRIDE * NA_MAX_S);
static_assert(NA_BYTES <= (size_t)RQA_NOALLOC_SCRATCH_BYTES, "scratch layout exceeds its array");

// The scratch itself: shared by every call on a device.  In host code this
// name is only a stand-in for the device array; kernels get the address that
// cudaGetSymbolAddress returns for the current device.
static __device__ __align__(256) unsigned char g_scratch[RQA_NOALLOC_SCRATCH_BYTES];

struct NaPlan {
    int S, K;
    SeriesDev sd[NA_MAX_S];
    uint64_t T[NA_MAX_S][NA_KMAX];
    int chunk[NA_MAX_S];       // bands per work item
    int item_begin[NA_MAX_S + 1];
};

// Per-device set-up: the device address of g_scratch and the SM count.
struct NaDevice {
    unsigned char *scratch = nullptr;
    int sm_count = 0;
};
constexpr int NA_MAX_DEVICES = 64;
NaDevice g_dev[NA_MAX_DEVICES];
std::mutex g_dev_mu;

// A pointer the kernels dereference must be memory the current device can
// address: its own device memory, or managed memory.
bool na_device_ptr(const void *p, int device)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    return at.type == cudaMemoryTypeDevice && at.device == device;
}

int na_setup(int device, NaDevice &out)
{
    std::lock_guard<std::mutex> lock(g_dev_mu);
    NaDevice &d = g_dev[device];
    if (!d.scratch) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return RQA_ERR_CUDA;
        }
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
            cudaGetLastError();
            return RQA_ERR_CUDA;
        }
        d.scratch = static_cast<unsigned char *>(p);
        d.sm_count = sms;
    }
    out = d;
    return RQA_OK;
}

// Writes the plan into the scratch and clears what must start at zero: the
// status word, the work-queue tickets and the group counts.  The counting
// histograms are cleared before each round and the selection tables by the
// select kernels themselves, as in rqa_eps_for_rr.
__global__ void k_na_setup(NaPlan pl, unsigned char *scr)
{
    SeriesDev *sd = reinterpret_cast<SeriesDev *>(scr + O_SERIES);
    uint64_t *T = reinterpret_cast<uint64_t *>(scr + O_T);
    Item *items = reinterpret_cast<Item *>(scr + O_ITEMS);
    const int t = threadIdx.x;
    if (t == 0) *reinterpret_cast<int *>(scr + O_STATUS) = 0;
    if (t < 64) reinterpret_cast<unsigned *>(scr + O_QUEUE)[t] = 0u;
    if (t < 3 * NA_MAX_S) reinterpret_cast<int32_t *>(scr + O_NGROUPS)[t] = 0;
    if (t < NA_MAX_S) scr[O_REDO + t] = 1;  // the plain coarse round for every series
    for (int s = 0; s < pl.S; ++s) {
        if (t == 0) sd[s] = pl.sd[s];
        if (t < pl.K) T[s * pl.K + t] = pl.T[s][t];
        const int n_it = pl.item_begin[s + 1] - pl.item_begin[s];
        for (int i = t; i < n_it; i += blockDim.x) {
            Item it;
            it.s = s;
            it.b_lo = i * pl.chunk[s];
            it.b_hi = min((i + 1) * pl.chunk[s], pl.sd[s].nbands);
            it.pad = 0;
            items[pl.item_begin[s] + i] = it;
        }
    }
}

__global__ void k_na_status(const unsigned char *scr, int *status_out)
{
    *status_out = *reinterpret_cast<const int *>(scr + O_STATUS);
}

}  // namespace
}  // namespace rqa

using namespace rqa;

extern "C" int rqa_eps_for_rr_noalloc(const rqa_batch *b, const int32_t *rr_num, int32_t rr_den,
                                      int32_t K, float *eps_out, uint64_t *count_le,
                                      uint64_t *count_lt, int *status_out, void *stream)
{
    // ---- host-side checks (nothing is enqueued if one fails)
    if (!b || !b->y || !b->offsets || !b->m || !b->tau || !eps_out || !rr_num)
        return RQA_ERR_INVALID_ARG;
    if (b->n_series < 1) return RQA_ERR_INVALID_ARG;
    if (b->n_series > NA_MAX_S) return RQA_ERR_CAPACITY;
    if (K < 1 || K > NA_KMAX || rr_den < 2 || b->offsets[0] != 0) return RQA_ERR_INVALID_ARG;
    for (int k = 0; k < K; ++k)
        if (rr_num[k] < 1 || rr_num[k] >= rr_den || (k && rr_num[k] <= rr_num[k - 1]))
            return RQA_ERR_INVALID_ARG;
    NaPlan pl;
    std::memset(&pl, 0, sizeof(pl));
    pl.S = b->n_series;
    pl.K = K;
    int n_items = 0;
    for (int s = 0; s < pl.S; ++s) {
        const int64_t n = b->offsets[s + 1] - b->offsets[s];
        if (n < 0 || b->m[s] < 1 || b->m[s] > RQA_M_MAX || b->tau[s] < 1) return RQA_ERR_INVALID_ARG;
        if (n > (int64_t)0x7fffffff - 64) return RQA_ERR_CAPACITY;
        const int64_t ne = n - (int64_t)(b->m[s] - 1) * b->tau[s];
        if (ne < 2) return RQA_ERR_TOO_SHORT;
        if (ne > RQA_NOALLOC_NE_MAX) return RQA_ERR_CAPACITY;
        SeriesDev &d = pl.sd[s];
        d.off = b->offsets[s];
        d.n = (int32_t)n;
        d.m = b->m[s];
        d.tau = b->tau[s];
        d.ne = (int32_t)ne;
        d.P = (uint64_t)ne * (uint64_t)(ne - 1) / 2;
        d.nbands = (int32_t)((ne - 1 + BAND - 1) / BAND);
        if (rqa_target_counts(d.P, rr_num, rr_den, K, pl.T[s]) != RQA_OK) return RQA_ERR_INVALID_ARG;
        // at least ITEM_MIN_BANDS bands (1024 diagonals) per item, at most
        // NA_MAX_ITEMS_PER_SERIES items
        int chunk = ITEM_MIN_BANDS;
        while ((d.nbands + chunk - 1) / chunk > NA_MAX_ITEMS_PER_SERIES) chunk *= 2;
        // the largest item is the first (the longest diagonals 1..chunk*BAND);
        // every Ne up to RQA_NOALLOC_NE_MAX passes, this guards the invariant
        const int64_t dl = std::min<int64_t>((int64_t)chunk * BAND, ne - 1);
        if ((uint64_t)(dl * ne - dl * (dl + 1) / 2) > NA_ITEM_CELLS_MAX) return RQA_ERR_CAPACITY;
        pl.chunk[s] = chunk;
        pl.item_begin[s] = n_items;
        n_items += (d.nbands + chunk - 1) / chunk;
    }
    pl.item_begin[pl.S] = n_items;

    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess || device < 0 || device >= NA_MAX_DEVICES) {
        cudaGetLastError();
        return RQA_ERR_CUDA;
    }
    if (!na_device_ptr(b->y, device) || !na_device_ptr(eps_out, device) ||
        (count_le && !na_device_ptr(count_le, device)) || (count_lt && !na_device_ptr(count_lt, device)) ||
        (status_out && !na_device_ptr(status_out, device)))
        return RQA_ERR_INVALID_ARG;
    NaDevice dv;
    if (int rc = na_setup(device, dv)) return rc;
    unsigned char *scr = dv.scratch;
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    // ---- the selection, as rqa_eps_for_rr runs it, on the fixed scratch
    int embed = E_GENERIC;
    {
        bool um = true, ut = true;
        for (int s = 1; s < pl.S; ++s) {
            um &= pl.sd[s].m == pl.sd[0].m;
            ut &= pl.sd[s].tau == pl.sd[0].tau;
        }
        const int m0 = pl.sd[0].m, t0 = pl.sd[0].tau;
        if (um && m0 <= 4) embed = m0;
        if (um && m0 == 1) embed = E_M1T1;
        if (um && ut && m0 == 3 && t0 == 1) embed = E_M3T1;
        if (um && ut && m0 == 3 && t0 == 3) embed = E_M3T3;
    }
    k_na_setup<<<1, 256, 0, st>>>(pl, scr);
    if (cudaGetLastError() != cudaSuccess) return RQA_ERR_CUDA;
    int *status = reinterpret_cast<int *>(scr + O_STATUS);
    if (launch_check_finite(b->y, b->offsets[pl.S], status, st) != cudaSuccess) return RQA_ERR_CUDA;

    SelBufs sb{};  // no hashed final-round table here: tab_hash = hash_mul = null
    sb.T = reinterpret_cast<const uint64_t *>(scr + O_T);
    sb.prefix = reinterpret_cast<uint32_t *>(scr + O_PREFIX);
    sb.level = reinterpret_cast<uint8_t *>(scr + O_LEVEL);
    sb.rank = reinterpret_cast<uint64_t *>(scr + O_RANK);
    sb.below = reinterpret_cast<uint64_t *>(scr + O_BELOW);
    sb.tab_sub = reinterpret_cast<int8_t *>(scr + O_TSUB);
    sb.tab_mid = reinterpret_cast<int8_t *>(scr + O_TMID);
    sb.tab_fin1 = reinterpret_cast<int8_t *>(scr + O_TFIN1);
    sb.tab_fin2 = reinterpret_cast<int8_t *>(scr + O_TFIN2);
    sb.fin2_stride = (int64_t)NA_KMAX * NFINE;
    int32_t *ng = reinterpret_cast<int32_t *>(scr + O_NGROUPS);
    sb.n_sub = ng;
    sb.n_mid = ng + pl.S;
    sb.n_fin = ng + 2 * pl.S;
    sb.range = reinterpret_cast<uint32_t *>(scr + O_RANGE);
    sb.redo = scr + O_REDO;
    sb.hist = reinterpret_cast<uint64_t *>(scr + O_HIST);
    sb.hstride = NCOARSE + (int64_t)(K > NSUB_MAX ? K : NSUB_MAX) * NFINE;

    CellArgs a{};
    a.y = b->y;
    a.series = reinterpret_cast<const SeriesDev *>(scr + O_SERIES);
    a.items = reinterpret_cast<const Item *>(scr + O_ITEMS);
    a.n_items = n_items;
    a.band = BAND;
    a.g0 = 0;
    a.gn = MID_GROUPS;  // K <= NA_KMAX < MID_GROUPS: one middle-round launch
    a.status = status;
    const int grid = (int)(n_items < dv.sm_count * 2 ? n_items : dv.sm_count * 2);
    const int rounds[3] = {R_COARSE, R_MID, R_FINAL};
    unsigned *queue = reinterpret_cast<unsigned *>(scr + O_QUEUE);
    for (int r = 0; r < 3; ++r) {
        if (cudaMemsetAsync(sb.hist, 0, sizeof(uint64_t) * sb.hstride * pl.S, st) != cudaSuccess) {
            cudaGetLastError();
            return RQA_ERR_CUDA;
        }
        a.queue = queue + 16 * r;
        if (launch_count(rounds[r], a, sb, K, grid < 1 ? 1 : grid, embed, st) != cudaSuccess)
            return RQA_ERR_CUDA;
        if (launch_select(rounds[r], sb, a.series, 0, pl.S, K, eps_out, count_le, count_lt, status,
                          st) != cudaSuccess)
            return RQA_ERR_CUDA;
    }
    if (status_out) {
        k_na_status<<<1, 1, 0, st>>>(scr, status_out);
        if (cudaGetLastError() != cudaSuccess) return RQA_ERR_CUDA;
    }
    return RQA_OK;
}
