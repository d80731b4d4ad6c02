// Host side of librqa: argument validation, work planning and the launch
// sequences behind the C ABI declared in include/rqa.h.
#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "rqa.h"
#include "rqa_learn.h"
#include "rqa_learn_internal.h"
#include "rqa_common.cuh"

using namespace rqa;

namespace {

struct DevBuf {
    void *p = nullptr;
    size_t cap = 0;
};

std::atomic<uint64_t> g_realloc_events{0};  // any scratch reallocation (graphs capture pointers)

int ensure(DevBuf &b, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    if (bytes <= b.cap) return RQA_OK;
    ++g_realloc_events;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.cap = 0;
    if (cudaMalloc(&b.p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return RQA_ERR_OOM;
    }
    b.cap = bytes;
    return RQA_OK;
}

template <class T>
T *P(DevBuf &b) { return reinterpret_cast<T *>(b.p); }

size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

}  // namespace

struct rqa_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int schedule = RQA_SCHED_BATCHED;
    int select = RQA_SELECT_AUTO;
    int band = 16;          // diagonals per band of the counting rounds
    int line_tile = 0;      // diagonals per register window of the line pass (0 = default)
    int unit_bands = 0;     // bands per line-pass work unit (0 = planned)
    int line_ctas = 0;      // persistent line-pass CTAs per SM (0 = all that fit)
    int line_stage = 0;     // line pass: series windows staged by bulk copies (1) or read per lane (0)
    float tuned_ms = 0.f;   // line-pass time of the last rqa_autotune choice
    bool tile_fixed = false;  // the caller chose the tile: rqa_autotune keeps it
    bool loi = false;         // RQA_FLAG_LOI: rates and DET over the whole matrix
    int bpsm = 0;
    int sm_count = 0;

    // scratch (grow-only)
    DevBuf arena;      // uploaded plan: series, targets, items, lmin, hist offsets
    DevBuf prefix, level, rank, below, tab_sub, tab_mid, tab_fin1, tab_fin2, tab_hash, ngroups, hist, krange,
        redo;
    DevBuf queue, status;
    DevBuf eps_tmp, le_tmp, lt_tmp, count, lmax, hshort;
    DevBuf meas;  // per-target L / ENTR when only their averages are asked for
    DevBuf grid_thr, grid_hist, grid_rr;  // the approximate grid search

    // learned bracket
    DevBuf mlp;                 // installed network parameters
    bool has_model = false;
    std::vector<int32_t> dom_m, dom_tau;  // embeddings the network was trained on (empty: any)
    float margin = 0.f;
    DevBuf feats, centre, ymlp, acts, bstats, learn_scratch;
    uint64_t sketch_seed = 1;

    // graph of the last rqa_det_avg call and its argument signature
    bool graphs = true;
    bool graph_valid = false;
    std::vector<uint64_t> graph_sig;
    cudaGraphExec_t graph_exec = nullptr;
    uint64_t graph_launches = 0;  // kernels in the graph
    uint64_t graph_replays = 0;
    uint64_t alloc_gen = 0;       // bumped whenever a scratch buffer moves

    // per-phase timing of the last call (batched schedule)
    bool timing = false;
    cudaEvent_t ev[7] = {};
    bool ev_recorded = false;
    uint64_t launches = 0;

    // pinned host staging of the plan upload
    void *h_stage = nullptr;
    size_t h_cap = 0;
    cudaEvent_t stage_done = nullptr;
    bool stage_pending = false;
};

namespace {

struct Plan {
    const float *y = nullptr;   // the batch's device buffer
    int S = 0, K = 0;
    int mt = 0;                 // Embed code of the batch (distance kernel variant)
    int64_t total = 0;          // values in the batch buffer
    std::vector<SeriesDev> sd;
    std::vector<uint64_t> T;    // S*K (empty if no targets)
    std::vector<Item> items_lpt;             // whole batch, largest first
    std::vector<Item> items_ser;             // grouped by series
    std::vector<int> ser_begin;              // S+1 into items_ser
    std::vector<int32_t> order;              // series by size, largest first
    std::vector<int64_t> uprefix;            // S+1 unit-count prefix along order
    int32_t chunk = 1;                       // bands per line-pass unit (batched)
    int32_t line_tile = LINE_TILE_DEFAULT;   // diagonals per register window of the line pass
    int32_t ne_max = 0;                      // largest Ne of the batch
    std::vector<int32_t> ident;              // 0..S-1
    std::vector<int64_t> uprefix1;           // [2s], [2s+1] = 0, units of s alone
    std::vector<int32_t> chunk1;             // bands per unit of s alone
    std::vector<uint8_t> dom;                // 1: the series may be bracketed
    bool any_dom = false;
    // device pointers into the arena after upload
    SeriesDev *d_sd = nullptr;
    uint64_t *d_T = nullptr;
    Item *d_lpt = nullptr;
    Item *d_ser = nullptr;
    int32_t *d_order = nullptr, *d_ident = nullptr;
    int64_t *d_uprefix = nullptr, *d_uprefix1 = nullptr;
    int32_t *d_lmin = nullptr;
    int64_t *d_hoff = nullptr;
    uint8_t *d_dom = nullptr;
};

int check_cuda(cudaError_t e)
{
    if (e == cudaSuccess) return RQA_OK;
    cudaGetLastError();
    return RQA_ERR_CUDA;
}

// A kernel launch through one of the launch wrappers: counted per context.
int launched(rqa_ctx *c, cudaError_t e)
{
    c->launches++;
    return check_cuda(e);
}

// Phase boundary i (0..6) of the timed sequence.
void mark(rqa_ctx *c, int i)
{
    if (c->timing && c->schedule == RQA_SCHED_BATCHED) {
        // "external": inside a stream capture this becomes an event-record node
        // of the graph, so replays record the phase boundaries too
        cudaEventRecordWithFlags(c->ev[i], c->stream, cudaEventRecordExternal);
        if (i == 6) c->ev_recorded = true;
    }
}

uint64_t band_cost(int64_t ne, int64_t d_lo, int64_t d_hi)
{
    // sum_{delta = d_lo}^{d_hi - 1} (ne - delta)
    const int64_t n = d_hi - d_lo;
    return (uint64_t)(n * ne - (d_lo + d_hi - 1) * n / 2);
}

void build_items(const SeriesDev &s, int sidx, int band, uint64_t target, int min_bands,
                 std::vector<Item> &out, std::vector<uint64_t> *costs)
{
    Item cur{sidx, 0, 0, 0};
    uint64_t acc = 0;
    for (int b = 0; b < s.nbands; ++b) {
        const int64_t d_lo = 1 + (int64_t)b * band;
        const int64_t d_hi = std::min<int64_t>(d_lo + band, s.ne);
        acc += band_cost(s.ne, d_lo, d_hi);
        cur.b_hi = b + 1;
        const bool enough = acc >= target && cur.b_hi - cur.b_lo >= min_bands &&
                            s.nbands - cur.b_hi >= min_bands;
        if (enough || acc >= ((uint64_t)1 << 30) || b + 1 == s.nbands) {
            out.push_back(cur);
            if (costs) costs->push_back(acc);
            cur.b_lo = b + 1;
            acc = 0;
        }
    }
}

int validate_batch(const rqa_batch *b)
{
    if (!b || !b->y || !b->offsets || !b->m || !b->tau || b->n_series < 1)
        return RQA_ERR_INVALID_ARG;
    if (b->offsets[0] != 0) return RQA_ERR_INVALID_ARG;
    for (int s = 0; s < b->n_series; ++s) {
        const int64_t n = b->offsets[s + 1] - b->offsets[s];
        if (n < 0) return RQA_ERR_INVALID_ARG;
        if (b->m[s] < 1 || b->m[s] > RQA_M_MAX || b->tau[s] < 1) return RQA_ERR_INVALID_ARG;
        if (n > (int64_t)0x7fffffff - 64) return RQA_ERR_CAPACITY;
        const int64_t ne = n - (int64_t)(b->m[s] - 1) * b->tau[s];
        if (ne < 2) return RQA_ERR_TOO_SHORT;
        if (ne > COUNT_NE_MAX) return RQA_ERR_CAPACITY;
    }
    return RQA_OK;
}

int validate_rr(const int32_t *rr_num, int32_t rr_den, int32_t K)
{
    if (!rr_num || K < 1 || K > RQA_K_MAX || rr_den < 2) return RQA_ERR_INVALID_ARG;
    for (int k = 0; k < K; ++k) {
        if (rr_num[k] < 1 || rr_num[k] >= rr_den) return RQA_ERR_INVALID_ARG;
        if (k && rr_num[k] <= rr_num[k - 1]) return RQA_ERR_INVALID_ARG;
    }
    return RQA_OK;
}

// Requested persistent grid: every item its CTA, at most blocks_per_sm per SM
// when the caller set it; the launchers further cap it at the CTAs the
// kernel can keep resident.
int persistent_grid(rqa_ctx *c, size_t n_items)
{
    const int bpsm = c->bpsm > 0 ? c->bpsm : 8;
    const size_t g = (size_t)c->sm_count * bpsm;
    return (int)std::max<size_t>(1, std::min(g, n_items));
}

int make_plan(rqa_ctx *c, const rqa_batch *b, const int32_t *rr_num, int32_t rr_den, int K,
              Plan &pl)
{
    const int S = b->n_series;
    pl.y = b->y;
    pl.S = S;
    pl.K = K;
    pl.sd.resize(S);
    int m0 = b->m[0], t0 = b->tau[0];
    bool uniform = true, uniform_tau = true;
    uint64_t total_cells = 0;
    for (int s = 0; s < S; ++s) {
        SeriesDev &d = pl.sd[s];
        d.off = b->offsets[s];
        d.n = (int32_t)(b->offsets[s + 1] - b->offsets[s]);
        d.m = b->m[s];
        d.tau = b->tau[s];
        d.ne = d.n - (d.m - 1) * d.tau;
        d.P = (uint64_t)d.ne * (uint64_t)(d.ne - 1) / 2;
        d.nbands = (d.ne - 1 + c->band - 1) / c->band;
        d.pad = 0;
        uniform &= (d.m == m0);
        uniform_tau &= (d.tau == t0);
        total_cells += d.P;
    }
    pl.total = b->offsets[S];
    // series the learned bracket may take: any when the bracket is forced or
    // the network's domain is unrestricted, else those with a trained embedding
    pl.dom.assign(S, 1);
    if (c->select != RQA_SELECT_BRACKET && !c->dom_m.empty())
        for (int s = 0; s < S; ++s) {
            bool in = false;
            for (size_t i = 0; i < c->dom_m.size() && !in; ++i)
                in = c->dom_m[i] == b->m[s] && c->dom_tau[i] == b->tau[s];
            pl.dom[s] = in ? 1 : 0;
        }
    pl.any_dom = false;
    for (int s = 0; s < S; ++s) pl.any_dom |= pl.dom[s] != 0;
    pl.mt = E_GENERIC;
    if (uniform && m0 <= 4) pl.mt = m0;
    if (uniform && m0 == 1) pl.mt = E_M1T1;  // tau plays no part when m = 1
    if (uniform && uniform_tau) {
        if (m0 == 3 && t0 == 1) pl.mt = E_M3T1;
        if (m0 == 3 && t0 == 3) pl.mt = E_M3T3;
    }
    if (rr_num) {
        pl.T.resize((size_t)S * K);
        for (int s = 0; s < S; ++s) {
            uint64_t *T = &pl.T[(size_t)s * K];
            if (rqa_target_counts(pl.sd[s].P, rr_num, rr_den, K, T) != RQA_OK)
                return RQA_ERR_INVALID_ARG;
            if (c->loi)  // whole matrix: 2 C + Ne >= ceil(rr Ne^2 / den)
                if (rqa_target_counts_loi((uint64_t)pl.sd[s].ne, rr_num, rr_den, K, T) != RQA_OK)
                    return RQA_ERR_INVALID_ARG;
        }
    }
    // CTA work items (counting rounds): runs of consecutive bands of one
    // series, about three per persistent CTA and at least four bands per warp,
    // sorted largest first.  Per series: the same rule within the series.
    const uint64_t ctas = (uint64_t)c->sm_count * 2;
    const uint64_t cap = (uint64_t)1 << 30;  // keeps 32-bit shared counters exact
    uint64_t tgt = std::max<uint64_t>(total_cells / (ctas * 3), 1);
    tgt = std::min(tgt, cap);
    std::vector<Item> items;
    std::vector<uint64_t> costs;
    for (int s = 0; s < S; ++s) build_items(pl.sd[s], s, c->band, tgt, ITEM_MIN_BANDS, items, &costs);
    std::vector<size_t> idx(items.size());
    for (size_t i = 0; i < idx.size(); ++i) idx[i] = i;
    std::stable_sort(idx.begin(), idx.end(), [&](size_t x, size_t y) { return costs[x] > costs[y]; });
    pl.items_lpt.resize(items.size());
    for (size_t i = 0; i < idx.size(); ++i) pl.items_lpt[i] = items[idx[i]];
    pl.ser_begin.assign(S + 1, 0);
    for (int s = 0; s < S; ++s) {
        uint64_t t = std::min(std::max<uint64_t>(pl.sd[s].P / (ctas * 3), 1), cap);
        build_items(pl.sd[s], s, c->band, t, ITEM_MIN_BANDS, pl.items_ser, nullptr);
        pl.ser_begin[s + 1] = (int)pl.items_ser.size();
    }
    // warp work units (line pass): runs of `chunk` bands of LINE_BAND
    // diagonals, series largest first; about eight units per warp so the tail
    // stays short while each unit's histogram flush is spread over many cells.
    // A unit covers at most 2^33 cells, so the warp's 32-bit counts of lines of
    // length >= 4 (each line and the cell after it: >= 5 cells) stay exact.
    const int64_t n_warps = (int64_t)c->sm_count * 16;  // resident warps of the line pass
    for (int s = 0; s < S; ++s) pl.ne_max = std::max(pl.ne_max, pl.sd[s].ne);
    const int64_t chunk_cap = std::max<int64_t>(1, ((int64_t)1 << 28) / std::max(pl.ne_max, 1));
    auto chunk_for = [&](int64_t bands) {
        int64_t ch = std::max<int64_t>(1, std::min<int64_t>(64, bands / (n_warps * 8)));
        if (c->unit_bands > 0) ch = c->unit_bands;  // a tuned size
        return (int32_t)std::min(ch, chunk_cap);
    };
    pl.line_tile = c->line_tile ? c->line_tile : LINE_TILE_DEFAULT;
    if (!lines_tile_ok(pl.mt, pl.line_tile)) pl.line_tile = LINE_TILE_DEFAULT;
    auto nbl = [&](int s) { return (int64_t)(pl.sd[s].ne - 1 + LINE_BAND - 1) / LINE_BAND; };
    int64_t total_bands = 0;
    for (int s = 0; s < S; ++s) total_bands += nbl(s);
    pl.chunk = chunk_for(total_bands);
    pl.order.resize(S);
    for (int s = 0; s < S; ++s) pl.order[s] = s;
    std::stable_sort(pl.order.begin(), pl.order.end(),
                     [&](int x, int y) { return pl.sd[x].P > pl.sd[y].P; });
    pl.uprefix.assign(S + 1, 0);
    for (int i = 0; i < S; ++i)
        pl.uprefix[i + 1] = pl.uprefix[i] + (nbl(pl.order[i]) + pl.chunk - 1) / pl.chunk;
    pl.ident.resize(S);
    pl.uprefix1.resize(2 * (size_t)S);
    pl.chunk1.resize(S);
    for (int s = 0; s < S; ++s) {
        pl.ident[s] = s;
        pl.chunk1[s] = chunk_for(nbl(s));
        pl.uprefix1[2 * s] = 0;
        pl.uprefix1[2 * s + 1] = (nbl(s) + pl.chunk1[s] - 1) / pl.chunk1[s];
    }
    return RQA_OK;
}

// Copy the plan (and optional lmin list / histogram offsets) to the device.
int upload_plan(rqa_ctx *c, Plan &pl, const int32_t *lmin, int n_lmin, const int64_t *hoff)
{
    const size_t o_sd = 0;
    const size_t o_T = align16(o_sd + pl.sd.size() * sizeof(SeriesDev));
    const size_t o_lpt = align16(o_T + pl.T.size() * sizeof(uint64_t));
    const size_t o_ser = align16(o_lpt + pl.items_lpt.size() * sizeof(Item));
    const size_t o_order = align16(o_ser + pl.items_ser.size() * sizeof(Item));
    const size_t o_upre = align16(o_order + pl.order.size() * sizeof(int32_t));
    const size_t o_ident = align16(o_upre + pl.uprefix.size() * sizeof(int64_t));
    const size_t o_upre1 = align16(o_ident + pl.ident.size() * sizeof(int32_t));
    const size_t o_lmin = align16(o_upre1 + pl.uprefix1.size() * sizeof(int64_t));
    const size_t o_hoff = align16(o_lmin + (size_t)n_lmin * sizeof(int32_t));
    const size_t o_dom = align16(o_hoff + (hoff ? (size_t)(pl.S + 1) * sizeof(int64_t) : 0));
    const size_t total = align16(o_dom + pl.dom.size());

    if (c->stage_pending) {
        if (cudaEventSynchronize(c->stage_done) != cudaSuccess) return check_cuda(cudaGetLastError());
        c->stage_pending = false;
    }
    if (total > c->h_cap) {
        if (c->h_stage) cudaFreeHost(c->h_stage);
        c->h_stage = nullptr;
        c->h_cap = 0;
        if (cudaHostAlloc(&c->h_stage, total, cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            return RQA_ERR_OOM;
        }
        c->h_cap = total;
    }
    if (int rc = ensure(c->arena, total)) return rc;
    c->graph_valid = false;  // the arena is about to hold another plan
    char *h = static_cast<char *>(c->h_stage);
    std::memcpy(h + o_sd, pl.sd.data(), pl.sd.size() * sizeof(SeriesDev));
    if (!pl.T.empty()) std::memcpy(h + o_T, pl.T.data(), pl.T.size() * sizeof(uint64_t));
    std::memcpy(h + o_lpt, pl.items_lpt.data(), pl.items_lpt.size() * sizeof(Item));
    std::memcpy(h + o_ser, pl.items_ser.data(), pl.items_ser.size() * sizeof(Item));
    std::memcpy(h + o_order, pl.order.data(), pl.order.size() * sizeof(int32_t));
    std::memcpy(h + o_upre, pl.uprefix.data(), pl.uprefix.size() * sizeof(int64_t));
    std::memcpy(h + o_ident, pl.ident.data(), pl.ident.size() * sizeof(int32_t));
    std::memcpy(h + o_upre1, pl.uprefix1.data(), pl.uprefix1.size() * sizeof(int64_t));
    if (n_lmin) std::memcpy(h + o_lmin, lmin, (size_t)n_lmin * sizeof(int32_t));
    if (hoff) std::memcpy(h + o_hoff, hoff, (size_t)(pl.S + 1) * sizeof(int64_t));
    std::memcpy(h + o_dom, pl.dom.data(), pl.dom.size());
    char *d = static_cast<char *>(c->arena.p);
    if (int rc = check_cuda(cudaMemcpyAsync(d, h, total, cudaMemcpyHostToDevice, c->stream))) return rc;
    if (int rc = check_cuda(cudaEventRecord(c->stage_done, c->stream))) return rc;
    c->stage_pending = true;
    pl.d_sd = reinterpret_cast<SeriesDev *>(d + o_sd);
    pl.d_T = reinterpret_cast<uint64_t *>(d + o_T);
    pl.d_lpt = reinterpret_cast<Item *>(d + o_lpt);
    pl.d_ser = reinterpret_cast<Item *>(d + o_ser);
    pl.d_order = reinterpret_cast<int32_t *>(d + o_order);
    pl.d_uprefix = reinterpret_cast<int64_t *>(d + o_upre);
    pl.d_ident = reinterpret_cast<int32_t *>(d + o_ident);
    pl.d_uprefix1 = reinterpret_cast<int64_t *>(d + o_upre1);
    pl.d_lmin = reinterpret_cast<int32_t *>(d + o_lmin);
    pl.d_hoff = reinterpret_cast<int64_t *>(d + o_hoff);
    pl.d_dom = reinterpret_cast<uint8_t *>(d + o_dom);
    return RQA_OK;
}

int64_t hist_stride(int K) { return NCOARSE + (int64_t)std::max(K, NSUB_MAX) * NFINE; }

int ensure_select_bufs(rqa_ctx *c, int S, int K)
{
    const size_t sk = (size_t)S * K;
    int rc = RQA_OK;
    if ((rc = ensure(c->prefix, sk * 4))) return rc;
    if ((rc = ensure(c->level, sk))) return rc;
    if ((rc = ensure(c->rank, sk * 8))) return rc;
    if ((rc = ensure(c->below, sk * 8))) return rc;
    if ((rc = ensure(c->tab_sub, (size_t)S * NCOARSE))) return rc;
    if ((rc = ensure(c->tab_mid, (size_t)S * NCOARSE))) return rc;
    if ((rc = ensure(c->tab_fin1, (size_t)S * NCOARSE))) return rc;
    if ((rc = ensure(c->tab_fin2, (size_t)S * KMAX * NFINE))) return rc;
    if ((rc = ensure(c->tab_hash, (size_t)S * NHASH * 4))) return rc;
    if ((rc = ensure(c->ngroups, (size_t)S * 4 * sizeof(int32_t)))) return rc;
    if ((rc = ensure(c->krange, (size_t)S * 2 * sizeof(uint32_t)))) return rc;
    if ((rc = ensure(c->redo, (size_t)S))) return rc;
    if ((rc = ensure(c->hist, (size_t)S * hist_stride(K) * 8))) return rc;
    if ((rc = ensure(c->eps_tmp, sk * 4))) return rc;
    if ((rc = ensure(c->le_tmp, sk * 8))) return rc;
    if ((rc = ensure(c->lt_tmp, sk * 8))) return rc;
    return RQA_OK;
}

SelBufs sel_bufs(rqa_ctx *c, const Plan &pl)
{
    SelBufs sb{};
    sb.T = pl.d_T;
    sb.prefix = P<uint32_t>(c->prefix);
    sb.level = P<uint8_t>(c->level);
    sb.rank = P<uint64_t>(c->rank);
    sb.below = P<uint64_t>(c->below);
    sb.tab_sub = P<int8_t>(c->tab_sub);
    sb.tab_mid = P<int8_t>(c->tab_mid);
    sb.tab_fin1 = P<int8_t>(c->tab_fin1);
    sb.tab_fin2 = P<int8_t>(c->tab_fin2);
    sb.fin2_stride = (int64_t)KMAX * NFINE;
    int32_t *ng = P<int32_t>(c->ngroups);
    sb.n_sub = ng;
    sb.n_mid = ng + pl.S;
    sb.n_fin = ng + 2 * pl.S;
    sb.tab_hash = P<uint32_t>(c->tab_hash);
    sb.hash_mul = reinterpret_cast<uint32_t *>(ng + 3 * pl.S);
    sb.hist = P<uint64_t>(c->hist);
    sb.hstride = hist_stride(pl.K);
    sb.range = P<uint32_t>(c->krange);
    sb.redo = P<uint8_t>(c->redo);
    return sb;
}


// Zero the queue tickets of n launches; returns the first ticket pointer.
// Counting launches of one selection (per series in the per-series
// schedule): bracket/coarse, middle rounds of MID_GROUPS groups, final.
int select_launches(int K) { return 3 + (K + MID_GROUPS - 1) / MID_GROUPS; }
// Line-pass launches: groups of at most LINE_KMAX targets.
int line_groups(int K) { return (K + LINE_KMAX - 1) / LINE_KMAX; }

int reset_queue(rqa_ctx *c, int n, unsigned **q)
{
    if (int rc = ensure(c->queue, (size_t)n * 64)) return rc;
    if (int rc = check_cuda(cudaMemsetAsync(c->queue.p, 0, (size_t)n * 64, c->stream))) return rc;
    *q = P<unsigned>(c->queue);
    return RQA_OK;
}

// Exact selection for series [s0, s0+ns) using the given item list: three
// counting rounds, the first one split by the learned bracket if asked.
int run_select(rqa_ctx *c, const Plan &pl, const SelBufs &sb, const Item *items, int n_items,
               int s0, int ns, unsigned *&q, float *eps, uint64_t *le, uint64_t *lt, bool bracket)
{
    const int K = pl.K;
    const int grid = persistent_grid(c, (size_t)n_items);
    CellArgs a{};
    a.y = pl.y;
    a.series = pl.d_sd;
    a.items = items;
    a.n_items = n_items;
    a.band = c->band;
    a.status = P<int>(c->status);
    const size_t hbytes = (size_t)ns * sb.hstride * 8;
    uint64_t *hbase = sb.hist + (int64_t)s0 * sb.hstride;
    if (bracket) {
        float *feats = P<float>(c->feats) + (int64_t)s0 * FEATURES;
        float *centre = P<float>(c->centre) + s0;
        float *ym = P<float>(c->ymlp) + (int64_t)s0 * MLP_OUT;
        if (int rc = launched(c, launch_sketch(pl.y, pl.d_sd, s0, ns, c->sketch_seed, feats, centre,
                                               nullptr, c->stream)))
            return rc;
        if (int rc = check_cuda(mlp_forward(P<float>(c->mlp), feats, ns, ym, P<float>(c->acts),
                                            c->stream)))
            return rc;
        c->launches += 3;
        if (int rc = launched(c, launch_bracket(ym, centre, c->margin, ns, K, pl.d_dom + s0,
                                                sb.tab_sub + (int64_t)s0 * NCOARSE, sb.n_sub + s0,
                                                sb.range + 2 * (int64_t)s0, c->stream)))
            return rc;
    } else {
        // plain selection: the coarse round runs for every series
        if (int rc = check_cuda(cudaMemsetAsync(sb.redo + s0, 1, (size_t)ns, c->stream))) return rc;
    }
    // bracket: split round, then the plain coarse round only for series with a
    // target outside its bracket; then the middle and final rounds
    const int rounds[4] = {R_COARSE_SUB, R_COARSE, R_MID, R_FINAL};
    for (int r = bracket ? 0 : 1; r < 4; ++r) {
        if (int rc = check_cuda(cudaMemsetAsync(hbase, 0, hbytes, c->stream))) return rc;
        // the middle round counts at most MID_GROUPS groups per launch
        for (int g0 = 0; g0 == 0 || (rounds[r] == R_MID && g0 < K); g0 += MID_GROUPS) {
            a.g0 = g0;
            a.gn = MID_GROUPS;
            a.queue = q;
            q += 16;
            if (int rc = launched(c, launch_count(rounds[r], a, sb, K, grid, pl.mt, c->stream)))
                return rc;
        }
        if (int rc = launched(c, launch_select(rounds[r], sb, pl.d_sd, s0, ns, K, eps, le, lt,
                                               P<int>(c->status), c->stream)))
            return rc;
        if (r == 0)
            if (int rc = launched(c, launch_bracket_stats(sb.level + (int64_t)s0 * K, pl.d_dom + s0, ns, K,
                                                          P<unsigned long long>(c->bstats), c->stream)))
                return rc;
        if (r >= 1) mark(c, 1 + r);
    }
    return RQA_OK;
}

// Whether this call's targets are the ones the bracket network predicts.
bool rr_matches_model(const int32_t *rr_num, int32_t rr_den, int K)
{
    if (K != MLP_K || !rr_num) return false;
    for (int k = 0; k < K; ++k)
        if ((int64_t)rr_num[k] * 100 != (int64_t)(k + 1) * rr_den) return false;
    return true;
}

int ensure_bracket_bufs(rqa_ctx *c, int S)
{
    int rc = RQA_OK;
    if ((rc = ensure(c->feats, (size_t)S * FEATURES * 4))) return rc;
    if ((rc = ensure(c->centre, (size_t)S * 4))) return rc;
    if ((rc = ensure(c->ymlp, (size_t)S * MLP_OUT * 4))) return rc;
    if ((rc = ensure(c->acts, (size_t)S * 2 * HIDDEN * 4))) return rc;
    if ((rc = ensure(c->bstats, 16))) return rc;
    return RQA_OK;
}

int select_all(rqa_ctx *c, const rqa_batch *b, Plan &pl, float *eps, uint64_t *le, uint64_t *lt,
               bool bracket)
{
    const SelBufs sb = sel_bufs(c, pl);
    if (bracket) {
        if (int rc = ensure_bracket_bufs(c, pl.S)) return rc;
        if (int rc = check_cuda(cudaMemsetAsync(c->bstats.p, 0, 16, c->stream))) return rc;
    }
    mark(c, 0);
    if (int rc = launched(c, launch_check_finite(b->y, pl.total, P<int>(c->status), c->stream)))
        return rc;
    mark(c, 1);
    if (int rc = check_cuda(cudaMemsetAsync(c->ngroups.p, 0, (size_t)pl.S * 4 * sizeof(int32_t),
                                            c->stream)))
        return rc;
    unsigned *q = nullptr;
    if (c->schedule == RQA_SCHED_PER_SERIES) {
        if (int rc = reset_queue(c, select_launches(pl.K) * pl.S, &q)) return rc;
        for (int s = 0; s < pl.S; ++s) {
            const int ib = pl.ser_begin[s], ie = pl.ser_begin[s + 1];
            if (int rc = run_select(c, pl, sb, pl.d_ser + ib, ie - ib, s, 1, q, eps, le, lt, bracket))
                return rc;
        }
        return RQA_OK;
    }
    if (int rc = reset_queue(c, select_launches(pl.K), &q)) return rc;
    return run_select(c, pl, sb, pl.d_lpt, (int)pl.items_lpt.size(), 0, pl.S, q, eps, le, lt,
                      bracket);
}

int ensure_line_bufs(rqa_ctx *c, int S, int K)
{
    const size_t sk = (size_t)S * K;
    int rc = RQA_OK;
    if ((rc = ensure(c->count, sk * 8))) return rc;
    if ((rc = ensure(c->lmax, sk * 4))) return rc;
    if ((rc = ensure(c->hshort, sk * LSH * 8))) return rc;
    return RQA_OK;
}

// The line pass over every series; fills count / lmax / hshort (and hist).
int run_lines(rqa_ctx *c, const Plan &pl, const float *eps, uint64_t *hist, const int64_t *d_hoff,
              LineBufs &lb, bool vert = false)
{
    const int S = pl.S, K = pl.K;
    const size_t sk = (size_t)S * K;
    lb.eps = eps;
    lb.count = P<uint64_t>(c->count);
    lb.lmax = P<uint32_t>(c->lmax);
    lb.hshort = P<uint64_t>(c->hshort);
    lb.hist = hist;
    lb.hist_off = d_hoff;
    lb.kstride = K;
    lb.loi = vert && c->loi;  // only vertical lines run through the identity cells
    if (int rc = check_cuda(cudaMemsetAsync(lb.count, 0, sk * 8, c->stream))) return rc;
    if (int rc = check_cuda(cudaMemsetAsync(lb.lmax, 0, sk * 4, c->stream))) return rc;
    if (int rc = check_cuda(cudaMemsetAsync(lb.hshort, 0, sk * LSH * 8, c->stream))) return rc;
    CellArgs a{};
    a.y = pl.y;
    a.series = pl.d_sd;
    a.band = c->band;
    a.line_tile = pl.line_tile;
    a.line_ctas = c->line_ctas;
    a.line_stage = c->line_stage;
    a.y_len = pl.total;
    a.status = P<int>(c->status);
    unsigned *q = nullptr;
    const int full_grid = persistent_grid(c, (size_t)1 << 30);
    auto grid_for = [&](int64_t units) {
        return (int)std::max<int64_t>(1, std::min<int64_t>(full_grid, (units + WARPS - 1) / WARPS));
    };
    // targets in groups of at most LINE_KMAX (one lane each), one pass per group
    const int ng = line_groups(K), gsz = (K + ng - 1) / ng;
    auto launch_groups = [&]() -> int {
        for (int g = 0; g < ng; ++g) {
            lb.k0 = g * gsz;
            a.queue = q;
            q += 16;
            const int kg = std::min(gsz, K - lb.k0);
            const int grid = grid_for(a.n_units);
            if (int rc = launched(c, vert ? launch_vlines(a, lb, kg, grid, pl.mt, c->stream)
                                          : launch_lines(a, lb, kg, grid, pl.mt, c->stream)))
                return rc;
        }
        return RQA_OK;
    };
    int rc = RQA_OK;
    if (c->schedule == RQA_SCHED_PER_SERIES) {
        if ((rc = reset_queue(c, S * ng, &q))) return rc;
        for (int s = 0; s < S && rc == RQA_OK; ++s) {
            a.order = pl.d_ident + s;
            a.uprefix = pl.d_uprefix1 + 2 * (size_t)s;
            a.n_pos = 1;
            a.chunk = pl.chunk1[s];
            a.n_units = pl.uprefix1[2 * (size_t)s + 1];
            rc = launch_groups();
        }
    } else {
        if ((rc = reset_queue(c, ng, &q))) return rc;
        a.order = pl.d_order;
        a.uprefix = pl.d_uprefix;
        a.n_pos = S;
        a.chunk = pl.chunk;
        a.n_units = pl.uprefix[S];
        rc = launch_groups();
    }
    lb.k0 = 0;  // the finalisation kernels read all K targets
    return rc;
}

// Line pass plus the requested outputs.  hist/hoff come from the caller.
int lines_and_outputs(rqa_ctx *c, const Plan &pl, const float *eps, const rqa_line_outputs *lo,
                      LineBufs &lb)
{
    uint64_t *hist = lo ? lo->hist : nullptr;
    if (hist)
        if (int rc = check_cuda(cudaMemsetAsync(hist, 0, (size_t)lo->hist_offsets[pl.S] * 8, c->stream)))
            return rc;
    if (int rc = run_lines(c, pl, eps, hist, hist ? pl.d_hoff : nullptr, lb)) return rc;
    mark(c, 5);
    return RQA_OK;
}

int line_outputs_tail(rqa_ctx *c, const Plan &pl, const rqa_line_outputs *lo, LineBufs &lb)
{
    if (!lo) return RQA_OK;
    const size_t sk = (size_t)pl.S * pl.K;
    if (lo->hist || lo->stencil)
        if (int rc = launched(c, launch_finalize_hist(lb, pl.d_sd, pl.S, pl.K, lo->stencil, c->stream)))
            return rc;
    if (lo->lmax)
        if (int rc = check_cuda(cudaMemcpyAsync(lo->lmax, lb.lmax, sk * 4, cudaMemcpyDeviceToDevice,
                                                c->stream)))
            return rc;
    if (lo->count)
        if (int rc = check_cuda(cudaMemcpyAsync(lo->count, lb.count, sk * 8, cudaMemcpyDeviceToDevice,
                                                c->stream)))
            return rc;
    return RQA_OK;
}

int validate_hist(const rqa_batch *b, int K, const uint64_t *hist, const int64_t *hoff, int extra = 0)
{
    if (!hist) return RQA_OK;
    if (!hoff) return RQA_ERR_INVALID_ARG;
    if (hoff[0] != 0) return RQA_ERR_CAPACITY;
    for (int s = 0; s < b->n_series; ++s) {
        const int64_t ne = (b->offsets[s + 1] - b->offsets[s]) - (int64_t)(b->m[s] - 1) * b->tau[s];
        if (hoff[s + 1] - hoff[s] != (int64_t)K * (ne - 1 + extra)) return RQA_ERR_CAPACITY;
    }
    return RQA_OK;
}

// Selection mode of a call: bracket with a model and matching targets.
int use_bracket(rqa_ctx *c, const int32_t *rr_num, int32_t rr_den, int K, bool *out)
{
    *out = false;
    if (c->select == RQA_SELECT_RADIX) return RQA_OK;
    if (c->select == RQA_SELECT_BRACKET && !c->has_model) return RQA_ERR_NO_MODEL;
    const bool match = rr_matches_model(rr_num, rr_den, K);
    if (c->select == RQA_SELECT_BRACKET && !match) return RQA_ERR_INVALID_ARG;
    *out = c->has_model && match;
    return RQA_OK;
}

}  // namespace

// ====================================================================== ABI
extern "C" {

int rqa_abi_version(void) { return RQA_ABI_VERSION; }

const char *rqa_error_string(int code)
{
    switch (code) {
    case RQA_OK: return "ok";
    case RQA_ERR_INVALID_ARG: return "invalid argument";
    case RQA_ERR_TOO_SHORT: return "series too short (fewer than two embedded vectors)";
    case RQA_ERR_NONFINITE: return "series holds a non-finite value";
    case RQA_ERR_CUDA: return "CUDA runtime error";
    case RQA_ERR_OOM: return "out of device or pinned host memory";
    case RQA_ERR_TIMEOUT: return "a bounded device wait timed out";
    case RQA_ERR_CAPACITY: return "buffer too small or size limit exceeded";
    case RQA_ERR_UNSORTED: return "thresholds not ascending, negative or NaN";
    case RQA_ERR_NO_MODEL: return "bracket selection requested without a model";
    case RQA_ERR_INTERNAL: return "internal inconsistency in device counts";
    default: return "unknown error";
    }
}

int rqa_target_counts(uint64_t Pc, const int32_t *rr_num, int32_t rr_den, int32_t K,
                      uint64_t *T_out)
{
    if (!rr_num || !T_out || K < 1 || rr_den < 1 || Pc < 1) return RQA_ERR_INVALID_ARG;
    for (int k = 0; k < K; ++k) {
        if (rr_num[k] < 1 || rr_num[k] >= rr_den) return RQA_ERR_INVALID_ARG;
        const unsigned __int128 num = (unsigned __int128)(uint64_t)rr_num[k] * Pc;
        const unsigned __int128 t = (num + (unsigned __int128)(rr_den - 1)) / (unsigned)rr_den;
        T_out[k] = (uint64_t)t;
    }
    return RQA_OK;
}

int rqa_target_counts_loi(uint64_t ne, const int32_t *rr_num, int32_t rr_den, int32_t K,
                          uint64_t *T_out)
{
    if (!rr_num || !T_out || K < 1 || rr_den < 1 || ne < 2 || ne > ((uint64_t)1 << 32))
        return RQA_ERR_INVALID_ARG;
    for (int k = 0; k < K; ++k) {
        if (rr_num[k] < 1 || rr_num[k] >= rr_den) return RQA_ERR_INVALID_ARG;
        const unsigned __int128 n = ne;
        const unsigned __int128 full =
            ((unsigned __int128)(uint64_t)rr_num[k] * n * n + (unsigned)(rr_den - 1)) / (unsigned)rr_den;
        if (full <= n) return RQA_ERR_INVALID_ARG;  // the identity line alone reaches this rate
        T_out[k] = (uint64_t)((full - n + 1) / 2);
    }
    return RQA_OK;
}

int rqa_create(rqa_ctx **out, const rqa_config *cfg)
{
    if (!out) return RQA_ERR_INVALID_ARG;
    *out = nullptr;
    rqa_config def;
    std::memset(&def, 0, sizeof(def));
    if (!cfg) cfg = &def;
    for (int i = 0; i < 3; ++i)
        if (cfg->reserved[i]) return RQA_ERR_INVALID_ARG;
    if (cfg->flags & ~(RQA_FLAG_NO_GRAPHS | RQA_FLAG_LOI)) return RQA_ERR_INVALID_ARG;
    if (cfg->schedule != RQA_SCHED_BATCHED && cfg->schedule != RQA_SCHED_PER_SERIES)
        return RQA_ERR_INVALID_ARG;
    if (cfg->select < RQA_SELECT_AUTO || cfg->select > RQA_SELECT_BRACKET) return RQA_ERR_INVALID_ARG;
    if (cfg->tile != 0 && cfg->tile != 8 && cfg->tile != 16 && cfg->tile != 32)
        return RQA_ERR_INVALID_ARG;
    if (cfg->blocks_per_sm < 0 || cfg->blocks_per_sm > 8) return RQA_ERR_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || cfg->device < 0 || cfg->device >= ndev) {
        cudaGetLastError();
        return RQA_ERR_CUDA;
    }
    if (cudaSetDevice(cfg->device) != cudaSuccess) return check_cuda(cudaGetLastError());
    rqa_ctx *c = new (std::nothrow) rqa_ctx;
    if (!c) return RQA_ERR_OOM;
    c->device = cfg->device;
    c->stream = static_cast<cudaStream_t>(cfg->stream);
    c->schedule = cfg->schedule;
    c->select = cfg->select;
    c->band = BAND;
    c->line_tile = cfg->tile;
    c->tile_fixed = cfg->tile != 0;
    c->graphs = !(cfg->flags & RQA_FLAG_NO_GRAPHS);
    c->loi = (cfg->flags & RQA_FLAG_LOI) != 0;
    c->bpsm = cfg->blocks_per_sm;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, c->device) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->stage_done, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return RQA_ERR_CUDA;
    }
    c->sm_count = prop.multiProcessorCount;
    if (ensure(c->status, 64) != RQA_OK || cudaMemset(c->status.p, 0, 64) != cudaSuccess) {
        cudaGetLastError();
        rqa_destroy(c);
        return RQA_ERR_OOM;
    }
    *out = c;
    return RQA_OK;
}

void rqa_destroy(rqa_ctx *c)
{
    if (!c) return;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    DevBuf *bufs[] = {&c->arena, &c->prefix, &c->level, &c->rank, &c->below, &c->tab_sub,
                      &c->tab_mid, &c->tab_fin1, &c->tab_fin2, &c->tab_hash, &c->ngroups, &c->hist,
                      &c->krange, &c->meas, &c->grid_thr, &c->grid_hist, &c->grid_rr,
                      &c->redo,
                      &c->queue,
                      &c->status, &c->eps_tmp, &c->le_tmp, &c->lt_tmp, &c->count, &c->lmax,
                      &c->hshort, &c->mlp, &c->feats, &c->centre, &c->ymlp, &c->acts,
                      &c->bstats, &c->learn_scratch};
    for (DevBuf *b : bufs)
        if (b->p) cudaFree(b->p);
    if (c->h_stage) cudaFreeHost(c->h_stage);
    if (c->stage_done) cudaEventDestroy(c->stage_done);
    for (int i = 0; i < 7; ++i)
        if (c->ev[i]) cudaEventDestroy(c->ev[i]);
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    cudaGetLastError();
    delete c;
}

int rqa_status(rqa_ctx *c)
{
    if (!c) return RQA_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return check_cuda(cudaGetLastError());
    int st = 0;
    if (cudaMemcpy(&st, c->status.p, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return check_cuda(cudaGetLastError());
    if (st) cudaMemset(c->status.p, 0, sizeof(int));
    return st;
}

int rqa_device_info(rqa_ctx *c, int *sm_count, int *tile, int *blocks_per_sm)
{
    if (!c) return RQA_ERR_INVALID_ARG;
    if (sm_count) *sm_count = c->sm_count;
    if (tile) *tile = c->line_tile ? c->line_tile : LINE_TILE_DEFAULT;
    if (blocks_per_sm) *blocks_per_sm = c->bpsm;  // 0: as many as each kernel keeps resident
    return RQA_OK;
}

int rqa_eps_for_rr(rqa_ctx *c, const rqa_batch *b, const int32_t *rr_num, int32_t rr_den,
                   int32_t K, float *eps_out, uint64_t *count_le, uint64_t *count_lt)
{
    if (!c || !eps_out) return RQA_ERR_INVALID_ARG;
    if (int rc = validate_batch(b)) return rc;
    if (int rc = validate_rr(rr_num, rr_den, K)) return rc;
    bool bracket = false;
    if (int rc = use_bracket(c, rr_num, rr_den, K, &bracket)) return rc;
    cudaSetDevice(c->device);
    Plan pl;
    if (int rc = make_plan(c, b, rr_num, rr_den, K, pl)) return rc;
    bracket = bracket && pl.any_dom;
    if (int rc = ensure_select_bufs(c, pl.S, K)) return rc;
    if (int rc = upload_plan(c, pl, nullptr, 0, nullptr)) return rc;
    return select_all(c, b, pl, eps_out, count_le, count_lt, bracket);
}

int rqa_det_avg(rqa_ctx *c, const rqa_batch *b, const int32_t *rr_num, int32_t rr_den,
                const float *eps, int32_t K, const int32_t *lmin, int32_t n_lmin, double *det_out,
                double *det_avg, float *eps_used, const rqa_line_outputs *lo)
{
    if (!c || !det_avg || !lmin || n_lmin < 1 || n_lmin > RQA_LMIN_MAX) return RQA_ERR_INVALID_ARG;
    if (K < 1 || K > RQA_K_MAX) return RQA_ERR_INVALID_ARG;
    for (int j = 0; j < n_lmin; ++j)
        if (lmin[j] < 1 || lmin[j] > LSH + 1) return RQA_ERR_INVALID_ARG;
    if (int rc = validate_batch(b)) return rc;
    if (lo)
        if (int rc = validate_hist(b, K, lo->hist, lo->hist_offsets)) return rc;
    bool bracket = false;
    if (!eps) {
        if (int rc = validate_rr(rr_num, rr_den, K)) return rc;
        if (int rc = use_bracket(c, rr_num, rr_den, K, &bracket)) return rc;
    }
    cudaSetDevice(c->device);
    Plan pl;
    if (int rc = make_plan(c, b, eps ? nullptr : rr_num, rr_den, K, pl)) return rc;
    if (pl.ne_max > LINE_NE_MAX) return RQA_ERR_CAPACITY;
    bracket = bracket && pl.any_dom;
    // every scratch buffer sized before anything is enqueued (and captured)
    if (int rc = ensure_line_bufs(c, pl.S, K)) return rc;
    if (!eps)
        if (int rc = ensure_select_bufs(c, pl.S, K)) return rc;
    if (bracket)
        if (int rc = ensure_bracket_bufs(c, pl.S)) return rc;
    if (int rc = ensure(c->queue, (size_t)(std::max(select_launches(K), line_groups(K)) * pl.S + 8) * 64))
        return rc;
    const int64_t *hoff = (lo && lo->hist) ? lo->hist_offsets : nullptr;

    // the call's signature: every argument the launch sequence depends on
    const bool use_graph = c->graphs && c->stream != nullptr;
    std::vector<uint64_t> sig;
    auto make_sig = [&]() {
        sig.clear();
        auto put = [&](uint64_t v) { sig.push_back(v); };
        auto ptr = [&](const void *p) { put((uint64_t)(uintptr_t)p); };
        put((uint64_t)pl.S); put((uint64_t)K); put((uint64_t)n_lmin); put((uint64_t)rr_den);
        put(bracket); put((uint64_t)c->schedule); put((uint64_t)pl.line_tile); put((uint64_t)c->unit_bands); put((uint64_t)c->line_ctas); put((uint64_t)c->line_stage); put(c->timing);
        for (int s = 0; s < pl.S; ++s) put(pl.dom[s]);
        put(c->loi);
        uint32_t mb;
        std::memcpy(&mb, &c->margin, 4);
        put(mb);
        put(g_realloc_events.load());
        ptr(b->y); ptr(eps); ptr(det_out); ptr(det_avg); ptr(eps_used);
        ptr(lo ? lo->hist : nullptr); ptr(lo ? lo->lmax : nullptr);
        ptr(lo ? lo->count : nullptr); ptr(lo ? lo->stencil : nullptr);
        for (int s = 0; s <= pl.S; ++s) put((uint64_t)b->offsets[s]);
        for (int s = 0; s < pl.S; ++s) put(((uint64_t)(uint32_t)b->m[s] << 32) | (uint32_t)b->tau[s]);
        for (int k = 0; !eps && k < K; ++k) put((uint64_t)rr_num[k]);
        for (int j = 0; j < n_lmin; ++j) put((uint64_t)lmin[j]);
        for (int s = 0; hoff && s <= pl.S; ++s) put((uint64_t)hoff[s]);
    };
    if (use_graph) {
        make_sig();
        if (c->graph_valid && c->graph_exec && sig == c->graph_sig) {
            if (int rc = check_cuda(cudaGraphLaunch(c->graph_exec, c->stream))) return rc;
            c->launches += c->graph_launches;
            c->graph_replays++;
            return RQA_OK;
        }
    }
    if (int rc = upload_plan(c, pl, lmin, n_lmin, hoff)) return rc;

    auto body = [&]() -> int {
        const float *e = eps;
        if (!eps) {
            if (int rc = select_all(c, b, pl, P<float>(c->eps_tmp), P<uint64_t>(c->le_tmp),
                                    P<uint64_t>(c->lt_tmp), bracket))
                return rc;
            e = P<float>(c->eps_tmp);
        } else {
            mark(c, 0);
            if (int rc = launched(c, launch_check_finite(b->y, pl.total, P<int>(c->status), c->stream)))
                return rc;
            for (int i = 1; i <= 4; ++i) mark(c, i);
        }
        LineBufs lb;
        if (int rc = lines_and_outputs(c, pl, e, lo, lb)) return rc;
        if (int rc = launched(c, launch_finalize_det(lb, pl.d_sd, pl.S, K, pl.d_lmin, n_lmin, det_out,
                                                     det_avg, c->loi, c->stream)))
            return rc;
        if (int rc = line_outputs_tail(c, pl, lo, lb)) return rc;
        mark(c, 6);
        if (eps_used)
            if (int rc = check_cuda(cudaMemcpyAsync(eps_used, e, (size_t)pl.S * K * 4,
                                                    cudaMemcpyDeviceToDevice, c->stream)))
                return rc;
        return RQA_OK;
    };
    if (!use_graph) return body();

    // record the sequence once, then launch the recording (and replay it for
    // identical calls); any failure falls back to launching directly
    const uint64_t l0 = c->launches;
    if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return body();
    }
    const int rc = body();
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(c->stream, &g);
    cudaGraphExec_t ex = nullptr;
    if (rc != RQA_OK || ec != cudaSuccess || !g || cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        c->launches = l0;
        return body();
    }
    cudaGraphDestroy(g);
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    c->graph_exec = ex;
    c->graph_launches = c->launches - l0;
    make_sig();  // after the upload, which may have moved the arena
    c->graph_sig = sig;
    c->graph_valid = true;
    return check_cuda(cudaGraphLaunch(ex, c->stream));
}

int rqa_line_hist(rqa_ctx *c, const rqa_batch *b, const float *eps, int32_t K, uint64_t *hist,
                  const int64_t *hist_offsets, uint32_t *lmax, uint64_t *count, uint64_t *stencil)
{
    if (!c || !eps || K < 1 || K > RQA_K_MAX) return RQA_ERR_INVALID_ARG;
    if (int rc = validate_batch(b)) return rc;
    if (int rc = validate_hist(b, K, hist, hist_offsets)) return rc;
    cudaSetDevice(c->device);
    Plan pl;
    if (int rc = make_plan(c, b, nullptr, 0, K, pl)) return rc;
    if (pl.ne_max > LINE_NE_MAX) return RQA_ERR_CAPACITY;
    if (int rc = ensure_line_bufs(c, pl.S, K)) return rc;
    if (int rc = upload_plan(c, pl, nullptr, 0, hist ? hist_offsets : nullptr)) return rc;
    mark(c, 0);
    if (int rc = launched(c, launch_check_finite(b->y, pl.total, P<int>(c->status), c->stream)))
        return rc;
    for (int i = 1; i <= 4; ++i) mark(c, i);
    rqa_line_outputs lo{hist, hist_offsets, lmax, count, stencil};
    LineBufs lb;
    if (int rc = lines_and_outputs(c, pl, eps, &lo, lb)) return rc;
    if (int rc = line_outputs_tail(c, pl, &lo, lb)) return rc;
    mark(c, 6);
    return RQA_OK;
}

int rqa_line_measures(rqa_ctx *c, const rqa_batch *b, int32_t K, const uint64_t *hist,
                      const int64_t *hist_offsets, const int32_t *lmin, int32_t n_lmin, double *L_out,
                      double *entr_out, double *L_avg, double *entr_avg)
{
    if (!c || !hist || !lmin || n_lmin < 1 || n_lmin > RQA_LMIN_MAX || K < 1 || K > RQA_K_MAX)
        return RQA_ERR_INVALID_ARG;
    for (int j = 0; j < n_lmin; ++j)
        if (lmin[j] < 1) return RQA_ERR_INVALID_ARG;
    if (int rc = validate_batch(b)) return rc;
    if (int rc = validate_hist(b, K, hist, hist_offsets)) return rc;
    if (!L_out && !entr_out && !L_avg && !entr_avg) return RQA_OK;
    cudaSetDevice(c->device);
    Plan pl;
    if (int rc = make_plan(c, b, nullptr, 0, K, pl)) return rc;
    const size_t n = (size_t)pl.S * K * n_lmin;
    double *L = L_out, *E = entr_out;
    if ((L_avg && !L) || (entr_avg && !E)) {
        if (int rc = ensure(c->meas, 2 * n * sizeof(double))) return rc;
        if (L_avg && !L) L = P<double>(c->meas);
        if (entr_avg && !E) E = P<double>(c->meas) + n;
    }
    if (int rc = upload_plan(c, pl, lmin, n_lmin, hist_offsets)) return rc;
    return launched(c, launch_line_measures(hist, pl.d_hoff, pl.S, K, pl.d_lmin, n_lmin, L, E, L_avg,
                                            entr_avg, c->loi, c->stream));
}

int rqa_vline_hist(rqa_ctx *c, const rqa_batch *b, const float *eps, int32_t K, uint64_t *vhist,
                   const int64_t *vhist_offsets, uint32_t *vmax, uint64_t *vmass)
{
    if (!c || !eps || K < 1 || K > RQA_K_MAX) return RQA_ERR_INVALID_ARG;
    if (int rc = validate_batch(b)) return rc;
    if (int rc = validate_hist(b, K, vhist, vhist_offsets, c->loi ? 1 : 0)) return rc;
    cudaSetDevice(c->device);
    // the vertical pass runs the default register window
    const int saved = c->line_tile;
    c->line_tile = LINE_TILE_DEFAULT;
    Plan pl;
    const int rcp = make_plan(c, b, nullptr, 0, K, pl);
    c->line_tile = saved;
    if (rcp) return rcp;
    if (pl.ne_max > LINE_NE_MAX) return RQA_ERR_CAPACITY;
    if (int rc = ensure_line_bufs(c, pl.S, K)) return rc;
    if (int rc = upload_plan(c, pl, nullptr, 0, vhist ? vhist_offsets : nullptr)) return rc;
    if (int rc = launched(c, launch_check_finite(b->y, pl.total, P<int>(c->status), c->stream)))
        return rc;
    if (vhist)
        if (int rc = check_cuda(cudaMemsetAsync(vhist, 0, (size_t)vhist_offsets[pl.S] * 8, c->stream)))
            return rc;
    LineBufs lb{};
    if (int rc = run_lines(c, pl, eps, vhist, vhist ? pl.d_hoff : nullptr, lb, true)) return rc;
    lb.loi = c->loi;
    if (vhist)
        if (int rc = launched(c, launch_finalize_hist(lb, pl.d_sd, pl.S, K, nullptr, c->stream)))
            return rc;
    const size_t sk = (size_t)pl.S * K;
    if (vmax)
        if (int rc = check_cuda(cudaMemcpyAsync(vmax, lb.lmax, sk * 4, cudaMemcpyDeviceToDevice, c->stream)))
            return rc;
    if (vmass)
        if (int rc = check_cuda(cudaMemcpyAsync(vmass, lb.count, sk * 8, cudaMemcpyDeviceToDevice, c->stream)))
            return rc;
    return RQA_OK;
}

int rqa_lam_tt(rqa_ctx *c, const rqa_batch *b, int32_t K, const uint64_t *vhist,
               const int64_t *vhist_offsets, const int32_t *vmin, int32_t n_vmin, double *lam_out,
               double *tt_out, double *lam_avg, double *tt_avg)
{
    if (!c || !vhist || !vmin || n_vmin < 1 || n_vmin > RQA_LMIN_MAX || K < 1 || K > RQA_K_MAX)
        return RQA_ERR_INVALID_ARG;
    for (int j = 0; j < n_vmin; ++j)
        if (vmin[j] < 1) return RQA_ERR_INVALID_ARG;
    if (int rc = validate_batch(b)) return rc;
    if (int rc = validate_hist(b, K, vhist, vhist_offsets, c->loi ? 1 : 0)) return rc;
    if (!lam_out && !tt_out && !lam_avg && !tt_avg) return RQA_OK;
    cudaSetDevice(c->device);
    Plan pl;
    if (int rc = make_plan(c, b, nullptr, 0, K, pl)) return rc;
    const size_t n = (size_t)pl.S * K * n_vmin;
    double *lam = lam_out, *tt = tt_out;
    if ((lam_avg && !lam) || (tt_avg && !tt)) {
        if (int rc = ensure(c->meas, 2 * n * sizeof(double))) return rc;
        if (lam_avg && !lam) lam = P<double>(c->meas);
        if (tt_avg && !tt) tt = P<double>(c->meas) + n;
    }
    if (int rc = upload_plan(c, pl, vmin, n_vmin, vhist_offsets)) return rc;
    return launched(c, launch_lam_tt(vhist, pl.d_hoff, pl.S, K, pl.d_lmin, n_vmin, lam, tt, lam_avg,
                                     tt_avg, c->stream));
}

int rqa_eps_approx(rqa_ctx *c, const rqa_batch *b, const int32_t *rr_num, int32_t rr_den, int32_t K,
                   int32_t n_thr, float *eps_out, double *rr_out, uint64_t *count_out)
{
    if (!c || !eps_out || n_thr < 1 || n_thr > 1024) return RQA_ERR_INVALID_ARG;
    if (int rc = validate_batch(b)) return rc;
    if (int rc = validate_rr(rr_num, rr_den, K)) return rc;
    cudaSetDevice(c->device);
    const bool loi = c->loi;
    c->loi = false;  // the grid search counts the upper triangle only
    Plan pl;
    const int rcp = make_plan(c, b, rr_num, rr_den, K, pl);
    c->loi = loi;
    if (rcp) return rcp;
    if (int rc = upload_plan(c, pl, nullptr, 0, nullptr)) return rc;
    if (int rc = ensure(c->grid_thr, (size_t)pl.S * n_thr * 4)) return rc;
    if (int rc = ensure(c->grid_hist, (size_t)pl.S * (n_thr + 1) * 8)) return rc;
    if (int rc = ensure(c->grid_rr, (size_t)K * 4)) return rc;
    if (int rc = check_cuda(cudaMemcpyAsync(c->grid_rr.p, rr_num, (size_t)K * 4, cudaMemcpyHostToDevice,
                                            c->stream)))
        return rc;
    if (int rc = check_cuda(cudaMemsetAsync(c->grid_hist.p, 0, (size_t)pl.S * (n_thr + 1) * 8, c->stream)))
        return rc;
    if (int rc = launched(c, launch_check_finite(b->y, pl.total, P<int>(c->status), c->stream)))
        return rc;
    unsigned *q = nullptr;
    if (int rc = reset_queue(c, 1, &q)) return rc;
    CellArgs a{};
    a.y = pl.y;
    a.series = pl.d_sd;
    a.items = pl.d_lpt;
    a.n_items = (int)pl.items_lpt.size();
    a.band = c->band;
    a.queue = q;
    a.status = P<int>(c->status);
    c->launches += 2;  // grid and selection kernels
    return launched(c, launch_grid_select(a, pl.S, n_thr, P<float>(c->grid_thr), P<uint64_t>(c->grid_hist),
                                          P<int32_t>(c->grid_rr), rr_den, K, eps_out, rr_out, count_out,
                                          persistent_grid(c, (size_t)a.n_items), pl.mt, c->stream));
}

int rqa_set_timing(rqa_ctx *c, int enable)
{
    if (!c) return RQA_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    if (enable && !c->ev[0]) {
        for (int i = 0; i < 7; ++i)
            if (cudaEventCreate(&c->ev[i]) != cudaSuccess) return check_cuda(cudaGetLastError());
    }
    c->timing = enable != 0;
    c->ev_recorded = false;
    return RQA_OK;
}

int rqa_phase_times(rqa_ctx *c, float *ms, int n)
{
    if (!c || !ms || n < 6) return RQA_ERR_INVALID_ARG;
    for (int i = 0; i < 6; ++i) ms[i] = 0.f;
    if (!c->timing || !c->ev_recorded) return RQA_OK;
    cudaSetDevice(c->device);
    if (cudaEventSynchronize(c->ev[6]) != cudaSuccess) return check_cuda(cudaGetLastError());
    for (int i = 0; i < 6; ++i)
        if (cudaEventElapsedTime(&ms[i], c->ev[i], c->ev[i + 1]) != cudaSuccess)
            return check_cuda(cudaGetLastError());
    return RQA_OK;
}

uint64_t rqa_kernel_launches(rqa_ctx *c) { return c ? c->launches : 0; }

uint64_t rqa_graph_replays(rqa_ctx *c) { return c ? c->graph_replays : 0; }

int rqa_set_tuning(rqa_ctx *c, const rqa_tuning *t)
{
    if (!c || !t) return RQA_ERR_INVALID_ARG;
    if (t->tile != 0 && t->tile != 8 && t->tile != 16 && t->tile != 32) return RQA_ERR_INVALID_ARG;
    if (t->unit_bands < 0 || t->unit_bands > 64 || t->line_ctas < 0 || t->line_ctas > 8 ||
        (t->stage != 0 && t->stage != 1))
        return RQA_ERR_INVALID_ARG;
    c->line_tile = t->tile;
    c->unit_bands = t->unit_bands;
    c->line_ctas = t->line_ctas;
    c->line_stage = t->stage;
    return RQA_OK;
}

int rqa_get_tuning(rqa_ctx *c, rqa_tuning *t)
{
    if (!c || !t) return RQA_ERR_INVALID_ARG;
    t->tile = c->line_tile ? c->line_tile : LINE_TILE_DEFAULT;
    t->unit_bands = c->unit_bands;
    t->line_ctas = c->line_ctas;
    t->stage = c->line_stage;
    t->ms = c->tuned_ms;
    return RQA_OK;
}

int rqa_autotune(rqa_ctx *c, const rqa_batch *b, const int32_t *rr_num, int32_t rr_den, int32_t K,
                 rqa_tuning *out)
{
    if (!c) return RQA_ERR_INVALID_ARG;
    if (int rc = validate_batch(b)) return rc;
    if (int rc = validate_rr(rr_num, rr_den, K)) return rc;
    cudaSetDevice(c->device);
    // sample: the longest prefix of the batch under ~2e10 cells (at least one series)
    rqa_batch sb = *b;
    uint64_t cells = 0;
    int j = 0;
    for (; j < b->n_series; ++j) {
        const int64_t ne = (b->offsets[j + 1] - b->offsets[j]) - (int64_t)(b->m[j] - 1) * b->tau[j];
        const uint64_t pc = (uint64_t)ne * (uint64_t)(ne - 1) / 2;
        if (j > 0 && cells + pc > (uint64_t)2e10) break;
        cells += pc;
    }
    sb.n_series = j;
    const int saved[4] = {c->line_tile, c->unit_bands, c->line_ctas, c->line_stage};
    c->line_stage = 0;
    c->unit_bands = 0;  // the planned unit size, for the probe's plan
    c->line_ctas = 0;
    Plan probe;
    const int rcp = make_plan(c, &sb, nullptr, 0, K, probe);
    c->unit_bands = saved[1];
    c->line_ctas = saved[2];
    c->line_stage = saved[3];
    if (rcp) return rcp;
    if (probe.ne_max > LINE_NE_MAX) return RQA_ERR_CAPACITY;
    if (int rc = ensure(c->eps_tmp, (size_t)sb.n_series * K * 4)) return rc;
    float *eps = P<float>(c->eps_tmp);
    const int saved_select = c->select;
    c->select = RQA_SELECT_RADIX;  // thresholds only: the plain selection suffices
    int rc = rqa_eps_for_rr(c, &sb, rr_num, rr_den, K, eps, nullptr, nullptr);
    c->select = saved_select;
    if (rc) return rc;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return check_cuda(cudaGetLastError());
    c->unit_bands = 0;
    c->line_ctas = 0;
    c->line_stage = 0;
    // the line pass over the probe with the context's current knobs, best of two
    auto time_lines = [&](float *best) {
        float t_min = 3.4e38f;
        for (int rep = 0; rep < 2 && rc == RQA_OK; ++rep) {
            cudaEventRecord(e0, c->stream);
            rc = rqa_line_hist(c, &sb, eps, K, nullptr, nullptr, nullptr, nullptr, nullptr);
            cudaEventRecord(e1, c->stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) rc = check_cuda(cudaGetLastError());
            float ms = 0.f;
            if (rc == RQA_OK && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) t_min = std::min(t_min, ms);
        }
        *best = t_min;
    };
    float best_ms = 3.4e38f;
    // 1. register window (kept when the caller fixed it)
    int best_tile = c->line_tile ? c->line_tile : LINE_TILE_DEFAULT;
    if (!c->tile_fixed) {
        const int cand[3] = {8, 16, 32};
        for (int ci = 0; ci < 3 && rc == RQA_OK; ++ci) {
            if (!lines_tile_ok(probe.mt, cand[ci])) continue;
            c->line_tile = cand[ci];
            float ms = 0.f;
            time_lines(&ms);
            if (ms < best_ms) {
                best_ms = ms;
                best_tile = cand[ci];
            }
        }
    }
    c->line_tile = best_tile;
    if (best_ms == 3.4e38f && rc == RQA_OK) time_lines(&best_ms);
    // 2. bands per work unit: half and twice the planned size
    int best_units = 0;
    const int planned = probe.chunk;
    const int ucand[2] = {std::max(1, planned / 2), std::min(64, planned * 2)};
    for (int ci = 0; ci < 2 && rc == RQA_OK; ++ci) {
        if (ucand[ci] == planned) continue;
        c->unit_bands = ucand[ci];
        float ms = 0.f;
        time_lines(&ms);
        if (ms < best_ms) {
            best_ms = ms;
            best_units = ucand[ci];
        }
    }
    c->unit_bands = best_units;
    // 3. CTAs per SM: all that fit, or six
    int best_ctas = 0;
    if (rc == RQA_OK) {
        c->line_ctas = 6;
        float ms = 0.f;
        time_lines(&ms);
        if (ms < best_ms) {
            best_ms = ms;
            best_ctas = 6;
        }
    }
    c->line_ctas = best_ctas;
    // 4. series windows staged by bulk copies, where the variant exists
    int best_stage = 0;
    if (rc == RQA_OK && lines_stage_ok(probe.mt, c->line_tile)) {
        c->line_stage = 1;
        float ms = 0.f;
        time_lines(&ms);
        if (ms < best_ms) {
            best_ms = ms;
            best_stage = 1;
        }
    }
    c->line_stage = best_stage;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != RQA_OK) {
        c->line_tile = saved[0];
        c->unit_bands = saved[1];
        c->line_ctas = saved[2];
        c->line_stage = saved[3];
        return rc;
    }
    c->tuned_ms = best_ms;
    if (out) rqa_get_tuning(c, out);
    return RQA_OK;
}

// ---------------------------------------------------------- learned bracket
int rqa_sketch(rqa_ctx *c, const rqa_batch *b, uint64_t seed, float *feats, float *centre,
               float *qdist)
{
    if (!c || !feats) return RQA_ERR_INVALID_ARG;
    if (int rc = validate_batch(b)) return rc;
    cudaSetDevice(c->device);
    Plan pl;
    if (int rc = make_plan(c, b, nullptr, 0, 1, pl)) return rc;
    if (int rc = upload_plan(c, pl, nullptr, 0, nullptr)) return rc;
    return launched(c, launch_sketch(b->y, pl.d_sd, 0, pl.S, seed, feats, centre, qdist, c->stream));
}

int rqa_mlp_forward(rqa_ctx *c, const float *params, const float *X, int32_t B, float *Y,
                    float *acts)
{
    if (!c || !params || !X || !Y || B < 1) return RQA_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    if (!acts) {
        if (int rc = ensure(c->learn_scratch, (size_t)B * 2 * HIDDEN * 4)) return rc;
        acts = P<float>(c->learn_scratch);
    }
    c->launches += 3;
    return check_cuda(mlp_forward(params, X, B, Y, acts, c->stream));
}

int rqa_mlp_backward(rqa_ctx *c, const float *params, const float *X, const float *acts,
                     const float *Y, const float *T, int32_t B, float tau_lo, float tau_hi,
                     float *grads, float *loss)
{
    if (!c || !params || !X || !acts || !Y || !T || !grads || B < 1) return RQA_ERR_INVALID_ARG;
    if (!(tau_lo > 0.f && tau_lo < 1.f && tau_hi > 0.f && tau_hi < 1.f)) return RQA_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    if (int rc = ensure(c->learn_scratch, (size_t)B * (MLP_OUT + 2 * HIDDEN) * 4)) return rc;
    c->launches += 10;
    return check_cuda(mlp_backward(params, X, acts, Y, T, B, tau_lo, tau_hi, grads, loss,
                                   P<float>(c->learn_scratch), c->stream));
}

int rqa_adam_step(rqa_ctx *c, float *params, const float *grads, float *m, float *v, int64_t n,
                  int32_t t, float lr, float beta1, float beta2, float eps)
{
    if (!c || !params || !grads || !m || !v || n < 1 || t < 1) return RQA_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    return launched(c, adam_step(params, grads, m, v, n, t, lr, beta1, beta2, eps, c->stream));
}

int rqa_set_bracket_model(rqa_ctx *c, const float *params, float margin)
{
    if (!c || !(margin >= 0.f)) return RQA_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    if (!params) {
        c->has_model = false;
        return RQA_OK;
    }
    if (int rc = ensure(c->mlp, (size_t)MLP_PARAMS * 4)) return rc;
    if (int rc = check_cuda(cudaMemcpyAsync(c->mlp.p, params, (size_t)MLP_PARAMS * 4,
                                            cudaMemcpyDeviceToDevice, c->stream)))
        return rc;
    c->has_model = true;
    c->margin = margin;
    return RQA_OK;
}

int rqa_log_labels(rqa_ctx *c, const float *eps, const float *centre, int32_t S, int32_t K, float *T)
{
    if (!c || !eps || !centre || !T || S < 1 || K < 1) return RQA_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    return launched(c, launch_log_labels(eps, centre, S, K, T, c->stream));
}

int rqa_bracket_eval(rqa_ctx *c, const float *Y, const float *T, int32_t B, int32_t K, float tau_lo,
                     float tau_hi, float margin, double *loss_sum, uint64_t *inside, double *width_sum)
{
    if (!c || !Y || !T || !loss_sum || !inside || !width_sum || B < 1 || K < 1)
        return RQA_ERR_INVALID_ARG;
    if (!(tau_lo > 0.f && tau_lo < 1.f && tau_hi > 0.f && tau_hi < 1.f && margin >= 0.f))
        return RQA_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    return launched(c, launch_bracket_eval(Y, T, B, K, tau_lo, tau_hi, margin, loss_sum,
                                           reinterpret_cast<unsigned long long *>(inside), width_sum,
                                           c->stream));
}

int rqa_gather_rows(rqa_ctx *c, const float *src, const int64_t *idx, int32_t n, int32_t width, float *dst)
{
    if (!c || !src || !idx || !dst || n < 1 || width < 1) return RQA_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    return launched(c, launch_gather_rows(src, idx, n, width, dst, c->stream));
}

int rqa_set_bracket_domain(rqa_ctx *c, const int32_t *m, const int32_t *tau, int32_t n)
{
    if (!c || n < 0 || n > 64 || (n > 0 && (!m || !tau))) return RQA_ERR_INVALID_ARG;
    for (int i = 0; i < n; ++i)
        if (m[i] < 1 || tau[i] < 1) return RQA_ERR_INVALID_ARG;
    c->dom_m.assign(m, m + n);
    c->dom_tau.assign(tau, tau + n);
    return RQA_OK;
}

int rqa_bracket_stats(rqa_ctx *c, uint64_t *hits, uint64_t *misses)
{
    if (!c) return RQA_ERR_INVALID_ARG;
    uint64_t hm[2] = {0, 0};
    if (c->bstats.p) {
        cudaSetDevice(c->device);
        if (cudaStreamSynchronize(c->stream) != cudaSuccess) return check_cuda(cudaGetLastError());
        if (cudaMemcpy(hm, c->bstats.p, 16, cudaMemcpyDeviceToHost) != cudaSuccess)
            return check_cuda(cudaGetLastError());
    }
    if (hits) *hits = hm[0];
    if (misses) *misses = hm[1];
    return RQA_OK;
}

}  // extern "C"
