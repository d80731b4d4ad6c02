"""GB300-native averaged recurrence quantification analysis.

For each delay-embedded FP32 series: exact thresholds eps_k for K target
recurrence rates, determinism DET(eps_k) over the never-materialised
recurrence matrix, its average over k, and the diagonal line-length histogram
(Pánis, Adámek & Marwan, Sect. 2-4).  The work runs in hand-written sm_103a
CUDA kernels behind a C ABI (``include/rqa.h``); this package is its Python
binding (``abi``) plus a few conveniences that allocate outputs as tensors.
"""
from __future__ import annotations

from typing import Dict, Optional, Sequence

import numpy as np

from .abi import (  # noqa: F401
    Batch, Context, RqaError, exported_symbols, lib,
    rqa_abi_version, rqa_create, rqa_destroy, rqa_det_avg, rqa_device_info,
    rqa_error_string, rqa_eps_for_rr, rqa_line_hist, rqa_status, rqa_target_counts,
    rqa_target_counts_loi,
    rqa_set_timing, rqa_phase_times, rqa_kernel_launches,
    rqa_sketch, rqa_mlp_forward, rqa_mlp_backward, rqa_adam_step, rqa_set_bracket_model,
    rqa_set_bracket_domain, rqa_bracket_stats, rqa_log_labels, rqa_bracket_eval, rqa_gather_rows, RQA_MLP_PARAMS, RQA_MLP_ACTS, RQA_MLP_OUT,
    rqa_eps_for_rr_noalloc, RQA_NOALLOC_MAX_SERIES, RQA_NOALLOC_NE_MAX, RQA_NOALLOC_K_MAX,
    rqa_graph_replays, rqa_autotune, rqa_set_tuning, rqa_get_tuning, RQA_FLAG_NO_GRAPHS, RQA_FLAG_LOI, rqa_line_measures,
    rqa_vline_hist, rqa_lam_tt, rqa_eps_approx,
    RQA_SCHED_BATCHED, RQA_SCHED_PER_SERIES, RQA_SELECT_AUTO, RQA_SELECT_BRACKET,
    RQA_SELECT_RADIX, RQA_K_MAX, RQA_LMIN_MAX, RQA_FEATURES,
)


def eps_for_rr(ctx: Context, batch: Batch, rr_num: Sequence[int], rr_den: int) -> Dict[str, "object"]:
    """Thresholds and counts as CUDA tensors of shape (S, K)."""
    import torch
    S, K = batch.n_series, len(rr_num)
    dev = batch.y.device
    eps = torch.empty((S, K), dtype=torch.float32, device=dev)
    le = torch.empty((S, K), dtype=torch.uint64, device=dev)
    lt = torch.empty((S, K), dtype=torch.uint64, device=dev)
    rqa_eps_for_rr(ctx, batch, rr_num, rr_den, eps, le, lt)
    return {"eps": eps, "count_le": le, "count_lt": lt}


def det_avg(ctx: Context, batch: Batch, rr_num: Optional[Sequence[int]], rr_den: int,
            lmin: Sequence[int] = (2,), eps=None, K: Optional[int] = None,
            lines: bool = False) -> Dict[str, "object"]:
    """DET_k(lmin) (S, K, L), its mean over k (S, L) and the thresholds used;
    with lines=True also the full histograms, L_max, C_k and stencil counts of
    the same pass."""
    import torch
    S = batch.n_series
    K = len(rr_num) if K is None else K
    dev = batch.y.device
    det = torch.empty((S, K, len(lmin)), dtype=torch.float64, device=dev)
    avg = torch.empty((S, len(lmin)), dtype=torch.float64, device=dev)
    used = torch.empty((S, K), dtype=torch.float32, device=dev)
    out = {"det": det, "det_avg": avg, "eps": used}
    if lines:
        hoff = batch.hist_offsets(K)
        out.update(hist=torch.empty(int(hoff[-1]), dtype=torch.uint64, device=dev), hist_offsets=hoff,
                   lmax=torch.empty((S, K), dtype=torch.uint32, device=dev),
                   count=torch.empty((S, K), dtype=torch.uint64, device=dev),
                   stencil=torch.empty((S, K), dtype=torch.uint64, device=dev))
        rqa_det_avg(ctx, batch, rr_num, rr_den, eps, K, lmin, det, avg, used, out["hist"], hoff,
                    out["lmax"], out["count"], out["stencil"])
    else:
        rqa_det_avg(ctx, batch, rr_num, rr_den, eps, K, lmin, det, avg, used)
    return out


def line_measures(ctx: Context, batch: Batch, hist, hist_offsets, K: int,
                  lmin: Sequence[int] = (2,)) -> Dict[str, "object"]:
    """Average line length L and line-length entropy ENTR per target (S, K, L)
    and their means over the targets (S, L), from a full line histogram."""
    import torch
    S = batch.n_series
    dev = batch.y.device
    out = {"L": torch.empty((S, K, len(lmin)), dtype=torch.float64, device=dev),
           "entr": torch.empty((S, K, len(lmin)), dtype=torch.float64, device=dev),
           "L_avg": torch.empty((S, len(lmin)), dtype=torch.float64, device=dev),
           "entr_avg": torch.empty((S, len(lmin)), dtype=torch.float64, device=dev)}
    rqa_line_measures(ctx, batch, K, hist, hist_offsets, lmin, out["L"], out["entr"], out["L_avg"],
                      out["entr_avg"])
    return out


def eps_approx(ctx: Context, batch: Batch, rr_num: Sequence[int], rr_den: int,
               n_thr: int = 400) -> Dict[str, "object"]:
    """The paper's approximate search: grid thresholds closest to each target
    RR, their rates and counts (S, K)."""
    import torch
    S, K = batch.n_series, len(rr_num)
    dev = batch.y.device
    out = {"eps": torch.empty((S, K), dtype=torch.float32, device=dev),
           "rr": torch.empty((S, K), dtype=torch.float64, device=dev),
           "count": torch.empty((S, K), dtype=torch.uint64, device=dev)}
    rqa_eps_approx(ctx, batch, rr_num, rr_den, n_thr, out["eps"], out["rr"], out["count"])
    return out


def vline_offsets(batch: Batch, K: int, loi: bool = False) -> np.ndarray:
    """Packed offsets of vertical-line histograms: K*(Ne-1) per series, K*Ne
    when the context counts the line of identity."""
    off = np.zeros(batch.n_series + 1, dtype=np.int64)
    off[1:] = np.cumsum(K * (batch.ne - 1 + (1 if loi else 0)))
    return off


def vline_hist(ctx: Context, batch: Batch, eps, K: int, loi: bool = False) -> Dict[str, "object"]:
    """Vertical-line histograms V_k(l) (packed), longest vertical line and
    vertical mass per target."""
    import torch
    S = batch.n_series
    dev = batch.y.device
    voff = vline_offsets(batch, K, loi)
    out = {"vhist": torch.empty(int(voff[-1]), dtype=torch.uint64, device=dev), "vhist_offsets": voff,
           "vmax": torch.empty((S, K), dtype=torch.uint32, device=dev),
           "vmass": torch.empty((S, K), dtype=torch.uint64, device=dev)}
    rqa_vline_hist(ctx, batch, eps, K, out["vhist"], voff, out["vmax"], out["vmass"])
    return out


def lam_tt(ctx: Context, batch: Batch, vhist, vhist_offsets, K: int,
           vmin: Sequence[int] = (2,)) -> Dict[str, "object"]:
    """Laminarity and trapping time per target (S, K, V) and their means (S, V)."""
    import torch
    S = batch.n_series
    dev = batch.y.device
    out = {"lam": torch.empty((S, K, len(vmin)), dtype=torch.float64, device=dev),
           "tt": torch.empty((S, K, len(vmin)), dtype=torch.float64, device=dev),
           "lam_avg": torch.empty((S, len(vmin)), dtype=torch.float64, device=dev),
           "tt_avg": torch.empty((S, len(vmin)), dtype=torch.float64, device=dev)}
    rqa_lam_tt(ctx, batch, K, vhist, vhist_offsets, vmin, out["lam"], out["tt"], out["lam_avg"],
               out["tt_avg"])
    return out


def line_hist(ctx: Context, batch: Batch, eps, K: int, full: bool = True) -> Dict[str, "object"]:
    """Full P_k(l) histograms (packed per series), L_max, C_k and stencil counts."""
    import torch
    S = batch.n_series
    dev = batch.y.device
    hoff = batch.hist_offsets(K) if full else None
    hist = torch.empty(int(hoff[-1]) if full else 0, dtype=torch.uint64, device=dev) if full else None
    lmax = torch.empty((S, K), dtype=torch.uint32, device=dev)
    cnt = torch.empty((S, K), dtype=torch.uint64, device=dev)
    st = torch.empty((S, K), dtype=torch.uint64, device=dev)
    rqa_line_hist(ctx, batch, eps, K, hist, hoff, lmax, cnt, st)
    return {"hist": hist, "hist_offsets": hoff, "lmax": lmax, "count": cnt, "stencil": st}


def unpack_hist(hist_np: np.ndarray, hoff: np.ndarray, batch: Batch, K: int):
    """Split a packed histogram into per-series (K, Ne-1) arrays."""
    out = []
    for s in range(batch.n_series):
        ne = int(batch.ne[s])
        out.append(hist_np[hoff[s]:hoff[s + 1]].reshape(K, ne - 1))
    return out
