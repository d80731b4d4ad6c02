"""NumPy oracle for exact RR-preselected thresholds and (averaged) determinism.

TEST INFRASTRUCTURE: only the tests, the smoke check and the benchmark's CPU
baseline use this module.

Notation (Sect. 2, Eq. 1-4): a scalar series y[0..N-1] (FP32) is delay
embedded with dimension m and delay tau (Sect. 3.3),
    x_i = (y[i], y[i+tau], ..., y[i+(m-1)tau]),   i = 0 .. Ne-1,
    Ne = N - (m-1) tau.
(The paper writes the delays backwards, x(t) = [y(t), y(t-tau), ...]; indexing
forwards gives the same set of vectors, shifted by (m-1)tau, hence the same
distances and diagonal lines.)  Distances use the maximum norm (Sect. 2):
    d_ij = max_q |y[i+q tau] - y[j+q tau]|        (FP32 subtract, abs, max).

Readings of the paper (the paper is silent or ambiguous on these):

* Only the upper triangle i < j is used (Sect. 4 computes on j > i); the line
  of identity is excluded from every count.  P = Ne (Ne - 1) / 2 pairs.
* RR targets are rationals rr_num / rr_den (the paper's RR in per cent is
  rr_num / 100).  The target count is T = ceil(rr_num * P / rr_den) in exact
  integers.
* The threshold for a target is the T-th smallest distance, eps (Sect. 2
  fixes the recurrence rate first and takes the eps that yields it).  A cell is
  recurrent iff d_ij <= eps.  (Eq. 2 sets H(0) = 0, i.e. strict d < eps; the
  inclusive form is Eq. 1 evaluated at the next float above eps, and is the
  only reading under which an all-equal-distance series has any recurrence.)
  The achieved count C = #{d <= eps} satisfies #{d < eps} < T <= C.
* DET (Eq. 4) over the upper triangle: sum_{l >= lmin} l P(l) / C, where P(l)
  counts maximal runs of recurrent cells along each diagonal j - i = delta.
  Both triangles hold the same lines, so the ratio equals the full-matrix ratio
  without the line of identity.  DET is a ratio of exact integers in FP64.
* Averaged DET (Eq. avgDET): the FP64 sum of DET over the K targets in their
  given order, divided by K.
"""
from __future__ import annotations

from typing import Dict, Sequence, Tuple

import numpy as np


def embedded_count(n: int, m: int, tau: int) -> int:
    """Ne = N - (m-1) tau, the number of delay vectors (Sect. 3.3)."""
    return int(n) - (int(m) - 1) * int(tau)


def pair_count(ne: int) -> int:
    """P = Ne (Ne - 1) / 2 off-diagonal pairs of the upper triangle (Sect. 4)."""
    return ne * (ne - 1) // 2


def target_counts(p: int, rr_num: Sequence[int], rr_den: int) -> np.ndarray:
    """T_k = ceil(rr_num_k * P / rr_den) in exact integers (Eq. 3 inverted)."""
    out = []
    for r in rr_num:
        num = int(r) * int(p)
        out.append(-((-num) // int(rr_den)))
    return np.array(out, dtype=np.uint64)


def target_counts_loi(ne: int, rr_num: Sequence[int], rr_den: int) -> np.ndarray:
    """Upper-triangle targets when RR counts the whole Ne x Ne matrix with the
    line of identity, as Eq. 3 is written: a rate needs 2 C + Ne >=
    ceil(rr_num Ne^2 / rr_den) recurrent cells (C upper-triangle cells, both
    triangles alike, Ne diagonal cells always recurrent), so
    T_k = ceil((ceil(rr_num Ne^2 / rr_den) - Ne) / 2).  A rate the line of
    identity reaches by itself (T_k <= 0) has no threshold: ValueError."""
    out = []
    for r in rr_num:
        full = -((-int(r) * int(ne) * int(ne)) // int(rr_den))
        t = -((-(full - int(ne))) // 2)
        if t <= 0:
            raise ValueError("the line of identity alone reaches this recurrence rate")
        out.append(t)
    return np.array(out, dtype=np.uint64)


def diagonal_distances(y: np.ndarray, m: int, tau: int, delta: int) -> np.ndarray:
    """d(i, i+delta) for i = 0 .. Ne-delta-1, maximum norm in FP32 (Eq. 1)."""
    y = np.asarray(y, dtype=np.float32)
    ne = embedded_count(len(y), m, tau)
    i = np.arange(ne - delta)
    d = np.abs(y[i] - y[i + delta])
    for q in range(1, m):
        d = np.maximum(d, np.abs(y[i + q * tau] - y[i + delta + q * tau]))
    return d.astype(np.float32)


def all_distances(y: np.ndarray, m: int, tau: int) -> np.ndarray:
    """All P upper-triangle distances, diagonal by diagonal (delta = 1 .. Ne-1)."""
    ne = embedded_count(len(y), m, tau)
    if ne < 2:
        return np.zeros(0, dtype=np.float32)
    return np.concatenate([diagonal_distances(y, m, tau, dl) for dl in range(1, ne)])


def eps_for_rr(y: np.ndarray, m: int, tau: int, rr_num: Sequence[int], rr_den: int,
               dist: np.ndarray = None, loi: bool = False) -> Dict[str, np.ndarray]:
    """Exact thresholds by sorting all distances (Sect. 2: RR fixed first, eps from it).

    Returns eps (FP32), T, count_le = #{d <= eps}, count_lt = #{d < eps} (upper
    triangle).  loi: RR over the whole matrix with the line of identity
    (target_counts_loi) instead of over the upper triangle.
    """
    d = all_distances(y, m, tau) if dist is None else dist
    p = d.shape[0]
    if p == 0:
        raise ValueError("fewer than two embedded vectors")
    ne = embedded_count(len(y), m, tau)
    t = target_counts_loi(ne, rr_num, rr_den) if loi else target_counts(p, rr_num, rr_den)
    s = np.sort(d, kind="stable")
    eps = s[(t - 1).astype(np.int64)].astype(np.float32)
    le = np.searchsorted(s, eps, side="right").astype(np.uint64)
    lt = np.searchsorted(s, eps, side="left").astype(np.uint64)
    return {"eps": eps, "T": t, "count_le": le, "count_lt": lt}


def _runs(mask: np.ndarray) -> np.ndarray:
    """Lengths of the maximal runs of True in a 1-D boolean array."""
    if mask.size == 0:
        return np.zeros(0, dtype=np.int64)
    padded = np.concatenate(([False], mask, [False])).astype(np.int8)
    diff = np.diff(padded)
    starts = np.flatnonzero(diff == 1)
    ends = np.flatnonzero(diff == -1)
    return (ends - starts).astype(np.int64)


def line_hist(y: np.ndarray, m: int, tau: int, eps: Sequence[float]) -> Dict[str, np.ndarray]:
    """Diagonal line statistics of the upper triangle for each threshold.

    For every threshold k: hist[k, l-1] = P_k(l), the number of maximal
    diagonal runs of length l (l = 1 .. Ne-1; Eq. 4 and Sect. 4); count =
    number of recurrent cells; stencil = recurrent cells with a recurrent
    diagonal neighbour (i-1, j-1) or (i+1, j+1); lmax = longest run.
    """
    y = np.asarray(y, dtype=np.float32)
    eps = np.asarray(eps, dtype=np.float32)
    k = eps.shape[0]
    ne = embedded_count(len(y), m, tau)
    hist = np.zeros((k, max(ne - 1, 0)), dtype=np.uint64)
    count = np.zeros(k, dtype=np.uint64)
    stencil = np.zeros(k, dtype=np.uint64)
    lmax = np.zeros(k, dtype=np.uint32)
    for dl in range(1, ne):
        d = diagonal_distances(y, m, tau, dl)
        # rec[k, i] = R^k_{i, i+dl}: one row per threshold along this diagonal.
        rec = d[None, :] <= eps[:, None]
        count += rec.sum(axis=1).astype(np.uint64)
        nb = np.zeros_like(rec)
        nb[:, 1:] |= rec[:, :-1]
        nb[:, :-1] |= rec[:, 1:]
        stencil += (rec & nb).sum(axis=1).astype(np.uint64)
        # Maximal runs: +1 where a run starts, -1 one past where it ends.
        padded = np.zeros((k, rec.shape[1] + 2), dtype=np.int8)
        padded[:, 1:-1] = rec
        edge = np.diff(padded, axis=1)
        ks, starts = np.nonzero(edge == 1)      # row-major: sorted by (k, position)
        ke, ends = np.nonzero(edge == -1)
        assert np.array_equal(ks, ke)
        lens = ends - starts
        if lens.size:
            np.add.at(hist, (ks, lens - 1), np.uint64(1))
            np.maximum.at(lmax, ks, lens.astype(np.uint32))
    return {"hist": hist, "count": count, "stencil": stencil, "lmax": lmax}


def approx_thresholds(y: np.ndarray, n_thr: int = 400) -> np.ndarray:
    """The fixed threshold grid of the paper's approximate search (described in
    its source as a comment, Sect. 2): every series mapped onto [0, 1] and RR
    evaluated at n_thr thresholds.  Reading: thresholds i/n_thr, i = 1..n_thr,
    of the [0, 1]-normalised series, i.e. in the series' own units
    thr_i = float32(i) * (range / n_thr) with range = max(y) - min(y), every
    operation in FP32 (correctly rounded), so any implementation reproduces the
    grid bit for bit."""
    y = np.asarray(y, dtype=np.float32)
    rng = np.float32(np.float32(y.max()) - np.float32(y.min()))
    scale = np.float32(rng / np.float32(n_thr))
    return (np.arange(1, n_thr + 1, dtype=np.float32) * scale).astype(np.float32)


def eps_approx(y: np.ndarray, m: int, tau: int, rr_num: Sequence[int], rr_den: int,
               n_thr: int = 400) -> Dict[str, np.ndarray]:
    """The paper's approximate eps search: RR at every grid threshold
    (approx_thresholds), then for each target the threshold whose RR is the
    closest to it (ties: the lower threshold).  Counts over the upper triangle
    (recurrent iff d <= thr).  Returns eps (FP32), rr (achieved RR, FP64
    fraction), count (#{d <= eps}) and the full grid counts."""
    d = np.sort(all_distances(y, m, tau), kind="stable")
    p = d.shape[0]
    thr = approx_thresholds(y, n_thr)
    c = np.searchsorted(d, thr, side="right").astype(np.int64)   # C_j = #{d <= thr_j}
    eps, rr, cnt = [], [], []
    for r in rr_num:
        # |C_j / P - r / den| compared exactly as |C_j den - r P|
        err = [abs(int(cj) * int(rr_den) - int(r) * int(p)) for cj in c]
        j = int(np.argmin(err))                                    # first minimum: lower threshold
        eps.append(thr[j])
        cnt.append(int(c[j]))
        rr.append(float(c[j]) / float(p))
    return {"eps": np.array(eps, dtype=np.float32), "rr": np.array(rr, dtype=np.float64),
            "count": np.array(cnt, dtype=np.uint64), "grid_count": c.astype(np.uint64), "thr": thr}


def column_distances(y: np.ndarray, m: int, tau: int, j: int) -> np.ndarray:
    """d(i, j) for i = 0 .. Ne-1 (the whole column j, d(j, j) = 0), FP32."""
    y = np.asarray(y, dtype=np.float32)
    ne = embedded_count(len(y), m, tau)
    i = np.arange(ne)
    d = np.abs(y[i] - y[j])
    for q in range(1, m):
        d = np.maximum(d, np.abs(y[i + q * tau] - y[j + q * tau]))
    return d.astype(np.float32)


def vline_hist(y: np.ndarray, m: int, tau: int, eps: Sequence[float],
               loi: bool = False) -> Dict[str, np.ndarray]:
    """Vertical line statistics of the whole recurrence matrix per threshold.

    Sect. 2 notes that the averaging applies to other RQA measures; the
    vertical-line ones (laminarity LAM, trapping time TT; Marwan et al. 2007,
    Phys. Rep. 438, Sect. 5.1) count maximal runs of recurrent cells along each
    column j of the Ne x Ne matrix.  The line of identity is left out (the cell
    (j, j) ends a run) unless loi, where it is recurrent like every d = 0 cell.
    vhist[k, l-1] = V_k(l) for l = 1 .. Ne-1 (loi: 1 .. Ne, one more column),
    vmax = longest vertical line.
    """
    y = np.asarray(y, dtype=np.float32)
    eps = np.asarray(eps, dtype=np.float32)
    k = eps.shape[0]
    ne = embedded_count(len(y), m, tau)
    nl = ne if loi else max(ne - 1, 0)
    vhist = np.zeros((k, nl), dtype=np.uint64)
    vmax = np.zeros(k, dtype=np.uint32)
    for j in range(ne):
        d = column_distances(y, m, tau, j)
        rec = d[None, :] <= eps[:, None]
        if not loi:
            rec[:, j] = False
        for kk in range(k):
            runs = _runs(rec[kk])
            if runs.size:
                np.add.at(vhist[kk], runs - 1, 1)
                vmax[kk] = max(int(vmax[kk]), int(runs.max()))
    return {"vhist": vhist, "vmax": vmax}


def lam_tt(vhist: np.ndarray, count: np.ndarray, vmin: Sequence[int], ne: int,
           loi: bool = False) -> Dict[str, np.ndarray]:
    """LAM_k(vmin) = sum_{l >= vmin} l V_k(l) / (recurrent cells of the matrix)
    and TT_k(vmin) = sum_{l >= vmin} l V_k(l) / sum_{l >= vmin} V_k(l), FP64
    ratios of exact integers.  The recurrent cells are 2 C_k (both triangles,
    count = upper-triangle C_k), plus Ne with loi.  TT is NaN when no vertical
    line is vmin long.  Shapes (K, len(vmin))."""
    k = vhist.shape[0]
    lam = np.zeros((k, len(vmin)), dtype=np.float64)
    tt = np.zeros((k, len(vmin)), dtype=np.float64)
    for kk in range(k):
        row = [int(v) for v in vhist[kk]]
        rec = 2 * int(count[kk]) + (ne if loi else 0)
        for j, vm in enumerate(vmin):
            mass = sum(l * c for l, c in enumerate(row, start=1) if l >= vm)
            nv = sum(c for l, c in enumerate(row, start=1) if l >= vm)
            lam[kk, j] = float(mass) / float(rec)
            tt[kk, j] = float(mass) / float(nv) if nv else float("nan")
    return {"lam": lam, "tt": tt}


def det_from_hist(hist: np.ndarray, count: np.ndarray, lmin: Sequence[int],
                  loi: bool = False) -> np.ndarray:
    """DET_k(lmin) = sum_{l >= lmin} l P_k(l) / C_k in FP64 (Eq. 4).

    With no recurrent cell (C_k = 0, only possible for thresholds the caller
    gives) Eq. 4 is 0/0: undefined, returned as NaN (the IEEE quotient 0.0/0.0).
    loi: over the whole matrix with the line of identity, as Eq. 4 is written:
    every upper-triangle line twice plus the identity line of length Ne =
    hist.shape[1] + 1, i.e. (2 sum_{l >= lmin} l P_k(l) + Ne [Ne >= lmin]) /
    (2 C_k + Ne).  Returns an array of shape (K, len(lmin)).
    """
    k, lmax_len = hist.shape
    ne = lmax_len + 1
    out = np.zeros((k, len(lmin)), dtype=np.float64)
    lengths = np.arange(1, lmax_len + 1, dtype=object)
    for kk in range(k):
        row = [int(v) for v in hist[kk]]
        for j, lm in enumerate(lmin):
            num = sum(int(l) * c for l, c in zip(lengths, row) if l >= lm)
            den = int(count[kk])
            if loi:
                num = 2 * num + (ne if ne >= lm else 0)
                den = 2 * den + ne
            out[kk, j] = float(num) / float(den) if den else float("nan")
    return out


def det_avg(det: np.ndarray) -> np.ndarray:
    """Averaged DET (Eq. avgDET): FP64 sum over k in order, then / K."""
    k = det.shape[0]
    acc = np.zeros(det.shape[1], dtype=np.float64)
    for kk in range(k):
        acc = acc + det[kk]
    return acc / np.float64(k)


def line_measures(hist: np.ndarray, lmin: Sequence[int], loi: bool = False) -> Dict[str, np.ndarray]:
    """Average diagonal line length L and line-length entropy ENTR (K, len(lmin)).

    Sect. 2 closes by noting that the averaging over RR applies to other RQA
    measures as well; these two are the usual diagonal-line measures next to
    DET (Marwan et al. 2007, Phys. Rep. 438, Sect. 5.1), over lines of length
    >= lmin of the upper triangle (both triangles hold the same lines, so the
    ratios equal the full-matrix ones without the line of identity):
        N_l  = sum_{l >= lmin} P(l)                  (number of lines)
        L    = sum_{l >= lmin} l P(l) / N_l          (FP64 ratio of exact integers;
                                                      NaN when N_l = 0)
        ENTR = -sum_{l >= lmin} p(l) ln p(l),  p(l) = P(l) / N_l
               (natural logarithm, FP64, summed over l ascending; 0 when N_l = 0).
    loi: the whole matrix with the line of identity (P(l) -> 2 P(l), plus one
    line of length Ne = hist.shape[1] + 1), as for det_from_hist.
    """
    k, nl = hist.shape
    L = np.zeros((k, len(lmin)), dtype=np.float64)
    E = np.zeros((k, len(lmin)), dtype=np.float64)
    for kk in range(k):
        row = [int(v) for v in hist[kk]]
        if loi:  # whole matrix: each line twice, plus the identity line of length Ne
            row = [2 * c for c in row] + [1]
        for j, lm in enumerate(lmin):
            n_lines = sum(c for l, c in enumerate(row, start=1) if l >= lm)
            mass = sum(l * c for l, c in enumerate(row, start=1) if l >= lm)
            L[kk, j] = float(mass) / float(n_lines) if n_lines else float("nan")
            ent = 0.0
            for l, c in enumerate(row, start=1):
                if l >= lm and c:
                    pl = float(c) / float(n_lines)
                    ent = ent - pl * float(np.log(pl))
            E[kk, j] = ent
    return {"L": L, "entr": E}


def measure_avg(v: np.ndarray) -> np.ndarray:
    """Average of a per-target measure over the K targets (the same reduction
    as Eq. avgDET): FP64 sum in k order, then / K."""
    return det_avg(v)


def rqa_det_avg(y: np.ndarray, m: int, tau: int, rr_num: Sequence[int], rr_den: int,
                lmin: Sequence[int] = (2,), loi: bool = False) -> Dict[str, np.ndarray]:
    """The whole hot path on one series: eps_k, line statistics, DET_k, mean."""
    sel = eps_for_rr(y, m, tau, rr_num, rr_den, loi=loi)
    lines = line_hist(y, m, tau, sel["eps"])
    det = det_from_hist(lines["hist"], lines["count"], lmin, loi=loi)
    out = dict(sel)
    out.update(lines)
    out["det"] = det
    out["det_avg"] = det_avg(det)
    return out
