"""Averaged DET for every RR* and the sorting rate S of Sect. 3 (Eq. 5).

The paper judges a measure by how well it orders series of one kind of
dynamics by their signal-to-noise ratio: n series at n SNR levels, repeated
for several noise realisations.  For one realisation, x_j is the place of
series j when the n series are ordered by the measure (ascending), y_j = j its
place in the SNR order (ascending), z the reversed y; S compares the summed
departure |x - y| with the worst case |z - y| (Eq. 5):

    S = (sum_i sum_j |z_j - y_j| - sum_i sum_j |x_j - y_j|) / sum_i sum_j |z_j - y_j|

in per cent: 100 for a perfect order.  Equal measure values keep the SNR
order between them (a stable sort), a reading the paper does not state.
"""
from __future__ import annotations

from typing import Sequence

import numpy as np


def det_avg_prefix(det: np.ndarray) -> np.ndarray:
    """DET averaged over RR = 1..RR* for every RR* (Eq. avgDET): det has the
    targets RR = 1, 2, ... along its second-to-last axis; entry r of the
    result is the FP64 mean of the first r + 1 targets, summed in order."""
    det = np.asarray(det, dtype=np.float64)
    out = np.empty_like(det)
    acc = np.zeros(det.shape[:-2] + det.shape[-1:], dtype=np.float64)
    for k in range(det.shape[-2]):
        acc = acc + det[..., k, :]
        out[..., k, :] = acc / np.float64(k + 1)
    return out


def sorting_rate(measure: np.ndarray) -> float:
    """S in per cent (Eq. 5).  measure[i, j]: the measure of series j (SNR
    level j, ascending) in realisation i."""
    m = np.asarray(measure, dtype=np.float64)
    if m.ndim != 2 or m.shape[1] < 2:
        raise ValueError("measure must be (realisations, n >= 2 SNR levels)")
    n = m.shape[1]
    y = np.arange(1, n + 1)
    z = y[::-1]
    worst = 0
    dep = 0
    for row in m:
        order = np.argsort(row, kind="stable")   # series indices by ascending measure
        x = np.empty(n, dtype=np.int64)
        x[order] = y                             # place of each series in that order
        dep += int(np.abs(x - y).sum())
        worst += int(np.abs(z - y).sum())
    return 100.0 * (worst - dep) / worst


def sorting_rates(det: np.ndarray, averaged: bool = True) -> np.ndarray:
    """S for every target column: det[i, j, k] is DET_k (one lmin) of series j
    (SNR ascending) in realisation i.  averaged: S of the mean DET over
    RR = 1..RR* for each RR* (the paper's averaged approach), else of DET at
    each single RR."""
    d = np.asarray(det, dtype=np.float64)
    if averaged:
        d = det_avg_prefix(d[..., None])[..., 0]
    return np.array([sorting_rate(d[:, :, k]) for k in range(d.shape[2])])
