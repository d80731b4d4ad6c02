"""Shared test helpers: run the CUDA path through the C ABI and the CPU oracle
on the same seeded inputs, and compare element by element."""
from __future__ import annotations

from typing import Dict, List, Sequence

import numpy as np

RR20 = list(range(1, 21))


def oracle_series(y: np.ndarray, m: int, tau: int, rr: Sequence[int], den: int,
                  lmin: Sequence[int] = (2,), full_hist: bool = True) -> Dict[str, np.ndarray]:
    """Oracle results for one series: sort-based eps (NumPy), diagonal scans (C)."""
    from oracle import c_oracle as CO
    from oracle import rqa_oracle as O
    d = CO.distances(y, m, tau)
    sel = O.eps_for_rr(y, m, tau, rr, den, dist=d)
    del d
    lines = CO.lines(y, m, tau, sel["eps"], full_hist=True)
    det = O.det_from_hist(lines["hist"], lines["count"], lmin)
    out = dict(sel)
    out.update(lines)
    out["det"] = det
    out["det_avg"] = O.det_avg(det)
    if not full_hist:
        out.pop("hist")
    return out


def gpu_run(series: List[np.ndarray], m, tau, rr: Sequence[int], den: int,
            lmin: Sequence[int] = (2,), schedule: int = 0, select: int = 1,
            hist: bool = True) -> Dict[str, object]:
    """eps_for_rr, det_avg (one call, eps selected inside) and line_hist."""
    import torch
    import paper_2208_09136_gb300 as rqa
    ctx = rqa.Context(device=0, schedule=schedule, select=select)
    batch = rqa.Batch.from_numpy(series, m, tau, device=0)
    K = len(rr)
    sel = rqa.eps_for_rr(ctx, batch, rr, den)
    da = rqa.det_avg(ctx, batch, rr, den, lmin=lmin)
    lh = rqa.line_hist(ctx, batch, sel["eps"], K, full=hist)
    code = rqa.rqa_status(ctx)
    assert code == 0, rqa.rqa_error_string(code)
    torch.cuda.synchronize()
    out = {
        "eps": sel["eps"].cpu().numpy(),
        "count_le": sel["count_le"].cpu().numpy(),
        "count_lt": sel["count_lt"].cpu().numpy(),
        "det": da["det"].cpu().numpy(),
        "det_avg": da["det_avg"].cpu().numpy(),
        "eps_det": da["eps"].cpu().numpy(),
        "lmax": lh["lmax"].cpu().numpy(),
        "count": lh["count"].cpu().numpy(),
        "stencil": lh["stencil"].cpu().numpy(),
        "batch": batch,
    }
    if hist:
        out["hist"] = rqa.unpack_hist(lh["hist"].cpu().numpy(), lh["hist_offsets"], batch, K)
    ctx.close()
    return out


def assert_series_equal(g: Dict[str, object], s: int, ref: Dict[str, np.ndarray], tag: str = ""):
    """Bit-exact comparison of series s of a GPU run with its oracle result."""
    where = f"{tag} series {s}"
    assert np.array_equal(g["eps"][s], ref["eps"]), (where, "eps", g["eps"][s], ref["eps"])
    assert np.array_equal(g["eps_det"][s], ref["eps"]), (where, "eps (det_avg)")
    assert np.array_equal(g["count_le"][s], ref["count_le"]), (where, "count_le")
    assert np.array_equal(g["count_lt"][s], ref["count_lt"]), (where, "count_lt")
    assert np.array_equal(g["count"][s], ref["count"]), (where, "count")
    assert np.array_equal(g["stencil"][s], ref["stencil"]), (where, "stencil")
    assert np.array_equal(g["lmax"][s], ref["lmax"]), (where, "lmax")
    if "hist" in g and "hist" in ref:
        assert np.array_equal(g["hist"][s], ref["hist"]), (where, "hist")
    # DET is an FP64 ratio of identical integers: bit-exact
    assert np.array_equal(g["det"][s], ref["det"]), (where, "det", g["det"][s], ref["det"])
    assert np.array_equal(g["det_avg"][s], ref["det_avg"]), (where, "det_avg")
