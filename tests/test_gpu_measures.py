"""L (average diagonal line length) and ENTR (line-length entropy) per target
and averaged over the targets, from the line pass's full histograms, against
the oracle.  L is a ratio of exact integers and must match bit for bit; ENTR
sums FP64 terms -p ln p: the device log and the host log may differ by one
ulp per term and the two sides add the terms in different orders, so for n
non-negative terms the sums agree within about (n + 2) * 2^-52 relative; the
test allows 1e-11 (n <= 10^4 here)."""
import math

import numpy as np
import pytest

from oracle import rqa_oracle as O
from tests._helpers import RR20, oracle_series

pytestmark = pytest.mark.gpu

LMIN = (1, 2, 3, 5)


def _series(seed, sizes):
    rng = np.random.default_rng(seed)
    out = []
    for i, n in enumerate(sizes):
        t = np.arange(n)
        if i % 3 == 0:
            out.append(rng.standard_normal(n).astype(np.float32))
        elif i % 3 == 1:
            out.append((np.sin(2 * np.pi * t / 20.3) + 0.2 * rng.standard_normal(n)).astype(np.float32))
        else:
            x = np.empty(n)
            x[0] = rng.uniform(0.1, 0.9)
            for j in range(1, n):
                x[j] = 4.0 * x[j - 1] * (1.0 - x[j - 1])
            out.append(x.astype(np.float32))
    return out


def _check(rqa, ctx, ys, m, tau, rr):
    batch = rqa.Batch.from_numpy(ys, m, tau)
    K = len(rr)
    lines = rqa.det_avg(ctx, batch, rr, 100, lmin=(2,), lines=True)
    out = rqa.line_measures(ctx, batch, lines["hist"], lines["hist_offsets"], K, LMIN)
    assert rqa.rqa_status(ctx) == 0
    got = {k: v.cpu().numpy() for k, v in out.items()}
    for s, y in enumerate(ys):
        ref_lines = oracle_series(y, m, tau, rr, 100, lmin=(2,))
        ref = O.line_measures(ref_lines["hist"], LMIN)
        np.testing.assert_array_equal(got["L"][s], ref["L"])  # NaN where no line is that long
        np.testing.assert_allclose(got["entr"][s], ref["entr"], rtol=1e-11, atol=1e-15)
        np.testing.assert_array_equal(got["L_avg"][s], O.measure_avg(ref["L"]))
        np.testing.assert_allclose(got["entr_avg"][s], O.measure_avg(ref["entr"]), rtol=1e-11, atol=1e-15)


def test_measures_mixed_series(rqa_lib):
    ctx = rqa_lib.Context()
    _check(rqa_lib, ctx, _series(3, [50, 700, 3000, 5001, 90]), 3, 2, RR20)
    ctx.close()


def test_measures_constant_series_closed_form(rqa_lib):
    """Constant series: one line of each length 1..Ne-1, so L is the mean of
    lmin..Ne-1 and ENTR = ln(Ne - lmin) for every target."""
    rqa = rqa_lib
    ctx = rqa.Context()
    n = 300
    batch = rqa.Batch.from_numpy([np.full(n, 2.5, dtype=np.float32)], 1, 1)
    lines = rqa.det_avg(ctx, batch, [1, 50, 99], 100, lmin=(2,), lines=True)
    out = rqa.line_measures(ctx, batch, lines["hist"], lines["hist_offsets"], 3, LMIN)
    L, E = out["L"].cpu().numpy()[0], out["entr"].cpu().numpy()[0]
    for j, lm in enumerate(LMIN):
        ls = list(range(lm, n))
        assert np.all(L[:, j] == sum(ls) / len(ls))
        assert np.allclose(E[:, j], math.log(len(ls)), rtol=1e-12)
    ctx.close()


def test_measures_averages_only(rqa_lib):
    """Averages without per-target outputs (context scratch) equal those with."""
    import torch
    rqa = rqa_lib
    ctx = rqa.Context()
    ys = _series(8, [400, 1200])
    batch = rqa.Batch.from_numpy(ys, 3, 3)
    lines = rqa.det_avg(ctx, batch, RR20, 100, lmin=(2,), lines=True)
    full = rqa.line_measures(ctx, batch, lines["hist"], lines["hist_offsets"], 20, LMIN)
    la = torch.empty((2, len(LMIN)), dtype=torch.float64, device="cuda")
    ea = torch.empty_like(la)
    rqa.rqa_line_measures(ctx, batch, 20, lines["hist"], lines["hist_offsets"], LMIN, None, None, la, ea)
    assert rqa.rqa_status(ctx) == 0
    torch.testing.assert_close(la, full["L_avg"], rtol=0, atol=0, equal_nan=True)  # NaN: no line >= lmin
    torch.testing.assert_close(ea, full["entr_avg"], rtol=0, atol=0)
    ctx.close()


def test_measures_rejects_bad_arguments(rqa_lib):
    rqa = rqa_lib
    ctx = rqa.Context()
    batch = rqa.Batch.from_numpy(_series(1, [100]), 1, 1)
    lines = rqa.det_avg(ctx, batch, RR20, 100, lmin=(2,), lines=True)
    with pytest.raises(rqa.RqaError):
        rqa.line_measures(ctx, batch, lines["hist"], lines["hist_offsets"], 20, (0,))
    bad = np.array(lines["hist_offsets"])
    bad[0] = 1  # packed offsets must start at 0
    with pytest.raises(rqa.RqaError):
        rqa.line_measures(ctx, batch, lines["hist"], bad, 20, (2,))
    ctx.close()
