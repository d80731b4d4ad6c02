"""The paper's approximate eps search (a fixed grid of thresholds on the
[0,1]-normalised series, closest RR per target) against the oracle, bit for
bit, then DET at those thresholds; on series without heavy ties the exact
selection's rates are at least as close to the targets."""
import numpy as np
import pytest

from oracle import c_oracle as CO
from oracle import rqa_oracle as O

pytestmark = pytest.mark.gpu


def _series(seed):
    rng = np.random.default_rng(seed)
    t = np.arange(800)
    return [rng.standard_normal(300).astype(np.float32),
            (np.sin(2 * np.pi * t / 20.3) + 0.3 * rng.standard_normal(800)).astype(np.float32),
            (np.arange(150) % 11).astype(np.float32) * 0.5]


@pytest.mark.parametrize("n_thr", [400, 25, 1024])
def test_grid_search_against_oracle(rqa_lib, n_thr):
    rqa = rqa_lib
    ys = _series(n_thr)
    m, tau, rr = 3, 2, list(range(1, 100))
    ctx = rqa.Context(select=rqa.RQA_SELECT_RADIX)
    batch = rqa.Batch.from_numpy(ys, m, tau)
    g = rqa.eps_approx(ctx, batch, rr, 100, n_thr)
    det = rqa.det_avg(ctx, batch, None, 100, eps=g["eps"], K=len(rr), lmin=(2, 3))
    ex = rqa.eps_for_rr(ctx, batch, rr, 100)
    assert rqa.rqa_status(ctx) == 0
    eps, rate, cnt = (g[k].cpu().numpy() for k in ("eps", "rr", "count"))
    d = det["det"].cpu().numpy()
    ex_le = ex["count_le"].cpu().numpy()
    err_grid, err_exact = [], []
    for s, y in enumerate(ys):
        ref = O.eps_approx(y, m, tau, rr, 100, n_thr)
        assert np.array_equal(eps[s], ref["eps"]), s
        assert np.array_equal(rate[s], ref["rr"]), s
        assert np.array_equal(cnt[s], ref["count"]), s
        L = CO.lines(y, m, tau, ref["eps"], full_hist=True)
        assert np.array_equal(d[s], O.det_from_hist(L["hist"], L["count"], (2, 3))), s
        P = int(batch.ne[s]) * (int(batch.ne[s]) - 1) // 2
        t = np.array(rr) / 100.0
        if s < 2:  # continuous values; the integer sawtooth's ties make any rule overshoot
            err_grid.append(np.abs(ref["rr"] - t).mean())
            err_exact.append(np.abs(ex_le[s].astype(np.float64) / P - t).mean())
    # the exact rule takes the smallest eps reaching each rate: with few ties it
    # lands within a few cells of the target, the grid within half a grid step
    assert np.mean(err_exact) <= np.mean(err_grid)
    ctx.close()


def test_grid_search_rejects_bad_sizes(rqa_lib):
    import torch
    rqa = rqa_lib
    ctx = rqa.Context()
    batch = rqa.Batch.from_numpy([np.arange(50, dtype=np.float32)], 1, 1)
    out = torch.empty(2, dtype=torch.float32, device="cuda")
    for n_thr in (0, 1025):
        with pytest.raises(rqa.RqaError):
            rqa.rqa_eps_approx(ctx, batch, [10, 20], 100, n_thr, out)
    ctx.close()
