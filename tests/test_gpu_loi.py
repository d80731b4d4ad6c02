"""RQA_FLAG_LOI: recurrence rate and DET with the line of identity counted
(Eq. 3 and Eq. 4 over the whole matrix, as printed), against the oracle's
whole-matrix reading: thresholds and counts bit-exact, DET and L bit-exact
(FP64 ratios of the same integers), ENTR within the tolerance derived in
tests/test_gpu_measures.py."""
import numpy as np
import pytest

from oracle import c_oracle as CO
from oracle import rqa_oracle as O

pytestmark = pytest.mark.gpu

LMIN = (1, 2, 3, 5)
RR = list(range(1, 21)) + [35, 50, 80, 99]


def _series(seed):
    rng = np.random.default_rng(seed)
    t = np.arange(900)
    return [rng.standard_normal(240).astype(np.float32),
            (np.sin(2 * np.pi * t / 20.3) + 0.2 * rng.standard_normal(900)).astype(np.float32),
            np.full(130, 0.5, np.float32)]


@pytest.mark.parametrize("schedule", [0, 1])
def test_loi_against_oracle(rqa_lib, schedule):
    rqa = rqa_lib
    ys = _series(5)
    m, tau = 3, 2
    ctx = rqa.Context(schedule=schedule, select=rqa.RQA_SELECT_RADIX, flags=rqa.RQA_FLAG_LOI)
    batch = rqa.Batch.from_numpy(ys, m, tau)
    sel = rqa.eps_for_rr(ctx, batch, RR, 100)
    da = rqa.det_avg(ctx, batch, RR, 100, lmin=LMIN, lines=True)
    meas = rqa.line_measures(ctx, batch, da["hist"], da["hist_offsets"], len(RR), LMIN)
    assert rqa.rqa_status(ctx) == 0
    hist = rqa.unpack_hist(da["hist"].cpu().numpy(), da["hist_offsets"], batch, len(RR))
    got = {k: v.cpu().numpy() for k, v in list(sel.items()) + list(da.items()) + list(meas.items())
           if hasattr(v, "cpu")}
    for s, y in enumerate(ys):
        ref = O.eps_for_rr(y, m, tau, RR, 100, loi=True)
        assert np.array_equal(got["eps"][s], ref["eps"]), s
        assert np.array_equal(got["count_le"][s], ref["count_le"]), s
        assert np.array_equal(got["count_lt"][s], ref["count_lt"]), s
        L = CO.lines(y, m, tau, ref["eps"], full_hist=True)
        assert np.array_equal(hist[s], L["hist"]), s
        det = O.det_from_hist(L["hist"], L["count"], LMIN, loi=True)
        assert np.array_equal(got["det"][s], det), s
        assert np.array_equal(got["det_avg"][s], O.det_avg(det)), s
        lm = O.line_measures(L["hist"], LMIN, loi=True)
        np.testing.assert_array_equal(got["L"][s], lm["L"])
        np.testing.assert_allclose(got["entr"][s], lm["entr"], rtol=1e-11, atol=1e-15)
    # the constant series: every cell recurrent, DET(1) = 1, DET(2) = 1 - 2 / Ne^2
    ne = 130 - (m - 1) * tau
    assert np.all(got["det"][2][:, 0] == 1.0)
    assert np.all(got["det"][2][:, 1] == (ne * ne - 2) / (ne * ne))
    ctx.close()


def test_loi_rejects_rates_the_identity_line_reaches(rqa_lib):
    rqa = rqa_lib
    ctx = rqa.Context(flags=rqa.RQA_FLAG_LOI)
    batch = rqa.Batch.from_numpy([np.random.default_rng(1).standard_normal(60).astype(np.float32)], 1, 1)
    with pytest.raises(rqa.RqaError) as ei:  # ceil(0.01 * 60^2) = 36 <= Ne = 60
        rqa.eps_for_rr(ctx, batch, [1, 2, 5], 100)
    assert ei.value.code == 1
    sel = rqa.eps_for_rr(ctx, batch, [2, 5], 100)  # ceil(0.02 * 3600) = 72 > 60
    assert rqa.rqa_status(ctx) == 0
    ref = O.eps_for_rr(np.asarray(batch.y.cpu().numpy()), 1, 1, [2, 5], 100, loi=True)
    assert np.array_equal(sel["eps"].cpu().numpy()[0], ref["eps"])
    ctx.close()
