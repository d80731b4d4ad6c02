"""Vertical lines of the whole recurrence matrix (rqa_vline_hist) and
laminarity / trapping time (rqa_lam_tt) against the oracle, bit for bit:
histograms, longest lines, the vertical mass (= every recurrent cell), and
LAM/TT as FP64 ratios of the same integers."""
import numpy as np
import pytest

from oracle import rqa_oracle as O

pytestmark = pytest.mark.gpu

VMIN = (1, 2, 3, 5)


def _series(seed):
    rng = np.random.default_rng(seed)
    t = np.arange(700)
    x = np.empty(300)
    x[0] = 0.3
    for j in range(1, 300):
        x[j] = 4.0 * x[j - 1] * (1.0 - x[j - 1])
    return [rng.standard_normal(97).astype(np.float32),
            (np.sin(2 * np.pi * t / 20.3) + 0.2 * rng.standard_normal(700)).astype(np.float32),
            x.astype(np.float32), np.full(66, 0.25, np.float32), rng.standard_normal(9).astype(np.float32)]


def _check(rqa, ys, m, tau, rr, schedule, loi):
    flags = rqa.RQA_FLAG_LOI if loi else 0
    ctx = rqa.Context(schedule=schedule, select=rqa.RQA_SELECT_RADIX, flags=flags)
    batch = rqa.Batch.from_numpy(ys, m, tau)
    K = len(rr)
    sel = rqa.eps_for_rr(ctx, batch, rr, 100)
    v = rqa.vline_hist(ctx, batch, sel["eps"], K, loi=loi)
    lt = rqa.lam_tt(ctx, batch, v["vhist"], v["vhist_offsets"], K, VMIN)
    assert rqa.rqa_status(ctx) == 0
    vh = v["vhist"].cpu().numpy()
    off = v["vhist_offsets"]
    eps = sel["eps"].cpu().numpy()
    cle = sel["count_le"].cpu().numpy()
    got = {k: t.cpu().numpy() for k, t in lt.items()}
    vmax, vmass = v["vmax"].cpu().numpy(), v["vmass"].cpu().numpy()
    for s, y in enumerate(ys):
        ne = int(batch.ne[s])
        ref = O.vline_hist(y, m, tau, eps[s], loi=loi)
        h = vh[off[s]:off[s + 1]].reshape(K, -1)
        assert np.array_equal(h, ref["vhist"]), s
        assert np.array_equal(vmax[s], ref["vmax"]), s
        assert np.array_equal(vmass[s].astype(np.int64), 2 * cle[s].astype(np.int64) + (ne if loi else 0)), s
        r = O.lam_tt(ref["vhist"], cle[s], VMIN, ne, loi=loi)
        np.testing.assert_array_equal(got["lam"][s], r["lam"])
        np.testing.assert_array_equal(got["tt"][s], r["tt"])
        np.testing.assert_array_equal(got["lam_avg"][s], O.measure_avg(r["lam"]))
        np.testing.assert_array_equal(got["tt_avg"][s], O.measure_avg(r["tt"]))
    ctx.close()


@pytest.mark.parametrize("schedule", [0, 1])
@pytest.mark.parametrize("m,tau", [(3, 3), (1, 1), (2, 2)])
def test_vertical_lines(rqa_lib, schedule, m, tau):
    _check(rqa_lib, _series(11), m, tau, list(range(1, 21)), schedule, False)


def test_vertical_lines_two_target_groups(rqa_lib):
    _check(rqa_lib, _series(12), 3, 1, list(range(2, 82, 2)), 0, False)  # K = 40: two sweeps


@pytest.mark.parametrize("schedule", [0, 1])
def test_vertical_lines_identity_counted(rqa_lib, schedule):
    ys = [y for y in _series(13) if len(y) > 120]
    _check(rqa_lib, ys, 3, 2, list(range(1, 21)), schedule, True)
