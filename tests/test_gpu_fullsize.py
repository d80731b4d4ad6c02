"""Full-size parity on the 296-series workload, in the configuration bench.py
times (batched schedule, learned bracket, one rqa_det_avg call with line
outputs): every short series against the oracle in full; long series
(N = 10^5, 5*10^9 cells each) through the oracle's streaming selection
certificate on a sample, one of them through the oracle's full line scan,
and all of them through invariants that hold at any size."""
import numpy as np
import pytest

from tests._helpers import RR20, oracle_series

pytestmark = pytest.mark.gpu

LMIN = (2, 3, 5)


@pytest.fixture(scope="module")
def full_run(rqa_lib):
    import torch
    rqa = rqa_lib
    from paper_2208_09136_gb300 import bracket
    from synth import workload
    w = workload("full-296")
    flat, offsets, m, tau = w.pack()
    ctx = rqa.Context(device=0, select=rqa.RQA_SELECT_BRACKET)
    bracket.install(ctx)
    y = torch.from_numpy(flat).cuda()
    batch = rqa.Batch(y, offsets, m, tau)
    out = rqa.det_avg(ctx, batch, RR20, 100, lmin=LMIN, lines=True)
    assert rqa.rqa_status(ctx) == 0
    hits, misses = rqa.rqa_bracket_stats(ctx)
    sel = rqa.eps_for_rr(ctx, batch, RR20, 100)  # the selection alone, for its own counts
    assert rqa.rqa_status(ctx) == 0
    res = {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in out.items()}
    res["sel_eps"] = sel["eps"].cpu().numpy()
    res["sel_le"] = sel["count_le"].cpu().numpy()
    res["sel_lt"] = sel["count_lt"].cpu().numpy()
    res["hist_list"] = rqa.unpack_hist(res["hist"], res["hist_offsets"], batch, 20)
    ctx.close()
    return w, flat, offsets, m, tau, res, (hits, misses)


def test_bracket_statistics(full_run):
    _, _, offsets, _, _, res, (hits, misses) = full_run
    assert hits + misses == (len(offsets) - 1) * 20
    assert misses / (hits + misses) < 0.05


def test_line_mass_equals_selection_count(full_run):
    """C_k from the line pass (sum of l P_k(l)) against the selection's own
    #{d <= eps_k}, and the counting certificate #{d < eps_k} < T_k <= C_k,
    on every series: two independent counts of the same recurrent cells."""
    _, _, offsets, m, tau, res, _ = full_run
    assert np.array_equal(res["sel_eps"], res["eps"])
    assert np.array_equal(res["sel_le"], res["count"])
    for s in range(len(offsets) - 1):
        ne = int(offsets[s + 1] - offsets[s]) - (int(m[s]) - 1) * int(tau[s])
        P = ne * (ne - 1) // 2
        T = np.array([-((-r * P) // 100) for r in RR20], dtype=np.uint64)
        assert np.all(res["sel_lt"][s] < T) and np.all(T <= res["sel_le"][s]), s


def test_invariants_every_series(full_run):
    _, _, offsets, m, tau, res, _ = full_run
    for s in range(len(offsets) - 1):
        h = res["hist_list"][s].astype(np.int64)
        L = np.arange(1, h.shape[1] + 1, dtype=np.int64)
        mass = (h * L[None, :]).sum(axis=1)
        C = res["count"][s].astype(np.int64)
        assert np.array_equal(mass, C), s                                   # sum l P(l) = C_k
        assert np.array_equal(res["stencil"][s].astype(np.int64), C - h[:, 0]), s  # S = C - P(1)
        lmax = np.array([np.nonzero(row)[0].max() + 1 if row.any() else 0 for row in h])
        assert np.array_equal(res["lmax"][s].astype(np.int64), lmax), s
        assert np.all(np.diff(res["eps"][s]) >= 0) and np.all(np.diff(C) >= 0), s
        ne = int(offsets[s + 1] - offsets[s]) - (int(m[s]) - 1) * int(tau[s])
        P = ne * (ne - 1) // 2
        T = np.array([-((-r * P) // 100) for r in RR20])
        assert np.all(C >= T), s
        for j, lm in enumerate(LMIN):
            num = (h[:, lm - 1:] * L[None, lm - 1:]).sum(axis=1)
            assert np.array_equal(res["det"][s][:, j], num.astype(np.float64) / C.astype(np.float64))
        avg = np.zeros(len(LMIN))
        for k in range(20):
            avg = avg + res["det"][s][k]
        assert np.array_equal(res["det_avg"][s], avg / 20.0)


def test_short_series_against_oracle(full_run):
    _, flat, offsets, m, tau, res, _ = full_run
    n = np.diff(offsets)
    for s in np.nonzero(n < 20000)[0]:
        y = flat[offsets[s]:offsets[s + 1]]
        ref = oracle_series(y, int(m[s]), int(tau[s]), RR20, 100, lmin=LMIN)
        assert np.array_equal(res["eps"][s], ref["eps"]), s
        assert np.array_equal(res["count"][s], ref["count"]), s
        assert np.array_equal(res["hist_list"][s], ref["hist"]), s
        assert np.array_equal(res["det"][s], ref["det"]), s
        assert np.array_equal(res["det_avg"][s], ref["det_avg"]), s


def test_long_series_sampled_against_oracle(full_run):
    """One long series per signal type and SNR (24 of the 96): thresholds
    proven exact by the oracle's counting certificate #{d < eps} < T <=
    #{d <= eps} (and C_k equal to the oracle's count); the 0 dB sine series
    also through the oracle's full diagonal scan (histograms, stencil,
    L_max)."""
    from oracle import c_oracle as CO
    w, flat, offsets, m, tau, res, _ = full_run
    snrs = sorted({sp.snr_db for sp in w.specs if sp.n == 100_000})
    assert len(snrs) == 8
    picks = []
    for kind in ("sine", "logistic", "lorenz"):
        for snr in ([0.0] + [v for v in snrs if v != 0.0]):
            picks.append(next(i for i, sp in enumerate(w.specs) if sp.kind == kind and sp.n == 100_000
                              and sp.snr_db == snr))
    for idx, s in enumerate(picks):
        y = flat[offsets[s]:offsets[s + 1]]
        ne = len(y) - (int(m[s]) - 1) * int(tau[s])
        P = ne * (ne - 1) // 2
        T = np.array([-((-r * P) // 100) for r in RR20], dtype=np.int64)
        le, lt = CO.count(y, int(m[s]), int(tau[s]), res["eps"][s])
        assert np.all(lt.astype(np.int64) < T) and np.all(T <= le.astype(np.int64)), s
        assert np.array_equal(le, res["count"][s]), s
        if idx == 0:
            L = CO.lines(y, int(m[s]), int(tau[s]), res["eps"][s], full_hist=True)
            assert np.array_equal(L["hist"], res["hist_list"][s])
            assert np.array_equal(L["stencil"], res["stencil"][s])
            assert np.array_equal(L["lmax"], res["lmax"][s])
