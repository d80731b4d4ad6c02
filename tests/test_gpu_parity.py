"""GPU parity: the CUDA path through the C ABI against the CPU oracle, bit for
bit (thresholds, counts, line histograms, DET and its average)."""
import numpy as np
import pytest

from tests._helpers import RR20, assert_series_equal, gpu_run, oracle_series

pytestmark = pytest.mark.gpu

SCHEDS = [0, 1]  # batched persistent launch, per-series launches


@pytest.mark.parametrize("schedule", SCHEDS)
def test_logistic_n100(rqa_lib, schedule):
    from synth import workload
    w = workload("logistic-n100")
    ys = w.series()
    sp = w.specs[0]
    g = gpu_run(ys, sp.m, sp.tau, RR20, 100, lmin=(2, 3, 5), schedule=schedule)
    ref = oracle_series(ys[0], sp.m, sp.tau, RR20, 100, lmin=(2, 3, 5))
    assert_series_equal(g, 0, ref, "logistic-n100")


@pytest.mark.parametrize("n,m,tau", [(2, 1, 1), (3, 1, 1), (3, 2, 1), (5, 2, 3), (33, 1, 1),
                                     (34, 1, 1), (65, 3, 1), (97, 4, 2), (130, 5, 3)])
def test_tiny_and_ragged_lengths(rqa_lib, n, m, tau):
    rng = np.random.default_rng(n * 100 + m * 10 + tau)
    ys = [rng.standard_normal(n).astype(np.float32)]
    rr = [1, 10, 25, 50, 75, 99]
    g = gpu_run(ys, m, tau, rr, 100, lmin=(1, 2, 3, 5))
    ref = oracle_series(ys[0], m, tau, rr, 100, lmin=(1, 2, 3, 5))
    assert_series_equal(g, 0, ref, f"n={n}")


def test_constant_ramp_sawtooth(rqa_lib):
    ys = [np.full(300, 1.25, np.float32), np.arange(200, dtype=np.float32),
          (np.arange(250) % 7).astype(np.float32), np.zeros(40, np.float32)]
    for m, tau in [(1, 1), (3, 2)]:
        g = gpu_run(ys, m, tau, RR20, 100, lmin=(2, 3, 5))
        for s, y in enumerate(ys):
            ref = oracle_series(y, m, tau, RR20, 100, lmin=(2, 3, 5))
            assert_series_equal(g, s, ref, f"closed-form m={m}")
        # constant series: one line of every length, DET = 1 - lmin(lmin-1)/2/P
        ne = 300 - (m - 1) * tau
        p = ne * (ne - 1) // 2
        assert np.all(g["hist"][0] == 1)
        assert g["det"][0, 0, 0] == (p - 1) / p


@pytest.mark.parametrize("schedule", SCHEDS)
def test_mixed_batch_generic_path(rqa_lib, schedule):
    """Uneven lengths, mixed m and tau (generic distance path), exact ties."""
    rng = np.random.default_rng(77)
    ys, ms, taus = [], [], []
    for i in range(40):
        m = int(rng.integers(1, 7))
        tau = int(rng.integers(1, 5))
        n = int(rng.integers((m - 1) * tau + 2, 420))
        y = rng.standard_normal(n)
        if i % 3 == 0:
            y = np.round(y * 2) / 2  # coarse values: many tied distances
        ys.append(y.astype(np.float32))
        ms.append(m)
        taus.append(tau)
    g = gpu_run(ys, ms, taus, RR20, 100, lmin=(2, 3, 5), schedule=schedule)
    for s, y in enumerate(ys):
        ref = oracle_series(y, ms[s], taus[s], RR20, 100, lmin=(2, 3, 5))
        assert_series_equal(g, s, ref, "mixed")


@pytest.mark.parametrize("m,tau", [(1, 1), (2, 1), (3, 1), (3, 3), (4, 2), (5, 1)])
def test_uniform_embedding_paths(rqa_lib, m, tau):
    rng = np.random.default_rng(m * 7 + tau)
    t = np.arange(700)
    ys = [(np.sin(2 * np.pi * t / 20.3) + 0.3 * rng.standard_normal(700)).astype(np.float32),
          rng.standard_normal(513).astype(np.float32)]
    g = gpu_run(ys, m, tau, RR20, 100, lmin=(2, 3, 5))
    for s, y in enumerate(ys):
        assert_series_equal(g, s, oracle_series(y, m, tau, RR20, 100, lmin=(2, 3, 5)), f"m={m}")


@pytest.mark.parametrize("rr,den", [([50], 100), (list(range(1, 32)), 100), ([1, 99], 100),
                                    ([1, 2, 3], 7), (list(range(3, 97, 3)), 100)])
def test_threshold_counts(rqa_lib, rr, den):
    rr = rr[:31]
    rng = np.random.default_rng(len(rr))
    ys = [rng.standard_normal(400).astype(np.float32),
          (np.round(rng.standard_normal(300) * 3) / 3).astype(np.float32)]
    g = gpu_run(ys, 2, 1, rr, den, lmin=(2,))
    for s, y in enumerate(ys):
        assert_series_equal(g, s, oracle_series(y, 2, 1, rr, den, lmin=(2,)), f"K={len(rr)}")


def test_long_lines_global_histogram(rqa_lib):
    """Noise-free sine: diagonal lines far longer than the shared-memory part of
    the histogram, so the long-line path to global memory is exercised."""
    t = np.arange(3000)
    ys = [np.sin(2 * np.pi * t / 20.3).astype(np.float32)]
    g = gpu_run(ys, 3, 1, RR20, 100, lmin=(2, 3, 5))
    ref = oracle_series(ys[0], 3, 1, RR20, 100, lmin=(2, 3, 5))
    assert ref["lmax"].max() > 500
    assert_series_equal(g, 0, ref, "sine")


@pytest.mark.parametrize("schedule", SCHEDS)
def test_lorenz_n1e4(rqa_lib, schedule):
    from synth import workload
    w = workload("lorenz-n1e4")
    ys = w.series()
    sp = w.specs[0]
    g = gpu_run(ys, sp.m, sp.tau, RR20, 100, lmin=(2, 3, 5), schedule=schedule)
    picks = range(4) if schedule == 0 else [3]
    for s in picks:
        ref = oracle_series(ys[s], sp.m, sp.tau, RR20, 100, lmin=(2, 3, 5))
        assert_series_equal(g, s, ref, "lorenz-n1e4")


def test_batched_720_sampled(rqa_lib):
    """The 720-series uneven batch in one persistent launch per phase; every
    N=100 and N=1000 series and a sample of the N=10^4 series vs the oracle."""
    from synth import workload
    w = workload("batched-720")
    ys = w.series()
    g = gpu_run(ys, 3, 1, RR20, 100, lmin=(2,), hist=False)
    rng = np.random.default_rng(0)
    big = [i for i, sp in enumerate(w.specs) if sp.n == 10_000]
    picks = [i for i, sp in enumerate(w.specs) if sp.n < 10_000] + list(rng.choice(big, 4, replace=False))
    for s in picks:
        ref = oracle_series(ys[s], 3, 1, RR20, 100, lmin=(2,), full_hist=False)
        assert_series_equal(g, s, ref, "batched-720")


def test_schedules_agree_bitwise(rqa_lib):
    rng = np.random.default_rng(5)
    ys = [rng.standard_normal(int(n)).astype(np.float32) for n in rng.integers(50, 3000, 12)]
    a = gpu_run(ys, 3, 2, RR20, 100, lmin=(2, 3), schedule=0)
    b = gpu_run(ys, 3, 2, RR20, 100, lmin=(2, 3), schedule=1)
    for key in ("eps", "count_le", "count_lt", "det", "det_avg", "lmax", "count", "stencil"):
        assert np.array_equal(a[key], b[key]), key
    for s in range(len(ys)):
        assert np.array_equal(a["hist"][s], b["hist"][s])


def test_det_nan_without_recurrences(rqa_lib):
    """Caller thresholds below every distance leave C_k = 0: DET_k is then 0/0,
    NaN on both sides, and so is the average over the targets; the other
    targets and series stay finite and bit-exact."""
    import torch
    import paper_2208_09136_gb300 as rqa
    from oracle import rqa_oracle as O
    rng = np.random.default_rng(21)
    ys = [np.cumsum(rng.uniform(1.0, 2.0, 300)).astype(np.float32),  # every |step| >= 1
          rng.standard_normal(500).astype(np.float32)]
    eps_np = np.array([[0.5, 3.0], [0.05, 0.2]], dtype=np.float32)
    ctx = rqa.Context(device=0)
    batch = rqa.Batch.from_numpy(ys, 1, 1)
    eps = torch.from_numpy(eps_np).cuda()
    out = rqa.det_avg(ctx, batch, None, 0, lmin=(2, 3), eps=eps, K=2, lines=True)
    assert rqa.rqa_status(ctx) == 0
    det = out["det"].cpu().numpy()
    avg = out["det_avg"].cpu().numpy()
    for s, y in enumerate(ys):
        lines = O.line_hist(y, 1, 1, eps_np[s])
        ref = O.det_from_hist(lines["hist"], lines["count"], (2, 3))
        assert np.array_equal(det[s], ref, equal_nan=True), (s, det[s], ref)
        assert np.array_equal(avg[s], O.det_avg(ref), equal_nan=True)
        assert np.array_equal(out["count"].cpu().numpy()[s], lines["count"])
    assert np.isnan(det[0, 0]).all() and np.isfinite(det[0, 1]).all()
    ctx.close()


def test_device_errors_reported(rqa_lib):
    import torch
    import paper_2208_09136_gb300 as rqa
    ctx = rqa.Context(device=0)
    y = np.random.default_rng(1).standard_normal(100).astype(np.float32)
    batch = rqa.Batch.from_numpy([y], 1, 1)
    # unsorted thresholds supplied by the caller
    eps = torch.tensor([[0.5, 0.2]], dtype=torch.float32, device="cuda")
    rqa.line_hist(ctx, batch, eps, 2)
    assert rqa.rqa_status(ctx) == 8
    # NaN in the series
    y2 = y.copy()
    y2[17] = np.nan
    batch2 = rqa.Batch.from_numpy([y2], 1, 1)
    rqa.eps_for_rr(ctx, batch2, [1, 2], 100)
    assert rqa.rqa_status(ctx) == 3
    assert rqa.rqa_status(ctx) == 0  # cleared after reading
    # host-side validation
    for bad, den in (([0], 100), ([5, 5], 100), ([100], 100), (list(range(1, 129)), 1000)):
        with pytest.raises(rqa.RqaError):  # zero, repeated, = den, K > RQA_K_MAX
            rqa.eps_for_rr(ctx, batch, bad, den)
    short = rqa.Batch.from_numpy([y[:4]], 3, 2)  # Ne = 0
    with pytest.raises(rqa.RqaError) as ei:
        rqa.eps_for_rr(ctx, short, [1, 2], 100)
    assert ei.value.code == 2
    ctx.close()


@pytest.mark.parametrize("schedule", SCHEDS)
def test_rr_up_to_99(rqa_lib, schedule):
    """RR = 1..99 % (Sect. 2 averages up to RR* = 99): 99 targets per call,
    middle round in windows of 48 groups and the line pass in five sweeps of
    at most 20 targets; bit-exact against the oracle."""
    rng = np.random.default_rng(99)
    ys = [rng.standard_normal(300).astype(np.float32),
          (np.sin(2 * np.pi * np.arange(1500) / 20.3) + 0.3 * rng.standard_normal(1500)).astype(np.float32),
          (np.arange(120) % 9).astype(np.float32)]
    rr = list(range(1, 100))
    g = gpu_run(ys, 3, 2, rr, 100, lmin=(2, 3, 5), schedule=schedule)
    for s, y in enumerate(ys):
        ref = oracle_series(y, 3, 2, rr, 100, lmin=(2, 3, 5))
        assert_series_equal(g, s, ref, "RR 1..99")


@pytest.mark.parametrize("K", [20, 21, 31, 32, 40, 41, 62, 63, 127])
def test_target_count_group_boundaries(rqa_lib, K):
    """K around the 20-target line-pass sweeps, the 31-target fixed-scratch
    limit and the 48-group middle-round windows, up to K = RQA_K_MAX = 127
    (rr_den = 128)."""
    rng = np.random.default_rng(K)
    ys = [rng.standard_normal(400).astype(np.float32), rng.standard_normal(77).astype(np.float32)]
    rr = list(range(1, K + 1))
    g = gpu_run(ys, 2, 1, rr, 128, lmin=(2, 4))
    for s, y in enumerate(ys):
        ref = oracle_series(y, 2, 1, rr, 128, lmin=(2, 4))
        assert_series_equal(g, s, ref, f"K={K}")


def test_noalloc_rejects_more_than_31_targets(rqa_lib):
    import torch
    rqa = rqa_lib
    batch = rqa.Batch.from_numpy([np.ones(50, np.float32)], 1, 1)
    eps = torch.empty(32, dtype=torch.float32, device="cuda")
    with pytest.raises(rqa.RqaError):
        rqa.rqa_eps_for_rr_noalloc(batch, list(range(1, 33)), 100, eps)
