"""CUDA-graph replay of rqa_det_avg and the line-pass autotuner.

A call with the same arguments as the previous one on a caller-owned stream
replays the recorded launch sequence; every decision of the sequence is taken
on the device, so new series values behind the same pointer must give the
oracle's results again, bit for bit."""
import numpy as np
import pytest

from tests._helpers import RR20, oracle_series

pytestmark = pytest.mark.gpu

LMIN = (2, 3, 5)


def _series(seed, sizes):
    rng = np.random.default_rng(seed)
    out = []
    for i, n in enumerate(sizes):
        t = np.arange(n)
        if i % 3 == 0:
            out.append(rng.standard_normal(n).astype(np.float32))
        elif i % 3 == 1:
            out.append((np.sin(2 * np.pi * t / 20.3) + 0.3 * rng.standard_normal(n)).astype(np.float32))
        else:
            x = np.empty(n)
            x[0] = rng.uniform(0.1, 0.9)
            for j in range(1, n):
                x[j] = 4.0 * x[j - 1] * (1.0 - x[j - 1])
            out.append(x.astype(np.float32))
    return out


class _Run:
    """Fixed device buffers for repeated rqa_det_avg calls on one stream."""

    def __init__(self, rqa, ctx, ys, m, tau, stream):
        import torch
        self.rqa, self.ctx, self.stream = rqa, ctx, stream
        with torch.cuda.stream(stream):
            self.batch = rqa.Batch.from_numpy(ys, m, tau)
            S, K = self.batch.n_series, 20
            self.hoff = self.batch.hist_offsets(K)
            self.det = torch.empty((S, K, len(LMIN)), dtype=torch.float64, device="cuda")
            self.avg = torch.empty((S, len(LMIN)), dtype=torch.float64, device="cuda")
            self.eps = torch.empty((S, K), dtype=torch.float32, device="cuda")
            self.hist = torch.empty(int(self.hoff[-1]), dtype=torch.uint64, device="cuda")
            self.lmax = torch.empty((S, K), dtype=torch.uint32, device="cuda")
            self.cnt = torch.empty((S, K), dtype=torch.uint64, device="cuda")
            self.st = torch.empty((S, K), dtype=torch.uint64, device="cuda")
        stream.synchronize()

    def call(self, rr=RR20, lmin=LMIN):
        import torch
        for t in (self.det, self.avg, self.eps, self.hist, self.lmax, self.cnt, self.st):
            with torch.cuda.stream(self.stream):
                t.fill_(7)  # stale values must not survive a replay
        self.rqa.rqa_det_avg(self.ctx, self.batch, rr, 100, None, len(rr), lmin, self.det, self.avg,
                             self.eps, self.hist, self.hoff, self.lmax, self.cnt, self.st)
        self.stream.synchronize()
        code = self.rqa.rqa_status(self.ctx)
        assert code == 0, self.rqa.rqa_error_string(code)
        return {"det": self.det.cpu().numpy(), "det_avg": self.avg.cpu().numpy(),
                "eps": self.eps.cpu().numpy(), "lmax": self.lmax.cpu().numpy(),
                "count": self.cnt.cpu().numpy(), "stencil": self.st.cpu().numpy(),
                "hist": self.rqa.unpack_hist(self.hist.cpu().numpy(), self.hoff, self.batch, 20)}


def _same(a, b):
    """Equal results of two calls (hist is a list of per-series arrays)."""
    assert a.keys() == b.keys()
    for key in a:
        if key == "hist":
            assert len(a[key]) == len(b[key])
            for s, (x, y) in enumerate(zip(a[key], b[key])):
                assert np.array_equal(x, y), (key, s)
        else:
            assert np.array_equal(a[key], b[key]), key


def _against_oracle(res, ys, m, tau):
    for s, y in enumerate(ys):
        ref = oracle_series(y, m, tau, RR20, 100, lmin=LMIN)
        for key in ("eps", "det", "det_avg", "lmax", "count", "stencil"):
            assert np.array_equal(res[key][s], ref[key]), (s, key)
        assert np.array_equal(res["hist"][s], ref["hist"]), s


@pytest.mark.parametrize("schedule", [0, 1])
def test_replay_bit_exact_and_counted(rqa_lib, schedule):
    import torch
    rqa = rqa_lib
    stream = torch.cuda.Stream()
    ys = _series(21, [64, 700, 2500, 5000, 33])
    ctx = rqa.Context(stream=stream, schedule=schedule, select=rqa.RQA_SELECT_RADIX)
    run = _Run(rqa, ctx, ys, 3, 2, stream)
    first = run.call()
    l1 = rqa.rqa_kernel_launches(ctx)
    assert rqa.rqa_graph_replays(ctx) == 0
    for i in range(2):
        _same(run.call(), first)
    assert rqa.rqa_graph_replays(ctx) == 2
    assert rqa.rqa_kernel_launches(ctx) == 3 * l1  # a replay counts the kernels it holds
    _against_oracle(first, ys, 3, 2)
    # the same call with graphs off gives the same bits
    ctx2 = rqa.Context(stream=stream, schedule=schedule, select=rqa.RQA_SELECT_RADIX,
                       flags=rqa.RQA_FLAG_NO_GRAPHS)
    run2 = _Run(rqa, ctx2, ys, 3, 2, stream)
    for _ in range(2):
        _same(run2.call(), first)
    assert rqa.rqa_graph_replays(ctx2) == 0
    ctx.close()
    ctx2.close()


def test_replay_follows_new_values_behind_the_same_pointer(rqa_lib):
    import torch
    rqa = rqa_lib
    stream = torch.cuda.Stream()
    sizes = [900, 3100, 150]
    ys_a, ys_b = _series(5, sizes), _series(6, sizes)
    ctx = rqa.Context(stream=stream, select=rqa.RQA_SELECT_RADIX)
    run = _Run(rqa, ctx, ys_a, 3, 3, stream)
    run.call()
    with torch.cuda.stream(stream):
        run.batch.y.copy_(torch.from_numpy(np.concatenate(ys_b)).cuda())
    res_b = run.call()
    assert rqa.rqa_graph_replays(ctx) == 1
    _against_oracle(res_b, ys_b, 3, 3)
    ctx.close()


def test_changed_arguments_record_again(rqa_lib):
    import torch
    rqa = rqa_lib
    stream = torch.cuda.Stream()
    ys = _series(8, [400, 1200])
    ctx = rqa.Context(stream=stream, select=rqa.RQA_SELECT_RADIX)
    run = _Run(rqa, ctx, ys, 2, 1, stream)
    a = run.call()
    b = run.call(lmin=(2, 4, 6))  # other lmin: a new recording, not a replay
    assert rqa.rqa_graph_replays(ctx) == 0
    assert np.array_equal(a["eps"], b["eps"]) and np.array_equal(a["det"][:, :, 0], b["det"][:, :, 0])
    c = run.call(rr=list(range(2, 22)))  # other targets
    assert rqa.rqa_graph_replays(ctx) == 0
    for s, y in enumerate(ys):
        ref = oracle_series(y, 2, 1, list(range(2, 22)), 100, lmin=LMIN)
        assert np.array_equal(c["eps"][s], ref["eps"]) and np.array_equal(c["det"][s], ref["det"])
    # another call in between (line histograms with other thresholds) moves the
    # plan the recording reads: the next rqa_det_avg must record again
    rqa.line_hist(ctx, run.batch, run.eps, 20)
    d = run.call(rr=list(range(2, 22)))
    assert rqa.rqa_graph_replays(ctx) == 0
    _same(c, d)
    ctx.close()


def test_autotune_picks_a_supported_tile_and_stays_exact(rqa_lib):
    import torch
    rqa = rqa_lib
    stream = torch.cuda.Stream()
    ys = _series(13, [6000, 800, 4000])
    ctx = rqa.Context(stream=stream, select=rqa.RQA_SELECT_RADIX)
    run = _Run(rqa, ctx, ys, 3, 3, stream)
    t = rqa.rqa_autotune(ctx, run.batch, RR20, 100)
    assert t["tile"] in (8, 16, 32) and 0 <= t["unit_bands"] <= 64 and t["line_ctas"] in (0, 6)
    assert t["stage"] in (0, 1)
    assert t["ms"] > 0
    assert rqa.rqa_device_info(ctx)["tile"] == t["tile"]
    assert {k: v for k, v in rqa.rqa_get_tuning(ctx).items() if k != "ms"} == \
        {k: v for k, v in t.items() if k != "ms"}
    res = run.call()
    _against_oracle(res, ys, 3, 3)
    # every knob setting gives the same results: the smallest units, few CTAs
    rqa.rqa_set_tuning(ctx, tile=8, unit_bands=1, line_ctas=1)
    _against_oracle(run.call(), ys, 3, 3)
    rqa.rqa_set_tuning(ctx, tile=32, unit_bands=64, line_ctas=8)
    _against_oracle(run.call(), ys, 3, 3)
    # series windows staged by bulk copies, both windows
    for tile in (16, 32):
        rqa.rqa_set_tuning(ctx, tile=tile, stage=1)
        assert rqa.rqa_get_tuning(ctx)["stage"] == 1
        _against_oracle(run.call(), ys, 3, 3)
    with pytest.raises(rqa.RqaError):
        rqa.rqa_set_tuning(ctx, tile=12)
    with pytest.raises(rqa.RqaError):
        rqa.rqa_set_tuning(ctx, stage=2)
    # a context created with an explicit tile keeps it
    ctx2 = rqa.Context(stream=stream, select=rqa.RQA_SELECT_RADIX, tile=8)
    assert rqa.rqa_autotune(ctx2, run.batch, RR20, 100)["tile"] == 8
    ctx.close()
    ctx2.close()


def test_phase_times_on_replay(rqa_lib):
    """Phase boundaries are event nodes of the recording: a replay times its
    phases like a direct run does."""
    import torch
    rqa = rqa_lib
    stream = torch.cuda.Stream()
    ys = _series(17, [3000, 5000])
    ctx = rqa.Context(stream=stream, select=rqa.RQA_SELECT_RADIX)
    rqa.rqa_set_timing(ctx, True)
    run = _Run(rqa, ctx, ys, 3, 3, stream)
    for i in range(3):
        run.call()
        ms = rqa.rqa_phase_times(ctx)
        assert np.all(ms >= 0) and ms[4] > 0, ms  # the line pass takes time
    assert rqa.rqa_graph_replays(ctx) == 2
    ctx.close()


def test_replay_with_learned_bracket(rqa_lib):
    """The bench configuration: batched schedule, learned bracket, one call
    replayed; bit-identical to a radix-selection run without graphs and to
    the oracle."""
    import os
    import torch
    rqa = rqa_lib
    from paper_2208_09136_gb300 import bracket
    if not os.path.exists(bracket.MODEL_PATH):
        pytest.skip("no trained model file")
    stream = torch.cuda.Stream()
    ys = _series(31, [3000, 700, 5000, 150])
    ctx = rqa.Context(stream=stream, select=rqa.RQA_SELECT_BRACKET)
    bracket.install(ctx)
    run = _Run(rqa, ctx, ys, 3, 3, stream)
    first = run.call()
    for _ in range(2):
        _same(run.call(), first)
    assert rqa.rqa_graph_replays(ctx) == 2
    hits, misses = rqa.rqa_bracket_stats(ctx)
    assert hits + misses == len(ys) * 20
    ref_ctx = rqa.Context(stream=stream, select=rqa.RQA_SELECT_RADIX, flags=rqa.RQA_FLAG_NO_GRAPHS)
    _same(_Run(rqa, ref_ctx, ys, 3, 3, stream).call(), first)
    _against_oracle(first, ys, 3, 3)
    ctx.close()
    ref_ctx.close()
