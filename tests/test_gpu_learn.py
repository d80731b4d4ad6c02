"""GPU checks of the learned bracket: sketch, network forward/backward and
Adam against the FP64 oracle, and exactness of bracketed selection (with an
untrained and, when present, the trained network)."""
import os

import numpy as np
import pytest

from oracle import mlp_oracle as MO
from tests._helpers import RR20, oracle_series

pytestmark = pytest.mark.gpu


def _series(seed, sizes, kind="mix"):
    rng = np.random.default_rng(seed)
    out = []
    for i, n in enumerate(sizes):
        t = np.arange(n)
        if i % 2:
            out.append(rng.standard_normal(n).astype(np.float32))
        else:
            out.append((np.sin(2 * np.pi * t / 20.3) + 0.2 * rng.standard_normal(n)).astype(np.float32))
    return out


def test_sketch_matches_oracle(rqa_lib):
    import torch
    rqa = rqa_lib
    ys = _series(1, [50, 300, 1000, 4097, 20000])
    ctx = rqa.Context()
    batch = rqa.Batch.from_numpy(ys, [3, 1, 3, 2, 3], [3, 1, 1, 5, 3])
    S = batch.n_series
    feats = torch.empty((S, 131), dtype=torch.float32, device="cuda")
    centre = torch.empty(S, dtype=torch.float32, device="cuda")
    qd = torch.empty((S, 128), dtype=torch.float32, device="cuda")
    rqa.rqa_sketch(ctx, batch, 12345, feats, centre, qd)
    assert rqa.rqa_status(ctx) == 0
    f, c, q = feats.cpu().numpy(), centre.cpu().numpy(), qd.cpu().numpy()
    for s in range(S):
        x, cc, qq = MO.sketch_features(ys[s], int(batch.m[s]), int(batch.tau[s]), s, 12345)
        assert np.array_equal(q[s], qq)                 # sampled distances: exact
        assert abs(c[s] - cc) <= 2e-6 * max(1.0, abs(cc))
        assert np.allclose(f[s], x, rtol=1e-5, atol=2e-6)


def _oracle_params(seed=3):
    return MO.init_params(seed)


def test_mlp_forward_backward_adam(rqa_lib):
    import torch
    rqa = rqa_lib
    ctx = rqa.Context()
    rng = np.random.default_rng(9)
    compared = 0
    for B in (1, 37, 256, 300):
        p = (_oracle_params() * 0.5).astype(np.float32)
        X = rng.standard_normal((B, 131)).astype(np.float32)
        T = rng.standard_normal((B, 20)).astype(np.float32)
        dp = torch.from_numpy(p).cuda()
        dX = torch.from_numpy(X).cuda()
        dT = torch.from_numpy(T).cuda()
        Y = torch.empty((B, 40), dtype=torch.float32, device="cuda")
        acts = torch.empty((B, 512), dtype=torch.float32, device="cuda")
        rqa.rqa_mlp_forward(ctx, dp, dX, Y, acts)
        ref = MO.forward(p, X)
        y = Y.cpu().numpy()
        scale = np.abs(ref["Y"]).max()
        assert np.abs(y - ref["Y"]).max() <= 1e-5 * scale + 1e-6
        flat = acts.cpu().numpy().ravel()
        h1, h2 = flat[:B * 256].reshape(B, 256), flat[B * 256:].reshape(B, 256)  # H1 block, H2 block
        assert np.allclose(h1, ref["H1"], rtol=1e-4, atol=1e-5 * np.abs(ref["H1"]).max())
        assert np.allclose(h2, ref["H2"], rtol=1e-4, atol=1e-5 * np.abs(ref["H2"]).max())
        g = torch.empty_like(dp)
        loss = torch.empty(1, dtype=torch.float32, device="cuda")
        rqa.rqa_mlp_backward(ctx, dp, dX, acts, Y, dT, 0.05, 0.95, g, loss)
        rl, rg = MO.backward(p, X, T, 0.05, 0.95)
        gg = g.cpu().numpy()
        assert abs(float(loss.item()) - rl) <= 1e-4 * max(1.0, abs(rl))
        # A unit whose pre-activation rounds to the other side of zero in FP32
        # (or an output exactly on a loss kink) changes the gradient by design;
        # compare only batches where both sides took the same branches.
        same = (np.array_equal(h1 > 0, ref["H1"] > 0) and
                np.array_equal(h2 > 0, ref["H2"] > 0) and
                np.array_equal(np.repeat(T, 2, axis=1) >= y, np.repeat(T, 2, axis=1) >= ref["Y"]))
        if same:
            compared += 1
            assert np.abs(gg - rg).max() <= 2e-4 * np.abs(rg).max() + 1e-7
        # one Adam step
        m = torch.zeros_like(dp)
        v = torch.zeros_like(dp)
        p2 = dp.clone()
        rqa.rqa_adam_step(ctx, p2, g, m, v, 1, 1e-3)
        ref_p, _, _ = MO.adam(p.astype(np.float64), gg.astype(np.float64), 0.0, 0.0, 1, lr=1e-3)
        assert np.allclose(p2.cpu().numpy(), ref_p, rtol=1e-5, atol=1e-6)
    assert compared >= 3
    assert rqa.rqa_status(ctx) == 0


def _select(rqa, ys, m, tau, model, schedule=0):
    import torch
    ctx = rqa.Context(schedule=schedule, select=rqa.RQA_SELECT_BRACKET if model is not None
                      else rqa.RQA_SELECT_RADIX)
    if model is not None:
        rqa.rqa_set_bracket_model(ctx, torch.from_numpy(model).cuda(), 0.05)
    batch = rqa.Batch.from_numpy(ys, m, tau)
    out = rqa.eps_for_rr(ctx, batch, RR20, 100)
    da = rqa.det_avg(ctx, batch, RR20, 100, lmin=(2, 3, 5))
    code = rqa.rqa_status(ctx)
    assert code == 0, rqa.rqa_error_string(code)
    stats = rqa.rqa_bracket_stats(ctx) if model is not None else None
    res = {k: v.cpu().numpy() for k, v in out.items()}
    res.update(det=da["det"].cpu().numpy(), det_avg=da["det_avg"].cpu().numpy())
    ctx.close()
    return res, stats


@pytest.mark.parametrize("schedule", [0, 1])
def test_bracketed_selection_exact_with_untrained_model(rqa_lib, schedule):
    """A random network misses most intervals: every threshold must still be
    exact (the full selection takes over)."""
    ys = _series(4, [120, 900, 3000, 7000, 64])
    model = MO.init_params(11)
    got, (hits, misses) = _select(rqa_lib, ys, 3, 3, model, schedule)
    base, _ = _select(rqa_lib, ys, 3, 3, None, schedule)
    for key in ("eps", "count_le", "count_lt", "det", "det_avg"):
        assert np.array_equal(got[key], base[key]), key
    assert hits + misses == len(ys) * 20
    for s, y in enumerate(ys):
        ref = oracle_series(y, 3, 3, RR20, 100, lmin=(2, 3, 5), full_hist=False)
        assert np.array_equal(got["eps"][s], ref["eps"])
        assert np.array_equal(got["det"][s], ref["det"])


def test_bracket_rejects_other_targets(rqa_lib):
    import torch
    rqa = rqa_lib
    ctx = rqa.Context(select=rqa.RQA_SELECT_BRACKET)
    batch = rqa.Batch.from_numpy(_series(2, [200]), 3, 3)
    with pytest.raises(rqa.RqaError) as ei:
        rqa.eps_for_rr(ctx, batch, RR20, 100)
    assert ei.value.code == 9  # no model installed
    rqa.rqa_set_bracket_model(ctx, torch.from_numpy(MO.init_params(1)).cuda(), 0.0)
    with pytest.raises(rqa.RqaError):
        rqa.eps_for_rr(ctx, batch, list(range(1, 11)), 100)  # the network predicts 20 targets
    ctx.close()


def test_trained_model_hits_and_stays_exact(rqa_lib):
    """The trained network on held-out long Lorenz series (N = 10^5,
    m = tau = 3, SNR -10/0/10 dB): thresholds equal the radix selection bit
    for bit and are proven exact by the oracle's counting certificate
    #{d < eps_k} < T_k <= #{d <= eps_k} (one streaming pass over the 5*10^9
    cells of each series, no sort), and most intervals hold (each miss costs
    the full selection for its series)."""
    from oracle import c_oracle as CO
    from paper_2208_09136_gb300 import bracket
    if not os.path.exists(bracket.MODEL_PATH):
        pytest.skip("no trained model file")
    from synth import workload
    w = workload("lorenz-n1e5-eval")
    ys = w.series()
    model = bracket.load_model()["params"]
    got, (hits, misses) = _select(rqa_lib, ys, 3, 3, model)
    base, _ = _select(rqa_lib, ys, 3, 3, None)
    for key in ("eps", "count_le", "count_lt", "det", "det_avg"):
        assert np.array_equal(got[key], base[key]), key
    assert hits + misses == 60
    assert hits >= 54, (hits, misses)
    for s, y in enumerate(ys):
        ne = len(y) - 6
        P = ne * (ne - 1) // 2
        T = np.array([-((-r * P) // 100) for r in RR20], dtype=np.int64)
        le, lt = CO.count(y, 3, 3, got["eps"][s])
        assert np.all(lt.astype(np.int64) < T) and np.all(T <= le.astype(np.int64)), s
        assert np.array_equal(le, got["count_le"][s]) and np.array_equal(lt, got["count_lt"][s]), s


def _timed_det_avg(rqa, ys, m, tau, learned, reps=2):
    """Phase times (ms) of rqa_det_avg in the batched schedule, the fastest of
    reps calls, and the call's outputs."""
    import torch
    from paper_2208_09136_gb300 import bracket
    stream = torch.cuda.Stream()
    ctx = rqa.Context(stream=stream, select=rqa.RQA_SELECT_AUTO if learned else rqa.RQA_SELECT_RADIX)
    if learned:
        bracket.install(ctx)
    rqa.rqa_set_timing(ctx, True)
    with torch.cuda.stream(stream):
        batch = rqa.Batch.from_numpy(ys, m, tau)
    best = None
    for _ in range(reps + 1):
        with torch.cuda.stream(stream):
            out = rqa.det_avg(ctx, batch, RR20, 100, lmin=(2, 3, 5))
        stream.synchronize()
        ph = rqa.rqa_phase_times(ctx)
        best = ph if best is None else np.minimum(best, ph)
    assert rqa.rqa_status(ctx) == 0
    stats = rqa.rqa_bracket_stats(ctx) if learned else None
    res = {k: v.cpu().numpy() for k, v in out.items()}
    ctx.close()
    return best, res, stats


def test_trained_model_gain_on_long_series(rqa_lib):
    """What the trained network buys on the held-out long series: with its
    intervals the selection skips the middle counting pass (its phase does no
    work) and takes less time in all than the radix selection of the same
    batched schedule, with identical outputs."""
    from paper_2208_09136_gb300 import bracket
    if not os.path.exists(bracket.MODEL_PATH):
        pytest.skip("no trained model file")
    from synth import workload
    ys = workload("lorenz-n1e5-eval").series()
    rad, r_out, _ = _timed_det_avg(rqa_lib, ys, 3, 3, False)
    lrn, l_out, (hits, misses) = _timed_det_avg(rqa_lib, ys, 3, 3, True)
    for key in ("eps", "det", "det_avg"):
        assert np.array_equal(l_out[key], r_out[key]), key
    assert hits == 60 and misses == 0, (hits, misses)
    # phases: [1] coarse or bracket round + select, [2] middle round, [3] final round
    assert lrn[2] < 0.05 * rad[2], (lrn, rad)
    assert lrn[1] + lrn[2] + lrn[3] < rad[1] + rad[2] + rad[3], (lrn, rad)


def test_auto_selection_keeps_to_the_training_domain(rqa_lib):
    """RQA_SELECT_AUTO brackets only series whose embedding the network was
    trained on (m = tau = 3 here): a batch of other embeddings runs the plain
    selection (no bracketed target counted), a mixed batch brackets exactly
    its m = tau = 3 series; results equal the radix selection bit for bit."""
    import torch
    rqa = rqa_lib
    from paper_2208_09136_gb300 import bracket
    if not os.path.exists(bracket.MODEL_PATH):
        pytest.skip("no trained model file")
    assert bracket.load_model()["domain"] == [(3, 3)]
    ys = _series(41, [400, 2500, 1200, 800])
    for m, tau, n_in in (([1, 1, 1, 1], [1, 1, 1, 1], 0), ([3, 3, 3, 3], [1, 1, 1, 1], 0),
                         ([3, 3, 3, 1], [3, 1, 3, 1], 2)):
        ctx = rqa.Context(select=rqa.RQA_SELECT_AUTO)
        bracket.install(ctx)
        batch = rqa.Batch.from_numpy(ys, m, tau)
        got = rqa.eps_for_rr(ctx, batch, RR20, 100)
        hits, misses = rqa.rqa_bracket_stats(ctx)
        assert rqa.rqa_status(ctx) == 0
        assert hits + misses == 20 * n_in, (m, tau, hits, misses)
        ref_ctx = rqa.Context(select=rqa.RQA_SELECT_RADIX)
        ref = rqa.eps_for_rr(ref_ctx, batch, RR20, 100)
        for key in ("eps", "count_le", "count_lt"):
            assert np.array_equal(got[key].cpu().numpy(), ref[key].cpu().numpy()), (key, m, tau)
        ctx.close()
        ref_ctx.close()
    # the domain can be lifted: every series is bracketed again
    ctx = rqa.Context(select=rqa.RQA_SELECT_AUTO)
    bracket.install(ctx)
    rqa.rqa_set_bracket_domain(ctx, [])
    rqa.eps_for_rr(ctx, rqa.Batch.from_numpy(ys, 1, 1), RR20, 100)
    assert sum(rqa.rqa_bracket_stats(ctx)) == 80
    ctx.close()


def test_training_arithmetic_kernels(rqa_lib):
    """The label, validation and gather kernels the trainer uses, against
    NumPy: labels ln(max(eps, 2^-126)) - c within FP32 rounding of the
    logarithm, the inside count exactly (the same FP32 comparisons), the loss
    and width sums to double rounding, the gather exactly."""
    import torch
    rqa = rqa_lib
    rng = np.random.default_rng(17)
    ctx = rqa.Context()
    S, K = 300, 20
    eps = (np.exp(rng.uniform(-9, 2, (S, K))) * (rng.random((S, K)) > 0.01)).astype(np.float32)
    centre = rng.uniform(-3, 1, S).astype(np.float32)
    T = torch.empty((S, K), dtype=torch.float32, device="cuda")
    rqa.rqa_log_labels(ctx, torch.from_numpy(eps).cuda(), torch.from_numpy(centre).cuda(), T)
    ref = np.log(np.maximum(eps.astype(np.float64), 2.0 ** -126)) - centre[:, None].astype(np.float64)
    got = T.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(got - ref) <= 4e-7 * np.maximum(1.0, np.abs(ref)))
    # validation sums over rows of predictions
    B = 257
    Y = rng.standard_normal((B, 2 * K)).astype(np.float32)
    Y[:, 1::2] = Y[:, 0::2] + np.abs(Y[:, 1::2])
    Tt = rng.standard_normal((B, K)).astype(np.float32)
    out = (torch.empty(1, dtype=torch.float64, device="cuda"),
           torch.empty(1, dtype=torch.uint64, device="cuda"),
           torch.empty(1, dtype=torch.float64, device="cuda"))
    tl, th, mg = np.float32(0.005), np.float32(0.995), np.float32(0.05)
    rqa.rqa_bracket_eval(ctx, torch.from_numpy(Y).cuda(), torch.from_numpy(Tt).cuda(), float(tl),
                         float(th), float(mg), out)
    loss, inside, width = (v.cpu().item() for v in out)
    lo, hi = Y[:, 0::2], Y[:, 1::2]
    rl, rh = Tt - lo, Tt - hi
    pl = np.where(rl >= 0, tl * rl, (tl - np.float32(1)) * rl).astype(np.float64)
    ph = np.where(rh >= 0, th * rh, (th - np.float32(1)) * rh).astype(np.float64)
    assert abs(loss - (pl.sum() + ph.sum())) <= 1e-9 * max(1.0, abs(loss))
    assert inside == int(((Tt >= lo - mg) & (Tt <= hi + mg)).sum())
    assert abs(width - ((hi + mg) - (lo - mg)).astype(np.float64).sum()) <= 1e-9 * abs(width)
    # gather
    idx = rng.integers(0, S, 77)
    src = rng.standard_normal((S, 131)).astype(np.float32)
    dst = torch.empty((77, 131), dtype=torch.float32, device="cuda")
    rqa.rqa_gather_rows(ctx, torch.from_numpy(src).cuda(), torch.from_numpy(idx).cuda(), dst)
    assert np.array_equal(dst.cpu().numpy(), src[idx])
    assert rqa.rqa_status(ctx) == 0
    ctx.close()
