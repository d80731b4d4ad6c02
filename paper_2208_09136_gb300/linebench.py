"""Time the line pass alone on a named workload.

``python -m paper_2208_09136_gb300.linebench WORKLOAD [REPS] [TILE] [STAGE]``

Builds the workload's batch on cuda:0, selects the thresholds for RR = 1..20 %
once (``rqa_eps_for_rr``, radix selection), then runs ``rqa_line_hist`` (full
histograms) REPS times, each timed with CUDA events on the context's stream,
and prints one line per run.  TILE fixes the cell phase's register window
(8, 16 or 32; 0 = the default); STAGE = 1 stages the series windows in
shared memory by bulk copies (where the variant exists).  Besides the workloads of ``synth``, "mix-m3t3"
is a 12-series m = tau = 3 set (sine, logistic, Lorenz x SNR -10/0/10/20 dB,
N = 2e4): the headline workload's line statistics at a size a full profiler
capture handles.
"""
from __future__ import annotations

import sys

import numpy as np


def batch_arrays(name: str):
    """(flat series, offsets, m, tau) of a workload name."""
    if name == "mix-m3t3":
        from synth.series import SeriesSpec, _make_many
        specs = [SeriesSpec(kind=k, n=20000, snr_db=s, seed=5, m=3, tau=3)
                 for k in ("sine", "logistic", "lorenz") for s in (-10.0, 0.0, 10.0, 20.0)]
        ys = _make_many(specs, cache=False)
        offsets = np.concatenate([[0], np.cumsum([len(v) for v in ys])]).astype(np.int64)
        flat = np.concatenate(ys).astype(np.float32)
        return flat, offsets, np.full(len(ys), 3, np.int32), np.full(len(ys), 3, np.int32)
    from synth import workload
    return workload(name).pack()


def main(argv=None) -> int:
    import torch
    from . import abi
    argv = sys.argv[1:] if argv is None else argv
    name = argv[0] if argv else "batched-720"
    reps = int(argv[1]) if len(argv) > 1 else 3
    tile = int(argv[2]) if len(argv) > 2 else 0
    stage = int(argv[3]) if len(argv) > 3 else 0
    flat, offsets, m, tau = batch_arrays(name)
    stream = torch.cuda.Stream()
    ctx = abi.Context(stream=stream, select=abi.RQA_SELECT_RADIX, tile=tile)
    abi.rqa_set_tuning(ctx, tile, 0, 0, stage)
    with torch.cuda.stream(stream):
        y = torch.from_numpy(flat).cuda()
    batch = abi.Batch(y, offsets, m, tau)
    rr = list(range(1, 21))
    eps = torch.empty((batch.n_series, 20), dtype=torch.float32, device="cuda")
    with torch.cuda.stream(stream):
        abi.rqa_eps_for_rr(ctx, batch, rr, 100, eps)
    stream.synchronize()
    ne = np.diff(offsets) - (m.astype(np.int64) - 1) * tau
    cells = int((ne * (ne - 1) // 2).sum())
    hoff = batch.hist_offsets(20)
    hist = torch.empty(int(hoff[-1]), dtype=torch.uint64, device="cuda")
    for r in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        with torch.cuda.stream(stream):
            abi.rqa_line_hist(ctx, batch, eps, 20, hist, hoff)
        e1.record(stream)
        stream.synchronize()
        ms = e0.elapsed_time(e1)
        print(f"{name} tile={abi.rqa_device_info(ctx)['tile']} stage={stage} run {r}: {ms:.2f} ms, "
              f"{cells / (ms * 1e-3):.4g} cells/s")
    code = abi.rqa_status(ctx)
    ctx.close()
    if code:
        print(f"device error {code}: {abi.rqa_error_string(code)}")
        return 1
    return 0


if __name__ == "__main__":
    sys.exit(main())
