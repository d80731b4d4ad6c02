"""Time whole averaged-DET steps on a named workload, phase by phase.

``python -m paper_2208_09136_gb300.stepbench WORKLOAD [REPS] [SELECT]``

Builds the workload's batch on cuda:0 and runs ``rqa_det_avg`` (K = 20,
RR = 1..20 %, lmin 2, 3, 5, full histograms) REPS times on one stream after
one warm-up call, with the context's phase events on.  SELECT is "auto" (the
learned bracket where the model's domain allows, radix elsewhere; the
default) or "radix".  Prints one line per run: the step time from CUDA events
and the time of each phase (finiteness check, the three counting rounds
with their selections, line pass, finalisation).
"""
from __future__ import annotations

import sys

import numpy as np

PHASES = ["finite", "coarse", "middle", "final", "lines", "finalize"]


def main(argv=None) -> int:
    import torch
    from . import abi, bracket
    from .linebench import batch_arrays
    argv = sys.argv[1:] if argv is None else argv
    name = argv[0] if argv else "batched-720"
    reps = int(argv[1]) if len(argv) > 1 else 3
    mode = argv[2] if len(argv) > 2 else "auto"
    flat, offsets, m, tau = batch_arrays(name)
    stream = torch.cuda.Stream()
    sel = abi.RQA_SELECT_AUTO if mode == "auto" else abi.RQA_SELECT_RADIX
    ctx = abi.Context(stream=stream, select=sel)
    if mode == "auto":
        bracket.install(ctx)
    with torch.cuda.stream(stream):
        y = torch.from_numpy(flat).cuda()
    batch = abi.Batch(y, offsets, m, tau)
    S, K, lmin = batch.n_series, 20, (2, 3, 5)
    rr = list(range(1, K + 1))
    hoff = batch.hist_offsets(K)
    with torch.cuda.stream(stream):
        det = torch.empty((S, K, len(lmin)), dtype=torch.float64, device="cuda")
        avg = torch.empty((S, len(lmin)), dtype=torch.float64, device="cuda")
        eps = torch.empty((S, K), dtype=torch.float32, device="cuda")
        hist = torch.empty(int(hoff[-1]), dtype=torch.uint64, device="cuda")
        lmax = torch.empty((S, K), dtype=torch.uint32, device="cuda")
        cnt = torch.empty((S, K), dtype=torch.uint64, device="cuda")
    abi.rqa_set_timing(ctx, True)

    def step():
        with torch.cuda.stream(stream):
            abi.rqa_det_avg(ctx, batch, rr, 100, None, K, lmin, det, avg, eps, hist, hoff, lmax,
                            cnt, None)

    step()
    stream.synchronize()
    for r in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        stream.synchronize()
        ph = np.asarray(abi.rqa_phase_times(ctx), dtype=np.float64)
        parts = " ".join(f"{n}={v:.2f}" for n, v in zip(PHASES, ph))
        print(f"{name} select={mode} run {r}: {e0.elapsed_time(e1):.2f} ms  {parts}")
    code = abi.rqa_status(ctx)
    ctx.close()
    if code:
        print(f"device error {code}: {abi.rqa_error_string(code)}")
        return 1
    return 0


if __name__ == "__main__":
    sys.exit(main())
