#!/usr/bin/env python
"""Throughput benchmark of the averaged-RQA hot path on GB300.

One step = the whole hot path over one batch: exact thresholds eps_k for
K = 20 recurrence rates (1..20 %), then one line pass over every upper-triangle
cell giving C_k, L_max, the full diagonal line-length histograms P_k(l),
DET_k(lmin) for lmin in {2, 3, 5} and their averages -- a single
``rqa_det_avg`` call through the C ABI.  Default workload: 96 series of
N = 10^5 (sine / logistic / Lorenz x 8 SNRs x 4 seeds) plus 200 series with
N log-uniform in [10^2, 10^4], m = 3, tau = 3 (synthetic stand-ins for the
paper's Sect. 3 data).

Prints ONE JSON line (rank 0).  ``--impl reference`` times the CPU oracle on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = ("series/sec & recurrence cells/sec for averaged DET (K=20), bit-exact, "
          "batched+MLP vs plain")
UNIT = "recurrence cells/s"
RR = list(range(1, 21))
LMIN = [2, 3, 5]


def env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", default="full-296")
    ap.add_argument("--form", default="auto", choices=["auto", "batched", "plain"])
    ap.add_argument("--no-plain", action="store_true", help="skip the per-series comparison")
    ap.add_argument("--no-radix", action="store_true",
                    help="skip the batched radix-selection comparison")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-small", action="store_true",
                    help="skip the per-call latency of a one-series batch")
    ap.add_argument("--cpu-cells", type=float, default=1.2e8,
                    help="cells of the oracle's bounded sample")
    ap.add_argument("--tile", type=int, default=0,
                    help="line-pass register window: 8, 16 or 32 diagonals (0 = tuned)")
    ap.add_argument("--select", default="auto", choices=["auto", "radix"],
                    help="auto: learned bracket when a model file exists")
    return ap.parse_args()


# ----------------------------------------------------------------- helpers
def workload_desc(name):
    return {
        "full-296": "96 x N=1e5 (sine/logistic/Lorenz x 8 SNR x 4 seeds) + 200 x N~logU[1e2,1e4]; "
                    "m=3 tau=3; K=20 RR=1..20%; lmin {2,3,5}; full P(l), L_max",
        "batched-720": "720 series {sine,logistic,Lorenz} x 8 SNR x 10 seeds x N in {1e2,1e3,1e4}; "
                       "m=3 tau=1; K=20; lmin {2,3,5}",
        "lorenz-n1e4": "4 Lorenz x series N=1e4, SNR {-10,0,10,20} dB, m=3 tau=3, K=20",
    }.get(name, name)


def cells_of(offsets, m, tau):
    n = np.diff(offsets).astype(np.int64)
    ne = n - (m.astype(np.int64) - 1) * tau
    return ne * (ne - 1) // 2


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu)], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def file_hash(path):
    return hashlib.sha256(open(path, "rb").read()).hexdigest()[:16]


def profile_traffic(kernel_key, workload):
    """DRAM bytes per launch of a kernel from a committed ncu summary, if it was
    taken on this workload and the kernel source has not changed since."""
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))[kernel_key]
        src = os.path.join(ROOT, rec["source"])
        if file_hash(src) != rec["source_sha"] or rec.get("workload") != workload:
            return None
        return rec
    except Exception:
        return None


# ----------------------------------------------------------------- oracle arm
def oracle_sample(flat, offsets, m, tau, budget_cells):
    """Series indices of a bounded sample: short series first, then longer."""
    cells = cells_of(offsets, m, tau)
    order = np.argsort(cells, kind="stable")
    pick, tot = [], 0
    for i in order:
        if tot >= budget_cells:
            break
        pick.append(int(i))
        tot += int(cells[i])
    return pick, tot


def run_oracle(flat, offsets, m, tau, pick):
    from oracle import c_oracle as CO
    from oracle import rqa_oracle as O
    t0 = time.perf_counter()
    for i in pick:
        y = flat[offsets[i]:offsets[i + 1]]
        d = CO.distances(y, int(m[i]), int(tau[i]))
        sel = O.eps_for_rr(y, int(m[i]), int(tau[i]), RR, 100, dist=d)
        del d
        lines = CO.lines(y, int(m[i]), int(tau[i]), sel["eps"], full_hist=True)
        det = O.det_from_hist(lines["hist"], lines["count"], LMIN)
        O.det_avg(det)
    return time.perf_counter() - t0


def max_over_ranks(x: float, dist, device) -> float:
    """Largest value of x over the ranks (x itself without a process group)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(cells_per_rank: int, world: int, ms_max: float) -> float:
    """Weak scaling: every rank processes its own copy of the workload, the job
    finishes with the slowest rank."""
    return world * cells_per_rank / (ms_max * 1e-3)


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


# ----------------------------------------------------------------- main
def main():
    args = parse()
    rank = env_int("RANK", 0)
    world = env_int("WORLD_SIZE", 1)
    local_rank = env_int("LOCAL_RANK", 0)

    from synth import workload
    w = workload(args.workload)

    if args.impl == "reference":
        if rank != 0:
            return 0
        flat, offsets, m, tau = w.pack()
        from oracle import c_oracle as CO
        CO.build()
        pick, cells = oracle_sample(flat, offsets, m, tau, args.cpu_cells)
        times = []
        for s in range(args.warmup + args.steps):
            t = run_oracle(flat, offsets, m, tau, pick)
            if s >= args.warmup:
                times.append(t)
        sec = sum(times) / len(times)
        val = cells / sec
        sample = (f"{len(pick)} shortest series of the workload ({cells:.3e} cells) per step; "
                  f"oracle = NumPy sort for eps + C diagonal scans (OpenMP) + FP64 DET")
        print(json.dumps({
            "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": args.workload, "desc": workload_desc(args.workload),
                       "sample": sample},
            "series_per_s": len(pick) / sec,
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": CO.num_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        }), flush=True)
        return 0

    import torch
    import paper_2208_09136_gb300 as rqa

    dist = None
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
    dev = local_rank if torch.cuda.is_available() else 0
    torch.cuda.set_device(dev)

    flat, offsets, m, tau = w.pack()
    cells = cells_of(offsets, m, tau)
    total_cells = int(cells.sum())
    S, K = len(offsets) - 1, len(RR)
    form = args.form
    from paper_2208_09136_gb300 import bracket
    have_model = os.path.exists(bracket.MODEL_PATH) and form != "plain" and args.select == "auto"
    if form == "auto":
        form = "batched"
    stream = torch.cuda.Stream(device=dev)
    sched = rqa.RQA_SCHED_PER_SERIES if form == "plain" else rqa.RQA_SCHED_BATCHED

    with torch.cuda.stream(stream):
        y = torch.from_numpy(flat).to(f"cuda:{dev}")
        batch = rqa.Batch(y, offsets, m, tau)
        hoff = batch.hist_offsets(K)
        det = torch.empty((S, K, len(LMIN)), dtype=torch.float64, device=dev)
        avg = torch.empty((S, len(LMIN)), dtype=torch.float64, device=dev)
        eps = torch.empty((S, K), dtype=torch.float32, device=dev)
        hist = torch.empty(int(hoff[-1]), dtype=torch.uint64, device=dev)
        lmax = torch.empty((S, K), dtype=torch.uint32, device=dev)
        cnt = torch.empty((S, K), dtype=torch.uint64, device=dev)
        flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2
    stream.synchronize()

    def make_ctx(schedule, learned=False):
        c = rqa.Context(device=dev, stream=stream, schedule=schedule,
                        select=rqa.RQA_SELECT_AUTO if learned else rqa.RQA_SELECT_RADIX,
                        tile=args.tile)
        if learned:
            bracket.install(c)
        return c

    def step(ctx, yb=None):
        b = batch if yb is None else yb
        rqa.rqa_det_avg(ctx, b, RR, 100, None, K, LMIN, det, avg, eps, hist, hoff, lmax, cnt, None)

    def barrier():
        torch.cuda.synchronize(dev)
        if dist is not None:
            dist.barrier()

    ctx = make_ctx(sched, have_model)
    from paper_2208_09136_gb300 import tuning
    tuned = tuning.tuned(ctx, batch, RR, 100)  # cached or timed now; keeps --tile when one was given
    rqa.rqa_set_timing(ctx, True)
    for _ in range(args.warmup):
        step(ctx)
    barrier()
    code = rqa.rqa_status(ctx)
    if code:
        raise SystemExit(f"device error: {rqa.rqa_error_string(code)}")

    clocks = ClockSampler(dev)
    launches0 = rqa.rqa_kernel_launches(ctx)
    replays0 = rqa.rqa_graph_replays(ctx)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    phase = np.zeros(6, dtype=np.float64)
    barrier()
    clocks.start()
    for i in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(i & 0xff)  # evict L2 between steps (outside the timed events)
        ev[i][0].record(stream)
        step(ctx)
        ev[i][1].record(stream)
        stream.synchronize()
        phase += rqa.rqa_phase_times(ctx)
    barrier()
    clk = clocks.stop()
    launches = rqa.rqa_kernel_launches(ctx) - launches0
    replays = rqa.rqa_graph_replays(ctx) - replays0
    bstats = rqa.rqa_bracket_stats(ctx) if have_model else None
    ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
    code = rqa.rqa_status(ctx)
    if code:
        raise SystemExit(f"device error: {rqa.rqa_error_string(code)}")
    phase /= args.steps

    ms_max = max_over_ranks(ms, dist, dev)
    value = whole_job_rate(total_cells, world, ms_max)
    series_per_s = world * S / (ms_max * 1e-3)

    # plain per-series form of the same step, for comparison
    plain = None
    if not args.no_plain and form != "plain":
        pctx = make_ctx(rqa.RQA_SCHED_PER_SERIES)
        step(pctx)
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n_plain = max(1, min(2, args.steps))
        pms = 0.0
        for i in range(n_plain):
            with torch.cuda.stream(stream):
                flush.fill_(i & 0xff)
            e0.record(stream)
            step(pctx)
            e1.record(stream)
            stream.synchronize()
            pms += e0.elapsed_time(e1)
        pms /= n_plain
        if rqa.rqa_status(pctx):
            raise SystemExit("device error in the per-series form")
        plain = {"form": "plain per-series (one launch sequence per series, radix select)",
                 "value": total_cells / (pms * 1e-3), "series_per_s": S / (pms * 1e-3),
                 "ms_per_step": pms, "steps": n_plain}
        pctx.close()

    # the same batched schedule with the full radix selection: what the
    # learned bracket gains on this workload
    radix = None
    if not args.no_radix and form != "plain" and have_model:
        rctx = make_ctx(rqa.RQA_SCHED_BATCHED)  # radix select
        # the same line-pass knobs as the timed context, so the two legs differ in the
        # selection alone
        rqa.rqa_set_tuning(rctx, tuned["tile"], tuned["unit_bands"], tuned["line_ctas"], tuned["stage"])
        rqa.rqa_set_timing(rctx, True)
        step(rctx)
        stream.synchronize()
        n_rad = max(1, min(3, args.steps))
        rms, rph = 0.0, np.zeros(6, dtype=np.float64)
        for i in range(n_rad):
            with torch.cuda.stream(stream):
                flush.fill_(i & 0xff)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step(rctx)
            e1.record(stream)
            stream.synchronize()
            rms += e0.elapsed_time(e1)
            rph += rqa.rqa_phase_times(rctx)
        rms /= n_rad
        rph /= n_rad
        if rqa.rqa_status(rctx):
            raise SystemExit("device error in the radix form")
        rms = max_over_ranks(rms, dist, dev)
        radix = {"form": "batched, full radix selection (no network), the timed context's line-pass knobs",
                 "value": world * total_cells / (rms * 1e-3), "series_per_s": world * S / (rms * 1e-3),
                 "ms_per_step": rms, "steps": n_rad,
                 "phase_ms": {n: round(float(v), 4) for n, v in
                              zip(["finite check", "coarse round", "middle round", "final round",
                                   "line pass", "finalize"], rph)},
                 "learned_over_radix_series_per_s": (world * S / (ms_max * 1e-3)) / (world * S / (rms * 1e-3))}
        rctx.close()

    # end to end through the C ABI from pinned host buffers
    e2e = None
    if not args.no_e2e:
        h_y = torch.from_numpy(flat).pin_memory()
        h_avg = torch.empty((S, len(LMIN)), dtype=torch.float64).pin_memory()
        h_det = torch.empty((S, K, len(LMIN)), dtype=torch.float64).pin_memory()
        h_eps = torch.empty((S, K), dtype=torch.float32).pin_memory()
        with torch.cuda.stream(stream):
            y2 = torch.empty_like(y)
        yb = rqa.Batch(y2, offsets, m, tau)
        n_e2e = max(1, min(3, args.steps))
        tot = 0.0
        for i in range(n_e2e + 1):
            with torch.cuda.stream(stream):
                flush.fill_(i & 0xff)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            with torch.cuda.stream(stream):
                y2.copy_(h_y, non_blocking=True)
            step(ctx, yb)
            with torch.cuda.stream(stream):
                h_avg.copy_(avg, non_blocking=True)
                h_det.copy_(det, non_blocking=True)
                h_eps.copy_(eps, non_blocking=True)
            e1.record(stream)
            stream.synchronize()
            if i > 0:
                tot += e0.elapsed_time(e1)
        ems = max_over_ranks(tot / n_e2e, dist, dev)
        e2e = {"value": whole_job_rate(total_cells, world, ems), "unit": UNIT,
               "h2d_bytes_per_step": int(h_y.numel() * 4),
               "d2h_bytes_per_step": int((h_avg.numel() + h_det.numel()) * 8 + h_eps.numel() * 4),
               "ms_per_step": ems, "note": "series H2D, DET/avg DET/eps D2H; P(l) stays on device"}

    # latency of one call on a one-series batch (N = 100 logistic map, m = tau = 1),
    # where the step is bound by launches, not by cells: median of single calls,
    # with the inputs resident and end to end (series H2D, DET averages D2H)
    small = None
    if rank == 0 and not args.no_small:
        from synth import workload as make_workload
        sflat, soff, sm_, stau = make_workload("logistic-n100").pack()
        sK = len(RR)
        with torch.cuda.stream(stream):
            sy = torch.from_numpy(sflat).to(f"cuda:{dev}")
            sb = rqa.Batch(sy, soff, sm_, stau)
            shoff = sb.hist_offsets(sK)
            s_det = torch.empty((1, sK, len(LMIN)), dtype=torch.float64, device=dev)
            s_avg = torch.empty((1, len(LMIN)), dtype=torch.float64, device=dev)
            s_eps = torch.empty((1, sK), dtype=torch.float32, device=dev)
            s_hist = torch.empty(int(shoff[-1]), dtype=torch.uint64, device=dev)
        h_sy = torch.from_numpy(sflat).pin_memory()
        h_savg = torch.empty((1, len(LMIN)), dtype=torch.float64).pin_memory()
        sctx = rqa.Context(device=dev, stream=stream, schedule=rqa.RQA_SCHED_BATCHED,
                           select=rqa.RQA_SELECT_RADIX)

        def small_call(e2e_copies):
            if e2e_copies:
                with torch.cuda.stream(stream):
                    sy.copy_(h_sy, non_blocking=True)
            rqa.rqa_det_avg(sctx, sb, RR, 100, None, sK, LMIN, s_det, s_avg, s_eps, s_hist, shoff,
                            None, None, None)
            if e2e_copies:
                with torch.cuda.stream(stream):
                    h_savg.copy_(s_avg, non_blocking=True)

        res = {}
        for label, copies in (("resident", False), ("e2e", True)):
            for _ in range(20):
                small_call(copies)
            stream.synchronize()
            t = []
            for _ in range(100):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                small_call(copies)
                e1.record(stream)
                stream.synchronize()
                t.append(e0.elapsed_time(e1))
            res[label] = statistics.median(t)
        if rqa.rqa_status(sctx):
            raise SystemExit("device error in the one-series calls")
        sctx.close()
        small = {"workload": "logistic-n100: 1 series, N = 100, m = tau = 1, K = 20, radix select",
                 "ms_per_call": res["resident"], "e2e_ms_per_call": res["e2e"],
                 "calls": 100, "stat": "median of single calls (CUDA events on the call's stream)"}

    # roofline of the dominant kernel (line pass): issue-limited integer/FP32 ALU
    peaks = measured_peaks()
    sm = rqa.rqa_device_info(ctx)["sm_count"]
    f_max = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    peak_ops = sm * 128 * f_max                       # lane-ops/s
    mm = int(m[0])
    names = ["finite check", "coarse round", "middle round", "final round", "line pass", "finalize"]
    dom = int(np.argmax(phase))
    ops_cell = {4: (2 * mm - 1) + 5 + 0.2, 1: (2 * mm - 1) + 2, 2: (2 * mm - 1) + 2,
                3: (2 * mm - 1) + 2}.get(dom, 0.0)
    achieved = total_cells * ops_cell / (phase[dom] * 1e-3) if phase[dom] > 0 else 0.0
    traffic = profile_traffic("lines" if dom == 4 else "count", args.workload)
    roofline = {"bound": "alu", "kernel": names[dom], "achieved": achieved / 1e12,
                "peak": peak_ops / 1e12, "unit": "Tops/s (lane-ops)",
                "frac": achieved / peak_ops if peak_ops else None,
                "traffic": None if traffic is None else traffic["bytes_per_launch"],
                "ncu": None if traffic is None or "issue_active_pct" not in traffic else {
                    "issue_active_pct": traffic["issue_active_pct"],
                    "alu_pipe_pct": traffic["alu_pipe_pct"],
                    "warp_inst_per_32_cells": traffic["warp_inst_per_32_cells"],
                    "source": "profiles/traffic.json: DRAM bytes from one ncu pass of this kernel on this "
                              "workload; issue, ALU and instructions from " + traffic.get("inst_source", "")},
                "ops_per_cell": ops_cell,
                "peak_note": f"{sm} SMs x 128 lanes x {f_max/1e6:.0f} MHz (max SM clock)"}

    cpu = None
    if rank == 0 and not args.no_cpu:
        from oracle import c_oracle as CO
        CO.build()
        pick, pcells = oracle_sample(flat, offsets, m, tau, args.cpu_cells)
        sec = run_oracle(flat, offsets, m, tau, pick)
        cpu = {"value": pcells / sec, "unit": UNIT, "cores": CO.num_threads(), "kind": "oracle",
               "sample": f"{len(pick)} shortest series of the workload, {pcells:.3e} cells, "
                         f"{sec:.1f} s (NumPy sort eps + OpenMP C diagonal scans + FP64 DET)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "desc": workload_desc(args.workload),
                       "form": f"{form} + radix select" if not have_model else f"{form} + learned bracket",
                       "series": S, "cells_per_step": total_cells, "l2": "flushed between steps",
                       "line_tuning": {k: tuned[k] for k in ("tile", "unit_bands", "line_ctas", "stage")},
                       "line_tuning_from": ("--tile + " if args.tile else "") +
                                           ("tuning cache" if tuned["cached"] else "rqa_autotune"),
                       "parallelism": f"replicas x{world} (series-independent)"},
            "series_per_s": series_per_s,
            "phase_ms": {n: round(float(v), 4) for n, v in zip(names, phase)},
            "gpu_launches": int(launches),
            "graph_replays": int(replays),
            "bracket": None if bstats is None else {"hits": bstats[0], "misses": bstats[1],
                                                    "miss_rate": bstats[1] / max(1, sum(bstats))},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "plain": plain,
            "radix": radix,
            "small_batch": small,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
