"""Thin ctypes binding of ``librqa.so`` (the C ABI in ``include/rqa.h``).

Only argument marshalling happens here: torch tensors supply device buffers
and streams, NumPy arrays the host-side arrays.  Every step of the method runs
in the library's CUDA kernels; there is no fallback, and loading fails loudly
if the library has not been built.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

from .build import LIB

c_int = ctypes.c_int
c_i32 = ctypes.c_int32
c_i64 = ctypes.c_int64
c_u64 = ctypes.c_uint64
c_vp = ctypes.c_void_p

RQA_SCHED_BATCHED, RQA_SCHED_PER_SERIES = 0, 1
RQA_SELECT_AUTO, RQA_SELECT_RADIX, RQA_SELECT_BRACKET = 0, 1, 2
RQA_K_MAX = 127
RQA_NOALLOC_K_MAX = 31
RQA_NOALLOC_NE_MAX = 1 << 20
RQA_LMIN_MAX = 8
RQA_FEATURES = 131
RQA_MLP_HIDDEN = 256
RQA_MLP_OUT = 40
RQA_MLP_PARAMS = 256 * 131 + 256 + 256 * 256 + 256 + 40 * 256 + 40
RQA_MLP_ACTS = 512


class RqaError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {rqa_error_string(code)} (code {code})")


class _Config(ctypes.Structure):
    _fields_ = [("device", c_int), ("stream", c_vp), ("schedule", c_int), ("select", c_int),
                ("tile", c_int), ("blocks_per_sm", c_int), ("flags", c_int), ("reserved", c_int * 3)]


RQA_FLAG_NO_GRAPHS = 1
RQA_FLAG_LOI = 2


class _Batch(ctypes.Structure):
    _fields_ = [("y", c_vp), ("offsets", c_vp), ("m", c_vp), ("tau", c_vp), ("n_series", c_i32)]


class _LineOutputs(ctypes.Structure):
    _fields_ = [("hist", c_vp), ("hist_offsets", c_vp), ("lmax", c_vp), ("count", c_vp),
                ("stencil", c_vp)]


_lib: Optional[ctypes.CDLL] = None

_SIGS = {
    "rqa_abi_version": ([], c_int),
    "rqa_error_string": ([c_int], ctypes.c_char_p),
    "rqa_create": ([ctypes.POINTER(c_vp), ctypes.POINTER(_Config)], c_int),
    "rqa_destroy": ([c_vp], None),
    "rqa_status": ([c_vp], c_int),
    "rqa_device_info": ([c_vp, c_vp, c_vp, c_vp], c_int),
    "rqa_target_counts": ([c_u64, c_vp, c_i32, c_i32, c_vp], c_int),
    "rqa_target_counts_loi": ([c_u64, c_vp, c_i32, c_i32, c_vp], c_int),
    "rqa_eps_for_rr": ([c_vp, ctypes.POINTER(_Batch), c_vp, c_i32, c_i32, c_vp, c_vp, c_vp], c_int),
    "rqa_det_avg": ([c_vp, ctypes.POINTER(_Batch), c_vp, c_i32, c_vp, c_i32, c_vp, c_i32, c_vp,
                     c_vp, c_vp, ctypes.POINTER(_LineOutputs)], c_int),
    "rqa_set_timing": ([c_vp, c_int], c_int),
    "rqa_phase_times": ([c_vp, c_vp, c_int], c_int),
    "rqa_kernel_launches": ([c_vp], c_u64),
    "rqa_graph_replays": ([c_vp], c_u64),
    "rqa_line_measures": ([c_vp, ctypes.POINTER(_Batch), c_i32, c_vp, c_vp, c_vp, c_i32, c_vp, c_vp,
                           c_vp, c_vp], c_int),
    "rqa_eps_approx": ([c_vp, ctypes.POINTER(_Batch), c_vp, c_i32, c_i32, c_i32, c_vp, c_vp, c_vp], c_int),
    "rqa_vline_hist": ([c_vp, ctypes.POINTER(_Batch), c_vp, c_i32, c_vp, c_vp, c_vp, c_vp], c_int),
    "rqa_lam_tt": ([c_vp, ctypes.POINTER(_Batch), c_i32, c_vp, c_vp, c_vp, c_i32, c_vp, c_vp, c_vp,
                    c_vp], c_int),
    "rqa_autotune": ([c_vp, ctypes.POINTER(_Batch), c_vp, c_i32, c_i32, c_vp], c_int),
    "rqa_set_tuning": ([c_vp, c_vp], c_int),
    "rqa_get_tuning": ([c_vp, c_vp], c_int),
    "rqa_line_hist": ([c_vp, ctypes.POINTER(_Batch), c_vp, c_i32, c_vp, c_vp, c_vp, c_vp, c_vp],
                      c_int),
    "rqa_sketch": ([c_vp, ctypes.POINTER(_Batch), c_u64, c_vp, c_vp, c_vp], c_int),
    "rqa_mlp_forward": ([c_vp, c_vp, c_vp, c_i32, c_vp, c_vp], c_int),
    "rqa_mlp_backward": ([c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_i32, ctypes.c_float, ctypes.c_float,
                          c_vp, c_vp], c_int),
    "rqa_adam_step": ([c_vp, c_vp, c_vp, c_vp, c_vp, c_i64, c_i32, ctypes.c_float, ctypes.c_float,
                       ctypes.c_float, ctypes.c_float], c_int),
    "rqa_set_bracket_model": ([c_vp, c_vp, ctypes.c_float], c_int),
    "rqa_set_bracket_domain": ([c_vp, c_vp, c_vp, c_i32], c_int),
    "rqa_log_labels": ([c_vp, c_vp, c_vp, c_i32, c_i32, c_vp], c_int),
    "rqa_bracket_eval": ([c_vp, c_vp, c_vp, c_i32, c_i32, ctypes.c_float, ctypes.c_float,
                          ctypes.c_float, c_vp, c_vp, c_vp], c_int),
    "rqa_gather_rows": ([c_vp, c_vp, c_vp, c_i32, c_i32, c_vp], c_int),
    "rqa_bracket_stats": ([c_vp, c_vp, c_vp], c_int),
    "rqa_eps_for_rr_noalloc": ([ctypes.POINTER(_Batch), c_vp, c_i32, c_i32, c_vp, c_vp, c_vp, c_vp,
                                c_vp], c_int),
}


def exported_symbols():
    return sorted(_SIGS)


def lib() -> ctypes.CDLL:
    """Load librqa.so (built by ``build()``); raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise RuntimeError(f"librqa.so is not built ({LIB}); run "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB)
        for name, (args, res) in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def rqa_error_string(code: int) -> str:
    try:
        return lib().rqa_error_string(code).decode()
    except Exception:
        return "error"


def rqa_abi_version() -> int:
    return int(lib().rqa_abi_version())


def _check(rc: int, where: str):
    if rc != 0:
        raise RqaError(rc, where)


def _np_ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(c_vp)


def _dev_ptr(t, dtype, n: Optional[int] = None, name: str = "buffer"):
    """Device pointer of a contiguous CUDA tensor of the given dtype (or None)."""
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if n is not None and t.numel() < n:
        raise ValueError(f"{name} holds {t.numel()} elements, needs {n}")
    return c_vp(t.data_ptr())


class Batch:
    """S series back to back in one CUDA FP32 tensor, with host metadata."""

    def __init__(self, y, offsets, m, tau):
        import torch
        self.y = y
        self.offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        S = len(self.offsets) - 1
        self.m = np.ascontiguousarray(np.broadcast_to(np.asarray(m, dtype=np.int32), (S,)))
        self.tau = np.ascontiguousarray(np.broadcast_to(np.asarray(tau, dtype=np.int32), (S,)))
        if not isinstance(y, torch.Tensor) or not y.is_cuda or y.dtype != torch.float32:
            raise TypeError("y must be a CUDA float32 tensor")
        if not y.is_contiguous() or y.numel() < int(self.offsets[-1]):
            raise ValueError("y must be contiguous and hold offsets[-1] values")

    @property
    def n_series(self) -> int:
        return len(self.offsets) - 1

    @property
    def ne(self) -> np.ndarray:
        n = np.diff(self.offsets)
        return n - (self.m.astype(np.int64) - 1) * self.tau

    def hist_offsets(self, K: int) -> np.ndarray:
        off = np.zeros(self.n_series + 1, dtype=np.int64)
        off[1:] = np.cumsum(K * (self.ne - 1))
        return off

    def _c(self) -> _Batch:
        return _Batch(c_vp(self.y.data_ptr()), _np_ptr(self.offsets), _np_ptr(self.m),
                      _np_ptr(self.tau), self.n_series)

    @staticmethod
    def from_numpy(series: Sequence[np.ndarray], m, tau, device: int = 0) -> "Batch":
        import torch
        offsets = np.zeros(len(series) + 1, dtype=np.int64)
        offsets[1:] = np.cumsum([len(s) for s in series])
        flat = np.concatenate([np.asarray(s, dtype=np.float32) for s in series])
        y = torch.from_numpy(flat).to(f"cuda:{device}")
        return Batch(y, offsets, m, tau)


class Context:
    """An ``rqa_ctx``: device, stream, schedule and scratch memory."""

    def __init__(self, device: int = 0, stream=None, schedule: int = RQA_SCHED_BATCHED,
                 select: int = RQA_SELECT_AUTO, tile: int = 0, blocks_per_sm: int = 0,
                 flags: int = 0):
        import torch
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        handle = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        cfg = _Config(device, c_vp(handle), schedule, select, tile, blocks_per_sm, int(flags),
                      (c_int * 3)())
        p = c_vp()
        _check(lib().rqa_create(ctypes.byref(p), ctypes.byref(cfg)), "rqa_create")
        self._p = p
        self.device = device

    @property
    def handle(self):
        return self._p

    def close(self):
        if getattr(self, "_p", None) is not None and self._p.value:
            lib().rqa_destroy(self._p)
            self._p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rqa_create(device: int = 0, stream=None, schedule: int = RQA_SCHED_BATCHED,
               select: int = RQA_SELECT_AUTO, tile: int = 0, blocks_per_sm: int = 0) -> Context:
    return Context(device, stream, schedule, select, tile, blocks_per_sm)


def rqa_destroy(ctx: Context):
    ctx.close()


def rqa_status(ctx: Context) -> int:
    return int(lib().rqa_status(ctx.handle))


def rqa_device_info(ctx: Context):
    sm, tile, bpsm = c_int(), c_int(), c_int()
    _check(lib().rqa_device_info(ctx.handle, ctypes.byref(sm), ctypes.byref(tile),
                                 ctypes.byref(bpsm)), "rqa_device_info")
    return {"sm_count": sm.value, "tile": tile.value, "blocks_per_sm": bpsm.value}


def rqa_target_counts(P: int, rr_num: Sequence[int], rr_den: int) -> np.ndarray:
    rr = np.ascontiguousarray(rr_num, dtype=np.int32)
    out = np.zeros(len(rr), dtype=np.uint64)
    _check(lib().rqa_target_counts(int(P), _np_ptr(rr), int(rr_den), len(rr), _np_ptr(out)),
           "rqa_target_counts")
    return out


def rqa_target_counts_loi(ne: int, rr_num: Sequence[int], rr_den: int) -> np.ndarray:
    rr = np.ascontiguousarray(rr_num, dtype=np.int32)
    out = np.zeros(len(rr), dtype=np.uint64)
    _check(lib().rqa_target_counts_loi(int(ne), _np_ptr(rr), int(rr_den), len(rr), _np_ptr(out)),
           "rqa_target_counts_loi")
    return out


def rqa_eps_for_rr(ctx: Context, batch: Batch, rr_num, rr_den: int, eps_out, count_le=None,
                   count_lt=None):
    import torch
    rr = np.ascontiguousarray(rr_num, dtype=np.int32)
    n = batch.n_series * len(rr)
    b = batch._c()
    _check(lib().rqa_eps_for_rr(ctx.handle, ctypes.byref(b), _np_ptr(rr), int(rr_den), len(rr),
                                _dev_ptr(eps_out, torch.float32, n, "eps_out"),
                                _dev_ptr(count_le, torch.uint64, n, "count_le"),
                                _dev_ptr(count_lt, torch.uint64, n, "count_lt")), "rqa_eps_for_rr")


def rqa_det_avg(ctx: Context, batch: Batch, rr_num, rr_den: int, eps, K: int, lmin, det_out,
                det_avg, eps_used=None, hist=None, hist_offsets=None, lmax=None, count=None,
                stencil=None):
    import torch
    rr = None if rr_num is None else np.ascontiguousarray(rr_num, dtype=np.int32)
    lm = np.ascontiguousarray(lmin, dtype=np.int32)
    S = batch.n_series
    b = batch._c()
    hoff = None if hist_offsets is None else np.ascontiguousarray(hist_offsets, dtype=np.int64)
    lo = None
    if any(v is not None for v in (hist, lmax, count, stencil)):
        lo = _LineOutputs(_dev_ptr(hist, torch.uint64, None if hoff is None else int(hoff[-1]), "hist"),
                          _np_ptr(hoff), _dev_ptr(lmax, torch.uint32, S * K, "lmax"),
                          _dev_ptr(count, torch.uint64, S * K, "count"),
                          _dev_ptr(stencil, torch.uint64, S * K, "stencil"))
    _check(lib().rqa_det_avg(ctx.handle, ctypes.byref(b), _np_ptr(rr), int(rr_den),
                             _dev_ptr(eps, torch.float32, S * K, "eps"), int(K), _np_ptr(lm),
                             len(lm), _dev_ptr(det_out, torch.float64, S * K * len(lm), "det_out"),
                             _dev_ptr(det_avg, torch.float64, S * len(lm), "det_avg"),
                             _dev_ptr(eps_used, torch.float32, S * K, "eps_used"),
                             None if lo is None else ctypes.byref(lo)), "rqa_det_avg")


def rqa_set_timing(ctx: Context, enable: bool = True):
    _check(lib().rqa_set_timing(ctx.handle, int(bool(enable))), "rqa_set_timing")


def rqa_phase_times(ctx: Context) -> np.ndarray:
    out = np.zeros(6, dtype=np.float32)
    _check(lib().rqa_phase_times(ctx.handle, _np_ptr(out), 6), "rqa_phase_times")
    return out


def rqa_kernel_launches(ctx: Context) -> int:
    return int(lib().rqa_kernel_launches(ctx.handle))


def rqa_line_measures(ctx: Context, batch: Batch, K: int, hist, hist_offsets, lmin, L_out=None,
                      entr_out=None, L_avg=None, entr_avg=None):
    import torch
    S = batch.n_series
    lm = np.ascontiguousarray(lmin, dtype=np.int32)
    hoff = np.ascontiguousarray(hist_offsets, dtype=np.int64)
    b = batch._c()
    n = S * K * len(lm)
    _check(lib().rqa_line_measures(ctx.handle, ctypes.byref(b), int(K),
                                   _dev_ptr(hist, torch.uint64, int(hoff[-1]), "hist"), _np_ptr(hoff),
                                   _np_ptr(lm), len(lm),
                                   _dev_ptr(L_out, torch.float64, n, "L_out"),
                                   _dev_ptr(entr_out, torch.float64, n, "entr_out"),
                                   _dev_ptr(L_avg, torch.float64, S * len(lm), "L_avg"),
                                   _dev_ptr(entr_avg, torch.float64, S * len(lm), "entr_avg")),
           "rqa_line_measures")


def rqa_eps_approx(ctx: Context, batch: Batch, rr_num, rr_den: int, n_thr: int, eps_out, rr_out=None,
                   count_out=None):
    import torch
    rr = np.ascontiguousarray(rr_num, dtype=np.int32)
    S, K = batch.n_series, len(rr)
    b = batch._c()
    _check(lib().rqa_eps_approx(ctx.handle, ctypes.byref(b), _np_ptr(rr), int(rr_den), K, int(n_thr),
                                _dev_ptr(eps_out, torch.float32, S * K, "eps_out"),
                                _dev_ptr(rr_out, torch.float64, S * K, "rr_out"),
                                _dev_ptr(count_out, torch.uint64, S * K, "count_out")), "rqa_eps_approx")


def rqa_vline_hist(ctx: Context, batch: Batch, eps, K: int, vhist=None, vhist_offsets=None,
                   vmax=None, vmass=None):
    import torch
    S = batch.n_series
    hoff = None if vhist_offsets is None else np.ascontiguousarray(vhist_offsets, dtype=np.int64)
    b = batch._c()
    _check(lib().rqa_vline_hist(ctx.handle, ctypes.byref(b), _dev_ptr(eps, torch.float32, S * K, "eps"),
                                int(K),
                                _dev_ptr(vhist, torch.uint64, None if hoff is None else int(hoff[-1]), "vhist"),
                                None if hoff is None else _np_ptr(hoff),
                                _dev_ptr(vmax, torch.uint32, S * K, "vmax"),
                                _dev_ptr(vmass, torch.uint64, S * K, "vmass")), "rqa_vline_hist")


def rqa_lam_tt(ctx: Context, batch: Batch, K: int, vhist, vhist_offsets, vmin, lam_out=None,
               tt_out=None, lam_avg=None, tt_avg=None):
    import torch
    S = batch.n_series
    vm = np.ascontiguousarray(vmin, dtype=np.int32)
    hoff = np.ascontiguousarray(vhist_offsets, dtype=np.int64)
    b = batch._c()
    n = S * K * len(vm)
    _check(lib().rqa_lam_tt(ctx.handle, ctypes.byref(b), int(K),
                            _dev_ptr(vhist, torch.uint64, int(hoff[-1]), "vhist"), _np_ptr(hoff),
                            _np_ptr(vm), len(vm), _dev_ptr(lam_out, torch.float64, n, "lam_out"),
                            _dev_ptr(tt_out, torch.float64, n, "tt_out"),
                            _dev_ptr(lam_avg, torch.float64, S * len(vm), "lam_avg"),
                            _dev_ptr(tt_avg, torch.float64, S * len(vm), "tt_avg")), "rqa_lam_tt")


def rqa_graph_replays(ctx: Context) -> int:
    return int(lib().rqa_graph_replays(ctx.handle))


class _Tuning(ctypes.Structure):
    _fields_ = [("tile", c_int), ("unit_bands", c_int), ("line_ctas", c_int), ("stage", c_int),
                ("ms", ctypes.c_float)]


def _tuning_dict(t: "_Tuning") -> dict:
    return {"tile": t.tile, "unit_bands": t.unit_bands, "line_ctas": t.line_ctas, "stage": t.stage,
            "ms": float(t.ms)}


def rqa_autotune(ctx: Context, batch: Batch, rr_num, rr_den: int) -> dict:
    """Time the line pass's knobs on (a prefix of) this batch and keep the
    fastest in the context; returns them as a dict."""
    rr = np.ascontiguousarray(rr_num, dtype=np.int32)
    b = batch._c()
    t = _Tuning()
    _check(lib().rqa_autotune(ctx.handle, ctypes.byref(b), _np_ptr(rr), int(rr_den), len(rr),
                              ctypes.byref(t)), "rqa_autotune")
    return _tuning_dict(t)


def rqa_set_tuning(ctx: Context, tile: int = 0, unit_bands: int = 0, line_ctas: int = 0,
                   stage: int = 0):
    t = _Tuning(int(tile), int(unit_bands), int(line_ctas), int(stage), 0.0)
    _check(lib().rqa_set_tuning(ctx.handle, ctypes.byref(t)), "rqa_set_tuning")


def rqa_get_tuning(ctx: Context) -> dict:
    t = _Tuning()
    _check(lib().rqa_get_tuning(ctx.handle, ctypes.byref(t)), "rqa_get_tuning")
    return _tuning_dict(t)


def rqa_line_hist(ctx: Context, batch: Batch, eps, K: int, hist=None, hist_offsets=None,
                  lmax=None, count=None, stencil=None):
    import torch
    S = batch.n_series
    hoff = None if hist_offsets is None else np.ascontiguousarray(hist_offsets, dtype=np.int64)
    b = batch._c()
    _check(lib().rqa_line_hist(ctx.handle, ctypes.byref(b), _dev_ptr(eps, torch.float32, S * K, "eps"),
                               int(K),
                               _dev_ptr(hist, torch.uint64, None if hoff is None else int(hoff[-1]),
                                        "hist"),
                               _np_ptr(hoff), _dev_ptr(lmax, torch.uint32, S * K, "lmax"),
                               _dev_ptr(count, torch.uint64, S * K, "count"),
                               _dev_ptr(stencil, torch.uint64, S * K, "stencil")), "rqa_line_hist")


# ------------------------------------------------------------ learned bracket
def rqa_sketch(ctx: Context, batch: Batch, seed: int, feats, centre=None, qdist=None):
    import torch
    S = batch.n_series
    b = batch._c()
    _check(lib().rqa_sketch(ctx.handle, ctypes.byref(b), int(seed) & ((1 << 64) - 1),
                            _dev_ptr(feats, torch.float32, S * RQA_FEATURES, "feats"),
                            _dev_ptr(centre, torch.float32, S, "centre"),
                            _dev_ptr(qdist, torch.float32, S * 128, "qdist")), "rqa_sketch")


def rqa_mlp_forward(ctx: Context, params, X, Y, acts=None):
    import torch
    B = X.shape[0]
    _check(lib().rqa_mlp_forward(ctx.handle, _dev_ptr(params, torch.float32, RQA_MLP_PARAMS, "params"),
                                 _dev_ptr(X, torch.float32, B * RQA_FEATURES, "X"), int(B),
                                 _dev_ptr(Y, torch.float32, B * RQA_MLP_OUT, "Y"),
                                 _dev_ptr(acts, torch.float32, B * RQA_MLP_ACTS, "acts")),
           "rqa_mlp_forward")


def rqa_mlp_backward(ctx: Context, params, X, acts, Y, T, tau_lo: float, tau_hi: float, grads,
                     loss=None):
    import torch
    B = X.shape[0]
    _check(lib().rqa_mlp_backward(ctx.handle, _dev_ptr(params, torch.float32, RQA_MLP_PARAMS, "params"),
                                  _dev_ptr(X, torch.float32, B * RQA_FEATURES, "X"),
                                  _dev_ptr(acts, torch.float32, B * RQA_MLP_ACTS, "acts"),
                                  _dev_ptr(Y, torch.float32, B * RQA_MLP_OUT, "Y"),
                                  _dev_ptr(T, torch.float32, B * (RQA_MLP_OUT // 2), "T"), int(B),
                                  float(tau_lo), float(tau_hi),
                                  _dev_ptr(grads, torch.float32, RQA_MLP_PARAMS, "grads"),
                                  _dev_ptr(loss, torch.float32, 1, "loss")), "rqa_mlp_backward")


def rqa_adam_step(ctx: Context, params, grads, m, v, t: int, lr: float, beta1: float = 0.9,
                  beta2: float = 0.999, eps: float = 1e-8):
    import torch
    n = params.numel()
    _check(lib().rqa_adam_step(ctx.handle, _dev_ptr(params, torch.float32, n, "params"),
                               _dev_ptr(grads, torch.float32, n, "grads"),
                               _dev_ptr(m, torch.float32, n, "m"), _dev_ptr(v, torch.float32, n, "v"),
                               int(n), int(t), float(lr), float(beta1), float(beta2), float(eps)),
           "rqa_adam_step")


def rqa_set_bracket_model(ctx: Context, params, margin: float = 0.0):
    import torch
    _check(lib().rqa_set_bracket_model(ctx.handle,
                                       _dev_ptr(params, torch.float32, RQA_MLP_PARAMS, "params"),
                                       float(margin)), "rqa_set_bracket_model")


def rqa_set_bracket_domain(ctx: Context, pairs):
    """The (m, tau) embeddings the installed network was trained on; [] = any."""
    pairs = list(pairs)
    m = np.ascontiguousarray([p[0] for p in pairs], dtype=np.int32)
    tau = np.ascontiguousarray([p[1] for p in pairs], dtype=np.int32)
    _check(lib().rqa_set_bracket_domain(ctx.handle, _np_ptr(m) if pairs else None,
                                        _np_ptr(tau) if pairs else None, len(pairs)),
           "rqa_set_bracket_domain")


def rqa_log_labels(ctx: Context, eps, centre, T_out):
    """T_out (S x K) = ln(max(eps, 2^-126)) - centre[:, None], on the device."""
    import torch
    S, K = int(eps.shape[0]), int(eps.shape[1])
    _check(lib().rqa_log_labels(ctx.handle, _dev_ptr(eps, torch.float32, S * K, "eps"),
                                _dev_ptr(centre, torch.float32, S, "centre"), S, K,
                                _dev_ptr(T_out, torch.float32, S * K, "T_out")), "rqa_log_labels")


def rqa_bracket_eval(ctx: Context, Y, T, tau_lo: float, tau_hi: float, margin: float, out):
    """Summed pinball loss, targets inside the widened intervals and summed
    width, into out = (float64 scalar, uint64 scalar, float64 scalar) tensors."""
    import torch
    B, K = int(T.shape[0]), int(T.shape[1])
    loss, inside, width = out
    _check(lib().rqa_bracket_eval(ctx.handle, _dev_ptr(Y, torch.float32, B * 2 * K, "Y"),
                                  _dev_ptr(T, torch.float32, B * K, "T"), B, K, float(tau_lo),
                                  float(tau_hi), float(margin), _dev_ptr(loss, torch.float64, 1, "loss"),
                                  _dev_ptr(inside, torch.uint64, 1, "inside"),
                                  _dev_ptr(width, torch.float64, 1, "width")), "rqa_bracket_eval")


def rqa_gather_rows(ctx: Context, src, idx, dst):
    """dst[r] = src[idx[r]] for rows of src.shape[1] floats (idx: device int64)."""
    import torch
    n, width = int(idx.shape[0]), int(src.shape[1])
    _check(lib().rqa_gather_rows(ctx.handle, _dev_ptr(src, torch.float32, None, "src"),
                                 _dev_ptr(idx, torch.int64, n, "idx"), n, width,
                                 _dev_ptr(dst, torch.float32, n * width, "dst")), "rqa_gather_rows")


def rqa_bracket_stats(ctx: Context):
    h, m = c_u64(), c_u64()
    _check(lib().rqa_bracket_stats(ctx.handle, ctypes.byref(h), ctypes.byref(m)), "rqa_bracket_stats")
    return int(h.value), int(m.value)


# ------------------------------------------------------------ no allocation
RQA_NOALLOC_MAX_SERIES = 4


def rqa_eps_for_rr_noalloc(batch: Batch, rr_num, rr_den: int, eps_out, count_le=None,
                           count_lt=None, status_out=None, stream=None):
    """Thresholds without any device allocation (see rqa.h): at most
    RQA_NOALLOC_MAX_SERIES series, on the current device and the given torch
    stream (default: the current stream)."""
    import torch
    rr = np.ascontiguousarray(rr_num, dtype=np.int32)
    n = batch.n_series * len(rr)
    if stream is None:
        stream = torch.cuda.current_stream()
    b = batch._c()
    _check(lib().rqa_eps_for_rr_noalloc(ctypes.byref(b), _np_ptr(rr), int(rr_den), len(rr),
                                        _dev_ptr(eps_out, torch.float32, n, "eps_out"),
                                        _dev_ptr(count_le, torch.uint64, n, "count_le"),
                                        _dev_ptr(count_lt, torch.uint64, n, "count_lt"),
                                        _dev_ptr(status_out, torch.int32, 1, "status_out"),
                                        c_vp(stream.cuda_stream)), "rqa_eps_for_rr_noalloc")
