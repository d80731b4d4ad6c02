"""ctypes wrapper of the plain-C oracle (``rqa_oracle.c``).

TEST INFRASTRUCTURE: used by the tests, the smoke check and the benchmark's
CPU baseline only.  ``build()`` compiles the C file with gcc (no fast-math,
no FP contraction, OpenMP over diagonals).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Dict, Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "rqa_oracle.c")
LIB = os.path.join(HERE, "_build", "liborc.so")

_lib: Optional[ctypes.CDLL] = None


def build(force: bool = False) -> str:
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-o", tmp, SRC])
        os.replace(tmp, LIB)
    return LIB


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(LIB)
        P = ctypes.c_void_p
        i64 = ctypes.c_int64
        i32 = ctypes.c_int
        L.orc_distances.argtypes = [P, i64, i32, i32, P]
        L.orc_count.argtypes = [P, i64, i32, i32, P, i32, P, P, i32]
        L.orc_lines.argtypes = [P, i64, i32, i32, P, i32, P, P, P, P, P, i32, i32]
        L.orc_num_threads.argtypes = []
        for f in (L.orc_distances, L.orc_count, L.orc_lines, L.orc_num_threads):
            f.restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def num_threads() -> int:
    return int(lib().orc_num_threads())


def distances(y: np.ndarray, m: int, tau: int) -> np.ndarray:
    y = np.ascontiguousarray(y, dtype=np.float32)
    ne = len(y) - (m - 1) * tau
    out = np.empty(max(ne * (ne - 1) // 2, 0), dtype=np.float32)
    lib().orc_distances(_ptr(y), len(y), m, tau, _ptr(out))
    return out


def count(y: np.ndarray, m: int, tau: int, thr: Sequence[float], threads: int = 0):
    """(#{d <= t_k}, #{d < t_k}) for every threshold; the selection certificate."""
    y = np.ascontiguousarray(y, dtype=np.float32)
    thr = np.ascontiguousarray(thr, dtype=np.float32)
    le = np.zeros(len(thr), dtype=np.uint64)
    lt = np.zeros(len(thr), dtype=np.uint64)
    rc = lib().orc_count(_ptr(y), len(y), m, tau, _ptr(thr), len(thr), _ptr(le), _ptr(lt), threads)
    if rc != 0:
        raise ValueError("orc_count rejected its arguments")
    return le, lt


def lines(y: np.ndarray, m: int, tau: int, eps: Sequence[float], full_hist: bool = True,
          n_short: int = 0, threads: int = 0) -> Dict[str, np.ndarray]:
    """Diagonal line statistics per threshold (see ``orc_lines``)."""
    y = np.ascontiguousarray(y, dtype=np.float32)
    eps = np.ascontiguousarray(eps, dtype=np.float32)
    K = len(eps)
    ne = len(y) - (m - 1) * tau
    hist = np.zeros((K, max(ne - 1, 0)), dtype=np.uint64) if full_hist else None
    short = np.zeros((K, n_short), dtype=np.uint64) if n_short > 0 else None
    cnt = np.zeros(K, dtype=np.uint64)
    st = np.zeros(K, dtype=np.uint64)
    lmax = np.zeros(K, dtype=np.uint32)
    rc = lib().orc_lines(_ptr(y), len(y), m, tau, _ptr(eps), K,
                         _ptr(hist) if hist is not None else None,
                         _ptr(cnt), _ptr(st), _ptr(lmax),
                         _ptr(short) if short is not None else None, n_short, threads)
    if rc != 0:
        raise ValueError("orc_lines rejected its arguments")
    out = {"count": cnt, "stencil": st, "lmax": lmax}
    if hist is not None:
        out["hist"] = hist
    if short is not None:
        out["short_hist"] = short
    return out
