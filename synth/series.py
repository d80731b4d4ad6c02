"""Seeded synthetic time series with the shapes of the paper's workloads.

The paper's own data (RobPer sine light curves, its logistic-map and Lorenz
runs with unpublished noise realisations; Sect. 3.1-3.3) are not available, so
these generators stand in for them.  Every series is produced in FP64 from a
NumPy PCG64 stream that is fully determined by its ``SeriesSpec`` and then cast
to FP32, the precision the method works in.

Readings of the paper used here:

* Logistic map ``x_{n+1} = r x_n (1 - x_n)`` (Sect. 3.2).  The workloads use
  r = 4 (the paper's r = 3.679 is available through ``r=``); x0 ~ U(0.1, 0.9);
  the first 1000 iterates are dropped.  An orbit that reaches exactly 0 or 1
  (absorbing in FP64) or has zero variance is redrawn from the same stream.
* Lorenz system (Sect. 3.3) with sigma = 10, rho = 28, beta = 8/3.  The printed
  y-equation lacks its ``- y`` term; the standard system is used.  Classical
  RK4 with dt = 0.01, x0 = (1, 1, 1) + 0.1 N(0, 1)^3, 5000 transient steps,
  then the x component every 5 steps, z-scored in FP64.
* Sine (Sect. 3.1 stand-in): ``sin(2 pi n / 20.3 + phi)``, phi ~ U(0, 2 pi).
* Noise (Sect. 3): SNR is var(signal) / var(noise); given in dB here, so
  sigma = sqrt(var(clean) / 10^(dB / 10)), Gaussian, drawn after the signal's
  own draws from the same stream.  Clean + noise is summed in FP64.
"""
from __future__ import annotations

import math
import os
from dataclasses import dataclass, field
from typing import Dict, List, Sequence

import numpy as np

KIND_CODE = {"sine": 1, "logistic": 2, "lorenz": 3}
KINDS = ("sine", "logistic", "lorenz")


@dataclass(frozen=True)
class SeriesSpec:
    kind: str
    n: int
    snr_db: float
    seed: int
    m: int = 1
    tau: int = 1

    def rng(self) -> np.random.Generator:
        snr_code = int(round((self.snr_db + 1000.0) * 1000.0))
        return np.random.default_rng([int(self.seed), KIND_CODE[self.kind], int(self.n), snr_code])


def logistic(n: int, rng: np.random.Generator, r: float = 4.0, transient: int = 1000) -> np.ndarray:
    """Logistic-map orbit of length n in FP64 (Sect. 3.2)."""
    for _ in range(64):
        x = rng.uniform(0.1, 0.9)
        for _ in range(transient):
            x = r * x * (1.0 - x)
        out = np.empty(n, dtype=np.float64)
        ok = True
        for t in range(n):
            out[t] = x
            if x <= 0.0 or x >= 1.0:
                ok = False
                break
            x = r * x * (1.0 - x)
        if ok and np.var(out) > 0.0:
            return out
    raise RuntimeError("logistic map: no admissible orbit in 64 draws")


def _lorenz_batch(x0: np.ndarray, n: int, dt: float = 0.01, every: int = 5,
                  transient: int = 5000, sigma: float = 10.0, rho: float = 28.0,
                  beta: float = 8.0 / 3.0) -> np.ndarray:
    """Classical RK4 for a batch of Lorenz initial states; returns x samples (B, n)."""
    x = x0[:, 0].copy()
    y = x0[:, 1].copy()
    z = x0[:, 2].copy()
    h = dt
    h2 = 0.5 * dt
    h6 = dt / 6.0

    def f(x, y, z):
        return sigma * (y - x), x * (rho - z) - y, x * y - beta * z

    out = np.empty((x0.shape[0], n), dtype=np.float64)
    total = transient + n * every
    k = 0
    for step in range(total):
        ax, ay, az = f(x, y, z)
        bx, by, bz = f(x + h2 * ax, y + h2 * ay, z + h2 * az)
        cx, cy, cz = f(x + h2 * bx, y + h2 * by, z + h2 * bz)
        dx, dy, dz = f(x + h * cx, y + h * cy, z + h * cz)
        x = x + h6 * (ax + 2.0 * bx + 2.0 * cx + dx)
        y = y + h6 * (ay + 2.0 * by + 2.0 * cy + dy)
        z = z + h6 * (az + 2.0 * bz + 2.0 * cz + dz)
        s = step + 1 - transient
        if s > 0 and s % every == 0:
            out[:, k] = x
            k += 1
    assert k == n
    return out


def lorenz_x(n: int, rng: np.random.Generator) -> np.ndarray:
    """z-scored Lorenz x component of length n in FP64 (Sect. 3.3)."""
    x0 = np.array([[1.0, 1.0, 1.0]]) + 0.1 * rng.standard_normal((1, 3))
    x = _lorenz_batch(x0, n)[0]
    return (x - x.mean()) / x.std()


def sine(n: int, rng: np.random.Generator, period: float = 20.3) -> np.ndarray:
    phi = rng.uniform(0.0, 2.0 * math.pi)
    t = np.arange(n, dtype=np.float64)
    return np.sin(2.0 * math.pi * t / period + phi)


def add_noise_db(clean: np.ndarray, snr_db: float, rng: np.random.Generator) -> np.ndarray:
    var_s = float(np.var(clean))
    sd = math.sqrt(var_s / (10.0 ** (snr_db / 10.0)))
    return clean + sd * rng.standard_normal(clean.shape[0])


_CACHE_DIR = os.environ.get("RQA_SYNTH_CACHE", os.path.join("/tmp", "rqa_synth_cache"))


def _cache_path(spec: SeriesSpec) -> str:
    return os.path.join(_CACHE_DIR, f"{spec.kind}_{spec.n}_{spec.snr_db:+.3f}_{spec.seed}.npy")


def make_series(spec: SeriesSpec, cache: bool = True) -> np.ndarray:
    """FP32 series for one spec (embedding parameters are carried separately)."""
    path = _cache_path(spec)
    if cache and os.path.exists(path):
        try:
            arr = np.load(path)
            if arr.dtype == np.float32 and arr.shape == (spec.n,):
                return arr
        except Exception:
            pass
    rng = spec.rng()
    if spec.kind == "logistic":
        clean = logistic(spec.n, rng)
    elif spec.kind == "lorenz":
        clean = lorenz_x(spec.n, rng)
    elif spec.kind == "sine":
        clean = sine(spec.n, rng)
    else:
        raise ValueError(spec.kind)
    out = add_noise_db(clean, spec.snr_db, rng).astype(np.float32)
    if cache and spec.n >= 20000:
        try:
            os.makedirs(_CACHE_DIR, exist_ok=True)
            tmp = path + f".{os.getpid()}.tmp.npy"
            np.save(tmp, out)
            os.replace(tmp, path)
        except OSError:
            pass
    return out


def _make_many(specs: Sequence[SeriesSpec], cache: bool = True) -> List[np.ndarray]:
    """Like make_series over a list.  All uncached Lorenz runs are integrated
    as one RK4 batch up to the longest of them; each series keeps its own
    first N samples, so the arithmetic per series is that of a lone run."""
    out: List[np.ndarray] = [None] * len(specs)  # type: ignore
    pending: List[int] = []
    for idx, sp in enumerate(specs):
        if sp.kind == "lorenz" and not (cache and os.path.exists(_cache_path(sp))):
            pending.append(idx)
        else:
            out[idx] = make_series(sp, cache=cache)
    if pending:
        rngs = [specs[i].rng() for i in pending]
        x0 = np.stack([np.array([1.0, 1.0, 1.0]) + 0.1 * r.standard_normal(3) for r in rngs])
        n_max = max(specs[i].n for i in pending)
        xs = _lorenz_batch(x0, n_max)
        for row, (i, r) in enumerate(zip(pending, rngs)):
            n = specs[i].n
            x = xs[row, :n]
            clean = (x - x.mean()) / x.std()
            y = add_noise_db(clean, specs[i].snr_db, r).astype(np.float32)
            out[i] = y
            if cache and n >= 20000:
                try:
                    os.makedirs(_CACHE_DIR, exist_ok=True)
                    p = _cache_path(specs[i])
                    tmp = p + f".{os.getpid()}.tmp.npy"
                    np.save(tmp, y)
                    os.replace(tmp, p)
                except OSError:
                    pass
    return out


@dataclass
class Workload:
    name: str
    specs: List[SeriesSpec]
    rr_num: List[int] = field(default_factory=lambda: list(range(1, 21)))
    rr_den: int = 100
    lmin: List[int] = field(default_factory=lambda: [2])
    hist: bool = False

    def series(self, cache: bool = True) -> List[np.ndarray]:
        return _make_many(self.specs, cache=cache)

    def pack(self, cache: bool = True):
        """Concatenated FP32 series + int64 offsets + int32 m, tau arrays."""
        ys = self.series(cache=cache)
        offsets = np.zeros(len(ys) + 1, dtype=np.int64)
        offsets[1:] = np.cumsum([len(y) for y in ys])
        flat = np.concatenate(ys).astype(np.float32) if ys else np.zeros(0, np.float32)
        m = np.array([s.m for s in self.specs], dtype=np.int32)
        tau = np.array([s.tau for s in self.specs], dtype=np.int32)
        return flat, offsets, m, tau


SNR_C3 = [-20.0, -15.0, -10.0, -5.0, 0.0, 5.0, 10.0, 20.0]


def _logu_int(rng: np.random.Generator, lo: float, hi: float) -> int:
    return int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))


def workload(name: str) -> Workload:
    """Named synthetic workloads with the paper's shapes (Sect. 3)."""
    if name == "logistic-n100":
        return Workload(name, [SeriesSpec("logistic", 100, 10.0, 1, 1, 1)])
    if name == "lorenz-n1e4":
        return Workload(name, [SeriesSpec("lorenz", 10_000, s, 2, 3, 3) for s in (-10.0, 0.0, 10.0, 20.0)],
                        hist=True)
    if name == "batched-720":
        specs = [SeriesSpec(k, n, s, seed, 3, 1)
                 for n in (100, 1000, 10_000) for k in KINDS for s in SNR_C3 for seed in range(10)]
        return Workload(name, specs)
    if name == "train-20000":
        rng = np.random.default_rng(20000)
        specs = []
        for i in range(20000):
            kind = KINDS[i % 3]
            n = _logu_int(rng, 100, 10_000)
            snr = float(np.round(rng.uniform(-20.0, 20.0), 3))
            specs.append(SeriesSpec(kind, n, snr, 1000 + i, 3, 3))
        return Workload(name, specs)
    if name == "lorenz-n1e5-eval":
        return Workload(name, [SeriesSpec("lorenz", 100_000, s, 90_000 + i, 3, 3)
                               for i, s in enumerate((-10.0, 0.0, 10.0))])
    if name in ("full-296", "full-296-short"):
        specs = [SeriesSpec(k, 100_000, s, seed, 3, 3) for k in KINDS for s in SNR_C3 for seed in range(4)]
        rng = np.random.default_rng(7)
        short = []
        for i in range(200):
            n = _logu_int(rng, 100, 10_000)
            kind = KINDS[int(rng.integers(0, 3))]
            snr = SNR_C3[int(rng.integers(0, len(SNR_C3)))]
            short.append(SeriesSpec(kind, n, snr, 7_000 + i, 3, 3))
        if name == "full-296-short":
            return Workload(name, short, lmin=[2, 3, 5], hist=True)
        return Workload(name, specs + short, lmin=[2, 3, 5], hist=True)
    raise KeyError(name)


WORKLOADS = ("logistic-n100", "lorenz-n1e4", "batched-720", "train-20000",
             "lorenz-n1e5-eval", "full-296", "full-296-short")
