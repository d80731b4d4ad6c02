"""FP64 oracle of the learned threshold bracket -- TEST INFRASTRUCTURE.

Used only by the tests (and nowhere in the product path) to check the CUDA
sketch, MLP forward/backward and Adam kernels.  The paper has no learned part;
this restates the library's own definition of it, step by step:

1. Sketch.  For series s of a batch and a 64-bit seed, 4096 random pairs of
   embedded vectors are drawn with SplitMix64 (Steele, Lea & Flood, OOPSLA
   2014; the 64-bit output function with the published constants), used as a
   counter-based generator: the series key is k_s = mix(seed XOR
   (s + 1) * 0xD1B54A32D192ED03) and the t-th draw is
   u_t = mix(k_s + (t + 1) * 0x9E3779B97F4A7C15), where mix() is the SplitMix64
   output function.  Pair p uses a = u_{2p}, b = u_{2p+1}:
   i = a mod Ne, j' = b mod (Ne - 1), j = j' + [j' >= i]  (so i != j).
   Distances d = max_q |y[i+q tau] - y[j+q tau]| in FP32 (Eq. 1).
2. Features: the 4096 distances sorted ascending, quantile b (b = 0..127) is
   sorted[32 b + 16]; f_b = ln(max(q_b, 2^-126)); centre c = f_64; inputs
   x_b = f_b - c (b < 128), x_128 = log10 N, x_129 = m, x_130 = tau.
3. Network 131 -> 256 -> 256 -> 40 with ReLU between layers (three linear
   layers; W as [out][in], row-major).  Output 2k is the lower and 2k+1 the
   upper end of the bracket of ln(eps_k) - c.
4. Loss: pinball (quantile) loss, mean over the batch and the 2K outputs,
   quantile tau_lo for the lower and tau_hi for the upper ends.
5. Adam (Kingma & Ba 2015) with bias correction.
"""
from __future__ import annotations

from typing import Dict, Tuple

import numpy as np

MASK = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15
SERIES_MULT = 0xD1B54A32D192ED03
N_PAIRS = 4096
N_BINS = 128
N_FEAT = 131
HIDDEN = 256
K_OUT = 20
LAYERS = [(N_FEAT, HIDDEN), (HIDDEN, HIDDEN), (HIDDEN, 2 * K_OUT)]


def splitmix_mix(z: int) -> int:
    """SplitMix64 output function (the published 64-bit finaliser)."""
    z &= MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
    return z ^ (z >> 31)


def splitmix_stream(seed: int, n: int):
    """The sequential SplitMix64 generator: state += gamma, output mix(state)."""
    x = seed & MASK
    out = []
    for _ in range(n):
        x = (x + GAMMA) & MASK
        out.append(splitmix_mix(x))
    return out


def sketch_pairs(ne: int, s: int, seed: int) -> Tuple[np.ndarray, np.ndarray]:
    key = splitmix_mix((seed ^ (((s + 1) * SERIES_MULT) & MASK)) & MASK)
    ii = np.empty(N_PAIRS, dtype=np.int64)
    jj = np.empty(N_PAIRS, dtype=np.int64)
    for p in range(N_PAIRS):
        a = splitmix_mix((key + (2 * p + 1) * GAMMA) & MASK)
        b = splitmix_mix((key + (2 * p + 2) * GAMMA) & MASK)
        i = a % ne
        j = b % (ne - 1)
        if j >= i:
            j += 1
        ii[p] = i
        jj[p] = j
    return ii, jj


def sketch_distances(y: np.ndarray, m: int, tau: int, s: int, seed: int) -> np.ndarray:
    y = np.asarray(y, dtype=np.float32)
    ne = len(y) - (m - 1) * tau
    ii, jj = sketch_pairs(ne, s, seed)
    d = np.abs(y[ii] - y[jj])
    for q in range(1, m):
        d = np.maximum(d, np.abs(y[ii + q * tau] - y[jj + q * tau]))
    return np.sort(d.astype(np.float32))


def sketch_features(y: np.ndarray, m: int, tau: int, s: int, seed: int):
    """(x[131] FP64, centre c, the 128 FP32 quantile distances)."""
    srt = sketch_distances(y, m, tau, s, seed)
    q = srt[32 * np.arange(N_BINS) + 16]
    f = np.log(np.maximum(q.astype(np.float64), 2.0 ** -126))
    c = f[64]
    x = np.zeros(N_FEAT, dtype=np.float64)
    x[:N_BINS] = f - c
    x[128] = np.log10(len(y))
    x[129] = m
    x[130] = tau
    return x, c, q


def n_params() -> int:
    return sum(o * i + o for i, o in LAYERS)


def unpack(params: np.ndarray):
    """Split the flat parameter vector into [(W[out][in], b[out]), ...]."""
    out = []
    off = 0
    for i, o in LAYERS:
        W = params[off:off + o * i].reshape(o, i)
        off += o * i
        b = params[off:off + o]
        off += o
        out.append((W, b))
    return out


def forward(params: np.ndarray, X: np.ndarray) -> Dict[str, np.ndarray]:
    (W1, b1), (W2, b2), (W3, b3) = unpack(np.asarray(params, dtype=np.float64))
    X = np.asarray(X, dtype=np.float64)
    Z1 = X @ W1.T + b1
    H1 = np.maximum(Z1, 0.0)
    Z2 = H1 @ W2.T + b2
    H2 = np.maximum(Z2, 0.0)
    Y = H2 @ W3.T + b3
    return {"Z1": Z1, "H1": H1, "Z2": Z2, "H2": H2, "Y": Y}


def pinball(Y: np.ndarray, T: np.ndarray, tau_lo: float, tau_hi: float):
    """Mean quantile loss and its gradient w.r.t. Y (B x 2K); T is B x K."""
    B, two_k = Y.shape
    taus = np.tile([tau_lo, tau_hi], two_k // 2)
    Tt = np.repeat(T, 2, axis=1)
    r = Tt - Y
    loss = np.where(r >= 0, taus * r, (taus - 1.0) * r)
    g = np.where(r >= 0, -taus, 1.0 - taus) / (B * two_k)
    return float(loss.sum() / (B * two_k)), g


def backward(params: np.ndarray, X: np.ndarray, T: np.ndarray, tau_lo: float, tau_hi: float):
    """(loss, flat gradient) of the mean pinball loss, by the chain rule."""
    (W1, b1), (W2, b2), (W3, b3) = unpack(np.asarray(params, dtype=np.float64))
    f = forward(params, X)
    loss, dY = pinball(f["Y"], np.asarray(T, dtype=np.float64), tau_lo, tau_hi)
    gW3 = dY.T @ f["H2"]
    gb3 = dY.sum(axis=0)
    dH2 = dY @ W3
    dZ2 = dH2 * (f["Z2"] > 0)
    gW2 = dZ2.T @ f["H1"]
    gb2 = dZ2.sum(axis=0)
    dH1 = dZ2 @ W2
    dZ1 = dH1 * (f["Z1"] > 0)
    gW1 = dZ1.T @ np.asarray(X, dtype=np.float64)
    gb1 = dZ1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return loss, g


def adam(params, grads, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (t counts from 1); returns new (params, m, v)."""
    m = b1 * m + (1 - b1) * grads
    v = b2 * v + (1 - b2) * grads * grads
    mhat = m / (1 - b1 ** t)
    vhat = v / (1 - b2 ** t)
    return params - lr * mhat / (np.sqrt(vhat) + eps), m, v


def init_params(seed: int = 0) -> np.ndarray:
    """He-uniform weights, zero biases (FP32)."""
    rng = np.random.default_rng(seed)
    parts = []
    for i, o in LAYERS:
        lim = np.sqrt(6.0 / i)
        parts.append(rng.uniform(-lim, lim, size=o * i))
        parts.append(np.zeros(o))
    return np.concatenate(parts).astype(np.float32)
