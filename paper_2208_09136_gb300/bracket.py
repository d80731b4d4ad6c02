"""Training and storage of the learned threshold bracket.

The network (``include/rqa_learn.h``) maps a series' distance sketch to
intervals of ln(eps_k) for RR = 1..20 %.  It is trained here on the GPU with
the library's own kernels only: exact thresholds from ``rqa_eps_for_rr``
(radix selection) are the labels, ``rqa_sketch`` gives the inputs, and
``rqa_mlp_forward`` / ``rqa_mlp_backward`` / ``rqa_adam_step`` fit it with
the pinball loss at quantiles tau_lo / tau_hi.  PyTorch only allocates.

Model file: 8-byte magic ``RQAMLP02``, uint32 parameter count, float32
margin, float32 tau_lo, float32 tau_hi, uint32 number of training
embeddings n, n pairs of int32 (m, tau), the float32 parameters, uint32
CRC-32 of the embedding and parameter bytes.  (``RQAMLP01`` files, without
the embeddings, load with an unrestricted domain.)  ``python -m
paper_2208_09136_gb300.bracket train --out FILE`` trains one.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import struct
import sys
import time
import zlib
from typing import Dict, Optional

import numpy as np

from . import abi

MAGIC = b"RQAMLP02"
MAGIC_V1 = b"RQAMLP01"
MODEL_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "models")
MODEL_PATH = os.path.join(MODEL_DIR, "bracket_mlp.bin")
RR = list(range(1, 21))
LAYERS = [(131, 256), (256, 256), (256, 40)]
TINY = 2.0 ** -126


def save_model(path: str, params: np.ndarray, margin: float, tau_lo: float, tau_hi: float,
               domain=((3, 3),)):
    """domain: the (m, tau) embeddings of the training series."""
    params = np.ascontiguousarray(params, dtype=np.float32)
    assert params.size == abi.RQA_MLP_PARAMS
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    dom = np.ascontiguousarray(list(domain), dtype=np.int32).reshape(-1, 2)
    body = dom.tobytes() + params.tobytes()
    with open(path, "wb") as f:
        f.write(MAGIC)
        f.write(struct.pack("<Ifff", params.size, margin, tau_lo, tau_hi))
        f.write(struct.pack("<I", dom.shape[0]))
        f.write(body)
        f.write(struct.pack("<I", zlib.crc32(body) & 0xFFFFFFFF))


def load_model(path: str = MODEL_PATH) -> Dict[str, object]:
    raw = open(path, "rb").read()
    if raw[:8] not in (MAGIC, MAGIC_V1):
        raise ValueError(f"{path}: not a bracket model")
    n, margin, tau_lo, tau_hi = struct.unpack("<Ifff", raw[8:24])
    pos, domain = 24, []
    if raw[:8] == MAGIC:
        (nd,) = struct.unpack("<I", raw[24:28])
        pos = 28
        dom = np.frombuffer(raw[pos:pos + 8 * nd], dtype=np.int32).reshape(-1, 2)
        domain = [(int(a), int(b)) for a, b in dom]
        pos += 8 * nd
    if n != abi.RQA_MLP_PARAMS or len(raw) != pos + 4 * n + 4:
        raise ValueError(f"{path}: wrong size")
    body = raw[24 if raw[:8] == MAGIC_V1 else 28:pos + 4 * n]
    (crc,) = struct.unpack("<I", raw[pos + 4 * n:])
    if zlib.crc32(body) & 0xFFFFFFFF != crc:
        raise ValueError(f"{path}: checksum mismatch")
    return {"params": np.frombuffer(raw[pos:pos + 4 * n], dtype=np.float32).copy(),
            "margin": margin, "tau_lo": tau_lo, "tau_hi": tau_hi, "domain": domain}


def install(ctx: abi.Context, path: str = MODEL_PATH, margin: Optional[float] = None):
    """Load a model file and install it in a context, with its training
    domain (RQA_SELECT_AUTO brackets only series with those embeddings);
    returns the model dict."""
    import torch
    m = load_model(path)
    t = torch.from_numpy(m["params"]).to(f"cuda:{ctx.device}")
    abi.rqa_set_bracket_model(ctx, t, m["margin"] if margin is None else margin)
    abi.rqa_set_bracket_domain(ctx, m["domain"])
    torch.cuda.synchronize(ctx.device)
    return m


def init_params(seed: int = 0) -> np.ndarray:
    """He-uniform weights, zero biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for i, o in LAYERS:
        lim = math.sqrt(6.0 / i)
        parts.append(rng.uniform(-lim, lim, size=o * i))
        parts.append(np.zeros(o))
    return np.concatenate(parts).astype(np.float32)


def make_dataset(specs, device: int = 0, chunk: int = 2000, seed: int = 1):
    """Sketch features X (n x 131) and targets T = ln(max(eps_k, 2^-126)) - c
    (n x 20), on the GPU, for the series of the given specs: exact thresholds
    by rqa_eps_for_rr, features by rqa_sketch, labels by rqa_log_labels."""
    import torch
    from synth.series import _make_many
    ctx = abi.Context(device=device, select=abi.RQA_SELECT_RADIX)
    dev = f"cuda:{device}"
    n = len(specs)
    X = torch.empty((n, 131), dtype=torch.float32, device=dev)
    T = torch.empty((n, 20), dtype=torch.float32, device=dev)
    for a in range(0, n, chunk):
        part = specs[a:a + chunk]
        ys = _make_many(part, cache=False)
        batch = abi.Batch.from_numpy(ys, [sp.m for sp in part], [sp.tau for sp in part], device)
        S = batch.n_series
        eps = torch.empty((S, 20), dtype=torch.float32, device=dev)
        abi.rqa_eps_for_rr(ctx, batch, RR, 100, eps)
        centre = torch.empty(S, dtype=torch.float32, device=dev)
        abi.rqa_sketch(ctx, batch, seed, X[a:a + S], centre)
        abi.rqa_log_labels(ctx, eps, centre, T[a:a + S])
        code = abi.rqa_status(ctx)
        if code:
            raise RuntimeError(abi.rqa_error_string(code))
    ctx.close()
    return X, T


def train(workload: str = "train-20000", epochs: int = 60, batch_size: int = 256,
          lr: float = 2e-3, tau_lo: float = 0.005, tau_hi: float = 0.995, seed: int = 0,
          device: int = 0, val_frac: float = 0.1, log=print) -> Dict[str, object]:
    import torch
    from synth import workload as wl
    t0 = time.time()
    specs = wl(workload).specs
    X, T = make_dataset(specs, device)
    n = X.shape[0]
    rng = np.random.default_rng(seed)
    perm = rng.permutation(n)
    n_val = int(n * val_frac)
    val_idx = torch.from_numpy(perm[:n_val]).to(X.device)
    tr_idx = perm[n_val:]
    log(f"dataset: {n} series ({n - n_val} train / {n_val} val), {time.time() - t0:.1f} s")

    ctx = abi.Context(device=device)
    dev = X.device
    params = torch.from_numpy(init_params(seed)).to(dev)
    grads = torch.zeros_like(params)
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    B = batch_size
    Y = torch.empty((B, 40), dtype=torch.float32, device=dev)
    acts = torch.empty((B, 512), dtype=torch.float32, device=dev)
    xb = torch.empty((B, 131), dtype=torch.float32, device=dev)
    tb = torch.empty((B, 20), dtype=torch.float32, device=dev)
    Xv = torch.empty((n_val, 131), dtype=torch.float32, device=dev)
    Tv = torch.empty((n_val, 20), dtype=torch.float32, device=dev)
    abi.rqa_gather_rows(ctx, X, val_idx, Xv)
    abi.rqa_gather_rows(ctx, T, val_idx, Tv)
    step = 0
    steps_per_epoch = len(tr_idx) // B
    total = epochs * steps_per_epoch
    hist = []
    for ep in range(epochs):
        order = torch.from_numpy(rng.permutation(tr_idx)).to(dev)
        ep_loss = 0.0
        for i in range(steps_per_epoch):
            idx = order[i * B:(i + 1) * B]
            abi.rqa_gather_rows(ctx, X, idx, xb)
            abi.rqa_gather_rows(ctx, T, idx, tb)
            abi.rqa_mlp_forward(ctx, params, xb, Y, acts)
            abi.rqa_mlp_backward(ctx, params, xb, acts, Y, tb, tau_lo, tau_hi, grads, loss)
            step += 1
            cur_lr = lr * 0.5 * (1.0 + math.cos(math.pi * step / total))  # cosine decay
            abi.rqa_adam_step(ctx, params, grads, m, v, step, cur_lr)
            if i % 16 == 0:
                ep_loss += float(loss.item())
        vl = evaluate(ctx, params, Xv, Tv, tau_lo, tau_hi)
        hist.append(vl)
        if ep % 5 == 0 or ep == epochs - 1:
            log(f"epoch {ep:3d} val loss {vl['loss']:.5f} cover {vl['cover']:.4f} "
                f"width {vl['width']:.4f} ({time.time() - t0:.1f} s)")
    out = {"params": params.cpu().numpy(), "tau_lo": tau_lo, "tau_hi": tau_hi, "val": hist[-1],
           "seconds": time.time() - t0, "domain": sorted({(sp.m, sp.tau) for sp in specs})}
    ctx.close()
    return out


def evaluate(ctx, params, X, T, tau_lo, tau_hi, margin: float = 0.0):
    """Validation loss (mean pinball loss of the 40 outputs), fraction of
    targets inside [lo - margin, hi + margin] and the mean widened interval
    width (ln units), all computed by rqa_bracket_eval."""
    import torch
    n = X.shape[0]
    Y = torch.empty((n, 40), dtype=torch.float32, device=X.device)
    abi.rqa_mlp_forward(ctx, params, X, Y)
    out = (torch.empty(1, dtype=torch.float64, device=X.device),
           torch.empty(1, dtype=torch.uint64, device=X.device),
           torch.empty(1, dtype=torch.float64, device=X.device))
    abi.rqa_bracket_eval(ctx, Y, T, tau_lo, tau_hi, margin, out)
    loss, inside, width = (float(v.cpu().item()) for v in out)
    m = n * T.shape[1]
    return {"loss": loss / (2 * m), "cover": inside / m, "width": width / m}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__)
    sub = ap.add_subparsers(dest="cmd", required=True)
    t = sub.add_parser("train")
    t.add_argument("--out", default=MODEL_PATH)
    t.add_argument("--epochs", type=int, default=60)
    t.add_argument("--workload", default="train-20000")
    t.add_argument("--margin", type=float, default=0.05)
    t.add_argument("--device", type=int, default=0)
    a = ap.parse_args(argv)
    if a.cmd == "train":
        res = train(a.workload, epochs=a.epochs, device=a.device)
        save_model(a.out, res["params"], a.margin, res["tau_lo"], res["tau_hi"], res["domain"])
        print(json.dumps({"saved": a.out, "val": res["val"], "seconds": res["seconds"],
                          "margin": a.margin}))
    return 0


if __name__ == "__main__":
    sys.exit(main())
