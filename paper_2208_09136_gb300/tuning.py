"""A JSON cache of the line pass's tuned knobs (``rqa_autotune``).

The best register window, work-unit size and CTAs per SM depend on the GPU and
on the batch's shape, not on its values, so a tuning result is stored under
a key made of the GPU name and SM count and the batch's class: the largest
series length as a power-of-two bucket, the embedding (m, tau, or "mixed")
and the number of thresholds K.  ``tuned()`` looks the key up, installs a
stored result with ``rqa_set_tuning`` or else runs ``rqa_autotune`` and stores
what it chose.  Any setting gives the same results; only the time differs.

Default file: $RQA_TUNE_CACHE, else ~/.cache/rqa/tuning.json.
"""
from __future__ import annotations

import json
import math
import os
from typing import Optional

import numpy as np

from . import abi


def cache_path() -> str:
    return os.environ.get("RQA_TUNE_CACHE") or os.path.join(
        os.path.expanduser("~"), ".cache", "rqa", "tuning.json")


def batch_key(gpu_name: str, sm_count: int, offsets, m, tau, K: int) -> str:
    """The cache key of a batch on a GPU."""
    n = np.diff(np.asarray(offsets, dtype=np.int64))
    n_bucket = int(math.ceil(math.log2(max(int(n.max()), 2))))
    m = np.asarray(m)
    tau = np.asarray(tau)
    emb = f"m{int(m[0])}t{int(tau[0])}" if (m == m[0]).all() and (tau == tau[0]).all() else "mixed"
    return f"{gpu_name}|sm{int(sm_count)}|n2^{n_bucket}|{emb}|K{int(K)}"


def load(path: Optional[str] = None) -> dict:
    try:
        with open(path or cache_path()) as f:
            data = json.load(f)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}


def store(entries: dict, path: Optional[str] = None):
    path = path or cache_path()
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    tmp = f"{path}.{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(entries, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tuned(ctx: abi.Context, batch: abi.Batch, rr_num, rr_den: int, path: Optional[str] = None,
          gpu_name: Optional[str] = None) -> dict:
    """The context's line-pass knobs for this batch: from the cache when the
    key is there, else tuned now (and stored).  Returns the knobs with
    "cached" telling which."""
    if gpu_name is None:
        import torch
        gpu_name = torch.cuda.get_device_name(ctx.device)
    sm = abi.rqa_device_info(ctx)["sm_count"]
    key = batch_key(gpu_name, sm, batch.offsets, batch.m, batch.tau, len(rr_num))
    entries = load(path)
    hit = entries.get(key)
    if isinstance(hit, dict) and {"tile", "unit_bands", "line_ctas"} <= set(hit):
        abi.rqa_set_tuning(ctx, hit["tile"], hit["unit_bands"], hit["line_ctas"], hit.get("stage", 0))
        return dict(abi.rqa_get_tuning(ctx), cached=True, key=key)
    got = abi.rqa_autotune(ctx, batch, rr_num, rr_den)
    entries = load(path)  # another process may have written meanwhile
    entries[key] = {k: got[k] for k in ("tile", "unit_bands", "line_ctas", "stage", "ms")}
    store(entries, path)
    return dict(got, cached=False, key=key)
