"""Seeded synthetic inputs for averaged RQA.

This package only *produces input series*: it holds none of the method's
arithmetic (no distances, thresholds, recurrence or line counting).  Both the
CUDA path (through the tests and the benchmark) and the CPU oracle consume the
arrays it returns, so neither depends on the other.
"""
from .series import (  # noqa: F401
    logistic, lorenz_x, sine, add_noise_db, make_series,
    SeriesSpec, Workload, workload, WORKLOADS,
)
