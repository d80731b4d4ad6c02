"""rqa_eps_for_rr_noalloc: thresholds for callers that cannot allocate device
memory when they need them (their scratch is a fixed array inside the
library).  Its results must equal those of rqa_eps_for_rr bit for bit, call
after call, since every call reuses -- and so must first clear -- the same
scratch.  This file is collected last on purpose."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

RR = list(range(1, 21))


def _batches():
    rng = np.random.default_rng(2024)
    t = np.arange(3000)
    first = ([(np.sin(2 * np.pi * t[:700] / 20.3) + 0.3 * rng.standard_normal(700)).astype(np.float32),
              rng.standard_normal(2000).astype(np.float32),
              (np.round(rng.standard_normal(150) * 2) / 2).astype(np.float32)], 3, 3)
    second = ([rng.standard_normal(int(n)).astype(np.float32) for n in (3000, 64, 999, 1500)], 1, 1)
    return [first, second]


def test_noalloc_equals_eps_for_rr_on_consecutive_calls(rqa_lib):
    import torch
    rqa = rqa_lib
    ctx = rqa.Context(select=rqa.RQA_SELECT_RADIX)
    for ys, m, tau in _batches():
        batch = rqa.Batch.from_numpy(ys, m, tau)
        S, K = batch.n_series, len(RR)
        ref = rqa.eps_for_rr(ctx, batch, RR, 100)
        assert rqa.rqa_status(ctx) == 0
        eps = torch.empty((S, K), dtype=torch.float32, device="cuda")
        le = torch.empty((S, K), dtype=torch.uint64, device="cuda")
        lt = torch.empty((S, K), dtype=torch.uint64, device="cuda")
        st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        rqa.rqa_eps_for_rr_noalloc(batch, RR, 100, eps, le, lt, st)
        torch.cuda.synchronize()
        assert int(st.item()) == 0
        assert np.array_equal(eps.cpu().numpy(), ref["eps"].cpu().numpy())
        assert np.array_equal(le.cpu().numpy(), ref["count_le"].cpu().numpy())
        assert np.array_equal(lt.cpu().numpy(), ref["count_lt"].cpu().numpy())
    ctx.close()


def test_noalloc_rejects_too_many_series(rqa_lib):
    import torch
    rqa = rqa_lib
    ys = [np.random.default_rng(s).standard_normal(100).astype(np.float32)
          for s in range(rqa.RQA_NOALLOC_MAX_SERIES + 1)]
    batch = rqa.Batch.from_numpy(ys, 1, 1)
    eps = torch.empty((batch.n_series, 20), dtype=torch.float32, device="cuda")
    with pytest.raises(rqa.RqaError) as ei:
        rqa.rqa_eps_for_rr_noalloc(batch, RR, 100, eps)
    assert ei.value.code == 7  # RQA_ERR_CAPACITY


def test_noalloc_limits_of_its_layout(rqa_lib):
    """The fixed scratch at its limits: K = RQA_NOALLOC_K_MAX targets (the
    final round's per-target tables at full stride), four series with four
    different embeddings (the generic distance kernels), and one series long
    enough (N = 6 * 10^5) that its work items hold twice the usual bands; bit
    for bit the results of rqa_eps_for_rr, on two calls in a row."""
    import torch
    rqa = rqa_lib
    rng = np.random.default_rng(77)
    K = rqa.RQA_NOALLOC_K_MAX
    rr = list(range(1, K + 1))
    t = np.arange(600_000)
    cases = [
        ([rng.standard_normal(n).astype(np.float32) for n in (900, 1500, 400, 2500)],
         [1, 2, 3, 4], [1, 2, 3, 1]),
        ([(np.sin(2 * np.pi * t / 20.3) + 0.5 * rng.standard_normal(t.size)).astype(np.float32)],
         [3], [3]),
    ]
    ctx = rqa.Context(select=rqa.RQA_SELECT_RADIX)
    for ys, m, tau in cases:
        batch = rqa.Batch.from_numpy(ys, m, tau)
        S = batch.n_series
        ref = rqa.eps_for_rr(ctx, batch, rr, 100)
        assert rqa.rqa_status(ctx) == 0
        for _ in range(2):
            eps = torch.empty((S, K), dtype=torch.float32, device="cuda")
            le = torch.empty((S, K), dtype=torch.uint64, device="cuda")
            lt = torch.empty((S, K), dtype=torch.uint64, device="cuda")
            st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
            rqa.rqa_eps_for_rr_noalloc(batch, rr, 100, eps, le, lt, st)
            torch.cuda.synchronize()
            assert int(st.item()) == 0
            assert np.array_equal(eps.cpu().numpy(), ref["eps"].cpu().numpy())
            assert np.array_equal(le.cpu().numpy(), ref["count_le"].cpu().numpy())
            assert np.array_equal(lt.cpu().numpy(), ref["count_lt"].cpu().numpy())
    ctx.close()


def test_noalloc_rejects_buffers_of_the_host(rqa_lib):
    """Outputs the device cannot address (here: host memory) are refused
    before anything is enqueued."""
    import ctypes
    import torch
    rqa = rqa_lib
    from paper_2208_09136_gb300 import abi
    batch = rqa.Batch.from_numpy([np.random.default_rng(3).standard_normal(200).astype(np.float32)], 1, 1)
    host_eps = np.empty(20, dtype=np.float32)
    rr = np.arange(1, 21, dtype=np.int32)
    b = batch._c()
    rc = abi.lib().rqa_eps_for_rr_noalloc(ctypes.byref(b), rr.ctypes.data, 100, 20,
                                         ctypes.c_void_p(host_eps.ctypes.data), None, None, None,
                                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 1  # RQA_ERR_INVALID_ARG
