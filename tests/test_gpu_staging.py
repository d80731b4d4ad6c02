"""Series windows staged by bulk copies into shared memory (rqa_tuning.stage).

The staged line pass must give the unstaged one's outputs bit for bit, and
the oracle's: for series lengths of every residue mod 4 (the copies start on
16-byte boundaries, so each series puts its rows at another offset in the
buffers), a last series that ends at the end of the batch buffer (its last
interior blocks cannot widen their copies past it and read directly), and a
batch buffer that is not 16-byte aligned (no copies at all)."""
import numpy as np
import pytest

from tests._helpers import RR20, oracle_series

pytestmark = pytest.mark.gpu

SIZES = [5001, 3334, 2223, 1112, 777]


def _series(seed, sizes):
    rng = np.random.default_rng(seed)
    out = []
    for i, n in enumerate(sizes):
        t = np.arange(n)
        if i % 2 == 0:
            out.append((np.sin(2 * np.pi * t / 17.7) + 0.2 * rng.standard_normal(n)).astype(np.float32))
        else:
            out.append(rng.standard_normal(n).astype(np.float32))
    return out


def _lines(rqa, ctx, batch, eps, tile, stage):
    import torch
    rqa.rqa_set_tuning(ctx, tile=tile, stage=stage)
    out = rqa.line_hist(ctx, batch, eps, 20, full=True)
    torch.cuda.synchronize()
    code = rqa.rqa_status(ctx)
    assert code == 0, rqa.rqa_error_string(code)
    return {"hist": rqa.unpack_hist(out["hist"].cpu().numpy(), out["hist_offsets"], batch, 20),
            "lmax": out["lmax"].cpu().numpy(), "count": out["count"].cpu().numpy()}


def _same(a, b, tag):
    assert np.array_equal(a["lmax"], b["lmax"]), (tag, "lmax")
    assert np.array_equal(a["count"], b["count"]), (tag, "count")
    for s, (x, y) in enumerate(zip(a["hist"], b["hist"])):
        assert np.array_equal(x, y), (tag, "hist", s)


@pytest.mark.parametrize("m,tau", [(3, 3), (3, 1)])
def test_staged_windows_match_unstaged_and_oracle(rqa_lib, m, tau):
    import torch
    rqa = rqa_lib
    ys = _series(31 + tau, SIZES)
    ctx = rqa.Context(device=0, select=rqa.RQA_SELECT_RADIX)
    batch = rqa.Batch.from_numpy(ys, m, tau, device=0)
    eps = rqa.eps_for_rr(ctx, batch, RR20, 100)["eps"]
    torch.cuda.synchronize()
    base = _lines(rqa, ctx, batch, eps, 16, 0)
    for tile in (16, 32):
        _same(_lines(rqa, ctx, batch, eps, tile, 1), base, f"staged tile {tile}")
    # the oracle, on the two shortest series (the others agree with them above)
    for s in (3, 4):
        ref = oracle_series(ys[s], m, tau, RR20, 100)
        assert np.array_equal(eps.cpu().numpy()[s], ref["eps"])
        assert np.array_equal(base["hist"][s], ref["hist"]), s
        assert np.array_equal(base["lmax"][s], ref["lmax"]), s
        assert np.array_equal(base["count"][s], ref["count"]), s
    ctx.close()


def test_staging_skipped_for_unaligned_buffer(rqa_lib):
    import torch
    rqa = rqa_lib
    ys = _series(7, SIZES[:3])
    flat = np.concatenate(ys)
    offsets = np.concatenate([[0], np.cumsum([len(v) for v in ys])])
    store = torch.zeros(len(flat) + 1, dtype=torch.float32, device="cuda")
    store[1:] = torch.from_numpy(flat).cuda()
    y = store[1:]  # 4 bytes past a 16-byte boundary
    assert y.data_ptr() % 16 == 4
    ctx = rqa.Context(device=0, select=rqa.RQA_SELECT_RADIX)
    batch = rqa.Batch(y, offsets, 3, 3)
    eps = rqa.eps_for_rr(ctx, batch, RR20, 100)["eps"]
    torch.cuda.synchronize()
    ref = rqa.Batch.from_numpy(ys, 3, 3, device=0)
    eps_ref = rqa.eps_for_rr(ctx, ref, RR20, 100)["eps"]
    assert torch.equal(eps, eps_ref)
    _same(_lines(rqa, ctx, batch, eps, 32, 1), _lines(rqa, ctx, ref, eps_ref, 32, 0), "unaligned")
    ctx.close()
