"""The sorting-rate evaluation of Sect. 3 on synthetic groups: DET_RR for
RR = 1..99 % from one GPU call per group, averaged over RR = 1..RR* for every
RR*, and S (Eq. 5) for the averaged and the single-RR approach.  The GPU DET
values equal the oracle's bit for bit, so S must too."""
import numpy as np
import pytest

from paper_2208_09136_gb300.sorting import sorting_rates
from tests._helpers import oracle_series

pytestmark = pytest.mark.gpu

SNR_DB = np.linspace(-20.0, 25.0, 10)
RR99 = list(range(1, 100))


def _group(seed, n=400):
    """Ten logistic-map series (r = 4) at ten SNR levels, one realisation."""
    rng = np.random.default_rng(seed)
    x = np.empty(n + 500)
    x[0] = rng.uniform(0.1, 0.9)
    for j in range(1, len(x)):
        x[j] = 4.0 * x[j - 1] * (1.0 - x[j - 1])
    clean = x[500:]
    var = clean.var()
    return [(clean + rng.standard_normal(n) * np.sqrt(var / 10 ** (db / 10))).astype(np.float32)
            for db in SNR_DB]


def test_sorting_rate_from_gpu_det_equals_oracle(rqa_lib):
    rqa = rqa_lib
    ctx = rqa.Context(select=rqa.RQA_SELECT_RADIX)
    det_gpu, det_orc = [], []
    for i in range(3):
        ys = _group(100 + i)
        batch = rqa.Batch.from_numpy(ys, 2, 1)
        det_gpu.append(rqa.det_avg(ctx, batch, RR99, 100, lmin=(2,))["det"].cpu().numpy()[:, :, 0])
        det_orc.append(np.stack([oracle_series(y, 2, 1, RR99, 100, lmin=(2,), full_hist=False)["det"][:, 0]
                                 for y in ys]))
    assert rqa.rqa_status(ctx) == 0
    g, o = np.stack(det_gpu), np.stack(det_orc)            # (realisations, SNR levels, RR)
    assert np.array_equal(g, o)
    s_avg, s_one = sorting_rates(g, averaged=True), sorting_rates(g, averaged=False)
    assert np.array_equal(s_avg, sorting_rates(o, averaged=True))
    assert s_avg.shape == (99,) and np.all((s_avg >= 0) & (s_avg <= 100))
    # deterministic dynamics under rising SNR: DET orders the series far better than chance
    assert s_avg[-1] > 50.0 and s_one[0] > 50.0
    ctx.close()
