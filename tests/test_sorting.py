"""Sorting rate S (Eq. 5) and the averaged DET for every RR* (Eq. avgDET):
the worked cases the definition fixes."""
import numpy as np
import pytest

from paper_2208_09136_gb300.sorting import det_avg_prefix, sorting_rate, sorting_rates


def test_sorting_rate_extremes():
    n = 10
    good = np.tile(np.arange(n, dtype=float), (10, 1))     # measure rises with SNR
    assert sorting_rate(good) == 100.0
    assert sorting_rate(good[:, ::-1]) == 0.0              # fully reversed
    # the paper's worst case for n = 10 and ten realisations is 500
    y = np.arange(1, 11)
    assert 10 * np.abs(y[::-1] - y).sum() == 500


def test_sorting_rate_one_swap():
    """Swapping two neighbours in one of ten realisations departs by 2 of 500."""
    m = np.tile(np.arange(10, dtype=float), (10, 1))
    m[3, [4, 5]] = m[3, [5, 4]]
    assert sorting_rate(m) == pytest.approx(100.0 * (500 - 2) / 500)


def test_sorting_rate_ties_keep_snr_order():
    m = np.zeros((2, 4))
    assert sorting_rate(m) == 100.0


def test_det_avg_prefix_and_rates():
    det = np.array([[[0.1], [0.3], [0.2]]])                 # one series, three targets
    p = det_avg_prefix(det)[0, :, 0]
    assert list(p) == [0.1, (0.1 + 0.3) / 2, (0.1 + 0.3 + 0.2) / 3]
    rng = np.random.default_rng(0)
    d = np.sort(rng.random((5, 6, 4)), axis=1)              # every target sorts perfectly
    assert np.all(sorting_rates(d, averaged=False) == 100.0)
    assert np.all(sorting_rates(d, averaged=True) == 100.0)
    with pytest.raises(ValueError):
        sorting_rate(np.zeros(3))
