"""Pins of the learned-bracket oracle (sketch, network, loss, Adam) to
published test vectors, closed forms and finite differences."""
import numpy as np
import pytest

from oracle import mlp_oracle as MO
from oracle import rqa_oracle as O


def test_splitmix64_published_vectors():
    # SplitMix64 reference outputs for seeds 0 and 1234567
    assert MO.splitmix_stream(0, 3) == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    assert MO.splitmix_stream(1234567, 3) == [6457827717110365317, 3203168211198807973,
                                              9817491932198370423]


def test_counter_form_equals_sequential_stream():
    key = 0x0123456789ABCDEF
    seq = MO.splitmix_stream(key, 10)
    for t in range(10):
        assert seq[t] == MO.splitmix_mix(key + (t + 1) * MO.GAMMA)


@pytest.mark.parametrize("ne", [2, 3, 5, 1000, 99994])
def test_sketch_pairs_valid(ne):
    i, j = MO.sketch_pairs(ne, 3, 42)
    assert np.all(i != j) and i.min() >= 0 and j.min() >= 0 and i.max() < ne and j.max() < ne
    if ne == 5:  # 20 ordered pairs, each ~ 4096/20 = 205 times
        counts = np.bincount(i * 5 + j, minlength=25)
        used = counts[[a * 5 + b for a in range(5) for b in range(5) if a != b]]
        assert used.min() > 140 and used.max() < 270


def test_sketch_distances_match_distance_definition():
    rng = np.random.default_rng(3)
    y = rng.standard_normal(300).astype(np.float32)
    m, tau = 3, 2
    ne = 300 - (m - 1) * tau
    i, j = MO.sketch_pairs(ne, 7, 99)
    lo, hi = np.minimum(i, j), np.maximum(i, j)
    ref = np.array([O.diagonal_distances(y, m, tau, int(h - l))[l] for l, h in zip(lo, hi)],
                   dtype=np.float32)
    assert np.array_equal(MO.sketch_distances(y, m, tau, 7, 99), np.sort(ref))


def test_sketch_features_layout():
    rng = np.random.default_rng(4)
    y = rng.standard_normal(500).astype(np.float32)
    x, c, q = MO.sketch_features(y, 3, 3, 0, 1)
    srt = MO.sketch_distances(y, 3, 3, 0, 1)
    assert np.array_equal(q, srt[16::32])
    assert x[64] == 0.0 and np.all(np.diff(x[:128]) >= 0)
    assert c == np.log(float(srt[32 * 64 + 16]))
    assert x[128] == np.log10(500) and x[129] == 3 and x[130] == 3
    # scale invariance of the inputs: y * 4 shifts only the centre
    x4, c4, _ = MO.sketch_features(y * np.float32(4), 3, 3, 0, 1)
    assert np.allclose(x4, x, atol=1e-12) and abs(c4 - c - np.log(4)) < 1e-12


def test_forward_small_explicit():
    p = MO.init_params(1).astype(np.float64)
    X = np.random.default_rng(2).standard_normal((3, MO.N_FEAT))
    f = MO.forward(p, X)
    (W1, b1), (W2, b2), (W3, b3) = MO.unpack(p)
    for r in range(3):
        h1 = [max(0.0, sum(W1[o, i] * X[r, i] for i in range(MO.N_FEAT)) + b1[o]) for o in range(5)]
        assert np.allclose(f["H1"][r, :5], h1, rtol=1e-12, atol=1e-12)
    assert f["Y"].shape == (3, 40)


def test_pinball_closed_form():
    T = np.array([[1.0, 2.0]])
    Y = np.array([[1.0, 1.0, 0.0, 3.0]])  # (lo, hi) per target
    loss, g = MO.pinball(Y, T, 0.1, 0.9)
    # residuals r = T - Y: 0, 0, 2, -1 ; losses 0, 0, 0.1*2, (0.9-1)*(-1)
    assert loss == pytest.approx((0.2 + 0.1) / 4)
    assert np.allclose(g, np.array([[-0.1, -0.9, -0.1, 0.1]]) / 4)


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(5)
    p = MO.init_params(3).astype(np.float64) * 0.5
    X = rng.standard_normal((4, MO.N_FEAT))
    T = rng.standard_normal((4, MO.K_OUT))
    loss, g = MO.backward(p, X, T, 0.05, 0.95)
    idx = rng.choice(p.size, 60, replace=False)
    h = 1e-6
    for k in idx:
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        fd = (MO.backward(pp, X, T, 0.05, 0.95)[0] - MO.backward(pm, X, T, 0.05, 0.95)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 + 1e-4 * abs(g[k]), (k, fd, g[k])


def test_adam_first_step_is_sign_step():
    g = np.array([0.3, -2.0, 1e-3])
    p, m, v = MO.adam(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, lr=0.01, eps=0.0)
    assert np.allclose(p, -0.01 * np.sign(g))
