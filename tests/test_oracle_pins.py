"""Pins of the CPU oracle to facts fixed by the paper's definitions and by
mathematics -- not to the oracle itself.

Each pin is chosen so that a plausible slip in the oracle (an off-by-one in
the target count, a strict/inclusive mix-up, a dropped delay coordinate, a
transposed diagonal, a lost line at a diagonal's end) fails at least one test:

* a hand-worked 4-point example (tests/golden/hand_example_4pt.json) and its line
  measures, vertical lines and line-of-identity reading (hand_example_4pt_measures.json);
* brute force over the FULL N x N matrix with ordered pairs (a different
  formulation of Eq. 1-4: every count is exactly twice the upper-triangle one);
* closed forms: constant series, integer ramp, sawtooth;
* invariants: selection certificate, monotonicity, histogram mass, stencil vs
  histogram, negation / time reversal / power-of-two scaling;
* the i.i.d.-noise expectation DET ~ 1 - (1 - r)^2 (m = 1, large N).
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import rqa_oracle as O
from oracle import c_oracle as CO

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
RR = list(range(1, 21))


# ---------------------------------------------------------------- hand example
def test_hand_example_matches_worked_values():
    g = json.load(open(os.path.join(GOLDEN, "hand_example_4pt.json")))
    y = np.array(g["y"], dtype=np.float32)
    r = O.rqa_det_avg(y, g["m"], g["tau"], g["rr_num"], g["rr_den"], lmin=(2,))
    assert r["eps"].tolist() == g["eps"]
    assert r["T"].tolist() == g["T"]
    assert r["count_le"].tolist() == g["count_le"]
    assert r["count_lt"].tolist() == g["count_lt"]
    assert r["hist"].tolist() == g["hist"]
    assert r["stencil"].tolist() == g["stencil"]
    assert r["lmax"].tolist() == g["lmax"]
    assert r["det"][:, 0].tolist() == g["det_lmin2"]
    assert float(r["det_avg"][0]) == g["det_avg_lmin2"]


def _eq_or_nan(got, want, rtol=0.0):
    """want None means undefined (NaN); otherwise equal within rtol."""
    got = np.asarray(got, dtype=np.float64).ravel()
    flat = [np.nan if w is None else w for w in np.asarray(want, dtype=object).ravel()]
    want = np.asarray(flat, dtype=np.float64)
    assert np.array_equal(np.isnan(got), np.isnan(want))
    ok = ~np.isnan(want)
    assert np.allclose(got[ok], want[ok], rtol=rtol, atol=0.0), (got, want)


def test_hand_example_measures_vertical_lines_and_identity_line():
    """L, ENTR, vertical lines, LAM and TT, and the line-of-identity reading
    of Eq. 3 and Eq. 4, against values worked by hand for the 4-point series
    (tests/golden/hand_example_4pt_measures.json)."""
    g = json.load(open(os.path.join(GOLDEN, "hand_example_4pt_measures.json")))
    y = np.array(g["y"], dtype=np.float32)
    m, tau = g["m"], g["tau"]
    eps = np.array(g["eps"], dtype=np.float32)
    lines = O.line_hist(y, m, tau, eps)
    lm = O.line_measures(lines["hist"], g["lmin"])
    _eq_or_nan(lm["L"], g["L"])
    _eq_or_nan(lm["entr"], g["entr"], rtol=1e-15)
    v = O.vline_hist(y, m, tau, eps)
    assert v["vhist"].tolist() == g["vhist"]
    assert v["vmax"].tolist() == g["vmax"]
    lt = O.lam_tt(v["vhist"], lines["count"], g["vmin"], 4)
    _eq_or_nan(lt["lam"], g["lam"])
    _eq_or_nan(lt["tt"], g["tt"])

    h = g["loi"]
    sel = O.eps_for_rr(y, m, tau, h["rr_num"], h["rr_den"], loi=True)
    assert sel["T"].tolist() == h["T"]
    assert sel["eps"].tolist() == h["eps"]
    assert sel["count_le"].tolist() == h["count_le"]
    ll = O.line_hist(y, m, tau, sel["eps"])
    _eq_or_nan(O.det_from_hist(ll["hist"], ll["count"], [2], loi=True)[:, 0], h["det_lmin2"], rtol=1e-15)
    lml = O.line_measures(ll["hist"], [2], loi=True)
    _eq_or_nan(lml["L"][:, 0], h["L_lmin2"], rtol=1e-15)
    _eq_or_nan(lml["entr"][:, 0], h["entr_lmin2"], rtol=1e-14)
    vl = O.vline_hist(y, m, tau, sel["eps"], loi=True)
    assert vl["vhist"].tolist() == h["vhist"]
    ltl = O.lam_tt(vl["vhist"], ll["count"], [2], 4, loi=True)
    _eq_or_nan(ltl["lam"][:, 0], h["lam_vmin2"], rtol=1e-15)
    _eq_or_nan(ltl["tt"][:, 0], h["tt_vmin2"], rtol=1e-15)


# ------------------------------------------------------------ target counts
@pytest.mark.parametrize("p", [1, 2, 3, 4753, 49975003, 4999350021, 2**62 // 100])
def test_target_count_is_smallest_integer_reaching_rate(p):
    for num, den in [(1, 100), (7, 100), (20, 100), (99, 100), (1, 3), (2, 7)]:
        t = int(O.target_counts(p, [num], den)[0])
        # T/P >= num/den and (T-1)/P < num/den, in exact rationals
        assert Fraction(t, p) >= Fraction(num, den)
        assert Fraction(t - 1, p) < Fraction(num, den)


# ------------------------------------------------- full-matrix brute force
def _d32(y, i, j, m, tau):
    d = np.float32(0.0)
    for q in range(m):
        v = np.float32(abs(np.float32(y[i + q * tau]) - np.float32(y[j + q * tau])))
        d = v if q == 0 else (v if v > d else d)
    return d


def _brute_full(y, m, tau, rr_num, rr_den, lmin):
    """Full ordered-pair matrix without the line of identity, pure Python."""
    n = len(y)
    ne = n - (m - 1) * tau
    D = [[_d32(y, i, j, m, tau) if i != j else None for j in range(ne)] for i in range(ne)]
    vals = sorted({D[i][j] for i in range(ne) for j in range(ne) if i != j})
    npairs = ne * (ne - 1)  # ordered
    out = []
    for num in rr_num:
        need = -((-num * npairs) // rr_den)  # ceil over ordered pairs
        eps = None
        for v in vals:  # smallest distance value whose ordered count reaches the target
            if sum(1 for i in range(ne) for j in range(ne) if i != j and D[i][j] <= v) >= need:
                eps = v
                break
        rec = [[(i != j) and D[i][j] <= eps for j in range(ne)] for i in range(ne)]
        c2 = sum(rec[i][j] for i in range(ne) for j in range(ne))
        lt2 = sum(1 for i in range(ne) for j in range(ne) if i != j and D[i][j] < eps)
        # lines on every diagonal of the full matrix except the main one
        hist2 = [0] * ne
        for off in range(-(ne - 1), ne):
            if off == 0:
                continue
            run = 0
            cells = [(i, i + off) for i in range(ne) if 0 <= i + off < ne]
            for cell in cells + [None]:
                if cell is not None and rec[cell[0]][cell[1]]:
                    run += 1
                else:
                    if run:
                        hist2[run] += 1
                    run = 0
        det = [sum(l * hist2[l] for l in range(lm, ne)) / c2 for lm in lmin]
        out.append(dict(eps=eps, c2=c2, lt2=lt2, hist2=hist2, det=det))
    return out


@pytest.mark.parametrize("seed,n,m,tau", [(0, 12, 1, 1), (1, 17, 2, 1), (2, 20, 3, 2),
                                          (3, 9, 1, 1), (4, 33, 3, 3), (5, 25, 2, 4)])
def test_oracle_equals_full_matrix_brute_force(seed, n, m, tau):
    rng = np.random.default_rng(seed)
    # coarse values force many exact ties
    y = (rng.integers(0, 6, size=n) * 0.25).astype(np.float32) if seed % 2 else \
        rng.standard_normal(n).astype(np.float32)
    rr_num, rr_den, lmin = [1, 5, 13, 20, 37, 50], 100, (2, 3, 5)
    orc = O.rqa_det_avg(y, m, tau, rr_num, rr_den, lmin)
    ref = _brute_full(y, m, tau, rr_num, rr_den, lmin)
    for k, b in enumerate(ref):
        assert orc["eps"][k] == b["eps"]
        assert 2 * int(orc["count_le"][k]) == b["c2"]
        assert 2 * int(orc["count_lt"][k]) == b["lt2"]
        ne = n - (m - 1) * tau
        for l in range(1, ne):
            assert 2 * int(orc["hist"][k, l - 1]) == b["hist2"][l]
        for j in range(len(lmin)):
            assert orc["det"][k, j] == pytest.approx(b["det"][j], abs=0, rel=1e-15)


# ------------------------------------------------------------- closed forms
@pytest.mark.parametrize("n,m,tau", [(40, 1, 1), (31, 3, 2), (64, 2, 5)])
def test_constant_series_closed_form(n, m, tau):
    y = np.full(n, 0.7, dtype=np.float32)
    ne = n - (m - 1) * tau
    p = ne * (ne - 1) // 2
    r = O.rqa_det_avg(y, m, tau, RR, 100, lmin=(2, 3, 5))
    assert np.all(r["eps"] == 0.0)
    assert np.all(r["count_le"] == p) and np.all(r["count_lt"] == 0)
    assert np.all(r["hist"] == 1)           # one line of every length 1..Ne-1
    assert np.all(r["lmax"] == ne - 1)
    for j, lm in enumerate((2, 3, 5)):
        exact = 1.0 - (lm * (lm - 1) // 2) / p
        assert np.all(r["det"][:, j] == (p - lm * (lm - 1) // 2) / p)
        assert abs(r["det"][0, j] - exact) < 1e-15


@pytest.mark.parametrize("n,m,tau", [(50, 1, 1), (45, 3, 2)])
def test_ramp_closed_form(n, m, tau):
    y = np.arange(n, dtype=np.float32)       # d_ij = j - i exactly for any m, tau
    ne = n - (m - 1) * tau
    p = ne * (ne - 1) // 2
    r = O.rqa_det_avg(y, m, tau, RR, 100, lmin=(2,))
    for k, num in enumerate(RR):
        t = -((-num * p) // 100)
        e = 1
        while sum(ne - dl for dl in range(1, e + 1)) < t:
            e += 1
        assert r["eps"][k] == np.float32(e)
        assert int(r["count_le"][k]) == sum(ne - dl for dl in range(1, e + 1))
        assert int(r["count_lt"][k]) == sum(ne - dl for dl in range(1, e))
        expect = np.zeros(ne - 1, dtype=np.uint64)
        for dl in range(1, e + 1):
            expect[ne - dl - 1] += 1               # diagonal dl is one full line
        assert np.array_equal(r["hist"][k], expect)
        assert int(r["lmax"][k]) == ne - 1


def test_sawtooth_zero_threshold_lines():
    p_, n = 7, 70
    y = (np.arange(n) % p_).astype(np.float32)
    ne = n
    pairs = ne * (ne - 1) // 2
    zero_cells = sum(ne - q * p_ for q in range(1, (ne - 1) // p_ + 1))
    r = O.rqa_det_avg(y, 1, 1, RR, 100, lmin=(2,))
    for k, num in enumerate(RR):
        t = -((-num * pairs) // 100)
        if t <= zero_cells:
            assert r["eps"][k] == 0.0
            assert int(r["count_le"][k]) == zero_cells
            expect = np.zeros(ne - 1, dtype=np.uint64)
            for q in range(1, (ne - 1) // p_ + 1):
                expect[ne - q * p_ - 1] += 1
            assert np.array_equal(r["hist"][k], expect)
        else:
            assert r["eps"][k] >= 1.0


# --------------------------------------------------------------- invariants
def _series(kind, n, seed):
    rng = np.random.default_rng(seed)
    if kind == "noise":
        return rng.standard_normal(n).astype(np.float32)
    t = np.arange(n)
    return (np.sin(2 * np.pi * t / 20.3) + 0.1 * rng.standard_normal(n)).astype(np.float32)


@pytest.mark.parametrize("kind,n,m,tau", [("noise", 300, 1, 1), ("sine", 400, 3, 3), ("sine", 257, 2, 1)])
def test_invariants(kind, n, m, tau):
    y = _series(kind, n, 11)
    r = O.rqa_det_avg(y, m, tau, RR, 100, lmin=(2, 3, 5))
    t = r["T"].astype(np.int64)
    le = r["count_le"].astype(np.int64)
    lt = r["count_lt"].astype(np.int64)
    assert np.all(lt < t) and np.all(t <= le)                      # certificate
    assert np.all(np.diff(r["eps"]) >= 0) and np.all(np.diff(le) >= 0)  # monotone in k
    L = np.arange(1, r["hist"].shape[1] + 1, dtype=np.int64)
    mass = (r["hist"].astype(np.int64) * L[None, :]).sum(axis=1)
    assert np.array_equal(mass, le)                               # sum l P(l) = C
    assert np.array_equal(r["count"].astype(np.int64), le)
    s_from_hist = le - r["hist"][:, 0].astype(np.int64)
    assert np.array_equal(r["stencil"].astype(np.int64), s_from_hist)  # S = C - P(1)
    assert np.array_equal(r["det"][:, 0], r["stencil"].astype(np.float64) / le.astype(np.float64))
    # independent certificate from the C oracle
    cle, clt = CO.count(y, m, tau, r["eps"])
    assert np.array_equal(cle.astype(np.int64), le) and np.array_equal(clt.astype(np.int64), lt)


@pytest.mark.parametrize("m,tau", [(1, 1), (3, 2)])
def test_metamorphic_negation_reversal_scaling(m, tau):
    y = _series("noise", 180, 5)
    base = O.rqa_det_avg(y, m, tau, RR, 100, lmin=(2, 3))
    for y2, scale in [(-y, 1.0), (y[::-1].copy(), 1.0), (y * np.float32(8.0), 8.0),
                      (y * np.float32(0.125), 0.125)]:
        r = O.rqa_det_avg(y2, m, tau, RR, 100, lmin=(2, 3))
        assert np.array_equal(r["eps"], (base["eps"] * np.float32(scale)).astype(np.float32))
        for key in ("count_le", "count_lt", "hist", "stencil", "lmax", "det", "det_avg"):
            assert np.array_equal(r[key], base[key]), key


def test_delay_coordinates_all_used():
    # A series whose second delay coordinate alone separates two vectors: dropping
    # any coordinate of the maximum norm changes the distances.
    y = np.array([0, 0, 5, 0, 0, 0, 9, 0], dtype=np.float32)
    d = O.all_distances(y, 3, 2)
    # vectors: x0=(0,5,0) x1=(0,0,0) x2=(5,0,9) x3=(0,0,0)
    assert d.tolist() == [5.0, 9.0, 9.0, 9.0, 0.0, 5.0]


# ---------------------------------------------------- statistical closed form
def test_iid_noise_det_matches_independence_expectation():
    """m = 1, i.i.d. Gaussian noise: off the first diagonal, neighbouring cells of
    a diagonal use disjoint samples, so P(recurrent neighbour | recurrent) is
    1 - (1 - r)^2 in the interior and r at a diagonal's two ends."""
    n = 1500
    y = np.random.default_rng(123).standard_normal(n).astype(np.float32)
    rr = [5, 10, 20]
    r = O.eps_for_rr(y, 1, 1, rr, 100)
    for k, eps in enumerate(r["eps"]):
        rate = float(r["count_le"][k]) / (n * (n - 1) / 2)
        exp_s = 0.0
        exp_c = 0.0
        for dl in range(2, n):
            ln = n - dl
            exp_c += ln * rate
            if ln == 1:
                continue
            exp_s += rate * ((ln - 2) * (1 - (1 - rate) ** 2) + 2 * rate)
        obs = CO.lines(y, 1, 1, [eps], full_hist=False)
        d1 = O.diagonal_distances(y, 1, 1, 1) <= eps
        nb1 = np.zeros_like(d1)
        nb1[1:] |= d1[:-1]
        nb1[:-1] |= d1[1:]
        s1 = int((d1 & nb1).sum())
        c_off = int(obs["count"][0]) - int(d1.sum())
        s_off = int(obs["stencil"][0]) - s1
        det_off = s_off / c_off
        expect = exp_s / exp_c
        assert abs(det_off - expect) < 0.01, (rate, det_off, expect)
        # a one-sided neighbour rule would give ~ r, far outside the band
        assert abs(det_off - rate) > 0.03


# --------------------------------------------- C oracle against NumPy oracle
@pytest.mark.parametrize("n,m,tau", [(200, 1, 1), (333, 3, 3), (150, 2, 7)])
def test_c_oracle_agrees_with_numpy_oracle(n, m, tau):
    y = _series("sine", n, 3)
    r = O.rqa_det_avg(y, m, tau, RR, 100)
    assert np.array_equal(CO.distances(y, m, tau), O.all_distances(y, m, tau))
    L = CO.lines(y, m, tau, r["eps"], full_hist=True, n_short=8)
    for key in ("hist", "count", "stencil", "lmax"):
        assert np.array_equal(L[key], r[key]), key
    assert np.array_equal(L["short_hist"], r["hist"][:, :8])


def test_c_oracle_many_targets():
    """RR = 1..99 and 1..127 of 128 (the targets a call may hold): the C scans
    equal the NumPy oracle's for every target."""
    y = _series("logistic", 150, 5)
    for rr, den in ((list(range(1, 100)), 100), (list(range(1, 128)), 128)):
        r = O.rqa_det_avg(y, 2, 1, rr, den)
        L = CO.lines(y, 2, 1, r["eps"], full_hist=True)
        for key in ("hist", "count", "stencil", "lmax"):
            assert np.array_equal(L[key], r[key]), (den, key)


# ------------------------------------------------------------- L and ENTR
def test_line_measures_closed_forms():
    """L and ENTR on histograms with known answers: one length only (ENTR 0,
    L that length), equal counts of n lengths (ENTR ln n), lmin above every
    line (L NaN, ENTR 0), and a worked mixture."""
    K = 1
    h = np.zeros((K, 20), dtype=np.uint64)
    h[0, 6] = 5                                   # five lines of length 7
    r = O.line_measures(h, [1, 2, 7, 8])
    assert list(r["L"][0, :3]) == [7.0, 7.0, 7.0] and math.isnan(r["L"][0, 3])
    assert list(r["entr"][0]) == [0.0, 0.0, 0.0, 0.0]
    h = np.zeros((1, 10), dtype=np.uint64)
    h[0, [1, 3, 4, 8]] = 3                        # lengths 2, 4, 5, 9, three each
    r = O.line_measures(h, [1, 3, 6])
    assert r["entr"][0, 0] == pytest.approx(math.log(4), rel=1e-15)
    assert r["entr"][0, 1] == pytest.approx(math.log(3), rel=1e-15)
    assert r["entr"][0, 2] == 0.0
    assert r["L"][0, 0] == (2 + 4 + 5 + 9) / 4 and r["L"][0, 1] == (4 + 5 + 9) / 3
    h = np.zeros((1, 4), dtype=np.uint64)
    h[0, 0], h[0, 1], h[0, 3] = 2, 1, 1           # p = 1/2, 1/4, 1/4
    r = O.line_measures(h, [1])
    assert r["entr"][0, 0] == pytest.approx(1.5 * math.log(2), rel=1e-15)
    assert r["L"][0, 0] == (2 * 1 + 2 + 4) / 4


@pytest.mark.parametrize("n,m,tau", [(40, 1, 1), (31, 3, 2)])
def test_line_measures_constant_series(n, m, tau):
    """Constant series: one line of every length 1..Ne-1 (the upper triangle's
    diagonals are all fully recurrent), so for lines >= lmin:
    L = mean of lmin..Ne-1 and ENTR = ln(Ne - lmin)."""
    y = np.full(n, 0.75, dtype=np.float32)
    ne = n - (m - 1) * tau
    res = O.rqa_det_avg(y, m, tau, [1, 50], 100, (2,))
    lm = [1, 2, 5]
    r = O.line_measures(res["hist"], lm)
    for j, l0 in enumerate(lm):
        ls = list(range(l0, ne))
        assert r["L"][0, j] == pytest.approx(sum(ls) / len(ls), rel=1e-15)
        assert r["entr"][0, j] == pytest.approx(math.log(len(ls)), rel=1e-13)


@pytest.mark.parametrize("seed,n,m,tau", [(1, 17, 2, 1), (4, 33, 3, 3)])
def test_line_measures_full_matrix_brute_force(seed, n, m, tau):
    """L and ENTR from the full ordered-pair matrix (every line counted twice,
    by pure-Python run scanning) equal the oracle's upper-triangle values."""
    rng = np.random.default_rng(seed)
    y = (rng.integers(0, 6, size=n) * 0.25).astype(np.float32) if seed % 2 else \
        rng.standard_normal(n).astype(np.float32)
    rr_num, lmin = [5, 20, 50], (1, 2, 3)
    orc = O.rqa_det_avg(y, m, tau, rr_num, 100, lmin)
    r = O.line_measures(orc["hist"], lmin)
    for k, b in enumerate(_brute_full(y, m, tau, rr_num, 100, lmin)):
        h2 = b["hist2"]
        for j, lm in enumerate(lmin):
            nl = sum(h2[l] for l in range(lm, len(h2)))
            if nl == 0:
                assert math.isnan(r["L"][k, j]) and r["entr"][k, j] == 0.0
                continue
            L2 = sum(l * h2[l] for l in range(lm, len(h2))) / nl
            E2 = -sum((h2[l] / nl) * math.log(h2[l] / nl) for l in range(lm, len(h2)) if h2[l])
            assert r["L"][k, j] == pytest.approx(L2, rel=1e-15)
            assert r["entr"][k, j] == pytest.approx(E2, rel=1e-13, abs=1e-15)


# ------------------------------------------------- line of identity (Eq. 3-4 as written)
def _brute_full_loi(y, m, tau, rr_num, rr_den, lmin):
    """Eq. 3 and Eq. 4 over the whole Ne x Ne matrix, main diagonal included,
    by pure-Python counting and run scanning of every diagonal."""
    n = len(y)
    ne = n - (m - 1) * tau
    D = [[_d32(y, i, j, m, tau) if i != j else np.float32(0.0) for j in range(ne)] for i in range(ne)]
    vals = sorted({D[i][j] for i in range(ne) for j in range(ne) if i != j})
    out = []
    for num in rr_num:
        need = -((-num * ne * ne) // rr_den)
        eps = next(v for v in vals if sum(1 for i in range(ne) for j in range(ne) if D[i][j] <= v) >= need)
        rec = [[D[i][j] <= eps for j in range(ne)] for i in range(ne)]
        cfull = sum(rec[i][j] for i in range(ne) for j in range(ne))
        hist = [0] * (ne + 1)
        for off in range(-(ne - 1), ne):
            run = 0
            cells = [(i, i + off) for i in range(ne) if 0 <= i + off < ne]
            for cell in cells + [None]:
                if cell is not None and rec[cell[0]][cell[1]]:
                    run += 1
                else:
                    if run:
                        hist[run] += 1
                    run = 0
        det = [sum(l * hist[l] for l in range(lm, ne + 1)) / cfull for lm in lmin]
        nls = [sum(hist[l] for l in range(lm, ne + 1)) for lm in lmin]
        L = [sum(l * hist[l] for l in range(lm, ne + 1)) / nl for lm, nl in zip(lmin, nls)]
        E = [-sum((hist[l] / nl) * math.log(hist[l] / nl) for l in range(lm, ne + 1) if hist[l])
             for lm, nl in zip(lmin, nls)]
        out.append(dict(eps=eps, cfull=cfull, det=det, L=L, E=E))
    return out


@pytest.mark.parametrize("seed,n,m,tau", [(0, 14, 1, 1), (1, 19, 2, 1), (2, 24, 3, 2)])
def test_loi_reading_equals_full_matrix_brute_force(seed, n, m, tau):
    """With the line of identity counted (Eq. 3-4 as printed): eps, the full
    recurrence count 2C + Ne, DET, L and ENTR against the whole matrix."""
    rng = np.random.default_rng(seed)
    y = (rng.integers(0, 5, size=n) * 0.5).astype(np.float32) if seed % 2 else \
        rng.standard_normal(n).astype(np.float32)
    ne = n - (m - 1) * tau
    rr_num = [r for r in (10, 20, 35, 50, 80) if -((-r * ne * ne) // 100) > ne]
    lmin = (1, 2, 3)
    orc = O.rqa_det_avg(y, m, tau, rr_num, 100, lmin, loi=True)
    meas = O.line_measures(orc["hist"], lmin, loi=True)
    for k, b in enumerate(_brute_full_loi(y, m, tau, rr_num, 100, lmin)):
        assert orc["eps"][k] == b["eps"]
        assert 2 * int(orc["count_le"][k]) + ne == b["cfull"]
        for j in range(len(lmin)):
            assert orc["det"][k, j] == pytest.approx(b["det"][j], rel=1e-15)
            assert meas["L"][k, j] == pytest.approx(b["L"][j], rel=1e-15)
            assert meas["entr"][k, j] == pytest.approx(b["E"][j], rel=1e-13, abs=1e-15)


def test_loi_constant_series_and_rejection():
    """Constant series: every cell recurrent at eps = 0, so DET(1) = 1 exactly
    and DET(2) = 1 - 2 / Ne^2 (only the two corner cells are single points);
    a rate that the identity line alone reaches has no threshold."""
    ne = 50
    r = O.rqa_det_avg(np.full(ne, 3.0, np.float32), 1, 1, [5, 60], 100, (1, 2), loi=True)
    assert np.all(r["eps"] == 0.0)
    assert np.all(r["det"][:, 0] == 1.0)
    assert np.all(r["det"][:, 1] == (ne * ne - 2) / (ne * ne))
    with pytest.raises(ValueError):
        O.target_counts_loi(50, [2], 100)  # ceil(0.02 * 2500) = 50 <= Ne
    assert list(O.target_counts_loi(50, [3], 100)) == [13]  # ceil((75 - 50) / 2)


# ------------------------------------------------------------- vertical lines
def _brute_vertical(y, m, tau, eps, loi):
    n = len(y)
    ne = n - (m - 1) * tau
    out = []
    for e in eps:
        hist = [0] * (ne + 1)
        for j in range(ne):
            run = 0
            for i in list(range(ne)) + [None]:
                rec = i is not None and (i != j or loi) and _d32(y, i, j, m, tau) <= e if i != j \
                    else (i is not None and loi)
                if rec:
                    run += 1
                else:
                    if run:
                        hist[run] += 1
                    run = 0
        out.append(hist)
    return out


@pytest.mark.parametrize("seed,n,m,tau,loi", [(0, 15, 1, 1, False), (1, 21, 2, 1, False),
                                              (2, 26, 3, 2, True), (3, 18, 2, 3, True)])
def test_vertical_lines_brute_force(seed, n, m, tau, loi):
    """V_k(l) by scanning every column of the matrix cell by cell, LAM and TT
    from it, and the symmetry of the matrix: the vertical lines are the
    horizontal lines, so the vertical mass equals the recurrence count."""
    rng = np.random.default_rng(seed)
    y = (rng.integers(0, 5, size=n) * 0.5).astype(np.float32) if seed % 2 else \
        rng.standard_normal(n).astype(np.float32)
    ne = n - (m - 1) * tau
    rr = [10, 30, 60]
    sel = O.eps_for_rr(y, m, tau, rr, 100)
    v = O.vline_hist(y, m, tau, sel["eps"], loi=loi)
    for k, h in enumerate(_brute_vertical(y, m, tau, sel["eps"], loi)):
        assert [int(x) for x in v["vhist"][k]] == h[1:1 + v["vhist"].shape[1]]
        assert int(v["vmax"][k]) == max([l for l in range(len(h)) if h[l]], default=0)
    mass = (v["vhist"].astype(np.int64) * np.arange(1, v["vhist"].shape[1] + 1)).sum(axis=1)
    assert np.array_equal(mass, 2 * sel["count_le"].astype(np.int64) + (ne if loi else 0))
    lt = O.lam_tt(v["vhist"], sel["count_le"], (1, 2), ne, loi=loi)
    assert np.all(lt["lam"][:, 0] == 1.0)        # every recurrent cell is on a vertical line
    for k in range(len(rr)):
        row = [int(x) for x in v["vhist"][k]]
        n2 = sum(row[1:])
        m2 = sum(l * c for l, c in enumerate(row, start=1) if l >= 2)
        assert lt["tt"][k, 1] == m2 / n2 if n2 else math.isnan(lt["tt"][k, 1])


def test_vertical_lines_constant_series():
    """Constant series: column j is recurrent everywhere but at (j, j), so it
    holds one line of length j and one of length Ne-1-j: V(l) = 2 for every
    l = 1..Ne-1; with the identity line counted each column is one line of
    length Ne."""
    ne = 30
    y = np.full(ne, 1.5, np.float32)
    v = O.vline_hist(y, 1, 1, np.array([0.0], np.float32))
    assert np.all(v["vhist"][0] == 2) and int(v["vmax"][0]) == ne - 1
    v2 = O.vline_hist(y, 1, 1, np.array([0.0], np.float32), loi=True)
    assert int(v2["vhist"][0, ne - 1]) == ne and int(v2["vhist"][0, :ne - 1].sum()) == 0
    lt = O.lam_tt(v["vhist"], np.array([ne * (ne - 1) // 2]), (2,), ne)
    assert lt["lam"][0, 0] == (ne * (ne - 1) - 2) / (ne * (ne - 1))
    assert lt["tt"][0, 0] == (ne * (ne - 1) - 2) / (2 * (ne - 2))


# ------------------------------------------------- the paper's approximate eps search
def test_approx_grid_and_brute_force():
    """Grid counts by counting every pair against every grid value, the
    closest-RR choice by scanning all grid points, and the grid's own
    definition (i * range / n in FP32)."""
    rng = np.random.default_rng(3)
    y = rng.standard_normal(40).astype(np.float32)
    n_thr = 25
    r = O.eps_approx(y, 2, 1, [5, 20, 50, 90], 100, n_thr)
    rg = np.float32(y.max()) - np.float32(y.min())
    assert np.array_equal(r["thr"], np.float32(np.arange(1, n_thr + 1)) * np.float32(rg / np.float32(n_thr)))
    ne = 39
    d = [_d32(y, i, j, 2, 1) for i in range(ne) for j in range(i + 1, ne)]
    P = len(d)
    grid = [sum(1 for v in d if v <= t) for t in r["thr"]]
    assert [int(c) for c in r["grid_count"]] == grid
    assert grid[-1] == P                                   # the top threshold is the range
    for k, rr in enumerate([5, 20, 50, 90]):
        best = min(range(n_thr), key=lambda j: (abs(grid[j] / P - rr / 100), j))
        assert r["eps"][k] == r["thr"][best] and int(r["count"][k]) == grid[best]
        assert r["rr"][k] == grid[best] / P


def test_approx_error_bound():
    """The achieved RR is within half a grid step's RR jump of the target."""
    rng = np.random.default_rng(4)
    y = np.sin(np.arange(300) * 0.31).astype(np.float32) + 0.1 * rng.standard_normal(300).astype(np.float32)
    r = O.eps_approx(y, 3, 2, list(range(1, 100)), 100)
    P = pair = (300 - 4) * (300 - 5) // 2
    c = np.concatenate(([0], r["grid_count"].astype(np.int64)))
    for k, rr in enumerate(range(1, 100)):
        t = rr / 100
        j = int(np.searchsorted(c / P, t))
        lo, hi = c[max(j - 1, 0)] / P, c[min(j, len(c) - 1)] / P
        assert abs(r["rr"][k] - t) <= max(t - lo, hi - t) + 1e-15


def test_det_undefined_without_recurrences():
    """Thresholds below the smallest distance leave no recurrent cell: Eq. 4 is
    then 0/0, which the oracle returns as NaN (the IEEE quotient); the average
    over the targets is NaN too.  The smallest distance is taken by brute force
    over all pairs, independent of the oracle's own distance routine."""
    y = np.array([0.0, 1.0, 3.0, 7.0, 15.0, 31.0], dtype=np.float32)  # distinct gaps
    dmin = min(abs(float(y[i]) - float(y[j])) for i in range(len(y)) for j in range(i + 1, len(y)))
    assert dmin == 1.0
    eps = np.array([0.5, 2.0], dtype=np.float32)  # below dmin, then above it
    lines = O.line_hist(y, 1, 1, eps)
    assert int(lines["count"][0]) == 0 and int(lines["hist"][0].sum()) == 0
    det = O.det_from_hist(lines["hist"], lines["count"], (2, 3))
    assert np.isnan(det[0]).all()
    # the second threshold: cells with d <= 2 are (0,1) and (1,2): one line of
    # length 2 on the first diagonal, so DET_2 = 2/2 and DET_3 = 0/2
    assert int(lines["count"][1]) == 2
    assert det[1].tolist() == [1.0, 0.0]
    assert np.isnan(O.det_avg(det)).all()


def test_c_oracle_compiles_without_openmp(tmp_path):
    """The plain-C oracle is standard C99: it builds with and without OpenMP."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle",
                       "rqa_oracle.c")
    for flags in ([], ["-fopenmp"]):
        out = tmp_path / ("o%d.o" % len(flags))
        p = subprocess.run([cc, "-std=c99", "-O1", "-Wall", "-Werror", "-c", src, "-o", str(out)] + flags,
                           capture_output=True, text=True)
        assert p.returncode == 0, p.stderr
