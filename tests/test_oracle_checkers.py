"""Pins of the oracle routines that serve as checkers at full size, of the
lag-cube window, and of the trispectrum's composition.

- ``c3_at`` and ``c3_rows`` compute the Problem Statement's third moment
  time average at chosen lags; they are the FP64 reference of every
  full-size c3 check and of the bench's accuracy figure.  Each is pinned to
  ``c3`` (itself pinned by the index-triple enumeration), to that
  enumeration directly, and to the zero the estimator gives where a lag
  reaches past the series.
- ``window3`` is pinned over the whole cube to the hand-worked Parzen
  values of ``tests/golden/parzen_values.txt`` and to the rectangular rule.
- The trispectrum (windowed c4, average over parts, (2 pi)^-3 transform) is
  pinned by exact identities: numpy's FFT of the wrapped windowed cumulant,
  T(0,0,0) = sum W c4 / (2 pi)^3, Parseval on the N^3 grid, Hermitian
  symmetry, symmetry under permutations of (k1, k2, k3), and the part
  average (Algorithm DBS step 6).
"""
import itertools
import math
import os

import numpy as np
import pytest

import hos_synth

TWO_PI = 2.0 * math.pi
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _triples(y, pairs):
    """c3 at the given lag pairs by enumerating ordered index triples
    (a, a + w1, a + w2) with all three inside the series."""
    n = y.size
    out = []
    for w1, w2 in pairs:
        s = 0.0
        for a in range(n):
            b, c = a + w1, a + w2
            if 0 <= b < n and 0 <= c < n:
                s += y[a] * y[b] * y[c]
        out.append(s / n)
    return np.array(out)


# --------------------------------------------------------------------- c3_at
def test_c3_at_matches_pinned_c3_on_random_lags(oracle):
    n, L = 57, 9
    y = oracle.demean(hos_synth.exp_noise(n, 31))
    full = oracle.c3(y, L)
    rng = np.random.default_rng(5)
    lags = rng.integers(-L, L + 1, size=(200, 2))
    got = oracle.c3_at(y, lags)
    np.testing.assert_array_equal(got, full[lags[:, 0] + L, lags[:, 1] + L])


def test_c3_at_matches_index_triples_and_vanishes_past_the_series(oracle):
    n = 23
    y = hos_synth.exp_noise(n, 8)
    # lags inside the series, at its edge (|w| = n - 1) and past it (|w| >= n)
    pairs = [(0, 0), (1, 0), (0, 1), (-3, 5), (5, -3), (7, 7), (-22, 0), (0, 22), (22, 22), (-22, -22),
             (23, 0), (0, -23), (30, 1), (-1, -40), (22, -1), (11, -11)]
    got = oracle.c3_at(y, pairs)
    np.testing.assert_allclose(got, _triples(y, pairs), rtol=1e-13, atol=1e-15)
    for p, (w1, w2) in enumerate(pairs):
        if max(abs(w1), abs(w2), abs(w1 - w2)) >= n:
            assert got[p] == 0.0  # no index triple fits inside the series
    # a lag pair whose span is exactly n - 1 has one term
    assert oracle.c3_at(y, [(-(n - 1), 0)])[0] == pytest.approx(y[n - 1] * y[0] * y[n - 1] / n, rel=1e-15)


def test_c3_at_is_symmetric_and_order_preserving(oracle):
    y = oracle.demean(hos_synth.ar2(400, 12))
    pairs = np.array([(w1, w2) for w1 in range(-6, 7) for w2 in range(-6, 7)])
    a = oracle.c3_at(y, pairs)
    b = oracle.c3_at(y, pairs[:, ::-1])
    np.testing.assert_allclose(a, b, rtol=1e-13, atol=1e-16)
    # the output order follows the input order (a reversed list gives a reversed result)
    np.testing.assert_array_equal(oracle.c3_at(y, pairs[::-1]), a[::-1])


# --------------------------------------------------------------------- c3_rows
@pytest.mark.parametrize("lo_hi", [(-7, -7), (-7, -4), (-2, 3), (4, 7), (7, 7), (-7, 7)])
def test_c3_rows_matches_pinned_c3(oracle, lo_hi):
    lo, hi = lo_hi
    n, L = 64, 7
    y = oracle.demean(hos_synth.exp_noise(n, 40 + lo))
    full = oracle.c3(y, L)
    got = oracle.c3_rows(y, L, lo, hi)
    assert got.shape == (hi - lo + 1, 2 * L + 1)
    np.testing.assert_array_equal(got, full[lo + L:hi + L + 1])


def test_c3_rows_past_the_lag_square_and_the_series(oracle):
    """Rows outside [-L, L] (the bench samples rows of a larger square) and rows
    whose lag reaches past a short series."""
    n, L = 12, 5
    y = hos_synth.exp_noise(n, 77)
    got = oracle.c3_rows(y, L, 9, 13)
    pairs = [(w1, w2) for w1 in range(9, 14) for w2 in range(-L, L + 1)]
    np.testing.assert_allclose(got.ravel(), _triples(y, pairs), rtol=1e-13, atol=1e-16)
    assert np.all(got[3:] == 0.0)  # w1 >= n: no triple fits


# --------------------------------------------------------------------- window3
def _golden():
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "parzen_values.txt")) if ln.strip() and ln[0] != "#"]
    table = {}
    for L, w, d in rows:
        table[(int(L), int(w))] = float(d)
        table[(int(L), -int(w))] = float(d)
    return table


@pytest.mark.parametrize("L", [4, 6])
def test_window3_parzen_over_the_whole_cube(oracle, L):
    d = _golden()
    lags = range(-L, L + 1)
    for w1, w2, w3 in itertools.product(lags, repeat=3):
        want = d[(L, w1)] * d[(L, w2)] * d[(L, w3)]
        assert oracle.window3(w1, w2, w3, L, oracle.WIN_PARZEN) == pytest.approx(want, rel=1e-14, abs=1e-17)


@pytest.mark.parametrize("L", [1, 3, 6])
def test_window3_rect_over_the_whole_cube(oracle, L):
    for w1, w2, w3 in itertools.product(range(-L - 1, L + 2), repeat=3):
        want = 1.0 if max(abs(w1), abs(w2), abs(w3)) <= L - 1 else 0.0
        assert oracle.window3(w1, w2, w3, L, oracle.WIN_RECT) == want


# --------------------------------------------------------------------- trispectrum composition
def _wrapped_windowed_c4(oracle, c4, L, N, window):
    """Windowed c4 (weights from the golden table or the rectangular rule,
    not from the oracle's window routine) wrapped onto the N^3 grid."""
    W = 2 * L + 1
    lags = np.arange(-L, L + 1)
    if window == oracle.WIN_RECT:
        d = (np.abs(lags) <= L - 1).astype(float)
    else:
        g = _golden()
        d = np.array([g[(L, int(w))] for w in lags])
    Wc = c4 * d[:, None, None] * d[None, :, None] * d[None, None, :]
    grid = np.zeros((N, N, N))
    for a, b, c in itertools.product(range(W), repeat=3):
        grid[(a - L) % N, (b - L) % N, (c - L) % N] += Wc[a, b, c]
    return Wc, grid


@pytest.mark.parametrize("L,N,window", [(4, 8, 0), (4, 11, 0), (6, 12, 0), (4, 8, 2)])
def test_trispectrum_is_the_fft_of_the_windowed_c4(oracle, L, N, window):
    x = hos_synth.ma(300, 17 + N)
    T = oracle.trispectrum(x, L, N, window=window)
    c4 = oracle.c4(oracle.demean(x), L)
    _, grid = _wrapped_windowed_c4(oracle, c4, L, N, window)
    np.testing.assert_allclose(T, np.fft.fftn(grid) / TWO_PI ** 3, rtol=1e-10, atol=1e-13)


def test_trispectrum_origin_parseval_hermitian_permutations(oracle):
    L, N = 4, 8
    x = hos_synth.exp_noise(250, 21)
    T = oracle.trispectrum(x, L, N)
    c4 = oracle.c4(oracle.demean(x), L)
    Wc, _ = _wrapped_windowed_c4(oracle, c4, L, N, oracle.WIN_PARZEN)
    # origin: the plain sum of the windowed cumulant
    assert T[0, 0, 0].real == pytest.approx(Wc.sum() / TWO_PI ** 3, rel=1e-12)
    assert abs(T[0, 0, 0].imag) < 1e-14
    # Parseval: lags |w| <= L - 1 carry all the weight, no two alias on N >= 2L
    assert (np.abs(T) ** 2).sum() == pytest.approx(N ** 3 * (Wc ** 2).sum() / TWO_PI ** 6, rel=1e-11)
    # a real lag-domain function has a Hermitian transform
    k = np.arange(N)
    neg = (-k) % N
    np.testing.assert_allclose(T[np.ix_(neg, neg, neg)], np.conj(T), atol=1e-13)
    # c4 and the separable window are symmetric under any permutation of the lags
    for p in itertools.permutations(range(3)):
        np.testing.assert_allclose(np.transpose(T, p), T, atol=1e-13)


def test_trispectrum_part_average(oracle):
    # Algorithm DBS steps 1, 2 and 6 with c4: each part's mean removed and its
    # own 1/m, the parts' estimates averaged (the transform is linear)
    L, N, m = 3, 6, 70
    x = hos_synth.ma(3 * m, 44) + 0.3
    T = oracle.trispectrum(x, L, N, segment_len=m)
    parts = [oracle.trispectrum(x[p * m:(p + 1) * m], L, N) for p in range(3)]
    np.testing.assert_allclose(T, sum(parts) / 3, rtol=1e-12, atol=1e-15)
