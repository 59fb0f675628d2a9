"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

None of these checks retypes the oracle's loops: each one is a closed form,
an independent enumeration, an identity with a library routine (numpy's FFT),
or an invariant, chosen so that a dropped term, a wrong sign, a wrong index
or a transposed operand in the oracle fails at least one of them.
"""
import itertools
import math
import os

import numpy as np
import pytest

import hos_synth

TWO_PI = 2.0 * math.pi
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------- c3
def _c3_by_index_triples(y, L):
    """Enumerate every ordered index triple (a, b, c) of the series and file
    y[a] y[b] y[c] under the lags (b - a, c - a): the time average of the
    Problem Statement's third moment, reached without the lag loop."""
    n = y.size
    W = 2 * L + 1
    out = np.zeros((W, W))
    for a in range(n):
        for b in range(max(0, a - L), min(n, a + L + 1)):
            for c in range(max(0, a - L), min(n, a + L + 1)):
                out[b - a + L, c - a + L] += y[a] * y[b] * y[c]
    return out / n


@pytest.mark.parametrize("n,L", [(1, 1), (2, 3), (7, 3), (23, 5), (40, 12), (17, 20)])
def test_c3_matches_index_triple_enumeration(oracle, n, L):
    y = np.random.default_rng(n * 100 + L).standard_normal(n)
    np.testing.assert_allclose(oracle.c3(y, L), _c3_by_index_triples(y, L), rtol=1e-12, atol=1e-14)


def test_c3_six_symmetries(oracle):
    L = 9
    y = hos_synth.exp_noise(300, 7)
    c = oracle.c3(y, L)

    def at(w1, w2):
        return c[w1 + L, w2 + L]

    for w1 in range(-L, L + 1):
        for w2 in range(-L, L + 1):
            v = at(w1, w2)
            assert at(w2, w1) == pytest.approx(v, abs=1e-14)
            for a, b in [(-w1, w2 - w1), (w2 - w1, -w1), (-w2, w1 - w2), (w1 - w2, -w2)]:
                if abs(a) <= L and abs(b) <= L:
                    assert at(a, b) == pytest.approx(v, abs=1e-14)


def test_c3_spike_closed_form(oracle):
    # x = a * delta(i0) without mean removal: only the zero-lag product survives
    n, L, a, i0 = 50, 6, 1.7, 20
    x = np.zeros(n)
    x[i0] = a
    c = oracle.c3(x, L)
    expect = np.zeros_like(c)
    expect[L, L] = a ** 3 / n
    np.testing.assert_allclose(c, expect, atol=1e-15)
    # and the bispectrum is flat at a^3 / (n (2 pi)^2) with the rectangular window
    B = oracle.bispectrum(x, L, N=2 * L, window=oracle.WIN_RECT, remove_mean=False)
    np.testing.assert_allclose(B, np.full(B.shape, a ** 3 / n / TWO_PI ** 2), atol=1e-14)


def test_c3_dft_equals_direct_triple_product(oracle):
    """Over all lags, the 2-D transform of the biased sample c3 is exactly the
    direct method's raw bispectrum (1/n) Y(k1) Y(k2) conj(Y(k1+k2)) (Algorithm
    DBS step 4, with the conjugate on the third factor that the text drops).
    Y is the transform of the series sampled on the same grid (numpy FFT)."""
    n = 21
    L = n  # every lag |w| <= n - 1 present, rectangular window keeps them all
    for N in (8, 17, 48):
        y = oracle.demean(hos_synth.exp_noise(n, 11 + N))
        B = oracle.bispectrum(y, L, N=N, window=oracle.WIN_RECT, remove_mean=False)
        # DTFT of y at 2 pi k / N: fold the series modulo N then FFT
        folded = np.zeros(N)
        np.add.at(folded, np.arange(n) % N, y)
        Y = np.fft.fft(folded)
        k = np.arange(N)
        expect = Y[:, None] * Y[None, :] * np.conj(Y[(k[:, None] + k[None, :]) % N]) / n / TWO_PI ** 2
        np.testing.assert_allclose(B, expect, rtol=1e-10, atol=1e-12)


# --------------------------------------------------------------------- m4, c2, c4
def test_m4_dft_equals_quadruple_product(oracle):
    n = 11
    L = n
    N = 10
    y = hos_synth.exp_noise(n, 5)
    m = oracle.m4(y, L)
    T = oracle.dft3(m, L, N, -1.0, 1.0)
    folded = np.zeros(N)
    np.add.at(folded, np.arange(n) % N, y)
    Y = np.fft.fft(folded)
    k = np.arange(N)
    k1, k2, k3 = np.meshgrid(k, k, k, indexing="ij")
    expect = Y[k1] * Y[k2] * Y[k3] * np.conj(Y[(k1 + k2 + k3) % N]) / n
    np.testing.assert_allclose(T, expect, rtol=1e-10, atol=1e-12)


def test_c2_dft_equals_periodogram(oracle):
    n, N = 13, 40
    y = hos_synth.exp_noise(n, 9)
    c = oracle.c2(y, n - 1)
    # 1-D transform over lags [-(n-1), n-1]
    lags = np.arange(-(n - 1), n)
    k = np.arange(N)
    S = (c[None, :] * np.exp(-2j * np.pi * np.outer(k, lags) / N)).sum(1)
    folded = np.zeros(N)
    np.add.at(folded, np.arange(n) % N, y)
    Y = np.fft.fft(folded)
    np.testing.assert_allclose(S, np.abs(Y) ** 2 / n, rtol=1e-11, atol=1e-12)


def test_c4_alternating_sequence_closed_form(oracle):
    """y(i) = (-1)^i.  Counting the valid i of each sum gives
    c2(t) = (-1)^t (n - |t|) / n and
    m4(w) = (-1)^(w1+w2+w3) (n - (max(0,w) - min(0,w))) / n, hence c4."""
    n, L = 30, 4
    y = np.array([(-1.0) ** i for i in range(n)])

    def c2(t):
        return (-1) ** (t % 2) * (n - abs(t)) / n

    got = oracle.c4(y, L)
    for w1, w2, w3 in itertools.product(range(-L, L + 1), repeat=3):
        span = max(0, w1, w2, w3) - min(0, w1, w2, w3)
        m4 = (-1) ** ((w1 + w2 + w3) % 2) * (n - span) / n
        c4 = m4 - c2(w1) * c2(w3 - w2) - c2(w2) * c2(w3 - w1) - c2(w3) * c2(w2 - w1)
        assert got[w1 + L, w2 + L, w3 + L] == pytest.approx(c4, abs=1e-13)


def test_c4_spike_closed_form(oracle):
    n, L, a = 40, 3, 1.3
    x = np.zeros(n)
    x[17] = a
    got = oracle.c4(x, L)
    # m4 lives only at the origin; c2 only at lag 0 (= a^2/n); the three c2*c2
    # products are nonzero only where each pair of lags is equal and one is 0
    for w1, w2, w3 in itertools.product(range(-L, L + 1), repeat=3):
        m4 = a ** 4 / n if (w1, w2, w3) == (0, 0, 0) else 0.0
        c2 = lambda t: a * a / n if t == 0 else 0.0
        expect = m4 - c2(w1) * c2(w3 - w2) - c2(w2) * c2(w3 - w1) - c2(w3) * c2(w2 - w1)
        assert got[w1 + L, w2 + L, w3 + L] == pytest.approx(expect, abs=1e-15)
    assert got[L, L, L] == pytest.approx(a ** 4 / n - 3 * a ** 4 / n ** 2, rel=1e-13)


def test_c4_permutation_symmetry(oracle):
    L = 3
    y = oracle.demean(hos_synth.exp_noise(80, 3))
    c = oracle.c4(y, L)
    for p in itertools.permutations(range(3)):
        np.testing.assert_allclose(np.transpose(c, p), c, atol=1e-14)


# --------------------------------------------------------------------- window
def test_parzen_golden_values(oracle):
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "parzen_values.txt")) if ln.strip() and ln[0] != "#"]
    assert len(rows) >= 10
    for L, w, d in rows:
        assert oracle.parzen(int(w), int(L)) == pytest.approx(float(d), abs=1e-15)
        assert oracle.parzen(-int(w), int(L)) == pytest.approx(float(d), abs=1e-15)


def test_parzen_is_nonnegative_definite(oracle):
    # The Parzen window is a cubic B-spline: its transform is sinc^4-like and
    # never negative, so the smoothed spectrum of a periodogram stays >= 0.
    for L in (5, 16, 32):
        lags = np.arange(-L, L + 1)
        d = np.array([oracle.parzen(w, L) for w in lags])
        om = np.linspace(0, np.pi, 257)
        spec = (d[None, :] * np.cos(np.outer(om, lags))).sum(1)
        assert spec.min() > -1e-12


def test_window_shapes(oracle):
    L = 8
    for w1, w2 in itertools.product(range(-L, L + 1), repeat=2):
        sep = oracle.window2(w1, w2, L, oracle.WIN_PARZEN)
        assert sep == pytest.approx(oracle.parzen(w1, L) * oracle.parzen(w2, L))
        hexa = oracle.window2(w1, w2, L, oracle.WIN_PARZEN_SYM)
        if abs(w1 - w2) >= L:
            assert hexa == 0.0
        assert oracle.window2(w1, w2, L, oracle.WIN_RECT) == (1.0 if max(abs(w1), abs(w2)) <= L - 1 else 0.0)
        assert oracle.window3(w1, w2, 0, L) == pytest.approx(sep)


# --------------------------------------------------------------------- DFT
@pytest.mark.parametrize("L,N", [(3, 6), (3, 8), (5, 16), (4, 9)])
def test_dft2_matches_numpy_fft2(oracle, L, N):
    f = np.random.default_rng(L * N).standard_normal((2 * L + 1, 2 * L + 1))
    grid = np.zeros((N, N))
    for a in range(2 * L + 1):
        for b in range(2 * L + 1):
            grid[(a - L) % N, (b - L) % N] += f[a, b]
    np.testing.assert_allclose(oracle.dft2(f, L, N, -1.0, 1.0), np.fft.fft2(grid), rtol=1e-11, atol=1e-11)
    np.testing.assert_allclose(oracle.dft2(f, L, N, +1.0, 1.0), np.fft.ifft2(grid) * N * N, rtol=1e-11, atol=1e-11)


def test_dft3_matches_numpy_fftn(oracle):
    L, N = 2, 6
    f = np.random.default_rng(1).standard_normal((5, 5, 5))
    grid = np.zeros((N, N, N))
    for a, b, c in itertools.product(range(5), repeat=3):
        grid[(a - L) % N, (b - L) % N, (c - L) % N] += f[a, b, c]
    np.testing.assert_allclose(oracle.dft3(f, L, N, -1.0, 0.5), 0.5 * np.fft.fftn(grid), rtol=1e-11, atol=1e-11)


def test_bispectrum_parseval_and_hermitian(oracle):
    L, N = 6, 12
    x = hos_synth.exp_noise(200, 4)
    B = oracle.bispectrum(x, L, N)
    k = np.arange(N)
    np.testing.assert_allclose(B[(-k[:, None]) % N, (-k[None, :]) % N], np.conj(B), atol=1e-14)
    np.testing.assert_allclose(B, B.T, atol=1e-14)  # c3 and the separable window are symmetric
    y = oracle.demean(x)
    c = oracle.c3(y, L)
    Wc = np.array([[oracle.window2(a - L, b - L, L) for b in range(2 * L + 1)] for a in range(2 * L + 1)]) * c
    # Parseval on the N-grid (|w| = L carries zero weight, so no lag aliases)
    assert (np.abs(B) ** 2).sum() == pytest.approx(N * N * (Wc ** 2).sum() / TWO_PI ** 4, rel=1e-11)
    assert B[0, 0].real == pytest.approx(Wc.sum() / TWO_PI ** 2, rel=1e-12)


# --------------------------------------------------------------------- segments / mean removal
def test_demean_segments(oracle):
    x = hos_synth.exp_noise(103, 2) + 5.0
    y = oracle.demean(x, 25)
    for s0 in range(0, 103, 25):
        assert abs(y[s0:s0 + 25].mean()) < 1e-13
    np.testing.assert_allclose(oracle.demean(x, 0, remove_mean=False), x)


def test_bispectrum_segment_average(oracle):
    # Algorithm DBS step 6 applied to c3: with K parts the estimate is the
    # mean of the parts' own estimates (the transform is linear)
    L, N, m = 4, 8, 60
    x = hos_synth.exp_noise(3 * m, 8)
    B = oracle.bispectrum(x, L, N, segment_len=m)
    parts = [oracle.bispectrum(x[p * m:(p + 1) * m], L, N) for p in range(3)]
    np.testing.assert_allclose(B, sum(parts) / 3, rtol=1e-12, atol=1e-15)


# --------------------------------------------------------------------- statistics
def _zscore(samples, expect):
    s = np.asarray(samples)
    return abs(s.mean() - expect) / (s.std(ddof=1) / math.sqrt(s.size))


def test_flat_bispectrum_of_exp_noise(oracle):
    """Centred i.i.d. Exp(1) noise has c3(0,0) = 2 and c3 = 0 elsewhere, so the
    bispectrum is flat at 2 / (2 pi)^2.  The grid average of (2 pi)^2 B is the
    windowed c3 at the origin, whose expectation is exactly 2."""
    vals, pts = [], []
    for r in range(24):
        B = oracle.bispectrum(hos_synth.exp_noise(2048, 5000 + r), 32, 64, remove_mean=False)
        vals.append((B.real * TWO_PI ** 2).mean())
        pts.append(B[5, 9].real * TWO_PI ** 2)
    assert _zscore(vals, 2.0) < 4.0
    assert _zscore(pts, 2.0) < 4.0


def test_linear_filter_closed_form(oracle):
    """MA filter h driven by centred Exp(1) noise (gamma3 = 2):
    c3_true(w1,w2) = gamma3 sum_k h_k h_{k+w1} h_{k+w2}; the biased estimator
    without mean removal has expectation (1 - span(w)/n) c3_true(w).  Its
    windowed transform must match the seed average, and with the window and
    the span factor removed it is gamma3 H(f1) H(f2) conj(H(f1+f2)) / (2 pi)^2."""
    h = np.array(hos_synth.MA3)
    L, N, n = 8, 16, 1024

    def c3_true(w1, w2):
        s = 0.0
        for k in range(-10, 10):
            def hh(j):
                return h[j] if 0 <= j < h.size else 0.0
            s += hh(k) * hh(k + w1) * hh(k + w2)
        return 2.0 * s

    lags = range(-L, L + 1)
    ct = np.array([[c3_true(a, b) for b in lags] for a in lags])
    span = np.array([[max(0, a, b) - min(0, a, b) for b in lags] for a in lags])
    Wd = np.array([[oracle.window2(a, b, L) for b in lags] for a in lags])
    expect = oracle.dft2(Wd * (1 - span / n) * ct, L, N, -1.0, 1.0 / TWO_PI ** 2)
    # closed form of the unwindowed, infinite-n spectrum (all true lags are < L)
    H = np.fft.fft(h, N)
    k = np.arange(N)
    Hcf = 2.0 * H[:, None] * H[None, :] * np.conj(H[(k[:, None] + k[None, :]) % N]) / TWO_PI ** 2
    np.testing.assert_allclose(oracle.dft2(ct, L, N, -1.0, 1.0 / TWO_PI ** 2), Hcf, rtol=1e-12, atol=1e-13)
    samples = np.array([oracle.bispectrum(hos_synth.ma(n, 7000 + r), L, N, remove_mean=False)
                        for r in range(40)])
    for (a, b) in [(0, 0), (1, 2), (3, 5), (7, 1)]:
        assert _zscore(samples[:, a, b].real, expect[a, b].real) < 4.5
        if abs(expect[a, b].imag) > 1e-12:
            assert _zscore(samples[:, a, b].imag, expect[a, b].imag) < 4.5


def test_gaussian_bispectrum_vanishes(oracle):
    """For Gaussian X every cumulant above the second is zero (Some
    Applications), so the grid-average of B (= windowed c3(0,0)) is
    zero-mean across seeds."""
    vals = [oracle.bispectrum(np.random.default_rng(900 + r).standard_normal(1024), 8, 16).real.mean()
            for r in range(24)]
    assert _zscore(vals, 0.0) < 4.0


def test_flat_trispectrum_of_exp_noise(oracle):
    """Centred Exp(1) has fourth cumulant 6: the grid average of (2 pi)^3 T
    is the estimated c4(0,0,0), whose expectation is 6 + O(1/n)."""
    vals = [(oracle.trispectrum(hos_synth.exp_noise(4096, 300 + r), 3, 6, remove_mean=False).real
             * TWO_PI ** 3).mean() for r in range(40)]
    assert _zscore(vals, 6.0) < 4.0


# --------------------------------------------------------------------- gradient
def _principal_mask(N):
    k1, k2 = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    return (k2 <= k1) & (k1 + k2 < N // 2)


def test_gradient_central_differences(oracle):
    """dl/dx for l = sum over the principal domain of |B - B_t|^2 against
    central differences of the oracle's own forward (FP64)."""
    n, L, N = 40, 5, 10
    x = hos_synth.ar2(n, 31)
    Bt = oracle.bispectrum(hos_synth.ar2(n, 32), L, N)
    mask = _principal_mask(N)

    def loss(v):
        B = oracle.bispectrum(v, L, N)
        return (np.abs(B - Bt) ** 2 * mask).sum()

    G = 2.0 * (oracle.bispectrum(x, L, N) - Bt) * mask
    g = oracle.bispectrum_grad(x, L, G, N)
    h = 1e-6 * np.sqrt((x ** 2).mean())
    fd = np.empty(n)
    for i in range(n):
        e = np.zeros(n)
        e[i] = h
        fd[i] = (loss(x + e) - loss(x - e)) / (2 * h)
    assert np.abs(g - fd).max() <= 1e-6 * np.abs(fd).max()


def test_gradient_dot_product_identity(oracle):
    """<J v, G> = <v, J^T G> for the real-linear map dx -> dB, with J v taken
    by a small central difference of the forward along v."""
    n, L, N = 36, 4, 9
    x = hos_synth.exp_noise(n, 41)
    rng = np.random.default_rng(42)
    v = rng.standard_normal(n)
    G = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    eps = 1e-5
    Jv = (oracle.bispectrum(x + eps * v, L, N) - oracle.bispectrum(x - eps * v, L, N)) / (2 * eps)
    lhs = (Jv.real * G.real + Jv.imag * G.imag).sum()
    rhs = v @ oracle.bispectrum_grad(x, L, G, N)
    assert lhs == pytest.approx(rhs, rel=1e-8)


def test_sampled_gradient_matches_the_full_chain_rule(oracle):
    """grad_lag + dy_at (used to check large problems at chosen samples) give
    the same values as the central-difference-pinned bispectrum_grad."""
    n, L, N = 60, 7, 16
    x = hos_synth.ar2(n, 51)
    rng = np.random.default_rng(5)
    G = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    full = oracle.bispectrum_grad(x, L, G, N, remove_mean=False)
    dc = oracle.grad_lag(G, L, N)
    js = np.arange(n)
    np.testing.assert_allclose(oracle.dy_at(x, L, dc, js), full, rtol=1e-10, atol=1e-14)


def test_gradient_central_differences_n1024(oracle):
    """The FP64 gradient against central differences at n = 1024 on sampled
    coordinates (loss: principal-domain squared distance to a target)."""
    n, L, N = 1024, 8, 16
    x = hos_synth.ar2(n, 61)
    Bt = oracle.bispectrum(hos_synth.ar2(n, 62), L, N)
    mask = _principal_mask(N)
    G = 2.0 * (oracle.bispectrum(x, L, N) - Bt) * mask
    g = oracle.bispectrum_grad(x, L, G, N)
    h = 1e-6 * np.sqrt((x ** 2).mean())
    for i in np.random.default_rng(6).choice(n, 48, replace=False):
        e = np.zeros(n)
        e[i] = h
        lp = (np.abs(oracle.bispectrum(x + e, L, N) - Bt) ** 2 * mask).sum()
        lm = (np.abs(oracle.bispectrum(x - e, L, N) - Bt) ** 2 * mask).sum()
        assert (lp - lm) / (2 * h) == pytest.approx(g[i], rel=1e-6, abs=1e-6 * np.abs(g).max())
