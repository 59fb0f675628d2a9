"""Pins of the oracle's trispectrum gradient (the adjoint of the indirect
trispectrum, one part) against facts that do not come from its own loops:
central differences of the pinned forward, the dot-product identity of an
adjoint, numpy's inverse FFT for the transform step, and agreement of the
sampled route used for long series with the full chain rule."""
import math

import numpy as np
import pytest

import hos_synth

WIN_PARZEN, WIN_RECT = 0, 2


@pytest.mark.parametrize("window,remove_mean", [(WIN_PARZEN, True), (WIN_PARZEN, False), (WIN_RECT, True)])
def test_trispectrum_gradient_central_differences(oracle, window, remove_mean):
    """dl/dx for l = sum |T - T_t|^2 over the grid against central differences
    of the oracle's forward trispectrum (FP64)."""
    n, L, N = 24, 3, 8
    x = hos_synth.ar2(n, 71)
    Tt = oracle.trispectrum(hos_synth.ar2(n, 72), L, N, window=window, remove_mean=remove_mean)

    def loss(v):
        T = oracle.trispectrum(v, L, N, window=window, remove_mean=remove_mean)
        return (np.abs(T - Tt) ** 2).sum()

    G = 2.0 * (oracle.trispectrum(x, L, N, window=window, remove_mean=remove_mean) - Tt)
    g = oracle.trispectrum_grad(x, L, G, N, window=window, remove_mean=remove_mean)
    h = 1e-5 * np.sqrt((x ** 2).mean())
    fd = np.empty(n)
    for i in range(n):
        e = np.zeros(n)
        e[i] = h
        fd[i] = (loss(x + e) - loss(x - e)) / (2 * h)
    assert np.abs(g - fd).max() <= 1e-6 * np.abs(fd).max()


def test_trispectrum_gradient_dot_product_identity(oracle):
    """<J v, G> = <v, J^T G> for the real-linear map dx -> dT, J v by a central
    difference of the forward along v, G an arbitrary complex grid."""
    n, L, N = 30, 4, 8
    x = hos_synth.exp_noise(n, 73)
    rng = np.random.default_rng(74)
    v = rng.standard_normal(n)
    G = rng.standard_normal((N, N, N)) + 1j * rng.standard_normal((N, N, N))
    eps = 1e-5
    Jv = (oracle.trispectrum(x + eps * v, L, N) - oracle.trispectrum(x - eps * v, L, N)) / (2 * eps)
    lhs = (Jv.real * G.real + Jv.imag * G.imag).sum()
    rhs = v @ oracle.trispectrum_grad(x, L, G, N)
    assert lhs == pytest.approx(rhs, rel=1e-7)


@pytest.mark.parametrize("window", [WIN_PARZEN, WIN_RECT])
def test_grad_lag4_matches_numpy_inverse_fft(oracle, window):
    """Step 1: W(w) (2 pi)^-3 Re sum_k G(k) e^{+i 2 pi k.w/N} is N^3 times
    numpy's ifftn read at w mod N."""
    L, N = 3, 8
    rng = np.random.default_rng(75)
    G = rng.standard_normal((N, N, N)) + 1j * rng.standard_normal((N, N, N))
    dc = oracle.grad_lag4(G, L, N, window)
    full = np.fft.ifftn(G) * N ** 3
    W = 2 * L + 1
    ref = np.empty((W, W, W))
    for a in range(W):
        for b in range(W):
            for c in range(W):
                w1, w2, w3 = a - L, b - L, c - L
                ref[a, b, c] = (oracle.window3(w1, w2, w3, L, window) * full[w1 % N, w2 % N, w3 % N].real
                                / (2 * math.pi) ** 3)
    np.testing.assert_allclose(dc, ref, rtol=1e-11, atol=1e-13 * np.abs(ref).max())


def test_sampled_trispectrum_gradient_matches_the_full_chain_rule(oracle):
    """grad_lag4 + grad_c2 + dy4_at (the route used to check long series at
    chosen samples) give the full chain rule's values."""
    n, L, N = 40, 4, 8
    x = hos_synth.ar2(n, 76)
    rng = np.random.default_rng(77)
    G = rng.standard_normal((N, N, N)) + 1j * rng.standard_normal((N, N, N))
    full = oracle.trispectrum_grad(x, L, G, N, remove_mean=False)
    dc4 = oracle.grad_lag4(G, L, N)
    dc2 = oracle.grad_c2(dc4, oracle.c2(x, 2 * L), L)
    np.testing.assert_allclose(oracle.dy4_at(x, L, dc4, dc2, np.arange(n)), full, rtol=1e-10,
                               atol=1e-12 * np.abs(full).max())


def test_grad_c2_of_a_single_term(oracle):
    """dl/dc2 when dl/dc4 is one at a single lag triple: the three c2 c2
    products of c4 at (w1, w2, w3) give -c2(b) to c2(a) and -c2(a) to c2(b)."""
    L = 3
    W, T = 2 * L + 1, 2 * L
    c2v = np.random.default_rng(78).standard_normal(2 * T + 1)
    w = (2, -1, 1)
    dc4 = np.zeros((W, W, W))
    dc4[w[0] + L, w[1] + L, w[2] + L] = 1.0
    got = oracle.grad_c2(dc4, c2v, L)
    ref = np.zeros(2 * T + 1)
    for a, b in ((w[0], w[2] - w[1]), (w[1], w[2] - w[0]), (w[2], w[1] - w[0])):
        ref[a + T] -= c2v[b + T]
        ref[b + T] -= c2v[a + T]
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-15)
