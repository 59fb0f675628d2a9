"""Pins of the oracle's direct method (Algorithm DBS steps 1-6) against
numpy's FFT and independent array formulations, and against the closed
form of centred Exp(1) noise.  CPU only."""
import numpy as np
import pytest

import hos_synth


def numpy_raw(x, M, remove_mean=True, overlap=0):
    """Average over parts of (1/M) F(k1) F(k2) conj F(k1 + k2), F = numpy FFT;
    parts of M samples every M - overlap samples."""
    step = M - overlap
    starts = list(range(0, x.size - M + 1, step))
    K = len(starts)
    k = np.arange(M)
    acc = np.zeros((M, M), complex)
    for a in starts:
        y = x[a:a + M].astype(np.float64)
        if remove_mean:
            y = y - y.mean()
        F = np.fft.fft(y)
        acc += F[:, None] * F[None, :] * np.conj(F[(k[:, None] + k[None, :]) % M]) / M
    return acc / K


def roll_smooth(R, M3):
    """Box average over offsets lo .. lo + M3 - 1 on both axes, lo = -(M3 // 2),
    as a sum of cyclically shifted copies."""
    lo = -(M3 // 2)
    acc = np.zeros_like(R)
    for n1 in range(lo, lo + M3):
        for n2 in range(lo, lo + M3):
            acc += np.roll(R, (-n1, -n2), axis=(0, 1))
    return acc / (M3 * M3)


@pytest.mark.parametrize("M,K,rm", [(16, 1, True), (64, 3, True), (50, 2, False)])
def test_unsmoothed_direct_estimate_is_the_fft_triple_product(oracle, M, K, rm):
    x = hos_synth.ar2(M * K + 7, 3 + M)  # the 7 trailing samples are not used
    got = oracle.bispectrum_direct(x, M, 1, remove_mean=rm)
    ref = numpy_raw(x, M, rm)
    assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()


@pytest.mark.parametrize("M,overlap,n", [(32, 16, 200), (40, 10, 131), (16, 15, 40), (64, 0, 64)])
def test_overlapping_parts(oracle, M, overlap, n):
    """Parts every M - overlap samples (the trailing samples past the last
    whole part unused)."""
    x = hos_synth.ar2(n, 5 + overlap)
    got = oracle.bispectrum_direct(x, M, 3, overlap=overlap)
    ref = roll_smooth(numpy_raw(x, M, overlap=overlap), 3)
    assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()


@pytest.mark.parametrize("M,M3", [(32, 4), (32, 5), (40, 2), (24, 24)])
def test_box_smoothing_equals_shifted_copies(oracle, M, M3):
    x = hos_synth.ma(M * 2, 11 + M3)
    got = oracle.bispectrum_direct(x, M, M3)
    ref = roll_smooth(numpy_raw(x, M), M3)
    assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()


def test_box_smoothing_equals_circular_convolution(oracle):
    """The same smoothing as a product of 2-D DFTs (circular correlation with
    a box of M3 x M3 ones starting at offset lo)."""
    M, M3 = 48, 6
    x = hos_synth.exp_noise(M * 3, 5)
    R = numpy_raw(x, M)
    box = np.zeros((M, M))
    idx = np.arange(-(M3 // 2), -(M3 // 2) + M3) % M
    box[np.ix_(idx, idx)] = 1.0 / (M3 * M3)
    # S(k) = sum_n box(n) R(k + n): correlation = ifft(fft(R) * conj(fft(box))) for real box
    ref = np.fft.ifft2(np.fft.fft2(R) * np.conj(np.fft.fft2(box)))
    got = oracle.bispectrum_direct(x, M, M3)
    assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()


@pytest.mark.parametrize("M,K,M3", [(32, 1, 1), (64, 4, 5), (48, 3, 8)])
def test_grid_mean_is_the_parts_third_moment(oracle, M, K, M3):
    """Summing (1/M) F(k1)F(k2)F*(k1+k2) over the whole grid gives
    M^2 (1/M) sum_u y(u)^3 (the k-sums collapse to u = v = w), and box
    smoothing on the torus keeps the grid sum: the grid mean of the estimate
    is the parts' average third central moment, exactly."""
    x = hos_synth.ar2(M * K, 77 + M3)
    B = oracle.bispectrum_direct(x, M, M3)
    m3 = np.mean([np.mean((x[p * M:(p + 1) * M] - x[p * M:(p + 1) * M].mean()) ** 3) for p in range(K)])
    assert abs(B.mean().real - m3) <= 1e-10 * abs(m3)
    assert abs(B.mean().imag) <= 1e-10 * abs(m3)


def test_exp_noise_direct_estimate_is_its_third_cumulant(oracle):
    """Centred Exp(1) noise has third cumulant 2: the estimate's grid mean
    (the parts' third moment, previous pin) lies within 5 standard errors of
    2, the error taken from the sample's own spread of y^3."""
    M, K, M3 = 64, 64, 5
    x = hos_synth.exp_noise(M * K, 2024)
    B = oracle.bispectrum_direct(x, M, M3)
    y3 = np.concatenate([(x[p * M:(p + 1) * M] - x[p * M:(p + 1) * M].mean()) ** 3 for p in range(K)])
    se = y3.std() / np.sqrt(y3.size)
    assert abs(B.mean().real - 2.0) <= 5 * se
