"""Pins of the oracle's overlapping-part estimates (parts of m samples every
m - overlap samples, each demeaned, cumulants averaged) against the
segment-averaged estimate already pinned in test_oracle_pins, applied to the
series written out part after part, and against that estimate directly when
the parts do not overlap."""
import numpy as np
import pytest

import hos_synth


def _expanded(x, m, overlap):
    step = m - overlap
    K = (x.size - m) // step + 1
    return np.concatenate([x[k * step:k * step + m] for k in range(K)]), K


@pytest.mark.parametrize("n,m,o,L", [(300, 64, 16, 5), (257, 50, 49, 4), (400, 100, 1, 7), (120, 40, 39, 3)])
@pytest.mark.parametrize("rm", [True, False])
def test_overlap_equals_segments_of_the_expanded_series(oracle, n, m, o, L, rm):
    x = hos_synth.ar2(n, 91 + n)
    xe, K = _expanded(x, m, o)
    assert K >= 2
    got = oracle.bispectrum_overlap(x, L, 2 * L, remove_mean=rm, segment_len=m, overlap=o)
    ref = oracle.bispectrum(xe, L, 2 * L, remove_mean=rm, segment_len=m)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-14 * np.abs(ref).max())
    got4 = oracle.trispectrum_overlap(x, 3, 6, remove_mean=rm, segment_len=m, overlap=o)
    ref4 = oracle.trispectrum(xe, 3, 6, remove_mean=rm, segment_len=m)
    np.testing.assert_allclose(got4, ref4, rtol=1e-12, atol=1e-14 * np.abs(ref4).max())


def test_no_overlap_is_the_segment_average(oracle):
    """overlap = 0 and n a multiple of m: the parts are the plain partition."""
    x = hos_synth.exp_noise(360, 95)
    got = oracle.bispectrum_overlap(x, 6, 16, segment_len=90, overlap=0)
    np.testing.assert_allclose(got, oracle.bispectrum(x, 6, 16, segment_len=90), rtol=1e-12, atol=1e-16)


def test_overlap_cumulant_is_the_mean_of_part_cumulants(oracle):
    """The averaged c3 / c4 equals the mean of the pinned c3 / c4 of each
    demeaned part; a part count or step off by one fails it."""
    x = hos_synth.ar2(210, 96)
    m, o, L = 60, 20, 4
    step = m - o
    parts = [x[k * step:k * step + m] for k in range((x.size - m) // step + 1)]
    c3 = np.mean([oracle.c3(p - p.mean(), L) for p in parts], axis=0)
    np.testing.assert_allclose(oracle.cumulant_overlap(x, L, 3, segment_len=m, overlap=o), c3, rtol=1e-12,
                               atol=1e-15)
    c4 = np.mean([oracle.c4(p - p.mean(), 3) for p in parts], axis=0)
    np.testing.assert_allclose(oracle.cumulant_overlap(x, 3, 4, segment_len=m, overlap=o), c4, rtol=1e-12,
                               atol=1e-15)


def test_short_series_is_one_part(oracle):
    x = hos_synth.ar2(50, 97)
    np.testing.assert_allclose(oracle.bispectrum_overlap(x, 4, 8, segment_len=64, overlap=10),
                               oracle.bispectrum(x, 4, 8), rtol=1e-13, atol=1e-16)
