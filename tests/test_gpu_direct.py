"""GPU parity of the direct method (Algorithm DBS: part transforms, raw
triple products, window-sum box smoothing, average over parts) against the
FP64 oracle.  The path is FP32 (transform, products) with double-float
window sums; tolerance 1e-5 normwise, as the other FP32-class paths."""
import numpy as np
import pytest

import hos_synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no GPU", allow_module_level=True)

TOL = 1e-5


@pytest.fixture(scope="module")
def hos():
    from paper_1805_11775_gb300 import build
    build.build()
    import paper_1805_11775_gb300 as h
    return h


def normwise(got, ref):
    return np.abs(np.asarray(got, np.complex128) - ref).max() / np.abs(ref).max()


@pytest.mark.parametrize("n,M,M3,rm", [(64, 64, 1, True), (1000, 128, 8, True), (4096, 256, 5, True),
                                       (300, 100, 4, True), (777, 96, 3, False), (1024, 1024, 16, True),
                                       (96, 8, 8, True), (2048, 2048, 1, True), (40, 20, 20, True)])
def test_direct_matches_oracle(hos, oracle, n, M, M3, rm):
    """Power-of-two and other part lengths, odd and even boxes, a box the size
    of the grid, several parts with trailing samples, no mean removal."""
    x = hos_synth.ar2(n, 31 * n + M3)
    ref = oracle.bispectrum_direct(x, M, M3, remove_mean=rm)
    got = hos.bispectrum_direct(torch.from_numpy(x).cuda(), M, M3, remove_mean=rm).cpu().numpy()
    assert normwise(got, ref) <= TOL


@pytest.mark.parametrize("n,M,M3,overlap", [(1000, 128, 5, 64), (700, 96, 4, 30), (4096, 512, 16, 500)])
def test_direct_overlapping_parts(hos, oracle, n, M, M3, overlap):
    x = hos_synth.ma(n, n + overlap)
    ref = oracle.bispectrum_direct(x, M, M3, overlap=overlap)
    got = hos.bispectrum_direct(torch.from_numpy(x).cuda(), M, M3, overlap=overlap).cpu().numpy()
    assert normwise(got, ref) <= TOL


def test_direct_float32_input_many_parts(hos, oracle):
    x = hos_synth.ma(64 * 200, 9).astype(np.float32)
    ref = oracle.bispectrum_direct(x.astype(np.float64), 64, 6)
    got = hos.bispectrum_direct(torch.from_numpy(x).cuda(), 64, 6).cpu().numpy()
    assert normwise(got, ref) <= TOL


@pytest.mark.parametrize("M,M3", [(4096, 1), (8192, 279)])
def test_direct_large_grids(hos, M, M3):
    """Grids too large for the oracle's point-by-point smoothing: the
    unsmoothed estimate against numpy's FFT triple product (M = 4096), and for
    the paper's largest case (n = M = 8192, box 279) the exact identity that
    the grid mean is the third central moment, plus the k1 <-> k2 symmetry."""
    x = hos_synth.exp_noise(M, 8192 + M3)
    got = hos.bispectrum_direct(torch.from_numpy(x).cuda(), M, M3).cpu().numpy().astype(np.complex128)
    y = x - x.mean()
    if M3 == 1:
        F = np.fft.fft(y)
        k = np.arange(M)
        ref = F[:, None] * F[None, :] * np.conj(F[(k[:, None] + k[None, :]) % M]) / M
        assert normwise(got, ref) <= TOL
    m3 = np.mean(y ** 3)
    scale = np.abs(got).max()
    assert abs(got.mean().real - m3) <= 1e-5 * scale
    assert abs(got.mean().imag) <= 1e-5 * scale
    assert np.abs(got - got.T).max() <= 1e-5 * scale


def test_direct_argument_errors(hos):
    from paper_1805_11775_gb300._native import HosError
    # fewer samples than one part, box wider than the grid, empty box, one-point
    # grid, a non-power-of-two grid above 2048, a power of two above 8192,
    # overlap of a whole part, negative overlap
    for n, M, M3, ov in [(100, 200, 4, 0), (100, 64, 65, 0), (100, 64, 0, 0), (100, 1, 1, 0), (6000, 3000, 4, 0),
                         (32768, 16384, 4, 0), (100, 64, 4, 64), (100, 64, 4, -1)]:
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        with pytest.raises(HosError):
            hos.bispectrum_direct(x, M, M3, overlap=ov)
