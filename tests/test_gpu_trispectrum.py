"""GPU parity of the trispectrum path (c2, m4 over symmetric lag pairs, the
c2*c2 correction, window, 3-axis transform) against the FP64 oracle.
Normwise tolerances as for the bispectrum: split-bf16 tensor cores 1e-4,
3xTF32 and split-FP16 tensor cores 1e-5, FP32 SIMT 1e-5."""
import math

import numpy as np
import pytest

import hos_synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no GPU", allow_module_level=True)

TOL = {"bf16": 1e-4, "fp32": 1e-5, "simt": 1e-5, "fp16": 1e-5}
PRECS = ["simt", "fp32", "bf16", "fp16"]


@pytest.fixture(scope="module")
def hos():
    from paper_1805_11775_gb300 import build
    build.build()
    import paper_1805_11775_gb300 as h
    return h


def normwise(got, ref):
    return np.abs(np.asarray(got, dtype=np.complex128) - ref).max() / np.abs(ref).max()


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("n,L", [(5, 1), (40, 3), (700, 8), (1500, 13), (2100, 32), (1200, 64)])
def test_cumulant4_elementwise(hos, oracle, n, L, prec):
    x = hos_synth.ma(n, 5 * n + L)
    ref = oracle.c4(oracle.demean(x), L)[:2 * L, :2 * L, :2 * L]
    got = hos.cumulant4(torch.from_numpy(x).cuda(), L, precision=prec).cpu().numpy()
    assert np.abs(got - ref).max() <= TOL[prec] * np.abs(ref).max()


@pytest.mark.parametrize("prec", PRECS)
def test_cumulant4_is_symmetric(hos, prec):
    x = torch.from_numpy(hos_synth.exp_noise(5000, 2)).cuda()
    c = hos.cumulant4(x, 8, precision=prec).cpu().numpy()
    # w1 <-> w2 reads the same lag-pair partial sums; only the FP64 c2*c2
    # terms change order
    assert np.abs(np.transpose(c, (1, 0, 2)) - c).max() <= 1e-12 * np.abs(c).max()
    # swaps with w3 pair the samples differently, so they agree to FP32 rounding
    for perm in [(2, 1, 0), (0, 2, 1)]:
        assert np.abs(np.transpose(c, perm) - c).max() <= (1e-6 if prec == "simt" else TOL[prec]) * np.abs(c).max()


@pytest.fixture(scope="module")
def tri_ref(oracle):
    w = hos_synth.workload("trispectrum_n65536_L32")
    return w, oracle.trispectrum(w["x"].astype(np.float64), w["L"], w["N"])


@pytest.mark.parametrize("prec", PRECS)
def test_trispectrum_full_size_workload(hos, tri_ref, prec):
    """n = 65536 float32 MA(3) series, L = 32, 64^3 grid: the whole output
    against the oracle."""
    w, ref = tri_ref
    got = hos.trispectrum(torch.from_numpy(w["x"]).cuda(), w["L"], precision=prec).cpu().numpy()
    assert normwise(got, ref) <= TOL[prec]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("n,L,N,seg", [(3000, 6, 14, 0), (5000, 10, 20, 1700), (2500, 16, 32, 0)])
def test_trispectrum_grids_and_parts(hos, oracle, n, L, N, seg, prec):
    x = hos_synth.ar2(n, 3 * n)
    ref = oracle.trispectrum(x, L, N, segment_len=seg)
    got = hos.trispectrum(torch.from_numpy(x).cuda(), L, nfft=N, segment_len=seg, precision=prec).cpu().numpy()
    assert normwise(got, ref) <= TOL[prec]


def test_trispectrum_hermitian_and_flat_level(hos):
    """Centred Exp(1) noise: c4(0,0,0) estimates the fourth cumulant 6, so the
    grid average of (2 pi)^3 T is near 6, and T(-k) = conj T(k)."""
    x = torch.from_numpy(hos_synth.exp_noise(1 << 20, 12)).cuda()
    T = hos.trispectrum(x, 8, precision="bf16").cpu().numpy().astype(np.complex128)
    N = T.shape[0]
    k = np.arange(N)
    neg = T[(-k[:, None, None]) % N, (-k[None, :, None]) % N, (-k[None, None, :]) % N]
    assert np.abs(neg - np.conj(T)).max() <= 1e-6 * np.abs(T).max()
    assert abs(T.real.mean() * (2 * math.pi) ** 3 - 6.0) < 0.6


@pytest.mark.parametrize("N", [8, 16, 128])
def test_trispectrum_transform_sizes(hos, oracle, N):
    """3-D transform on radix-8 register passes: contiguous lines along the
    last axis, strided lines along the other two."""
    L = 3
    x = hos_synth.ar2(900, 5 * N)
    ref = oracle.trispectrum(x, L, N)
    got = hos.trispectrum(torch.from_numpy(x).cuda(), L, nfft=N, precision="fp32").cpu().numpy()
    assert normwise(got, ref) <= TOL["fp32"]


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp16"])
def test_trispectrum_batched_matches_oracle_per_series(hos, oracle, prec):
    """Series of uneven length (one empty, one shorter than the lag range) in
    one call: each spectrum against the oracle, and against a single call."""
    lens = np.array([900, 0, 2500, 40, 1700], dtype=np.int64)
    vals, offs = hos_synth.student_t_returns(lens, 21)
    L, N = 8, 16
    got = hos.trispectrum_batched(torch.from_numpy(vals).cuda(), offs, L, nfft=N, precision=prec).cpu().numpy()
    assert got.shape == (lens.size, N, N, N)
    for s in range(lens.size):
        x = vals[offs[s]:offs[s + 1]]
        if x.size == 0:
            assert np.abs(got[s]).max() == 0.0
            continue
        ref = oracle.trispectrum(x, L, N)
        assert normwise(got[s], ref) <= TOL[prec]
        one = hos.trispectrum(torch.from_numpy(x).cuda(), L, nfft=N, precision=prec).cpu().numpy()
        assert normwise(got[s], one) <= 2 * TOL[prec]


def test_trispectrum_batched_rejects_simt_and_parts(hos):
    from paper_1805_11775_gb300._native import HosError
    v = torch.zeros(100, dtype=torch.float64, device="cuda")
    with pytest.raises(HosError):
        hos.trispectrum_batched(v, [0, 50, 100], 4, precision="simt")
