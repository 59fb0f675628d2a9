"""GPU parity of the time-sliced long-series path: ranks emulated one after
another on one GPU through the same C-ABI calls a rank makes
(hos_series_sum, hos_cumulant3_slice, hos_bispectrum_from_cumulant), the
FP64 sums taken on the host.  The result must match the FP64 oracle at the
precision's tolerance (normwise, as the other parity tests) and one call
over the whole series.
"""
import math

import numpy as np
import pytest

import hos_synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no GPU", allow_module_level=True)

TOL = {"bf16": 1e-4, "fp32": 1e-5, "simt": 1e-5, "fp16": 1e-5}


@pytest.fixture(scope="module")
def hos():
    from paper_1805_11775_gb300 import build
    build.build()
    import paper_1805_11775_gb300 as h
    return h


def normwise(got, ref):
    d = np.abs(np.asarray(got, dtype=np.complex128) - ref).max()
    s = np.abs(ref).max()
    return d / s if s > 0 else d


def emulate_ranks(hos, x, L, world, prec, remove_mean=True):
    """c3 of the whole series from `world` slices, computed one after another."""
    from paper_1805_11775_gb300.shard import slice_with_halo
    xd = torch.from_numpy(x).cuda()
    pieces = [slice_with_halo(xd, r, world, L) for r in range(world)]
    total = sum(float(hos.series_sum(p[h0:p.numel() - h1]).item()) for p, h0, h1 in pieces)
    tot = torch.tensor([total], dtype=torch.float64, device="cuda")
    c3 = np.zeros((2 * L, 2 * L))
    for p, h0, h1 in pieces:
        c3 += hos.cumulant3_slice(p, L, h0, h1, tot, x.size, precision=prec, remove_mean=remove_mean).cpu().numpy()
    return c3


def test_series_sum_is_the_fp64_sum(hos):
    for n, dt in [(1, np.float64), (8191, np.float64), (8193, np.float32), (3 << 20, np.float64)]:
        x = hos_synth.ar2(n, n).astype(dt)
        got = float(hos.series_sum(torch.from_numpy(x).cuda()).item())
        ref = math.fsum(x.astype(np.float64))
        assert abs(got - ref) <= 1e-13 * max(1.0, np.abs(x).sum())


@pytest.mark.parametrize("prec", ["simt", "fp32", "bf16", "fp16"])
@pytest.mark.parametrize("n,L,world", [(5000, 32, 2), (7001, 40, 3), (3000, 128, 5), (100, 32, 5), (2049, 8, 8)])
def test_slices_sum_to_the_oracle_c3(hos, oracle, prec, n, L, world):
    x = hos_synth.ar2(n, 13 * n + world)
    ref = oracle.c3(oracle.demean(x), L)[:2 * L, :2 * L]
    got = emulate_ranks(hos, x, L, world, prec)
    assert np.abs(got - ref).max() <= TOL[prec] * np.abs(ref).max()


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp16"])
def test_slices_match_one_call_and_the_oracle_bispectrum(hos, oracle, prec):
    """Slices of a 2^16-sample series at L = 64 (several chunks per slice,
    ragged slice ends): c3 against one hos_cumulant3 call, B from the summed
    c3 against the oracle, float32 input, no mean removal."""
    n, L, world = 1 << 16, 64, 3
    x = hos_synth.ma(n, 4242).astype(np.float32)
    one = hos.cumulant3(torch.from_numpy(x).cuda(), L, precision=prec, remove_mean=False).cpu().numpy()
    got = emulate_ranks(hos, x, L, world, prec, remove_mean=False)
    assert np.abs(got - one).max() <= 2 * TOL[prec] * np.abs(one).max()
    B = hos.bispectrum_from_cumulant(torch.from_numpy(got).cuda(), L).cpu().numpy()
    ref = oracle.bispectrum(x.astype(np.float64), L, remove_mean=False)
    assert normwise(B, ref) <= TOL[prec]


@pytest.mark.parametrize("window,nfft", [("parzen", 0), ("parzen_sym", 48), ("rect", 40)])
def test_from_cumulant_reproduces_bispectrum_exactly(hos, window, nfft, monkeypatch):
    """The same c3 through either route gives the same grid: bit for bit
    when the bispectrum contracts the same lag pairs (the swap plan, which the
    raw cumulant uses), and within the FP32-class target under the default
    six-fold plan (each value then comes from the one image of its lag pair
    that the plan computes: the same sum in another order)."""
    x = torch.from_numpy(hos_synth.ar2(3000, 99)).cuda()
    L = 20
    c3 = hos.cumulant3(x, L, precision="fp32")
    a = hos.bispectrum_from_cumulant(c3, L, nfft=nfft, window=window).cpu().numpy()
    b = hos.bispectrum(x, L, nfft=nfft, precision="fp32", window=window).cpu().numpy()
    assert normwise(b, a.astype(np.complex128)) <= TOL["fp32"]
    monkeypatch.setenv("HOS_TILE_SCHEME", "swap")
    b = hos.bispectrum(x, L, nfft=nfft, precision="fp32", window=window).cpu().numpy()
    np.testing.assert_array_equal(a, b)


def test_sharded_single_rank_is_the_bispectrum(hos, oracle):
    x = hos_synth.ar2(6000, 5)
    L = 32
    got = hos.bispectrum_sharded(torch.from_numpy(x).cuda(), L, 0, 0, x.size, precision="fp32").cpu().numpy()
    assert normwise(got, oracle.bispectrum(x, L)) <= TOL["fp32"]


def test_slice_argument_errors(hos):
    from paper_1805_11775_gb300._native import HosError
    x = torch.zeros(100, dtype=torch.float64, device="cuda")
    tot = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(HosError):
        hos.cumulant3_slice(x, 8, 9, 0, tot, 1000)  # halo longer than L
    with pytest.raises(HosError):
        hos.cumulant3_slice(x, 8, 4, 4, tot, 50)  # n_total shorter than the window


# ------------------------------------------------------------------ fourth order


def emulate_ranks4(hos, x, L, world, prec, remove_mean=True):
    """(m4, c2) of the whole series from `world` slices (halo L before, 2L
    after), computed one after another; host FP64 sums."""
    from paper_1805_11775_gb300.shard import slice_with_halo
    xd = torch.from_numpy(x).cuda()
    pieces = [slice_with_halo(xd, r, world, L, halo_after=2 * L) for r in range(world)]
    total = sum(float(hos.series_sum(p[h0:p.numel() - h1]).item()) for p, h0, h1 in pieces)
    tot = torch.tensor([total], dtype=torch.float64, device="cuda")
    m4 = np.zeros((2 * L,) * 3)
    c2 = np.zeros(4 * L - 1)
    for p, h0, h1 in pieces:
        a, b = hos.moments4_slice(p, L, h0, h1, tot, x.size, precision=prec, remove_mean=remove_mean)
        m4 += a.cpu().numpy()
        c2 += b.cpu().numpy()
    return m4, c2


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp16"])
@pytest.mark.parametrize("n,L,world", [(6000, 8, 2), (9001, 16, 3), (4000, 32, 5), (300, 4, 7)])
def test_fourth_order_slices_match_the_oracle(hos, oracle, prec, n, L, world):
    """Joined slices: c4 (from the joined m4 and c2) against the oracle's c4,
    and the trispectrum from the joined moments against the oracle's."""
    x = hos_synth.ma(n, 17 * n + world)
    m4, c2 = emulate_ranks4(hos, x, L, world, prec)
    T = hos.trispectrum_from_moments(torch.from_numpy(m4).cuda(), torch.from_numpy(c2).cuda(), L).cpu().numpy()
    ref = oracle.trispectrum(x, L, 2 * L)
    assert normwise(T, ref) <= TOL[prec]
    c2f = lambda t: c2[t + 2 * L - 1]  # noqa: E731
    r4 = oracle.c4(oracle.demean(x), L)[:2 * L, :2 * L, :2 * L]
    c4 = np.empty_like(m4)
    for w1 in range(-L, L):
        for w2 in range(-L, L):
            w3 = np.arange(-L, L)
            c4[w1 + L, w2 + L] = (m4[w1 + L, w2 + L] - c2f(w1) * c2[w3 - w2 + 2 * L - 1]
                                  - c2f(w2) * c2[w3 - w1 + 2 * L - 1] - c2[w3 + 2 * L - 1] * c2f(w2 - w1))
    assert np.abs(c4 - r4).max() <= TOL[prec] * np.abs(r4).max()


def test_fourth_order_sharded_single_rank_is_the_trispectrum(hos):
    """One rank (no process group): trispectrum_sharded equals hos_trispectrum
    to FP32 rounding (the same contraction, the c2 sums split otherwise)."""
    x = hos_synth.ma(20000, 23)
    xd = torch.from_numpy(x).cuda()
    a = hos.trispectrum_sharded(xd, 16, 0, 0, x.size, precision="fp32").cpu().numpy()
    b = hos.trispectrum(xd, 16, precision="fp32").cpu().numpy()
    assert normwise(a, b) <= 1e-6


def test_fourth_order_slice_argument_errors(hos):
    x = torch.from_numpy(hos_synth.ma(3000, 29)).cuda()
    tot = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(hos.HosError):
        hos.moments4_slice(x, 8, 0, 17, tot, 10000)  # halo after 2L + 1
    with pytest.raises(hos.HosError):
        hos.moments4_slice(x, 8, 9, 0, tot, 10000)  # halo before L + 1
    with pytest.raises(hos.HosError):
        hos.moments4_slice(x, 8, 0, 0, tot, 10000, precision="simt")
