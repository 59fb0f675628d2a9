"""GPU parity of the bispectrum path (C ABI -> sm_103a kernels) against the
FP64 oracle.

Tolerances (normwise: max |got - ref| / max |ref| per output tensor), as the
accuracy targets of the contraction precisions:
  split-bf16 tensor cores 1e-4; 3xTF32 tensor cores 1e-5; split-FP16 tensor
  cores (FP32-class) 1e-5; FP32 SIMT 1e-5.  Plain TF32 is reported, not gated.
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
PRECS = ["simt", "fp32", "bf16", "fp16"]
TWO_PI = 2 * math.pi


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


def lag_slice(c_oracle, L):
    """Oracle c3 over [-L, L]^2 -> the library's [-L, L-1]^2 layout."""
    return c_oracle[:2 * L, :2 * L]


# ------------------------------------------------------------- workload 1
@pytest.mark.parametrize("prec", PRECS)
def test_bispectrum_n2048_L32(hos, oracle, prec):
    w = hos_synth.workload("bispectrum_n2048_L32")
    ref = oracle.bispectrum(w["x"], w["L"], w["N"])
    got = hos.bispectrum(torch.from_numpy(w["x"]).cuda(), w["L"], precision=prec).cpu().numpy()
    assert normwise(got, ref) <= TOL[prec]
    assert hos.device_status() == 0


# ------------------------------------------------------------- cumulant, tiles, ragged tails
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("n,L", [(1, 1), (2, 3), (3, 1), (7, 2), (100, 64), (1500, 31), (5000, 32),
                                 (3000, 128), (2600, 200), (9000, 256)])
def test_cumulant3_elementwise(hos, oracle, prec, n, L):
    x = hos_synth.ar2(n, 10 * n + L)
    ref = lag_slice(oracle.c3(oracle.demean(x), L), L)
    got = hos.cumulant3(torch.from_numpy(x).cuda(), L, precision=prec).cpu().numpy()
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= TOL[prec] * scale + 1e-300


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("n,L,N,window", [(1500, 31, 64, "parzen"), (3000, 128, 256, "parzen"),
                                          (2600, 50, 100, "parzen"), (800, 12, 40, "parzen_sym"),
                                          (800, 12, 24, "rect"), (4100, 256, 512, "parzen")])
def test_bispectrum_elementwise(hos, oracle, prec, n, L, N, window):
    x = hos_synth.ma(n, 77 + n)
    wk = {"parzen": oracle.WIN_PARZEN, "parzen_sym": oracle.WIN_PARZEN_SYM, "rect": oracle.WIN_RECT}[window]
    ref = oracle.bispectrum(x, L, N, window=wk)
    got = hos.bispectrum(torch.from_numpy(x).cuda(), L, nfft=N, precision=prec, window=window).cpu().numpy()
    assert normwise(got, ref) <= TOL[prec]


@pytest.mark.parametrize("N", [2, 4, 8, 16, 32, 128, 1024, 2048, 4096])
def test_transform_sizes(hos, oracle, N):
    """Every power-of-two grid size: radix-2 lines below 8 points, radix-8
    register passes (one to four of them, the last of radix 8, 4 or 2) from 8
    up to 4096.  Few lags keep the oracle's transform cheap on big grids."""
    L = min(3, N // 2)
    x = hos_synth.ar2(700, N)
    ref = oracle.bispectrum(x, L, N)
    got = hos.bispectrum(torch.from_numpy(x).cuda(), L, nfft=N, precision="fp32").cpu().numpy()
    assert normwise(got, ref) <= TOL["fp32"]


@pytest.mark.parametrize("prec", PRECS)
def test_symmetric_window_leaves_out_zero_tiles(hos, oracle, prec):
    """With d(w1 - w2) in the window, lag tiles where |w1 - w2| >= L
    everywhere are not contracted (1 of 10 tiles at tile width 128, 2 of 20
    at 64, L = 256); their grid entries are zero like the window."""
    x = hos_synth.ma(3000, 5)
    L = 256
    ref = oracle.bispectrum(x, L, 512, window=oracle.WIN_PARZEN_SYM)
    xd = torch.from_numpy(x).cuda()
    for tile_n in (128, 64):
        got = hos.bispectrum(xd, L, precision=prec, window="parzen_sym", tile_n=tile_n).cpu().numpy()
        assert normwise(got, ref) <= TOL[prec]


@pytest.mark.parametrize("tile_n,flush", [(128, 1), (256, 3), (64, 2)])
def test_tile_and_flush_variants_agree(hos, oracle, tile_n, flush):
    x = hos_synth.ar2(7000, 5)
    L = 100
    ref = lag_slice(oracle.c3(oracle.demean(x), L), L)
    for prec in ("bf16", "fp32", "fp16"):
        got = hos.cumulant3(torch.from_numpy(x).cuda(), L, precision=prec, tile_n=tile_n,
                            flush_chunks=flush).cpu().numpy()
        assert np.abs(got - ref).max() <= TOL[prec] * np.abs(ref).max()


def test_float32_input_and_no_mean_removal(hos, oracle):
    x = (hos_synth.exp_noise(3000, 3) + 0.25).astype(np.float32)
    for rm in (True, False):
        ref = oracle.bispectrum(x.astype(np.float64), 40, 80, remove_mean=rm)
        got = hos.bispectrum(torch.from_numpy(x).cuda(), 40, precision="fp32", remove_mean=rm).cpu().numpy()
        assert normwise(got, ref) <= 1e-5


def test_segments_average(hos, oracle):
    x = hos_synth.ar2(10_000, 8)
    ref = oracle.bispectrum(x, 24, 48, segment_len=3000)
    for prec in PRECS:
        got = hos.bispectrum(torch.from_numpy(x).cuda(), 24, precision=prec, segment_len=3000).cpu().numpy()
        assert normwise(got, ref) <= TOL[prec]


def test_zero_and_nan_inputs(hos):
    z = torch.zeros(5000, dtype=torch.float64, device="cuda")
    for prec in PRECS:
        assert torch.count_nonzero(hos.bispectrum(z, 32, precision=prec)).item() == 0
    x = torch.from_numpy(hos_synth.exp_noise(5000, 1)).cuda()
    x[1234] = float("nan")
    B = hos.bispectrum(x, 32, precision="bf16")
    assert torch.isnan(B.real).any()


def test_deterministic(hos):
    x = torch.from_numpy(hos_synth.ar2(50_000, 2)).cuda()
    for prec in PRECS:
        a = hos.bispectrum(x, 128, precision=prec)
        b = hos.bispectrum(x, 128, precision=prec)
        assert torch.equal(a, b)


# ------------------------------------------------------------- batching
def test_batched_matches_oracle_per_series(hos, oracle):
    """Intraday-return shaped series (symmetric Student-t): their true c3 is
    zero, so B is sampling noise about 200 times smaller than the sum of the
    absolute lag products (sum_w W c3(|y|) / max|B|), and the tensor cores'
    FP32 accumulation error (about 1e-8 of the partial sum per MMA step)
    shows through amplified: a batch's FP32-class plans keep each FP32
    partial within 192 MMA steps (3xTF32: 512-sample chunks; split FP16: one
    chunk per partial), which meets the 1e-5 target here.  Every precision
    at its target."""
    lens = np.array([0, 1, 700, 2500, 1024, 3100, 17, 2048], dtype=np.int64)
    vals, offs = hos_synth.student_t_returns(lens, 11)
    L, N = 40, 80
    for prec in PRECS:
        got = hos.bispectrum_batched(torch.from_numpy(vals).cuda(), torch.from_numpy(offs), L,
                                     precision=prec).cpu().numpy()
        for s in range(lens.size):
            seg = vals[offs[s]:offs[s + 1]]
            if seg.size == 0:
                assert np.count_nonzero(got[s]) == 0
                continue
            ref = oracle.bispectrum(seg, L, N)
            if np.abs(ref).max() == 0:  # a one-sample series is all mean: B = 0
                assert np.abs(got[s]).max() <= 1e-30
                continue
            assert normwise(got[s], ref) <= TOL[prec], (prec, s)


def test_batched_host_pipeline_matches_one_device_call(hos):
    """Host input with a pinned host output: series in groups whose copies
    overlap the next group's compute; the same spectra as one device call
    within the 3xTF32 target (the groups' contraction splits differ, so the
    FP32 accumulation order differs)."""
    lens = hos_synth.intraday_lengths(37, 5)
    vals, offs = hos_synth.student_t_returns(lens, 6)
    L, N = 16, 32
    dev = hos.bispectrum_batched(torch.from_numpy(vals).cuda(), offs, L, precision="fp32").cpu().numpy()
    out = torch.empty((lens.size, N, N), dtype=torch.complex64).pin_memory()
    got = hos.bispectrum_batched(torch.from_numpy(vals).pin_memory(), offs, L, precision="fp32", out=out,
                                 pipeline=4).numpy()
    assert normwise(got, dev) <= TOL["fp32"]


def test_batched_equals_single_calls(hos):
    lens = hos_synth.intraday_lengths(24, 4)
    vals, offs = hos_synth.student_t_returns(lens, 4)
    xb = torch.from_numpy(vals).cuda()
    Bb = hos.bispectrum_batched(xb, torch.from_numpy(offs), 128, precision="bf16")
    for s in range(0, 24, 5):
        Bs = hos.bispectrum(xb[offs[s]:offs[s + 1]].contiguous(), 128, precision="bf16")
        assert normwise(Bb[s].cpu().numpy(), Bs.cpu().numpy().astype(np.complex128)) <= 2e-5


def test_batched_many_series_reduction_matches_single_calls(hos):
    """128 series and more take the reduction's many-group kernels (four
    vectors per thread, one-window series in a kernel of their own): each
    series' spectrum equals its single call's within the split-bf16 target."""
    lens = hos_synth.intraday_lengths(160, 9)
    vals, offs = hos_synth.student_t_returns(lens, 9)
    xb = torch.from_numpy(vals).cuda()
    Bb = hos.bispectrum_batched(xb, torch.from_numpy(offs), 128, precision="bf16").cpu().numpy()
    for s in list(range(0, 160, 23)) + [159]:
        Bs = hos.bispectrum(xb[offs[s]:offs[s + 1]].contiguous(), 128, precision="bf16").cpu().numpy()
        assert normwise(Bb[s], Bs.astype(np.complex128)) <= 1e-4, s


# ------------------------------------------------------------- long workload at full size
@pytest.fixture(scope="module")
def long_inputs():
    w = hos_synth.workload("long_bispectrum_n2M_L256")
    return w


@pytest.mark.parametrize("prec", ["bf16", "fp32"])
def test_long_full_size_sampled_lags(hos, oracle, long_inputs, prec):
    """n = 2^21, L = 256: lags sampled over the whole square (including every
    tile, the mirrored ones and the boundary lags) against the oracle's
    per-lag sums."""
    x, L = long_inputs["x"], long_inputs["L"]
    y = oracle.demean(x)
    rng = np.random.default_rng(0)
    lags = np.concatenate([rng.integers(-L, L, size=(40, 2)),
                           np.array([[0, 0], [-L, -L], [L - 1, L - 1], [-L, L - 1], [L - 1, -L], [1, 2], [2, 1],
                                     [-5, 7], [200, -100], [-100, 200]])])
    ref = oracle.c3_at(y, lags)
    got = hos.cumulant3(torch.from_numpy(x).cuda(), L, precision=prec).cpu().numpy()
    g = got[lags[:, 0] + L, lags[:, 1] + L]
    assert np.abs(g - ref).max() <= TOL[prec] * abs(oracle.c3_at(y, [[0, 0]])[0])


@pytest.mark.parametrize("prec", ["bf16", "fp32"])
def test_long_full_size_spectrum_properties(hos, oracle, long_inputs, prec):
    """At full size the transform is checked through properties that hold at
    any size: Hermitian symmetry, B(k1,k2) = B(k2,k1), and the inverse
    transform at sampled lags equals (2 pi)^-2 W(w) c3(w) from the oracle."""
    x, L, N = long_inputs["x"], long_inputs["L"], long_inputs["N"]
    B = hos.bispectrum(torch.from_numpy(x).cuda(), L, precision=prec).cpu().numpy().astype(np.complex128)
    k = np.arange(N)
    scale = np.abs(B).max()
    assert np.abs(B[(-k[:, None]) % N, (-k[None, :]) % N] - np.conj(B)).max() <= 1e-6 * scale
    assert np.abs(B - B.T).max() <= 1e-6 * scale
    y = oracle.demean(x)
    lags = np.array([[0, 0], [1, 0], [3, -2], [10, 20], [-40, 17], [100, 101], [-200, 50], [250, -250]])
    ref = oracle.c3_at(y, lags) * np.array([oracle.window2(a, b, L) for a, b in lags]) / TWO_PI ** 2
    ph = np.exp(2j * np.pi * (np.outer(lags[:, 0], k)[:, :, None] + np.outer(lags[:, 1], k)[:, None, :]) / N)
    inv = (B[None, :, :] * ph).sum(axis=(1, 2)).real / (N * N)
    assert np.abs(inv - ref).max() <= TOL[prec] * abs(ref[0])


# ------------------------------------------------------------- failure detection, tracing
def test_device_timeout_is_reported_without_a_fault(hos):
    assert hos.selftest_timeout(2000) == 5  # HOS_ERR_TIMEOUT
    hos.reset_device_status()
    torch.cuda.synchronize()
    assert hos.device_status() == 0
    x = torch.from_numpy(hos_synth.exp_noise(4096, 9)).cuda()
    B = hos.bispectrum(x, 32)
    torch.cuda.synchronize()
    assert torch.isfinite(B.real).all() and hos.device_status() == 0


def test_stage_times_and_launch_count(hos):
    x = torch.from_numpy(hos_synth.exp_noise(100_000, 9)).cuda()
    n0 = hos.launch_count()
    hos.set_profiling(True)
    hos.bispectrum(x, 64, precision="bf16")
    st = hos.stage_times()
    hos.set_profiling(False)
    assert [s for s, _ in st] == ["prep", "contract", "reduce", "transform"]
    assert all(ms >= 0 for _, ms in st)
    assert hos.launch_count() - n0 >= 7
    assert hos.last_contraction() == "c3_tcgen05_split_bf16"


def test_plain_tf32_is_reported(hos, oracle):
    """One plain TF32 product per term has no accuracy target: its normwise
    error against the oracle is printed for the record (the factors carry 11
    significant bits), checked only for being finite and small."""
    w = hos_synth.workload("bispectrum_n2048_L32")
    ref = oracle.bispectrum(w["x"], w["L"], w["N"])
    got = hos.bispectrum(torch.from_numpy(w["x"]).cuda(), w["L"], precision="tf32").cpu().numpy()
    err = normwise(got, ref)
    print(f"plain TF32 bispectrum n=2048 L=32: normwise error {err:.3e} ({hos.last_contraction()})")
    assert hos.last_contraction() == "c3_tcgen05_tf32"
    assert np.isfinite(err) and err < 1e-2


def test_split_fp16_scales_any_magnitude(hos, oracle):
    """The split-FP16 planes are scaled per series by a power of two; series of
    very small and very large magnitude (and a batch mixing them) keep the
    FP32-class accuracy."""
    base = hos_synth.ar2(6000, 41)
    for mag in (1e-6, 1.0, 3e5):
        x = base * mag
        ref = oracle.bispectrum(x, 64, 128)
        got = hos.bispectrum(torch.from_numpy(x).cuda(), 64, precision="fp16").cpu().numpy()
        assert normwise(got, ref) <= TOL["fp16"], mag
    lens = np.array([1500, 2600, 900], dtype=np.int64)
    vals = np.concatenate([hos_synth.ar2(1500, 42) * 1e-5, hos_synth.ar2(2600, 43) * 1e4, hos_synth.ar2(900, 44)])
    offs = np.concatenate([[0], np.cumsum(lens)])
    got = hos.bispectrum_batched(torch.from_numpy(vals).cuda(), offs, 32, precision="fp16").cpu().numpy()
    for s in range(3):
        ref = oracle.bispectrum(vals[offs[s]:offs[s + 1]], 32, 64)
        assert normwise(got[s], ref) <= TOL["fp16"], s


def test_batched_workload_full_size_sampled(hos, oracle):
    """The batched workload at full size (4096 intraday-shaped series, lengths
    2000..20000, L = 128, 256 x 256 grids) in one call: sixteen spectra
    across the batch (first, last, shortest, longest and twelve spread out)
    against the oracle at the split-bf16 and split-FP16 targets."""
    w = hos_synth.workload("batched_4096x_L128")
    vals, offs = w["x"], w["offsets"]
    lens = np.diff(offs)
    pick = sorted({0, lens.size - 1, int(lens.argmin()), int(lens.argmax())} |
                  set(np.linspace(1, lens.size - 2, 12).astype(int).tolist()))
    refs = {s: oracle.bispectrum(vals[offs[s]:offs[s + 1]], 128, 256) for s in pick}
    vd = torch.from_numpy(vals).cuda()
    for prec in ("bf16", "fp16"):
        got = hos.bispectrum_batched(vd, offs, 128, precision=prec, max_len=int(lens.max()))
        for s in pick:
            assert normwise(got[s].cpu().numpy(), refs[s]) <= TOL[prec], (prec, s)
