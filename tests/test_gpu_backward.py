"""GPU parity of the bispectrum adjoint (hos_bispectrum_backward and the
autograd wrapper) against the oracle's FP64 gradient, which is itself pinned
by central differences.  Normwise tolerances: 1e-5 for the FP32-class
adjoints (precision "fp32" / "simt" on the CUDA cores, "fp16": split FP16 of
power-of-two scaled operands on the tensor cores), 1e-4 for the split-bf16
tensor-core adjoint."""
import numpy as np
import pytest

import hos_synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no GPU", allow_module_level=True)

TOL = {"fp32": 1e-5, "simt": 1e-5, "bf16": 1e-4, "fp16": 1e-5}


@pytest.fixture(scope="module")
def hos():
    from paper_1805_11775_gb300 import build
    build.build()
    import paper_1805_11775_gb300 as h
    return h


def principal_mask(N):
    k1, k2 = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    return (k2 <= k1) & (k1 + k2 < N // 2)


def normwise(got, ref):
    return np.abs(got - ref).max() / np.abs(ref).max()


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp16"])
@pytest.mark.parametrize("n,L,N,window,rm", [(40, 5, 10, "parzen", True), (300, 12, 24, "parzen", False),
                                             (2000, 40, 80, "parzen", True), (1500, 33, 70, "rect", True),
                                             (900, 20, 40, "parzen_sym", False), (5000, 128, 256, "parzen", True),
                                             (4321, 100, 200, "parzen", True), (700, 130, 260, "parzen", False)])
def test_backward_matches_oracle(hos, oracle, n, L, N, window, rm, prec):
    x = hos_synth.ar2(n, 7 * n)
    rng = np.random.default_rng(n)
    G = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    wk = {"parzen": oracle.WIN_PARZEN, "parzen_sym": oracle.WIN_PARZEN_SYM, "rect": oracle.WIN_RECT}[window]
    ref = oracle.bispectrum_grad(x, L, G, N, window=wk, remove_mean=rm)
    got = hos.bispectrum_backward(torch.from_numpy(x).cuda(), torch.from_numpy(G.astype(np.complex64)), L, nfft=N,
                                  window=window, remove_mean=rm, precision=prec).cpu().numpy()
    assert normwise(got, ref) <= TOL[prec]


@pytest.mark.parametrize("N", [8, 16, 1024])
def test_backward_transform_sizes(hos, oracle, N):
    """The adjoint transform (sign +1) on radix-8 register passes of every
    last-pass radix (8: N = 8, 2: N = 16, 2: N = 1024 after three)."""
    L = 3
    x = hos_synth.ar2(600, 11 * N)
    rng = np.random.default_rng(N)
    G = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    ref = oracle.bispectrum_grad(x, L, G, N)
    got = hos.bispectrum_backward(torch.from_numpy(x).cuda(), torch.from_numpy(G.astype(np.complex64)), L, nfft=N,
                                  precision="fp32").cpu().numpy()
    assert normwise(got, ref) <= TOL["fp32"]


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp16"])
def test_autograd_bispectrum_matching_loss(hos, oracle, prec):
    """l = sum over the principal domain of |B(x) - B_target|^2 through
    torch.autograd; the gradient equals the oracle's for the same G."""
    n, L = 3000, 32
    N = 2 * L
    x = torch.from_numpy(hos_synth.ar2(n, 1)).cuda().float().requires_grad_(True)
    Bt = hos.bispectrum(torch.from_numpy(hos_synth.ar2(n, 2)).cuda().float(), L)
    mask = torch.from_numpy(principal_mask(N)).cuda()
    B = hos.bispectrum_ad(x, L, precision=prec)
    loss = ((B - Bt).abs() ** 2 * mask).sum()
    loss.backward()
    G = (2 * (B.detach() - Bt) * mask).cpu().numpy().astype(np.complex128)
    ref = oracle.bispectrum_grad(x.detach().cpu().numpy().astype(np.float64), L, G, N)
    assert normwise(x.grad.cpu().numpy(), ref) <= TOL[prec]


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp16"])
def test_backward_full_size_sampled(hos, oracle, prec):
    """n = 2^18 float32 AR(2), L = 128, 256 x 256 grid, loss against the
    bispectrum of a second seeded series: the gradient at sampled samples
    (mean removal off, so each sample's gradient is local)."""
    w = hos_synth.workload("differentiable_n262144_L128")
    x, xt, L, N = w["x"], w["target_x"], w["L"], w["N"]
    xd = torch.from_numpy(x).cuda()
    B = hos.bispectrum(xd, L, precision="fp32", remove_mean=False)
    Bt = hos.bispectrum(torch.from_numpy(xt).cuda(), L, precision="fp32", remove_mean=False)
    G = (2 * (B - Bt) * torch.from_numpy(principal_mask(N)).cuda()).cpu().numpy()
    dx = hos.bispectrum_backward(xd, torch.from_numpy(G), L, remove_mean=False, precision=prec).cpu().numpy()
    dc = oracle.grad_lag(G.astype(np.complex128), L, N)
    rng = np.random.default_rng(3)
    js = np.concatenate([[0, 1, L, x.size - 1, x.size - L], rng.integers(0, x.size, 300)])
    ref = oracle.dy_at(x.astype(np.float64), L, dc, js)
    assert np.abs(dx[js] - ref).max() <= TOL[prec] * np.abs(ref).max()


# ------------------------------------------------------------------ trispectrum adjoint
@pytest.mark.parametrize("n,L,N,window,rm", [(40, 3, 6, "parzen", True), (700, 4, 8, "parzen", False),
                                             (1000, 8, 16, "rect", True), (1500, 13, 30, "parzen", True),
                                             (2000, 16, 32, "parzen", True), (800, 32, 64, "parzen", False),
                                             (500, 1, 2, "parzen", True), (300, 48, 96, "rect", False),
                                             (200, 64, 128, "parzen", True), (333, 5, 17, "parzen", True)])
@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_trispectrum_backward_matches_oracle(hos, oracle, n, L, N, window, rm, prec):
    """Split-bf16 and split-FP16 adjoints of the trispectrum against the
    oracle's FP64 chain rule (pinned by central differences), random complex
    dl/dT."""
    x = hos_synth.ar2(n, 13 * n + L)
    rng = np.random.default_rng(n + L)
    G = rng.standard_normal((N, N, N)) + 1j * rng.standard_normal((N, N, N))
    wk = {"parzen": oracle.WIN_PARZEN, "rect": oracle.WIN_RECT}[window]
    ref = oracle.trispectrum_grad(x, L, G, N, window=wk, remove_mean=rm)
    got = hos.trispectrum_backward(torch.from_numpy(x).cuda(), torch.from_numpy(G.astype(np.complex64)), L, nfft=N,
                                   window=window, remove_mean=rm, precision=prec).cpu().numpy()
    assert normwise(got, ref) <= TOL[prec]


def test_autograd_trispectrum_matching_loss(hos, oracle):
    """l = sum |T(x) - T_target|^2 through torch.autograd; the gradient equals
    the oracle's for the same dl/dT."""
    n, L = 2000, 16
    N = 2 * L
    x = torch.from_numpy(hos_synth.ar2(n, 21)).cuda().float().requires_grad_(True)
    Tt = hos.trispectrum(torch.from_numpy(hos_synth.ar2(n, 22)).cuda().float(), L)
    T = hos.trispectrum_ad(x, L)
    loss = ((T - Tt).abs() ** 2).sum()
    loss.backward()
    G = (2 * (T.detach() - Tt)).cpu().numpy().astype(np.complex128)
    ref = oracle.trispectrum_grad(x.detach().cpu().numpy().astype(np.float64), L, G, N)
    assert normwise(x.grad.cpu().numpy(), ref) <= TOL["bf16"]


def test_trispectrum_backward_full_size_sampled(hos, oracle):
    """The trispectrum workload's series (n = 65536, L = 32, 64^3 grid), loss
    against a second seeded series' trispectrum: the gradient at sampled
    samples, edges included (mean removal off, so each sample's gradient is
    local), from the oracle's transform, c2 and per-sample steps."""
    w = hos_synth.workload("trispectrum_n65536_L32")
    x, L = w["x"], 32
    N = 2 * L
    xd = torch.from_numpy(x).cuda()
    T = hos.trispectrum(xd, L, precision="fp32", remove_mean=False)
    Tt = hos.trispectrum(torch.from_numpy(hos_synth.ar2(x.size, 5)).cuda(), L, precision="fp32", remove_mean=False)
    G = (2 * (T - Tt)).cpu().numpy()
    dx = hos.trispectrum_backward(xd, torch.from_numpy(G), L, remove_mean=False).cpu().numpy()
    x64 = x.astype(np.float64)
    dc4 = oracle.grad_lag4(G.astype(np.complex128), L, N)
    dc2 = oracle.grad_c2(dc4, oracle.c2(x64, 2 * L), L)
    rng = np.random.default_rng(4)
    js = np.concatenate([[0, 1, L, 2 * L, x.size - 1, x.size - L, x.size - 2 * L], rng.integers(0, x.size, 57)])
    ref = oracle.dy4_at(x64, L, dc4, dc2, js)
    assert np.abs(dx[js] - ref).max() <= TOL["bf16"] * np.abs(ref).max()


@pytest.mark.parametrize("kw", [{"precision": "fp32"}, {"precision": "simt"}, {"window": "parzen_sym"}])
def test_trispectrum_backward_unsupported(hos, kw):
    x = torch.from_numpy(hos_synth.ar2(500, 9)).cuda()
    G = torch.zeros((16, 16, 16), dtype=torch.complex64)
    with pytest.raises(hos.HosError):
        hos.trispectrum_backward(x, G, 8, **kw)
    with pytest.raises(hos.HosError):
        hos.trispectrum_backward(x, torch.zeros((130, 130, 130), dtype=torch.complex64), 65)
