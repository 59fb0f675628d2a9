"""Every entry point's launches can be captured in a CUDA graph (no host
synchronisation, no allocation once the workspace and outputs exist) and a
replay reproduces the eager result bit for bit."""
import numpy as np
import pytest

import hos_synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no GPU", allow_module_level=True)


@pytest.fixture(scope="module")
def hos():
    from paper_1805_11775_gb300 import build
    build.build()
    import paper_1805_11775_gb300 as h
    return h


def _replay_equals_eager(fn):
    eager = fn().clone()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        out = fn()
    g.replay()
    torch.cuda.synchronize()
    a, b = eager.cpu().numpy(), out.cpu().numpy()
    assert a.shape == b.shape
    assert np.array_equal(a.view(np.uint8), b.view(np.uint8))
    g.replay()  # a second replay into the same buffers
    torch.cuda.synchronize()
    assert np.array_equal(a.view(np.uint8), out.cpu().numpy().view(np.uint8))


@pytest.mark.parametrize("prec", ["bf16", "fp32", "simt", "fp16"])
def test_bispectrum_graph(hos, prec):
    x = torch.from_numpy(hos_synth.ar2(20000, 41)).cuda()
    ws = hos.Workspace()
    out = torch.empty((64, 64), dtype=torch.complex64, device="cuda")
    _replay_equals_eager(lambda: hos.bispectrum(x, 32, precision=prec, out=out, workspace=ws))


def test_bispectrum_overlap_graph(hos):
    x = torch.from_numpy(hos_synth.ar2(20000, 42)).cuda()
    ws = hos.Workspace()
    out = torch.empty((48, 48), dtype=torch.complex64, device="cuda")
    _replay_equals_eager(lambda: hos.bispectrum(x, 24, segment_len=4096, segment_overlap=1024, out=out,
                                                workspace=ws))


@pytest.mark.parametrize("prec", ["bf16", "fp32", "fp16"])
def test_trispectrum_graph(hos, prec):
    x = torch.from_numpy(hos_synth.ma(30000, 43)).cuda()
    ws = hos.Workspace()
    out = torch.empty((32, 32, 32), dtype=torch.complex64, device="cuda")
    _replay_equals_eager(lambda: hos.trispectrum(x, 16, precision=prec, out=out, workspace=ws))


def test_batched_graph(hos):
    rng = np.random.default_rng(44)
    lens = rng.integers(100, 5000, 40)
    offs = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    vals = hos_synth.exp_noise(int(offs[-1]), 45)
    vd, od = torch.from_numpy(vals).cuda(), torch.from_numpy(offs).cuda()
    ws = hos.Workspace()
    out = torch.empty((40, 32, 32), dtype=torch.complex64, device="cuda")
    _replay_equals_eager(lambda: hos.bispectrum_batched(vd, od, 16, out=out, workspace=ws,
                                                        max_len=int(lens.max())))


def test_backward_graphs(hos):
    x = torch.from_numpy(hos_synth.ar2(30000, 46)).cuda().float()
    gB = torch.randn((64, 64), dtype=torch.complex64, device="cuda")
    gT = torch.randn((32, 32, 32), dtype=torch.complex64, device="cuda")
    ws1, ws2 = hos.Workspace(), hos.Workspace()
    _replay_equals_eager(lambda: hos.bispectrum_backward(x, gB, 32, workspace=ws1))
    _replay_equals_eager(lambda: hos.trispectrum_backward(x, gT, 16, workspace=ws2))


def test_direct_graph(hos):
    x = torch.from_numpy(hos_synth.ar2(4096, 47)).cuda()
    ws = hos.Workspace()
    out = torch.empty((1024, 1024), dtype=torch.complex64, device="cuda")
    _replay_equals_eager(lambda: hos.bispectrum_direct(x, 1024, 31, overlap=512, out=out, workspace=ws))
