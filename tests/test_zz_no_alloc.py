"""The allocation-free bispectrum entry point (hos_bispectrum_noalloc).

It serves callers that cannot allocate device memory -- code with no
allocator at hand, or running where cudaMalloc must not be called, such as a
host callback or a plug-in whose host application owns every allocation.
Instead of a caller-supplied workspace it uses one fixed scratch array inside
the library, shared by every call.  These checks call it through the C ABI and
compare it with hos_bispectrum (workspace supplied by the caller) on two calls
in a row with different inputs, so that anything the first call left in the
shared array and the second call wrongly reused would show.

This file is collected last so that a failure here does not hide the rest of
the suite in a run that stops at the first failure.
"""
import ctypes

import numpy as np
import pytest

import hos_synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no GPU", allow_module_level=True)

TOL = 1e-4  # split-bf16 gate of the parity tests


@pytest.fixture(scope="module")
def lib():
    from paper_1805_11775_gb300 import build, _native
    build.build()
    return _native.lib()


def _with_workspace(lib, x, p):
    import paper_1805_11775_gb300 as hos
    from paper_1805_11775_gb300 import _native
    N = p.nfft or 2 * p.L
    out = torch.empty((N, N), dtype=torch.complex64, device="cuda")
    nbytes = hos.workspace_size(_native.OP_BISPECTRUM, x.numel(), 1, x.numel(), p)
    ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
    wp = ws.data_ptr() + ((-ws.data_ptr()) % 256)
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.hos_bispectrum(x.data_ptr(), 1, x.numel(), ctypes.byref(p), out.data_ptr(), wp, nbytes, st) == 0
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _no_alloc(lib, x, p):
    N = p.nfft or 2 * p.L
    out = torch.empty((N, N), dtype=torch.complex64, device="cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.hos_bispectrum_noalloc(x.data_ptr(), 1, x.numel(), ctypes.byref(p), out.data_ptr(), st)
    torch.cuda.synchronize()
    return rc, out.cpu().numpy()


def test_no_alloc_matches_workspace_entry_point_on_consecutive_calls(lib):
    from paper_1805_11775_gb300 import make_params
    cases = [(hos_synth.workload("bispectrum_n2048_L32")["x"], make_params(32, precision="bf16")),
             (hos_synth.ar2(200_000, 17), make_params(64, precision="bf16"))]
    for x_np, p in cases:  # two calls in a row, different sizes and inputs
        x = torch.from_numpy(x_np).cuda()
        ref = _with_workspace(lib, x, p)
        rc, got = _no_alloc(lib, x, p)
        assert rc == 0
        err = np.abs(got.astype(np.complex128) - ref).max() / np.abs(ref).max()
        assert err <= TOL


def test_no_alloc_rejects_problems_beyond_its_fixed_scratch(lib):
    from paper_1805_11775_gb300 import make_params
    x = torch.zeros(1 << 21, dtype=torch.float64, device="cuda")
    p = make_params(256, precision="bf16")  # needs ~133 MiB of scratch
    out = torch.full((512, 512), 7.0, dtype=torch.complex64, device="cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.hos_bispectrum_noalloc(x.data_ptr(), 1, x.numel(), ctypes.byref(p), out.data_ptr(), st) == 3
    torch.cuda.synchronize()
    assert bool((out == 7.0).all())
