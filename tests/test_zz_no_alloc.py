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


@pytest.fixture(scope="module")
def lib():
    from paper_1805_11775_gb300 import build, _native
    build.build()
    return _native.lib()


def _dtype(x):
    return 1 if x.dtype == torch.float64 else 0


def _with_workspace(lib, x, p):
    import paper_1805_11775_gb300 as hos
    from paper_1805_11775_gb300 import _native
    N = p.nfft or 2 * p.L
    out = torch.empty((N, N), dtype=torch.complex64, device="cuda")
    nbytes = hos.workspace_size(_native.OP_BISPECTRUM, x.numel(), 1, x.numel(), p)
    ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
    wp = ws.data_ptr() + ((-ws.data_ptr()) % 256)
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.hos_bispectrum(x.data_ptr(), _dtype(x), x.numel(), ctypes.byref(p), out.data_ptr(), wp, nbytes,
                              st) == 0
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _no_alloc(lib, x, p):
    N = p.nfft or 2 * p.L
    out = torch.empty((N, N), dtype=torch.complex64, device="cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.hos_bispectrum_noalloc(x.data_ptr(), _dtype(x), x.numel(), ctypes.byref(p), out.data_ptr(), st)
    torch.cuda.synchronize()
    return rc, out.cpu().numpy()


def _status(lib):
    v = ctypes.c_int32(-1)
    assert lib.hos_bispectrum_noalloc_status(ctypes.byref(v)) == 0
    return v.value


def test_no_alloc_matches_workspace_entry_point_on_consecutive_calls(lib):
    from paper_1805_11775_gb300 import make_params
    small = hos_synth.workload("bispectrum_n2048_L32")["x"]
    cases = [
        # a large problem first, so that the small ones after it run on its leftovers
        (hos_synth.ar2(200_000, 17), make_params(64, precision="bf16")),
        (small, make_params(32, precision="bf16")),
        (hos_synth.exp_noise(small.size, 23), make_params(32, precision="bf16")),  # same shape, new input
        (hos_synth.ar2(30_000, 19), make_params(40, nfft=96, precision="fp32")),
        (hos_synth.ar2(30_000, 21).astype(np.float32), make_params(40, nfft=96, precision="fp32")),
        (hos_synth.ar2(40_000, 25), make_params(16, precision="bf16", segment_len=4096, segment_overlap=1024)),
        (small, make_params(32, precision="bf16")),  # the first small case again, after all the others
    ]
    for x_np, p in cases:
        x = torch.from_numpy(x_np).cuda()
        ref = _with_workspace(lib, x, p)
        rc, got = _no_alloc(lib, x, p)
        assert rc == 0
        assert _status(lib) == 0
        assert np.array_equal(got, ref), (x_np.size, p.L, p.precision)


def test_no_alloc_rejects_problems_beyond_its_fixed_scratch(lib):
    from paper_1805_11775_gb300 import make_params
    x = torch.zeros(1 << 21, dtype=torch.float64, device="cuda")
    p = make_params(256, precision="bf16")  # needs ~100 MiB of scratch
    out = torch.full((512, 512), 7.0, dtype=torch.complex64, device="cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.hos_bispectrum_noalloc(x.data_ptr(), 1, x.numel(), ctypes.byref(p), out.data_ptr(), st) == 3
    # an unknown dtype code is refused before anything is enqueued
    q = make_params(8, precision="bf16")
    assert lib.hos_bispectrum_noalloc(x.data_ptr(), 7, 100, ctypes.byref(q), out.data_ptr(), st) == 1
    torch.cuda.synchronize()
    assert bool((out == 7.0).all())
