"""Host-side checks of the C ABI (no GPU needed): the library builds for
sm_103a, loads, exports every entry point include/hos.h declares, and
rejects bad arguments synchronously without touching the device."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hos.h")

pytestmark = pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                                reason="nvcc not available")


@pytest.fixture(scope="module")
def lib():
    from paper_1805_11775_gb300 import build, _native
    build.build()
    return _native.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hos_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_the_header():
    from paper_1805_11775_gb300 import _native
    assert set(declared_functions()) == set(_native._SIGS)


def test_params_struct_matches_header():
    from paper_1805_11775_gb300 import _native
    text = open(HEADER).read()
    body = text[text.index("typedef struct {"):text.index("} hos_params;")]
    fields = re.findall(r"int32_t\s+(\w+);", body)
    assert [f for f, _ in _native.HosParams._fields_] == fields


def _params(**kw):
    from paper_1805_11775_gb300 import make_params
    return make_params(**kw)


def test_status_strings(lib):
    for s in range(7):
        assert lib.hos_status_string(s)
    assert b"sm_103a" in lib.hos_version()


def test_invalid_arguments_return_synchronously(lib):
    from paper_1805_11775_gb300 import _native
    p = _params(L=32)
    dummy = ctypes.c_void_p(0x1000)
    # null pointers, bad sizes, bad dtype: rejected before any CUDA call
    assert lib.hos_bispectrum(None, 1, 100, ctypes.byref(p), dummy, dummy, 1 << 20, None) == 1
    assert lib.hos_bispectrum(dummy, 7, 100, ctypes.byref(p), dummy, dummy, 1 << 20, None) == 1
    assert lib.hos_bispectrum(dummy, 1, 0, ctypes.byref(p), dummy, dummy, 1 << 20, None) == 1
    for bad in (dict(L=0), dict(L=32, nfft=10), dict(L=32, precision=5), dict(L=32, precision=-1), dict(L=32, window=5),
                dict(L=32, tile_n=48), dict(L=32, segment_len=-1),
                dict(L=32, chunk_len=100), dict(L=32, chunk_len=2048), dict(L=32, chunk_len=-64)):
        q = _params(**bad)
        assert lib.hos_bispectrum(dummy, 1, 100, ctypes.byref(q), dummy, dummy, 1 << 20, None) == 1, bad
    big = _params(L=2048)
    assert lib.hos_bispectrum(dummy, 1, 100, ctypes.byref(big), dummy, dummy, 1 << 20, None) == 2
    # workspace too small
    assert lib.hos_bispectrum(dummy, 1, 100, ctypes.byref(p), dummy, dummy, 16, None) == 3
    assert lib.hos_bispectrum_batched(dummy, 1, None, 3, 10, 5, ctypes.byref(p), dummy, dummy, 1 << 30, None) == 1
    assert lib.hos_get_device_status(None, None) == 1
    assert _native.STATUS_NAMES[3] == "HOS_ERR_WORKSPACE"
    # time slices: halos longer than L, a whole series shorter than its slice,
    # parts inside a slice, null pointers
    ws = ctypes.c_void_p(0x100000)
    assert lib.hos_cumulant3_slice(dummy, 1, 100, 33, 0, dummy, 1000, ctypes.byref(p), dummy, ws, 1 << 30, None) == 1
    assert lib.hos_cumulant3_slice(dummy, 1, 100, 4, 4, dummy, 107, ctypes.byref(p), dummy, ws, 1 << 30, None) == 1
    seg = _params(L=32, segment_len=50)
    assert lib.hos_cumulant3_slice(dummy, 1, 100, 0, 0, dummy, 100, ctypes.byref(seg), dummy, ws, 1 << 30,
                                   None) == 1
    assert lib.hos_cumulant3_slice(dummy, 1, 100, 0, 0, None, 100, ctypes.byref(p), dummy, ws, 1 << 30, None) == 1
    assert lib.hos_series_sum(dummy, 1, 0, dummy, ws, 1 << 20, None) == 1
    assert lib.hos_series_sum(dummy, 1, 100, dummy, ws, 8, None) == 3
    assert lib.hos_bispectrum_from_cumulant(None, ctypes.byref(p), dummy, ws, 1 << 20, None) == 1
    assert lib.hos_bispectrum_from_cumulant(dummy, ctypes.byref(_params(L=32, nfft=8)), dummy, ws, 1 << 20,
                                            None) == 1
    assert lib.hos_bispectrum_from_cumulant(dummy, ctypes.byref(p), dummy, ws, 64, None) == 3


def test_workspace_size_grows_with_the_problem(lib):
    from paper_1805_11775_gb300 import workspace_size, _native
    p = _params(L=256)
    a = workspace_size(_native.OP_BISPECTRUM, 1 << 16, 1, 1 << 16, p)
    b = workspace_size(_native.OP_BISPECTRUM, 1 << 21, 1, 1 << 21, p)
    assert 0 < a < b
    c = workspace_size(_native.OP_BISPECTRUM_BATCHED, 45_000_000, 4096, 20000, _params(L=128))
    assert c > 4096 * 256 * 256 * 4  # at least the transform grid
    # the full-size long workload stays far below the device memory
    assert b < 2 << 30


def test_trispectrum_backward_workspace_and_limits(lib):
    """The trispectrum adjoint's workspace holds the adjoint grid, the per-block
    row partials ((2L)^2 / 128 blocks x n floats) and the rest; precisions other
    than the split ones (bf16, FP16), L > 64 and the symmetric window are
    refused on the host."""
    from paper_1805_11775_gb300 import workspace_size, _native, HosError
    n = 1 << 16
    a = workspace_size(_native.OP_TRISPECTRUM_BACKWARD, n, 1, n, _params(L=32, precision=1))
    assert a > 32 * n * 4 + 64 ** 3 * 8
    b = workspace_size(_native.OP_TRISPECTRUM_BACKWARD, n, 1, n, _params(L=64, precision=1))
    assert b > a
    assert workspace_size(_native.OP_TRISPECTRUM_BACKWARD, n, 1, n, _params(L=32, precision="fp16")) > 0
    for bad in (_params(L=32, precision="fp32"), _params(L=32, precision="tf32"), _params(L=32, precision="simt"),
                _params(L=65, precision=1),
                _params(L=32, precision=1, window=1), _params(L=32, precision=1, segment_len=1000)):
        with pytest.raises(HosError):
            workspace_size(_native.OP_TRISPECTRUM_BACKWARD, n, 1, n, bad)
    dummy = ctypes.c_void_p(16)
    ws = ctypes.c_void_p(256)
    p = _params(L=8, precision=1)
    assert lib.hos_trispectrum_backward(None, 0, 100, ctypes.byref(p), dummy, dummy, ws, 1 << 20, None) == 1
    assert lib.hos_trispectrum_backward(dummy, 0, 100, ctypes.byref(p), dummy, dummy, ws, 64, None) == 3


def test_overlap_workspace_and_checks(lib):
    """Overlapping parts: the workspace holds the parts written out (K x m
    samples) beyond the plan for K x m samples; bad overlaps are refused on
    the host, and ops without parts refuse any overlap."""
    from paper_1805_11775_gb300 import workspace_size, _native, HosError
    n, m, o = 100_000, 4096, 1024
    K = (n - m) // (m - o) + 1
    plain = workspace_size(_native.OP_BISPECTRUM, K * m, 1, K * m, _params(L=64, segment_len=m))
    ov = workspace_size(_native.OP_BISPECTRUM, n, 1, n, _params(L=64, segment_len=m, segment_overlap=o))
    assert ov >= plain + K * m * 8
    same = workspace_size(_native.OP_BISPECTRUM, 3000, 1, 3000, _params(L=64, segment_len=m, segment_overlap=o))
    assert same == workspace_size(_native.OP_BISPECTRUM, 3000, 1, 3000, _params(L=64, segment_len=m))
    for bad in (_params(L=8, segment_len=100, segment_overlap=100), _params(L=8, segment_overlap=5),
                _params(L=8, segment_len=100, segment_overlap=-1)):
        with pytest.raises(HosError):
            workspace_size(_native.OP_BISPECTRUM, n, 1, n, bad)
    for op in (_native.OP_BISPECTRUM_BATCHED, _native.OP_TRISPECTRUM_BACKWARD, _native.OP_SERIES_SUM):
        with pytest.raises(HosError):
            workspace_size(op, n, 1, n, _params(L=8, segment_len=100, segment_overlap=5, precision=1))


def test_fourth_order_slice_checks(lib):
    """Time slices of the fourth order: workspace sizes, and halos, precision
    and segment checks on the host."""
    from paper_1805_11775_gb300 import workspace_size, _native, HosError
    a = workspace_size(_native.OP_MOMENTS4_SLICE, 50_000, 1, 50_000, _params(L=32, precision=1))
    assert a > 0
    f = workspace_size(_native.OP_TRISPECTRUM_FROM_MOMENTS, 0, 1, 0, _params(L=32, precision=1))
    assert f >= 64 ** 3 * 4
    assert workspace_size(_native.OP_MOMENTS4_SLICE, 50_000, 1, 50_000, _params(L=32, precision="tf32")) > 0
    with pytest.raises(HosError):
        workspace_size(_native.OP_MOMENTS4_SLICE, 50_000, 1, 50_000, _params(L=32, precision="simt"))
    with pytest.raises(HosError):
        workspace_size(_native.OP_MOMENTS4_SLICE, 50_000, 1, 50_000, _params(L=65, precision=1))
    dummy = ctypes.c_void_p(16)
    ws = ctypes.c_void_p(256)
    p = _params(L=8, precision=1)
    # halo_after 2L + 1 and halo_before L + 1 are refused; so is n_total too short
    assert lib.hos_moments4_slice(dummy, 0, 1000, 0, 17, dummy, 5000, ctypes.byref(p), dummy, dummy, ws, 1 << 30,
                                  None) == 1
    assert lib.hos_moments4_slice(dummy, 0, 1000, 9, 0, dummy, 5000, ctypes.byref(p), dummy, dummy, ws, 1 << 30,
                                  None) == 1
    assert lib.hos_moments4_slice(dummy, 0, 1000, 8, 16, dummy, 1000, ctypes.byref(p), dummy, dummy, ws, 1 << 30,
                                  None) == 1
    assert lib.hos_trispectrum_from_moments(None, dummy, ctypes.byref(p), dummy, ws, 1 << 30, None) == 1


_FAULT_CHILD = r'''
import ctypes, json, sys
sys.path.insert(0, sys.argv[1])
from paper_1805_11775_gb300 import _native, make_params
lib = _native.lib()
d = ctypes.c_void_p(1 << 20)      # never dereferenced: every call stops before any GPU work
ws = ctypes.c_void_p(1 << 30)     # 256-byte aligned
big = ctypes.c_size_t(1 << 40)
out = {}
p = make_params(16, precision=1)
out["bispectrum"] = lib.hos_bispectrum(d, 1, 5000, ctypes.byref(p), d, ws, big, None)
out["trispectrum"] = lib.hos_trispectrum(d, 1, 5000, ctypes.byref(make_params(8, precision=1)), d, ws, big, None)
out["backward"] = lib.hos_bispectrum_backward(d, 1, 5000, ctypes.byref(p), d, d, ws, big, None)
out["tri_backward"] = lib.hos_trispectrum_backward(d, 1, 5000, ctypes.byref(make_params(8, precision=1)), d, d, ws,
                                                   big, None)
out["overlap"] = lib.hos_bispectrum(d, 1, 50000, ctypes.byref(make_params(16, precision=1, segment_len=4096,
                                                                          segment_overlap=1024)), d, ws, big, None)
print(json.dumps(out))
'''


@pytest.mark.parametrize("fault,status", [("workspace", 3), ("cuda", 4)])
def test_host_fault_injection(lib, fault, status):
    """HOS_FAULT=workspace / cuda: every entry point reports the injected
    status after its argument checks, before anything reaches a GPU (runs
    here without one)."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, HOS_FAULT=fault)
    r = subprocess.run([sys.executable, "-c", _FAULT_CHILD, root], env=env, capture_output=True, text=True,
                       timeout=120)
    assert r.returncode == 0, r.stderr
    got = json.loads(r.stdout.strip().splitlines()[-1])
    assert all(v == status for v in got.values()), got
