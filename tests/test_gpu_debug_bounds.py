"""The bounds-checking build (HOS_DEBUG_BOUNDS) on the GPU.

In that build the contraction checks, before it issues them, that every bulk
copy stays inside its series' zero-padded block of the sample planes and
every partial tile goes to a slot inside the workspace; a violation is
recorded as HOS_ERR_DEVICE_FAULT in the status word and the kernel stops
before the access (no trap, no fault).  These tests run the small parity
shapes through that build in a child process (HOS_LIB selects it) and
require status 0 and oracle parity; then they make the check fire on purpose
by reporting a one-slot workspace to it (HOS_DEBUG_SHRINK_SLOTS=1, nothing
is accessed out of bounds) and require the fault status, and a clean status
from the next call."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no GPU", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import json, os, sys
sys.path.insert(0, sys.argv[1])
import numpy as np, torch
import hos_synth, oracle
import paper_1805_11775_gb300 as hos
from paper_1805_11775_gb300 import _native
assert _native.LIB_PATH.endswith("libhos_debug_bounds.so"), _native.LIB_PATH
def nw(a, b):
    return float(np.abs(np.asarray(a, np.complex128) - b).max() / np.abs(b).max())
out = {}
ws = hos.Workspace()
def status():
    torch.cuda.synchronize()
    return hos.device_status(ws)
if sys.argv[2] == "parity":
    for prec, tol in (("bf16", 1e-4), ("fp32", 1e-5), ("tf32", 3e-3)):
        for n, L, kw in ((3000, 40, {}), (9000, 200, {}), (5000, 24, {"segment_len": 1300}),
                         (4000, 16, {"segment_len": 1000, "segment_overlap": 300}), (700, 100, {})):
            x = hos_synth.ar2(n, n + L)
            B = hos.bispectrum(torch.from_numpy(x).cuda(), L, precision=prec, workspace=ws, **kw).cpu().numpy()
            if "segment_overlap" in kw:
                ref = oracle.bispectrum_overlap(x, L, 2 * L, segment_len=kw["segment_len"], overlap=kw["segment_overlap"])
            else:
                ref = oracle.bispectrum(x, L, 2 * L, segment_len=kw.get("segment_len", 0))
            out[f"bis_{prec}_{n}_{L}"] = [nw(B, ref), status(), tol]
    lens = np.array([0, 700, 2500, 17, 2048], dtype=np.int64)
    vals, offs = hos_synth.student_t_returns(lens, 3)
    got = hos.bispectrum_batched(torch.from_numpy(vals).cuda(), offs, 40, workspace=ws).cpu().numpy()
    out["batched"] = [max(nw(got[s], oracle.bispectrum(vals[offs[s]:offs[s + 1]], 40, 80))
                          for s in range(lens.size) if lens[s] > 0), status(), 1e-4]
    for prec, tol in (("bf16", 1e-4), ("fp32", 2e-5)):
        x = hos_synth.ma(3000, 5)
        T = hos.trispectrum(torch.from_numpy(x).cuda(), 8, precision=prec, workspace=ws).cpu().numpy()
        out[f"tri_{prec}"] = [nw(T, oracle.trispectrum(x, 8, 16)), status(), tol]
else:
    x = torch.from_numpy(hos_synth.ar2(20000, 9)).cuda()
    hos.reset_device_status(ws)
    os.environ["HOS_DEBUG_SHRINK_SLOTS"] = "1"
    hos.bispectrum(x, 64, workspace=ws)
    out["shrunk"] = status()
    del os.environ["HOS_DEBUG_SHRINK_SLOTS"]
    hos.reset_device_status(ws)
    B = hos.bispectrum(x, 64, workspace=ws).cpu().numpy()
    out["after"] = status()
    out["after_err"] = nw(B, oracle.bispectrum(x.cpu().numpy(), 64))
print(json.dumps(out))
'''


@pytest.fixture(scope="module")
def debug_lib():
    from paper_1805_11775_gb300 import build
    return build.build(debug_bounds=True)


def _run(debug_lib, mode):
    env = dict(os.environ, HOS_LIB=debug_lib)
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT, mode], env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_bounds_checked_build_passes_the_parity_shapes(debug_lib):
    out = _run(debug_lib, "parity")
    for k, (err, st, tol) in out.items():
        assert st == 0, (k, st)
        assert err <= tol, (k, err)


def test_bounds_check_records_a_fault_and_stops(debug_lib):
    out = _run(debug_lib, "shrink")
    assert out["shrunk"] == 6  # HOS_ERR_DEVICE_FAULT
    assert out["after"] == 0
    assert out["after_err"] <= 1e-4
