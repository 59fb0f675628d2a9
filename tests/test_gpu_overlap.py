"""GPU parity of overlapping parts on the indirect path (segment_len with
segment_overlap: parts of segment_len samples every segment_len - overlap
samples, each demeaned, cumulants averaged) against the oracle's FP64
overlapping-part estimates, which are pinned against the plain segment
average of the parts written out."""
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
    return np.abs(np.asarray(got, dtype=np.complex128) - ref).max() / np.abs(ref).max()


@pytest.mark.parametrize("prec", ["simt", "fp32", "bf16", "fp16"])
@pytest.mark.parametrize("n,m,o,L,N,rm", [(5000, 1024, 256, 16, 32, True), (3001, 700, 699, 8, 20, False),
                                          (2100, 1000, 1, 32, 64, True), (9000, 2048, 1024, 40, 80, True)])
def test_bispectrum_overlap_matches_oracle(hos, oracle, prec, n, m, o, L, N, rm):
    x = hos_synth.ar2(n, 7 * n + o)
    ref = oracle.bispectrum_overlap(x, L, N, remove_mean=rm, segment_len=m, overlap=o)
    got = hos.bispectrum(torch.from_numpy(x).cuda(), L, nfft=N, precision=prec, remove_mean=rm, segment_len=m,
                         segment_overlap=o).cpu().numpy()
    assert normwise(got, ref) <= TOL[prec]


@pytest.mark.parametrize("prec", ["simt", "fp32", "bf16", "fp16"])
def test_trispectrum_overlap_matches_oracle(hos, oracle, prec):
    n, m, o, L = 4000, 1000, 500, 8
    x = hos_synth.ma(n, 31)
    ref = oracle.trispectrum_overlap(x, L, 2 * L, segment_len=m, overlap=o)
    got = hos.trispectrum(torch.from_numpy(x).cuda(), L, precision=prec, segment_len=m,
                          segment_overlap=o).cpu().numpy()
    assert normwise(got, ref) <= TOL[prec]


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp16"])
def test_cumulants_overlap_match_oracle(hos, oracle, prec):
    n, m, o = 3000, 800, 300
    x = hos_synth.ar2(n, 33)
    L3, L4 = 12, 6
    c3 = hos.cumulant3(torch.from_numpy(x).cuda(), L3, precision=prec, segment_len=m, segment_overlap=o).cpu().numpy()
    r3 = oracle.cumulant_overlap(x, L3, 3, segment_len=m, overlap=o)[:2 * L3, :2 * L3]
    assert np.abs(c3 - r3).max() <= TOL[prec] * np.abs(r3).max()
    c4 = hos.cumulant4(torch.from_numpy(x).cuda(), L4, precision=prec, segment_len=m, segment_overlap=o).cpu().numpy()
    r4 = oracle.cumulant_overlap(x, L4, 4, segment_len=m, overlap=o)[:2 * L4, :2 * L4, :2 * L4]
    assert np.abs(c4 - r4).max() <= TOL[prec] * np.abs(r4).max()


def test_short_series_with_overlap_is_one_part(hos):
    x = torch.from_numpy(hos_synth.ar2(900, 35)).cuda()
    a = hos.bispectrum(x, 10, precision="fp32", segment_len=1000, segment_overlap=100).cpu().numpy()
    b = hos.bispectrum(x, 10, precision="fp32").cpu().numpy()
    assert np.array_equal(a, b)


def test_overlap_argument_errors(hos):
    x = torch.from_numpy(hos_synth.ar2(3000, 37)).cuda()
    for kw in ({"segment_len": 500, "segment_overlap": 500}, {"segment_len": 0, "segment_overlap": 10},
               {"segment_len": 500, "segment_overlap": -1}):
        with pytest.raises(hos.HosError):
            hos.bispectrum(x, 8, **kw)
    from paper_1805_11775_gb300 import _native
    for op in (_native.OP_BISPECTRUM_BATCHED, _native.OP_BISPECTRUM_BACKWARD, _native.OP_TRISPECTRUM_BATCHED):
        with pytest.raises(hos.HosError):
            hos.workspace_size(op, 3000, 1, 3000, hos.make_params(8, segment_len=500, segment_overlap=10))
