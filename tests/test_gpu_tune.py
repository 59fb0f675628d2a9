"""The autotuner on the GPU: tune_bispectrum_batched times every candidate
(tile_n, flush_chunks) on a small batch of intraday-shaped series, stores the
fastest in its cache, and the next call with automatic knobs runs that plan
(hos_last_plan names it); the tuned result matches the FP64 oracle per series
at the split-bf16 tolerance."""
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


def test_tuner_stores_and_applies_its_choice(hos, oracle, tmp_path, monkeypatch):
    from paper_1805_11775_gb300 import tune
    monkeypatch.setenv("HOS_TUNE_CACHE", str(tmp_path / "tune.json"))
    monkeypatch.setattr(tune, "_cache", None)
    lens = hos_synth.intraday_lengths(48, 31)
    vals, offs = hos_synth.student_t_returns(lens, 32)
    L, N = 128, 256
    vd = torch.from_numpy(vals).cuda()
    best, times = tune.tune_bispectrum_batched(vd, offs, L, precision="bf16", repeats=2)
    assert set(times) == set(tune.candidates(L, "bf16")) and best in times
    assert all(t > 0 for t in times.values())
    # stored under this device and library version, and found again
    monkeypatch.setattr(tune, "_cache", None)
    assert tune.lookup("bispectrum_batched", L, vd.numel(), lens.size, "bf16") == best
    got = hos.bispectrum_batched(vd, offs, L, precision="bf16").cpu().numpy()
    plan = hos.last_plan()
    assert f"tile_n={best[0]} " in plan and f"flush={best[1]} " in plan, plan
    assert f"kc={best[2] or 1024} " in plan, plan
    for s in (0, 7, 23, 47):
        ref = oracle.bispectrum(vals[offs[s]:offs[s + 1]], L, N)
        assert np.abs(got[s] - ref).max() / np.abs(ref).max() <= 1e-4, s
