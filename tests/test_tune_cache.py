"""Autotuner cache logic (no GPU): keys, candidate sets, corrupt-cache recovery."""
import json

import pytest

from paper_1805_11775_gb300 import tune


def test_candidates_respect_precision_and_lag_range():
    assert all(f <= 2 for _, f, _ in tune.candidates(256, "fp32"))
    # the FP32-class candidates keep a partial's MMA steps within their budget
    steps = {"fp32": 384 / 1024, "fp16": 192 / 1024}
    for prec, per_sample in steps.items():
        assert max(f * c * per_sample for _, f, c in tune.candidates(256, prec)) <= 384
        assert max(f * c * per_sample for _, f, c in tune.candidates(256, prec, batched=True)) <= 192
    assert {t for t, _, _ in tune.candidates(256, "bf16")} == {128, 256}
    assert {t for t, _, _ in tune.candidates(40, "bf16")} == {128}


def test_key_buckets_sizes():
    a = tune.key("GB300", "bispectrum", 128, 3000, 1, "bf16")
    b = tune.key("GB300", "bispectrum", 128, 4000, 1, "bf16")
    c = tune.key("GB300", "bispectrum", 128, 5000, 1, "bf16")
    assert a == b != c


def test_key_names_the_library_version():
    a = tune.key("GB300", "bispectrum", 128, 3000, 1, "bf16", "hos-gb300 0.1")
    b = tune.key("GB300", "bispectrum", 128, 3000, 1, "bf16", "hos-gb300 0.2")
    assert a != b


def test_corrupt_cache_is_rebuilt(tmp_path, monkeypatch):
    p = tmp_path / "tune.json"
    p.write_text("{not json")
    monkeypatch.setenv("HOS_TUNE_CACHE", str(p))
    monkeypatch.setattr(tune, "_cache", None)
    assert tune._load() == {}
    tune._cache["k"] = {"tile_n": 256, "flush_chunks": 8, "ms": 1.0}
    tune._save()
    assert json.loads(p.read_text())["k"]["flush_chunks"] == 8


def test_store_choice_round_trip(tmp_path, monkeypatch):
    """Storing a choice takes the cache lock and loads the cache inside it
    (the lock is reentrant), saves, and a fresh load finds the choice."""
    import threading
    p = tmp_path / "tune.json"
    monkeypatch.setenv("HOS_TUNE_CACHE", str(p))
    monkeypatch.setattr(tune, "_cache", None)
    done = []
    t = threading.Thread(target=lambda: (tune.store_choice("k|x", (256, 8, 512), 1.5), done.append(1)))
    t.start()
    t.join(timeout=10)
    assert done, "store_choice did not return"
    monkeypatch.setattr(tune, "_cache", None)
    assert tune._load()["k|x"] == {"tile_n": 256, "flush_chunks": 8, "chunk_len": 512, "ms": 1.5}
