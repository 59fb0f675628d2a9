"""Host mirror of the contraction plans (no GPU): hos_check_plan runs, on the
CPU and with the code the kernels use, the series layout, every CTA's walk
over the cost-weighted stream-K split, the slots the partial tiles go to, the
reduction's reading of those slots, the bounds and 16-byte alignment of
every bulk copy, and which computed element gives each lag pair of the square
its value.  A plan passes when every (series, tile, chunk) is run exactly
once, every partial is read exactly once from its own (series, tile), no copy
leaves its series' zero-padded block, and every lag pair has one source."""
import ctypes
import os
import shutil

import numpy as np
import pytest

import hos_synth

pytestmark = pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                                reason="nvcc not available")

OP_BISPECTRUM, OP_TRISPECTRUM, OP_BATCHED = 0, 1, 2


@pytest.fixture(scope="module")
def lib():
    from paper_1805_11775_gb300 import build, _native
    build.build()
    return _native.lib()


def check(lib, op, n, p, ctas, offsets=None):
    msg = ctypes.create_string_buffer(512)
    if offsets is not None:
        offs = np.ascontiguousarray(offsets, dtype=np.int64)
        rc = lib.hos_check_plan(op, int(offs[-1]), offs.size - 1, offs.ctypes.data, ctypes.byref(p), ctas, msg, 512)
    else:
        rc = lib.hos_check_plan(op, n, 1, None, ctypes.byref(p), ctas, msg, 512)
    return rc, msg.value.decode()


def test_workload_plans(lib):
    from paper_1805_11775_gb300 import make_params
    for prec in ("bf16", "fp32", "tf32", "simt", "fp16"):
        ctas = 608 if prec == "simt" else 152
        for n, L in ((2048, 32), (1 << 21, 256), (1 << 18, 128)):
            rc, m = check(lib, OP_BISPECTRUM, n, make_params(L, precision=prec), ctas)
            assert rc == 0, (prec, n, L, m)
    w = hos_synth.workload("batched_4096x_L128")
    for prec in ("bf16", "fp32"):
        rc, m = check(lib, OP_BATCHED, 0, make_params(128, precision=prec), 152, w["offsets"])
        assert rc == 0, (prec, m)
    for prec in ("bf16", "fp32", "tf32"):
        rc, m = check(lib, OP_TRISPECTRUM, 65536, make_params(32, precision=prec), 152)
        assert rc == 0, (prec, m)


def test_tile_schemes(lib, monkeypatch):
    """L = 256.  Six-fold (default for the windowed spectra): rows w1 in
    [0, L), each row block's columns from w1 to w1 + L - 1 in 256-wide tiles,
    four tiles, cost 32 per chunk (L = 128: one tile).  Swap plan
    (HOS_TILE_SCHEME=swap): each row block's 256-wide tiles start at the
    multiple of 256 at or below its diagonal block, six tiles, cost 48.
    Diagonal start: row blocks of 512, 384, 256 and 128 columns, four
    256-wide and two 128-wide tiles, cost 40 (1280 columns / 32)."""
    from paper_1805_11775_gb300 import make_params
    monkeypatch.delenv("HOS_TILE_SCHEME", raising=False)
    rc, m = check(lib, OP_BISPECTRUM, 1 << 21, make_params(256), 152)
    assert rc == 0 and "4 tiles (cost 32 per chunk)" in m, m
    rc, m = check(lib, OP_BISPECTRUM, 1 << 18, make_params(128), 152)
    assert rc == 0 and "1 tiles (cost 8 per chunk)" in m, m
    rc, m = check(lib, OP_BISPECTRUM, 1 << 18, make_params(128, window="parzen_sym"), 152)
    assert rc == 0 and "1 tiles (cost 8 per chunk)" in m, m
    monkeypatch.setenv("HOS_TILE_SCHEME", "swap")
    rc, m = check(lib, OP_BISPECTRUM, 1 << 21, make_params(256), 152)
    assert rc == 0 and "6 tiles (cost 48 per chunk)" in m, m
    monkeypatch.setenv("HOS_TILE_SCHEME", "diagonal")
    rc, m = check(lib, OP_BISPECTRUM, 1 << 21, make_params(256), 152)
    assert rc == 0 and "6 tiles (cost 40 per chunk)" in m, m
    rc, m = check(lib, OP_BISPECTRUM, 1 << 18, make_params(128), 152)
    assert rc == 0 and "2 tiles (cost 12 per chunk)" in m, m


def set_scheme(monkeypatch, scheme):
    if scheme == "six":
        monkeypatch.delenv("HOS_TILE_SCHEME", raising=False)
    else:
        monkeypatch.setenv("HOS_TILE_SCHEME", scheme)


def test_fundamental_set_brute_force():
    """The six-fold plans' reading: with y zero outside the series,
    c3(w1, w2) = c3(w2, w1) = c3(-w1, w2 - w1), and every lag pair of
    (-L, L)^2 has exactly one image in {0 <= w1 < L, w1 <= w2 < w1 + L}.
    Counted here by brute force over the six images, independently of the
    library."""
    for L in (1, 2, 3, 5, 8, 13):
        for w1 in range(-L + 1, L):
            for w2 in range(-L + 1, L):
                imgs = {(w1, w2), (w2, w1), (-w1, w2 - w1), (w2 - w1, -w1), (-w2, w1 - w2), (w1 - w2, -w2)}
                reps = [(a, b) for a, b in imgs if 0 <= a < L and a <= b < a + L]
                assert len(reps) == 1, (L, w1, w2, reps)


@pytest.mark.parametrize("scheme", ["six", "swap", "diagonal"])
def test_random_single_series_plans(lib, monkeypatch, scheme):
    from paper_1805_11775_gb300 import make_params
    set_scheme(monkeypatch, scheme)
    rng = np.random.default_rng(7)
    for _ in range(300):
        L = int(rng.choice([1, 2, 3, 5, 16, 31, 32, 40, 64, 100, 127, 128, 129, 200, 256, 300, 512, 700, 1024]))
        n = int(rng.choice([1, 2, 100, 1023, 1024, 1025, 5000, 40000, 300000]))
        prec = str(rng.choice(["bf16", "fp32", "tf32", "simt", "fp16"]))
        tile = int(rng.choice([0, 0, 32, 64, 128, 256]))
        flush = int(rng.choice([0, 0, 1, 3, 16, 33]))
        win = str(rng.choice(["parzen", "parzen_sym", "rect"]))
        seg = int(rng.choice([0, 0, 0, 700, 4096]))
        ctas = int(rng.choice([1, 2, 7, 148, 152, 608]))
        kc = int(rng.choice([0, 0, 64, 256, 512, 960]))
        p = make_params(L, precision=prec, tile_n=tile, flush_chunks=flush, window=win, segment_len=seg,
                        chunk_len=kc)
        rc, m = check(lib, OP_BISPECTRUM, n, p, ctas)
        assert rc == 0, (L, n, prec, tile, flush, win, seg, ctas, kc, m)


@pytest.mark.parametrize("scheme", ["six", "swap", "diagonal"])
def test_random_batched_plans(lib, monkeypatch, scheme):
    from paper_1805_11775_gb300 import make_params
    set_scheme(monkeypatch, scheme)
    rng = np.random.default_rng(11)
    for _ in range(60):
        S = int(rng.integers(1, 300))
        lens = rng.integers(0, 6000, S)
        lens[rng.random(S) < 0.2] = 0  # empty series
        offs = np.concatenate([[0], np.cumsum(lens)])
        L = int(rng.choice([4, 32, 64, 100, 128, 256]))
        prec = str(rng.choice(["bf16", "fp32", "tf32", "simt", "fp16"]))
        ctas = int(rng.choice([1, 5, 152, 608]))
        p = make_params(L, precision=prec, flush_chunks=int(rng.choice([0, 1, 2, 16])),
                        chunk_len=int(rng.choice([0, 0, 128, 512])))
        rc, m = check(lib, OP_BATCHED, 0, p, ctas, offs)
        assert rc == 0, (S, L, prec, ctas, m)


def test_random_fourth_order_plans(lib):
    from paper_1805_11775_gb300 import make_params
    rng = np.random.default_rng(13)
    for _ in range(80):
        L = int(rng.choice([1, 2, 4, 8, 16, 20, 32, 64]))
        n = int(rng.choice([1, 50, 1000, 4096, 65536, 100001]))
        prec = str(rng.choice(["bf16", "fp32", "tf32", "fp16"]))
        seg = int(rng.choice([0, 0, 1500]))
        ctas = int(rng.choice([1, 3, 152]))
        kc = int(rng.choice([0, 0, 64, 256]))
        rc, m = check(lib, OP_TRISPECTRUM, n, make_params(L, precision=prec, segment_len=seg, chunk_len=kc), ctas)
        assert rc == 0, (L, n, prec, seg, ctas, m)
