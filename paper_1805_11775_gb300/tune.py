"""Autotuner for the contraction's tile width and flush length.

For a problem shape (op, L, size bucket, series-count bucket, precision) it
times every candidate (tile_n, flush_chunks) through the C ABI with CUDA
events on the current stream, keeps the fastest, and stores it in a JSON
cache (``$HOS_TUNE_CACHE``, default ``~/.cache/hos_gb300/tune.json``) keyed by
the device name and the library version (a rebuilt library with changed
kernels does not reuse old choices).  The public calls consult the cache when
the caller leaves ``tile_n`` / ``flush_chunks`` at 0.  The 3xTF32 path keeps
short flushes only: its FP32 accumulation error grows with the MMA steps one
partial holds.

tile_n is the widest lag tile: 256 gives each 128-row block of the lag square
tiles of 256 columns (and a narrower last one), 128 gives 128-column tiles
throughout (twice the tiles, half the MMA width); the flush length sets how
many 1024-sample chunks a tile accumulates in FP32 before its partial sum goes
to the reduction (more: fewer partials to reduce, longer FP32 sums).
"""
from __future__ import annotations

import json
import math
import os
import threading

_lock = threading.RLock()  # _load() runs inside tune()'s critical section
_cache = None


def cache_path() -> str:
    return os.environ.get("HOS_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "hos_gb300", "tune.json"))


def _load():
    global _cache
    with _lock:
        if _cache is None:
            try:
                with open(cache_path()) as f:
                    _cache = json.load(f)
            except (OSError, ValueError):  # missing or corrupt: start afresh
                _cache = {}
    return _cache


def _save():
    path = cache_path()
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = f"{path}.{os.getpid()}.tmp"
        with open(tmp, "w") as f:
            json.dump(_cache, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass


def _bucket(v: int) -> int:
    return int(math.ceil(math.log2(max(int(v), 1))))


def library_version() -> str:
    from . import _native
    return _native.lib().hos_version().decode()


def key(device_name: str, op: str, L: int, n_total: int, n_series: int, precision: str, version: str = "") -> str:
    return f"{version}|{device_name}|{op}|L{L}|n2^{_bucket(n_total)}|S2^{_bucket(n_series)}|{precision}"


def lookup(op: str, L: int, n_total: int, n_series: int, precision: str):
    """(tile_n, flush_chunks, chunk_len) tuned for this shape on the current device, or None."""
    import torch
    if not torch.cuda.is_available():
        return None
    k = key(torch.cuda.get_device_name(), op, L, n_total, n_series, precision, library_version())
    v = _load().get(k)
    return (int(v["tile_n"]), int(v["flush_chunks"]), int(v.get("chunk_len", 0))) if v else None


def candidates(L: int, precision: str, batched: bool = False):
    """(tile_n, flush_chunks, chunk_len) to time.  Each precision keeps the
    FP32 sum of one partial within the MMA steps its target allows (the
    tensor cores' accumulation error grows with them, about 1e-8 a step):
    FP32-class 384 for one series, 192 for a batch of short series (the
    least well conditioned); split-bf16 3,072."""
    two_l = 2 * L
    tiles = sorted({t for t in (128, 256) if t <= max(32, 1 << (two_l - 1).bit_length())} or {0})
    if precision in ("fp32", "3xtf32"):  # 384 MMA steps per 1024-sample chunk
        knobs = ((1, 512), (2, 256)) if batched else ((1, 1024), (1, 512), (2, 512))
        return [(t, f, c) for t in tiles for (f, c) in knobs]
    if precision in ("fp16", "split_fp16"):  # 192 MMA steps per 1024-sample chunk
        knobs = ((1, 1024), (2, 512)) if batched else ((1, 1024), (2, 1024), (2, 512), (4, 512))
        return [(t, f, c) for t in tiles for (f, c) in knobs]
    # split-bf16 (1e-4 target): flushes up to 16 chunks (3,072 MMA steps, about
    # 3e-5 on the long workload), a third of the target
    return [(t, f, 0) for t in tiles for f in (4, 8, 16)]


def tune(run, op: str, L: int, n_total: int, n_series: int, precision: str, repeats: int = 5, store: bool = True):
    """Time ``run(tile_n, flush_chunks, chunk_len)`` for every candidate; cache the best.

    ``run`` enqueues one call on the current stream.  Returns
    (best (tile_n, flush_chunks, chunk_len), {candidate: ms})."""
    import torch
    times = {}
    for cand in candidates(L, precision, batched=n_series > 1):
        run(*cand)  # first call: workspace growth, kernel attributes
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(repeats):
            run(*cand)
        e1.record()
        torch.cuda.synchronize()
        times[cand] = e0.elapsed_time(e1) / repeats
    best = min(times, key=times.get)
    if store:
        store_choice(key(torch.cuda.get_device_name(), op, L, n_total, n_series, precision, library_version()), best,
                     times[best])
    return best, times


def store_choice(k: str, best, ms: float) -> None:
    """Record a tuned (tile_n, flush_chunks, chunk_len) under key k and save the cache."""
    with _lock:
        cache = _load()
        cache[k] = {"tile_n": best[0], "flush_chunks": best[1], "chunk_len": best[2], "ms": ms}
        _save()


def tune_bispectrum(x, L: int, precision: str = "bf16", repeats: int = 5):
    import paper_1805_11775_gb300 as hos
    return tune(lambda t, f, c: hos.bispectrum(x, L, precision=precision, tile_n=t, flush_chunks=f, chunk_len=c),
                "bispectrum", L, x.numel(), 1, precision, repeats)


def tune_bispectrum_batched(values, offsets, L: int, precision: str = "bf16", repeats: int = 3, max_len=None):
    import paper_1805_11775_gb300 as hos
    S = len(offsets) - 1
    return tune(lambda t, f, c: hos.bispectrum_batched(values, offsets, L, precision=precision, tile_n=t,
                                                       flush_chunks=f, chunk_len=c, max_len=max_len),
                "bispectrum_batched", L, values.numel(), S, precision, repeats)
