"""Seeded synthetic inputs shaped like the paper's motivating workloads.

This module holds input generators only -- none of the estimator's
arithmetic -- so that the oracle and the CUDA path can share them.

The paper generates its series after Ravishanker's and Jones' guidelines
(Experimental Results, Test Platform); those generators are not available,
so these stand in: centred i.i.d. Exp(1) noise, AR(2) and MA(3) filters of
that noise, and Student-t returns of intraday length (Introduction: series of
up to 20,000 samples per trading day).  All draws use numpy's PCG64.
"""
from __future__ import annotations

import numpy as np

AR2 = (0.5, -0.3)                 # x_t = 0.5 x_{t-1} - 0.3 x_{t-2} + e_t
MA3 = (1.0, 0.6, -0.4, 0.2)       # x_t = e_t + 0.6 e_{t-1} - 0.4 e_{t-2} + 0.2 e_{t-3}
BURN_IN = 4096


def exp_noise(n: int, seed: int) -> np.ndarray:
    """Centred i.i.d. Exp(1) noise: mean 0, variance 1, third cumulant 2, fourth 6."""
    rng = np.random.default_rng(seed)
    return rng.exponential(1.0, int(n)) - 1.0


def ar2(n: int, seed: int, a=AR2, burn_in: int = BURN_IN) -> np.ndarray:
    """AR(2) driven by centred Exp(1) noise; the first ``burn_in`` samples are dropped."""
    e = exp_noise(int(n) + burn_in, seed)
    x = np.empty_like(e)
    x1 = x2 = 0.0
    a1, a2 = a
    # plain recursion; scipy.signal.lfilter gives the same values faster
    try:
        from scipy.signal import lfilter
        x = lfilter([1.0], [1.0, -a1, -a2], e)
    except Exception:  # pragma: no cover - scipy missing
        for t in range(e.size):
            v = a1 * x1 + a2 * x2 + e[t]
            x[t] = v
            x2, x1 = x1, v
    return np.ascontiguousarray(x[burn_in:])


def ma(n: int, seed: int, h=MA3) -> np.ndarray:
    """Moving average of centred Exp(1) noise with taps h (no burn-in needed)."""
    h = np.asarray(h, dtype=np.float64)
    e = exp_noise(int(n) + h.size - 1, seed)
    return np.ascontiguousarray(np.convolve(e, h, mode="valid"))


def student_t_returns(lengths, seed: int, df: float = 4.0, std: float = 1e-3):
    """Concatenated i.i.d. Student-t(df) series scaled to standard deviation ``std``.

    Returns (values float64, offsets int64 of length S+1)."""
    rng = np.random.default_rng(seed)
    lengths = np.asarray(lengths, dtype=np.int64)
    total = int(lengths.sum())
    scale = std / np.sqrt(df / (df - 2.0))
    vals = rng.standard_t(df, total) * scale
    offsets = np.zeros(lengths.size + 1, dtype=np.int64)
    np.cumsum(lengths, out=offsets[1:])
    return vals, offsets


def intraday_lengths(S: int, seed: int, lo: int = 2000, hi: int = 20000) -> np.ndarray:
    """S series lengths uniform on the integers [lo, hi]."""
    rng = np.random.default_rng(seed)
    return rng.integers(lo, hi + 1, size=int(S), dtype=np.int64)


# ---- the five workloads ------------------------------------------------
# (n, L, grid, dtype, generator) -- seeds are 1000 + workload number.

def workload(name: str, small: bool = False):
    """Inputs of a named workload.  ``small`` shrinks the series (not L)."""
    if name == "bispectrum_n2048_L32":
        return {"x": exp_noise(2048, 1001), "L": 32, "N": 64}
    if name == "long_bispectrum_n2M_L256":
        n = 1 << 21 if not small else 1 << 14
        return {"x": ar2(n, 1002), "L": 256, "N": 512}
    if name == "trispectrum_n65536_L32":
        n = 65536 if not small else 4096
        return {"x": ma(n, 1003).astype(np.float32), "L": 32, "N": 64}
    if name == "batched_4096x_L128":
        S = 4096 if not small else 16
        lens = intraday_lengths(S, 1004)
        vals, offs = student_t_returns(lens, 1004)
        return {"x": vals, "offsets": offs, "L": 128, "N": 256}
    if name == "differentiable_n262144_L128":
        n = 1 << 18 if not small else 4096
        return {"x": ar2(n, 1005).astype(np.float32), "target_x": ar2(n, 2005).astype(np.float32),
                "L": 128, "N": 256}
    if name == "differentiable_trispectrum_n65536_L32":
        n = 65536 if not small else 4096
        return {"x": ma(n, 1006).astype(np.float32), "target_x": ma(n, 2006).astype(np.float32), "L": 32, "N": 64}
    raise KeyError(name)
