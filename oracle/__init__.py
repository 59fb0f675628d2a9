"""FP64 CPU oracle for the indirect bispectrum / trispectrum estimator.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``.  The library path never imports it.

The arithmetic lives in ``hos_oracle.c`` (plain loops, FP64); this module
compiles it with gcc on first use and marshals numpy arrays to it.  Lag
arrays cover ``[-L, L]`` on every axis (index ``w + L``); spectra are complex
``[k1][k2]`` (or ``[k1][k2][k3]``) on the unshifted grid ``k = 0..N-1``.

Window kinds: 0 = Parzen (separable), 1 = Parzen with the extra factor
d(w1 - w2), 2 = rectangular over ``|w| <= L - 1``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hos_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libhos_oracle.so")
_lock = threading.Lock()
_lib = None

WIN_PARZEN, WIN_PARZEN_SYM, WIN_RECT = 0, 1, 2

_D = ctypes.POINTER(ctypes.c_double)
_I64 = ctypes.c_int64


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP) into oracle/_build/."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-fno-fast-math", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.hos_oracle_parzen.restype = ctypes.c_double
            lib.hos_oracle_parzen.argtypes = [_I64, _I64]
            lib.hos_oracle_window2.restype = ctypes.c_double
            lib.hos_oracle_window2.argtypes = [_I64, _I64, _I64, ctypes.c_int]
            lib.hos_oracle_window3.restype = ctypes.c_double
            lib.hos_oracle_window3.argtypes = [_I64, _I64, _I64, _I64, ctypes.c_int]
            lib.hos_oracle_demean.argtypes = [_D, _I64, _I64, ctypes.c_int, _D]
            lib.hos_oracle_c2.argtypes = [_D, _I64, _I64, _D]
            lib.hos_oracle_c3.argtypes = [_D, _I64, _I64, _D]
            lib.hos_oracle_c3_at.argtypes = [_D, _I64, ctypes.POINTER(_I64), _I64, _D]
            lib.hos_oracle_c3_rows.argtypes = [_D, _I64, _I64, _I64, _I64, _D]
            lib.hos_oracle_m4.argtypes = [_D, _I64, _I64, _D]
            lib.hos_oracle_c4.argtypes = [_D, _I64, _I64, _D]
            lib.hos_oracle_dft2.argtypes = [_D, _I64, _I64, ctypes.c_double, ctypes.c_double, _D]
            lib.hos_oracle_dft3.argtypes = [_D, _I64, _I64, ctypes.c_double, ctypes.c_double, _D]
            lib.hos_oracle_bispectrum.argtypes = [_D, _I64, _I64, _I64, ctypes.c_int, ctypes.c_int, _I64, _D]
            lib.hos_oracle_trispectrum.argtypes = [_D, _I64, _I64, _I64, ctypes.c_int, ctypes.c_int, _I64, _D]
            lib.hos_oracle_bispectrum_grad.argtypes = [_D, _I64, _I64, _I64, ctypes.c_int, ctypes.c_int, _D, _D]
            lib.hos_oracle_grad_lag.argtypes = [_D, _I64, _I64, ctypes.c_int, _D]
            lib.hos_oracle_dy_at.argtypes = [_D, _I64, _I64, _D, ctypes.POINTER(_I64), _I64, _D]
            lib.hos_oracle_bispectrum_direct.argtypes = [_D, _I64, _I64, _I64, _I64, ctypes.c_int, _D]
            lib.hos_oracle_bispectrum_overlap.argtypes = [_D, _I64, _I64, _I64, ctypes.c_int, ctypes.c_int, _I64,
                                                          _I64, _D]
            lib.hos_oracle_trispectrum_overlap.argtypes = [_D, _I64, _I64, _I64, ctypes.c_int, ctypes.c_int, _I64,
                                                           _I64, _D]
            lib.hos_oracle_cumulant_overlap.argtypes = [_D, _I64, _I64, ctypes.c_int, ctypes.c_int, _I64, _I64, _D]
            lib.hos_oracle_trispectrum_grad.argtypes = [_D, _I64, _I64, _I64, ctypes.c_int, ctypes.c_int, _D, _D]
            lib.hos_oracle_grad_lag4.argtypes = [_D, _I64, _I64, ctypes.c_int, _D]
            lib.hos_oracle_grad_c2.argtypes = [_D, _D, _I64, _D]
            lib.hos_oracle_dy4_at.argtypes = [_D, _I64, _I64, _D, _D, ctypes.POINTER(_I64), _I64, _D]
            _lib = lib
    return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _p(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _complex(buf: np.ndarray, shape) -> np.ndarray:
    return buf.view(np.complex128).reshape(shape)


def parzen(w: int, L: int) -> float:
    return _load().hos_oracle_parzen(int(w), int(L))


def window2(w1: int, w2: int, L: int, kind: int = WIN_PARZEN) -> float:
    return _load().hos_oracle_window2(int(w1), int(w2), int(L), int(kind))


def window3(w1: int, w2: int, w3: int, L: int, kind: int = WIN_PARZEN) -> float:
    return _load().hos_oracle_window3(int(w1), int(w2), int(w3), int(L), int(kind))


def demean(x, segment_len: int = 0, remove_mean: bool = True) -> np.ndarray:
    x = _f64(x)
    y = np.empty_like(x)
    _load().hos_oracle_demean(_p(x), x.size, int(segment_len), int(bool(remove_mean)), _p(y))
    return y


def c2(y, T: int) -> np.ndarray:
    """c2[t + T], t in [-T, T]."""
    y = _f64(y)
    out = np.empty(2 * T + 1)
    _load().hos_oracle_c2(_p(y), y.size, int(T), _p(out))
    return out


def c3(y, L: int) -> np.ndarray:
    """c3[w1 + L, w2 + L] over [-L, L]^2 (y already mean-removed)."""
    y = _f64(y)
    W = 2 * L + 1
    out = np.empty(W * W)
    _load().hos_oracle_c3(_p(y), y.size, int(L), _p(out))
    return out.reshape(W, W)


def c3_at(y, lags) -> np.ndarray:
    """c3 at explicit lag pairs, lags shape (P, 2)."""
    y = _f64(y)
    lg = np.ascontiguousarray(np.asarray(lags, dtype=np.int64).reshape(-1, 2))
    out = np.empty(lg.shape[0])
    _load().hos_oracle_c3_at(_p(y), y.size, lg.ctypes.data_as(ctypes.POINTER(_I64)), lg.shape[0], _p(out))
    return out


def c3_rows(y, L: int, w1_lo: int, w1_hi: int) -> np.ndarray:
    y = _f64(y)
    W = 2 * L + 1
    out = np.empty((w1_hi - w1_lo + 1) * W)
    _load().hos_oracle_c3_rows(_p(y), y.size, int(L), int(w1_lo), int(w1_hi), _p(out))
    return out.reshape(w1_hi - w1_lo + 1, W)


def m4(y, L: int) -> np.ndarray:
    y = _f64(y)
    W = 2 * L + 1
    out = np.empty(W ** 3)
    _load().hos_oracle_m4(_p(y), y.size, int(L), _p(out))
    return out.reshape(W, W, W)


def c4(y, L: int) -> np.ndarray:
    y = _f64(y)
    W = 2 * L + 1
    out = np.empty(W ** 3)
    _load().hos_oracle_c4(_p(y), y.size, int(L), _p(out))
    return out.reshape(W, W, W)


def dft2(f, L: int, N: int, sign: float = -1.0, scale: float = 1.0) -> np.ndarray:
    f = _f64(f)
    out = np.empty(N * N * 2)
    _load().hos_oracle_dft2(_p(f), int(L), int(N), float(sign), float(scale), _p(out))
    return _complex(out, (N, N))


def dft3(f, L: int, N: int, sign: float = -1.0, scale: float = 1.0) -> np.ndarray:
    f = _f64(f)
    out = np.empty(N ** 3 * 2)
    _load().hos_oracle_dft3(_p(f), int(L), int(N), float(sign), float(scale), _p(out))
    return _complex(out, (N, N, N))


def bispectrum(x, L: int, N: int = 0, window: int = WIN_PARZEN, remove_mean: bool = True,
               segment_len: int = 0) -> np.ndarray:
    x = _f64(x)
    N = N or 2 * L
    out = np.empty(N * N * 2)
    _load().hos_oracle_bispectrum(_p(x), x.size, int(L), int(N), int(window), int(bool(remove_mean)),
                                  int(segment_len), _p(out))
    return _complex(out, (N, N))


def trispectrum(x, L: int, N: int = 0, window: int = WIN_PARZEN, remove_mean: bool = True,
                segment_len: int = 0) -> np.ndarray:
    x = _f64(x)
    N = N or 2 * L
    out = np.empty(N ** 3 * 2)
    _load().hos_oracle_trispectrum(_p(x), x.size, int(L), int(N), int(window), int(bool(remove_mean)),
                                   int(segment_len), _p(out))
    return _complex(out, (N, N, N))


def bispectrum_overlap(x, L: int, N: int = 0, window: int = WIN_PARZEN, remove_mean: bool = True,
                       segment_len: int = 0, overlap: int = 0) -> np.ndarray:
    """Parts of segment_len samples every segment_len - overlap samples (trailing
    samples past the last whole part unused), each demeaned, c3 averaged."""
    x = _f64(x)
    N = N or 2 * L
    out = np.empty(N * N * 2)
    _load().hos_oracle_bispectrum_overlap(_p(x), x.size, int(L), int(N), int(window), int(bool(remove_mean)),
                                          int(segment_len), int(overlap), _p(out))
    return _complex(out, (N, N))


def trispectrum_overlap(x, L: int, N: int = 0, window: int = WIN_PARZEN, remove_mean: bool = True,
                        segment_len: int = 0, overlap: int = 0) -> np.ndarray:
    x = _f64(x)
    N = N or 2 * L
    out = np.empty(N ** 3 * 2)
    _load().hos_oracle_trispectrum_overlap(_p(x), x.size, int(L), int(N), int(window), int(bool(remove_mean)),
                                           int(segment_len), int(overlap), _p(out))
    return _complex(out, (N, N, N))


def cumulant_overlap(x, L: int, order: int, remove_mean: bool = True, segment_len: int = 0,
                     overlap: int = 0) -> np.ndarray:
    """The parts' average c3 over [-L, L]^2 (order 3) or c4 over [-L, L]^3 (order 4)."""
    x = _f64(x)
    W = 2 * L + 1
    out = np.empty(W ** (order - 1))
    _load().hos_oracle_cumulant_overlap(_p(x), x.size, int(L), int(order), int(bool(remove_mean)),
                                        int(segment_len), int(overlap), _p(out))
    return out.reshape((W,) * (order - 1))


def bispectrum_grad(x, L: int, G, N: int = 0, window: int = WIN_PARZEN, remove_mean: bool = True) -> np.ndarray:
    """dl/dx for a loss with dl/dRe B + i dl/dIm B = G (complex N x N)."""
    x = _f64(x)
    N = N or 2 * L
    g = np.ascontiguousarray(np.asarray(G, dtype=np.complex128).reshape(N, N)).view(np.float64).ravel()
    out = np.empty_like(x)
    _load().hos_oracle_bispectrum_grad(_p(x), x.size, int(L), int(N), int(window), int(bool(remove_mean)),
                                       _p(np.ascontiguousarray(g)), _p(out))
    return out


def grad_lag(G, L: int, N: int, window: int = WIN_PARZEN) -> np.ndarray:
    """dl/dc3 over [-L, L]^2 for dl/dRe B + i dl/dIm B = G (complex N x N)."""
    g = np.ascontiguousarray(np.asarray(G, dtype=np.complex128).reshape(N, N)).view(np.float64).ravel()
    W = 2 * L + 1
    out = np.empty(W * W)
    _load().hos_oracle_grad_lag(_p(np.ascontiguousarray(g)), int(L), int(N), int(window), _p(out))
    return out.reshape(W, W)


def dy_at(y, L: int, dc, js) -> np.ndarray:
    """Gradient with respect to the mean-removed samples y at indices js."""
    y = _f64(y)
    dcf = _f64(dc)
    jj = np.ascontiguousarray(np.asarray(js, dtype=np.int64))
    out = np.empty(jj.size)
    _load().hos_oracle_dy_at(_p(y), y.size, int(L), _p(dcf), jj.ctypes.data_as(ctypes.POINTER(_I64)), jj.size,
                             _p(out))
    return out


def trispectrum_grad(x, L: int, G, N: int = 0, window: int = WIN_PARZEN, remove_mean: bool = True) -> np.ndarray:
    """dl/dx for a loss with dl/dRe T + i dl/dIm T = G (complex N x N x N)."""
    x = _f64(x)
    N = N or 2 * L
    g = np.ascontiguousarray(np.asarray(G, dtype=np.complex128).reshape(N, N, N)).view(np.float64).ravel()
    out = np.empty_like(x)
    _load().hos_oracle_trispectrum_grad(_p(x), x.size, int(L), int(N), int(window), int(bool(remove_mean)),
                                        _p(np.ascontiguousarray(g)), _p(out))
    return out


def grad_lag4(G, L: int, N: int, window: int = WIN_PARZEN) -> np.ndarray:
    """dl/dc4 over [-L, L]^3 for dl/dRe T + i dl/dIm T = G (complex N^3)."""
    g = np.ascontiguousarray(np.asarray(G, dtype=np.complex128).reshape(N, N, N)).view(np.float64).ravel()
    W = 2 * L + 1
    out = np.empty(W ** 3)
    _load().hos_oracle_grad_lag4(_p(np.ascontiguousarray(g)), int(L), int(N), int(window), _p(out))
    return out.reshape(W, W, W)


def grad_c2(dc4, c2v, L: int) -> np.ndarray:
    """dl/dc2(t), t in [-2L, 2L], from dl/dc4 over [-L, L]^3 and c2 over [-2L, 2L]."""
    d = _f64(dc4)
    c = _f64(c2v)
    out = np.empty(4 * L + 1)
    _load().hos_oracle_grad_c2(_p(d), _p(c), int(L), _p(out))
    return out


def dy4_at(y, L: int, dc4, dc2, js) -> np.ndarray:
    """Trispectrum gradient with respect to the mean-removed samples y at indices js."""
    y = _f64(y)
    d4 = _f64(dc4)
    d2 = _f64(dc2)
    jj = np.ascontiguousarray(np.asarray(js, dtype=np.int64))
    out = np.empty(jj.size)
    _load().hos_oracle_dy4_at(_p(y), y.size, int(L), _p(d4), _p(d2), jj.ctypes.data_as(ctypes.POINTER(_I64)),
                              jj.size, _p(out))
    return out


def bispectrum_direct(x, M: int, M3: int, remove_mean: bool = True, overlap: int = 0) -> np.ndarray:
    """Algorithm DBS: parts of M samples (every M - overlap samples), raw (1/M)
    F(k1)F(k2)F*(k1+k2), M3 x M3 box smoothing (indices mod M), average over
    parts.  (M, M) complex, [k1][k2]."""
    x = _f64(x)
    out = np.empty(M * M * 2)
    _load().hos_oracle_bispectrum_direct(_p(x), x.size, int(M), int(M3), int(overlap), int(bool(remove_mean)),
                                         _p(out))
    return _complex(out, (M, M))


def threads() -> int:
    """OpenMP threads the oracle uses (OMP_NUM_THREADS, else all host cores)."""
    v = os.environ.get("OMP_NUM_THREADS")
    return int(v) if v and v.isdigit() else (os.cpu_count() or 1)
