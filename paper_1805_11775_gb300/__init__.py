"""GB300 (sm_103a) higher-order spectra: the smoothed sample bispectrum and
trispectrum of a series, computed the indirect way (sample cumulant, lag
window, Fourier transform), after Mamun et al., "Efficient Sequential and
Parallel Algorithms for Estimating Higher Order Spectra" (Problem Statement;
Algorithm DBS steps 1, 2 and 6 for the parts and their averaging).

PyTorch supplies device memory and the current stream; the computation runs
in ``libhos.so`` (hand-written CUDA for sm_103a) through its C ABI.

    >>> import paper_1805_11775_gb300 as hos
    >>> B = hos.bispectrum(x_cuda, L=256, precision="bf16")      # (512, 512) complex64
"""
from __future__ import annotations

import ctypes
import threading

import numpy as np

from . import _native
from ._native import HosError, HosParams

__all__ = ["bispectrum", "bispectrum_batched", "trispectrum", "trispectrum_batched", "cumulant3", "cumulant4",
           "bispectrum_backward", "trispectrum_backward", "BispectrumFn", "TrispectrumFn", "bispectrum_ad",
           "trispectrum_ad", "bispectrum_direct", "series_sum", "cumulant3_slice", "bispectrum_from_cumulant",
           "bispectrum_sharded", "moments4_slice", "trispectrum_from_moments", "trispectrum_sharded", "Workspace", "workspace_size", "device_status", "reset_device_status",
           "selftest_timeout", "set_profiling", "stage_times", "launch_count", "last_contraction", "last_plan", "HosError",
           "PRECISIONS", "WINDOWS"]

PRECISIONS = {"fp32": 0, "3xtf32": 0, "bf16": 1, "split_bf16": 1, "tf32": 2, "simt": 3, "simt_fp32": 3, "fp16": 4,
              "split_fp16": 4}
WINDOWS = {"parzen": 0, "parzen_sym": 1, "rect": 2}


def _torch():
    import torch
    return torch


def make_params(L, nfft=0, precision="bf16", window="parzen", remove_mean=True, segment_len=0, tile_n=0,
                flush_chunks=0, segment_overlap=0, chunk_len=0) -> HosParams:
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    win = WINDOWS[window] if isinstance(window, str) else int(window)
    return HosParams(int(L), int(nfft or 0), prec, win, int(bool(remove_mean)), int(segment_len or 0),
                     int(tile_n or 0), int(flush_chunks or 0), int(segment_overlap or 0), int(chunk_len or 0))


def _tuned(op, L, n_total, n_series, precision, tile_n, flush_chunks, chunk_len=0):
    """The caller's knobs, else the autotuner's cached choice, else automatic:
    (tile_n, flush_chunks, chunk_len)."""
    if tile_n or flush_chunks or chunk_len:
        return tile_n, flush_chunks, chunk_len
    from . import tune
    r = tune.lookup(op, L, n_total, n_series, precision if isinstance(precision, str) else str(precision))
    return r if r else (0, 0, 0)


def workspace_size(op: int, n_total: int, n_series: int, max_len: int, params: HosParams) -> int:
    out = ctypes.c_size_t(0)
    _native.check(_native.lib().hos_workspace_size(op, int(n_total), int(n_series), int(max_len),
                                                   ctypes.byref(params), ctypes.byref(out)), "hos_workspace_size")
    return int(out.value)


class Workspace:
    """A growable device scratch buffer (a torch uint8 tensor) for the library."""

    def __init__(self, device=None):
        self.device = device
        self.buf = None

    def get(self, nbytes: int):
        torch = _torch()
        nbytes = max(int(nbytes), 256)
        if self.buf is None or self.buf.numel() < nbytes:
            dev = self.device if self.device is not None else torch.device("cuda", torch.cuda.current_device())
            self.buf = None
            self.buf = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
        return self.buf

    def ptr(self):
        p = self.buf.data_ptr()
        return p + ((-p) % 256)

    def nbytes(self):
        return self.buf.numel() - ((-self.buf.data_ptr()) % 256)


_default_ws = {}
_ws_lock = threading.Lock()


def _workspace(ws, device):
    if ws is not None:
        return ws
    with _ws_lock:
        key = (device.type, device.index)
        if key not in _default_ws:
            _default_ws[key] = Workspace(device)
        return _default_ws[key]


def _stream(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _prepare(x):
    """Return (device tensor, was_host).  Host input is copied to the GPU."""
    torch = _torch()
    if isinstance(x, np.ndarray):
        x = torch.from_numpy(np.ascontiguousarray(x))
    if x.dtype not in (torch.float32, torch.float64):
        raise TypeError("x must be float32 or float64")
    host = x.device.type != "cuda"
    if host:
        x = x.to("cuda", non_blocking=True)
    return x.contiguous(), host


def _out_buffers(out, shape, device):
    """(device result buffer, host tensor to fill or None).  A host ``out``
    (pinned for a fast copy) receives the result after the device computes it."""
    torch = _torch()
    if out is not None and out.device.type == "cuda":
        return out, None
    dev = torch.empty(shape, dtype=torch.complex64, device=device)
    return dev, out


def _finish(dev, host_out, host_input):
    if host_out is not None:
        host_out.copy_(dev)
        return host_out
    return dev.cpu() if host_input else dev


def _dtype_code(x):
    torch = _torch()
    return _native.F64 if x.dtype == torch.float64 else _native.F32


def bispectrum(x, L, nfft=0, precision="bf16", window="parzen", remove_mean=True, segment_len=0, tile_n=0,
               flush_chunks=0, out=None, workspace=None, stream=None, segment_overlap=0, chunk_len=0):
    """Smoothed sample bispectrum B[k1, k2] (complex64, nfft x nfft, default nfft = 2L).

    ``precision``: "bf16" (split-bf16 tensor cores), "fp32" (3xTF32 tensor
    cores), "fp16" (split FP16 of the series scaled by a power of two:
    FP32-class at the split-bf16 rate), "tf32" (one plain TF32 product, no
    accuracy target) or "simt" (FP32 CUDA cores).  Host input returns a host result; a
    host ``out`` (pinned for speed) receives the result.  ``segment_len`` > 0
    averages parts of that many samples; ``segment_overlap`` makes them
    overlap (parts start every segment_len - segment_overlap samples)."""
    torch = _torch()
    xd, host = _prepare(x)
    tile_n, flush_chunks, chunk_len = _tuned("bispectrum", L, xd.numel(), 1, precision, tile_n, flush_chunks,
                                             chunk_len)
    p = make_params(L, nfft, precision, window, remove_mean, segment_len, tile_n, flush_chunks, segment_overlap,
                    chunk_len)
    N = p.nfft or 2 * p.L
    dev, host_out = _out_buffers(out, (N, N), xd.device)
    ws = _workspace(workspace, xd.device)
    ws.get(workspace_size(_native.OP_BISPECTRUM, xd.numel(), 1, xd.numel(), p))
    _native.check(_native.lib().hos_bispectrum(xd.data_ptr(), _dtype_code(xd), xd.numel(), ctypes.byref(p),
                                               dev.data_ptr(), ws.ptr(), ws.nbytes(), _stream(stream)),
                  "hos_bispectrum")
    return _finish(dev, host_out, host)


def _batched_pipelined(values, offs, L, p, out, workspace, groups):
    """Host input and pinned host output: the series in `groups` contiguous
    groups of about equal sample counts, each group's input copied and
    computed on the current stream while the previous group's spectra are
    copied to the host on a second stream (two device output buffers)."""
    torch = _torch()
    from .shard import series_shard
    N = p.nfft or 2 * p.L
    cuts = [series_shard(offs, g, groups) for g in range(groups)]
    cuts = [(a, b) for a, b in cuts if b > a]
    smax = max(b - a for a, b in cuts)
    lmax = int(np.max(offs[1:] - offs[:-1])) if offs.size > 1 else 0
    comp = torch.cuda.current_stream()
    copy = torch.cuda.Stream()
    bufs = [torch.empty((smax, N, N), dtype=torch.complex64, device="cuda") for _ in range(2)]
    ws = _workspace(workspace, torch.device("cuda"))
    ws.get(max(workspace_size(_native.OP_BISPECTRUM_BATCHED, int(offs[b] - offs[a]), b - a, lmax, p)
               for a, b in cuts))
    freed = [None, None]
    for g, (a, b) in enumerate(cuts):
        buf = bufs[g % 2]
        if freed[g % 2] is not None:
            comp.wait_event(freed[g % 2])  # the copy out of this buffer is done
        vd = values[int(offs[a]):int(offs[b])].to("cuda", non_blocking=True)
        od = torch.from_numpy(offs[a:b + 1] - offs[a]).to("cuda", non_blocking=True)
        _native.check(_native.lib().hos_bispectrum_batched(vd.data_ptr(), _dtype_code(vd), od.data_ptr(), b - a,
                                                           vd.numel(), lmax, ctypes.byref(p), buf.data_ptr(),
                                                           ws.ptr(), ws.nbytes(), ctypes.c_void_p(comp.cuda_stream)),
                      "hos_bispectrum_batched")
        done = torch.cuda.Event()
        done.record(comp)
        copy.wait_event(done)
        with torch.cuda.stream(copy):
            out[a:b].copy_(buf[:b - a], non_blocking=True)
        freed[g % 2] = torch.cuda.Event()
        freed[g % 2].record(copy)
        vd.record_stream(comp)
    copy.synchronize()
    comp.synchronize()
    return out


def bispectrum_batched(values, offsets, L, nfft=0, precision="bf16", window="parzen", remove_mean=True, tile_n=0,
                       flush_chunks=0, out=None, workspace=None, stream=None, max_len=None, pipeline=4,
                       chunk_len=0):
    """Bispectra of S series concatenated in ``values`` with ``offsets`` (S+1).

    Returns (S, nfft, nfft) complex64.  With host ``values`` and a pinned host
    ``out``, the series go in ``pipeline`` groups whose transfers overlap the
    next group's compute (``pipeline=1``: one call)."""
    torch = _torch()
    if (pipeline > 1 and out is not None and out.device.type == "cpu" and out.is_pinned()
            and not (isinstance(values, torch.Tensor) and values.device.type == "cuda") and stream is None):
        offs_h = np.ascontiguousarray(np.asarray(offsets.cpu() if isinstance(offsets, torch.Tensor) else offsets,
                                                 dtype=np.int64))
        vals_h = values if isinstance(values, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(values))
        if vals_h.dtype not in (torch.float32, torch.float64):
            raise TypeError("values must be float32 or float64")
        S = offs_h.size - 1
        if S >= 2 * pipeline:
            tile_n, flush_chunks, chunk_len = _tuned("bispectrum_batched", L, vals_h.numel(), S, precision, tile_n,
                                                     flush_chunks, chunk_len)
            p = make_params(L, nfft, precision, window, remove_mean, 0, tile_n, flush_chunks, 0, chunk_len)
            return _batched_pipelined(vals_h, offs_h, L, p, out, workspace, pipeline)
    vd, host = _prepare(values)
    offs = torch.as_tensor(offsets, dtype=torch.int64)
    if max_len is None:
        oh = offs.cpu() if offs.device.type == "cuda" else offs
        max_len = int((oh[1:] - oh[:-1]).max().item()) if oh.numel() > 1 else 0
    od = offs.to(vd.device, non_blocking=True).contiguous()
    S = od.numel() - 1
    tile_n, flush_chunks, chunk_len = _tuned("bispectrum_batched", L, vd.numel(), S, precision, tile_n, flush_chunks,
                                             chunk_len)
    p = make_params(L, nfft, precision, window, remove_mean, 0, tile_n, flush_chunks, 0, chunk_len)
    N = p.nfft or 2 * p.L
    dev, host_out = _out_buffers(out, (S, N, N), vd.device)
    ws = _workspace(workspace, vd.device)
    ws.get(workspace_size(_native.OP_BISPECTRUM_BATCHED, vd.numel(), S, max_len, p))
    _native.check(_native.lib().hos_bispectrum_batched(vd.data_ptr(), _dtype_code(vd), od.data_ptr(), S, vd.numel(),
                                                       int(max_len), ctypes.byref(p), dev.data_ptr(), ws.ptr(),
                                                       ws.nbytes(), _stream(stream)), "hos_bispectrum_batched")
    return _finish(dev, host_out, host)


def cumulant3(x, L, precision="bf16", remove_mean=True, segment_len=0, tile_n=0, flush_chunks=0, workspace=None,
              stream=None, segment_overlap=0, chunk_len=0):
    """Unwindowed sample c3 over [-L, L-1]^2 (float64, (2L, 2L), index w + L)."""
    torch = _torch()
    xd, host = _prepare(x)
    p = make_params(L, 0, precision, "parzen", remove_mean, segment_len, tile_n, flush_chunks, segment_overlap,
                    chunk_len)
    out = torch.empty((2 * p.L, 2 * p.L), dtype=torch.float64, device=xd.device)
    ws = _workspace(workspace, xd.device)
    ws.get(workspace_size(_native.OP_CUMULANT3, xd.numel(), 1, xd.numel(), p))
    _native.check(_native.lib().hos_cumulant3(xd.data_ptr(), _dtype_code(xd), xd.numel(), ctypes.byref(p),
                                              out.data_ptr(), ws.ptr(), ws.nbytes(), _stream(stream)),
                  "hos_cumulant3")
    return out.cpu() if host else out


def trispectrum(x, L, nfft=0, precision="bf16", window="parzen", remove_mean=True, segment_len=0, flush_chunks=0,
                out=None, workspace=None, stream=None, segment_overlap=0, chunk_len=0):
    """Smoothed sample trispectrum T[k1, k2, k3] (complex64, nfft^3)."""
    torch = _torch()
    xd, host = _prepare(x)
    p = make_params(L, nfft, precision, window, remove_mean, segment_len, 0, flush_chunks, segment_overlap,
                    chunk_len)
    N = p.nfft or 2 * p.L
    dev, host_out = _out_buffers(out, (N, N, N), xd.device)
    ws = _workspace(workspace, xd.device)
    ws.get(workspace_size(_native.OP_TRISPECTRUM, xd.numel(), 1, xd.numel(), p))
    _native.check(_native.lib().hos_trispectrum(xd.data_ptr(), _dtype_code(xd), xd.numel(), ctypes.byref(p),
                                                dev.data_ptr(), ws.ptr(), ws.nbytes(), _stream(stream)),
                  "hos_trispectrum")
    return _finish(dev, host_out, host)


def trispectrum_batched(values, offsets, L, nfft=0, precision="bf16", window="parzen", remove_mean=True,
                        flush_chunks=0, out=None, workspace=None, stream=None, max_len=None):
    """Trispectra of S series concatenated in ``values`` with ``offsets`` (S+1):
    (S, nfft, nfft, nfft) complex64.  Tensor-core precisions ("bf16", "fp32")."""
    torch = _torch()
    vd, host = _prepare(values)
    offs = torch.as_tensor(offsets, dtype=torch.int64)
    if max_len is None:
        oh = offs.cpu() if offs.device.type == "cuda" else offs
        max_len = int((oh[1:] - oh[:-1]).max().item()) if oh.numel() > 1 else 0
    od = offs.to(vd.device, non_blocking=True).contiguous()
    S = od.numel() - 1
    p = make_params(L, nfft, precision, window, remove_mean, 0, 0, flush_chunks)
    N = p.nfft or 2 * p.L
    dev, host_out = _out_buffers(out, (S, N, N, N), vd.device)
    ws = _workspace(workspace, vd.device)
    ws.get(workspace_size(_native.OP_TRISPECTRUM_BATCHED, vd.numel(), S, max_len, p))
    _native.check(_native.lib().hos_trispectrum_batched(vd.data_ptr(), _dtype_code(vd), od.data_ptr(), S, vd.numel(),
                                                        int(max_len), ctypes.byref(p), dev.data_ptr(), ws.ptr(),
                                                        ws.nbytes(), _stream(stream)), "hos_trispectrum_batched")
    return _finish(dev, host_out, host)


def cumulant4(x, L, precision="bf16", remove_mean=True, segment_len=0, flush_chunks=0, workspace=None, stream=None,
              segment_overlap=0):
    """Unwindowed sample c4 over [-L, L-1]^3 (float64, (2L, 2L, 2L))."""
    torch = _torch()
    xd, host = _prepare(x)
    p = make_params(L, 0, precision, "parzen", remove_mean, segment_len, 0, flush_chunks, segment_overlap)
    out = torch.empty((2 * p.L,) * 3, dtype=torch.float64, device=xd.device)
    ws = _workspace(workspace, xd.device)
    ws.get(workspace_size(_native.OP_CUMULANT4, xd.numel(), 1, xd.numel(), p))
    _native.check(_native.lib().hos_cumulant4(xd.data_ptr(), _dtype_code(xd), xd.numel(), ctypes.byref(p),
                                              out.data_ptr(), ws.ptr(), ws.nbytes(), _stream(stream)),
                  "hos_cumulant4")
    return out.cpu() if host else out


def series_sum(x, workspace=None, stream=None):
    """FP64 sum of x in the library's fixed order: a float64 device tensor of shape (1,)."""
    torch = _torch()
    xd, _ = _prepare(x)
    out = torch.empty(1, dtype=torch.float64, device=xd.device)
    ws = _workspace(workspace, xd.device)
    ws.get(workspace_size(_native.OP_SERIES_SUM, xd.numel(), 1, xd.numel(), make_params(1)))
    _native.check(_native.lib().hos_series_sum(xd.data_ptr(), _dtype_code(xd), xd.numel(), out.data_ptr(), ws.ptr(),
                                               ws.nbytes(), _stream(stream)), "hos_series_sum")
    return out


def cumulant3_slice(x, L, halo_before, halo_after, total_sum, n_total, precision="bf16", remove_mean=True, tile_n=0,
                    flush_chunks=0, workspace=None, stream=None):
    """One time slice's share of c3 of a longer series (float64, (2L, 2L)).

    ``x`` holds ``halo_before`` samples before the slice, the slice, and
    ``halo_after`` samples after it (each <= L, fewer only at the series'
    ends); ``total_sum`` is a float64 device tensor with the whole series' sum
    and ``n_total`` its length.  Summing the slices' results gives c3 of the
    whole series."""
    torch = _torch()
    xd, _ = _prepare(x)
    n_slice = xd.numel() - int(halo_before) - int(halo_after)
    p = make_params(L, 0, precision, "parzen", remove_mean, 0, tile_n, flush_chunks)
    tot = total_sum.to(device=xd.device, dtype=torch.float64).contiguous()
    out = torch.empty((2 * p.L, 2 * p.L), dtype=torch.float64, device=xd.device)
    ws = _workspace(workspace, xd.device)
    ws.get(workspace_size(_native.OP_CUMULANT3_SLICE, max(n_slice, 0), 1, max(n_slice, 0), p))
    _native.check(_native.lib().hos_cumulant3_slice(xd.data_ptr(), _dtype_code(xd), n_slice, int(halo_before),
                                                    int(halo_after), tot.data_ptr(), int(n_total), ctypes.byref(p),
                                                    out.data_ptr(), ws.ptr(), ws.nbytes(), _stream(stream)),
                  "hos_cumulant3_slice")
    return out


def bispectrum_from_cumulant(c3, L, nfft=0, window="parzen", out=None, workspace=None, stream=None):
    """Window, scale and transform a c3 of :func:`cumulant3`'s layout into B."""
    torch = _torch()
    cd = c3.to(torch.float64).contiguous()
    p = make_params(L, nfft, "bf16", window)
    N = p.nfft or 2 * p.L
    if out is None:
        out = torch.empty((N, N), dtype=torch.complex64, device=cd.device)
    ws = _workspace(workspace, cd.device)
    ws.get(workspace_size(_native.OP_BISPECTRUM_FROM_C3, 0, 1, 0, p))
    _native.check(_native.lib().hos_bispectrum_from_cumulant(cd.data_ptr(), ctypes.byref(p), out.data_ptr(), ws.ptr(),
                                                             ws.nbytes(), _stream(stream)),
                  "hos_bispectrum_from_cumulant")
    return out


def bispectrum_sharded(x_local, L, halo_before, halo_after, n_total, nfft=0, precision="bf16", window="parzen",
                       remove_mean=True, group=None, workspace=None):
    """Bispectrum of one long series whose time slices are spread over the
    ranks of ``group`` (one GPU each; see :func:`shard.time_slices`).

    ``x_local`` is this rank's slice with its halo.  Two FP64 sum
    all-reduces: the series' total (for the mean) and the (2L)^2 c3.  Every
    rank returns the full B.  Without an initialised process group this is
    the single-rank case."""
    import torch.distributed as dist
    distributed = dist.is_available() and dist.is_initialized()
    xd, _ = _prepare(x_local)
    own = xd[int(halo_before):xd.numel() - int(halo_after)]
    tot = series_sum(own, workspace=workspace)
    if distributed:
        dist.all_reduce(tot, op=dist.ReduceOp.SUM, group=group)
    c3 = cumulant3_slice(xd, L, halo_before, halo_after, tot, n_total, precision, remove_mean, workspace=workspace)
    if distributed:
        dist.all_reduce(c3, op=dist.ReduceOp.SUM, group=group)
    return bispectrum_from_cumulant(c3, L, nfft, window, workspace=workspace)


def moments4_slice(x, L, halo_before, halo_after, total_sum, n_total, precision="bf16", remove_mean=True,
                   flush_chunks=0, workspace=None, stream=None):
    """One time slice's share of the fourth moment and of c2 of a longer
    series: (m4 float64 (2L, 2L, 2L), c2 float64 (4L - 1,)).

    ``x`` holds ``halo_before`` (<= L) samples before the slice, the slice,
    and ``halo_after`` (<= 2L) after it, fewer only at the series' ends
    (:func:`shard.time_slices` with ``halo_after=2 * L``).  Summing the
    slices' m4 and c2 gives the whole series' (time averages over n_total)."""
    torch = _torch()
    xd, _ = _prepare(x)
    n_slice = xd.numel() - int(halo_before) - int(halo_after)
    p = make_params(L, 0, precision, "parzen", remove_mean, 0, 0, flush_chunks)
    tot = total_sum.to(device=xd.device, dtype=torch.float64).contiguous()
    m4 = torch.empty((2 * p.L,) * 3, dtype=torch.float64, device=xd.device)
    c2 = torch.empty(4 * p.L - 1, dtype=torch.float64, device=xd.device)
    ws = _workspace(workspace, xd.device)
    ws.get(workspace_size(_native.OP_MOMENTS4_SLICE, max(n_slice, 0), 1, max(n_slice, 0), p))
    _native.check(_native.lib().hos_moments4_slice(xd.data_ptr(), _dtype_code(xd), n_slice, int(halo_before),
                                                   int(halo_after), tot.data_ptr(), int(n_total), ctypes.byref(p),
                                                   m4.data_ptr(), c2.data_ptr(), ws.ptr(), ws.nbytes(),
                                                   _stream(stream)), "hos_moments4_slice")
    return m4, c2


def trispectrum_from_moments(m4, c2, L, nfft=0, window="parzen", out=None, workspace=None, stream=None):
    """c4 = m4 - (three c2 c2 products), window, scale and 3-D transform: T
    from joined time-slice moments (:func:`moments4_slice`)."""
    torch = _torch()
    md = m4.to(torch.float64).contiguous()
    cd = c2.to(device=md.device, dtype=torch.float64).contiguous()
    p = make_params(L, nfft, "bf16", window)
    N = p.nfft or 2 * p.L
    if out is None:
        out = torch.empty((N, N, N), dtype=torch.complex64, device=md.device)
    ws = _workspace(workspace, md.device)
    ws.get(workspace_size(_native.OP_TRISPECTRUM_FROM_MOMENTS, 0, 1, 0, p))
    _native.check(_native.lib().hos_trispectrum_from_moments(md.data_ptr(), cd.data_ptr(), ctypes.byref(p),
                                                             out.data_ptr(), ws.ptr(), ws.nbytes(), _stream(stream)),
                  "hos_trispectrum_from_moments")
    return out


def trispectrum_sharded(x_local, L, halo_before, halo_after, n_total, nfft=0, precision="bf16", window="parzen",
                        remove_mean=True, group=None, workspace=None):
    """Trispectrum of one long series whose time slices are spread over the
    ranks of ``group`` (one GPU each; slices from :func:`shard.time_slices`
    with ``halo_after=2 * L``).  Three FP64 sum all-reduces: the series'
    total, the (2L)^3 fourth moment and the 4L - 1 c2.  Every rank returns
    the full T."""
    import torch.distributed as dist
    distributed = dist.is_available() and dist.is_initialized()
    xd, _ = _prepare(x_local)
    own = xd[int(halo_before):xd.numel() - int(halo_after)]
    tot = series_sum(own, workspace=workspace)
    if distributed:
        dist.all_reduce(tot, op=dist.ReduceOp.SUM, group=group)
    m4, c2 = moments4_slice(xd, L, halo_before, halo_after, tot, n_total, precision, remove_mean,
                            workspace=workspace)
    if distributed:
        dist.all_reduce(m4, op=dist.ReduceOp.SUM, group=group)
        dist.all_reduce(c2, op=dist.ReduceOp.SUM, group=group)
    return trispectrum_from_moments(m4, c2, L, nfft, window, workspace=workspace)


def bispectrum_direct(x, M, M3, remove_mean=True, overlap=0, out=None, workspace=None, stream=None):
    """The paper's direct method (Algorithm DBS): parts of M samples (every
    M - overlap samples), raw (1/M) F(k1) F(k2) F*(k1+k2), M3 x M3 box
    smoothing by window sums, average over parts.  (M, M) complex64 over the
    whole grid, [k1][k2]."""
    xd, host = _prepare(x)
    dev, host_out = _out_buffers(out, (int(M), int(M)), xd.device)
    nbytes = ctypes.c_size_t(0)
    _native.check(_native.lib().hos_bispectrum_direct_workspace_size(xd.numel(), int(M), int(M3), int(overlap),
                                                                       ctypes.byref(nbytes)),
                  "hos_bispectrum_direct_workspace_size")
    ws = _workspace(workspace, xd.device)
    ws.get(nbytes.value)
    _native.check(_native.lib().hos_bispectrum_direct(xd.data_ptr(), _dtype_code(xd), xd.numel(), int(M), int(M3),
                                                      int(overlap), int(bool(remove_mean)), dev.data_ptr(), ws.ptr(),
                                                      ws.nbytes(), _stream(stream)), "hos_bispectrum_direct")
    return _finish(dev, host_out, host)


def bispectrum_backward(x, dB, L, nfft=0, precision="bf16", window="parzen", remove_mean=True, workspace=None,
                        stream=None):
    """dl/dx given dB = dl/dRe B + i dl/dIm B."""
    torch = _torch()
    xd, host = _prepare(x)
    p = make_params(L, nfft, precision, window, remove_mean, 0)
    g = dB.to(xd.device).to(torch.complex64).contiguous()
    dx = torch.empty_like(xd)
    ws = _workspace(workspace, xd.device)
    ws.get(workspace_size(_native.OP_BISPECTRUM_BACKWARD, xd.numel(), 1, xd.numel(), p))
    _native.check(_native.lib().hos_bispectrum_backward(xd.data_ptr(), _dtype_code(xd), xd.numel(), ctypes.byref(p),
                                                        g.data_ptr(), dx.data_ptr(), ws.ptr(), ws.nbytes(),
                                                        _stream(stream)), "hos_bispectrum_backward")
    return dx.cpu() if host else dx


class BispectrumFn:
    """torch.autograd.Function wrapper, created lazily so that importing the
    package does not import torch."""
    _cls = None

    @classmethod
    def get(cls):
        if cls._cls is None:
            torch = _torch()

            class _Fn(torch.autograd.Function):
                @staticmethod
                def forward(ctx, x, L, nfft, precision, window, remove_mean):
                    ctx.save_for_backward(x)
                    ctx.cfg = (L, nfft, precision, window, remove_mean)
                    return bispectrum(x, L, nfft, precision, window, remove_mean)

                @staticmethod
                def backward(ctx, gB):
                    (x,) = ctx.saved_tensors
                    L, nfft, precision, window, remove_mean = ctx.cfg
                    dx = bispectrum_backward(x, gB, L, nfft, precision, window, remove_mean)
                    return dx, None, None, None, None, None

            cls._cls = _Fn
        return cls._cls


def bispectrum_ad(x, L, nfft=0, precision="bf16", window="parzen", remove_mean=True):
    """Differentiable bispectrum (torch autograd)."""
    return BispectrumFn.get().apply(x, L, nfft, precision, window, remove_mean)


def trispectrum_backward(x, dT, L, nfft=0, precision="bf16", window="parzen", remove_mean=True, workspace=None,
                         stream=None):
    """dl/dx given dT = dl/dRe T + i dl/dIm T (nfft^3).  Split-bf16 tensor-core
    adjoint only (precision "bf16" or "fp16"), L <= 64, one part."""
    torch = _torch()
    xd, host = _prepare(x)
    p = make_params(L, nfft, precision, window, remove_mean, 0)
    g = dT.to(xd.device).to(torch.complex64).contiguous()
    dx = torch.empty_like(xd)
    ws = _workspace(workspace, xd.device)
    ws.get(workspace_size(_native.OP_TRISPECTRUM_BACKWARD, xd.numel(), 1, xd.numel(), p))
    _native.check(_native.lib().hos_trispectrum_backward(xd.data_ptr(), _dtype_code(xd), xd.numel(),
                                                         ctypes.byref(p), g.data_ptr(), dx.data_ptr(), ws.ptr(),
                                                         ws.nbytes(), _stream(stream)), "hos_trispectrum_backward")
    return dx.cpu() if host else dx


class TrispectrumFn:
    """torch.autograd.Function wrapper of the trispectrum, created lazily."""
    _cls = None

    @classmethod
    def get(cls):
        if cls._cls is None:
            torch = _torch()

            class _Fn(torch.autograd.Function):
                @staticmethod
                def forward(ctx, x, L, nfft, precision, window, remove_mean):
                    ctx.save_for_backward(x)
                    ctx.cfg = (L, nfft, precision, window, remove_mean)
                    return trispectrum(x, L, nfft, precision, window, remove_mean)

                @staticmethod
                def backward(ctx, gT):
                    (x,) = ctx.saved_tensors
                    L, nfft, precision, window, remove_mean = ctx.cfg
                    dx = trispectrum_backward(x, gT, L, nfft, precision, window, remove_mean)
                    return dx, None, None, None, None, None

            cls._cls = _Fn
        return cls._cls


def trispectrum_ad(x, L, nfft=0, precision="bf16", window="parzen", remove_mean=True):
    """Differentiable trispectrum (torch autograd; split-bf16 forward and adjoint)."""
    return TrispectrumFn.get().apply(x, L, nfft, precision, window, remove_mean)


def device_status(workspace=None) -> int:
    torch = _torch()
    ws = _workspace(workspace, torch.device("cuda", torch.cuda.current_device()))
    if ws.buf is None:
        return 0
    v = ctypes.c_int32(0)
    _native.check(_native.lib().hos_get_device_status(ws.ptr(), ctypes.byref(v)), "hos_get_device_status")
    return int(v.value)


def reset_device_status(workspace=None, stream=None):
    torch = _torch()
    ws = _workspace(workspace, torch.device("cuda", torch.cuda.current_device()))
    if ws.buf is not None:
        _native.check(_native.lib().hos_reset_device_status(ws.ptr(), _stream(stream)), "hos_reset_device_status")


def selftest_timeout(timeout_us=1000, workspace=None, stream=None) -> int:
    """Run the device-side timeout self test; returns the status word it left."""
    torch = _torch()
    ws = _workspace(workspace, torch.device("cuda", torch.cuda.current_device()))
    ws.get(256)
    reset_device_status(ws, stream)
    _native.check(_native.lib().hos_selftest_timeout(ws.ptr(), ws.nbytes(), int(timeout_us), _stream(stream)),
                  "hos_selftest_timeout")
    torch.cuda.synchronize()
    return device_status(ws)


def set_profiling(on: bool):
    _native.lib().hos_set_profiling(int(bool(on)))


def stage_times():
    """[(stage name, ms)] of the last call made while profiling was on."""
    arr = (ctypes.c_float * 8)()
    n = ctypes.c_int32(0)
    _native.check(_native.lib().hos_get_stage_times(arr, 8, ctypes.byref(n)), "hos_get_stage_times")
    return [(_native.lib().hos_stage_name(i).decode(), float(arr[i])) for i in range(n.value)]


def launch_count() -> int:
    return int(_native.lib().hos_launch_count())


def last_contraction() -> str:
    return _native.lib().hos_last_contraction().decode()


def last_plan() -> str:
    """The last call's contraction plan (tile widths, flush, chunk, CTAs), as text."""
    return _native.lib().hos_last_plan().decode()
