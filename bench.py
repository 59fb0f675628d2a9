#!/usr/bin/env python3
"""Benchmark: cumulant lag-terms/s of the long bispectrum workload on GB300.

Workload (one step): the smoothed sample bispectrum of one AR(2) series of
n = 2^21 samples (centred Exp(1) innovations), Parzen lag window L = 256,
512 x 512 grid: FP64 mean removal, c3 contraction on the tensor cores,
FP64 reduction + window, 2-D transform.  Metric unit: n (2L+1)^2 lag terms.

  python bench.py [--gpus N --steps K --warmup W --precision bf16|fp32|simt]
  python bench.py --impl reference      # the FP64 CPU oracle on a bounded sample

Multi-GPU (torchrun, N > 1), weak scaling (2^21 samples per rank): the long
workload becomes one series of N x 2^21 samples cut into time slices (each
rank its slice plus L-sample halos; FP64 all-reduces of the series' sum and
of c3; every rank transforms); the other workloads run one independent copy
per rank.  Rank 0 prints the max-over-ranks time.  --time-slices runs the
sliced layout on one rank.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "long_bispectrum_n2M_L256"
METRIC = "cumulant lag-terms/s (n*(2L+1)^(k-1)) and % tensor peak, split-BF16 vs FP32, same GPU"
UNIT = "lag-terms/s"


def units_of(n, L, k=3):
    return n * (2 * L + 1) ** (k - 1)


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [v.strip() for v in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def kernel_source_hash():
    import hashlib
    h = hashlib.sha256()
    for f in ("c3_tc.cu", "hos_internal.cuh"):
        with open(os.path.join(ROOT, "paper_1805_11775_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(prec):
    """DRAM bytes per launch of the contraction from the committed ncu summary,
    or None when the kernel source has changed since those counters were taken."""
    path = os.path.join(ROOT, "profiles", f"c3_tc_{prec}_long_n2M_L256.md")
    if not os.path.exists(path):
        return None
    fields = {}
    with open(path) as f:
        for ln in f:
            if ":" in ln and ln.split(":")[0].strip() in ("kernel_source_sha256_16", "traffic_bytes_per_launch"):
                k, v = ln.split(":", 1)
                fields[k.strip()] = v.strip()
    if fields.get("kernel_source_sha256_16") != kernel_source_hash():
        return None
    return int(fields["traffic_bytes_per_launch"]) if "traffic_bytes_per_launch" in fields else None


def cpu_baseline(x, L, n, seconds_target=10.0):
    """The FP64 oracle as it stands, on this host's cores, over a bounded
    sample of the same workload: whole rows w1 of the lag square (every w2,
    every sample), extrapolated per lag term."""
    import oracle
    y = oracle.demean(x)
    rows = 2
    t0 = time.perf_counter()
    oracle.c3_rows(y, L, 0, rows - 1)
    dt = time.perf_counter() - t0
    rows = max(2, min(2 * L, int(rows * seconds_target / max(dt, 1e-3))))
    t0 = time.perf_counter()
    ref = oracle.c3_rows(y, L, -(rows // 2), -(rows // 2) + rows - 1)
    dt = time.perf_counter() - t0
    terms = rows * (2 * L + 1) * n
    return {"value": terms / dt, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
            "sample": f"c3 rows w1 in [{-(rows // 2)}, {-(rows // 2) + rows - 1}] x all {2 * L + 1} w2 x n={n} "
                      f"({terms:.3e} lag terms, {dt:.1f} s)"}, (-(rows // 2), ref)


def accuracy(hos, torch, x, L, prec, lo, ref, knobs=None):
    """Normwise error of the timed path's output (same input, contraction
    precision, plan, tile width, flush and chunk length as the timed steps)
    over the oracle rows the CPU baseline computed: B is brought back to the
    lag grid by an FP64 inverse transform, (2 pi)^2 ifft2(B)[w1, w2] =
    W(w1, w2) c3(w1, w2), and compared with the window times the oracle's c3:
    max |d| / max |ref|."""
    import numpy as np
    import oracle
    B = hos.bispectrum(torch.from_numpy(x).cuda(), L, precision=prec, **(knobs or {}))
    N = B.shape[0]
    G = (torch.fft.ifft2(B.to(torch.complex128)).real * (2 * math.pi) ** 2).cpu().numpy()
    rows = ref.shape[0]
    w1 = np.arange(lo, lo + rows)
    w2 = np.arange(-L, L)
    got = G[(w1 % N)[:, None], (w2 % N)[None, :]]
    win = np.array([[oracle.window2(int(a), int(b), L) for b in w2] for a in w1])
    want = win * ref[:, :2 * L]
    return {"vs": "FP64 oracle", "quantity": "W c3 (the lag grid of B, FP64 inverse transform)", "max_rel_err":
            float(np.abs(got - want).max() / np.abs(want).max()),
            "sample": f"rows w1 in [{lo}, {lo + rows - 1}] x w2 in [{-L}, {L - 1}]"}


def run_reference(args):
    import hos_synth
    import oracle
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    oracle.build()
    w = hos_synth.workload(WORKLOAD)
    x, L = w["x"], w["L"]
    n = x.size
    y = oracle.demean(x)
    rows = 8
    times = []
    for step in range(args.warmup + args.steps):
        r0 = -L + (step * rows) % (2 * L + 1 - rows)
        t0 = time.perf_counter()
        oracle.c3_rows(y, L, r0, r0 + rows - 1)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            times.append(dt)
    terms = rows * (2 * L + 1) * n
    value = terms / statistics.mean(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": n, "L": L, "grid": w["N"]},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
                             "sample": f"each step: c3 of {rows} rows w1 x all {2 * L + 1} w2 x n={n}"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def principal_mask(N):
    import numpy as np
    k1, k2 = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    return (k2 <= k1) & (k1 + k2 < N // 2)


def plan_fields(plan):
    """{'tile_n': .., 'tiles': .., 'cols': .., 'kc': ..} from hos_last_plan's text."""
    out = {}
    for tok in plan.split():
        if "=" in tok:
            k, v = tok.split("=", 1)
            if v.isdigit():
                out[k] = int(v)
    return out


def c3_tc_flops(lens, products, plan):
    """Executed tensor-core flops of the c3 contraction from the plan the call
    ran: 128 rows x the tiles' columns added up x padded samples x products x 2
    (rows from each 128-row block's diagonal block on)."""
    f = plan_fields(plan)
    kc = f.get("kc", 1024)
    kpad = sum(math.ceil(int(n) / kc) * kc for n in lens)
    return 128 * f["cols"] * kpad * products * 2, (
        f"{f['tiles']} tiles x 128 rows, {f['cols']} columns in all x {kpad} padded samples x {products} products"
        f" x 2 flops")


def m4_flops(L, n, prec):
    """Executed flops of the m4 contraction.  Tensor cores: 128-pair tiles of
    the lag triangle w1 <= w2 x next_pow2(2L) columns w3 x padded samples x 3
    products x 2 (chunks of 1024 samples, 128 for 3xTF32 and split FP16;
    one product for plain TF32).  SIMT: FFMA over pair rows x w3 rounded to
    16 x samples rounded to 4096."""
    two_l = 2 * L
    npairs = two_l * (two_l + 1) // 2
    rows = math.ceil(npairs / 128) * 128
    if prec in ("bf16", "fp32", "fp16", "tf32"):
        cols = max(32, 1 << (two_l - 1).bit_length())
        kc = {"fp32": 128, "fp16": 128}.get(prec, 1024)
        kpad = math.ceil(n / kc) * kc
        prod = 1 if prec == "tf32" else 3
        return rows * cols * kpad * 2 * prod, (f"{rows} lag pairs x {cols} w3 x {kpad} padded samples x {prod} products"
                                               f" x 2 flops")
    w3 = 16 * math.ceil(two_l / 16)
    kpad = math.ceil(n / 4096) * 4096
    return rows * w3 * kpad * 2, f"{rows} lag pairs x {w3} w3 x {kpad} samples x 2 flops (FFMA)"


def adjoint4_flops(L, n):
    """Executed flops of the trispectrum adjoint contraction
    D[u, (w1, w2)] = sum_w3 y(u + w3) Gs(w1, w2, w3) (split-bf16): blocks of 128
    (w1, w2) combinations x 128-row u tiles x 2L rounded to 16 lags w3 x 3
    products x 2."""
    two_l = 2 * L
    kpad = 16 * math.ceil(two_l / 16)
    nb, nut = math.ceil(two_l * two_l / 128), math.ceil(n / 128)
    return nb * nut * 128 * 128 * kpad * 6, (
        f"{nb} (w1, w2) blocks x {nut} u tiles x 128 x 128 x {kpad} lags w3 x 3 products x 2 flops")


def adjoint_flops(L, n, prec):
    """Executed flops of the adjoint contraction U = Hankel(y) Gs.  Tensor
    cores (split-bf16 or split FP16, L <= 128): 128-row tiles of u x 128-lag
    blocks of w1 x 2L rounded to 16 lags w2 x 3 products x 2.  SIMT (fp32,
    tf32 and simt precisions): 2 flops per (u, w1, w2)."""
    two_l = 2 * L
    if prec in ("bf16", "fp16") and L <= 128:
        kpad = 16 * math.ceil(two_l / 16)
        nb, nut = math.ceil(two_l / 128), math.ceil(n / 128)
        return nb * nut * 128 * 128 * kpad * 6, (
            f"{nb} lag blocks x {nut} u tiles x 128 x 128 x {kpad} lags x 3 products x 2 flops")
    return n * two_l * two_l * 2, f"{n} u x {two_l} x {two_l} lags x 2 flops (FFMA)"


def make_workload(name, prec, rank, hos, torch, series=0, time_slices=False):
    """Device-resident inputs, the step closure, the e2e closure, lag-term
    units per step, and the dominant kernel's executed work."""
    import numpy as np

    import hos_synth
    ws = hos.Workspace()
    if name == "direct_bispectrum_n8192_M3_279":
        # the paper's direct method at its largest reported size: one part
        # (K = 1, M = n = 8192), 279 x 279 box smoothing
        M, M3 = 8192, 279
        x_host = hos_synth.ar2(M, 1006)
        xd = torch.from_numpy(x_host).cuda()
        out = torch.empty((M, M), dtype=torch.complex64, device="cuda")
        step = lambda: hos.bispectrum_direct(xd, M, M3, out=out, workspace=ws)
        x_pin = torch.from_numpy(x_host).pin_memory()
        o_pin = torch.empty((M, M), dtype=torch.complex64).pin_memory()
        e2e = lambda: hos.bispectrum_direct(x_pin, M, M3, workspace=ws, out=o_pin)
        # the smoothing stage streams the M x M grid five times (raw write and read, column sums
        # write and read, result write), 8 bytes per complex64 point
        grid_bytes = 5 * M * M * 8
        return dict(step=step, e2e=e2e, units=1, metric="bispectra/s (direct method, n = M = 8192, box 279)",
                    unit="bispectra/s", paper_value=1.0 / 1.751, flops=0, work=f"5 passes x {M}^2 x 8 B",
                    roof={"bound": "hbm", "bytes": grid_bytes, "stage": "smooth"}, bound="hbm",
                    h2d=x_host.nbytes, d2h=M * M * 8, config={"n": M, "M": M, "M3": M3, "parts": 1})
    w = hos_synth.workload(name)
    L, N = w["L"], w["N"]
    products = {"bf16": 3, "fp32": 3, "tf32": 1, "fp16": 3}.get(prec, 1)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if name == "long_bispectrum_n2M_L256" and (world > 1 or time_slices):
        # one series of world x 2^21 samples, cut into time slices (one per
        # rank, L-sample halos); two FP64 all-reduces join the ranks
        import torch.distributed as dist
        joined = dist.is_available() and dist.is_initialized()

        from paper_1805_11775_gb300.shard import slice_with_halo
        n_rank = w["x"].size
        x_all = hos_synth.ar2(world * n_rank, 1002)
        xh, hb, ha = slice_with_halo(x_all, rank, world, L)
        xh = np.ascontiguousarray(xh)
        xd = torch.from_numpy(xh).cuda()
        step = lambda: hos.bispectrum_sharded(xd, L, hb, ha, x_all.size, precision=prec, workspace=ws)
        x_pin = torch.from_numpy(xh).pin_memory()
        e2e = lambda: hos.bispectrum_sharded(x_pin.to("cuda", non_blocking=True), L, hb, ha, x_all.size,
                                             precision=prec, workspace=ws).cpu()

        def profile():
            """Stage times of one step, the library calls traced one by one."""
            own = xd[hb:xd.numel() - ha]
            tot = hos.series_sum(own, workspace=ws)
            if joined:
                dist.all_reduce(tot)
            c3 = hos.cumulant3_slice(xd, L, hb, ha, tot, x_all.size, precision=prec, workspace=ws)
            st = dict(hos.stage_times())
            if joined:
                dist.all_reduce(c3)
            hos.bispectrum_from_cumulant(c3, L, workspace=ws)
            for k, v in hos.stage_times():
                st[k] = st.get(k, 0.0) + v
            return list(st.items())

        lens_ = [xh.size - hb - ha]
        return dict(step=step, e2e=e2e, profile=profile, units=units_of(xh.size - hb - ha, L),
                    flops_of=lambda plan: c3_tc_flops(lens_, products, plan), h2d=xh.nbytes, d2h=N * N * 8,
                    bound="tensor" if prec != "simt" else "alu",
                    config={"n": int(x_all.size), "n_per_rank": int(xh.size - hb - ha), "L": L, "grid": N,
                            "parallelism": f"time slices x{world}, FP64 all-reduce of c3"})
    from paper_1805_11775_gb300 import tune
    if name in ("long_bispectrum_n2M_L256", "bispectrum_n2048_L32"):
        x_host = w["x"] if rank == 0 else hos_synth.ar2(w["x"].size, 1002 + 100 * rank)
        xd = torch.from_numpy(x_host).cuda()
        out = torch.empty((N, N), dtype=torch.complex64, device="cuda")
        step = lambda: hos.bispectrum(xd, L, precision=prec, out=out, workspace=ws)
        x_pin = torch.from_numpy(x_host).pin_memory()
        o_pin = torch.empty((N, N), dtype=torch.complex64).pin_memory()
        e2e = lambda: hos.bispectrum(x_pin, L, precision=prec, workspace=ws, out=o_pin)
        extra = {"flops_of": lambda plan: c3_tc_flops([x_host.size], products, plan)}
        if name == "bispectrum_n2048_L32":  # small enough for the whole oracle spectrum

            def acc():
                import oracle
                ref = oracle.bispectrum(x_host, L, N)
                return {"vs": "FP64 oracle", "quantity": "B (whole grid)", "sample": "all of B",
                        "max_rel_err": float(np.abs(out.cpu().numpy() - ref).max() / np.abs(ref).max())}

            extra["accuracy"] = acc
        if prec != "simt":
            extra["tune"] = lambda: tune.tune_bispectrum(xd, L, precision=prec)
        return dict(step=step, e2e=e2e, units=units_of(x_host.size, L),
                    h2d=x_host.nbytes, d2h=N * N * 8, config={"n": int(x_host.size), "L": L, "grid": N},
                    bound="tensor" if products >= 1 and prec != "simt" else "alu", **extra)
    if name == "trispectrum_n65536_L32":
        x_host = w["x"]
        xd = torch.from_numpy(x_host).cuda()
        out = torch.empty((N, N, N), dtype=torch.complex64, device="cuda")
        step = lambda: hos.trispectrum(xd, L, precision=prec, out=out, workspace=ws)
        x_pin = torch.from_numpy(x_host).pin_memory()
        o_pin = torch.empty((N, N, N), dtype=torch.complex64).pin_memory()
        e2e = lambda: hos.trispectrum(x_pin, L, precision=prec, workspace=ws, out=o_pin)
        flops, work = m4_flops(L, x_host.size, prec)

        def acc():
            import oracle
            ref = oracle.trispectrum(x_host.astype(np.float64), L, N)
            got = out.cpu().numpy()
            return {"vs": "FP64 oracle", "quantity": "T (whole grid)",
                    "max_rel_err": float(np.abs(got - ref).max() / np.abs(ref).max()), "sample": "all of T"}

        return dict(step=step, e2e=e2e, accuracy=acc, units=units_of(x_host.size, L, k=4), flops=flops,
                    bound="tensor" if prec != "simt" else "alu", work=work,
                    h2d=x_host.nbytes, d2h=N ** 3 * 8, config={"n": int(x_host.size), "L": L, "grid": N})
    if name == "batched_4096x_L128":
        vals, offs = w["x"], w["offsets"]
        if series:  # a leading subset of the series (profiling a smaller case)
            offs = offs[:series + 1]
            vals = vals[:offs[-1]]
        lens = np.diff(offs)
        S = lens.size
        vd = torch.from_numpy(vals).cuda()
        od = torch.from_numpy(offs).cuda()
        out = torch.empty((S, N, N), dtype=torch.complex64, device="cuda")
        max_len = int(lens.max())
        step = lambda: hos.bispectrum_batched(vd, od, L, precision=prec, out=out, workspace=ws, max_len=max_len)
        v_pin = torch.from_numpy(vals).pin_memory()
        o_pin = torch.empty((S, N, N), dtype=torch.complex64).pin_memory()
        e2e = lambda: hos.bispectrum_batched(v_pin, offs, L, precision=prec, workspace=ws, max_len=max_len,
                                             out=o_pin)
        def acc():
            import oracle
            got = out[:8].cpu().numpy()
            err = 0.0
            for k in range(min(8, S)):
                ref = oracle.bispectrum(vals[offs[k]:offs[k + 1]], L, N)
                err = max(err, float(np.abs(got[k] - ref).max() / np.abs(ref).max()))
            return {"vs": "FP64 oracle", "quantity": "B per series (worst of the sample)", "max_rel_err": err,
                    "sample": "series 0..7, whole grids"}

        return dict(step=step, e2e=e2e, accuracy=acc, units=int((lens * (2 * L + 1) ** 2).sum()),
                    flops_of=lambda plan: c3_tc_flops(lens, products, plan),
                    tune=(lambda: tune.tune_bispectrum_batched(vd, od, L, precision=prec, repeats=3, max_len=max_len))
                    if prec != "simt" else None,
                    h2d=vals.nbytes + offs.nbytes, d2h=S * N * N * 8, bound="tensor" if prec != "simt" else "alu",
                    config={"series": S, "total_samples": int(lens.sum()), "L": L, "grid": N},
                    per_series=(vd, offs, L))
    if name == "differentiable_n262144_L128":
        x_host, t_host = w["x"], w["target_x"]
        xd = torch.from_numpy(x_host).cuda()
        Bt = hos.bispectrum(torch.from_numpy(t_host).cuda(), L, precision=prec)
        mask = torch.from_numpy(principal_mask(N)).cuda()
        out = torch.empty((N, N), dtype=torch.complex64, device="cuda")
        ws2 = hos.Workspace()

        def step():
            B = hos.bispectrum(xd, L, precision=prec, out=out, workspace=ws)
            G = 2.0 * (B - Bt) * mask  # gradient of sum_principal |B - Bt|^2
            return hos.bispectrum_backward(xd, G, L, workspace=ws2, precision=prec)

        x_pin = torch.from_numpy(x_host).pin_memory()

        def e2e():
            xg = x_pin.to("cuda", non_blocking=True)
            B = hos.bispectrum(xg, L, precision=prec, workspace=ws)
            G = 2.0 * (B - Bt) * mask
            return hos.bispectrum_backward(xg, G, L, workspace=ws2, precision=prec).cpu()

        # the step's last call is the adjoint: its contraction is the timed stage
        flops, work = adjoint_flops(L, x_host.size, prec)
        return dict(step=step, e2e=e2e, units=units_of(x_host.size, L), flops=flops, work=work,
                    h2d=x_host.nbytes, d2h=x_host.nbytes,
                    bound="tensor" if (prec in ("bf16", "fp16") and L <= 128) else "alu",
                    config={"n": int(x_host.size), "L": L, "grid": N, "step": "forward + adjoint"})
    if name == "differentiable_trispectrum_n65536_L32":
        x_host, t_host = w["x"], w["target_x"]
        xd = torch.from_numpy(x_host).cuda()
        Tt = hos.trispectrum(torch.from_numpy(t_host).cuda(), L)
        out = torch.empty((N, N, N), dtype=torch.complex64, device="cuda")
        ws2 = hos.Workspace()
        last_g = {}

        def step():
            T = hos.trispectrum(xd, L, out=out, workspace=ws, precision=prec)
            G = 2.0 * (T - Tt)  # gradient of sum |T - Tt|^2
            last_g["G"] = G
            return hos.trispectrum_backward(xd, G, L, workspace=ws2, precision=prec)

        x_pin = torch.from_numpy(x_host).pin_memory()

        def e2e():
            xg = x_pin.to("cuda", non_blocking=True)
            T = hos.trispectrum(xg, L, workspace=ws, precision=prec)
            return hos.trispectrum_backward(xg, 2.0 * (T - Tt), L, workspace=ws2, precision=prec).cpu()

        def acc():
            import oracle
            G = last_g["G"]
            dx = hos.trispectrum_backward(xd, G, L, remove_mean=False, precision=prec).cpu().numpy()
            x64 = x_host.astype(np.float64)
            dc4 = oracle.grad_lag4(G.cpu().numpy().astype(np.complex128), L, N)
            dc2 = oracle.grad_c2(dc4, oracle.c2(x64, 2 * L), L)
            js = np.concatenate([[0, 1, x64.size - 1], np.random.default_rng(9).integers(0, x64.size, 13)])
            ref = oracle.dy4_at(x64, L, dc4, dc2, js)
            return {"vs": "FP64 oracle", "quantity": "dl/dx (mean removal off, same dl/dT)",
                    "max_rel_err": float(np.abs(dx[js] - ref).max() / np.abs(ref).max()),
                    "sample": f"{js.size} samples incl. both ends"}

        flops, work = adjoint4_flops(L, x_host.size)
        return dict(step=step, e2e=e2e, accuracy=acc, units=units_of(x_host.size, L, k=4), flops=flops, work=work,
                    h2d=x_host.nbytes, d2h=x_host.nbytes, bound="tensor",
                    config={"n": int(x_host.size), "L": L, "grid": N, "step": "forward + adjoint"})
    raise KeyError(name)


def time_arm(wl, args, hos, torch, flush_buf, dist, local, world, sliced):
    """Warm up, capture one step in a CUDA graph (one rank, unless eager),
    time exactly args.steps steps with CUDA events (L2 flushed before each,
    outside the events, clocks sampled), then take the stage times from eager
    profiled passes when the timed steps could not trace them.  Returns
    (ms per step, max over ranks; stage times; launches in the timed region;
    clocks; launch mode; wall seconds of the timed region)."""
    step = wl["step"]
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    n0 = hos.launch_count()
    step()
    torch.cuda.synchronize()
    launches_per_step = hos.launch_count() - n0
    graph = None
    # one GPU: replay a captured CUDA graph of the step (the launches of every
    # stage, no host gaps); the time-sliced multi-rank step runs eagerly
    if args.graph or (not args.eager and not sliced):
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            step()
        graph.replay()
        torch.cuda.synchronize()

    traced = graph is None and "profile" not in wl  # stage times straight from each timed step
    hos.set_profiling(traced)
    clocks = Clocks(local)
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    stage_acc = {}
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = hos.launch_count()
    clocks.start()
    t_wall0 = time.perf_counter()
    for i in range(args.steps):
        flush_buf.zero_()  # evict the previous step's data from L2 (outside the events)
        ev0[i].record()
        if graph is not None:
            graph.replay()
        else:
            step()
        ev1[i].record()
        torch.cuda.synchronize()
        if traced:
            for name, ms in hos.stage_times():
                stage_acc.setdefault(name, []).append(ms)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    launches = hos.launch_count() - launches0
    clk = clocks.stop()
    hos.set_profiling(False)
    step_ms = [a.elapsed_time(b) for a, b in zip(ev0, ev1)]
    ms = statistics.mean(step_ms)
    if dist is not None:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    if not traced:
        # graph replays (or a step of several traced calls): the per-stage time
        # comes from an eager profiled pass over the same inputs
        hos.set_profiling(True)
        for _ in range(5):
            flush_buf.zero_()
            if "profile" in wl:
                st = wl["profile"]()
            else:
                step()
                torch.cuda.synchronize()
                st = hos.stage_times()
            for name, v in st:
                stage_acc.setdefault(name, []).append(v)
        hos.set_profiling(False)
    if graph is not None:
        launches = launches_per_step * args.steps  # replays re-run the captured launches
    mode = "cuda graph replay" if graph is not None else "eager (C ABI per step)"
    return ms, stage_acc, launches, clk, mode, t_wall


DTYPES = {"bf16": "bf16x3 (split-bf16, fp32 accumulate, fp64-class reduce)",
          "fp32": "tf32x3 (fp32-class, fp32 accumulate, fp64-class reduce)",
          "tf32": "tf32 (one product, fp32 accumulate, fp64-class reduce)",
          "fp16": "f16x3 (fp32-class: split-fp16 of the power-of-two scaled series, fp32 accumulate, "
                  "fp64-class reduce)",
          "simt": "f32"}


def tensor_peak(prec, pk, src):
    """Dense tensor peak of the contraction's operand type (TFLOP/s)."""
    if prec == "bf16":
        return pk["bf16_tflops"], f"bf16 dense, {src} burst"
    if prec == "fp16":  # the same dense rate as bf16 (kind::f16, nominal 2.25 PFLOP/s either way)
        return pk["bf16_tflops"], f"fp16 dense = {src} bf16 burst (same nominal rate)"
    return pk["bf16_tflops"] * (1.1 / 2.25), f"tf32 dense = {src} bf16 burst x 1.1/2.25 (nominal ratio)"


def run_ours(args):
    import torch

    import hos_synth
    import paper_1805_11775_gb300 as hos

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    prec = args.precision
    wl = make_workload(args.workload, prec, rank, hos, torch, args.series, args.time_slices)
    flush_buf = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")  # > L2 (129 MB)
    sliced = args.workload == WORKLOAD and (world > 1 or args.time_slices)
    autotune = None
    if not args.no_tune and not sliced and wl.get("tune"):
        # the project's autotuner picks the tile width and flush length for
        # this shape; the timed steps run with automatic knobs, i.e. its choice
        best, times = wl["tune"]()
        autotune = {"chosen": {"tile_n": best[0], "flush_chunks": best[1], "chunk_len": best[2]},
                    "candidates_ms": {f"tile_n={t} flush={f} chunk={c}": round(v, 4) for (t, f, c), v in times.items()}}
    ms, stage_acc, launches, clk, mode, t_wall = time_arm(wl, args, hos, torch, flush_buf, dist, local, world, sliced)
    contract_ms = statistics.mean(stage_acc.get("contract", [float("nan")]))
    contraction = hos.last_contraction()
    plan = hos.last_plan()
    if "flops_of" in wl:  # executed work of the plan the timed calls ran
        wl["flops"], wl["work"] = wl["flops_of"](plan)

    pk, src = peaks()
    if wl["bound"] == "tensor":
        peak, peak_note = tensor_peak(prec, pk, src)
    else:
        peak = 152 * 128 * 2 * 2.07e9 / 1e12
        peak_note = "FP32 FFMA: 152 SMs x 128 lanes x 2 flops x 2.07 GHz"
    roof_unit = "TFLOP/s"
    if "roof" in wl:  # a memory-bound stage: algorithmic bytes over its time
        stage_ms = statistics.mean(stage_acc.get(wl["roof"]["stage"], [float("nan")]))
        achieved = wl["roof"]["bytes"] / (stage_ms * 1e-3) / 1e9
        peak, peak_note, roof_unit = pk["hbm_gbs"], f"HBM copy, {src}", "GB/s"
    else:
        achieved = wl["flops"] / (contract_ms * 1e-3) / 1e12
    nsm = torch.cuda.get_device_properties(local).multi_processor_count
    per_clk = 8192 if prec in ("bf16", "fp16") else 4096
    clock_peak = nsm * per_clk * (clk["sm_mhz"] or 2070.0) * 1e6 / 1e12
    is_tc = contraction.startswith("c3_tcgen05")
    traffic = profiled_traffic(prec) if (is_tc and args.workload == WORKLOAD) else None

    e2e_t = []
    for i in range(max(3, min(50, args.steps // 2))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        wl["e2e"]()  # host input -> device, compute, result -> host
        e2e_t.append(time.perf_counter() - t0)
    e2e_s = statistics.median(e2e_t)

    extra = {}
    if "per_series" in wl and rank == 0:
        vd, offs, L = wl["per_series"]
        ws1 = hos.Workspace()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for s_ in range(offs.size - 1):
            hos.bispectrum(vd[offs[s_]:offs[s_ + 1]], L, precision=prec, workspace=ws1)
        e1.record()
        torch.cuda.synchronize()
        extra["per_series_launches_ms"] = e0.elapsed_time(e1)

    units = wl["units"] * world
    value = units / (ms * 1e-3)
    line = {
        "metric": wl.get("metric", METRIC),
        "value": value,
        "unit": wl.get("unit", UNIT),
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": value / wl["paper_value"] if "paper_value" in wl else None,
        "dtype": "f32 (transform, products), double-float window sums" if "roof" in wl else DTYPES[prec],
        "data": "synthetic",
        "config": dict({"workload": args.workload, "precision": prec, "contraction": contraction,
                        "plan": plan, "autotune": autotune,
                        "l2": "flushed between timed steps (256 MB write)",
                        "launch": mode,
                        "parallelism": "replicas" if world > 1 else "single"}, **wl["config"]),
        "stage_ms": {k: statistics.mean(v) for k, v in stage_acc.items()},
        "roofline": {"bound": wl["bound"], "kernel": contraction, "achieved": achieved, "peak": peak,
                     "unit": roof_unit, "frac": achieved / peak, "traffic": traffic, "peak_source": peak_note,
                     "frac_clock_matched": achieved / clock_peak if wl["bound"] == "tensor" else None,
                     "work": wl["work"]},
        "e2e": {"value": wl["units"] / e2e_s, "unit": wl.get("unit", UNIT), "h2d_bytes_per_step": int(wl["h2d"]),
                "d2h_bytes_per_step": int(wl["d2h"])},
        "gpu_launches": launches,
        "clocks": clk,
        "wall_s_timed": t_wall,
    }
    line.update(extra)
    ref_rows = None
    if rank == 0 and not args.no_cpu_baseline and "accuracy" in wl:
        line["accuracy"] = wl["accuracy"]()
    if rank == 0 and not args.no_cpu_baseline and args.workload == WORKLOAD:
        x_host = hos_synth.workload(WORKLOAD)["x"]
        line["cpu_baseline"], ref_rows = cpu_baseline(x_host, 256, x_host.size)
        line["accuracy"] = accuracy(hos, torch, x_host, 256, prec, *ref_rows,
                                    knobs=autotune["chosen"] if autotune else None)
    arms = [c for c in args.compare.split(",") if c and c != prec]
    if args.workload == "differentiable_trispectrum_n65536_L32":
        arms = [c for c in arms if c in ("bf16", "fp16")]  # the trispectrum adjoint's precisions
    if arms and world == 1 and "roof" not in wl:
        # the same workload in other precisions on the same GPU (the metric's
        # "split-BF16 vs FP32, same GPU"), timed the same way
        line["compare"] = []
        for cprec in arms:
            wl2 = make_workload(args.workload, cprec, rank, hos, torch, args.series, args.time_slices)
            tune2 = None
            if not args.no_tune and wl2.get("tune"):
                b2, _ = wl2["tune"]()
                tune2 = {"tile_n": b2[0], "flush_chunks": b2[1], "chunk_len": b2[2]}
            ms2, st2, launches2, clk2, mode2, _ = time_arm(wl2, args, hos, torch, flush_buf, dist, local, world,
                                                           sliced)
            c2_ms = statistics.mean(st2.get("contract", [float("nan")]))
            if "flops_of" in wl2:
                wl2["flops"], wl2["work"] = wl2["flops_of"](hos.last_plan())
            pk2, note2 = tensor_peak(cprec, pk, src)
            arm = {"precision": cprec, "dtype": DTYPES[cprec], "contraction": hos.last_contraction(),
                   "plan": hos.last_plan(), "autotune": tune2, "ms_per_step": ms2,
                   "value": wl2["units"] * world / (ms2 * 1e-3), "unit": wl2.get("unit", UNIT), "launch": mode2,
                   "stage_ms": {k: statistics.mean(v) for k, v in st2.items()}, "clocks": clk2,
                   "gpu_launches": launches2}
            if wl2["bound"] == "tensor":
                ach2 = wl2["flops"] / (c2_ms * 1e-3) / 1e12
                arm["roofline"] = {"bound": "tensor", "achieved": ach2, "peak": pk2, "unit": "TFLOP/s",
                                   "frac": ach2 / pk2, "peak_source": note2, "work": wl2["work"]}
            if ref_rows is not None:
                arm["accuracy"] = accuracy(hos, torch, x_host, 256, cprec, *ref_rows, knobs=tune2)
            elif rank == 0 and not args.no_cpu_baseline and "accuracy" in wl2:
                arm["accuracy"] = wl2["accuracy"]()
            line["compare"].append(arm)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16", choices=["bf16", "fp32", "tf32", "simt", "fp16"])
    ap.add_argument("--compare", default="fp32,fp16",
                    help="comma-separated precisions (bf16, fp32, fp16, tf32, simt) also timed on the same workload "
                         "and GPU (\"\" to skip)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="skip the autotuner (automatic tile width and flush)")
    ap.add_argument("--workload", default=WORKLOAD,
                    choices=[WORKLOAD, "bispectrum_n2048_L32", "trispectrum_n65536_L32", "batched_4096x_L128",
                             "differentiable_n262144_L128", "differentiable_trispectrum_n65536_L32",
                             "direct_bispectrum_n8192_M3_279"])
    ap.add_argument("--graph", action="store_true", help="capture one step in a CUDA graph and replay it "
                    "(the default on one rank)")
    ap.add_argument("--eager", action="store_true", help="launch every step's kernels eagerly instead")
    ap.add_argument("--series", type=int, default=0, help="batched workload: use only the first K series")
    ap.add_argument("--time-slices", action="store_true",
                    help="long workload: run the time-sliced path (the N > 1 layout) even on one rank")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
