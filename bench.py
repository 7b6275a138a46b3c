#!/usr/bin/env python
"""Benchmark: complex multi-component LU GFLOPS (8 n^3 / 3 / t) at n = 4096.

One step = one complex LU factorisation with partial pivoting (zgetrf) plus
one solve (zgetrs) of a fresh copy of a synthetic n x n matrix (Gaussian
leading limbs, canonical lower limbs, seed 1), i.e. one pass over the whole
hot path.  value = steps * 8 n^3 / 3 / elapsed, summed over ranks (each rank
an independent replica; the path has no data exchange).

The default step uses the Ozaki-scheme trailing update on the tensor cores
(nb = 128, factored as four 32-column sub-panels); the same step with the
plain FP64-pipe 4M update (nb = 64) is
timed right after it and reported under "plain", with both backward errors,
so that the speed-up is stated at equal accuracy.  The TD and QD steps (Ozaki
and plain, n = 4096) follow under "precisions", and the standalone complex
ZGEMM of m = n = k = 1024 (4M, 3M, Ozaki; DD, TD, QD) under "zgemm_1024".
FP64-pipe rooflines use the FP64 rate measured in the same run
(mclu_probe_fp64_rate) as their peak.

Other modes (one JSON line per point): --sweep (block width, the paper's
time-vs-K study), --slices-sweep (Ozaki slices per operand against accuracy,
the paper's divisions study), --zgemm (standalone ZGEMM workloads: 1024^3 per
precision with 3M against 4M, and 4096^3 DD / TD with entries spread over
2^+-20, Ozaki against plain).

Timing: W untimed warm-up steps, then K steps between a barrier +
torch.cuda.synchronize() on both sides, CUDA events on the library's stream,
max over ranks.  The matrix (537 MB in DD) is larger than L2 (129 MB), so no
explicit flush is needed.  SM clocks are sampled with nvidia-smi during the
timed region.  `e2e` repeats the step through the C ABI with pinned host
buffers: A and b are copied host->device and x device->host every step.

--impl reference times the CPU oracle (test infrastructure, not the product)
on the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# FP64-pipe operations (DADD/DMUL/DFMA, 1 each) per complex multiply-accumulate
# of the trailing update, as implemented in mc.cuh (leveled accumulator):
# one real product-accumulate costs 12 (DD), 45 (TD), 112 (QD); 4M uses 4 per
# complex MAC, 3M uses 3.
I_REAL = {"dd": 12, "td": 45, "qd": 112}
LIMBS = {"dd": 2, "td": 3, "qd": 4}
# FP64 peak: 1.25 TFLOP/s nominal on GB300 counting an FMA as 2 flops, i.e.
# 0.625e12 FP64 operations per second (2 per clock per SM at 2.07 GHz).
FP64_OPS_PEAK = 0.625e12
# Ozaki-scheme engine: slices S per precision; kept pairs p + q <= S - 1.
OZAKI_S = {"dd": 16, "td": 24, "qd": 32}
# DRAM traffic of the trailing-update kernel from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum of the first trailing update of
# the n = 4096 DD step: n2 = 3968 rows and columns, K = 256 realified).  It is
# reported, scaled to the average trailing launch by n2^2, only while the
# kernel source is the one it was taken on (sha1 of csrc/ozaki.cuh).
OZ_TRAFFIC = {"dd": {"bytes": 604965120 + 468543232, "n2": 3968, "src_sha1": "bdde21fd20155ef65d5b2e26c12829e015eb3623"}}
# ncu dram__bytes_read.sum + dram__bytes_write.sum of one cooperative panel
# launch (the first 32-column sub-panel of n = 2048: m = 2048 rows), valid
# while the kernel's source is unchanged
PANEL_TRAFFIC = {"dd": {"bytes": 2244096 + 39168, "m": 2048, "w": 32, "src_sha1": "c28d79383cdc2fa089319ef508a6aa90a1d22481"}}
# unit roundoff exponents: u = 2^-104 / 2^-157 / 2^-209
U_EXP = {"dd": 104, "td": 157, "qd": 209}


def fp64_peak(measured: float | None) -> tuple[float, str]:
    """FP64 operations per second for the alu rooflines: the rate measured in
    this run by mclu_probe_fp64_rate, else the nominal figure."""
    if measured:
        return measured, "measured FP64 DFMA rate (mclu_probe_fp64_rate, this run)"
    return FP64_OPS_PEAK, "nominal FP64 (1.25 TFLOP/s, FMA = 2)"


def measured_bf16_peak() -> tuple[float, str]:
    """Dense bf16 TFLOP/s from MEASURED_PEAKS.json (burst), else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]), "measured"
    except Exception:
        return 1900.0, "fallback"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="mclu", choices=["mclu", "reference"])
    p.add_argument("--prec", default="dd", choices=["dd", "td", "qd"])
    p.add_argument("--method", default="ozaki", choices=["4m", "3m", "unblocked", "ozaki", "strassen"])
    p.add_argument("--n", type=int, default=4096)
    p.add_argument("--nb", type=int, default=0, help="block width (0: 128 for ozaki, 64 otherwise)")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-plain", action="store_true", help="skip the plain 4M comparison of an ozaki run")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=15.0, help="target CPU seconds of the oracle sample")
    p.add_argument("--slices", type=int, default=0, help="Ozaki slices per operand (0: the precision's default)")
    p.add_argument("--sub-nb", type=int, default=0, help="Ozaki sub-panel width (0: the library's default)")
    p.add_argument("--no-precisions", action="store_true", help="skip the TD / QD steps of the default line")
    p.add_argument("--no-zgemm", action="store_true", help="skip the 1024^3 ZGEMM sub-object of the default line")
    p.add_argument("--slices-sweep", action="store_true",
                   help="LU + solve GFLOP/s and backward error against the Ozaki slice count, per precision")
    p.add_argument("--zgemm", action="store_true", help="standalone ZGEMM workloads, one JSON line per point")
    p.add_argument("--sweep", action="store_true",
                   help="block-width sweep instead of the benchmark line: LU + solve GFLOP/s for every method "
                        "and nb at --n (default 1024), plus the unblocked form; one JSON line per point")
    p.add_argument("--profile-step", action="store_true",
                   help="one untimed LU + solve of the workload (after one at n = 256) and nothing else: "
                        "the command that launch lists and ncu captures run")
    return p.parse_args()


def run_profile_step(args):
    """One factorisation + solve of the configured workload, untimed, after
    the same at n = 256 (kernels loaded, workspace pool warm), with no probe,
    clock sampler or oracle: a short, fixed launch sequence for profilers."""
    import torch
    from paper_2403_16013_gb300 import api, build, inputs
    build.build()
    torch.cuda.set_device(0)
    L = LIMBS[args.prec]
    nb = args.nb if args.nb else (128 if args.method == "ozaki" else 64)
    for n in (256, args.n):
        A = torch.from_numpy(inputs.gaussian_matrix(n, L, seed=1)).cuda()
        b = torch.from_numpy(inputs.complex_gaussian_vector(n, L, seed=2)).cuda()
        LU, ipiv, info = api.lu_factor(A, method=args.method, nb=nb, ozaki_slices=args.slices,
                                       sub_nb=args.sub_nb)
        api.lu_solve(LU, ipiv, b)
        torch.cuda.synchronize()
        if int(info.item()) != 0:
            raise SystemExit(f"profile step: info = {int(info.item())} at n = {n}")
    print(f"profile step ok: {args.prec} {args.method} n={args.n} nb={nb}", flush=True)


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl"
        dist.init_process_group(backend=backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, ws: int, device: str = "cuda") -> float:
    """Largest x over the ranks (the job is as slow as its slowest replica)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(ws: int, steps: int, flops_per_step: float, elapsed_ms: float) -> float:
    """Whole-job GFLOP/s: every rank factors its own replica, elapsed is the max over ranks."""
    return ws * steps * flops_per_step / (elapsed_ms * 1e-3) / 1e9


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.idx), "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except FileNotFoundError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.th.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "samples": len(sm),
                "reasons": sorted(reasons)}


def make_inputs(n: int, L: int):
    from paper_2403_16013_gb300 import inputs
    A = inputs.gaussian_matrix(n, L, seed=1)
    b = inputs.complex_gaussian_vector(n, L, seed=2)
    return A, b


def cpu_baseline(prec: str, target_s: float) -> dict:
    """Time the oracle (unblocked GEPP + solve, as it stands) on the host cores on
    a bounded sample: the largest n whose estimated run is about target_s."""
    import oracle
    L = LIMBS[prec]
    cores = oracle.num_threads()
    from paper_2403_16013_gb300 import inputs

    def run(n):
        A = inputs.gaussian_matrix(n, L, seed=1)
        b = inputs.complex_gaussian_vector(n, L, seed=2)
        t0 = time.perf_counter()
        LU, ipiv, info, _ = oracle.zgetrf(A)
        oracle.zgetrs(LU, ipiv, b)
        return time.perf_counter() - t0

    n0 = 96
    t0 = run(n0)
    n = int(n0 * (target_s / max(t0, 1e-3)) ** (1 / 3))
    n = max(n0, min(n, 1024))
    t = run(n) if n != n0 else t0
    return {"value": 8 * n ** 3 / 3 / t / 1e9, "unit": "GFLOP/s", "cores": cores, "kind": "oracle",
            "sample": f"complex {prec.upper()} LU+solve n={n} (unblocked oracle, {t:.1f} s), seed 1",
            "seconds": t}


def run_reference(args):
    ws, rank, _ = int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")), 0
    if rank != 0:
        return
    per_step = max(3.0, args.cpu_seconds / 3)
    vals = []
    for _ in range(args.warmup):
        cpu_baseline(args.prec, per_step / 4)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(cpu_baseline(args.prec, per_step))
    el = time.perf_counter() - t0
    v = statistics.median(x["value"] for x in vals)
    cb = dict(vals[-1])
    cb["value"] = v
    line = {"impl": "reference", "metric": "complex DD/TD/QD LU GFLOPS (8n^3/3/t) at n=4096", "value": v,
            "unit": "GFLOP/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": el / args.steps * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"complex {args.prec.upper()} LU + solve (CPU oracle sample of the n={args.n} "
                                   f"workload)", "n": args.n, "prec": args.prec},
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def panel_roofline(method: str, prec: str, n: int, nb: int, steps: int, prof: dict, el_ms: float,
                   fp64: float | None = None, sub_nb: int = 0):
    """Roofline of the cooperative panel kernel (FP64 pipe): the algorithmic
    FP64 operations of its multipliers and rank-1 updates (4 real
    product-accumulates of I_REAL operations per complex multiply-accumulate)
    per launch over the average event-timed launch duration."""
    panel_ms, panel_calls = prof["panel"]
    if not panel_calls:
        return None
    w = (sub_nb or 32) if method == "ozaki" else nb  # panel width of one launch
    macs = 0
    for s0 in range(0, n, w):
        ww = min(w, n - s0)
        m = n - s0
        for jc in range(ww):
            rows = m - jc - 1
            macs += rows * (ww - jc - 1) + rows  # rank-1 update + multiplier
    per_launch = macs * 4 * I_REAL[prec] / (panel_calls / steps)
    achieved = per_launch / (panel_ms / panel_calls * 1e-3)
    traffic, note = None, None
    cap = PANEL_TRAFFIC.get(prec)
    if cap and method == "ozaki" and w == cap["w"]:
        import hashlib
        with open(os.path.join(ROOT, "paper_2403_16013_gb300", "csrc", "panel_coop.cuh"), "rb") as f:
            if hashlib.sha1(f.read()).hexdigest() == cap["src_sha1"]:
                rows = [n - s0 for s0 in range(0, n, w)]
                traffic = cap["bytes"] * (sum(rows) / len(rows)) / cap["m"]
                note = "ncu dram read+write of one launch with m = 2048 rows, scaled to the average launch by rows"
    peak, src = fp64_peak(fp64)
    return {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "T FP64-ops/s",
            "frac": achieved / peak, "peak_source": src,
            "traffic": traffic, "traffic_note": note,
            "kernel": f"{'k_panel_coop' if LIMBS[prec] == 2 else 'k_panel_team'}<{LIMBS[prec]}> "
                      "(latency bound: a serial FP64 chain per column)",
            "ops_per_launch": per_launch, "avg_launch_ms": panel_ms / panel_calls, "share_of_step": panel_ms / el_ms}


def roofline(method: str, prec: str, n: int, nb: int, steps: int, prof: dict, el_ms: float,
             fp64: float | None = None, slices: int = 0):
    """Roofline of the trailing update: algorithmic work per launch (from n, nb
    and the method) over its average event-timed duration."""
    L = LIMBS[prec]
    gemm_ms, gemm_calls = prof["gemm"]
    if not gemm_calls:
        return None
    if method == "ozaki":
        S = slices or OZAKI_S[prec]
        pairs = S * (S + 1) // 2
        # realified real GEMM per kept slice pair: n2 x (2 n2) x (2 jb), 2 flops per MAC
        flops = 0.0
        for j0 in range(0, n, nb):
            jb = min(nb, n - j0)
            n2 = n - j0 - jb
            flops += pairs * 2.0 * n2 * (2 * n2) * (2 * jb)
        per_launch = flops / (gemm_calls / steps)
        achieved = per_launch / (gemm_ms / gemm_calls * 1e-3) / 1e12
        peak, src = measured_bf16_peak()
        traffic = None
        cap = OZ_TRAFFIC.get(prec)
        if cap and nb == 128 and n == 4096 and S == OZAKI_S[prec]:
            import hashlib
            with open(os.path.join(ROOT, "paper_2403_16013_gb300", "csrc", "ozaki.cuh"), "rb") as f:
                if hashlib.sha1(f.read()).hexdigest() == cap["src_sha1"]:
                    n2s = [n - j0 - min(nb, n - j0) for j0 in range(0, n, nb)]
                    n2s = [v for v in n2s if v > 0]
                    traffic = cap["bytes"] * (sum(v * v for v in n2s) / len(n2s)) / cap["n2"] ** 2
        return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "peak_source": src + " bf16 burst", "traffic": traffic,
                "traffic_note": None if traffic is None else
                "ncu dram read+write of the first trailing launch (n2 = 3968), scaled to the average launch by n2^2",
                "kernel": f"k_oz_gemm<{L},beta> (+ split kernels, counted in its time)",
                "flops_per_launch": per_launch, "avg_launch_ms": gemm_ms / gemm_calls,
                "share_of_step": gemm_ms / el_ms}
    if method in ("4m", "3m"):
        macs = 0
        for j0 in range(0, n, nb):
            jb = min(nb, n - j0)
            n2 = n - j0 - jb
            macs += n2 * n2 * jb
        per_mac = (3 if method == "3m" else 4) * I_REAL[prec]
        per_launch_ops = macs * per_mac / (gemm_calls / steps)
        achieved = per_launch_ops / (gemm_ms / gemm_calls * 1e-3)
        peak, src = fp64_peak(fp64)
        return {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "T FP64-ops/s",
                "frac": achieved / peak, "peak_source": src,
                "traffic": None, "kernel": f"k_gemm<{L},{'3M' if method == '3m' else '4M'},beta>",
                "ops_per_launch": per_launch_ops, "avg_launch_ms": gemm_ms / gemm_calls,
                "share_of_step": gemm_ms / el_ms}
    return None


def backward_error(api, A0, X, B0):
    """||b - A x||_inf / (||A||_inf ||x||_inf) (modulus norms), the residual
    formed by the library's ZGEMM (both forms tested against the exact product):
    DD and TD with the QD 4M product on the limbs zero-padded to four, which
    resolves it far below the bound; QD with the QD Ozaki product, whose
    C - A B epilogue is exact and whose slice truncation stays below
    2^-204 max|A_i.| max|x| (about 2^-216 of ||A|| ||x|| at n = 4096), below
    a QD residual."""
    import torch
    L = A0.shape[1]

    def pad(T):
        if L == 4:
            return T
        P = torch.zeros((2, 4) + tuple(T.shape[2:]), dtype=T.dtype, device=T.device)
        P[:, :L] = T
        return P

    R = api.zgemm(pad(A0), pad(X), C=pad(B0), method="ozaki" if L == 4 else "4m")
    r = torch.hypot(R[0].sum(dim=0), R[1].sum(dim=0)).max().item()
    anorm = torch.hypot(A0[0, 0], A0[1, 0]).sum(dim=0).max().item()
    xnorm = torch.hypot(X[0, 0], X[1, 0]).max().item()
    return r / (anorm * xnorm)


RESIDUAL_NOTE = ("b - A x by the library's ZGEMM: QD 4M on zero-padded limbs (DD, TD), QD Ozaki with its exact "
                 "C - A B epilogue (QD)")


def run_sweep(args):
    """Time-vs-K study of the blocked factorisation (the paper's Figs. 10/13/16
    analogue): LU + solve GFLOP/s against the block width for each trailing
    update, and the unblocked form, on one GPU."""
    import torch
    from paper_2403_16013_gb300 import api, binding, build
    build.build()
    binding.load()
    n = args.n if args.n != 4096 else 1024
    L, prec = LIMBS[args.prec], args.prec
    A_h, b_h = make_inputs(n, L)
    A0, b0 = torch.from_numpy(A_h).cuda(), torch.from_numpy(b_h).cuda()
    A, x = torch.empty_like(A0), torch.empty_like(b0)
    ipiv = torch.empty(n, dtype=torch.int32, device="cuda")
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    points = [("unblocked", 0)]
    for method in ("4m", "3m", "strassen", "ozaki"):
        for nb in (16, 32, 64, 96, 128, 192, 256):
            points.append((method, nb))
    for method, nb in points:
        def step():
            A.copy_(A0)
            api.lu_factor_(A, ipiv, info, method=method, nb=nb)
            x.copy_(b0)
            api.lu_solve(A, ipiv, x, inplace=True)
        step()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = max(1, args.steps)
        e0.record()
        for _ in range(reps):
            step()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        print(json.dumps({"sweep": True, "n": n, "prec": prec, "method": method, "nb": nb if nb else n,
                          "ms_per_step": ms, "value": 8.0 * n ** 3 / 3.0 / (ms * 1e-3) / 1e9, "unit": "GFLOP/s",
                          "info": int(info.item())}), flush=True)


def lu_step_fn(api, A, A0, x, b0, ipiv, info, method, nb, slices, sub_nb=0):
    def step():
        A.copy_(A0)
        oz = method == "ozaki"
        api.lu_factor_(A, ipiv, info, method=method, nb=nb, ozaki_slices=slices if oz else 0,
                       sub_nb=sub_nb if oz else 0)
        x.copy_(b0)
        api.lu_solve(A, ipiv, x, inplace=True)
    return step


def time_lu(ctx, prec, method, nb, steps, warmup, slices=0, sampler=None, ws=1, stream=None, fp64=None,
            warm_n=0, sub_nb=0):
    """LU + solve of the prec's benchmark matrix: warm-up steps (at order warm_n
    when given, which loads the kernels without the cost of full-size steps),
    then `steps` steps between barriers and CUDA events on the library's stream,
    with launch-class timing; returns value, phases, rooflines, backward error."""
    import torch
    api, binding = ctx["api"], ctx["binding"]
    n = ctx["n"]
    A0, b0 = ctx["inputs"][prec]
    A, x = torch.empty_like(A0), torch.empty_like(b0)
    ipiv = torch.empty(n, dtype=torch.int32, device="cuda")
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    step = lu_step_fn(api, A, A0, x, b0, ipiv, info, method, nb, slices, sub_nb)
    if warm_n:
        Aw = A0[:, :, :warm_n, :warm_n].contiguous()
        bw = b0[:, :, :, :warm_n].contiguous()
        Ax, xw = torch.empty_like(Aw), torch.empty_like(bw)
        ipw = torch.empty(warm_n, dtype=torch.int32, device="cuda")
        wstep = lu_step_fn(api, Ax, Aw, xw, bw, ipw, info, method, nb, slices, sub_nb)
        for _ in range(max(1, warmup)):
            wstep()
    else:
        for _ in range(warmup):
            step()
    torch.cuda.synchronize()
    if int(info.item()) != 0:
        raise RuntimeError(f"zgetrf info {int(info.item())} on the benchmark matrix")
    barrier(ws)
    torch.cuda.synchronize()
    if sampler is not None:
        sampler.start()
        time.sleep(0.4)
    binding.profile_begin(("gemm", "panel", "trsm", "laswp", "getrs", "other"))
    launches0 = binding.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    launches = binding.launch_count() - launches0
    prof = binding.profile_end()
    clocks = sampler.stop() if sampler is not None else None
    el_ms = max_over_ranks(e0.elapsed_time(e1), ws)
    if int(info.item()) != 0:
        raise RuntimeError(f"zgetrf info {int(info.item())} on the benchmark matrix")
    upd = roofline(method, prec, n, nb, steps, prof, el_ms, fp64=fp64, slices=slices)
    pan = panel_roofline(method, prec, n, nb, steps, prof, el_ms, fp64=fp64, sub_nb=sub_nb)
    # the "roofline" object describes the kernel with the largest share of the step
    first, second = (pan, upd) if (pan and (not upd or pan["share_of_step"] > upd["share_of_step"])) else (upd, pan)
    eta = backward_error(api, A0, x, b0)
    return {"el_ms": el_ms, "launches": launches, "prof": prof, "clocks": clocks, "steps": steps,
            "warmup": warmup, "value": job_throughput(ws, steps, 8.0 * n ** 3 / 3.0, el_ms),
            "backward_error": eta, "roofline": first, "roofline_secondary": second,
            "ipiv": ipiv}


def sub_object(r: dict, method: str, nb: int, slices: int, prec: str, n: int) -> dict:
    out = {"method": method, "nb": nb, "value": r["value"], "unit": "GFLOP/s", "ms_per_step": r["el_ms"] / r["steps"],
           "steps": r["steps"], "warmup": r["warmup"], "backward_error": r["backward_error"],
           "bound_16nu": 16.0 * n * 2.0 ** -U_EXP[prec], "roofline": r["roofline"],
           "roofline_secondary": r["roofline_secondary"],
           "phases_ms_per_step": {k: v[0] / r["steps"] for k, v in r["prof"].items()}}
    if method == "ozaki":
        out["ozaki_slices"] = slices or OZAKI_S[prec]
    return out


def zgemm_point(ctx, prec, method, m, n, k, reps, A, B, fp64=None, slices=0) -> dict:
    """Standalone C = A B (beta_mode 0): ms per call (CUDA events, after one
    warm-up call), GFLOP/s counted as 8 m n k, and the roofline of the kernel."""
    import torch
    api, binding = ctx["api"], ctx["binding"]
    api.zgemm(A, B, method=method, ozaki_slices=slices)
    torch.cuda.synchronize()
    binding.profile_begin(("gemm",))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        C = api.zgemm(A, B, method=method, ozaki_slices=slices)
    e1.record()
    torch.cuda.synchronize()
    prof = binding.profile_end()
    del C
    ms = e0.elapsed_time(e1) / reps
    # the product kernels' time; for Strassen the whole call (its block sums
    # and combinations are part of the method, and its product scopes nest)
    kern_ms = ms if method == "strassen" else prof["gemm"][0] / max(1, prof["gemm"][1])
    L = LIMBS[prec]
    out = {"prec": prec, "method": method, "m": m, "n": n, "k": k, "ms": ms, "value": 8.0 * m * n * k / (ms * 1e-3) / 1e9,
           "unit": "GFLOP/s"}
    if method == "ozaki":
        S = slices or OZAKI_S[prec]
        flops = S * (S + 1) // 2 * 2.0 * m * (2 * n) * (2 * k)
        peak, src = measured_bf16_peak()
        ach = flops / (kern_ms * 1e-3) / 1e12
        out["ozaki_slices"] = S
        out["roofline"] = {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                           "peak_source": src + " bf16 burst", "traffic": None,
                           "kernel": f"k_oz_gemm<{L},0> (+ split kernels)"}
    else:
        # Strassen: 7 of the 8 block products of 3M (one level of Winograd's variant)
        ops = float(m) * n * k * {"3m": 3.0, "4m": 4.0, "strassen": 3.0 * 7 / 8}[method] * I_REAL[prec]
        peak, src = fp64_peak(fp64)
        ach = ops / (kern_ms * 1e-3)
        out["roofline"] = {"bound": "alu", "achieved": ach / 1e12, "peak": peak / 1e12, "unit": "T FP64-ops/s",
                           "frac": ach / peak, "peak_source": src, "traffic": None,
                           "kernel": f"k_gemm<{L},{'4M' if method == '4m' else '3M'},0> (+ k_resum for 3M"
                                     f"{', block sums and combinations for Strassen' if method == 'strassen' else ''})"}
    return out


def setup(args, precs):
    import torch
    from paper_2403_16013_gb300 import api, binding, build
    build.build()
    binding.load()
    ctx = {"api": api, "binding": binding, "n": args.n, "inputs": {}}
    for prec in precs:
        A_h, b_h = make_inputs(args.n, LIMBS[prec])
        ctx["inputs"][prec] = (torch.from_numpy(A_h).cuda(), torch.from_numpy(b_h).cuda())
    return ctx


def run_slices_sweep(args):
    """The paper's divisions study (Sec. 4.1-4.3: how many Ozaki divisions each
    precision needs inside LU) on this engine: for each precision, LU + solve
    at --n with S, S-1, ... slices per operand, the backward error of each,
    and the plain 4M step's, one JSON line per point."""
    import torch
    torch.cuda.set_device(0)
    precs = [args.prec] if args.prec != "dd" or args.n != 4096 else ["dd", "td", "qd"]
    for prec in precs:
        ctx = setup(args, [prec])
        n = args.n
        plain = time_lu(ctx, prec, "4m", 64, 1, 1, warm_n=256)
        print(json.dumps({"slices_sweep": True, "prec": prec, "n": n, "method": "4m", "value": plain["value"],
                          "ms_per_step": plain["el_ms"], "backward_error": plain["backward_error"]}), flush=True)
        S = OZAKI_S[prec]
        for Se in range(S, max(1, S - 8), -1):
            r = time_lu(ctx, prec, "ozaki", 128, max(1, args.steps), 1, slices=Se)
            same = bool(torch.equal(r["ipiv"], plain["ipiv"]))
            print(json.dumps({"slices_sweep": True, "prec": prec, "n": n, "method": "ozaki", "ozaki_slices": Se,
                              "value": r["value"], "ms_per_step": r["el_ms"] / r["steps"],
                              "backward_error": r["backward_error"],
                              "eta_over_plain": r["backward_error"] / plain["backward_error"],
                              "bound_16nu": 16.0 * n * 2.0 ** -U_EXP[prec], "pivots_equal_plain": same}),
                  flush=True)
        del ctx
        torch.cuda.empty_cache()


def run_zgemm(args):
    """Standalone ZGEMM workloads: m = n = k = 1024 per precision, 4M / 3M /
    Ozaki on Gaussian limbs (seeds 1, 2); m = n = k = 4096 DD and TD with
    entries N(0,1) 2^e, e in [-20, 20] (seeds 3, 4), Ozaki against 4M."""
    import torch
    from paper_2403_16013_gb300 import inputs
    torch.cuda.set_device(0)
    ctx = setup(args, [])
    fp64 = ctx["binding"].probe_fp64_rate()
    for prec in ("dd", "td", "qd"):
        L = LIMBS[prec]
        A = torch.from_numpy(inputs.gaussian_matrix(1024, L, seed=1)).cuda()
        B = torch.from_numpy(inputs.gaussian_matrix(1024, L, seed=2)).cuda()
        for method in ("4m", "3m", "strassen", "ozaki"):
            r = zgemm_point(ctx, prec, method, 1024, 1024, 1024, max(1, args.steps), A, B, fp64=fp64)
            r["workload"] = "gaussian limbs 1024^3"
            print(json.dumps(r), flush=True)
    for prec in ("dd", "td"):
        L = LIMBS[prec]
        A = torch.from_numpy(inputs.spread_matrix(4096, 4096, L, seed=3, spread=20)).cuda()
        B = torch.from_numpy(inputs.spread_matrix(4096, 4096, L, seed=4, spread=20)).cuda()
        for method in ("ozaki", "4m"):
            r = zgemm_point(ctx, prec, method, 4096, 4096, 4096, 1, A, B, fp64=fp64)
            r["workload"] = "exponent spread 2^+-20, 4096^3"
            print(json.dumps(r), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.sweep:
        run_sweep(args)
        return
    if args.slices_sweep:
        run_slices_sweep(args)
        return
    if args.zgemm:
        run_zgemm(args)
        return
    if args.profile_step:
        run_profile_step(args)
        return
    import torch

    ws, rank, local = dist_init()
    torch.cuda.set_device(local)
    n, L, prec = args.n, LIMBS[args.prec], args.prec
    others = [] if (args.no_precisions or args.prec != "dd") else ["td", "qd"]
    ctx = setup(args, [prec])
    api, binding = ctx["api"], ctx["binding"]
    fp64 = binding.probe_fp64_rate()
    nb_of = lambda m: args.nb if args.nb else (128 if m == "ozaki" else 64)
    stream = torch.cuda.current_stream()
    method, nb = args.method, nb_of(args.method)
    main_run = time_lu(ctx, prec, method, nb, args.steps, args.warmup, slices=args.slices,
                       sampler=ClockSampler(local), ws=ws, stream=stream, fp64=fp64, sub_nb=args.sub_nb)
    bound = 16.0 * n * 2.0 ** -U_EXP[prec]
    A_bytes = ctx["inputs"][prec][0].numel() * 8
    line = {"metric": "complex DD/TD/QD LU GFLOPS (8n^3/3/t) at n=4096", "value": main_run["value"],
            "unit": "GFLOP/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": main_run["el_ms"] / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"complex {prec.upper()} LU (zgetrf, partial pivoting) + solve (zgetrs), n={n}, "
                                   f"nb={nb}, {method.upper()} trailing update, Gaussian limbs seed 1",
                       "n": n, "prec": prec, "method": method, "nb": nb,
                       "l2": "inputs larger than L2 (%.0f MB per matrix), no flush" % (A_bytes / 1e6),
                       "parallelism": f"replicas x{ws}"},
            "gpu_launches": main_run["launches"], "clocks": main_run["clocks"], "roofline": main_run["roofline"],
            "roofline_secondary": main_run["roofline_secondary"],
            "phases_ms_per_step": {k: v[0] / args.steps for k, v in main_run["prof"].items()},
            "accuracy": {"backward_error": main_run["backward_error"], "bound_16nu": bound,
                         "residual": RESIDUAL_NOTE},
            "fp64_measured_ops_per_s": fp64}
    if method == "ozaki":
        line["config"]["ozaki_slices"] = args.slices or OZAKI_S[prec]

    if method == "ozaki" and not args.no_plain:
        # the same step with the plain FP64-pipe 4M update, for the speed-up at equal accuracy
        plain = time_lu(ctx, prec, "4m", nb_of("4m"), min(args.steps, 5), min(args.warmup, 2), ws=ws,
                        stream=stream, fp64=fp64)
        line["plain"] = sub_object(plain, "4m", nb_of("4m"), 0, prec, n)
        line["ozaki_speedup_vs_plain"] = main_run["value"] / plain["value"]

    if not args.no_e2e:
        A_h = ctx["inputs"][prec][0].cpu().numpy()
        b_h = ctx["inputs"][prec][1].cpu().numpy()
        A_pin = torch.from_numpy(A_h).pin_memory()
        b_pin = torch.from_numpy(b_h).pin_memory()
        x_pin = torch.empty_like(b_pin).pin_memory()
        ipiv_pin = torch.empty(n, dtype=torch.int32).pin_memory()
        A = torch.empty_like(ctx["inputs"][prec][0])
        x = torch.empty_like(ctx["inputs"][prec][1])
        ipiv = torch.empty(n, dtype=torch.int32, device="cuda")
        info = torch.zeros(1, dtype=torch.int32, device="cuda")

        def e2e_step():
            A.copy_(A_pin, non_blocking=True)
            api.lu_factor_(A, ipiv, info, method=method, nb=nb, ozaki_slices=args.slices if method == "ozaki" else 0)
            x.copy_(b_pin, non_blocking=True)
            api.lu_solve(A, ipiv, x, inplace=True)
            x_pin.copy_(x, non_blocking=True)
            ipiv_pin.copy_(ipiv, non_blocking=True)

        e2e_step()
        torch.cuda.synchronize()
        barrier(ws)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(max(1, args.steps)):
            e2e_step()
        torch.cuda.synchronize()
        barrier(ws)
        el = max_over_ranks(time.perf_counter() - t0, ws)
        line["e2e"] = {"value": job_throughput(ws, max(1, args.steps), 8.0 * n ** 3 / 3.0, el * 1e3),
                       "unit": "GFLOP/s", "h2d_bytes_per_step": A_h.nbytes + b_h.nbytes,
                       "d2h_bytes_per_step": b_h.nbytes + 4 * n}
        del A, x, A_pin

    if others:
        # TD and QD at the same order: the Ozaki step (3 warm-up, up to 5 timed) and the plain 4M
        # step (warmed up at n = 256, one timed step: 7-20 s each at n = 4096)
        del ctx["inputs"][prec]
        line["precisions"] = {}
        for p2 in others:
            ctx2 = setup(args, [p2])
            oz = time_lu(ctx2, p2, "ozaki", 128, min(args.steps, 5), 3, ws=ws, stream=stream, fp64=fp64)
            pl = time_lu(ctx2, p2, "4m", 64, 1, 1, ws=ws, stream=stream, fp64=fp64, warm_n=256)
            line["precisions"][p2] = {"ozaki": sub_object(oz, "ozaki", 128, 0, p2, n),
                                      "plain": sub_object(pl, "4m", 64, 0, p2, n),
                                      "ozaki_speedup_vs_plain": oz["value"] / pl["value"]}
            del ctx2
            torch.cuda.empty_cache()

    if not args.no_zgemm:
        from paper_2403_16013_gb300 import inputs
        line["zgemm_1024"] = []
        for p2 in ("dd", "td", "qd"):
            L2 = LIMBS[p2]
            Ag = torch.from_numpy(inputs.gaussian_matrix(1024, L2, seed=1)).cuda()
            Bg = torch.from_numpy(inputs.gaussian_matrix(1024, L2, seed=2)).cuda()
            for m2 in ("4m", "3m", "ozaki"):
                line["zgemm_1024"].append(zgemm_point(ctx, p2, m2, 1024, 1024, 1024, 2, Ag, Bg, fp64=fp64))

    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(prec, args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
