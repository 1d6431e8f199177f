#!/usr/bin/env python
"""Benchmark of the structured-Gram solve + gradient over randomized digital nets.

Workload (solve20): base-2 digital net, Gray order, LMS + digital shift, n = 2^20 points,
d = 16, 64 randomizations per GPU (weak scaling), order-2 DSI kernel with weights
0.9^j, nugget 1e-8, one right-hand side y = exp(sum_j x_j / j) - const + N(0, 1e-6).
A step runs the whole path for every randomization: first column, eigenvalues (FWHT),
transformed right-hand side, spectral epilogue (quadratic form, log det, posterior
mean/variance), MLL gradient back-transform and reduction, and the solve with one
refinement step.  Inputs are resident in HBM (y alone is 256 MB, twice the L2).

The headline `value` is points/s (randomizations x n / step time) of the FP32 path
(FP32 column and transforms, FP64 / float-float reductions, one refinement step); beside
it the same step with the float-float first column (QK_F32W), the plain FP64 path, point
generation, and the FWHT / FFTBR transforms alone.  `--impl reference` times the FP64 CPU
oracle on a bounded sample of the same workload.

`--profile CASE` runs one small self-contained invocation of a hot kernel instead (for a
profiler: ncu -k <kernel> -c <n> python bench.py --profile fused --R 8); it prints "ok".
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import re
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "structured-Gram solve+grad points/s at n=2^20 (FP32-refined vs plain FP64), FWHT HBM GB/s"
UNIT = "points/s"

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum, bytes per launch) of the fused
# kernels at 64 randomizations of n = 2^20, d = 16, from one ncu capture, and the hash of the
# CUDA sources that capture ran (kernel_source_hash()).  A run whose sources differ reports
# traffic null: the counters belong to another version of the kernels.
NCU_TRAFFIC = {
    "src_hash": "a3fa2874c89e",
    "bytes_r64": {"k_fused_A": 1283025408, "k_fused_B": 1294175744, "k_fused_C": 1053564672},
    "fwht_bytes": 589224704,
}
# Nominal FP64 rate of GB300 (profiling recipe's table; FP64 is not a tensor-core path here).
FP64_PEAK_TFLOPS = 1.25


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--R", type=int, default=64, help="randomizations per GPU")
    ap.add_argument("--m", type=int, default=20)
    ap.add_argument("--refine", type=int, default=1, help="refinement steps of the FP32 solve")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 comparison timing")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--e2e-chunk", type=int, default=0,
                    help="randomizations per host-copy chunk (e2e); 0: the fastest of a few, timed before")
    ap.add_argument("--sched", default="auto", choices=["auto", "launches", "persistent"],
                    help="batched schedule: tuned (auto), per-phase launches or one persistent launch")
    ap.add_argument("--lag", type=int, default=1, help="persistent schedule: units between phases")
    ap.add_argument("--profile", default=None, choices=["fused", "fwht", "fftbr", "points", "col", "lattice"],
                    help="run one small case of a hot kernel (for a profiler) instead of the benchmark")
    ap.add_argument("--reps", type=int, default=2, help="--profile: runs after one warm-up")
    ap.add_argument("--fp64", action="store_true", help="--profile fused/fftbr/col: FP64")
    ap.add_argument("--wide", action="store_true", help="--profile fused/col: float-float first column")
    ap.add_argument("--two-pass", action="store_true", help="--profile fwht: two-launch form")
    ap.add_argument("--persistent", action="store_true", help="--profile fused / fftbr: one persistent launch")
    ap.add_argument("--d", type=int, default=16, help="--profile points/col: dimensions")
    return ap.parse_args()


# The sources the fused pipeline's and the batched FWHT's kernels are compiled from.
FUSED_SOURCES = ("qk_fused.cuh", "qk_fused.cu", "qk_fused_f32.cu", "qk_fused_f32c.cu", "qk_fused_f32w.cu",
                 "qk_fused_f64.cu", "qk_column.cuh", "qk_common.cuh", "qk_factors.cuh", "qk_internal.h")


def _code_only(text: bytes) -> bytes:
    """C / C++ source without its comments and blank lines (a comment never changes a kernel)."""
    t = re.sub(rb"/\*.*?\*/", b"", text, flags=re.S)
    t = re.sub(rb"//[^\n]*", b"", t)
    return b"\n".join(b" ".join(line.split()) for line in t.splitlines() if line.strip())


def kernel_source_hash() -> str:
    """Hash of the CUDA sources of the fused pipeline and the batched FWHT, comments left out
    (which kernel version a measurement belongs to)."""
    h = hashlib.sha256()
    for name in FUSED_SOURCES + ("../../include/qk.h",):
        f = os.path.join(ROOT, "paper_2502_14256_gb300", "csrc", name)
        with open(f, "rb") as fh:
            h.update(os.path.basename(f).encode() + _code_only(fh.read()))
    return h.hexdigest()[:12]


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons every 200 ms while running."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except FileNotFoundError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows if len(r) >= 9 for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(self.rows)}


# ------------------------------------------------------------- replicas
def replica_seed_offset(rank: int) -> int:
    """Replicas: every rank draws its own randomizations (no data exchange between ranks)."""
    return 1000 * rank


def max_over_ranks(x: float, torch, dist, world: int, device) -> float:
    """The slowest rank's time: the whole job ends when its last rank does."""
    if world <= 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: int, world: int, ms_max: float) -> float:
    """Whole-job units/s: every rank's units over the slowest rank's time."""
    return world * units_per_rank / (ms_max * 1e-3)


# ------------------------------------------------------------- the workload
def build_workload(qk, torch, dev, R, m, seed_offset=0):
    """Seeded inputs on the device: scrambled columns, shifts, weights and y."""
    from paper_2502_14256_gb300 import inputs
    wl = inputs.workload("solve20")
    d = wl.d
    n = 1 << m
    net = inputs.make_net(wl.seed + seed_offset, d, R, wl.order)
    u32 = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).to(dev)  # noqa: E731
    Cd, Sd, Dd = u32(net.C), u32(net.S), u32(net.D)
    Ct = torch.empty((R, d, 32), dtype=torch.int32, device=dev)
    qk.lms_setup(Cd, Sd, Ct)
    ps = qk.pointset(qk.QK_NET_B2, d, R, Ct=Ct, D=Dd, order=qk.QK_GRAY)
    # y from the points: generated on the device in chunks (input preparation, untimed)
    rng = inputs.SplitMix64(wl.seed + 17 + seed_offset)
    noise = torch.from_numpy(wl.noise_sigma * rng.normal(R * n)).to(dev).reshape(R, n)
    jj = torch.arange(1, d + 1, dtype=torch.float64, device=dev)
    const = float(np.prod(np.arange(1, d + 1) * np.expm1(1.0 / np.arange(1, d + 1))))
    y = torch.empty((R, 1, n), dtype=torch.float64, device=dev)
    X = torch.empty((1, n, d), dtype=torch.int32, device=dev)
    for r in range(R):
        qk.gen_points(ps, r, 1, 0, n, X)
        x = (X[0].to(torch.int64) & 0xFFFFFFFF).to(torch.float64) * 2.0 ** -32
        y[r, 0] = torch.exp((x / jj).sum(dim=1)) - const + noise[r]
    del X
    w = torch.tensor(inputs.workload("solve20").gamma, dtype=torch.float64, device=dev)
    return dict(wl=wl, d=d, n=n, R=R, m=m, ps=ps, keep=[Cd, Sd, Dd, Ct, w], w=w, y64=y, net=net)


class Pipeline:
    """One batched schedule (all randomizations) in a given precision (torch dtype or qk.F32W)."""

    def __init__(self, qk, torch, dev, W, dtype, refine, keep_lam=False):
        self.qk, self.torch = qk, torch
        R, n, d = W["R"], W["n"], W["d"]
        # every precision sees the same inputs: y rounded to FP32 once
        self.y = W["y64"].to(torch.float32).to(qk.data_dtype(dtype)).contiguous()
        self.c = torch.empty_like(self.y)
        self.lam = torch.empty((R, n), dtype=torch.float64, device=dev)
        self.out = torch.empty((R, 1, qk.QK_MLL_NOUT), dtype=torch.float64, device=dev)
        self.grad = torch.empty((R, 1, 2 * d + 2), dtype=torch.float64, device=dev)
        kern = qk.kernel(qk.QK_DSI, W["wl"].alpha, W["w"], W["wl"].zeta)
        # eigenvalues are an output only when asked for (the timed step does not write them)
        self.task = qk.Task(W["ps"], kern, W["m"], 1, W["wl"].eta, self.y.data_ptr(), self.c.data_ptr(),
                            self.lam.data_ptr() if keep_lam else None, self.out.data_ptr(),
                            self.grad.data_ptr())
        self.ws = qk.workspace(qk.batch_workspace_bytes([self.task], dtype), dev)
        qk.batch_plan([self.task], dtype, refine, self.ws)
        self.status = torch.zeros(1, dtype=torch.int32, device=dev)

    def step(self, stream=None):
        self.qk.batch_run(self.ws, self.status, stream=stream)

    def kernel_ms(self, torch, steps, stream):
        """Per-kernel device milliseconds per step: a separate pass of `steps` steps with a CUDA
        event pair around every kernel (on the launching stream)."""
        self.qk.batch_timing(self.ws, steps)
        time_steps(torch, self.step, steps, 0, stream)
        out = self.qk.batch_kernel_ms(self.ws)
        self.qk.batch_timing(self.ws, 0)
        return {k: (v[0] / steps, v[1] / steps) for k, v in out.items()}


def time_steps(torch, fn, steps, warmup, stream):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


# ------------------------------------------------------------ CPU baselines
def oracle_sample(W_host, m_sample, count=1, r_first=0):
    """Time the FP64 oracle (as it stands) on `count` whole randomizations of the workload
    at n = 2^m_sample (a bounded sample: its cost is close to linear in n, so points/s
    carries over); returns (points/s, sample text)."""
    from oracle import qk_oracle as o
    from paper_2502_14256_gb300 import inputs
    wl = W_host["wl"]
    net = W_host["net"]
    d = W_host["d"]
    n = 1 << m_sample
    c = o.effective_weights(wl.gamma, wl.log_ls)
    t0 = time.perf_counter()
    for q in range(count):
        r = (r_first + q) % net.R
        Ct = o.lms_scramble(net.C, net.S[r:r + 1])[0]
        X = o.net_points(Ct, net.D[r], np.arange(n), m_sample, wl.order)
        y = inputs.rhs_exp(X)
        k1 = o.first_column("dsi", wl.alpha, X, c, wl.zeta)
        lam = o.eigenvalues("dsi", k1, wl.eta)
        o.spectral_mll("dsi", lam, y, wl.zeta)
        o.spectral_mll_grad("dsi", wl.alpha, X, y, lam, c, wl.zeta)
        o.spectral_solve("dsi", lam, y)
    dt = time.perf_counter() - t0
    return count * n / dt, (f"{count} randomization(s) at n=2^{m_sample} (the workload has 2^{W_host['m']}), "
                            f"d={d}: oracle points, first column, spectrum, MLL, gradient and solve "
                            f"(numpy FP64, single thread, {dt:.1f} s)")


def workload_config(m, d, R, world):
    """The `config` object of both arms' JSON lines (the same workload)."""
    return {"workload": f"solve20: digital net (Gray, LMS+DS) n=2^{m}, d={d}, {R} randomizations/GPU, "
                        "DSI order 2, gamma_j=0.9^j, eta=1e-8, 1 rhs; FP32 column+FWHT, FP64 "
                        "division/logdet/variance, 1 refinement step",
            "global_batch": world * R, "seq_len": 1 << m, "parallelism": f"replicas x{world}",
            "l2": "inputs larger than L2 (y alone 256 MB)"}


def lattice_setup(qk, torch, dev, R, dt):
    """The differentiation workload's shape (rank-1 lattice n = 2^18, d = 32, SI kernel of
    smoothness 2, unit weights, nugget e^-12) as one planned batch task of R randomizations
    (shifts) in dtype dt: returns (workspace, status, points per run)."""
    from paper_2502_14256_gb300 import inputs
    wl = inputs.workload("diff")
    m, d = wl.ms[0], wl.d
    n = 1 << m
    lat = inputs.make_lattice(wl.seed, d, R, m)
    u32 = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).to(dev)  # noqa: E731
    gd, Dd = u32(lat.g), u32(lat.D)
    ps = qk.pointset(qk.QK_LATTICE, d, R, g=gd, D=Dd)
    w = torch.tensor(np.asarray(wl.gamma) * np.exp(wl.log_ls), dtype=torch.float64, device=dev)
    kern = qk.kernel(qk.QK_SI, wl.alpha, w, wl.zeta)
    X = torch.empty((R, n, d), dtype=torch.int32, device=dev)
    qk.gen_points(ps, 0, R, 0, n, X)
    x = (X.to(torch.int64) & 0xFFFFFFFF).to(torch.float64) * 2.0 ** -32
    jj = torch.arange(1, d + 1, dtype=torch.float64, device=dev)
    y64 = torch.prod(1.0 + (x - 0.5) / jj ** 2, dim=2).reshape(R, 1, n)
    del X, x
    y = y64.to(torch.float32).to(qk.data_dtype(dt)).contiguous()
    c = torch.empty_like(y)
    o = torch.empty((R, 1, qk.QK_MLL_NOUT), dtype=torch.float64, device=dev)
    g = torch.empty((R, 1, 2 * d + 2), dtype=torch.float64, device=dev)
    task = qk.Task(ps, kern, m, 1, wl.eta, y.data_ptr(), c.data_ptr(), None, o.data_ptr(), g.data_ptr())
    ws = qk.workspace(qk.batch_workspace_bytes([task], dt), dev)
    qk.batch_plan([task], dt, 1, ws)
    ws._keep = (ps, kern, gd, Dd, w, y, c, o, g)  # buffers the plan points at
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    return ws, status, R * n


def lattice_line(qk, torch, dev, stream, R=16):
    """The lattice setup (differentiation workload's shape) through the batched schedule:
    solve + MLL + gradient for R randomizations in FP64 and with the float-float first
    column; points/s and the time per op."""
    from paper_2502_14256_gb300 import inputs
    wl = inputs.workload("diff")
    out = {"workload": f"lattice n=2^{wl.ms[0]}, d={wl.d}, SI alpha={wl.alpha}, {R} shifts, nugget e^-12, 1 rhs",
           "points_per_step": R << wl.ms[0]}
    m, d = wl.ms[0], wl.d
    n = 1 << m
    # algorithmic FP64 flops of the FP64 step: column sweep 9 per (point, dimension) (the
    # factor x - x^2, its square and the polynomial, 5; the weight; p <- p + a + p a, 3),
    # gradient sweep 12 (the factor, 5; 1 + c K; the quotient; two accumulations, 4), 5 N
    # log2 N per complex transform of N (R/2 pairs each: eigenvalues, y forward; g and c
    # inverse), 20 per (frequency, vector) in the spectral step
    flops = R * n * d * (9 + 12) + 4 * (R // 2) * 5 * n * m + 20 * R * n
    for name, dt in (("fp64", torch.float64), ("f32w", qk.F32W)):
        ws, status, pts = lattice_setup(qk, torch, dev, R, dt)
        ms_ = time_steps(torch, lambda: qk.batch_run(ws, status), 3, 1, stream)
        qk.batch_timing(ws, 1)
        qk.batch_run(ws, status)
        per_op = {k: v[1] for k, v in qk.batch_kernel_ms(ws).items()}
        qk.batch_timing(ws, 0)
        out[name] = {"ms_per_step": ms_, "value": pts / (ms_ * 1e-3), "ops_ms": per_op}
        if name == "fp64":
            ach = flops / (ms_ * 1e-3) / 1e12
            out[name]["roofline"] = {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                                     "frac": ach / FP64_PEAK_TFLOPS, "scope": "whole step, algorithmic FP64 flops",
                                     "flops_per_step": flops,
                                     "peak_source": "nominal GB300 FP64 rate (1.25 TFLOP/s)"}
        del ws
    return out


# ------------------------------------------------------------- profile cases
def profile_case(args):
    """One small invocation of a hot kernel (1 warm-up + reps runs), for ncu -k ... -c ..."""
    import torch
    from paper_2502_14256_gb300 import build
    build.build()
    from paper_2502_14256_gb300 import inputs, qk
    dev = torch.device("cuda:0")
    R, m = args.R, args.m
    n = 1 << m
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    if args.profile == "fwht":
        x = torch.randn((R, n), dtype=torch.float32, device=dev)
        ws = qk.fwht_workspace(R, dev)
        plan = dict(mode=qk.QK_FWHT_TWO_PASS if args.two_pass else qk.QK_FWHT_PERSISTENT)
        run = lambda: qk.fwht_ws(m, x, ws, plan=plan, status=status)  # noqa: E731
    elif args.profile == "lattice":
        ws, lst, _ = lattice_setup(qk, torch, dev, R, torch.float64 if args.fp64 else qk.F32W)
        run = lambda: qk.batch_run(ws, lst)  # noqa: E731
    elif args.profile == "fftbr":
        x = torch.randn((R, 2 * n), dtype=torch.float64 if args.fp64 else torch.float32, device=dev)
        if args.persistent:
            fws = qk.fwht_workspace(R, dev)
            run = lambda: qk.fftbr_ws(m, x, ws=fws, status=status)  # noqa: E731
        else:
            run = lambda: qk.fftbr(m, x)  # noqa: E731
    else:
        wl = inputs.workload("solve20")
        d = args.d if args.profile in ("points", "col") else wl.d
        net = inputs.make_net(wl.seed, d, R, wl.order)
        u32 = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).to(dev)  # noqa: E731
        C, S, D = u32(net.C), u32(net.S), u32(net.D)
        Ct = torch.empty((R, d, 32), dtype=torch.int32, device=dev)
        qk.lms_setup(C, S, Ct)
        ps = qk.pointset(qk.QK_NET_B2, d, R, Ct=Ct, D=D, order=qk.QK_GRAY)
        w = torch.tensor(0.9 ** np.arange(1, d + 1), dtype=torch.float64, device=dev)
        kern = qk.kernel(qk.QK_DSI, wl.alpha, w, wl.zeta)
        if args.profile == "points":
            X = torch.empty((R, n, d), dtype=torch.int32, device=dev)
            run = lambda: qk.gen_points(ps, 0, R, 0, n, X)  # noqa: E731
        elif args.profile == "col":
            col = torch.empty((R, n), dtype=torch.float64 if (args.fp64 or args.wide) else torch.float32, device=dev)
            run = lambda: qk.kernel_col(ps, kern, 0, R, m, col, form=qk.QK_COL_P, wide=args.wide)  # noqa: E731
        else:
            dt = torch.float64 if args.fp64 else (qk.F32W if args.wide else torch.float32)
            g = torch.Generator(device=dev).manual_seed(wl.seed)
            y = torch.randn((R, 1, n), dtype=qk.data_dtype(dt), device=dev, generator=g)
            c = torch.empty_like(y)
            out = torch.empty((R, 1, qk.QK_MLL_NOUT), dtype=torch.float64, device=dev)
            grad = torch.empty((R, 1, 2 * d + 2), dtype=torch.float64, device=dev)
            task = qk.Task(ps, kern, m, 1, wl.eta, y.data_ptr(), c.data_ptr(), None, out.data_ptr(),
                           grad.data_ptr())
            ws = qk.workspace(qk.batch_workspace_bytes([task], dt))
            qk.batch_plan([task], dt, args.refine, ws)
            if args.persistent:
                qk.batch_schedule(ws, qk.QK_SCHED_PERSISTENT, 1)
            run = lambda: qk.batch_run(ws, status)  # noqa: E731
    for _ in range(1 + args.reps):
        run()
    torch.cuda.synchronize()
    qk.read_status(status)
    print("ok")
    return 0


# ---------------------------------------------------------------- main
def main():
    args = parse()
    if args.profile:
        return profile_case(args)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return 0
        from paper_2502_14256_gb300 import inputs
        wl = inputs.workload("solve20")
        net = inputs.make_net(wl.seed, wl.d, args.R, wl.order)
        W_host = dict(wl=wl, net=net, m=args.m, d=wl.d)
        times = []
        for q in range(args.warmup):
            oracle_sample(W_host, 10, 1, q)
        sample = ""
        for q in range(args.steps):
            v, sample = oracle_sample(W_host, min(16, args.m), 1, q)
            times.append(v)
        value = statistics.median(times)
        line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": workload_config(args.m, wl.d, args.R, args.gpus),
                "cpu_baseline": {"kind": "oracle", "value": value, "unit": UNIT, "cores": 1,
                                 "host_cores": os.cpu_count(), "sample": sample},
                "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return 0

    import torch
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    from paper_2502_14256_gb300 import build
    if rank == 0:
        build.build()
    if world > 1:
        dist.barrier()
    from paper_2502_14256_gb300 import qk

    W = build_workload(qk, torch, dev, args.R, args.m, seed_offset=replica_seed_offset(rank))
    stream = torch.cuda.current_stream()
    R, n, m, d = W["R"], W["n"], W["m"], W["d"]

    # ---- the headline: FP32-refined pipeline, device-resident inputs
    P32 = Pipeline(qk, torch, dev, W, torch.float32, refine=args.refine)
    if args.sched == "persistent":
        qk.batch_schedule(P32.ws, qk.QK_SCHED_PERSISTENT, args.lag)
    sched = {"mode": args.sched, "lag": args.lag if args.sched == "persistent" else 0}
    if args.sched == "auto":  # the library's schedule tuner picks launches vs one persistent launch
        sched = qk.batch_tune(P32.ws)
    for _ in range(args.warmup):
        P32.step()
    qk.read_status(P32.status)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    launches0 = qk.launch_count()
    ms = time_steps(torch, P32.step, args.steps, 0, stream)
    launches = qk.launch_count() - launches0
    clocks = sampler.stop()
    if world > 1:
        dist.barrier()
    ms = max_over_ranks(ms, torch, dist, world, dev)
    points_step = world * R * n
    value = job_throughput(R * n, world, ms)
    # per-kernel times of the same step, in a separate pass with CUDA events around each kernel
    kernel_ms = P32.kernel_ms(torch, args.steps, stream)

    # ---- end to end through the public API with host buffers (pinned)
    y_host = P32.y.cpu().pin_memory()
    c_host = torch.empty_like(P32.c, device="cpu").pin_memory()
    o_host = torch.empty_like(P32.out, device="cpu").pin_memory()
    g_host = torch.empty_like(P32.grad, device="cpu").pin_memory()
    host_io = [dict(y=y_host, c=c_host, out=o_host, grad=g_host)]

    chunk = {"r": args.e2e_chunk}

    def e2e_step():
        # the library's host path: chunks of randomizations copied in, computed and copied
        # back on overlapping streams
        qk.batch_run_host(P32.ws, host_io, chunk["r"], P32.status, stream=stream)

    if args.e2e_chunk == 0:
        # pick the chunk size (a chunk's kernels fill whole waves of resident CTAs only for
        # some sizes) by timing a few, before the timed region
        tried = {}
        for cr in (3, 4, 6, 8, 14, 16, 21, 32):
            if cr <= R:
                chunk["r"] = cr
                tried[cr] = time_steps(torch, e2e_step, 4, 1, stream)
        chunk["r"] = min(tried, key=tried.get)
    e2e_ms = time_steps(torch, e2e_step, max(2, args.steps // 2), 1, stream)
    e2e_ms = max_over_ranks(e2e_ms, torch, dist, world, dev)
    h2d = y_host.numel() * y_host.element_size()
    d2h = sum(t.numel() * t.element_size() for t in (c_host, o_host, g_host))
    del y_host, c_host, o_host, g_host, host_io

    # ---- stage timing of the FP32 path (which stage dominates)
    col = torch.empty((R, n), dtype=torch.float32, device=dev)
    kern = qk.kernel(qk.QK_DSI, W["wl"].alpha, W["w"], W["wl"].zeta)
    stage = {"kernel_col": time_steps(torch, lambda: qk.kernel_col(W["ps"], kern, 0, R, m, col, form=qk.QK_COL_P),
                                      3, 1, stream)}
    # doubling update (extensible n): eigenvalues of the 2^m-point sets from those of their
    # first 2^(m-1) points plus the new half's column and one half-length transform,
    # against computing the full column and transform
    lam_full = torch.empty((R, n), dtype=torch.float64, device=dev)
    lam_half = torch.empty((R, n // 2), dtype=torch.float64, device=dev)
    col_half = torch.empty((R, n // 2), dtype=torch.float32, device=dev)
    ws_e = qk.workspace(qk.workspace_bytes(qk.OP_EIGS, qk.QK_DSI, m, R, 1, torch.float32), dev)
    eta_ = W["wl"].eta

    def eig_full():
        qk.kernel_col(W["ps"], kern, 0, R, m, col, form=qk.QK_COL_P)
        qk.eigs(qk.QK_DSI, m, col, lam_full, zeta=W["wl"].zeta, eta=eta_, form=qk.QK_COL_P, ws=ws_e)

    qk.kernel_col(W["ps"], kern, 0, R, m - 1, col_half, form=qk.QK_COL_P)
    qk.eigs(qk.QK_DSI, m - 1, col_half, lam_half, zeta=W["wl"].zeta, eta=eta_, form=qk.QK_COL_P, ws=ws_e)

    def eig_extend():
        qk.kernel_col_at(W["ps"], kern, 0, R, n // 2, m - 1, col_half, form=qk.QK_COL_P)
        qk.eigs_extend(qk.QK_DSI, m - 1, col_half, lam_half, lam_full, zeta=W["wl"].zeta, eta=eta_,
                       form=qk.QK_COL_P, ws=ws_e)

    doubling = {"eigs_full_ms": time_steps(torch, eig_full, 3, 1, stream),
                "eigs_extend_ms": time_steps(torch, eig_extend, 3, 1, stream),
                "what": f"{R} x 2^{m} FP32 column + eigenvalues: from scratch vs from the first 2^{m - 1} points"}
    del lam_full, lam_half, col_half, ws_e, col

    peaks = {}
    pk_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk_path):
        peaks = json.load(open(pk_path))
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    src_hash = kernel_source_hash()
    ncu_ok = NCU_TRAFFIC["src_hash"] == src_hash and (R, m, d) == (64, 20, 16)

    # ---- point generation (a2): 32-bit words of every point, stored (R, n, d)
    Xp = torch.empty((R, n, d), dtype=torch.int32, device=dev)
    gen_ms = time_steps(torch, lambda: qk.gen_points(W["ps"], 0, R, 0, n, Xp), max(3, args.steps // 2), 1, stream)
    gen_bytes = 4 * R * n * d
    points = {"gbs": gen_bytes / (gen_ms * 1e-3) / 1e9, "ms": gen_ms, "bytes": gen_bytes,
              "frac_of_hbm": gen_bytes / (gen_ms * 1e-3) / 1e9 / hbm_peak, "peak": hbm_peak, "peak_source": peak_src,
              "shape": f"{R} x 2^{m} x {d} u32 (Gray order, LMS + digital shift), store-bound: 4 n d R bytes"}
    del Xp

    # FWHT alone on the same data volume (in place, FP32): HBM roofline of the transform
    xf = torch.randn((R, n), dtype=torch.float32, device=dev)
    fw_ws = qk.fwht_workspace(R, dev)
    fw_plan = qk.fwht_tune(m, xf, fw_ws)  # autotuned plan (xf is scratch here)
    fw_ms = time_steps(torch, lambda: qk.fwht_ws(m, xf, fw_ws), args.steps, 2, stream)
    fw2_ms = time_steps(torch, lambda: qk.fwht(m, xf), args.steps, 2, stream)
    fw_bytes = 2 * xf.numel() * 4  # one read + one write per element (the algorithmic minimum)
    fw_gbs = fw_bytes / (fw_ms * 1e-3) / 1e9
    del xf, fw_ws
    # FFTBR (the lattice transform) on R complex FP32 vectors of the same length
    xc = torch.randn((R, 2 * n), dtype=torch.float32, device=dev)
    ff_ws = qk.fwht_workspace(R, dev)
    ff_ms = time_steps(torch, lambda: qk.fftbr_ws(m, xc, ws=ff_ws), args.steps, 2, stream)
    ff2_ms = time_steps(torch, lambda: qk.fftbr(m, xc), args.steps, 2, stream)
    ff_bytes = 2 * xc.numel() * 4
    del xc, ff_ws

    # ---- the lattice (SI) path on the differentiation workload's shape
    lattice = lattice_line(qk, torch, dev, stream)

    # ---- the same step with the float-float first column (QK_F32W): its cost beside the headline
    PW = Pipeline(qk, torch, dev, W, qk.F32W, refine=args.refine, keep_lam=True)
    wide_ms = time_steps(torch, PW.step, max(3, args.steps // 2), 1, stream)
    wide = {"value": points_step / (wide_ms * 1e-3), "ms_per_step": wide_ms, "cost_vs_headline": wide_ms / ms,
            "kernels_ms_per_step": {k: v[1] for k, v in PW.kernel_ms(torch, 2, stream).items()}}

    # ---- plain FP64 pipeline beside it
    fp64 = None
    if not args.no_fp64:
        P64 = Pipeline(qk, torch, dev, W, torch.float64, refine=0, keep_lam=True)
        ms64 = time_steps(torch, P64.step, max(1, min(3, args.steps)), 1, stream)
        fp64 = {"value": points_step / (ms64 * 1e-3), "ms_per_step": ms64}
        k64 = P64.kernel_ms(torch, 1, stream)
        top64, (l64, t64) = max(k64.items(), key=lambda kv: kv[1][1])
        # FP64 FMA-pipe roofline of the FP64 path's longest kernel (algorithmic flops per
        # point below; 12-bit tile transforms in FP64)
        fl64 = {"k_fused_A": 8 * d + 2 * 12 + 2, "k_fused_C": 10 * d + 2 * 12 + 3}.get(top64)
        if fl64:
            ach = fl64 * R * n / (t64 / max(1.0, l64) * 1e-3) / 1e12
            fp64["roofline"] = {"kernel": top64, "bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS,
                                "unit": "TFLOP/s", "frac": ach / FP64_PEAK_TFLOPS,
                                "peak_source": "nominal GB300 FP64 rate (1.25 TFLOP/s)", "ms_per_launch": t64 / max(1.0, l64)}
        fp64["kernels_ms_per_step"] = {k: v[1] for k, v in k64.items()}
        # accuracy of the FP32 paths against the FP64 GPU path, per output (one untimed
        # FP32 run that also writes its eigenvalues)
        P32L = Pipeline(qk, torch, dev, W, torch.float32, refine=args.refine, keep_lam=True)
        P32L.step()
        PW.step()
        torch.cuda.synchronize()
        rel = lambda a, b: float((a.double() - b.double()).abs().max() / b.double().abs().max())  # noqa: E731
        for name, P in (("fp32_rel_err", P32L), ("wide_rel_err", PW)):
            errs = {"solve_c": rel(P.c, P64.c), "lambda": rel(P.lam, P64.lam),
                    "lambda_elementwise": float(((P.lam - P64.lam).abs() / P64.lam).max()),
                    "quad": rel(P.out[..., 0], P64.out[..., 0]), "logdet": rel(P.out[..., 1], P64.out[..., 1]),
                    "mll": rel(P.out[..., 2], P64.out[..., 2]), "post_mean": rel(P.out[..., 3], P64.out[..., 3]),
                    "post_var": rel(P.out[..., 4], P64.out[..., 4]), "grad_dc": rel(P.grad[..., :d], P64.grad[..., :d])}
            if name == "wide_rel_err":
                wide["rel_err_vs_fp64"] = errs
            else:
                fp64[name] = errs
        del P64, P32L
    del PW

    # ---- roofline of the dominant kernel of the timed step
    top_name, (top_launches, top_ms_step) = max(kernel_ms.items(), key=lambda kv: kv[1][1])
    top_ms = top_ms_step / max(1.0, top_launches)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    clk = (clocks.get("sm_max_mhz") or 2070.0) * 1e6
    # FP32 non-tensor peak from unit counts and clock: SMs x 128 FP32 lanes x 2 flop/FMA x clock
    fp32_peak = sms * 128 * 2 * clk / 1e12
    # algorithmic work per launch (per point and right-hand side, DSI order 2):
    #   gradient sweep 10 flops per dimension (K, f = 1 + c K, K/f, two accumulations),
    #   column sweep 8 flops per dimension (K, a = c K, p update),
    #   13-bit tile transforms 13 adds per vector.
    flops_per_point = {"k_fused_C": 10 * d + 2 * 13 + 3, "k_fused_A": 8 * d + 2 * 13 + 2}
    roof = None
    if top_name in flops_per_point:
        work = flops_per_point[top_name] * R * n
        ach = work / (top_ms * 1e-3) / 1e12
        tr = NCU_TRAFFIC["bytes_r64"].get(top_name) if ncu_ok else None
        roof = {"kernel": top_name, "bound": "alu", "achieved": ach, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": ach / fp32_peak, "traffic": tr,
                "traffic_source": (f"ncu dram__bytes_read.sum + dram__bytes_write.sum of this kernel, "
                                   f"sources {NCU_TRAFFIC['src_hash']}") if tr else "null: no capture of these sources",
                "ms_per_launch": top_ms,
                "peak_source": f"derived: {sms} SMs x 128 FP32 lanes x 2 flop x {clk / 1e9:.2f} GHz (sampled max clock)",
                "algorithmic_bytes": 20 * R * n if top_name == "k_fused_A" else 16 * R * n}

    cpu = None
    if rank == 0 and not args.no_cpu:
        v, sample = oracle_sample(W, min(18, m), 2, 0)  # ~10 s of host work
        cpu = {"value": v, "unit": UNIT, "cores": 1, "host_cores": os.cpu_count(), "kind": "oracle",
               "sample": sample}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(m, d, R, world),
            "e2e": {"value": points_step / (e2e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms, "chunk_r": chunk["r"]},
            "gpu_launches": launches,
            "gpu_launches_per_step": launches / max(1, args.steps),
            "fp64_plain": fp64,
            "wide": wide,
            "lattice": lattice,
            "schedule": sched,
            "stages_ms": stage,
            "doubling": doubling,
            "kernels_ms_per_step": {k: v[1] for k, v in kernel_ms.items()},
            "points": points,
            "fwht": {"gbs": fw_gbs, "ms": fw_ms, "frac_of_hbm": fw_gbs / hbm_peak, "bytes": fw_bytes,
                     "peak": hbm_peak, "peak_source": peak_src,
                     "shape": f"{R} x 2^{m} fp32, in place", "plan": fw_plan,
                     "traffic": NCU_TRAFFIC["fwht_bytes"] if ncu_ok else None,
                     "two_launch_ms": fw2_ms, "two_launch_gbs": fw_bytes / (fw2_ms * 1e-3) / 1e9},
            "fftbr": {"gbs": ff_bytes / (ff_ms * 1e-3) / 1e9, "ms": ff_ms, "bytes": ff_bytes,
                      "frac_of_hbm": ff_bytes / (ff_ms * 1e-3) / 1e9 / hbm_peak,
                      "shape": f"{R} x 2^{m} complex fp32, in place, both tile passes in one persistent launch",
                      "two_launch_ms": ff2_ms, "two_launch_gbs": ff_bytes / (ff2_ms * 1e-3) / 1e9},
            "roofline": roof,
            "kernel_sources": src_hash,
            "cpu_baseline": cpu,
            "clocks": clocks,
        }
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
