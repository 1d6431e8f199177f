"""Small, self-contained invocations of the library's hot kernels, for profiling one kernel
under a profiler (ncu -k <kernel> -c <n>) with inputs sized like the benchmark workload.

    python -m paper_2502_14256_gb300.profile_cases fwht  --m 20 --R 64 [--two-pass]
    python -m paper_2502_14256_gb300.profile_cases fftbr --m 20 --R 64 [--fp64]
    python -m paper_2502_14256_gb300.profile_cases fused --m 20 --R 8  [--refine 0|1] [--fp64] [--persistent]

`fwht` transforms R vectors of 2^m FP32 values in place (qk_fwht_ws, persistent plan with
the default lag unless --two-pass); `fused` runs the batched solve + MLL + gradient
schedule of the solve20 workload (DSI order 2, d = 16) on R randomizations.  Each case
runs `--reps` times after one warm-up and exits 0 on success.
"""
from __future__ import annotations

import argparse

import torch

from . import inputs, qk


def _fwht(args):
    x = torch.randn((args.R, 1 << args.m), dtype=torch.float32, device="cuda")
    ws = qk.fwht_workspace(args.R)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    plan = dict(mode=qk.QK_FWHT_TWO_PASS) if args.two_pass else dict(mode=qk.QK_FWHT_PERSISTENT)
    for _ in range(1 + args.reps):
        qk.fwht_ws(args.m, x, ws, plan=plan, status=status)
    torch.cuda.synchronize()
    qk.read_status(status)


def _fftbr(args):
    x = torch.randn((args.R, 2 << args.m), dtype=torch.float64 if args.fp64 else torch.float32, device="cuda")
    for _ in range(1 + args.reps):
        qk.fftbr(args.m, x)
    torch.cuda.synchronize()


def _fused(args):
    wl = inputs.workload("solve20")
    d, R, n = wl.d, args.R, 1 << args.m
    net = inputs.make_net(wl.seed, d, R, wl.order)
    u32 = lambda a: torch.from_numpy(a.astype("uint32").view("int32")).cuda()  # noqa: E731
    C, S, D = u32(net.C), u32(net.S), u32(net.D)
    Ct = torch.empty((R, d, 32), dtype=torch.int32, device="cuda")
    qk.lms_setup(C, S, Ct)
    ps = qk.pointset(qk.QK_NET_B2, d, R, Ct=Ct, D=D, order=qk.QK_GRAY)
    w = torch.tensor(wl.gamma, dtype=torch.float64, device="cuda")
    kern = qk.kernel(qk.QK_DSI, wl.alpha, w, wl.zeta)
    dt = torch.float64 if args.fp64 else torch.float32
    g = torch.Generator(device="cuda").manual_seed(wl.seed)
    y = torch.randn((R, 1, n), dtype=dt, device="cuda", generator=g)
    c = torch.empty_like(y)
    out = torch.empty((R, 1, qk.QK_MLL_NOUT), dtype=torch.float64, device="cuda")
    grad = torch.empty((R, 1, 2 * d + 2), dtype=torch.float64, device="cuda")
    task = qk.Task(ps, kern, args.m, 1, wl.eta, y.data_ptr(), c.data_ptr(), None, out.data_ptr(), grad.data_ptr())
    ws = qk.workspace(qk.batch_workspace_bytes([task], dt))
    qk.batch_plan([task], dt, args.refine, ws)
    if args.persistent:
        qk.batch_schedule(ws, qk.QK_SCHED_PERSISTENT, 1)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    for _ in range(1 + args.reps):
        qk.batch_run(ws, status)
    torch.cuda.synchronize()
    qk.read_status(status)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("case", choices=["fwht", "fftbr", "fused"])
    ap.add_argument("--m", type=int, default=20)
    ap.add_argument("--R", type=int, default=8)
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--refine", type=int, default=1)
    ap.add_argument("--fp64", action="store_true")
    ap.add_argument("--two-pass", action="store_true")
    ap.add_argument("--persistent", action="store_true", help="fused: one persistent launch")
    args = ap.parse_args(argv)
    {"fwht": _fwht, "fftbr": _fftbr, "fused": _fused}[args.case](args)
    print("ok")


if __name__ == "__main__":
    main()
