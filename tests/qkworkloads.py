"""Device-side builders for the named workloads (inputs.workload / inputs.mixed_batch):
generator columns, shifts and right-hand sides uploaded as the C ABI expects, plus the
host copies the oracle needs for sampled checks."""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import torch

from paper_2502_14256_gb300 import inputs


def _dev():
    return torch.device("cuda:0")


def _u32(a):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.uint32)).view(np.int32)).to(_dev())


@dataclass
class Inst:
    wl: inputs.Workload
    m: int
    R: int
    nrhs: int
    ps: object
    kern: object
    net: object = None
    lat: object = None
    keep: list = field(default_factory=list)
    y64: torch.Tensor = None


def build_instance(qk, wl, m, R, nrhs, seed_shift=0, y_kind=None):
    """Upload one instance (R randomizations, n = 2^m) and build y (R, nrhs, n) in FP64 on
    the device from the points: prod(1 + (x_j - 1/2)/j^2) or exp(sum x_j/j) - const + noise."""
    d = wl.d
    n = 1 << m
    keep = []
    if wl.kind == "net":
        net = inputs.make_net(wl.seed + seed_shift, d, R, wl.order)
        Cd, Sd, Dd = _u32(net.C), _u32(net.S), _u32(net.D)
        Ct = torch.empty((R, d, 32), dtype=torch.int32, device=_dev())
        qk.lms_setup(Cd, Sd, Ct)
        keep += [Cd, Sd, Dd, Ct]
        ps = qk.pointset(qk.QK_NET_B2, d, R, Ct=Ct, D=Dd, order=qk.QK_GRAY if wl.order == "gray" else qk.QK_NATURAL)
        lat = None
    else:
        lat = inputs.make_lattice(wl.seed + seed_shift, d, R, wl.extra.get("m_gen", m))
        gd, Dd = _u32(lat.g), _u32(lat.D)
        keep += [gd, Dd]
        ps = qk.pointset(qk.QK_LATTICE, d, R, g=gd, D=Dd)
        net = None
    c = np.asarray(wl.gamma) * np.exp(wl.log_ls)
    w = torch.tensor(c, dtype=torch.float64, device=_dev())
    keep.append(w)
    kern = qk.kernel(qk.QK_DSI if wl.family == "dsi" else qk.QK_SI, wl.alpha, w, wl.zeta)
    y = torch.empty((R, nrhs, n), dtype=torch.float64, device=_dev())
    X = torch.empty((1, n, d), dtype=torch.int32, device=_dev())
    jj = torch.arange(1, d + 1, dtype=torch.float64, device=_dev())
    const = float(np.prod(np.arange(1, d + 1) * np.expm1(1.0 / np.arange(1, d + 1))))
    kind = y_kind or wl.rhs
    # seeded Gaussian noise (an input, drawn by torch's generator; kept for the oracle side)
    gen = torch.Generator(device=_dev()).manual_seed(wl.seed + 77 + seed_shift)
    noise = None
    if kind == "exp" and wl.noise_sigma:
        noise = wl.noise_sigma * torch.randn((R, nrhs, n), dtype=torch.float64, device=_dev(), generator=gen)
    for r in range(R):
        qk.gen_points(ps, r, 1, 0, n, X)
        x = (X[0].to(torch.int64) & 0xFFFFFFFF).to(torch.float64) * 2.0 ** -32
        if kind == "exp":
            base = torch.exp((x / jj).sum(dim=1)) - const
            for q in range(nrhs):
                y[r, q] = base + (noise[r, q] if noise is not None else 0.0)
        else:
            base = torch.prod(1.0 + (x - 0.5) / jj ** 2, dim=1)
            for q in range(nrhs):
                y[r, q] = base * (1.0 + 0.1 * q)
    inst = Inst(wl, m, R, nrhs, ps, kern, net, lat, keep, y)
    inst.noise = noise
    inst.kind = kind
    return inst


def host_rhs(inst, r, X):
    """The right-hand sides of randomization r recomputed on the host from oracle points X
    (same formulas, same noise values)."""
    d = X.shape[1]
    n = X.shape[0]
    out = np.empty((inst.nrhs, n))
    if inst.kind == "exp":
        base = inputs.rhs_exp(X)
        for q in range(inst.nrhs):
            out[q] = base + (inst.noise[r, q].cpu().numpy() if inst.noise is not None else 0.0)
    else:
        base = inputs.rhs_product(X)
        for q in range(inst.nrhs):
            out[q] = base * (1.0 + 0.1 * q)
    return out


def host_points(inst, r, idx):
    """Oracle points of randomization r at positions idx (for sampled checks)."""
    from oracle import qk_oracle as o
    if inst.net is not None:
        Ct = o.lms_scramble(inst.net.C, inst.net.S[r:r + 1])[0]
        return o.net_points(Ct, inst.net.D[r], idx, inst.m, inst.wl.order)
    return o.lattice_points(inst.lat.g, inst.lat.D[r], idx)


def outputs(qk, inst, dtype, with_c=True, with_lam=True, with_grad=True, y_via=None, eta=None):
    """Output buffers and the task for one instance; dtype is a torch dtype or qk.F32W (FP32
    arrays); y_via rounds y through another dtype first (so that an FP64 run sees exactly the
    FP32 path's input); eta overrides the workload's nugget."""
    R, n, d = inst.R, 1 << inst.m, inst.wl.d
    y = (inst.y64.to(y_via) if y_via is not None else inst.y64).to(qk.data_dtype(dtype)).contiguous()
    bufs = {
        "y": y,
        "c": torch.zeros_like(y) if with_c else None,
        "lam": torch.zeros((R, n), dtype=torch.float64, device=_dev()) if with_lam else None,
        "out": torch.zeros((R, inst.nrhs, 5), dtype=torch.float64, device=_dev()),
        "grad": torch.zeros((R, inst.nrhs, 2 * d + 2), dtype=torch.float64, device=_dev()) if with_grad else None,
    }
    p = lambda t: t.data_ptr() if t is not None else None  # noqa: E731
    task = qk.Task(inst.ps, inst.kern, inst.m, inst.nrhs, inst.wl.eta if eta is None else eta, p(bufs["y"]), p(bufs["c"]), p(bufs["lam"]),
                   p(bufs["out"]), p(bufs["grad"]))
    return task, bufs


def run_tasks(qk, tasks, dtype, refine=0, graph=False, allow_floor=False, persistent=False):
    """Plan and run one schedule over tasks; optionally as ONE persistent launch
    (QK_SCHED_PERSISTENT), and optionally captured in a CUDA graph and replayed.
    Returns the workspace and the device status word (read and cleared here)."""
    ws = qk.workspace(qk.batch_workspace_bytes(tasks, dtype))
    status = torch.zeros(1, dtype=torch.int32, device=_dev())
    qk.batch_plan(tasks, dtype, refine, ws)
    if persistent:
        qk.batch_schedule(ws, qk.QK_SCHED_PERSISTENT, 1)
    if graph:
        qk.batch_run(ws, status)  # first call: module loading and shared-memory opt-ins
        torch.cuda.synchronize()
        s = torch.cuda.Stream()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                qk.batch_run(ws, status, stream=s)
        g.replay()
    else:
        qk.batch_run(ws, status)
    torch.cuda.synchronize()
    word = int(status.item())
    assert allow_floor or not word & qk.QK_STATUS_FLOOR, "an eigenvalue fell below the nugget"
    qk.read_status(status)
    return ws, word
