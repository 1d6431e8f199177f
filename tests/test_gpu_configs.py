"""The named workloads at their full sizes, through the batched C-ABI schedule, checked on
sampled outputs against the FP64 oracle (sampled because the oracle's spectral gradient is
O(d^2 n) and its dense forms O(n^3)) and, for the precision workload, FP32-refined against
the FP64 GPU path.  Oracle inputs are recomputed on the host from the oracle's own points."""
import math
import time

import numpy as np
import pytest
import torch

from oracle import qk_oracle as o
from paper_2502_14256_gb300 import inputs
from tests import qkcases as qc
from tests import qkworkloads as W

pytestmark = pytest.mark.gpu
F64, F32 = torch.float64, torch.float32


@pytest.fixture(scope="module")
def qk():
    from paper_2502_14256_gb300 import build
    build.build()
    from paper_2502_14256_gb300 import qk as q
    return q


def _oracle_check(inst, bufs, r, rhs_list, tol, check_grad=True, y_fp32=False):
    """Compare randomization r (given right-hand sides) with the oracle's spectral formulas;
    y_fp32: the GPU ran on y rounded to FP32, so the oracle takes the same rounded y."""
    fam = inst.wl.family
    n = 1 << inst.m
    X = W.host_points(inst, r, np.arange(n))
    c_w = o.effective_weights(inst.wl.gamma, inst.wl.log_ls)
    k1 = o.first_column(fam, inst.wl.alpha, X, c_w, inst.wl.zeta)
    lam = o.eigenvalues(fam, k1, inst.wl.eta)
    Y = W.host_rhs(inst, r, X)
    if y_fp32:
        Y = Y.astype(np.float32).astype(np.float64)
    got_lam = bufs["lam"][r].cpu().numpy() if bufs["lam"] is not None else None
    if got_lam is not None:
        assert qc.rel_err(got_lam, lam) < tol["lam"]
    cond = float(lam.max() / lam.min())
    for q in rhs_list:
        sp = o.spectral_mll(fam, lam, Y[q], inst.wl.zeta)
        go = bufs["out"][r, q].cpu().numpy()
        assert abs(go[0] - sp["quad"]) < tol["quad"] * abs(sp["quad"]), (go[0], sp["quad"])
        assert abs(go[1] - sp["logdet"]) < tol["logdet"] * abs(sp["logdet"])
        assert abs(go[2] - sp["mll"]) < tol["mll"] * abs(sp["mll"])
        assert abs(go[3] - sp["post_mean"]) < tol["mean"] * max(1.0, abs(sp["post_mean"]))
        if bufs["c"] is not None:
            c_ref = o.spectral_solve(fam, lam, Y[q])
            ctol = max(tol["c"], 20 * cond * qc.EPS64)
            assert qc.rel_err(bufs["c"][r, q].cpu().numpy(), c_ref) < ctol
        if check_grad and bufs["grad"] is not None:
            gr = o.spectral_mll_grad(fam, inst.wl.alpha, X, Y[q], lam, c_w, inst.wl.zeta)
            gg = bufs["grad"][r, q].cpu().numpy()
            d = inst.wl.d
            assert qc.rel_err(gg[:d], gr["dc"]) < tol["grad"], qc.rel_err(gg[:d], gr["dc"])
            assert abs(gg[d] - gr["deta"]) < tol["grad"] * max(1.0, abs(gr["deta"]))


TOL64 = dict(lam=1e-11, quad=1e-10, logdet=1e-11, mll=1e-10, mean=1e-10, c=1e-10, grad=1e-9)


def test_plain_workload_against_dense_oracle(qk):
    """n = 2^10, d = 4, order-1 DSI, FP64: every output against Cholesky / dense gradient."""
    wl = inputs.workload("plain")
    inst = W.build_instance(qk, wl, wl.ms[0], 1, 1, y_kind="product")
    task, bufs = W.outputs(qk, inst, F64)
    W.run_tasks(qk, [task], F64)
    n = 1 << inst.m
    X = W.host_points(inst, 0, np.arange(n))
    y = W.host_rhs(inst, 0, X)[0]
    K = o.gram_dense("dsi", wl.alpha, X, o.effective_weights(wl.gamma, wl.log_ls), wl.zeta, wl.eta)
    c_ref, logdet = o.cholesky_solve(K, y)
    mll = o.mll_dense(K, y)[0]
    mean, var = o.bc_posterior_dense(K, y, wl.zeta)
    g = o.mll_grad_dense("dsi", wl.alpha, X, y, wl.gamma, wl.log_ls, wl.eta, wl.zeta)
    out = bufs["out"][0, 0].cpu().numpy()
    assert qc.rel_err(bufs["c"][0, 0].cpu().numpy(), c_ref) < 1e-10
    assert abs(out[1] - logdet) < 1e-10 * abs(logdet)
    assert abs(out[2] - mll) < 1e-10 * abs(mll)
    assert abs(out[3] - mean) < 1e-10 * max(1, abs(mean))
    assert abs(out[4] - var) < 1e-10
    grad = bufs["grad"][0, 0].cpu().numpy()
    assert qc.rel_err(grad[:wl.d], g["dc"]) < 1e-9


def test_batch_workload_full_size(qk):
    """32 instances, m in 14..20, d = 16, 64 randomizations, 8 right-hand sides, order-2 DSI,
    FP64, the whole plan as ONE persistent launch (QK_SCHED_PERSISTENT) captured in a CUDA
    graph and replayed; sampled instances against the oracle."""
    wl = inputs.workload("batch")
    t0 = time.time()
    insts = [W.build_instance(qk, wl, m, wl.R, wl.nrhs, seed_shift=i) for i, m in enumerate(wl.ms)]
    small = int(np.argmin(wl.ms))
    big = int(np.argmax(wl.ms))
    # solutions and eigenvalues are requested for the sampled instances only (memory)
    tasks, bufs = zip(*[W.outputs(qk, inst, F64, with_c=i in (small, big), with_lam=i in (small, big))
                        for i, inst in enumerate(insts)])
    t1 = time.time()
    W.run_tasks(qk, list(tasks), F64, graph=True, persistent=True)
    t2 = time.time()
    print(f"\nbatch workload: {sum(1 << i.m for i in insts) * wl.R} points, inputs {t1 - t0:.1f} s, "
          f"schedule (plan, first run, graph replay) {t2 - t1:.2f} s")
    _oracle_check(insts[small], bufs[small], 0, range(wl.nrhs), TOL64)
    _oracle_check(insts[small], bufs[small], 37, [3, 7], TOL64)
    _oracle_check(insts[big], bufs[big], 63, [5], TOL64, check_grad=False)


def test_differentiation_workload_full_size(qk):
    """Lattice n = 2^18, d = 32, SI alpha = 2, log-lengthscales 0, nugget e^-12, FP64 MLL and
    gradient against the oracle's spectral formulas."""
    wl = inputs.workload("diff")
    inst = W.build_instance(qk, wl, wl.ms[0], 1, 1, y_kind="product")
    task, bufs = W.outputs(qk, inst, F64)
    W.run_tasks(qk, [task], F64)
    tol = dict(TOL64, grad=1e-8)
    _oracle_check(inst, bufs, 0, [0], tol)


def _rel(a, b):
    """Max-norm relative difference of a against b."""
    a, b = a.double(), b.double()
    return float((a - b).abs().max() / b.abs().max())


def test_precision_workload_fp32_refined_against_fp64(qk):
    """Net n = 2^24, d = 64, order-4 DSI, gamma_j = j^-3, nugget 1e-8, all 16 randomizations:
    the FP32 path with the float-float first column (QK_F32W) and one refinement step against
    the FP64 GPU path on the same FP32 right-hand side.  Spectrum-weighted outputs (quadratic
    form, log det, MLL, posterior mean and variance) within 1e-5; the solve and the gradient
    within max(1e-5, 20 cond eps64), the FP64 path's own forward-error scale; every eigenvalue
    element-wise within 1e-5 relative.  The first column is also checked against the oracle
    at sampled positions (the oracle's dense forms do not reach 2^24 points)."""
    wl = inputs.workload("precision")
    inst = W.build_instance(qk, wl, wl.ms[0], wl.R, 1, y_kind="product")
    n, d = 1 << inst.m, wl.d
    tw, bw = W.outputs(qk, inst, qk.F32W)
    _, word_w = W.run_tasks(qk, [tw], qk.F32W, refine=1, allow_floor=True)
    t64, b64 = W.outputs(qk, inst, F64, y_via=F32)
    _, word64 = W.run_tasks(qk, [t64], F64, allow_floor=True)
    assert not (word_w | word64) & qk.QK_STATUS_FLOOR, (word_w, word64)  # no eigenvalue reached the nugget
    worst, failures = {}, []
    for r in range(wl.R):
        lam64 = b64["lam"][r]
        cond = float(lam64.max() / lam64.min())
        loose = max(1e-5, 20 * cond * qc.EPS64)
        # every eigenvalue within 1e-5 relative or the float-float column's own floor
        floor = qc.ff_column_floor(lam64.cpu().numpy(), d)
        excess = float(((bw["lam"][r] - lam64).abs() - 1e-5 * lam64 - floor).max())
        errs = {"lambda_elementwise": float(((bw["lam"][r] - lam64).abs() / lam64).max()),
                "lambda_floor_rel": floor / float(lam64.min()),
                "quad": _rel(bw["out"][r, :, 0], b64["out"][r, :, 0]),
                "logdet": _rel(bw["out"][r, :, 1], b64["out"][r, :, 1]),
                "mll": _rel(bw["out"][r, :, 2], b64["out"][r, :, 2]),
                "post_mean": _rel(bw["out"][r, :, 3], b64["out"][r, :, 3]),
                "post_var": _rel(bw["out"][r, :, 4], b64["out"][r, :, 4]),
                "solve": _rel(bw["c"][r], b64["c"][r]),
                "grad": _rel(bw["grad"][r, :, :d], b64["grad"][r, :, :d])}
        print(f"\n  r={r} cond={cond:.2e} " + " ".join(f"{k}={v:.2e}" for k, v in errs.items()), end="")
        if excess > 0:
            failures.append((r, "lambda", excess))
        for k, v in errs.items():
            worst[k] = max(worst.get(k, 0.0), v)
            if k.startswith("lambda"):
                continue
            bound = loose if k in ("solve", "grad") else 1e-5
            if not v < bound:
                failures.append((r, k, v, bound))
    print("\nprecision workload (16 randomizations), QK_F32W vs FP64 GPU, worst: " +
          " ".join(f"{k}={v:.2e}" for k, v in worst.items()))
    assert not failures, failures
    # first column at sampled positions against the oracle (both GPU precisions)
    rng = np.random.default_rng(24)
    idx = np.concatenate([[0], np.sort(rng.choice(np.arange(1, n), 4095, replace=False))])
    X = W.host_points(inst, 3, idx)
    k1_ref = o.first_column("dsi", wl.alpha, X, o.effective_weights(wl.gamma, wl.log_ls), wl.zeta)
    for wide in (False, True):
        col = torch.empty((1, n), dtype=F64, device=qc.dev())
        qk.kernel_col(inst.ps, inst.kern, 3, 1, inst.m, col, wide=wide)
        got = col[0, torch.from_numpy(idx).to(qc.dev())].cpu().numpy()
        assert qc.rel_err(got, k1_ref) < (1e-13 if wide else 1e-14), (wide, qc.rel_err(got, k1_ref))


def test_solve20_workload_full_size(qk):
    """The benchmark's workload at its full size and in the launch configuration it times:
    net n = 2^20, d = 16, 64 randomizations, order-2 DSI, gamma_j = 0.9^j, eta = 1e-8, FP32
    column and transforms with one refinement step (the fused launch sequence).  Every
    randomization against the FP64 GPU path on the same FP32-rounded y (relative 1e-5 on the
    MLL, quadratic form, solve and gradient); the last randomization against the oracle's
    spectral formulas (~45 s of host work: the oracle's gradient is O(d^2 n))."""
    wl = inputs.workload("solve20")
    inst = W.build_instance(qk, wl, wl.ms[0], wl.R, wl.nrhs)
    t32, b32 = W.outputs(qk, inst, F32)
    W.run_tasks(qk, [t32], F32, refine=1, allow_floor=True)
    t64, b64 = W.outputs(qk, inst, F64, with_lam=False, y_via=F32)
    W.run_tasks(qk, [t64], F64, allow_floor=True)
    rel = lambda a, b: float((a.double() - b.double()).abs().max() / b.double().abs().max())  # noqa: E731
    d = wl.d
    errs = {"mll": rel(b32["out"][..., 2], b64["out"][..., 2]), "quad": rel(b32["out"][..., 0], b64["out"][..., 0]),
            "logdet": rel(b32["out"][..., 1], b64["out"][..., 1]), "solve": rel(b32["c"], b64["c"]),
            "grad": rel(b32["grad"][..., :d], b64["grad"][..., :d])}
    print("\nsolve20 FP32-refined vs FP64 GPU: " + " ".join(f"{k}={v:.2e}" for k, v in errs.items()))
    for k, v in errs.items():
        assert v < 1e-5, (k, v)
    del b64
    tol32 = dict(lam=1e-5, quad=1e-5, logdet=1e-5, mll=1e-5, mean=1e-5, c=1e-5, grad=1e-5)
    _oracle_check(inst, b32, wl.R - 1, [0], tol32, y_fp32=True)


def test_mixed_workload_full_size(qk):
    """256 instances (half lattice + SI alpha = 1, half net + DSI order 2), m in 12..22,
    d in {8, 32, 128}, nugget 1e-8: the FP32 schedule with the float-float first column
    (QK_F32W) and one refinement step, captured in a CUDA graph, against the FP64 GPU path on
    the eight smallest instances and the two largest of each family: MLL, quadratic form and
    log det within 1e-5, solve and gradient within max(1e-5, 20 cond eps64)."""
    wls = inputs.mixed_batch()
    t0 = time.time()
    insts = [W.build_instance(qk, wl, wl.ms[0], 1, 1, seed_shift=0, y_kind="product") for wl in wls]
    tasks, bufs = zip(*[W.outputs(qk, inst, qk.F32W) for inst in insts])
    t1 = time.time()
    _, word = W.run_tasks(qk, list(tasks), qk.F32W, refine=1, graph=True, allow_floor=True)
    t2 = time.time()
    print(f"\nmixed workload: {sum(1 << i.m for i in insts)} points, inputs {t1 - t0:.1f} s, "
          f"schedule {t2 - t1:.2f} s, status word {word}")
    size = [(1 << i.m) * i.wl.d for i in insts]
    order = list(np.argsort(size)[:8])
    for kind in ("net", "lattice"):
        order += [k for k in np.argsort(size)[::-1] if insts[k].wl.kind == kind][:2]
    for k in order:
        inst = insts[k]
        t64, b64 = W.outputs(qk, inst, F64, y_via=F32)
        W.run_tasks(qk, [t64], F64, allow_floor=True)
        bw = bufs[k]
        lam64 = b64["lam"][0]
        cond = float(lam64.max() / lam64.min())
        loose = max(1e-5, 20 * cond * qc.EPS64)
        d = inst.wl.d
        errs = {"mll": _rel(bw["out"][..., 2], b64["out"][..., 2]), "quad": _rel(bw["out"][..., 0], b64["out"][..., 0]),
                "logdet": _rel(bw["out"][..., 1], b64["out"][..., 1]),
                "solve": _rel(bw["c"], b64["c"]), "grad": _rel(bw["grad"][..., :d], b64["grad"][..., :d])}
        print(f"  {inst.wl.kind} m={inst.m} d={d} cond={cond:.1e}: " + " ".join(f"{a}={v:.2e}" for a, v in errs.items()))
        for key in ("out", "c", "grad"):
            assert torch.isfinite(bw[key]).all(), (k, key)
        for a, v in errs.items():
            assert v < (loose if a in ("solve", "grad") else 1e-5), (k, inst.wl.kind, inst.m, d, a, v)


@pytest.mark.parametrize("precision", ["float32w", "float32"])
def test_persistent_schedule_takes_the_fused_nets_of_a_mixed_plan(qk, precision):
    """A plan of mixed-workload instances: lattices, nets in and out of the fused size range
    and one net of another DSI order.  The persistent schedule takes the fused nets of the
    first net's order in one launch and runs the other tasks as their launch sequence after
    it; captured in a CUDA graph, the results equal the launch sequence's bit for bit."""
    import dataclasses
    wls = [wl for wl in inputs.mixed_batch() if wl.ms[0] <= 16][:20]
    odd = next(wl for wl in wls if wl.kind == "net" and wl.ms[0] >= 14)
    wls.append(dataclasses.replace(odd, name=odd.name + "-order4", alpha=4))
    insts = [W.build_instance(qk, wl, wl.ms[0], 1, 1, seed_shift=0, y_kind="product") for wl in wls]
    fused_nets = [i for i in insts if i.wl.kind == "net" and i.m >= 14 and i.wl.alpha == 2]
    assert fused_nets and any(i.wl.kind == "lattice" for i in insts) and any(
        i.wl.kind == "net" and i.m < 14 for i in insts), "the plan must mix persistent and launched tasks"
    dt = qk.F32W if precision == "float32w" else F32
    runs = []
    for persistent in (False, True):
        tasks, bufs = zip(*[W.outputs(qk, inst, dt) for inst in insts])
        W.run_tasks(qk, list(tasks), dt, refine=1, graph=True, allow_floor=True, persistent=persistent)
        runs.append(bufs)
    for k, (a, b) in enumerate(zip(*runs)):
        for key in ("out", "c", "lam", "grad"):
            assert torch.isfinite(a[key]).all(), (k, key)
            assert torch.equal(a[key], b[key]), (k, insts[k].wl.kind, insts[k].m, insts[k].wl.alpha, key)
