"""Lattice spectral operations carry two real vectors per complex transform (Sec. 5.2: the
DFT of a real vector is Hermitian, so a + i b transforms to A + i B and splits per frequency
pair k, n - k).  These tests cover what the pairing adds: odd batches (the last pair has an
empty half), vectors of different randomizations sharing a pair, and the combined MLL +
gradient + solve pass of lattice batch tasks, each against the oracle."""
import math

import numpy as np
import pytest
import torch

from oracle import qk_oracle as o
from tests import qkcases as qc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qk():
    from paper_2502_14256_gb300 import build
    build.build()
    from paper_2502_14256_gb300 import qk as q
    return q


F64, F32 = torch.float64, torch.float32


def _lattice(qk, R, d, m, eta, seed, alpha=2):
    case = qc.make_case("lattice", "si", alpha, d, R, seed=seed, c=0.6 ** np.arange(1, d + 1), zeta=1.2)
    kern = qc.kernel_of(case)
    n = 1 << m
    col = torch.empty((R, n), dtype=F64, device=qc.dev())
    qk.kernel_col(case.ps, kern, 0, R, m, col, form=qk.QK_COL_P)
    lam = torch.empty((R, n), dtype=F64, device=qc.dev())
    qk.eigs(qk.QK_SI, m, col, lam, zeta=case.zeta, eta=eta, form=qk.QK_COL_P)
    return case, kern, lam


def _rhs(X, nrhs):
    u = X.astype(np.float64) / 2.0 ** 32
    return np.stack([np.cos(2 * math.pi * (q + 1) * u[:, 0]) + 0.3 * u[:, 1] * u[:, 2] - 0.1 * q
                     for q in range(nrhs)])


@pytest.mark.parametrize("R,nrhs", [(1, 1), (3, 1), (1, 3), (3, 3)])
def test_odd_batches_of_eigs_solve_matvec(qk, R, nrhs):
    d, m, eta = 5, 11, 1e-4
    case, _, lam = _lattice(qk, R, d, m, eta, seed=5100 + 7 * R + nrhs)
    lam_h = lam.cpu().numpy()
    ys, lams = [], []
    for r in range(R):
        k1, X = case.k1_ref(r, m)
        want = o.eigenvalues("si", k1, eta)
        assert qc.lam_elementwise_ok(lam_h[r], want, 1e-10, qc.EPS64, m), qc.lam_elementwise_report(lam_h[r], want)
        ys.append(_rhs(X, nrhs))
        lams.append(want)
    Y = np.stack(ys)
    cref = np.stack([np.stack([o.spectral_solve("si", lams[r], Y[r, q]) for q in range(nrhs)]) for r in range(R)])
    cond = max(float(np.max(lv) / np.min(lv)) for lv in lams)
    y = torch.tensor(Y, dtype=F64, device=qc.dev())
    c = torch.empty_like(y)
    qk.solve(qk.QK_SI, m, lam, y, c)
    assert qc.rel_err(c.cpu().numpy(), cref) < max(1e-10, 20 * cond * qc.EPS64)
    # K c returns y
    u = torch.empty_like(y)
    qk.matvec(qk.QK_SI, m, lam, c, u)
    assert qc.rel_err(u.cpu().numpy(), Y) < 1e-12
    # FP32 data, one FP64-residual refinement step
    y32 = y.to(F32)
    c32 = torch.empty_like(y32)
    qk.solve(qk.QK_SI, m, lam, y32, c32, refine_steps=1)
    cref32 = np.stack([np.stack([o.spectral_solve("si", lams[r], y32[r, q].cpu().numpy().astype(np.float64))
                                 for q in range(nrhs)]) for r in range(R)])
    assert qc.rel_err(c32.cpu().numpy(), cref32) < max(1e-5, 20 * (cond * qc.EPS32) ** 2)


@pytest.mark.parametrize("R,nrhs", [(1, 1), (3, 1), (2, 3)])
def test_odd_batches_of_mll_and_gradient_vs_dense(qk, R, nrhs):
    d, m, eta = 3, 9, 1e-4
    gamma = np.array([0.9, 0.5, 0.3])
    log_ls = np.array([0.1, -0.2, 0.05])
    case = qc.make_case("lattice", "si", 2, d, R, seed=5200 + R + nrhs, c=o.effective_weights(gamma, log_ls), zeta=1.0)
    kern = qc.kernel_of(case)
    n = 1 << m
    col = torch.empty((R, n), dtype=F64, device=qc.dev())
    qk.kernel_col(case.ps, kern, 0, R, m, col, form=qk.QK_COL_P)
    lam = torch.empty((R, n), dtype=F64, device=qc.dev())
    qk.eigs(qk.QK_SI, m, col, lam, zeta=1.0, eta=eta, form=qk.QK_COL_P)
    ys, refs = [], []
    for r in range(R):
        X = case.points_ref(r, np.arange(n), m)
        Y = _rhs(X, nrhs)
        ys.append(Y)
        K = o.gram_dense("si", 2, X, case.c, 1.0, eta)
        rr = []
        for q in range(nrhs):
            mll, quad, logdet, _ = o.mll_dense(K, Y[q])
            mean, var = o.bc_posterior_dense(K, Y[q])
            g = o.mll_grad_dense("si", 2, X, Y[q], gamma, log_ls, eta)
            rr.append((quad, logdet, mll, mean, var, g))
        refs.append(rr)
    y = torch.tensor(np.stack(ys), dtype=F64, device=qc.dev())
    out = torch.empty((R, nrhs, 5), dtype=F64, device=qc.dev())
    grad = torch.empty((R, nrhs, 2 * d + 2), dtype=F64, device=qc.dev())
    qk.mll(case.ps, kern, 0, R, m, nrhs, eta, lam, y, out, grad)
    go, gg = out.cpu().numpy(), grad.cpu().numpy()
    for r in range(R):
        for q in range(nrhs):
            quad, logdet, mll, mean, var, g = refs[r][q]
            assert abs(go[r, q, 0] - quad) < 1e-10 * abs(quad)
            assert abs(go[r, q, 1] - logdet) < 1e-10 * max(1.0, abs(logdet))
            assert abs(go[r, q, 2] - mll) < 1e-10 * abs(mll)
            assert abs(go[r, q, 3] - mean) < 1e-10 * max(1.0, abs(mean))
            assert abs(go[r, q, 4] - var) < 1e-9
            assert qc.rel_err(gg[r, q, :d], g["dc"]) < 1e-9
            assert abs(gg[r, q, d] - g["deta"]) < 1e-9 * max(1.0, abs(g["deta"]))


@pytest.mark.parametrize("dtype", ["f64", "f32w", "f32"])
def test_lattice_batch_task_combined_pass(qk, dtype):
    """A lattice batch task runs column, eigenvalues and ONE pass for MLL, gradient and solve
    (one forward transform of y, one inverse transform giving both c and the gradient's u).
    Against the oracle's spectral outputs (n = 2^12) and the per-call FP64 ops."""
    d, R, nrhs, m, eta = 4, 3, 2, 12, 1e-6
    gamma = 0.8 ** np.arange(1, d + 1)
    case = qc.make_case("lattice", "si", 2, d, R, seed=5300, c=gamma, zeta=1.1)
    kern = qc.kernel_of(case)
    n = 1 << m
    ys, refs = [], []
    for r in range(R):
        k1, X = case.k1_ref(r, m)
        lv = o.eigenvalues("si", k1, eta)
        Y = _rhs(X, nrhs)
        ys.append(Y)
        refs.append((lv,))
    td = {"f64": F64, "f32w": qk.F32W, "f32": F32}[dtype]
    ddt = qk.data_dtype(td)
    y = torch.tensor(np.stack(ys), dtype=ddt, device=qc.dev())
    c = torch.zeros_like(y)
    lam = torch.zeros((R, n), dtype=F64, device=qc.dev())
    out = torch.zeros((R, nrhs, 5), dtype=F64, device=qc.dev())
    grad = torch.zeros((R, nrhs, 2 * d + 2), dtype=F64, device=qc.dev())
    task = qk.Task(case.ps, kern, m, nrhs, eta, y.data_ptr(), c.data_ptr(), lam.data_ptr(), out.data_ptr(),
                   grad.data_ptr())
    ws = qk.workspace(qk.batch_workspace_bytes([task], td))
    qk.batch_plan([task], td, 0, ws)
    qk.batch_run(ws)
    torch.cuda.synchronize()
    lam_h, c_h, o_h = lam.cpu().numpy(), c.cpu().numpy().astype(np.float64), out.cpu().numpy()
    # per-call FP64 reference on the same (rounded) data: gradient
    y64 = y.to(F64)
    lam_r = torch.empty((R, n), dtype=F64, device=qc.dev())
    col = torch.empty((R, n), dtype=F64, device=qc.dev())
    qk.kernel_col(case.ps, kern, 0, R, m, col, form=qk.QK_COL_P)
    qk.eigs(qk.QK_SI, m, col, lam_r, zeta=case.zeta, eta=eta, form=qk.QK_COL_P)
    out_r = torch.empty_like(out)
    grad_r = torch.empty_like(grad)
    qk.mll(case.ps, kern, 0, R, m, nrhs, eta, lam_r, y64, out_r, grad_r)
    g_h, g_r = grad.cpu().numpy(), grad_r.cpu().numpy()
    cond = max(float(np.max(rf[0]) / np.min(rf[0])) for rf in refs)
    for r in range(R):
        lv = refs[r][0]
        if dtype == "f32":
            assert qc.rel_err(lam_h[r], lv) < 1e-5
        else:
            assert qc.lam_elementwise_ok(lam_h[r], lv, 1e-10, 4 * qc.EPS64, m), qc.lam_elementwise_report(lam_h[r], lv)
        for q in range(nrhs):
            yq = y64[r, q].cpu().numpy()  # the data as the run saw it (FP32-rounded for f32w)
            cw = o.spectral_solve("si", lv, yq)
            mq = o.spectral_mll("si", lv, yq)
            quad, logdet = mq["quad"], mq["logdet"]
            if dtype == "f64":
                assert qc.rel_err(c_h[r, q], cw) < max(1e-10, 20 * cond * qc.EPS64)
                assert abs(o_h[r, q, 0] - quad) < 1e-10 * abs(quad)
                assert abs(o_h[r, q, 1] - logdet) < 1e-10 * max(1.0, abs(logdet))
                assert qc.rel_err(g_h[r, q], g_r[r, q]) < 1e-12
            elif dtype == "f32w":
                # FP64 forward transform of y and FP64 division: only the FP32 inverse rounds
                assert qc.rel_err(c_h[r, q], cw) < 1e-5
                assert abs(o_h[r, q, 0] - quad) < 1e-5 * abs(quad)
                assert abs(o_h[r, q, 1] - logdet) < 1e-5 * max(1.0, abs(logdet))
                # dMLL/deta = sum_w g_w: FP64 spectral sums
                assert abs(g_h[r, q, d] - g_r[r, q, d]) < 1e-6 * abs(g_r[r, q, d])
                # dMLL/dc_j = sum_i u_i dk1_i/dc_j summed by the FP32 sweep: its terms cancel
                # near the nugget floor, so the bound is the FP32 rounding of the terms,
                # eps32 sum_i |u_i dk1_i/dc_j| (u and dk1 from the oracle's pieces)
                X = case.points_ref(r, np.arange(n), m)
                yt = o.forward_transform("si", yq)
                gw = 0.5 * (np.abs(yt) ** 2 / lv ** 2 - 1.0 / lv)
                u = o.to_natural_order(np.fft.fft(gw).real, m)
                fac = [o.factor_values("si", 2, o.pair_difference("si", X[:, j], X[0, j])) for j in range(d)]
                for j in range(d):
                    dk = np.full(n, case.zeta)
                    for jj in range(d):
                        dk *= fac[jj] if jj == j else 1.0 + case.c[jj] * fac[jj]
                    bound = 1e-5 * abs(g_r[r, q, j]) + 8 * math.sqrt(32) * qc.EPS32 * float(np.sum(np.abs(u * dk)))
                    assert abs(g_h[r, q, j] - g_r[r, q, j]) < bound, (j, g_h[r, q, j], g_r[r, q, j], bound)
            else:
                assert np.all(np.isfinite(c_h[r, q])) and np.all(np.isfinite(g_h[r, q]))


@pytest.mark.parametrize("m", [14, 18, 21])
@pytest.mark.parametrize("dtype", ["f64", "f32w"])
def test_lattice_batch_task_against_oracle_at_scale(qk, m, dtype):
    """Lattice batch tasks (column, eigenvalues, one MLL + gradient + solve pass) against the
    oracle's spectral formulas at n = 2^14, 2^18 and 2^21: eigenvalues element-wise, the
    solve, quadratic form, log det, and the gradient (FP64: normwise; float-float column:
    bounded by the FP32 sweep's rounding of its cancelling terms)."""
    d, R, nrhs, eta = 4, 2, 1, 1e-4
    gamma = 0.7 ** np.arange(1, d + 1)
    case = qc.make_case("lattice", "si", 2, d, R, seed=5400 + m, c=gamma, zeta=0.9)
    kern = qc.kernel_of(case)
    n = 1 << m
    td = F64 if dtype == "f64" else qk.F32W
    ys, refs = [], []
    for r in range(R):
        k1, X = case.k1_ref(r, m)
        lv = o.eigenvalues("si", k1, eta)
        Y = _rhs(X, nrhs)
        ys.append(Y)
        refs.append((lv, X))
    y = torch.tensor(np.stack(ys), dtype=qk.data_dtype(td), device=qc.dev())
    c = torch.zeros_like(y)
    lam = torch.zeros((R, n), dtype=F64, device=qc.dev())
    out = torch.zeros((R, nrhs, 5), dtype=F64, device=qc.dev())
    grad = torch.zeros((R, nrhs, 2 * d + 2), dtype=F64, device=qc.dev())
    task = qk.Task(case.ps, kern, m, nrhs, eta, y.data_ptr(), c.data_ptr(), lam.data_ptr(), out.data_ptr(),
                   grad.data_ptr())
    ws = qk.workspace(qk.batch_workspace_bytes([task], td))
    qk.batch_plan([task], td, 0, ws)
    qk.batch_run(ws)
    torch.cuda.synchronize()
    lam_h, c_h, o_h, g_h = lam.cpu().numpy(), c.cpu().numpy().astype(np.float64), out.cpu().numpy(), grad.cpu().numpy()
    y_h = y.to(F64).cpu().numpy()
    for r in range(R):
        lv, X = refs[r]
        eps = qc.EPS64 if dtype == "f64" else 4 * qc.EPS64
        assert qc.lam_elementwise_ok(lam_h[r], lv, 1e-10, eps, m), qc.lam_elementwise_report(lam_h[r], lv)
        cond = float(np.max(lv) / np.min(lv))
        for q in range(nrhs):
            yq = y_h[r, q]
            cw = o.spectral_solve("si", lv, yq)
            sp = o.spectral_mll("si", lv, yq, case.zeta)
            gr = o.spectral_mll_grad("si", 2, X, yq, lv, case.c, case.zeta)
            tol = max(1e-10, 20 * cond * qc.EPS64) if dtype == "f64" else 1e-5
            assert qc.rel_err(c_h[r, q], cw) < tol, (qc.rel_err(c_h[r, q], cw), tol)
            qt = 1e-10 if dtype == "f64" else 1e-5
            # y^T K^-1 y moves by 2 c^T dy for a transform rounding dy ~ m eps ||y||: relative
            # 2 m eps ||c|| ||y|| / (y^T c), about m eps sqrt(cond) for these smooth y
            qq = max(qt, 4 * m * qc.EPS64 * math.sqrt(cond)) if dtype == "f64" else qt
            assert abs(o_h[r, q, 0] - sp["quad"]) < qq * abs(sp["quad"]), (o_h[r, q, 0], sp["quad"], qq)
            assert abs(o_h[r, q, 1] - sp["logdet"]) < qt * max(1.0, abs(sp["logdet"]))
            assert abs(o_h[r, q, 3] - sp["post_mean"]) < qt * max(1.0, abs(sp["post_mean"]))
            assert abs(g_h[r, q, d] - gr["deta"]) < 1e-8 * max(1.0, abs(gr["deta"]))
            # dMLL/dc_j = sum_i u_i dk1_i/dc_j over n points, its terms cancelling: bounded by
            # the sweep's rounding of the terms, eps sum_i |u_i dk1_i/dc_j| (u, dk1 from the
            # oracle's pieces), plus the relative target
            yt = o.forward_transform("si", yq)
            gw = 0.5 * (np.abs(yt) ** 2 / lv ** 2 - 1.0 / lv)
            u = o.to_natural_order(np.fft.fft(gw).real, m)
            fac = [o.factor_values("si", 2, o.pair_difference("si", X[:, j], X[0, j])) for j in range(d)]
            rel, eps = (1e-9, qc.EPS64) if dtype == "f64" else (1e-5, qc.EPS32)
            for j in range(d):
                dk = np.full(n, case.zeta)
                for jj in range(d):
                    dk *= fac[jj] if jj == j else 1.0 + case.c[jj] * fac[jj]
                bound = rel * abs(gr["dc"][j]) + 8 * math.sqrt(32) * eps * float(np.sum(np.abs(u * dk)))
                assert abs(g_h[r, q, j] - gr["dc"][j]) < bound, (j, g_h[r, q, j], gr["dc"][j], bound)
