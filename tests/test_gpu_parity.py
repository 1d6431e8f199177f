"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle, element by element.

Sizes span several CTA tiles and ragged ranges; tolerances: integer work bit-exact,
FP64 relative 1e-10 (solves, MLL) and 1e-12 (columns, eigenvalues), FP32 relative 1e-5
(after one refinement step for solves).
"""
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


# ------------------------------------------------------------------- points
@pytest.mark.parametrize("d,R", [(1, 1), (16, 5), (130, 2)])
def test_lms_setup_bit_exact(qk, d, R):
    case = qc.make_case("net", "dsi", 2, d, R, seed=100 + d)
    Ct = qc.u32_host(case.keep[3])
    assert np.array_equal(Ct, case.Ct_ref)


@pytest.mark.parametrize("order", ["natural", "gray"])
@pytest.mark.parametrize("d", [1, 4, 37])
def test_net_points_bit_exact(qk, order, d):
    case = qc.make_case("net", "dsi", 2, d, 3, seed=7 + d, order=order)
    for (i0, n) in [(0, 1), (0, 2), (0, 1 << 11), (5, 3001), (1 << 13, 777), ((1 << 20) - 9, 40)]:
        X = torch.empty((2, n, d), dtype=torch.int32, device=qc.dev())
        qk.gen_points(case.ps, 1, 2, i0, n, X)
        got = qc.u32_host(X)
        m = max(1, int(i0 + n - 1).bit_length())
        for r in (1, 2):
            want = o.net_points(case.Ct_ref[r], case.D[r], np.arange(i0, i0 + n), m, order)
            assert np.array_equal(got[r - 1], want), (i0, n, r)


@pytest.mark.parametrize("d", [1, 6, 40])
def test_lattice_points_bit_exact(qk, d):
    case = qc.make_case("lattice", "si", 2, d, 2, seed=50 + d)
    for (i0, n) in [(0, 1), (0, 1 << 12), (3, 5000), ((1 << 31) - 5, 17)]:
        X = torch.empty((2, n, d), dtype=torch.int32, device=qc.dev())
        qk.gen_points(case.ps, 0, 2, i0, n, X)
        got = qc.u32_host(X)
        for r in range(2):
            assert np.array_equal(got[r], o.lattice_points(case.g, case.D[r], np.arange(i0, i0 + n)))


# ------------------------------------------------------------- first column
FAMS = [("net", "dsi", 1), ("net", "dsi", 2), ("net", "dsi", 3), ("net", "dsi", 4),
        ("lattice", "si", 1), ("lattice", "si", 2)]


@pytest.mark.parametrize("kind,family,alpha", FAMS)
@pytest.mark.parametrize("m,d", [(0, 3), (3, 5), (11, 2), (13, 33)])
def test_kernel_col(qk, kind, family, alpha, m, d):
    c = 0.8 ** np.arange(1, d + 1)
    case = qc.make_case(kind, family, alpha, d, 3, seed=300 + 7 * m + d, c=c, zeta=1.7)
    kern = qc.kernel_of(case)
    n = 1 << m
    for dt, tol in ((F64, 1e-13), (F32, 4e-6 if alpha < 4 else 2e-5)):
        for form in (qk.QK_COL_K1, qk.QK_COL_P):
            col = torch.empty((2, n), dtype=dt, device=qc.dev())
            qk.kernel_col(case.ps, kern, 1, 2, m, col, form=form)
            got = col.cpu().numpy().astype(np.float64)
            for r in (1, 2):
                k1, _ = case.k1_ref(r, m)
                g = got[r - 1] if form == qk.QK_COL_K1 else case.zeta * (1.0 + got[r - 1])
                assert qc.rel_err(g, k1) < tol, (dt, form, r, qc.rel_err(g, k1))
    # float-float arithmetic on the FP32 pipes (QK_F32W), written as FP64: about 2^-46 per
    # factor, so the column agrees with the oracle to ~1e-13 where FP32 gives ~1e-6
    for form in (qk.QK_COL_K1, qk.QK_COL_P):
        col = torch.empty((2, n), dtype=F64, device=qc.dev())
        qk.kernel_col(case.ps, kern, 1, 2, m, col, form=form, wide=True)
        got = col.cpu().numpy()
        for r in (1, 2):
            k1, _ = case.k1_ref(r, m)
            g = got[r - 1] if form == qk.QK_COL_K1 else case.zeta * (1.0 + got[r - 1])
            assert qc.rel_err(g, k1) < 2e-13, ("wide", form, r, qc.rel_err(g, k1))
            if form == qk.QK_COL_P:  # p itself keeps its relative precision
                p_ref = k1 / case.zeta - 1.0
                assert qc.rel_err(got[r - 1], p_ref) < 2e-12, ("wide p", r, qc.rel_err(got[r - 1], p_ref))


# ---------------------------------------------------------------- spectrum
def _lam_ref(case, r, m, eta):
    k1, X = case.k1_ref(r, m)
    return o.eigenvalues(case.family, k1, eta), k1, X


@pytest.mark.parametrize("kind,family,alpha", [("net", "dsi", 2), ("net", "dsi", 4), ("lattice", "si", 1),
                                               ("lattice", "si", 2)])
@pytest.mark.parametrize("m", [1, 9, 13, 16])
def test_eigs(qk, kind, family, alpha, m):
    d = 6
    case = qc.make_case(kind, family, alpha, d, 2, seed=900 + m, c=0.5 ** np.arange(d), zeta=1.3)
    kern = qc.kernel_of(case)
    eta = 1e-6
    fam = qk.QK_DSI if family == "dsi" else qk.QK_SI
    for dt, tol in ((F64, 1e-12), (F32, 1e-5)):
        col = torch.empty((2, 1 << m), dtype=dt, device=qc.dev())
        qk.kernel_col(case.ps, kern, 0, 2, m, col, form=qk.QK_COL_P)
        lam = torch.empty((2, 1 << m), dtype=F64, device=qc.dev())
        status = torch.zeros(1, dtype=torch.int32, device=qc.dev())
        qk.eigs(fam, m, col, lam, zeta=case.zeta, eta=eta, form=qk.QK_COL_P, status=status)
        if dt == F64:
            qk.read_status(status)  # FP64 resolves every eigenvalue above the nugget
        # FP32 eigenvalues carry errors ~ eps32 * ||k1||, larger than the nugget at
        # this n: the smallest may go negative, which the status word then reports.
        got = lam.cpu().numpy()
        for r in range(2):
            want, _, _ = _lam_ref(case, r, m, eta)
            assert qc.rel_err(got[r], want) < tol, (dt, r, qc.rel_err(got[r], want))
            if dt == F64:
                # element-wise: every eigenvalue, the small ones included, to the rounding floor
                # of two FP64 transforms of k_1 (the library's and the oracle's)
                assert qc.lam_elementwise_ok(got[r], want, 1e-10, qc.EPS64, m), qc.lam_elementwise_report(got[r], want)
    # the float-float column (QK_F32W) then the FP64 transform: the same element-wise bound
    col = torch.empty((2, 1 << m), dtype=F64, device=qc.dev())
    qk.kernel_col(case.ps, kern, 0, 2, m, col, form=qk.QK_COL_P, wide=True)
    lam = torch.empty((2, 1 << m), dtype=F64, device=qc.dev())
    qk.eigs(fam, m, col, lam, zeta=case.zeta, eta=eta, form=qk.QK_COL_P)
    got = lam.cpu().numpy()
    for r in range(2):
        want, _, _ = _lam_ref(case, r, m, eta)
        assert qc.lam_elementwise_ok(got[r], want, 1e-10, qc.EPS64 * 4, m), qc.lam_elementwise_report(got[r], want)


def test_eigs_reports_non_positive_definite(qk):
    case = qc.make_case("net", "dsi", 2, 3, 1, seed=5)
    kern = qc.kernel_of(case)
    col = torch.empty((1, 256), dtype=F64, device=qc.dev())
    qk.kernel_col(case.ps, kern, 0, 1, 8, col)
    lam = torch.empty_like(col)
    status = torch.zeros(1, dtype=torch.int32, device=qc.dev())
    qk.eigs(qk.QK_DSI, 8, col, lam, eta=-1e6, status=status)
    with pytest.raises(qk.QKError) as e:
        qk.read_status(status)
    assert e.value.code == qk.QK_ENOTPD
    qk.read_status(status)  # cleared


def test_eigenvalues_below_the_nugget_are_raised_to_it(qk):
    """K + eta I has no eigenvalue below eta; a column whose transform dips below (here a
    kernel with a negative weight, so that K itself is indefinite) is floored at eta and
    flagged with the informational QK_STATUS_FLOOR bit, not an error."""
    case = qc.make_case("net", "dsi", 2, 3, 1, seed=5, c=np.array([-0.9, 0.3, 0.1]))
    kern = qc.kernel_of(case)
    col = torch.empty((1, 256), dtype=F64, device=qc.dev())
    qk.kernel_col(case.ps, kern, 0, 1, 8, col)
    lam = torch.empty_like(col)
    status = torch.zeros(1, dtype=torch.int32, device=qc.dev())
    eta = 1e-3
    qk.eigs(qk.QK_DSI, 8, col, lam, eta=eta, status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == qk.QK_STATUS_FLOOR
    got = lam.cpu().numpy()[0]
    want = o.eigenvalues("dsi", case.k1_ref(0, 8)[0], eta)
    assert np.all(got >= eta)
    assert np.array_equal(got == eta, want < eta)
    keep = want >= eta
    assert qc.rel_err(got[keep], want[keep]) < 1e-12
    qk.read_status(status)  # informational: not an error


def _setup_spectrum(qk, case, m, dt, eta, R):
    kern = qc.kernel_of(case)
    fam = qk.QK_DSI if case.family == "dsi" else qk.QK_SI
    col = torch.empty((R, 1 << m), dtype=dt, device=qc.dev())
    qk.kernel_col(case.ps, kern, 0, R, m, col, form=qk.QK_COL_P)
    lam = torch.empty((R, 1 << m), dtype=F64, device=qc.dev())
    qk.eigs(fam, m, col, lam, zeta=case.zeta, eta=eta, form=qk.QK_COL_P)
    return kern, fam, lam


@pytest.mark.parametrize("kind,family,alpha", [("net", "dsi", 1), ("net", "dsi", 2), ("lattice", "si", 1),
                                               ("lattice", "si", 2)])
@pytest.mark.parametrize("m", [4, 10, 14])
def test_solve_and_matvec(qk, kind, family, alpha, m):
    """Forward error against the oracle on moderately conditioned systems (eta = 1e-3):
    FP64 within max(1e-10, 20 cond eps64); FP32 + one refinement step (FP64 residual)
    within max(1e-5, 20 (cond eps32)^2); plain FP32 within 20 cond eps32."""
    d, R, nrhs, eta = 4, 2, 3, 1e-3
    case = qc.make_case(kind, family, alpha, d, R, seed=1200 + m, c=1.0 / np.arange(1, d + 1) ** 2)
    refs = []
    for r in range(R):
        lam_ref, k1, X = _lam_ref(case, r, m, eta)
        Y = np.stack([np.sin(3.0 * (q + 1) * X[:, 0] / 2 ** 32) + X[:, 1] / 2 ** 33 for q in range(nrhs)])
        if m <= 10:
            K = o.gram_dense(case.family, alpha, X, case.c, case.zeta, eta)
            Cref = o.cholesky_solve(K, Y.T)[0].T
        else:
            Cref = np.stack([o.spectral_solve(case.family, lam_ref, Y[q]) for q in range(nrhs)])
        refs.append((Y, Cref, lam_ref))
    y_h = np.stack([refs[r][0] for r in range(R)])
    cond = max(float(np.max(rf[2]) / np.min(rf[2])) for rf in refs)
    for dt, refine in ((F64, 0), (F32, 0), (F32, 1)):
        if dt == F64:
            tol = max(1e-10, 20 * cond * qc.EPS64)
        elif refine:
            tol = max(1e-5, 20 * (cond * qc.EPS32) ** 2)
        else:
            tol = 20 * cond * qc.EPS32
        _, fam, lam = _setup_spectrum(qk, case, m, F64 if refine else dt, eta, R)
        y = torch.tensor(y_h, dtype=dt, device=qc.dev())
        c = torch.empty_like(y)
        qk.solve(fam, m, lam, y, c, refine_steps=refine)
        got = c.cpu().numpy().astype(np.float64)
        for r in range(R):
            assert qc.rel_err(got[r], refs[r][1]) < tol, (dt, refine, r, qc.rel_err(got[r], refs[r][1]), tol)
        u = torch.empty_like(y)
        qk.matvec(fam, m, lam, c, u)
        # K c reproduces y up to the conditioning of the round trip
        eps = qc.EPS64 if dt == F64 else qc.EPS32
        assert qc.rel_err(u.cpu().numpy(), y_h) < max(1e-12 if dt == F64 else 2e-6, 20 * cond * eps)


@pytest.mark.parametrize("kind,family,alpha", [("net", "dsi", 2), ("lattice", "si", 2)])
def test_ill_conditioned_solve_has_small_backward_error(qk, kind, family, alpha):
    """eta = 1e-8, cond up to ~1e12: the residual y - K c (K applied by the oracle from
    its own eigenvalues) stays at FP64 rounding level even where the forward error cannot."""
    d, R, m, eta = 4, 1, 14, 1e-8
    case = qc.make_case(kind, family, alpha, d, R, seed=1300, c=1.0 / np.arange(1, d + 1) ** 2)
    lam_ref, k1, X = _lam_ref(case, 0, m, eta)
    Y = np.sin(5.0 * X[:, 0] / 2 ** 32)[None, None, :]
    _, fam, lam = _setup_spectrum(qk, case, m, F64, eta, R)
    y = torch.tensor(Y, dtype=F64, device=qc.dev())
    c = torch.empty_like(y)
    qk.solve(fam, m, lam, y, c)
    cg = c.cpu().numpy()[0, 0]
    res = Y[0, 0] - o.spectral_matvec(case.family, lam_ref, cg)
    # normwise backward error of a transform-based solve: |y - K c| <~ m eps |K| |c|
    bound = 8 * m * qc.EPS64 * float(np.max(lam_ref)) * float(np.max(np.abs(cg)))
    assert np.max(np.abs(res)) < bound, (np.max(np.abs(res)), bound)


# --------------------------------------------------------------- MLL + grad
@pytest.mark.parametrize("kind,family,alpha", [("net", "dsi", 1), ("net", "dsi", 2), ("net", "dsi", 4),
                                               ("lattice", "si", 1), ("lattice", "si", 2)])
def test_mll_and_gradient_vs_dense(qk, kind, family, alpha):
    d, R, nrhs, m, eta = 3, 2, 2, 8, 1e-4
    gamma = np.array([0.9, 0.5, 0.3])
    log_ls = np.array([0.1, -0.2, 0.05])
    case = qc.make_case(kind, family, alpha, d, R, seed=77, c=o.effective_weights(gamma, log_ls), zeta=1.0)
    kern, fam, lam = _setup_spectrum(qk, case, m, F64, eta, R)
    n = 1 << m
    ys = []
    refs = []
    for r in range(R):
        X = case.points_ref(r, np.arange(n), m)
        Y = np.stack([np.cos(2.0 * (q + 1) * X[:, 0] / 2 ** 32) + 0.1 * X[:, 2] / 2 ** 32 for q in range(nrhs)])
        ys.append(Y)
        K = o.gram_dense(case.family, alpha, X, case.c, 1.0, eta)
        rr = []
        for q in range(nrhs):
            mll, quad, logdet, _ = o.mll_dense(K, Y[q])
            mean, var = o.bc_posterior_dense(K, Y[q])
            g = o.mll_grad_dense(case.family, alpha, X, Y[q], gamma, log_ls, eta)
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
            assert qc.rel_err(gg[r, q, d + 1:2 * d + 1], g["dmean_dc"]) < 1e-8
            assert abs(gg[r, q, 2 * d + 1] - g["dmean_deta"]) < 1e-9 * max(1.0, abs(g["dmean_deta"]))


def test_mll_gradient_matches_finite_differences_on_gpu(qk):
    """Lattice + SI alpha=2, d=32, n=2^10, log-lengthscales 0 and log-nugget -12 (the
    differentiation workload at the dense-oracle size): central differences with
    h = 1e-6 of the GPU's own MLL against its hand-written gradient."""
    from paper_2502_14256_gb300 import inputs
    wl = inputs.workload("diff_small")
    d, m = wl.d, wl.ms[0]
    n = 1 << m
    lat = inputs.make_lattice(wl.seed, d, 1, wl.extra["m_gen"])
    X = o.lattice_points(lat.g, lat.D[0], np.arange(n))
    y_h = inputs.rhs_product(X)
    gd, Dd = qc.u32_tensor(lat.g), qc.u32_tensor(lat.D)
    ps = qk.pointset(qk.QK_LATTICE, d, 1, g=gd, D=Dd)

    def run(log_ls, log_eta):
        w = torch.tensor(o.effective_weights(wl.gamma, log_ls), dtype=F64, device=qc.dev())
        kern = qk.kernel(qk.QK_SI, wl.alpha, w, 1.0)
        col = torch.empty((1, n), dtype=F64, device=qc.dev())
        qk.kernel_col(ps, kern, 0, 1, m, col, form=qk.QK_COL_P)
        lam = torch.empty_like(col)
        qk.eigs(qk.QK_SI, m, col, lam, eta=math.exp(log_eta), form=qk.QK_COL_P)
        y = torch.tensor(y_h, dtype=F64, device=qc.dev()).reshape(1, 1, n)
        out = torch.empty((1, 1, 5), dtype=F64, device=qc.dev())
        grad = torch.empty((1, 1, 2 * d + 2), dtype=F64, device=qc.dev())
        qk.mll(ps, kern, 0, 1, m, 1, math.exp(log_eta), lam, y, out, grad)
        return out.cpu().numpy().ravel(), grad.cpu().numpy().ravel()

    log_ls = wl.log_ls.copy()
    log_eta = math.log(wl.eta)
    out0, g0 = run(log_ls, log_eta)
    cw = o.effective_weights(wl.gamma, log_ls)
    dtheta = cw * g0[:d]
    h = 1e-6
    for j in (0, 5, 31):
        e = np.zeros(d)
        e[j] = h
        fd = (run(log_ls + e, log_eta)[0][2] - run(log_ls - e, log_eta)[0][2]) / (2 * h)
        assert abs(fd - dtheta[j]) < 1e-5 * max(1.0, abs(fd)), (j, fd, dtheta[j])
    # dMLL/dlog(eta) is ~1e-19 here (K ~ 1e16 I): compare absolutely
    fd = (run(log_ls, log_eta + h)[0][2] - run(log_ls, log_eta - h)[0][2]) / (2 * h)
    assert abs(fd - wl.eta * g0[d]) < 1e-6
    # and the dense oracle's gradient at the same point
    gref = o.mll_grad_dense("si", wl.alpha, X, y_h, wl.gamma, log_ls, wl.eta)
    assert qc.rel_err(dtheta, gref["dtheta"]) < 1e-8


# ----------------------------------------------------------------- batching
def test_batch_schedule_matches_per_call_results_and_replays_in_a_graph(qk):
    tasks, keep, refs = [], [], []
    specs = [("net", "dsi", 2, 5, 3, 10, 2), ("lattice", "si", 1, 4, 2, 12, 1), ("net", "dsi", 1, 3, 2, 6, 3),
             ("lattice", "si", 2, 8, 1, 9, 2)]
    for t, (kind, family, alpha, d, R, m, nrhs) in enumerate(specs):
        case = qc.make_case(kind, family, alpha, d, R, seed=4000 + t, c=0.7 ** np.arange(1, d + 1))
        kern = qc.kernel_of(case)
        n = 1 << m
        y = torch.randn((R, nrhs, n), dtype=F64, device=qc.dev(), generator=torch.Generator(qc.dev()).manual_seed(t))
        out = torch.zeros((R, nrhs, 5), dtype=F64, device=qc.dev())
        grad = torch.zeros((R, nrhs, 2 * d + 2), dtype=F64, device=qc.dev())
        c = torch.zeros_like(y)
        lam = torch.zeros((R, n), dtype=F64, device=qc.dev())
        keep += [case, y, out, grad, c, lam]
        tasks.append(qk.Task(case.ps, kern, m, nrhs, 1e-5, y.data_ptr(), c.data_ptr(), lam.data_ptr(),
                             out.data_ptr(), grad.data_ptr()))
        # per-call reference
        _, fam, lam_r = _setup_spectrum(qk, case, m, F64, 1e-5, R)
        out_r = torch.empty_like(out)
        grad_r = torch.empty_like(grad)
        qk.mll(case.ps, kern, 0, R, m, nrhs, 1e-5, lam_r, y, out_r, grad_r)
        c_r = torch.empty_like(y)
        qk.solve(fam, m, lam_r, y, c_r)
        refs.append((lam_r, out_r, grad_r, c_r))
    ws = qk.workspace(qk.batch_workspace_bytes(tasks, F64))
    qk.batch_plan(tasks, F64, 0, ws)
    qk.batch_run(ws)
    torch.cuda.synchronize()

    def check():
        for t in range(len(specs)):
            lam, out, grad, c = keep[6 * t + 5], keep[6 * t + 2], keep[6 * t + 3], keep[6 * t + 4]
            lam_r, out_r, grad_r, c_r = refs[t]
            assert torch.allclose(lam, lam_r, rtol=1e-13, atol=0)
            assert torch.allclose(out, out_r, rtol=1e-12, atol=1e-13)
            assert torch.allclose(grad, grad_r, rtol=1e-10, atol=1e-12)
            assert torch.allclose(c, c_r, rtol=1e-12, atol=1e-12)

    check()
    for t in range(len(specs)):
        keep[6 * t + 2].zero_()
        keep[6 * t + 4].zero_()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            qk.batch_run(ws, stream=s)
    g.replay()
    torch.cuda.synchronize()
    check()


# --------------------------------------------------------- public transforms
@pytest.mark.parametrize("m", [0, 1, 5, 12, 13, 14, 16, 17, 18, 19, 20, 21, 24])
def test_fwht_fftbr_ifftbr(qk, m):
    n = 1 << m
    nvec = 3 if m < 20 else (2 if m < 24 else 1)
    rng = np.random.default_rng(m)
    x = rng.standard_normal((nvec, n))
    want = o.hadamard_apply(x) / math.sqrt(n)
    for dt, tol in ((F64, 1e-13), (F32, 1e-6 * max(1, m))):
        t = torch.tensor(x, dtype=dt, device=qc.dev())
        qk.fwht(m, t)
        assert qc.rel_err(t.cpu().numpy(), want) < tol, (dt, m)
    z = rng.standard_normal((nvec, n)) + 1j * rng.standard_normal((nvec, n))
    zw = np.fft.fft(o.to_linear_order(z, m), axis=-1) / math.sqrt(n)
    for dt, tol in ((F64, 1e-13), (F32, 2e-6 * max(1, m))):
        t = torch.tensor(np.stack([z.real, z.imag], axis=-1), dtype=dt, device=qc.dev()).contiguous()
        qk.fftbr(m, t)
        got = t.cpu().numpy()
        assert qc.rel_err(got[..., 0] + 1j * got[..., 1], zw) < tol, (dt, m)
        qk.ifftbr(m, t)
        got = t.cpu().numpy()
        assert qc.rel_err(got[..., 0] + 1j * got[..., 1], z) < tol, (dt, m)


@pytest.mark.parametrize("m", [13, 16, 17, 18, 19, 20])
def test_fftbr_persistent_equals_two_pass(qk, m):
    """qk_fftbr_ws: both passes of FFTBR / IFFTBR in one persistent launch, bit for bit the
    pass-by-pass transform (m = 13 and FP64 fall back to it), for several lags."""
    n = 1 << m
    nvec = 7
    rng = np.random.default_rng(700 + m)
    z = np.stack([rng.standard_normal((nvec, n)), rng.standard_normal((nvec, n))], axis=-1)
    for dt in (F32, F64):
        for inverse in (False, True):
            ref = torch.tensor(z, dtype=dt, device=qc.dev()).contiguous()
            (qk.ifftbr if inverse else qk.fftbr)(m, ref)
            for lag in (0, 1, 3, nvec):
                t = torch.tensor(z, dtype=dt, device=qc.dev()).contiguous()
                status = torch.zeros(1, dtype=torch.int32, device=qc.dev())
                qk.fftbr_ws(m, t, inverse=inverse, lag=lag, status=status)
                torch.cuda.synchronize()
                assert int(status.item()) == 0
                assert torch.equal(t, ref), (dt, inverse, lag)


# ------------------------------------------------------------ fused pipeline
def _abs_dk_sums(family, alpha, X, c, zeta):
    """sum_i |dk1_i/dc_j| for every j (the scale of the cancelling gradient sums)."""
    n, d = X.shape
    out = np.empty(d)
    fac = [o.factor_values(family, alpha, o.pair_difference(family, X[:, j], X[0, j])) for j in range(d)]
    for j in range(d):
        dk = np.full(n, float(zeta))
        for jj in range(d):
            dk *= fac[jj] if jj == j else 1.0 + c[jj] * fac[jj]
        out[j] = float(np.sum(np.abs(dk)))
    return out


def _batch_outputs(qk, case, m, nrhs, dt, y_h, eta, refine=0):
    kern = qc.kernel_of(case)
    R, n, d = case.R, 1 << m, case.d
    y = torch.tensor(y_h, dtype=qk.data_dtype(dt), device=qc.dev())
    c = torch.zeros_like(y)
    lam = torch.zeros((R, n), dtype=F64, device=qc.dev())
    out = torch.zeros((R, nrhs, 5), dtype=F64, device=qc.dev())
    grad = torch.zeros((R, nrhs, 2 * d + 2), dtype=F64, device=qc.dev())
    task = qk.Task(case.ps, kern, m, nrhs, eta, y.data_ptr(), c.data_ptr(), lam.data_ptr(), out.data_ptr(),
                   grad.data_ptr())
    ws = qk.workspace(qk.batch_workspace_bytes([task], dt))
    status = torch.zeros(1, dtype=torch.int32, device=qc.dev())
    qk.batch_plan([task], dt, refine, ws)
    qk.batch_run(ws, status)
    qk.read_status(status)
    return {k: v.cpu().numpy().astype(np.float64) for k, v in dict(c=c, lam=lam, out=out, grad=grad).items()}


def _data(qk, dt):
    return qk.data_dtype(dt)


F32W = "float32w"  # qk.F32W: FP32 arrays, float-float first column


@pytest.mark.parametrize("dt", [F64, F32, F32W])
@pytest.mark.parametrize("m,alpha,order,nrhs", [(13, 2, "gray", 2), (14, 1, "gray", 1), (16, 4, "natural", 3),
                                                (17, 3, "gray", 2), (20, 2, "gray", 1), (21, 2, "natural", 1),
                                                (22, 2, "gray", 1)])
def test_fused_schedule_matches_oracle(qk, dt, m, alpha, order, nrhs):
    """The batched schedule (fused three-phase kernels where the size allows, the standalone
    ops beyond) against the oracle's spectral formulas: lambda, solve, quadratic form, log
    det, MLL, posterior mean/variance and gradients, per randomization and right-hand side.
    FP64 at nugget 1e-6; the FP32 precisions with one refinement step: QK_F32W (float-float
    first column) at the workloads' nugget 1e-8 with 1e-5 tolerances; QK_F32 (FP32 column)
    at nugget 1e-3, above the eps32 ||p||_2 perturbation an FP32 column gives every eigenvalue."""
    if dt == F64 and m > 20:
        pytest.skip("FP64 fused sizes end at 2^20; larger runs the standalone path, covered elsewhere")
    if dt == F32 and m > 21:
        pytest.skip("m = 22 runs the standalone ops; covered for FP32 by the solve and MLL tests")
    d, R = 5, 2
    eta = {F64: 1e-6, F32: 1e-3, F32W: 1e-8}[dt]
    gamma = 0.8 ** np.arange(1, d + 1)
    case = qc.make_case("net", "dsi", alpha, d, R, seed=2000 + m, c=gamma, zeta=1.2, order=order)
    n = 1 << m
    rng = np.random.default_rng(m)
    y_h = np.empty((R, nrhs, n))
    refs = []
    for r in range(R):
        k1, X = case.k1_ref(r, m)
        lam_ref = o.eigenvalues("dsi", k1, eta)
        for q in range(nrhs):
            y_h[r, q] = np.cos((q + 1) * X[:, 0] / 2 ** 31) + 0.01 * rng.standard_normal(n)
        refs.append((X, lam_ref))
    got = _batch_outputs(qk, case, m, nrhs, dt, y_h, eta, refine=0 if dt == F64 else 1)
    if dt == F64:
        tol = dict(lam=1e-12, c=1e-10, quad=1e-11, logdet=1e-12, mll=1e-11, mean=1e-10, var=1e-10, grad=1e-9)
    else:
        # QK_F32 (FP32 column): its eigenvalues carry ~eps32 ||p||_2 absolute, which the
        # 1/lambda-weighted quadratic form feels at the 1e-5 level (order 4 at 2^16: 1.8e-5)
        tol = dict(lam=2e-6, c=1e-5, quad=1e-5 if dt == F32W else 3e-5, logdet=1e-5, mll=1e-5, mean=1e-5, var=1e-5,
                   grad=1e-4)
    for r in range(R):
        X, lam_ref = refs[r]
        assert qc.rel_err(got["lam"][r], lam_ref) < tol["lam"], (r, qc.rel_err(got["lam"][r], lam_ref))
        if dt == F32W:  # every eigenvalue to FP32 relative precision, down to the nugget
            el = np.abs(got["lam"][r] - lam_ref) / lam_ref
            assert el.max() < 1e-5, (r, float(el.max()), float(lam_ref.min()))
        for q in range(nrhs):
            y = y_h[r, q]
            c_ref = o.spectral_solve("dsi", lam_ref, y)
            sp = o.spectral_mll("dsi", lam_ref, y, case.zeta)
            gr = o.spectral_mll_grad("dsi", alpha, X, y, lam_ref, case.c, case.zeta)
            cond = float(lam_ref.max() / lam_ref.min())
            ctol = max(tol["c"], 20 * cond * qc.EPS64) if dt != F32 else max(tol["c"], 20 * cond * qc.EPS32)
            assert qc.rel_err(got["c"][r, q], c_ref) < ctol, (r, q, qc.rel_err(got["c"][r, q], c_ref))
            o_ = got["out"][r, q]
            assert abs(o_[0] - sp["quad"]) < tol["quad"] * abs(sp["quad"])
            assert abs(o_[1] - sp["logdet"]) < tol["logdet"] * max(1.0, abs(sp["logdet"]))
            assert abs(o_[2] - sp["mll"]) < tol["mll"] * abs(sp["mll"])
            assert abs(o_[3] - sp["post_mean"]) < tol["mean"] * max(1.0, abs(sp["post_mean"]))
            assert abs(o_[4] - sp["post_var"]) < tol["var"] * case.zeta
            g_ = got["grad"][r, q]
            assert qc.rel_err(g_[:d], gr["dc"]) < tol["grad"], (qc.rel_err(g_[:d], gr["dc"]))
            assert abs(g_[d] - gr["deta"]) < tol["grad"] * max(1.0, abs(gr["deta"]))
            # dMEAN/dc_j = -zeta sum(y) / lambda_0^2 * sum_i dk1_i/dc_j, a mean-zero sum:
            # summed in FP32 it loses about sqrt(L) eps32 sum_i |dk1_i/dc_j| (L = 32 terms
            # per thread before the FP64 reduction)
            if dt == F64:
                assert qc.rel_err(g_[d + 1:2 * d + 1], gr["dmean_dc"]) < tol["grad"] * 10
            else:
                absum = _abs_dk_sums("dsi", alpha, X, case.c, case.zeta)
                lam0 = float(lam_ref[0])
                scale = abs(case.zeta * float(np.sum(y)) / lam0 ** 2) * absum
                bound = 2e-4 * np.abs(gr["dmean_dc"]) + 8 * math.sqrt(32) * qc.EPS32 * scale
                assert np.all(np.abs(g_[d + 1:2 * d + 1] - gr["dmean_dc"]) < bound)


@pytest.mark.parametrize("path,dt,m", [("standalone", F64, 8), ("standalone", F32, 8),
                                       ("fused", F64, 14), ("fused", F32, 14)])
def test_gradient_with_exact_zero_factors(qk, path, dt, m):
    """DSI order 1 with c_1 = 2: K_1 = 1 - 3 2^-beta is -1/2 wherever the first coordinate of
    the difference is >= 1/2 (beta = 1), so 1 + c_1 K_1 = 0 exactly and k_1 vanishes at half
    the points.  dk_1/dc_1 there is the product of the other factors, which the sweeps reach
    only through their exact fallback; the oracle multiplies the factors explicitly.  The
    standalone case (2^8 points in a 2^11-point tile) also has padding points whose factors
    vanish."""
    d, R, alpha = 3, 2, 1
    eta = 1e-4 if dt == F64 else 1e-3
    c = np.array([2.0, 0.6, 0.4])
    case = qc.make_case("net", "dsi", alpha, d, R, seed=4242 + m, c=c, zeta=1.0, order="gray")
    n = 1 << m
    y_h = np.empty((R, 1, n))
    refs = []
    for r in range(R):
        k1, X = case.k1_ref(r, m)
        assert np.count_nonzero(k1 == 0.0) >= n // 4  # the degenerate case is present
        lam_ref = o.eigenvalues("dsi", k1, eta)
        y_h[r, 0] = np.cos(X[:, 1] / 2 ** 31) + X[:, 0] / 2 ** 33
        refs.append((X, float(lam_ref[0]),
                     o.spectral_mll_grad("dsi", alpha, X, y_h[r, 0], lam_ref, case.c, case.zeta)))
    if path == "fused":
        grad = _batch_outputs(qk, case, m, 1, dt, y_h, eta)["grad"]
    else:
        kern, _, lam = _setup_spectrum(qk, case, m, dt, eta, R)
        y = torch.tensor(y_h, dtype=dt, device=qc.dev())
        out = torch.empty((R, 1, 5), dtype=F64, device=qc.dev())
        g = torch.empty((R, 1, 2 * d + 2), dtype=F64, device=qc.dev())
        status = torch.zeros(1, dtype=torch.int32, device=qc.dev())
        qk.mll(case.ps, kern, 0, R, m, 1, eta, lam, y, out, g, status=status)
        qk.read_status(status)
        grad = g.cpu().numpy()
    for r in range(R):
        X, lam0, gr = refs[r]
        assert np.all(np.isfinite(grad[r, 0]))
        if dt == F64:
            assert qc.rel_err(grad[r, 0, :d], gr["dc"]) < 1e-9, qc.rel_err(grad[r, 0, :d], gr["dc"])
            assert qc.rel_err(grad[r, 0, d + 1:2 * d + 1], gr["dmean_dc"]) < 1e-8
        else:
            assert qc.rel_err(grad[r, 0, :d], gr["dc"]) < 2e-4, qc.rel_err(grad[r, 0, :d], gr["dc"])
            # a sum of mean-zero terms: absolute bound from the FP32 rounding of the terms
            absum = _abs_dk_sums("dsi", alpha, X, case.c, case.zeta)
            scale = abs(case.zeta * float(np.sum(y_h[r, 0])) / lam0 ** 2) * absum
            bound = 2e-4 * np.abs(gr["dmean_dc"]) + 8 * math.sqrt(32) * qc.EPS32 * scale
            assert np.all(np.abs(grad[r, 0, d + 1:2 * d + 1] - gr["dmean_dc"]) < bound)


@pytest.mark.parametrize("m,alpha,eta", [(15, 2, 1e-4), (18, 1, 1e-5), (20, 4, 1e-4)])
def test_fused_refinement_solves_the_fp32_operator(qk, m, alpha, eta):
    """One refinement step (refine_steps = 1) with the residual carried exactly
    (compensated forward transform and exact division residual): the FP32 solve then
    matches the exact solution of K^ c = y, K^ built from the same FP32 eigenvalues,
    to the rounding of the inverse transform; the unrefined solve does not."""
    d, R, nrhs = 5, 1, 2
    case = qc.make_case("net", "dsi", alpha, d, R, seed=3000 + m, c=0.9 ** np.arange(1, d + 1))
    n = 1 << m
    k1, X = case.k1_ref(0, m)
    rng = np.random.default_rng(m)
    y_h = np.stack([np.exp(X[:, 0] / 2 ** 32) + 0.1 * rng.standard_normal(n) for _ in range(nrhs)])[None]
    y32 = y_h.astype(np.float32).astype(np.float64)
    ref = _batch_outputs(qk, case, m, nrhs, F32, y_h, eta, refine=1)
    raw = _batch_outputs(qk, case, m, nrhs, F32, y_h, eta, refine=0)
    lam_hat = ref["lam"][0]
    assert np.array_equal(lam_hat, raw["lam"][0])
    for q in range(nrhs):
        c_exact = o.spectral_solve("dsi", lam_hat, y32[0, q])
        e1 = qc.rel_err(ref["c"][0, q], c_exact)
        e0 = qc.rel_err(raw["c"][0, q], c_exact)
        assert e1 < 8 * math.sqrt(m) * qc.EPS32, (e1, e0)
        assert e1 < e0, (e1, e0)


@pytest.mark.parametrize("chunk_r", [1, 3, 8])
def test_batch_run_host_matches_device_run(qk, chunk_r):
    """qk_batch_run_host (host buffers, chunked copies overlapping compute) gives the
    device-resident schedule's results bit for bit, for every chunk size."""
    from paper_2502_14256_gb300 import inputs
    from tests import qkworkloads as W
    wl = inputs.workload("solve20")
    for dtype, refine in ((torch.float32, 1), (torch.float64, 0)):
        inst = W.build_instance(qk, wl, 15, 8, 2)
        task, bufs = W.outputs(qk, inst, dtype)
        ws = qk.workspace(qk.batch_workspace_bytes([task], dtype))
        qk.batch_plan([task], dtype, refine, ws)
        status = torch.zeros(1, dtype=torch.int32, device=qc.dev())
        qk.batch_run(ws, status)
        torch.cuda.synchronize()
        qk.read_status(status)
        ref = {k: v.clone() for k, v in bufs.items() if v is not None}
        host = {k: torch.zeros_like(v, device="cpu").pin_memory() for k, v in ref.items()}
        host["y"] = ref["y"].cpu().pin_memory()
        for v in bufs.values():
            if v is not None:
                v.zero_()
        qk.batch_run_host(ws, [host], chunk_r, status)
        torch.cuda.synchronize()
        qk.read_status(status)
        for k in ("c", "lam", "out", "grad"):
            assert torch.equal(host[k], ref[k].cpu()), (k, dtype, chunk_r)


@pytest.mark.parametrize("dtype,refine,lag", [(torch.float32, 1, 1), (torch.float32, 0, 2), (torch.float64, 0, 1)])
def test_persistent_schedule_matches_launch_sequence(qk, dtype, refine, lag):
    """QK_SCHED_PERSISTENT (one launch, ticket-ordered unit phases, slot reuse) gives the
    launch sequence's results bit for bit, on uneven n (three tasks, m = 14, 16, 15) with
    several right-hand sides, also when captured in a CUDA graph and replayed."""
    from paper_2502_14256_gb300 import inputs
    from tests import qkworkloads as W
    wl = inputs.workload("batch")
    insts = [W.build_instance(qk, wl, m, R, 3, seed_shift=i) for i, (m, R) in enumerate([(14, 5), (16, 3), (15, 4)])]
    tasks, bufs = zip(*[W.outputs(qk, inst, dtype, with_lam=(i != 1)) for i, inst in enumerate(insts)])
    ws = qk.workspace(qk.batch_workspace_bytes(list(tasks), dtype))
    qk.batch_plan(list(tasks), dtype, refine, ws)
    status = torch.zeros(1, dtype=torch.int32, device=qc.dev())
    qk.batch_run(ws, status)
    torch.cuda.synchronize()
    qk.read_status(status)
    ref = [{k: v.clone() for k, v in b.items() if v is not None} for b in bufs]
    for b in bufs:
        for k, v in b.items():
            if v is not None and k != "y":
                v.fill_(float("nan"))
    qk.batch_schedule(ws, qk.QK_SCHED_PERSISTENT, lag)
    qk.batch_run(ws, status)
    torch.cuda.synchronize()
    qk.read_status(status)
    for i, b in enumerate(bufs):
        for k in ("c", "lam", "out", "grad"):
            if b[k] is not None:
                assert torch.equal(b[k], ref[i][k]), (i, k)
    # graph capture and replay of the single launch
    for b in bufs:
        for k, v in b.items():
            if v is not None and k != "y":
                v.zero_()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            qk.batch_run(ws, status, stream=s)
    g.replay()
    torch.cuda.synchronize()
    qk.read_status(status)
    for i, b in enumerate(bufs):
        assert torch.equal(b["out"], ref[i]["out"]) and torch.equal(b["grad"], ref[i]["grad"])


DOUBLING_CASES = [("net", "dsi", 2, "gray"), ("net", "dsi", 4, "natural"), ("lattice", "si", 2, "natural")]


@pytest.mark.parametrize("kind,family,alpha,order", DOUBLING_CASES)
def test_doubling_update_of_eigenvalues_and_transforms(qk, kind, family, alpha, order):
    """Sec. 5.4 doubling updates: the column of the n new points (qk_kernel_col_at) equals
    the second half of the 2n-point column bit for bit; qk_eigs_extend equals qk_eigs of
    the 2n column (and the oracle's update); qk_fwht_extend / qk_fftbr_extend equal the
    transform of the doubled vectors."""
    m, d, R = 11, 5, 2
    n = 1 << m
    case = qc.make_case(kind, family, alpha, d, R, seed=41, order=order, m_gen=20)
    kern = qc.kernel_of(case)
    fam = qk.QK_DSI if family == "dsi" else qk.QK_SI
    eta = 1e-6
    for dtype, tol in ((F64, 1e-12), (torch.float32, 2e-6)):
        for form in (qk.QK_COL_K1, qk.QK_COL_P):
            full = torch.empty((R, 2 * n), dtype=dtype, device=qc.dev())
            qk.kernel_col(case.ps, kern, 0, R, m + 1, full, form=form)
            old = torch.empty((R, n), dtype=dtype, device=qc.dev())
            qk.kernel_col(case.ps, kern, 0, R, m, old, form=form)
            new = torch.empty((R, n), dtype=dtype, device=qc.dev())
            qk.kernel_col_at(case.ps, kern, 0, R, n, m, new, form=form)
            assert torch.equal(old, full[:, :n]) and torch.equal(new, full[:, n:])
            status = torch.zeros(1, dtype=torch.int32, device=qc.dev())
            lam_old = torch.empty((R, n), dtype=F64, device=qc.dev())
            qk.eigs(fam, m, old, lam_old, eta=eta, form=form, status=status)
            lam_ext = torch.empty((R, 2 * n), dtype=F64, device=qc.dev())
            qk.eigs_extend(fam, m, new, lam_old, lam_ext, eta=eta, form=form, status=status)
            lam_full = torch.empty((R, 2 * n), dtype=F64, device=qc.dev())
            qk.eigs(fam, m + 1, full, lam_full, eta=eta, form=form, status=status)
            torch.cuda.synchronize()
            if dtype == F64:
                qk.read_status(status)
            else:
                status.zero_()
            assert qc.rel_err(lam_ext.cpu().numpy(), lam_full.cpu().numpy()) < tol, (dtype, form)
    # against the oracle's update on the oracle's own column (FP64)
    k2, _ = case.k1_ref(1, m + 1)
    lam1 = o.eigenvalues(family, k2[:n], eta)
    want = o.extend_eigenvalues(family, lam1, k2[n:])
    new = torch.from_numpy(np.ascontiguousarray(k2[n:])).to(qc.dev()).reshape(1, n)
    lam_old = torch.from_numpy(lam1).to(qc.dev()).reshape(1, n)
    got = torch.empty((1, 2 * n), dtype=F64, device=qc.dev())
    qk.eigs_extend(fam, m, new, lam_old, got, eta=eta)
    assert qc.rel_err(got.cpu().numpy()[0], want) < 1e-13
    # transforms of doubled vectors
    g = torch.Generator(device=qc.dev()).manual_seed(3)
    cplx = family == "si"
    width = 2 if cplx else 1
    for dtype, tol in ((F64, 1e-13), (torch.float32, 1e-6)):
        y = torch.randn((3, 2 * n * width), dtype=dtype, device=qc.dev(), generator=g)
        ref = y.clone()
        (qk.fftbr if cplx else qk.fwht)(m + 1, ref)
        halves = y.view(3, 2, n * width)
        xt_old = halves[:, 0].contiguous()
        (qk.fftbr if cplx else qk.fwht)(m, xt_old)
        x_new = halves[:, 1].contiguous()
        out = torch.empty_like(y)
        (qk.fftbr_extend if cplx else qk.fwht_extend)(m, xt_old, x_new, out)
        assert qc.rel_err(out.cpu().numpy(), ref.cpu().numpy()) < tol, dtype


def test_schedule_tuner_keeps_results(qk):
    """qk_batch_tune times the launch sequence and the persistent launch (each lag), keeps
    the fastest, and the plan's results are unchanged bit for bit."""
    from paper_2502_14256_gb300 import inputs
    from tests import qkworkloads as W
    wl = inputs.workload("batch")
    insts = [W.build_instance(qk, wl, m, R, 2, seed_shift=i) for i, (m, R) in enumerate([(15, 4), (16, 2)])]
    tasks, bufs = zip(*[W.outputs(qk, inst, torch.float32, with_lam=False) for inst in insts])
    ws = qk.workspace(qk.batch_workspace_bytes(list(tasks), torch.float32))
    qk.batch_plan(list(tasks), torch.float32, 1, ws)
    status = torch.zeros(1, dtype=torch.int32, device=qc.dev())
    qk.batch_run(ws, status)
    torch.cuda.synchronize()
    qk.read_status(status)
    ref = [{k: v.clone() for k, v in b.items() if v is not None} for b in bufs]
    choice = qk.batch_tune(ws)
    assert choice["mode"] in ("launches", "persistent") and choice["ms"] > 0
    for b in bufs:
        for k, v in b.items():
            if v is not None and k != "y":
                v.zero_()
    qk.batch_run(ws, status)
    torch.cuda.synchronize()
    qk.read_status(status)
    for i, b in enumerate(bufs):
        for k in ("c", "out", "grad"):
            assert torch.equal(b[k], ref[i][k]), (i, k, choice)


def test_empty_inputs_are_no_ops(qk):
    """Zero randomizations, vectors or tasks: every entry returns QK_OK and touches nothing."""
    case = qc.make_case("net", "dsi", 2, 3, 1, seed=5)
    kern = qc.kernel_of(case)
    empty = torch.empty((0, 1 << 10), dtype=F64, device=qc.dev())
    qk.kernel_col(case.ps, kern, 0, 0, 10, empty)
    lam = torch.empty((0, 1 << 10), dtype=F64, device=qc.dev())
    qk.eigs(qk.QK_DSI, 10, empty, lam, ws=qk.workspace(256))
    qk.fwht(10, empty)
    qk.fftbr(10, torch.empty((0, 2 << 10), dtype=F64, device=qc.dev()))
    qk.fwht_ws(15, torch.empty((0, 1 << 15), dtype=torch.float32, device=qc.dev()), ws=qk.workspace(256))
    ws = qk.workspace(256)
    qk.batch_plan([], F64, 0, ws)
    status = torch.zeros(1, dtype=torch.int32, device=qc.dev())
    qk.batch_run(ws, status)
    torch.cuda.synchronize()
    qk.read_status(status)
    assert int(status.item()) == 0


def test_fp64_quotient_of_the_gradient_sweeps(qk):
    """The FP64 sweeps' a / b (Newton steps on the FP32 reciprocal estimate) against numpy's
    correctly rounded division: within 2 ulp over a wide range of magnitudes and signs, and
    exactly the divide outside 2^-100 .. 2^100 (where the sweeps take it)."""
    rng = np.random.default_rng(17)
    n = 1 << 20
    b = rng.uniform(0.5, 1.0, n) * 2.0 ** rng.integers(-99, 99, n) * rng.choice([-1.0, 1.0], n)
    a = rng.standard_normal(n) * 2.0 ** rng.integers(-300, 300, n)
    # the sweeps' own argument range: 1 + c K near 1, and values close to powers of two
    b[:4096] = 1.0 + rng.uniform(-0.999, 3.0, 4096)
    b[4096:8192] = np.nextafter(2.0 ** rng.integers(-60, 60, 4096), 0.0)
    b[8192:8200] = [2.0 ** 101, -2.0 ** -101, 1e300, 1e-300, 5e-324, 0.0, np.inf, -np.inf]
    at = torch.tensor(a, dtype=F64, device=qc.dev())
    bt = torch.tensor(b, dtype=F64, device=qc.dev())
    q = qk.ratio_selftest(at, bt).cpu().numpy()
    with np.errstate(divide="ignore", invalid="ignore"):
        want = a / b
    fast = (np.abs(b) >= 2.0 ** -100) & (np.abs(b) <= 2.0 ** 100)
    ulp = np.spacing(np.abs(want[fast]))
    assert np.all(np.abs(q[fast] - want[fast]) <= 2 * ulp), float(np.max(np.abs(q[fast] - want[fast]) / ulp))
    slow = ~fast
    assert np.array_equal(q[slow], want[slow], equal_nan=True)
