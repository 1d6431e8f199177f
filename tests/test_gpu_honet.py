"""Higher-order nets on the GPU through the C ABI against the oracle (Sec. 4.3 interlacing
with higher-order LMS; Sec. 5.3 DSI kernels on their 64-digit points): interlaced columns
and points bit for bit, the first column in FP64 and FP32, and the spectral solve and MLL
pieces of an interlaced net with order-2 and order-4 kernels against dense Cholesky."""
import math

import numpy as np
import pytest
import torch

from oracle import qk_oracle as o
from paper_2502_14256_gb300 import inputs
from tests import qkcases as qc

pytestmark = pytest.mark.gpu
F64, F32 = torch.float64, torch.float32


@pytest.fixture(scope="module")
def qk():
    from paper_2502_14256_gb300 import build
    build.build()
    from paper_2502_14256_gb300 import qk as q
    return q


def _u64(a):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.uint64)).view(np.int64)).to(qc.dev())


def _ho_set(qk, d, alpha, R, order, seed):
    net = inputs.make_ho_net(seed, d, alpha, R, order)
    Cd, Sd = qc.u32_tensor(net.C), qc.u32_tensor(net.S)
    Ct = torch.empty((R, alpha * d, 32), dtype=torch.int32, device=qc.dev())
    qk.lms_setup(Cd, Sd, Ct)
    Chat = torch.empty((R, d, 32), dtype=torch.int64, device=qc.dev())
    qk.interlace(alpha, Ct, Chat)
    Dd = _u64(net.D)
    ps = qk.ho_pointset(d, R, Chat, Dd, order=qk.QK_GRAY if order == "gray" else qk.QK_NATURAL)
    Chat_ref = [o.interlace(o.lms_scramble(net.C, net.S[r:r + 1])[0], alpha) for r in range(R)]
    return ps, net, Chat, Chat_ref, [Cd, Sd, Ct, Chat, Dd]


@pytest.mark.parametrize("alpha,order", [(2, "gray"), (3, "natural"), (4, "gray")])
def test_interlaced_columns_and_points_bit_exact(qk, alpha, order):
    d, R = 5, 3
    ps, net, Chat, Chat_ref, keep = _ho_set(qk, d, alpha, R, order, 40 + alpha)
    got = Chat.cpu().numpy().view(np.uint64)
    for r in range(R):
        assert np.array_equal(got[r], Chat_ref[r]), r
    for i0, n in ((0, 4096), (4096 * 5 + 3, 2999)):
        X = torch.empty((2, n, d), dtype=torch.int64, device=qc.dev())
        qk.gen_points_ho(ps, 1, 2, i0, n, X)
        gx = X.cpu().numpy().view(np.uint64)
        for r in (1, 2):
            want = o.ho_net_points(Chat_ref[r], net.D[r], np.arange(i0, i0 + n), 20, order)
            assert np.array_equal(gx[r - 1], want), (r, i0)


@pytest.mark.parametrize("alpha_net,alpha_k", [(2, 1), (2, 2), (2, 3), (2, 4), (4, 2), (4, 4)])
@pytest.mark.parametrize("m", [3, 12])
def test_higher_order_first_column(qk, alpha_net, alpha_k, m):
    d, R, zeta = 4, 2, 1.3
    ps, net, Chat, Chat_ref, keep = _ho_set(qk, d, alpha_net, R, "gray", 50 + alpha_k)
    c = 0.8 ** np.arange(1, d + 1)
    w = torch.tensor(c, dtype=F64, device=qc.dev())
    kern = qk.kernel(qk.QK_DSI, alpha_k, w, zeta)
    n = 1 << m
    for dt, tol in ((F64, 1e-13), (F32, 2e-5)):
        for form in (qk.QK_COL_K1, qk.QK_COL_P):
            col = torch.empty((R, n), dtype=dt, device=qc.dev())
            qk.kernel_col_ho(ps, kern, 0, R, m, col, form=form)
            got = col.cpu().numpy().astype(np.float64)
            for r in range(R):
                X = o.ho_net_points(Chat_ref[r], net.D[r], np.arange(n), m, "gray")
                k1 = o.ho_first_column(alpha_k, X, c, zeta)
                g = got[r] if form == qk.QK_COL_K1 else zeta * (1.0 + got[r])
                assert qc.rel_err(g, k1) < tol, (dt, form, r, qc.rel_err(g, k1))


@pytest.mark.parametrize("alpha_net,alpha_k", [(2, 2), (2, 4), (3, 4)])
def test_higher_order_solve_and_mll_against_dense(qk, alpha_net, alpha_k):
    """An interlaced net with a DSI kernel of matching order: eigenvalues by the FWHT of the
    64-digit column, then solve and MLL pieces, against Cholesky on the dense Gram matrix."""
    d, R, m, zeta, eta = 3, 2, 9, 1.0, 1e-8
    n = 1 << m
    ps, net, Chat, Chat_ref, keep = _ho_set(qk, d, alpha_net, R, "gray", 60 + alpha_k)
    c = 0.7 ** np.arange(1, d + 1)
    w = torch.tensor(c, dtype=F64, device=qc.dev())
    kern = qk.kernel(qk.QK_DSI, alpha_k, w, zeta)
    col = torch.empty((R, n), dtype=F64, device=qc.dev())
    qk.kernel_col_ho(ps, kern, 0, R, m, col, form=qk.QK_COL_P)
    lam = torch.empty((R, n), dtype=F64, device=qc.dev())
    qk.eigs(qk.QK_DSI, m, col, lam, zeta=zeta, eta=eta, form=qk.QK_COL_P)
    y_h = np.empty((R, 1, n))
    Xs = []
    for r in range(R):
        X = o.ho_net_points(Chat_ref[r], net.D[r], np.arange(n), m, "gray")
        Xs.append(X)
        x = X.astype(np.float64) / 2.0 ** 64
        y_h[r, 0] = np.prod(1.0 + (x - 0.5) / np.arange(1, d + 1) ** 2, axis=1)
    y = torch.tensor(y_h, dtype=F64, device=qc.dev())
    csol = torch.empty_like(y)
    qk.solve(qk.QK_DSI, m, lam, y, csol)
    out = torch.empty((R, 1, qk.QK_MLL_NOUT), dtype=F64, device=qc.dev())
    qk.mll_spectrum(qk.QK_DSI, m, lam, y, out, zeta=zeta)
    got_c, got_o = csol.cpu().numpy(), out.cpu().numpy()
    for r in range(R):
        K = o.ho_gram_dense(alpha_k, Xs[r], c, zeta, eta)
        c_ref, logdet = o.cholesky_solve(K, y_h[r, 0])
        mll = o.mll_dense(K, y_h[r, 0])[0]
        mean, var = o.bc_posterior_dense(K, y_h[r, 0], zeta)
        lam_ref = np.linalg.eigvalsh(K)
        tol = qc.cond_tol(lam_ref, 1e-10, qc.EPS64)
        assert qc.rel_err(got_c[r, 0], c_ref) < tol, (r, qc.rel_err(got_c[r, 0], c_ref), tol)
        assert abs(got_o[r, 0, 1] - logdet) < 1e-10 * abs(logdet)
        assert abs(got_o[r, 0, 2] - mll) < 1e-9 * abs(mll), (got_o[r, 0, 2], mll)
        assert abs(got_o[r, 0, 3] - mean) < 1e-9 * max(1.0, abs(mean))
        assert abs(got_o[r, 0, 4] - var) < 1e-9 * max(1.0, abs(var)) + 1e-12


@pytest.mark.parametrize("alpha_net,alpha_k,dt", [(2, 2, F64), (2, 4, F64), (3, 3, F64), (2, 2, F32)])
def test_higher_order_mll_gradient_against_dense(qk, alpha_net, alpha_k, dt):
    """qk_mll_ho: MLL pieces and the gradient (factors recomputed from the 64-digit words)
    against the dense Cholesky forms on an interlaced net (2^8 points)."""
    d, R, m, zeta, eta = 3, 2, 8, 1.0, 1e-6
    n = 1 << m
    ps, net, Chat, Chat_ref, keep = _ho_set(qk, d, alpha_net, R, "gray", 70 + alpha_k)
    c = np.array([0.9, 0.5, 0.3])
    w = torch.tensor(c, dtype=F64, device=qc.dev())
    kern = qk.kernel(qk.QK_DSI, alpha_k, w, zeta)
    col = torch.empty((R, n), dtype=F64, device=qc.dev())
    qk.kernel_col_ho(ps, kern, 0, R, m, col, form=qk.QK_COL_P)
    lam = torch.empty((R, n), dtype=F64, device=qc.dev())
    qk.eigs(qk.QK_DSI, m, col, lam, zeta=zeta, eta=eta, form=qk.QK_COL_P)
    Xs = [o.ho_net_points(Chat_ref[r], net.D[r], np.arange(n), m, "gray") for r in range(R)]
    y_h = np.stack([np.cos(X[:, 0].astype(np.float64) / 2.0 ** 63) for X in Xs])[:, None, :]
    y = torch.tensor(y_h, dtype=dt, device=qc.dev())
    out = torch.empty((R, 1, qk.QK_MLL_NOUT), dtype=F64, device=qc.dev())
    grad = torch.empty((R, 1, 2 * d + 2), dtype=F64, device=qc.dev())
    qk.mll_ho(ps, kern, 0, R, m, 1, lam, y, out, grad)
    go, gg = out.cpu().numpy(), grad.cpu().numpy()
    tol = 1e-9 if dt == F64 else 2e-4
    for r in range(R):
        yr = y.cpu().numpy().astype(np.float64)[r, 0]
        K = o.ho_gram_dense(alpha_k, Xs[r], c, zeta, eta)
        mll = o.mll_dense(K, yr)[0]
        g = o.ho_mll_grad_dense(alpha_k, Xs[r], yr, c, eta, zeta)
        assert abs(go[r, 0, 2] - mll) < max(tol, 1e-10) * abs(mll), (r, go[r, 0, 2], mll)
        assert qc.rel_err(gg[r, 0, :d], g["dc"]) < tol, (r, qc.rel_err(gg[r, 0, :d], g["dc"]))
        assert abs(gg[r, 0, d] - g["deta"]) < tol * max(1.0, abs(g["deta"]))
