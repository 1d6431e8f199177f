"""The torch.autograd.Function over the library's MLL and posterior mean: gradients with
respect to weights, log-lengthscales and log-nugget against the oracle's dense gradient
(Cholesky; d MLL/d theta = c^T dK c/2 - tr(K^-1 dK)/2) and against central differences."""
import numpy as np
import pytest
import torch

from oracle import qk_oracle as o
from paper_2502_14256_gb300 import inputs
from tests import qkworkloads as W

pytestmark = pytest.mark.gpu
F64 = torch.float64


@pytest.fixture(scope="module")
def qk():
    from paper_2502_14256_gb300 import build
    build.build()
    from paper_2502_14256_gb300 import qk as q
    return q


def _params(wl, log_ls=None):
    dev = torch.device("cuda:0")
    gamma = torch.tensor(wl.gamma, dtype=F64, device=dev, requires_grad=True)
    th = torch.tensor(wl.log_ls if log_ls is None else log_ls, dtype=F64, device=dev, requires_grad=True)
    le = torch.tensor(np.log(wl.eta), dtype=F64, device=dev, requires_grad=True)
    return gamma, th, le


@pytest.mark.parametrize("name,log_ls", [("plain", [0.3, -0.2, 0.1, 0.0]), ("diff_small", None)])
def test_autograd_matches_dense_oracle(qk, name, log_ls):
    from paper_2502_14256_gb300.autograd import mll_and_mean
    wl = inputs.workload(name)
    if log_ls is not None:
        wl.log_ls = np.asarray(log_ls)
    m = wl.ms[0]
    inst = W.build_instance(qk, wl, m, 1, 1, y_kind="product")
    gamma, th, le = _params(wl)
    fam = qk.QK_DSI if wl.family == "dsi" else qk.QK_SI
    mll, mean = mll_and_mean(gamma, th, le, inst.y64, inst.ps, fam, wl.alpha, m, wl.zeta)
    g_mll = torch.autograd.grad(mll.sum(), (gamma, th, le), retain_graph=True)
    g_mean = torch.autograd.grad(mean.sum(), (gamma, th, le))
    X = W.host_points(inst, 0, np.arange(1 << m))
    y = W.host_rhs(inst, 0, X)[0]
    ref = o.mll_grad_dense(wl.family, wl.alpha, X, y, wl.gamma, wl.log_ls, wl.eta, wl.zeta)
    rel = lambda a, b: float(np.max(np.abs(np.asarray(a) - b)) / max(np.max(np.abs(b)), 1e-300))  # noqa: E731
    assert rel(g_mll[0].cpu().numpy(), ref["dgamma"]) < 1e-9
    assert rel(g_mll[1].cpu().numpy(), ref["dtheta"]) < 1e-9
    assert abs(float(g_mll[2]) - ref["dlog_eta"]) < 1e-9 * max(1.0, abs(ref["dlog_eta"]))
    c_w = o.effective_weights(wl.gamma, wl.log_ls)
    assert rel(g_mean[1].cpu().numpy(), c_w * ref["dmean_dc"]) < 1e-8
    assert abs(float(g_mean[2]) - wl.eta * ref["dmean_deta"]) < 1e-8 * max(1.0, abs(wl.eta * ref["dmean_deta"]))
    assert abs(float(mean) - ref["post_mean"]) < 1e-10 * max(1.0, abs(ref["post_mean"]))


def test_autograd_matches_central_differences(qk):
    """Central differences (h = 1e-6) of the library's own forward, through the Function."""
    from paper_2502_14256_gb300.autograd import mll_and_mean
    wl = inputs.workload("diff_small")
    m = wl.ms[0]
    inst = W.build_instance(qk, wl, m, 1, 1, y_kind="product")
    gamma, th, le = _params(wl)
    spec = (inst.ps, qk.QK_SI, wl.alpha, m, wl.zeta)

    def f(g, t, e):
        return mll_and_mean(g, t, e, inst.y64, spec[0], spec[1], spec[2], spec[3], spec[4])[0].sum()

    gg, gt, ge = torch.autograd.grad(f(gamma, th, le), (gamma, th, le))
    h = 1e-6
    with torch.no_grad():
        for j in (0, 5, 31):
            tp, tm = th.detach().clone(), th.detach().clone()
            tp[j] += h
            tm[j] -= h
            fd = (float(f(gamma.detach(), tp, le.detach())) - float(f(gamma.detach(), tm, le.detach()))) / (2 * h)
            assert abs(fd - float(gt[j])) < 1e-5 * max(1.0, abs(fd)), (j, fd, float(gt[j]))
        fd = (float(f(gamma.detach(), th.detach(), le.detach() + h))
              - float(f(gamma.detach(), th.detach(), le.detach() - h))) / (2 * h)
        assert abs(fd - float(ge)) < 1e-5 * max(1.0, abs(fd)), (fd, float(ge))
