"""torch.autograd.Function over the library's marginal log-likelihood and Bayesian-cubature
posterior mean (Sec. 3.2 with the spectral forms of Sec. 5.4).

The hyper-parameters are per-dimension weights gamma_j, log-lengthscales theta_j (effective
weight c_j = gamma_j exp(theta_j)) and the log-nugget log(eta).  The forward pass runs the
library's kernels: first column in the p = k_1/zeta - 1 form (qk_kernel_col), eigenvalues
(qk_eigs) and the MLL with its gradient block (qk_mll), whose hand-written gradient carries
g_w = (|y~_w|^2/lambda_w^2 - 1/lambda_w)/2 back through the transform and recomputes the
kernel factors.  The backward pass only contracts that block with the incoming gradients and
applies the chain rule from c_j and eta to the parameters.
"""
from __future__ import annotations

import torch

from . import qk


class BayesCubatureMLL(torch.autograd.Function):
    """Returns (mll, post_mean), each of shape (nr, nrhs), for randomizations r0 .. r0+nr-1.

    forward(gamma (d,), log_ls (d,), log_eta (), y (nr, nrhs, n), spec) with spec a
    tuple (ps, family, alpha, zeta, m, r0); gamma, log_ls, log_eta FP64 device tensors;
    y in the computation dtype (FP64 or FP32).  y is data: no gradient flows to it.
    """

    @staticmethod
    def forward(ctx, gamma, log_ls, log_eta, y, spec):
        ps, family, alpha, zeta, m, r0 = spec
        nr, nrhs, n = y.shape
        if n != 1 << m:
            raise ValueError(f"y has {n} points per right-hand side, 2^{m} expected")
        c = (gamma * torch.exp(log_ls)).to(torch.float64).contiguous()
        eta = float(torch.exp(log_eta))
        kern = qk.kernel(family, alpha, c, zeta)
        col = torch.empty((nr, n), dtype=y.dtype, device=y.device)
        qk.kernel_col(ps, kern, r0, nr, m, col, form=qk.QK_COL_P)
        lam = torch.empty((nr, n), dtype=torch.float64, device=y.device)
        status = torch.zeros(1, dtype=torch.int32, device=y.device)
        qk.eigs(family, m, col, lam, zeta=zeta, eta=eta, form=qk.QK_COL_P, status=status)
        out = torch.empty((nr, nrhs, qk.QK_MLL_NOUT), dtype=torch.float64, device=y.device)
        want_grad = any(ctx.needs_input_grad[:3])
        d = c.numel()
        grad = torch.empty((nr, nrhs, 2 * d + 2), dtype=torch.float64, device=y.device) if want_grad else None
        qk.mll(ps, kern, r0, nr, m, nrhs, eta, lam, y.contiguous(), out, grad, status=status)
        qk.read_status(status)
        if want_grad:
            ctx.save_for_backward(grad, c, torch.exp(log_ls), torch.exp(log_eta))
        ctx.d = d
        return out[..., qk.QK_MLL_MLL].clone(), out[..., qk.QK_MLL_MEAN].clone()

    @staticmethod
    def backward(ctx, g_mll, g_mean):
        grad, c, ls, eta = ctx.saved_tensors
        d = ctx.d
        g_mll = torch.zeros_like(grad[..., 0]) if g_mll is None else g_mll.to(torch.float64)
        g_mean = torch.zeros_like(grad[..., 0]) if g_mean is None else g_mean.to(torch.float64)
        dc = (g_mll[..., None] * grad[..., :d] + g_mean[..., None] * grad[..., d + 1:2 * d + 1]).sum(dim=(0, 1))
        deta = (g_mll * grad[..., d] + g_mean * grad[..., 2 * d + 1]).sum()
        return dc * ls, dc * c, deta * eta, None, None


def mll_and_mean(gamma, log_ls, log_eta, y, ps, family: int, alpha: int, m: int, zeta: float = 1.0, r0: int = 0):
    """Differentiable (mll, post_mean) of shape (nr, nrhs); see BayesCubatureMLL."""
    return BayesCubatureMLL.apply(gamma, log_ls, log_eta, y, (ps, family, alpha, zeta, m, r0))
