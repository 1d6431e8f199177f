"""RQMC integration on the GPU through the C ABI against the oracle: the six test integrands
of Sec. 6 at the points of nets (Gray and natural order) and lattices, with and without the
baker transform (Sec. 4.2), over ragged position ranges; the RQMC estimate and Student-t
interval of Sec. 3.1; the squared worst-case error of Sec. 3.2 (closed forms for equal and
optimal weights, general weights through the spectrum)."""
import math

import numpy as np
import pytest
import torch

from oracle import qk_oracle as o
from tests import qkcases as qc

pytestmark = pytest.mark.gpu
F64, F32 = torch.float64, torch.float32
DIMS = {"simple1": 1, "simple2": 2, "oakley": 2, "gfun": 3, "genz_osc": 5, "genz_cp": 7}


@pytest.fixture(scope="module")
def qk():
    from paper_2502_14256_gb300 import build
    build.build()
    from paper_2502_14256_gb300 import qk as q
    return q


@pytest.mark.parametrize("name", list(DIMS))
@pytest.mark.parametrize("kind,order", [("net", "gray"), ("net", "natural"), ("lattice", "natural")])
@pytest.mark.parametrize("baker", [False, True])
def test_integrand_values(qk, name, kind, order, baker):
    d, R = DIMS[name], 3
    case = qc.make_case(kind, "dsi" if kind == "net" else "si", 2, d, R, seed=700 + d, order=order)
    for i0, n in ((0, 4096), (2048 * 3 + 5, 3001)):
        for dt, tol in ((F64, 1e-14), (F32, 2e-6)):
            y = torch.empty((2, n), dtype=dt, device=qc.dev())
            qk.integrand(case.ps, 1, 2, i0, n, name, y, baker=baker)
            got = y.cpu().numpy().astype(np.float64)
            for r in (1, 2):
                X = case.points_ref(r, np.arange(i0, i0 + n), 20)
                x = X.astype(np.float64) / 2.0 ** 32
                want = o.integrand(name, o.baker(x) if baker else x)
                err = np.max(np.abs(got[r - 1] - want)) / max(1.0, np.max(np.abs(want)))
                assert err < tol, (name, kind, order, baker, dt, r, i0, err)


def test_rqmc_estimate_and_interval(qk):
    """The corner-peak Genz function in d = 50 with R = 10 randomizations of a 2^15-point net
    (the shape of the paper's RQMC example, Sec. 6): per-randomization means, estimate, sigma
    and the 99% Student-t half width against the oracle on the same values; the interval
    covers the exact mean."""
    d, R, m, tau = 50, 10, 15, 0.01
    n = 1 << m
    case = qc.make_case("net", "dsi", 2, d, R, seed=2025, order="gray")
    y = torch.empty((R, n), dtype=F64, device=qc.dev())
    qk.integrand(case.ps, 0, R, 0, n, "genz_cp", y)
    out = qk.rqmc(y, tau).cpu().numpy()
    est = o.rqmc_estimate(y.cpu().numpy(), tau)
    assert np.allclose(out[4:], est["mu_r"], rtol=1e-14, atol=0)
    for k, key in enumerate(("mu", "sigma", "half_width", "t")):
        assert math.isclose(out[k], est[key], rel_tol=1e-10), (key, out[k], est[key])
    exact = o.integrand_mean("genz_cp", 3)  # sanity of the 3-d closed form vs a 3-d run below
    y3 = torch.empty((R, n), dtype=F64, device=qc.dev())
    case3 = qc.make_case("net", "dsi", 2, 3, R, seed=2026, order="gray")
    qk.integrand(case3.ps, 0, R, 0, n, "genz_cp", y3)
    out3 = qk.rqmc(y3, tau).cpu().numpy()
    assert abs(out3[0] - exact) <= 2.0 * out3[2] + 1e-12, (out3[0], exact, out3[2])
    # FP32 values: the same reduction in FP64
    y32 = y.to(F32)
    out32 = qk.rqmc(y32, tau).cpu().numpy()
    est32 = o.rqmc_estimate(y32.cpu().numpy().astype(np.float64), tau)
    assert math.isclose(out32[0], est32["mu"], rel_tol=1e-12)


@pytest.mark.parametrize("kind,family,alpha", [("net", "dsi", 2), ("net", "dsi", 4), ("lattice", "si", 1),
                                               ("lattice", "si", 2)])
def test_discrepancy_closed_forms_against_dense_oracle(qk, kind, family, alpha):
    m, d, R, zeta = 8, 3, 2, 1.4
    n = 1 << m
    case = qc.make_case(kind, family, alpha, d, R, seed=800 + alpha, c=0.7 ** np.arange(1, d + 1), zeta=zeta)
    kern = qc.kernel_of(case)
    col = torch.empty((R, n), dtype=F64, device=qc.dev())
    qk.kernel_col(case.ps, kern, 0, R, m, col, form=qk.QK_COL_P)
    out = qk.discrepancy(qk.QK_DSI if family == "dsi" else qk.QK_SI, m, col, zeta=zeta).cpu().numpy()
    for r in range(R):
        _, X = case.k1_ref(r, m)
        w_eq = np.full(n, 1.0 / n)
        d_eq = o.discrepancy2_dense(family, alpha, X, case.c, zeta, w_eq)
        w_opt = o.optimal_weights_dense(family, alpha, X, case.c, zeta)
        d_opt = o.discrepancy2_dense(family, alpha, X, case.c, zeta, w_opt)
        # the dense forms cancel (zeta - 2 zeta + ...): absolute FP64 error about n eps zeta
        assert abs(out[r, 0] - d_eq) < 1e-12 * zeta * n, (r, out[r, 0], d_eq)
        assert abs(out[r, 1] - d_opt) < 1e-12 * zeta * n, (r, out[r, 1], d_opt)
        assert math.isclose(out[r, 2], w_opt.mean(), rel_tol=1e-10)


@pytest.mark.parametrize("kind,family,alpha,m", [("net", "dsi", 2, 9), ("net", "dsi", 3, 14),
                                                 ("lattice", "si", 2, 9), ("lattice", "si", 1, 14)])
def test_discrepancy_of_given_weights(qk, kind, family, alpha, m):
    """General weights through the spectrum: against the dense definition (m = 9) and the
    oracle's spectral form (m = 14); random weights and the equal weights as two vectors."""
    d, R, zeta, nw = 4, 2, 0.9, 3
    n = 1 << m
    case = qc.make_case(kind, family, alpha, d, R, seed=900 + m, c=0.6 ** np.arange(1, d + 1), zeta=zeta)
    kern = qc.kernel_of(case)
    fam = qk.QK_DSI if family == "dsi" else qk.QK_SI
    col = torch.empty((R, n), dtype=F64, device=qc.dev())
    qk.kernel_col(case.ps, kern, 0, R, m, col, form=qk.QK_COL_P)
    lam = torch.empty((R, n), dtype=F64, device=qc.dev())
    qk.eigs(fam, m, col, lam, zeta=zeta, eta=0.0, form=qk.QK_COL_P)
    rng = np.random.default_rng(m)
    w_h = np.abs(rng.standard_normal((R, nw, n))) / n
    w_h[:, 0] = 1.0 / n
    out = qk.discrepancy_weights(fam, m, lam, torch.tensor(w_h, dtype=F64, device=qc.dev()), zeta=zeta).cpu().numpy()
    for r in range(R):
        k1, X = case.k1_ref(r, m)
        lam_ref = o.eigenvalues(family, k1, 0.0)
        for q in range(nw):
            want = (o.discrepancy2_dense(family, alpha, X, case.c, zeta, w_h[r, q]) if m <= 9
                    else o.discrepancy2_spectral(family, lam_ref, w_h[r, q], zeta))
            assert abs(out[r, q] - want) < 1e-12 * zeta * max(1.0, abs(want) * n), (r, q, out[r, q], want)
