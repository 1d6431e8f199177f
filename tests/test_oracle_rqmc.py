"""Pins of the oracle's RQMC pieces against what the mathematics fixes (no GPU):
the six test integrands of Sec. 6 against their closed-form means (by quadrature), the
baker transform's mean preservation (Sec. 4.2), the Student-t interval of Sec. 3.1
against printed t-table values and a coverage experiment, and the squared worst-case
error of Sec. 3.2 (kappa_i = zeta, optimal weights, spectral = dense)."""
import math

import numpy as np
import pytest

from oracle import qk_oracle as o
from paper_2502_14256_gb300 import inputs

DIMS = {"simple1": 1, "simple2": 2, "oakley": 2, "gfun": 3, "genz_osc": 3, "genz_cp": 3}


def _grid(d, k):
    """Midpoints of the regular grid with 2^k cells per axis, shape (2^(k d), d)."""
    t = (np.arange(1 << k) + 0.5) / (1 << k)
    return np.stack(np.meshgrid(*([t] * d), indexing="ij"), axis=-1).reshape(-1, d)


@pytest.mark.parametrize("name", list(DIMS))
def test_integrand_means_match_closed_forms(name):
    d = DIMS[name]
    k = {1: 20, 2: 10, 3: 7}[d]
    x = _grid(d, k)
    quad = float(np.mean(o.integrand(name, x)))
    exact = o.integrand_mean(name, d)
    # midpoint rule: O(h^2) for these smooth (or cell-wise linear) integrands
    assert abs(quad - exact) < 2e-4 * max(1.0, abs(exact)), (name, quad, exact)
    # the baker transform maps U[0,1]^d to itself: same mean
    quad_b = float(np.mean(o.integrand(name, o.baker(x))))
    assert abs(quad_b - exact) < 2e-4 * max(1.0, abs(exact)), (name, quad_b, exact)


def test_gfun_second_moment():
    """The mean alone cannot tell a_j from -a_j here ({-1/2, 0, 1/2} is symmetric); the second
    moment can: E[(|4x - 2| - a)^2] = 4/3 - 2a + a^2 per factor (E|4x - 2|^2 = 4/3)."""
    d = 3
    a = (np.arange(1, d + 1) - 2.0) / 2.0
    want = float(np.prod((4.0 / 3.0 - 2.0 * a + a ** 2) / (1.0 + a) ** 2))
    x = _grid(d, 7)
    got = float(np.mean(o.integrand("gfun", x) ** 2))
    assert abs(got - want) < 1e-3 * want, (got, want)


def test_corner_peak_closed_form_in_one_and_two_dimensions():
    """The iterated-integration closed form against direct antiderivatives: d = 1 gives
    (1 - 1/(1 + c))/c; d = 2 gives (1/(1+c1+c2) - 1/(1+c1) - 1/(1+c2) + 1) / (2 c1 c2)."""
    c1 = o._genz_coefficients("corner", 1)[0]
    assert math.isclose(o.integrand_mean("genz_cp", 1), (1 - 1 / (1 + c1)) / c1, rel_tol=1e-14)
    a, b = o._genz_coefficients("corner", 2)
    want = (1 / (1 + a + b) - 1 / (1 + a) - 1 / (1 + b) + 1) / (2 * a * b)
    assert math.isclose(o.integrand_mean("genz_cp", 2), want, rel_tol=1e-12)
    x = _grid(2, 10)
    assert abs(np.mean(o.integrand("genz_cp", x)) - want) < 1e-6


def test_genz_coefficients_follow_their_kinds():
    c = o._genz_coefficients("oscillatory", 5)
    assert math.isclose(c.sum(), 4.5) and np.all(np.diff(np.log(c)) < 0)
    assert np.allclose(np.diff(np.log(c)), math.log(1e-8) / 5)  # geometric with ratio 1e-8^(1/d)
    c = o._genz_coefficients("corner", 4)
    assert math.isclose(c.sum(), 0.25) and np.allclose(c * np.arange(1, 5) ** 2, c[0])


def test_baker_transform_values():
    x = np.array([0.0, 0.25, 0.5, 0.75, 1.0 - 2.0 ** -32])
    assert np.array_equal(o.baker(x), [0.0, 0.5, 1.0, 0.5, 2.0 ** -31])


def test_student_t_interval_against_table_values():
    """t quantiles printed in standard t tables (two-sided 99% with 9 degrees of freedom:
    3.250; 95% with 14: 2.145; 90% with 4: 2.132), and the interval formula on a sample whose
    spread is known: rows y_r = r give mu = (R - 1)/2 and sigma^2 = R (R + 1)/12."""
    R = 10
    y = np.repeat(np.arange(R, dtype=np.float64)[:, None], 64, axis=1)
    est = o.rqmc_estimate(y, 0.01)
    assert round(est["t"], 3) == 3.250
    assert math.isclose(est["mu"], (R - 1) / 2)
    assert math.isclose(est["sigma"] ** 2, R * (R + 1) / 12)
    assert math.isclose(est["half_width"], est["t"] * est["sigma"] / math.sqrt(R))
    assert round(o.rqmc_estimate(np.zeros((15, 4)), 0.05)["t"], 3) == 2.145
    assert round(o.rqmc_estimate(np.zeros((5, 4)), 0.10)["t"], 3) == 2.132


def test_student_t_interval_covers_at_its_level():
    """With IID normal randomization means the interval covers the true mean for about
    100(1 - tau)% of repetitions (2000 repetitions of R = 8, tau = 0.1)."""
    rng = inputs.SplitMix64(77)
    reps, R, tau = 2000, 8, 0.1
    z = rng.normal(reps * R).reshape(reps, R, 1)
    hits = 0
    for k in range(reps):
        est = o.rqmc_estimate(z[k], tau)
        hits += abs(est["mu"]) <= est["half_width"]
    assert abs(hits / reps - (1 - tau)) < 0.025, hits / reps


@pytest.mark.parametrize("family,alpha", [("dsi", 1), ("dsi", 2), ("dsi", 3), ("dsi", 4), ("si", 1), ("si", 2)])
def test_kernel_integrates_to_zero_in_each_argument(family, alpha):
    """kappa_i = int K(u, x_i) du = zeta needs int_0^1 K_alpha(u, x) du = 0 for every x."""
    rng = inputs.SplitMix64(11 * alpha + (family == "si"))
    for x in rng.u32(4):
        assert abs(o.kernel_mean_1d(family, alpha, int(x))) < 2e-3 * (10.0 if alpha == 1 else 1.0)


@pytest.mark.parametrize("kind,family,alpha", [("net", "dsi", 2), ("net", "dsi", 4), ("lattice", "si", 1)])
def test_discrepancy_equal_and_optimal_weights(kind, family, alpha):
    """Equal weights 1/n: squared WCE = lambda_0/n - zeta (1 is the w = 0 eigenvector);
    optimal weights K^-1 kappa are the constant zeta/lambda_0 and reach zeta - zeta^2 n/lambda_0,
    the Bayesian-cubature posterior variance; any other weights do worse; the spectral form
    equals the dense one for random weights."""
    m, d, zeta = 7, 3, 1.3
    n = 1 << m
    c = 0.7 ** np.arange(1, d + 1)
    if kind == "net":
        net = inputs.make_net(500 + alpha, d, 1, "gray")
        X = o.net_points(o.lms_scramble(net.C, net.S)[0], net.D[0], np.arange(n), m, "gray")
    else:
        lat = inputs.make_lattice(500 + alpha, d, 1, m)
        X = o.lattice_points(lat.g, lat.D[0], np.arange(n))
    k1 = o.first_column(family, alpha, X, c, zeta)
    lam = o.eigenvalues(family, k1, 0.0)
    lam0 = float(lam[0])
    w_eq = np.full(n, 1.0 / n)
    assert math.isclose(o.discrepancy2_dense(family, alpha, X, c, zeta, w_eq), lam0 / n - zeta,
                        rel_tol=1e-9, abs_tol=1e-13)
    w_opt = o.optimal_weights_dense(family, alpha, X, c, zeta)
    assert np.allclose(w_opt, zeta / lam0, rtol=1e-9)
    d_opt = o.discrepancy2_dense(family, alpha, X, c, zeta, w_opt)
    K = o.gram_dense(family, alpha, X, c, zeta, 0.0)
    _, var = o.bc_posterior_dense(K, np.ones(n), zeta)
    assert math.isclose(d_opt, zeta - zeta ** 2 * n / lam0, rel_tol=1e-8, abs_tol=1e-13)
    assert math.isclose(d_opt, var, rel_tol=1e-8, abs_tol=1e-13)
    rng = np.random.default_rng(alpha)
    for _ in range(5):
        w = w_opt + 1e-3 * rng.standard_normal(n)
        assert o.discrepancy2_dense(family, alpha, X, c, zeta, w) > d_opt
        assert math.isclose(o.discrepancy2_spectral(family, lam, w, zeta),
                            o.discrepancy2_dense(family, alpha, X, c, zeta, w), rel_tol=1e-9)
