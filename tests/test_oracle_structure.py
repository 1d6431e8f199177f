"""Pins of the oracle's Gram-matrix algebra against dense definitions and mathematics.

* RSBT structure (Sec. 5.3): for a digitally shifted net in natural or Gray order,
  K[i, k] depends only on i XOR k.  Circulant structure (Sec. 5.2): a shifted lattice
  in linear order has K[l, l'] depending only on (l - l') mod n.
* Eigen-recipe (Sec. 5.4): the columns of H (DSI) or the bit-reversed Fourier vectors
  (SI) are eigenvectors with eigenvalues lambda = sqrt(n) conj(V) k_1; sorted, they
  equal numpy's eigvalsh of the dense Gram; Gray and natural order give the same set.
* Fast solve / log det / MLL / Bayesian cubature = Cholesky-based dense definitions.
* Dense gradient = central finite differences of the dense MLL (an independent check);
  spectral gradient = dense gradient.
"""
import math

import numpy as np
import pytest
import scipy.linalg

from oracle import qk_oracle as o
from paper_2502_14256_gb300 import inputs


def _net_points(m, d, order, seed=7, R=1, r=0):
    net = inputs.make_net(seed, d, R, order)
    Ct = o.lms_scramble(net.C, net.S)[r]
    return o.net_points(Ct, net.D[r], np.arange(1 << m), m, order)


def _lattice_points(m, d, seed=9):
    lat = inputs.make_lattice(seed, d, 1, max(m, 2))
    return o.lattice_points(lat.g, lat.D[0], np.arange(1 << m))


def test_hadamard_apply_matches_matrix_and_scipy():
    for m in range(0, 8):
        v = np.random.default_rng(m).standard_normal((3, 1 << m))
        H = o.hadamard_matrix(m)
        assert np.array_equal(H, scipy.linalg.hadamard(1 << m))
        assert np.allclose(o.hadamard_apply(v), v @ H.T, atol=1e-12)


@pytest.mark.parametrize("order", ["natural", "gray"])
@pytest.mark.parametrize("alpha", [1, 2, 4])
def test_dsi_gram_is_dyadic_convolution(order, alpha):
    m, d = 6, 3
    X = _net_points(m, d, order)
    K = o.gram_dense("dsi", alpha, X, np.array([1.0, 0.7, 0.3]))
    n = 1 << m
    i = np.arange(n)
    for k in range(n):
        assert np.array_equal(K[:, k], K[0, i ^ k])


def test_si_gram_is_circulant_in_linear_order():
    m, d = 6, 3
    X = _lattice_points(m, d)
    n = 1 << m
    K = o.gram_dense("si", 2, X, np.array([1.0, 0.5, 0.25]))
    rev = o.bit_reverse(np.arange(n), m).astype(np.int64)
    Klin = K[np.ix_(rev, rev)]  # linear-order point l is natural-order point R(l)
    l = np.arange(n)
    for s in range(n):
        assert np.allclose(Klin[l, (l + s) % n], Klin[0, s], rtol=0, atol=1e-13)


@pytest.mark.parametrize("order", ["natural", "gray"])
def test_dsi_eigen_recipe(order):
    m, d = 7, 4
    X = _net_points(m, d, order, seed=3)
    c = np.array([1.0, 0.5, 0.3, 0.2])
    eta = 1e-3
    K = o.gram_dense("dsi", 2, X, c, eta=eta)
    k1 = o.first_column("dsi", 2, X, c)
    lam = o.eigenvalues("dsi", k1, eta)
    H = o.hadamard_matrix(m)
    assert np.allclose(K @ H, H * lam[None, :], atol=1e-10 * np.abs(lam).max())
    assert np.allclose(np.sort(lam), np.linalg.eigvalsh(K), rtol=1e-10, atol=1e-12)


def test_gray_and_natural_spectra_agree():
    m, d = 8, 3
    c = np.array([0.9, 0.81, 0.729])
    lam = {}
    for order in ("natural", "gray"):
        X = _net_points(m, d, order, seed=13)
        lam[order] = np.sort(o.eigenvalues("dsi", o.first_column("dsi", 4, X, c), 1e-8))
    assert np.allclose(lam["natural"], lam["gray"], rtol=1e-12, atol=1e-13)


def test_si_eigen_recipe():
    m, d = 7, 3
    X = _lattice_points(m, d, seed=21)
    c = np.array([1.0, 0.5, 0.25])
    K = o.gram_dense("si", 1, X, c)
    k1 = o.first_column("si", 1, X, c)
    lam = o.eigenvalues("si", k1)
    n = 1 << m
    rev = o.bit_reverse(np.arange(n), m).astype(np.int64)
    w = np.arange(n)
    # Fourier vectors in linear order, read in natural order: f_w[i] = exp(2 pi i w R(i) / n)
    F = np.exp(2j * np.pi * np.outer(rev, w) / n)
    assert np.allclose(K @ F, F * lam[None, :], atol=1e-10 * np.abs(lam).max())
    assert np.allclose(np.sort(lam), np.linalg.eigvalsh(K), rtol=1e-10, atol=1e-10)


def test_nugget_shifts_every_eigenvalue():
    X = _net_points(6, 3, "gray")
    c = np.array([1.0, 0.5, 0.2])
    K0 = o.gram_dense("dsi", 1, X, c)
    K1 = o.gram_dense("dsi", 1, X, c, eta=0.125)
    assert np.allclose(np.linalg.eigvalsh(K1) - np.linalg.eigvalsh(K0), 0.125, atol=1e-12)


def test_first_column_does_not_depend_on_the_shift():
    net = inputs.make_net(55, 4, 3, "gray")
    Ct = o.lms_scramble(net.C, net.S)[0]
    c = np.ones(4)
    cols = [o.first_column("dsi", 2, o.net_points(Ct, net.D[r], np.arange(256), 8), c) for r in range(3)]
    assert np.array_equal(cols[0], cols[1]) and np.array_equal(cols[0], cols[2])
    lat = inputs.make_lattice(56, 4, 3, 8)
    cols = [o.first_column("si", 2, o.lattice_points(lat.g, lat.D[r], np.arange(256)), c) for r in range(3)]
    assert np.array_equal(cols[0], cols[1])


@pytest.mark.parametrize("family,alpha,order", [("dsi", 1, "gray"), ("dsi", 2, "natural"),
                                               ("dsi", 4, "gray"), ("si", 1, None), ("si", 2, None)])
def test_spectral_solve_logdet_mll_match_cholesky(family, alpha, order):
    m, d = 8, 4
    X = _net_points(m, d, order, seed=77) if family == "dsi" else _lattice_points(m, d, seed=78)
    gamma = 1.0 / np.arange(1, d + 1) ** 2
    eta = 1e-6
    y = inputs.rhs_product(X)
    K = o.gram_dense(family, alpha, X, gamma, eta=eta)
    c_ref, logdet_ref = o.cholesky_solve(K, y)
    mll_ref, quad_ref, _, _ = o.mll_dense(K, y)
    mean_ref, var_ref = o.bc_posterior_dense(K, y)
    lam = o.eigenvalues(family, o.first_column(family, alpha, X, gamma), eta)
    c = o.spectral_solve(family, lam, y)
    assert np.max(np.abs(c - c_ref)) < 1e-9 * np.max(np.abs(c_ref))
    assert np.allclose(o.spectral_matvec(family, lam, c), y, atol=1e-10 * np.abs(y).max())
    sp = o.spectral_mll(family, lam, y)
    assert abs(sp["logdet"] - logdet_ref) < 1e-9 * abs(logdet_ref)
    assert abs(sp["quad"] - quad_ref) < 1e-9 * abs(quad_ref)
    assert abs(sp["mll"] - mll_ref) < 1e-9 * abs(mll_ref)
    assert abs(sp["post_mean"] - mean_ref) < 1e-10 * max(1.0, abs(mean_ref))
    # posterior variance is a small difference: absolute check on the O(1) scale
    assert abs(sp["post_var"] - var_ref) < 1e-9


def _mll_at(family, alpha, X, y, gamma, log_ls, eta):
    K = o.gram_dense(family, alpha, X, o.effective_weights(gamma, log_ls), eta=eta)
    return o.mll_dense(K, y)[0]


def _post_mean_at(family, alpha, X, y, gamma, log_ls, eta):
    K = o.gram_dense(family, alpha, X, o.effective_weights(gamma, log_ls), eta=eta)
    return o.bc_posterior_dense(K, y)[0]


@pytest.mark.parametrize("family,alpha", [("dsi", 2), ("si", 2), ("dsi", 1)])
def test_dense_gradient_matches_finite_differences(family, alpha):
    m, d = 6, 3
    X = _net_points(m, d, "gray", seed=5) if family == "dsi" else _lattice_points(m, d, seed=6)
    y = inputs.rhs_product(X)
    gamma = np.array([0.8, 0.4, 0.2])
    log_ls = np.array([0.1, -0.2, 0.3])
    eta = 1e-3
    g = o.mll_grad_dense(family, alpha, X, y, gamma, log_ls, eta)
    h = 1e-5
    for j in range(d):
        e = np.zeros(d)
        e[j] = h
        fd = (_mll_at(family, alpha, X, y, gamma, log_ls + e, eta)
              - _mll_at(family, alpha, X, y, gamma, log_ls - e, eta)) / (2 * h)
        assert abs(fd - g["dtheta"][j]) < 1e-6 * max(1.0, abs(fd)), (j, fd, g["dtheta"][j])
        fdm = (_post_mean_at(family, alpha, X, y, gamma, log_ls + e, eta)
               - _post_mean_at(family, alpha, X, y, gamma, log_ls - e, eta)) / (2 * h)
        cw = o.effective_weights(gamma, log_ls)
        assert abs(fdm - cw[j] * g["dmean_dc"][j]) < 1e-7 * max(1.0, abs(fdm))
    le = math.log(eta)
    fd = (_mll_at(family, alpha, X, y, gamma, log_ls, math.exp(le + h))
          - _mll_at(family, alpha, X, y, gamma, log_ls, math.exp(le - h))) / (2 * h)
    assert abs(fd - g["dlog_eta"]) < 1e-6 * max(1.0, abs(fd))


@pytest.mark.parametrize("family,alpha,order", [("dsi", 2, "gray"), ("dsi", 4, "natural"),
                                               ("si", 1, None), ("si", 2, None)])
def test_spectral_gradient_matches_dense(family, alpha, order):
    m, d = 7, 3
    X = _net_points(m, d, order, seed=15) if family == "dsi" else _lattice_points(m, d, seed=16)
    y = inputs.rhs_product(X)
    gamma = np.array([1.0, 0.5, 0.25])
    log_ls = np.array([0.2, 0.0, -0.1])
    eta = 1e-4
    cw = o.effective_weights(gamma, log_ls)
    dense = o.mll_grad_dense(family, alpha, X, y, gamma, log_ls, eta)
    lam = o.eigenvalues(family, o.first_column(family, alpha, X, cw), eta)
    sp = o.spectral_mll_grad(family, alpha, X, y, lam, cw)
    assert np.allclose(sp["dc"], dense["dc"], rtol=1e-9, atol=1e-9 * np.abs(dense["dc"]).max())
    assert abs(sp["deta"] - dense["deta"]) < 1e-9 * max(1.0, abs(dense["deta"]))
    assert np.allclose(sp["dmean_dc"], dense["dmean_dc"], rtol=1e-9, atol=1e-12)
    assert abs(sp["dmean_deta"] - dense["dmean_deta"]) < 1e-9 * max(1.0, abs(dense["dmean_deta"]))


def test_gradient_with_exact_zero_factors_matches_dense_and_finite_differences():
    """DSI order 1 with c_1 = 2: 1 + c_1 K_1 = 0 exactly wherever the first coordinate of
    x_i (-) x_k is >= 1/2, so half of k_1 (and of every Gram row) vanishes.  The spectral
    gradient (explicit products, no division by the factor) must still equal the dense
    definition and central differences of the dense MLL in c_1 (K is polynomial in c)."""
    m, d, eta = 6, 3, 1e-3
    X = _net_points(m, d, "gray", seed=21)
    y = inputs.rhs_product(X)
    c = np.array([2.0, 0.6, 0.4])
    k1 = o.first_column("dsi", 1, X, c)
    assert np.count_nonzero(k1 == 0.0) == (1 << m) // 2
    lam = o.eigenvalues("dsi", k1, eta)
    sp = o.spectral_mll_grad("dsi", 1, X, y, lam, c)
    dense = o.mll_grad_dense("dsi", 1, X, y, c, np.zeros(d), eta)
    assert np.allclose(sp["dc"], dense["dc"], rtol=1e-9, atol=1e-9 * np.abs(dense["dc"]).max())
    assert np.allclose(sp["dmean_dc"], dense["dmean_dc"], rtol=1e-9, atol=1e-12)
    h = 1e-5
    mll = lambda cc: o.mll_dense(o.gram_dense("dsi", 1, X, cc, 1.0, eta), y)[0]  # noqa: E731
    fd = (mll(c + [h, 0, 0]) - mll(c - [h, 0, 0])) / (2 * h)
    assert abs(fd - dense["dc"][0]) < 1e-5 * max(1.0, abs(fd))


@pytest.mark.parametrize("family", ["dsi", "si"])
def test_scale_zeta_enters_posterior_as_in_the_dense_definition(family):
    m, d, zeta, eta = 7, 3, 2.5, 1e-5
    X = _net_points(m, d, "gray", seed=19) if family == "dsi" else _lattice_points(m, d, seed=20)
    y = inputs.rhs_product(X)
    c = np.array([0.6, 0.3, 0.1])
    K = o.gram_dense(family, 2, X, c, zeta=zeta, eta=eta)
    mean_ref, var_ref = o.bc_posterior_dense(K, y, zeta)
    lam = o.eigenvalues(family, o.first_column(family, 2, X, c, zeta=zeta), eta)
    sp = o.spectral_mll(family, lam, y, zeta)
    assert abs(sp["post_mean"] - mean_ref) < 1e-10 * max(1.0, abs(mean_ref))
    assert abs(sp["post_var"] - var_ref) < 1e-9
    assert abs(var_ref) > 1e-6


@pytest.mark.parametrize("family", ["dsi", "si"])
def test_doubling_update_of_transformed_data(family):
    """Sec. 5.4 update: the transform of [y; y_new] from the transforms of its halves."""
    rng = np.random.default_rng(5)
    m = 6
    n = 1 << m
    y = rng.standard_normal((3, 2 * n))
    full = o.forward_transform(family, y)
    ext = o.extend_transformed(family, o.forward_transform(family, y[:, :n]), o.forward_transform(family, y[:, n:]))
    assert np.allclose(ext, full, rtol=0, atol=1e-13)
    # the weights belong to the new half: putting them on the old half is wrong
    w = o.update_weights(family, m)
    if family == "si":
        a, b = o.forward_transform(family, y[:, :n]), o.forward_transform(family, y[:, n:])
        wrong = np.concatenate([w * a + b, w * a - b], axis=-1) / math.sqrt(2)
        assert not np.allclose(wrong, full, atol=1e-6)


@pytest.mark.parametrize("family,order", [("dsi", "natural"), ("dsi", "gray"), ("si", "natural")])
def test_doubling_update_of_eigenvalues(family, order):
    """Eigenvalues of the 2n-point Gram matrix from those of the first n points and the
    column entries of the n new points, against the dense 2n-point matrix."""
    m, d = 6, 3
    n = 1 << m
    c = np.array([1.0, 0.5, 0.25])
    alpha, eta = (2, 1e-3) if family == "dsi" else (1, 1e-3)
    if family == "dsi":
        X2, X1 = _net_points(m + 1, d, order, seed=31), _net_points(m, d, order, seed=31)
    else:
        lat = inputs.make_lattice(33, d, 1, 12)
        X2 = o.lattice_points(lat.g, lat.D[0], np.arange(2 * n))
        X1 = o.lattice_points(lat.g, lat.D[0], np.arange(n))
    assert np.array_equal(X2[:n], X1)  # the first n points of the doubled set are the n-point set
    k2 = o.first_column(family, alpha, X2, c)
    lam1 = o.eigenvalues(family, o.first_column(family, alpha, X1, c), eta)
    ext = o.extend_eigenvalues(family, lam1, k2[n:])
    assert np.allclose(ext, o.eigenvalues(family, k2, eta), rtol=0, atol=1e-12 * np.abs(ext).max())
    K2 = o.gram_dense(family, alpha, X2, c, eta=eta)
    assert np.allclose(np.sort(ext), np.linalg.eigvalsh(K2), rtol=1e-10, atol=1e-10)
