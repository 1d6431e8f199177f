"""Pins of the oracle's one-dimensional kernels against facts the paper and mathematics fix.

* DSI closed forms (Sec. 5.3 Theorem, with the readings listed in the oracle header)
  against an exact evaluation of the Walsh series of Eq. (DSI kernel).
* That exact evaluation against the pieces printed in Appendix B (s_1, s_2, s_3 and
  tilde s_4(0) = 1/294), read from tests/golden/dsi_proof_pieces.txt.
* The Walsh-function digit convention against the Lemma of Appendix B (Walsh
  coefficients of x, x^2, x^3), integrated exactly with rationals.
* SI kernels (Sec. 5.2) against their Fourier series evaluated with Hurwitz zeta.
"""
from fractions import Fraction
import math
import os

import numpy as np
import pytest
import scipy.special

from oracle import qk_oracle as o

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _words(seed=0, count=300):
    rng = np.random.default_rng(seed)
    rand = rng.integers(0, 2 ** 32, count, dtype=np.uint64).astype(np.uint32)
    dyadic = (np.arange(256, dtype=np.uint32) << np.uint32(24))
    edges = np.array([0, 1, 2, 3, 0x7FFFFFFF, 0x80000000, 0x80000001, 0xFFFFFFFF,
                      0x40000000, 0x3FFFFFFF, 0x00010000, 0x0000FFFF], dtype=np.uint32)
    return np.concatenate([rand, dyadic, edges])


@pytest.mark.parametrize("alpha", [1, 2, 3, 4])
def test_dsi_closed_form_matches_walsh_series(alpha):
    Z = _words(alpha)
    closed = o.dsi_kernel(alpha, Z)
    base, scale = (4.0, 2.0) if alpha == 1 else (2.0, 1.0)
    series = np.array([o.dsi_kernel_walsh_series(alpha, int(z), base=base, scale=scale) for z in Z])
    assert np.max(np.abs(closed - series)) < 4e-15


def test_dsi_special_values_at_zero():
    z0 = np.array([0], dtype=np.uint32)
    assert o.dsi_kernel(1, z0)[0] == 1.0
    assert abs(o.dsi_kernel(2, z0)[0] - 1.5) < 1e-15
    assert abs(o.dsi_kernel(3, z0)[0] - 25.0 / 18.0) < 1e-15
    assert abs(o.dsi_kernel(4, z0)[0] - 407.0 / 294.0) < 1e-15


def _golden_tilde_s4():
    with open(os.path.join(GOLDEN, "dsi_proof_pieces.txt")) as f:
        for line in f:
            if line.startswith("tilde_s4_at_0"):
                return float(Fraction(line.split()[1]))
    raise AssertionError("missing fixture")


def test_walsh_series_parts_match_printed_proof_pieces():
    """s_1, s_2, s_3 (Appendix B) from the exact series; tilde s_4(0) = 1/294."""
    for z in _words(7, 60):
        x = float(z) / 2 ** 32
        s1, s2, s3, ts4 = o.dsi_kernel_walsh_series(4, int(z), parts=True)
        S = float(o.walsh_power_series(np.array([z], dtype=np.uint32))[0])
        assert abs(s1 - (1 - 2 * x)) < 1e-15
        assert abs(s2 - (2 * x * x - 2 * x + 1.0 / 3.0)) < 1e-15
        assert abs(s3 - (-4.0 / 3.0 * x ** 3 + 2 * x * x - 2.0 / 3.0 * x + S / 24.0)) < 2e-15
    parts = o.dsi_kernel_walsh_series(4, 0, parts=True)
    assert abs(parts[-1] - _golden_tilde_s4()) < 1e-16


def _exact_walsh_coefficient(p, k):
    """int_0^1 x^p wal_k(x) dx, exactly: wal_k is constant on intervals of length 2^-(a_1+1)."""
    A = max(k.bit_length(), 1)
    lefts = (np.arange(1 << A, dtype=np.uint64) << np.uint64(32 - A)).astype(np.uint32)
    signs = o.walsh_function(k, lefts)
    total = Fraction(0)
    den = (p + 1) * (1 << (A * (p + 1)))
    for i in range(1 << A):
        total += int(signs[i]) * Fraction((i + 1) ** (p + 1) - i ** (p + 1), den)
    return total


def _lemma_value(p, k):
    if k == 0:
        return Fraction(1, p + 1)
    a = [t for t in range(k.bit_length() - 1, -1, -1) if (k >> t) & 1]
    F = lambda e: Fraction(2) ** e  # noqa: E731
    if p == 1:
        return -F(-a[0] - 2) if len(a) == 1 else Fraction(0)
    if p == 2:
        if len(a) == 1:
            return -F(-a[0] - 2)
        return F(-a[0] - a[1] - 3) if len(a) == 2 else Fraction(0)
    if len(a) == 1:
        return -F(-a[0] - 2) + F(-3 * a[0] - 5)
    if len(a) == 2:
        return 3 * F(-a[0] - a[1] - 4)
    if len(a) == 3:
        return -3 * F(-a[0] - a[1] - a[2] - 5)
    return Fraction(0)


def test_walsh_convention_reproduces_monomial_coefficients():
    """Lemma (Appendix B) fixes which digit wal_{2^a} reads: x_{a+1}, bit 31-a."""
    with open(os.path.join(GOLDEN, "walsh_monomials.txt")) as f:
        cases = [ln.split()[:2] for ln in f if ln[0].isdigit()]
    assert len(cases) == 12
    for p in (1, 2, 3):
        for k in range(0, 40):
            assert _exact_walsh_coefficient(p, k) == _lemma_value(p, k), (p, k)


def _si_fourier(alpha, p, q):
    """2 sum_{h>=1} cos(2 pi h p/q) / h^(2 alpha) by residues mod q and Hurwitz zeta."""
    s = 2 * alpha
    total = 0.0
    for r in range(1, q + 1):
        total += math.cos(2 * math.pi * r * p / q) * scipy.special.zeta(s, r / q)
    return 2.0 * total / q ** s


@pytest.mark.parametrize("alpha", [1, 2, 3])
def test_si_kernel_matches_fourier_series(alpha):
    for q in (1, 2, 3, 7, 16, 64):
        for p in range(q):
            got = float(o.si_kernel(alpha, p / q))
            want = _si_fourier(alpha, p, q)
            assert abs(got - want) < 1e-12 * max(1.0, abs(want)), (alpha, p, q)


def test_si_special_values():
    assert abs(float(o.si_kernel(1, 0.0)) - math.pi ** 2 / 3) < 1e-14
    assert abs(float(o.si_kernel(2, 0.0)) - math.pi ** 4 / 45) < 1e-13
    # periodic and symmetric: K(x) = K(1 - x) = K(x + 1)
    x = np.linspace(0, 1, 33)
    for a in (1, 2):
        assert np.allclose(o.si_kernel(a, x), o.si_kernel(a, 1 - x), atol=1e-13)
        assert np.allclose(o.si_kernel(a, x), o.si_kernel(a, x + 1), atol=1e-13)


@pytest.mark.parametrize("alpha", [1, 2, 3, 4])
def test_dsi_kernel_has_mean_zero(alpha):
    """Every Walsh term with k >= 1 integrates to 0; on a 2^T grid the sum over k < 2^T
    vanishes, so the grid mean is the tail over multiples of 2^T (tiny)."""
    T = 16
    Z = (np.arange(1 << T, dtype=np.uint32) << np.uint32(32 - T))
    assert abs(float(np.mean(o.dsi_kernel(alpha, Z)))) < 64 * 2.0 ** -T


@pytest.mark.parametrize("alpha", [1, 2])
def test_si_kernel_has_mean_zero(alpha):
    x = (np.arange(4096) + 0.5) / 4096
    assert abs(float(np.mean(o.si_kernel(alpha, x)))) < 1e-6


def test_dsi_kernel_is_positive_definite_on_a_net():
    """A product-weight DSI Gram over a small net must be SPD (smallest eigenvalue > 0)."""
    from paper_2502_14256_gb300 import inputs
    net = inputs.make_net(11, 3, 1)
    Ct = o.lms_scramble(net.C, net.S)[0]
    X = o.net_points(Ct, net.D[0], np.arange(256), 8, "natural")
    for alpha in (1, 2, 3, 4):
        K = o.gram_dense("dsi", alpha, X, np.array([1.0, 0.5, 0.25]))
        assert np.linalg.eigvalsh(K).min() > 0
