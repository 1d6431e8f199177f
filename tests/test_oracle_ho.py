"""Pins of the oracle's higher-order nets (Sec. 4.3, digital interlacing with higher-order LMS)
and of the DSI kernels on their 64-digit words (Sec. 5.3), without a GPU: the paper's worked
interlacing example, de-interlacing back to the underlying net (already pinned bit for bit),
the closed forms against the exact Walsh series with 64 digits, and the RSBT structure of
the Gram matrix that the fast transforms need."""
import os

import numpy as np
import pytest

from oracle import qk_oracle as o
from paper_2502_14256_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "interlace_example.txt")


def test_interlacing_reproduces_the_printed_example():
    """Sec. 4.3 prints the interlacing of four 2 x 2 matrices into two 4 x 2 ones; every
    assignment of bits to the sixteen entries a_{jtk} must land where the example puts it."""
    rows = [tuple(int(v) for v in line.split()) for line in open(GOLDEN) if line.strip() and not line.startswith("#")]
    rng = np.random.default_rng(4)
    for _ in range(32):
        a = rng.integers(0, 2, size=(4, 2, 2))  # a[j, t, k]: matrix j, digit t, column k
        A = np.zeros((4, 32), dtype=np.uint64)
        for j in range(4):
            for t in range(2):
                for k in range(2):
                    A[j, k] |= np.uint64(int(a[j, t, k])) << np.uint64(31 - t)
        H = o.interlace(A, 2, t_out=64)
        for jh, th, js, ts in rows:
            for k in range(2):
                got = int(H[jh - 1, k] >> np.uint64(63 - th)) & 1
                assert got == a[js - 1, ts, k], (jh, th, js, ts, k)
        # digits past alpha t_max of the example stay zero
        for jh in range(2):
            for k in range(2):
                assert int(H[jh, k]) & ((1 << 60) - 1) == 0


@pytest.mark.parametrize("alpha,order", [(2, "gray"), (3, "natural"), (4, "gray")])
def test_deinterlaced_points_are_the_underlying_scrambled_net(alpha, order):
    """Interlacing is digit-wise, so the interlaced net's points, de-interlaced, are the points
    of the alpha d-dimensional net with the same LMS (Sec. 4.3, higher-order LMS) and the
    de-interlaced shift, over the digits kept (64 of 32 alpha)."""
    d, R, m = 3, 2, 10
    net = inputs.make_ho_net(31 + alpha, d, alpha, R, order)
    idx = np.arange(1 << m)
    for r in range(R):
        Ct = o.lms_scramble(net.C, net.S[r:r + 1])[0]              # (alpha d, 32)
        Chat = o.interlace(Ct, alpha)
        X = o.ho_net_points(Chat, net.D[r], idx, m, order)
        D32 = o.deinterlace_point(net.D[r][None, :], alpha)[0]
        want = o.net_points(Ct, D32, idx, m, order)
        keep = min(64, 32 * alpha)
        mask = np.array([sum(1 << (31 - t // alpha) for t in range(keep) if t % alpha == u) for u in range(alpha)],
                        dtype=np.uint64)
        got = o.deinterlace_point(X, alpha)
        assert np.array_equal(got.astype(np.uint64), want.astype(np.uint64) & np.tile(mask, d)[None, :])


def test_interlacing_of_order_one_is_the_identity_on_the_words():
    net = inputs.make_net(5, 4, 1, "gray")
    H = o.interlace(net.C, 1)
    assert np.array_equal(H >> np.uint64(32), net.C.astype(np.uint64))


@pytest.mark.parametrize("alpha", [1, 2, 3, 4])
def test_64_digit_closed_forms_match_the_walsh_series(alpha):
    rng = inputs.SplitMix64(64 + alpha)
    words = [0, 1, 2, 3, 1 << 40, (1 << 64) - 1, 1 << 63]
    words += [int(h) << 32 | int(l) for h, l in zip(rng.u32(12), rng.u32(12))]
    words += [int(v) for v in rng.u32(6)]  # beta > 32: digits only in the low half
    base, scale = (4.0, 2.0) if alpha == 1 else (2.0, 1.0)
    for z in words:
        series = o.dsi_kernel_walsh_series(alpha, z, a_max=200, base=base, scale=scale, digits=64)
        closed = float(o.dsi_kernel_words(alpha, np.array([z], dtype=np.uint64), 64)[0])
        assert abs(series - closed) < 1e-13, (alpha, z, series, closed)


@pytest.mark.parametrize("alpha", [1, 2, 3, 4])
def test_64_digit_kernel_extends_the_32_digit_one(alpha):
    """A 64-digit word whose low half is zero is the 32-digit word of the same number."""
    Z = inputs.SplitMix64(7 * alpha).u32(64)
    Z64 = Z.astype(np.uint64) << np.uint64(32)
    assert np.allclose(o.dsi_kernel_words(alpha, Z64, 64), o.dsi_kernel(alpha, Z), rtol=0, atol=1e-15)


@pytest.mark.parametrize("alpha_net,alpha_k", [(2, 2), (2, 4), (3, 4)])
def test_higher_order_gram_is_rsbt_and_diagonalised_by_the_hadamard_transform(alpha_net, alpha_k):
    d, m = 2, 6
    n = 1 << m
    net = inputs.make_ho_net(90 + alpha_k, d, alpha_net, 1, "natural")
    Chat = o.interlace(o.lms_scramble(net.C, net.S)[0], alpha_net)
    X = o.ho_net_points(Chat, net.D[0], np.arange(n), m, "natural")
    c = np.array([0.8, 0.5])
    K = o.ho_gram_dense(alpha_k, X, c, 1.0)
    i = np.arange(n)
    assert np.allclose(K, K[0][i[:, None] ^ i[None, :]], rtol=0, atol=1e-14)  # K[i,k] = k_1[i xor k]
    lam = o.hadamard_apply(o.ho_first_column(alpha_k, X, c, 1.0))
    assert np.allclose(np.sort(lam), np.linalg.eigvalsh(K), rtol=1e-12, atol=1e-12 * lam.max())
    assert lam.min() > 0


def test_higher_order_dense_gradient_matches_central_differences():
    """The dense MLL gradient on an interlaced net against central differences (h = 1e-6) of
    the dense MLL in each weight and in the nugget."""
    d, m, alpha_k, eta = 2, 5, 4, 1e-3
    n = 1 << m
    net = inputs.make_ho_net(77, d, 2, 1, "gray")
    X = o.ho_net_points(o.interlace(o.lms_scramble(net.C, net.S)[0], 2), net.D[0], np.arange(n), m, "gray")
    x = X.astype(np.float64) / 2.0 ** 64
    y = np.prod(1.0 + (x - 0.5) / np.arange(1, d + 1) ** 2, axis=1)
    c = np.array([0.9, 0.4])
    g = o.ho_mll_grad_dense(alpha_k, X, y, c, eta, 1.0)
    h = 1e-6
    for j in range(d):
        cp, cm = c.copy(), c.copy()
        cp[j] += h
        cm[j] -= h
        fd = (o.mll_dense(o.ho_gram_dense(alpha_k, X, cp, 1.0, eta), y)[0]
              - o.mll_dense(o.ho_gram_dense(alpha_k, X, cm, 1.0, eta), y)[0]) / (2 * h)
        assert abs(fd - g["dc"][j]) < 1e-6 * max(1.0, abs(fd)), (j, fd, g["dc"][j])
    fd = (o.mll_dense(o.ho_gram_dense(alpha_k, X, c, 1.0, eta + h), y)[0]
          - o.mll_dense(o.ho_gram_dense(alpha_k, X, c, 1.0, eta - h), y)[0]) / (2 * h)
    assert abs(fd - g["deta"]) < 1e-5 * max(1.0, abs(fd))
