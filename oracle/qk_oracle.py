"""Plain FP64 CPU oracle for the structured-Gram kernel solve over randomized LD points.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or
execute this module: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code with the CUDA library (no kernels, headers, tables or helpers); it
takes every input as an explicit array, so the only thing the two sides have
in common is the seeded input generator.

Each function follows the paper (arXiv 2502.14256) as cited in its docstring:
definitions are written out (bit loops, dense n x n Gram matrices, Cholesky);
the O(n log n) spectral formulas of Sec. 5.4 are written in the paper's order
and are pinned against the dense definitions by the tests.

Readings of the paper used here (silent, garbled or ambiguous passages):

* Theorem in Sec. 5.3: ``-1+-beta(x)x`` is read as ``-1-beta(x)x`` (same for
  the x^3 term of K_4).
* ``wal_{2^a}(x) = (-1)^{x_{a+1}}`` with x_{a+1} the (a+1)-th binary digit of x
  (coefficient of 2^-(a+1)), i.e. bit (31-a) of the 32-bit word.
* beta(0) = t_nu(0) = 0 exactly as the theorem states; points carry
  t_max = 32 digits, digits past 32 are zero, so the K_4 series
  sum_a wal_{2^a}(x) 8^-a equals 8/7 - 2 sum_{a<32, x_{a+1}=1} 8^-a.
* Order-1 DSI kernel (the paper defers it to Dick & Pillichshammer):
  K_1(x) = 2 sum_{k>=1} wal_k(x) 4^{-mu_1(k)} = 1 - 3 * 2^{-beta(x)}, K_1(0) = 1.
* LMS matrices (Sec. 4.3): lower triangular, unit diagonal, uniform bits below.
* Nugget: K + eta I.  Lattice shift drawn on the 2^-32 grid.
* Effective product weight c_j = gamma_j * exp(theta_j) (theta = log-lengthscale).
* Zero-mean GP marginal log-likelihood and Bayesian cubature with
  kappa_i = int K(u, x_i) du = zeta (every one-dimensional K_alpha has mean 0).
"""
from __future__ import annotations

from fractions import Fraction
import math

import numpy as np
import scipy.linalg

TWO32 = 2.0 ** 32

# ----------------------------------------------------------------- digits (Sec. 4.1)


def bit_reverse(i, m: int):
    """R_m(i): flip the first m binary digits of i (Sec. 5.2), digit by digit."""
    i = np.asarray(i, dtype=np.uint64)
    out = np.zeros_like(i)
    for t in range(m):
        out |= ((i >> np.uint64(t)) & np.uint64(1)) << np.uint64(m - 1 - t)
    return out


def gray_code(i):
    """Index whose digits are the b=2 Gray code of i (Table "Gray code order", Sec. 4.3).

    Consecutive codes differ in exactly one digit; for base 2 this is i XOR (i >> 1).
    """
    i = np.asarray(i, dtype=np.uint64)
    return i ^ (i >> np.uint64(1))


# ------------------------------------------------------- bit matrices (Sec. 4.3)


def columns_to_matrix(cols) -> np.ndarray:
    """32x32 0/1 matrix M[t, k] = digit t of column k (digit t is bit 31 - t)."""
    cols = np.asarray(cols, dtype=np.uint64)
    M = np.zeros((32, cols.shape[-1]), dtype=np.int64)
    for t in range(32):
        M[t] = ((cols >> np.uint64(31 - t)) & np.uint64(1)).astype(np.int64)
    return M


def matrix_to_columns(M) -> np.ndarray:
    M = np.asarray(M, dtype=np.int64) % 2
    cols = np.zeros(M.shape[1], dtype=np.uint64)
    for t in range(32):
        cols |= M[t].astype(np.uint64) << np.uint64(31 - t)
    return cols.astype(np.uint32)


def rows_to_matrix(rows) -> np.ndarray:
    """32x32 0/1 matrix S[t, u] = bit (31 - u) of row mask t."""
    rows = np.asarray(rows, dtype=np.uint64)
    S = np.zeros((32, 32), dtype=np.int64)
    for u in range(32):
        S[:, u] = ((rows >> np.uint64(31 - u)) & np.uint64(1)).astype(np.int64)
    return S


def lms_scramble(C, S) -> np.ndarray:
    """Linear matrix scrambling C~_j = S_j C_j mod 2 (Sec. 4.3, "Linear matrix scrambling").

    C: (d, 32) generator columns; S: (R, d, 32) row masks.  Returns (R, d, 32).
    The product is an explicit integer matrix product reduced mod 2.
    """
    C = np.asarray(C, dtype=np.uint32)
    S = np.asarray(S, dtype=np.uint32)
    R, d = S.shape[0], S.shape[1]
    out = np.empty((R, d, 32), dtype=np.uint32)
    for j in range(d):
        Cm = columns_to_matrix(C[j])
        for r in range(R):
            out[r, j] = matrix_to_columns(rows_to_matrix(S[r, j]) @ Cm)
    return out


# ------------------------------------------------------------- points (Sec. 4.2-4.3)


def net_points(Ct, D, idx, m: int, order: str = "gray") -> np.ndarray:
    """Digitally shifted digital net points as 32-bit words (Sec. 4.3).

    z_ij = F_32(C~_j D_m(k) mod 2) with k = i (natural order) or the Gray code of i,
    x_ij = z_ij (+) Delta_j digit-wise mod 2 (XOR).  Ct: (d, 32); D: (d,);
    idx: positions in the sequence.  Returns (len(idx), d) uint32.
    """
    idx = np.asarray(idx, dtype=np.uint64)
    k = gray_code(idx) if order == "gray" else idx
    Ct = np.asarray(Ct, dtype=np.uint32)
    d = Ct.shape[0]
    X = np.zeros((idx.size, d), dtype=np.uint32)
    for t in range(m):
        digit = ((k >> np.uint64(t)) & np.uint64(1)).astype(bool)
        for j in range(d):
            X[digit, j] ^= Ct[j, t]
    X ^= np.asarray(D, dtype=np.uint32)[None, :]
    return X


def radical_inverse_word(idx) -> np.ndarray:
    """v(i) * 2^32 for i < 2^32 (Eq. for v(i), Sec. 4.1): sum_t i_{t-1} 2^(32-t)."""
    idx = np.asarray(idx, dtype=np.uint64)
    v = np.zeros_like(idx)
    for t in range(1, 33):
        v |= ((idx >> np.uint64(t - 1)) & np.uint64(1)) << np.uint64(32 - t)
    return v


def lattice_points(g, D, idx) -> np.ndarray:
    """Shifted rank-1 lattice in natural order as 32-bit words (Sec. 4.2).

    z_i = v(i) g mod 1, x_i = (z_i + Delta) mod 1 with Delta = D 2^-32.  In words:
    X = (v(i) 2^32 * g + D) mod 2^32, exact integer arithmetic.
    """
    v = radical_inverse_word(idx)
    g = np.asarray(g, dtype=np.uint64)
    D = np.asarray(D, dtype=np.uint64)
    with np.errstate(over="ignore"):
        Z = (v[:, None] * g[None, :]) & np.uint64(0xFFFFFFFF)
    return ((Z + D[None, :]) & np.uint64(0xFFFFFFFF)).astype(np.uint32)


# ------------------------------------------------------- DSI kernels (Sec. 5.3)


def beta_t(Z):
    """beta(x) = -floor(log2 x) and x = Z 2^-32 for 32-bit words Z; beta(0) = 0."""
    Z = np.asarray(Z, dtype=np.uint32)
    x = Z.astype(np.float64) / TWO32
    _, e = np.frexp(x)  # x = f 2^e with f in [1/2, 1) => floor(log2 x) = e - 1
    beta = np.where(Z != 0, 1 - e, 0).astype(np.int64)
    return beta, x


def dsi_kernel(alpha: int, Z) -> np.ndarray:
    """One-dimensional DSI kernel K_alpha(x) at x = Z 2^-32 (Theorem, Sec. 5.3).

    alpha 2, 3, 4 are the theorem's closed forms; alpha 1 is the first-order
    Walsh kernel 1 - 3 * 2^-beta (K_1(0) = 1).  t_nu(x) = 2^(-nu beta(x)), with
    t_nu(0) = 0 as the theorem sets it.
    """
    Z = np.asarray(Z, dtype=np.uint32)
    beta, x = beta_t(Z)
    nz = Z != 0
    b = beta.astype(np.float64)
    t1 = np.where(nz, np.ldexp(1.0, -beta), 0.0)
    t2 = np.where(nz, np.ldexp(1.0, -2 * beta), 0.0)
    t3 = np.where(nz, np.ldexp(1.0, -3 * beta), 0.0)
    if alpha == 1:
        return np.where(nz, 1.0 - 3.0 * t1, 1.0)
    if alpha == 2:
        return -1.0 - b * x + 2.5 * (1.0 - t1)
    if alpha == 3:
        return -1.0 + b * x ** 2 - 5.0 * (1.0 - t1) * x + (43.0 / 18.0) * (1.0 - t2)
    if alpha == 4:
        S = walsh_power_series(Z)
        return (-1.0 - (2.0 / 3.0) * b * x ** 3 + 5.0 * (1.0 - t1) * x ** 2
                - (43.0 / 9.0) * (1.0 - t2) * x + (701.0 / 294.0) * (1.0 - t3)
                + b * (S / 48.0 - 1.0 / 42.0))
    raise ValueError(f"DSI order {alpha} not supported")


def walsh_power_series(Z) -> np.ndarray:
    """sum_{a>=0} wal_{2^a}(x) / 2^(3a) for 32-digit x = Z 2^-32 (Theorem, K_4).

    wal_{2^a}(x) = (-1)^{x_{a+1}}; x_{a+1} = bit (31 - a); digits a >= 32 are 0.
    """
    Z = np.asarray(Z, dtype=np.uint64)
    s = np.full(Z.shape, 8.0 / 7.0)  # all digits zero: sum_a 8^-a
    for a in range(32):
        bit = ((Z >> np.uint64(31 - a)) & np.uint64(1)).astype(np.float64)
        s -= 2.0 * bit * 8.0 ** (-a)
    return s


def dsi_kernel_walsh_series(alpha: int, Z: int, a_max: int = 160, base: float = 2.0,
                            scale: float = 1.0, parts: bool = False, digits: int = 32):
    """Exact evaluation of the Walsh series of Eq. (DSI kernel), Sec. 5.3, for one word Z.

    K_alpha(x) = sum_{k>=1} wal_k(x) / base^{mu_alpha(k)} with mu_alpha(k) the sum of
    (a_l + 1) over the alpha leading set bits a_1 > a_2 > ... of k.  Split k by its
    set-bit set A: when |A| <= alpha every bit is weighted; when |A| > alpha the bits
    below a_alpha are free and sum to prod_{b<a_alpha}(1 + s_b) = 2^{a_alpha} if the
    first a_alpha digits of x are zero, else 0.  This gives elementary-symmetric sums
    over v_a = s_a base^-(a+1), s_a = (-1)^{x_{a+1}}, which are accumulated exactly up to
    a_max (every neglected term is below 2^-a_max * poly(a_max)).
    ``base=4, scale=2`` gives the first-order kernel reading.  With ``parts=True`` the
    result is (s_1, ..., s_{alpha-1}, tilde s_alpha): the sums over k with exactly nu
    nonzero digits and with at least alpha (the decomposition of Appendix B).  ``digits``
    is the word length t_max (x = Z 2^-digits; 64 for interlaced higher-order nets).
    """
    Z = int(Z)
    s = [(-1.0 if (a < digits and (Z >> (digits - 1 - a)) & 1) else 1.0) for a in range(a_max)]
    v = [s[a] * base ** (-(a + 1)) for a in range(a_max)]
    # sets with 1 <= |A| <= alpha - 1: elementary symmetric polynomials e_p(v)
    e = [1.0] + [0.0] * alpha
    for a in range(a_max):
        for p in range(alpha, 0, -1):
            e[p] += v[a] * e[p - 1]
    total = sum(e[1:alpha])
    # sets with |A| >= alpha: the smallest weighted bit a_alpha carries w_a = v_a P(a),
    # P(a) = 2^a when digits x_1..x_a vanish, else 0.  Ascending a, a is the new largest.
    F = [0.0] * (alpha + 1)
    for a in range(a_max):
        w = v[a] * 2.0 ** a if all_zero_below(a, Z, digits) else 0.0
        for q in range(alpha, 1, -1):
            F[q] += v[a] * F[q - 1]
        F[1] += w
    total += F[alpha]
    if parts:
        return [scale * x for x in e[1:alpha]] + [scale * F[alpha]]
    return scale * total


def walsh_function(k: int, Z) -> np.ndarray:
    """wal_k(x) = (-1)^{sum_a k_a x_{a+1}} in base 2 (Sec. 5.3), x = Z 2^-32, k < 2^32."""
    Z = np.asarray(Z, dtype=np.uint64)
    parity = np.zeros(Z.shape, dtype=np.uint64)
    for a in range(32):
        if (k >> a) & 1:
            parity ^= (Z >> np.uint64(31 - a)) & np.uint64(1)
    return 1.0 - 2.0 * parity.astype(np.float64)


def all_zero_below(a: int, Z: int, digits: int = 32) -> bool:
    """True when digits x_1..x_a of x = Z 2^-digits are all zero (free low bits sum to 2^a)."""
    if a == 0:
        return True
    if a >= digits:
        return Z == 0
    return (Z >> (digits - a)) == 0


# -------------------------------------------------------- SI kernels (Sec. 5.2)


def bernoulli_numbers(deg: int):
    """Exact Bernoulli numbers B_0..B_deg from sum_{k<=n} binom(n+1, k) B_k = 0 (B_1 = -1/2)."""
    B = [Fraction(1)]
    for n in range(1, deg + 1):
        B.append(-sum(math.comb(n + 1, k) * B[k] for k in range(n)) / (n + 1))
    return B


def bernoulli_poly(deg: int, x) -> np.ndarray:
    """B_deg(x) = sum_k binom(deg, k) B_k x^(deg - k)."""
    B = bernoulli_numbers(deg)
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros_like(x)
    for k in range(deg + 1):
        out += float(math.comb(deg, k) * B[k]) * x ** (deg - k)
    return out


def si_kernel(alpha: int, x) -> np.ndarray:
    """K_alpha(x) = (2 pi)^(2 alpha) / ((-1)^(alpha+1) (2 alpha)!) B_(2 alpha)(x mod 1) (Sec. 5.2)."""
    x = np.mod(np.asarray(x, dtype=np.float64), 1.0)
    coef = (2 * math.pi) ** (2 * alpha) / ((-1) ** (alpha + 1) * math.factorial(2 * alpha))
    return coef * bernoulli_poly(2 * alpha, x)


# ------------------------------------------------ product kernels, Gram matrices


def factor_values(family: str, alpha: int, diff_words) -> np.ndarray:
    """K_alpha at the digital difference (DSI) or difference mod 1 (SI) given as words."""
    diff_words = np.asarray(diff_words, dtype=np.uint32)
    if family == "dsi":
        return dsi_kernel(alpha, diff_words)
    return si_kernel(alpha, diff_words.astype(np.float64) / TWO32)


def pair_difference(family: str, Xa, Xb) -> np.ndarray:
    """x (-) x' digit-wise (XOR, Sec. 5.3) or (x - x') mod 1 (Sec. 5.2) as words."""
    Xa = np.asarray(Xa, dtype=np.uint64)
    Xb = np.asarray(Xb, dtype=np.uint64)
    if family == "dsi":
        return (Xa ^ Xb).astype(np.uint32)
    return ((Xa - Xb) & np.uint64(0xFFFFFFFF)).astype(np.uint32)


def effective_weights(gamma, log_ls) -> np.ndarray:
    return np.asarray(gamma, dtype=np.float64) * np.exp(np.asarray(log_ls, dtype=np.float64))


def kernel_rows(family, alpha, X, rows, c, zeta=1.0) -> np.ndarray:
    """Rows K(x_i, x_k) of the product-weight kernel (Eq. K_SI_prod / DSI analogue).

    K(x, x') = zeta prod_j (1 + c_j K_alpha(x_j, x'_j)) for the listed rows i, all k.
    """
    X = np.asarray(X, dtype=np.uint32)
    rows = np.atleast_1d(rows)
    out = np.full((rows.size, X.shape[0]), float(zeta))
    for j in range(X.shape[1]):
        diff = pair_difference(family, X[rows, j][:, None], X[None, :, j])
        out *= 1.0 + c[j] * factor_values(family, alpha, diff)
    return out


def gram_dense(family, alpha, X, c, zeta=1.0, eta=0.0) -> np.ndarray:
    """Dense n x n Gram matrix K = (K(x_i, x_k)) + eta I."""
    n = X.shape[0]
    K = kernel_rows(family, alpha, X, np.arange(n), c, zeta)
    return K + eta * np.eye(n)


def first_column(family, alpha, X, c, zeta=1.0) -> np.ndarray:
    """k_1 = (K(x_i, x_0))_i, the first column the fast methods need (Sec. 5.4)."""
    return kernel_rows(family, alpha, X, np.array([0]), c, zeta)[0]


def gram_weight_derivative(family, alpha, X, c, j, zeta=1.0) -> np.ndarray:
    """dK/dc_j = zeta K_alpha(x_j, x'_j) prod_{j' != j} (1 + c_j' K_alpha(...)) (dense)."""
    n = X.shape[0]
    out = np.full((n, n), float(zeta))
    for jj in range(X.shape[1]):
        diff = pair_difference(family, X[:, jj][:, None], X[None, :, jj])
        Kv = factor_values(family, alpha, diff)
        out *= Kv if jj == j else (1.0 + c[jj] * Kv)
    return out


# -------------------------------------------------- dense linear algebra (definitions)


def cholesky_solve(K, Y):
    """c = K^-1 Y and log det K by Cholesky K = L L^T (definition of the solve)."""
    L = np.linalg.cholesky(K)
    C = scipy.linalg.cho_solve((L, True), Y)
    logdet = 2.0 * float(np.sum(np.log(np.diag(L))))
    return C, logdet


def mll_dense(K, y):
    """Zero-mean GP marginal log-likelihood: -y^T K^-1 y / 2 - log det K / 2 - n log(2 pi) / 2."""
    c, logdet = cholesky_solve(K, y)
    quad = float(y @ c)
    n = K.shape[0]
    return -0.5 * quad - 0.5 * logdet - 0.5 * n * math.log(2 * math.pi), quad, logdet, c


def mll_grad_dense(family, alpha, X, y, gamma, log_ls, eta, zeta=1.0):
    """Dense gradient dMLL/dtheta = c^T (dK) c / 2 - tr(K^-1 dK) / 2 with c = K^-1 y.

    Returns dict with d/dc_j, d/dtheta_j (= c_j d/dc_j), d/dgamma_j, d/deta and
    d/dlog(eta), plus the Bayesian-cubature posterior mean zeta 1^T K^-1 y and its
    derivatives -(K^-1 kappa)^T dK c.
    """
    c_w = effective_weights(gamma, log_ls)
    K = gram_dense(family, alpha, X, c_w, zeta, eta)
    n, d = X.shape[0], X.shape[1]
    L = np.linalg.cholesky(K)
    cvec = scipy.linalg.cho_solve((L, True), y)
    Kinv = scipy.linalg.cho_solve((L, True), np.eye(n))
    kappa = np.full(n, float(zeta))
    a = Kinv @ kappa
    dc = np.empty(d)
    dmean = np.empty(d)
    for j in range(d):
        dK = gram_weight_derivative(family, alpha, X, c_w, j, zeta)
        dc[j] = 0.5 * cvec @ dK @ cvec - 0.5 * float(np.sum(Kinv * dK.T))
        dmean[j] = -a @ dK @ cvec
    deta = 0.5 * cvec @ cvec - 0.5 * float(np.trace(Kinv))
    return {
        "dc": dc,
        "dtheta": c_w * dc,
        "dgamma": np.exp(np.asarray(log_ls, dtype=np.float64)) * dc,
        "deta": deta,
        "dlog_eta": eta * deta,
        "post_mean": float(kappa @ cvec),
        "dmean_dc": dmean,
        "dmean_deta": float(-a @ cvec),
    }


def bc_posterior_dense(K, y, zeta=1.0):
    """Bayesian cubature: mean kappa^T K^-1 y, variance zeta - kappa^T K^-1 kappa, kappa = zeta 1."""
    n = K.shape[0]
    kappa = np.full(n, float(zeta))
    sol, _ = cholesky_solve(K, np.stack([y, kappa], axis=1))
    return float(kappa @ sol[:, 0]), float(zeta - kappa @ sol[:, 1])


# ---------------------------------------------------- fast transforms (Sec. 5.2-5.4)


def hadamard_matrix(m: int) -> np.ndarray:
    """H_0 = [1], H_{m+1} = [[H_m, H_m], [H_m, -H_m]] (Sec. 5.3)."""
    H = np.ones((1, 1))
    for _ in range(m):
        H = np.block([[H, H], [H, -H]])
    return H


def hadamard_apply(v) -> np.ndarray:
    """H_m v by the block recursion of Sec. 5.3 applied to a vector (last axis).

    With v = [a; b], H_{m+1} v = [H_m a + H_m b; H_m a - H_m b].
    """
    v = np.asarray(v, dtype=np.float64)
    n = v.shape[-1]
    if n == 1:
        return v.copy()
    half = n // 2
    a = hadamard_apply(v[..., :half])
    b = hadamard_apply(v[..., half:])
    return np.concatenate([a + b, a - b], axis=-1)


def to_linear_order(v_nat, m: int) -> np.ndarray:
    """Lattice data in natural order -> linear order: v_lin[l] = v_nat[R_m(l)] (Sec. 5.2)."""
    v_nat = np.asarray(v_nat)
    return v_nat[..., bit_reverse(np.arange(1 << m), m).astype(np.int64)]


def to_natural_order(v_lin, m: int) -> np.ndarray:
    """Inverse of to_linear_order: v_nat[i] = v_lin[R_m(i)]."""
    v_lin = np.asarray(v_lin)
    return v_lin[..., bit_reverse(np.arange(1 << m), m).astype(np.int64)]


def eigenvalues(family, k1, eta=0.0) -> np.ndarray:
    """lambda = sqrt(n) conj(V) k_1 (Sec. 5.4) plus the nugget eta.

    DSI: V = H/sqrt(n), so lambda = H k_1.  SI (natural-order lattice): V = T/sqrt(n),
    so lambda_w = sum_l k1_lin[l] W^{w l}, W = exp(-2 pi i / n) (numpy FFT), real for the
    symmetric kernel column.
    """
    k1 = np.asarray(k1, dtype=np.float64)
    n = k1.shape[-1]
    m = n.bit_length() - 1
    if family == "dsi":
        lam = hadamard_apply(k1)
    else:
        lam = np.fft.fft(to_linear_order(k1, m), axis=-1).real
    return lam + eta


def forward_transform(family, y) -> np.ndarray:
    """y~ = conj(V) y (orthonormal): H y / sqrt(n) or FFT of y in linear order / sqrt(n)."""
    y = np.asarray(y, dtype=np.float64)
    n = y.shape[-1]
    m = n.bit_length() - 1
    if family == "dsi":
        return hadamard_apply(y) / math.sqrt(n)
    return np.fft.fft(to_linear_order(y, m), axis=-1) / math.sqrt(n)


def inverse_transform(family, yt) -> np.ndarray:
    """V y~ back to natural order (real part for the real-valued results)."""
    n = yt.shape[-1]
    m = n.bit_length() - 1
    if family == "dsi":
        return hadamard_apply(np.real(yt)) / math.sqrt(n)
    return to_natural_order(np.fft.ifft(yt, axis=-1) * math.sqrt(n), m).real


def update_weights(family, m: int) -> np.ndarray:
    """Weights w_m of the doubling update (Sec. 5.4): all ones for the Hadamard matrix
    (nets), exp(-pi i k / 2^m) for the bit-reversed Fourier matrix (lattices)."""
    n = 1 << m
    if family == "dsi":
        return np.ones(n)
    return np.exp(-1j * np.pi * np.arange(n) / n)


def extend_transformed(family, yt_old, yt_new):
    """conj(V_{m+1}) [y; y_new] from yt_old = conj(V_m) y and yt_new = conj(V_m) y_new
    (Sec. 5.4 update; the weights multiply the new half):
    [yt_old + w yt_new, yt_old - w yt_new] / sqrt(2)."""
    yt_old = np.asarray(yt_old)
    m = yt_old.shape[-1].bit_length() - 1
    wy = update_weights(family, m) * np.asarray(yt_new)
    return np.concatenate([yt_old + wy, yt_old - wy], axis=-1) / math.sqrt(2.0)


def extend_eigenvalues(family, lam_old, k1_new):
    """Eigenvalues of the doubled Gram matrix from lam_old (those of the first n points,
    nugget included) and the first-column entries k1_new of the n new points: with
    t = sqrt(n) conj(V_m) k1_new, lam' = [lam_old + w t, lam_old - w t] (real)."""
    k1_new = np.asarray(k1_new, dtype=np.float64)
    n = k1_new.shape[-1]
    m = n.bit_length() - 1
    t = forward_transform(family, k1_new) * math.sqrt(n)
    wt = (update_weights(family, m) * t).real
    return np.concatenate([lam_old + wt, lam_old - wt], axis=-1)


def spectral_solve(family, lam, y):
    """K^-1 y = V (y~ / lambda) (Sec. 5.4)."""
    return inverse_transform(family, forward_transform(family, y) / lam)


def spectral_matvec(family, lam, y):
    """K y = V (y~ * lambda) (Sec. 5.4)."""
    return inverse_transform(family, forward_transform(family, y) * lam)


def spectral_mll(family, lam, y, zeta=1.0):
    """MLL pieces from the spectrum: quad = sum |y~|^2/lambda, log det = sum log lambda,
    posterior mean zeta 1^T K^-1 y = zeta sum(y)/lambda_0 and variance
    zeta - zeta^2 n / lambda_0 (the constant vector is the w = 0 eigenvector)."""
    yt = forward_transform(family, y)
    n = lam.shape[-1]
    quad = float(np.sum(np.abs(yt) ** 2 / lam))
    logdet = float(np.sum(np.log(lam)))
    mll = -0.5 * quad - 0.5 * logdet - 0.5 * n * math.log(2 * math.pi)
    mean = zeta * float(np.sum(y)) / float(lam[0])
    var = zeta - zeta * zeta * n / float(lam[0])
    return {"quad": quad, "logdet": logdet, "mll": mll, "post_mean": mean, "post_var": var}


def spectral_mll_grad(family, alpha, X, y, lam, c_w, zeta=1.0):
    """Gradient of the MLL through the spectrum (the structure fixes V, only lambda moves).

    dMLL/dtheta = sum_w g_w dlambda_w/dtheta with g_w = (|y~_w|^2/lambda_w^2 - 1/lambda_w)/2,
    and dlambda/dc_j = sqrt(n) conj(V) dk_1/dc_j, hence dMLL/dc_j = sum_i u_i dk1_i/dc_j with
    u = H g (DSI) or u_lin = FFT(g) (SI), mapped back to natural order.  dMLL/deta = sum g.
    """
    yt = forward_transform(family, y)
    n = lam.shape[-1]
    m = n.bit_length() - 1
    gw = 0.5 * (np.abs(yt) ** 2 / lam ** 2 - 1.0 / lam)
    if family == "dsi":
        u = hadamard_apply(gw)
    else:
        u = to_natural_order(np.fft.fft(gw).real, m)
    d = X.shape[1]
    dc = np.empty(d)
    dsum = np.empty(d)
    for j in range(d):
        dk1 = np.full(n, float(zeta))
        for jj in range(d):
            diff = pair_difference(family, X[:, jj], X[0, jj])
            Kv = factor_values(family, alpha, diff)
            dk1 *= Kv if jj == j else (1.0 + c_w[jj] * Kv)
        dc[j] = float(u @ dk1)
        dsum[j] = float(np.sum(dk1))
    ysum = float(np.sum(y))
    lam0 = float(lam[0])
    return {
        "dc": dc,
        "dtheta": c_w * dc,
        "deta": float(np.sum(gw)),
        "dmean_dc": -zeta * ysum * dsum / lam0 ** 2,
        "dmean_deta": -zeta * ysum / lam0 ** 2,
    }


# ------------------------------------------- test integrands and the baker transform


def baker(x) -> np.ndarray:
    """Baker (tent) transform x -> 1 - 2|x - 1/2| applied elementwise (Sec. 4.2): it maps the
    uniform distribution to itself, so it does not change an integrand's mean."""
    x = np.asarray(x, dtype=np.float64)
    return 1.0 - 2.0 * np.abs(x - 0.5)


def _genz_coefficients(kind: str, d: int) -> np.ndarray:
    """Genz coefficients (Sec. 6): oscillatory c_j = 4.5 ct_j / sum ct with
    ct_j = exp(j log(1e-8) / d) ("third kind"); corner peak c_j = 0.25 ct_j / sum ct with
    ct_j = 1/j^2 ("second kind"); j = 1..d."""
    j = np.arange(1, d + 1, dtype=np.float64)
    if kind == "oscillatory":
        ct = np.exp(j * math.log(1e-8) / d)
        return 4.5 * ct / ct.sum()
    ct = 1.0 / j ** 2
    return 0.25 * ct / ct.sum()


def integrand(name: str, x) -> np.ndarray:
    """The six test integrands of the numerical experiments (Sec. 6), x of shape (..., n, d):

    simple1   d = 1: x e^x - 1
    simple2   d = 2: x_2 e^{x_1 x_2} / (e - 2) - 1
    oakley    d = 2: g((x - 1/2)/50), g(t) = 5 + t_1 + t_2 + 2 cos t_1 + 2 cos t_2
    gfun      any d: prod_j (|4 x_j - 2| - a_j) / (1 + a_j), a_j = (j - 2)/2
    genz_osc  any d: cos(-sum_j c_j x_j), oscillatory coefficients
    genz_cp   any d: (1 + sum_j c_j x_j)^-(d + 1), corner-peak coefficients
    """
    x = np.asarray(x, dtype=np.float64)
    d = x.shape[-1]
    if name == "simple1":
        return x[..., 0] * np.exp(x[..., 0]) - 1.0
    if name == "simple2":
        return x[..., 1] * np.exp(x[..., 0] * x[..., 1]) / (math.e - 2.0) - 1.0
    if name == "oakley":
        t = (x - 0.5) / 50.0
        return 5.0 + t[..., 0] + t[..., 1] + 2.0 * np.cos(t[..., 0]) + 2.0 * np.cos(t[..., 1])
    if name == "gfun":
        a = (np.arange(1, d + 1, dtype=np.float64) - 2.0) / 2.0
        return np.prod((np.abs(4.0 * x - 2.0) - a) / (1.0 + a), axis=-1)
    if name == "genz_osc":
        return np.cos(-(x @ _genz_coefficients("oscillatory", d)))
    if name == "genz_cp":
        return (1.0 + x @ _genz_coefficients("corner", d)) ** (-(d + 1))
    raise KeyError(name)


def integrand_mean(name: str, d: int) -> float:
    """Exact means of the integrands over [0,1]^d (closed forms, for pinning):
    simple1, simple2: 0 (int_0^1 x e^x dx = 1; int int x_2 e^{x_1 x_2} = e - 2);
    oakley: 5 + 4 sin(1/100) / (1/100) (t uniform on [-1/100, 1/100]);
    gfun: prod_j (1 - a_j)/(1 + a_j) (E|4x - 2| = 1);
    genz_osc: Re prod_j (1 - e^{-i c_j}) / (i c_j);
    genz_cp: sum_{v in {0,1}^d} (-1)^|v| / (1 + c.v), over d! prod_j c_j (iterated integration)."""
    if name in ("simple1", "simple2"):
        return 0.0
    if name == "oakley":
        return 5.0 + 4.0 * math.sin(0.01) / 0.01
    if name == "gfun":
        a = (np.arange(1, d + 1, dtype=np.float64) - 2.0) / 2.0
        return float(np.prod((1.0 - a) / (1.0 + a)))
    if name == "genz_osc":
        c = _genz_coefficients("oscillatory", d)
        return float(np.real(np.prod((1.0 - np.exp(-1j * c)) / (1j * c))))
    if name == "genz_cp":
        c = _genz_coefficients("corner", d)
        total = Fraction(0)
        for mask in range(1 << d):
            v = [(mask >> j) & 1 for j in range(d)]
            s = 1.0 + sum(cj for cj, vj in zip(c, v) if vj)
            total += Fraction((-1) ** sum(v)) / Fraction(s)
        return float(total / (math.factorial(d) * Fraction(float(np.prod(c)))))
    raise KeyError(name)


# ------------------------------------------------- RQMC estimate with a Student-t interval


def rqmc_estimate(y, tau: float):
    """RQMC estimate from R randomizations (Sec. 3.1, Eq. RQMC): mu_r = mean_i y[r, i],
    mu = mean_r mu_r, sigma^2 = sum_r (mu_r - mu)^2 / (R - 1), and the 100(1 - tau)%
    interval mu +- t_{R-1, tau/2} sigma / sqrt(R) with the Student-t quantile (scipy)."""
    import scipy.stats
    y = np.asarray(y, dtype=np.float64)
    R = y.shape[0]
    mu_r = y.mean(axis=1)
    mu = float(mu_r.mean())
    sigma = float(np.sqrt(np.sum((mu_r - mu) ** 2) / (R - 1)))
    t_star = float(-scipy.stats.t.ppf(tau / 2.0, df=R - 1))
    return {"mu_r": mu_r, "mu": mu, "sigma": sigma, "t": t_star, "half_width": t_star * sigma / math.sqrt(R)}


# ---------------------------------- kernel discrepancy / worst-case error (Sec. 3.2)


def kernel_mean_1d(family: str, alpha: int, x_word: int, grid_bits: int = 16) -> float:
    """int_0^1 K_alpha(u, x) du for one 32-bit point x by the left-point rule on the 2^-grid
    grid (the grid is closed under (-) x's top digits, so for DSI kernels the rule sums
    K_alpha over a shifted grid); used to pin kappa_i = int K(u, x_i) du."""
    u = (np.arange(1 << grid_bits, dtype=np.uint64) << np.uint64(32 - grid_bits)).astype(np.uint32)
    diff = pair_difference(family, u, np.uint32(x_word))
    return float(np.mean(factor_values(family, alpha, diff)))


def discrepancy2_dense(family, alpha, X, c, zeta, w) -> float:
    """Squared worst-case error of the cubature sum_i w_i f(x_i) in the RKHS of K (Sec. 3.2):
    int int K - 2 sum_i w_i kappa_i + w^T K w, with the dense Gram matrix (no nugget),
    kappa_i = int K(u, x_i) du = zeta and int int K = zeta (each one-dimensional K_alpha
    integrates to zero, pinned by kernel_mean_1d)."""
    K = gram_dense(family, alpha, X, c, zeta, 0.0)
    w = np.asarray(w, dtype=np.float64)
    kappa = np.full(X.shape[0], float(zeta))
    return float(zeta - 2.0 * w @ kappa + w @ K @ w)


def optimal_weights_dense(family, alpha, X, c, zeta, eta=0.0) -> np.ndarray:
    """Weights minimising the squared worst-case error: w* = K^-1 kappa (Sec. 3.2), by Cholesky."""
    K = gram_dense(family, alpha, X, c, zeta, eta)
    sol, _ = cholesky_solve(K, np.full(X.shape[0], float(zeta)))
    return sol


def discrepancy2_spectral(family, lam, w, zeta) -> float:
    """The same squared worst-case error through the spectrum (Sec. 5.4): w^T K w = w . K w with
    K w = V(w~ lambda)."""
    w = np.asarray(w, dtype=np.float64)
    return float(zeta - 2.0 * zeta * np.sum(w) + w @ spectral_matvec(family, lam, w))


# ------------------------------------------- higher-order digital nets (Sec. 4.3)


def interlace(A, alpha: int, t_out: int = 64) -> np.ndarray:
    """Digital interlacing of order alpha (Sec. 4.3, "Digital interlacing for higher-order
    nets"): generator columns A (alpha d, 32) of 32-digit words (column k, bit 31 - t =
    digit t) -> d interlaced matrices with alpha 32 digits, of which the first t_out are
    kept (digits past t_out lie below 2^-t_out).  Entry (t, k) of the j-th interlaced matrix
    (1-based j) is entry (floor(t / alpha), k) of matrix alpha (j - 1) + (t mod alpha) + 1.
    Returns (d, 32) uint64 words, bit (63 - t) = digit t (t < t_out <= 64)."""
    A = np.asarray(A, dtype=np.uint64)
    d = A.shape[0] // alpha
    t_max = min(t_out, 32 * alpha)
    out = np.zeros((d, 32), dtype=np.uint64)
    for j in range(1, d + 1):
        for t in range(t_max):
            src = alpha * (j - 1) + (t % alpha) + 1          # 1-based source matrix
            t_src = t // alpha
            bit = (A[src - 1] >> np.uint64(31 - t_src)) & np.uint64(1)
            out[j - 1] |= bit << np.uint64(63 - t)
    return out


def ho_net_points(Chat, D, idx, m: int, order: str = "gray") -> np.ndarray:
    """Higher-order digital net points as 64-digit words: z = Chat_j D_m(k) mod 2 with k = i
    or its Gray code, digitally shifted by the 64-digit D_j (Sec. 4.3).  Chat: (d, 32) uint64
    interlaced columns; D: (d,) uint64.  Returns (len(idx), d) uint64."""
    idx = np.asarray(idx, dtype=np.uint64)
    k = gray_code(idx) if order == "gray" else idx
    Chat = np.asarray(Chat, dtype=np.uint64)
    d = Chat.shape[0]
    X = np.zeros((idx.size, d), dtype=np.uint64)
    for t in range(m):
        digit = ((k >> np.uint64(t)) & np.uint64(1)).astype(bool)
        for j in range(d):
            X[digit, j] ^= Chat[j, t]
    X ^= np.asarray(D, dtype=np.uint64)[None, :]
    return X


def deinterlace_point(Xhat, alpha: int, digits: int = 64) -> np.ndarray:
    """The alpha d coordinates (as 32-digit words, digits beyond those kept set to 0) whose
    interlacing gives the points Xhat (n, d) uint64: coordinate alpha j + u takes digits
    u, u + alpha, u + 2 alpha, ... of Xhat_j (0-based)."""
    Xhat = np.asarray(Xhat, dtype=np.uint64)
    n, d = Xhat.shape
    out = np.zeros((n, alpha * d), dtype=np.uint64)
    for j in range(d):
        for t in range(min(digits, 32 * alpha)):
            bit = (Xhat[:, j] >> np.uint64(63 - t)) & np.uint64(1)
            out[:, alpha * j + t % alpha] |= bit << np.uint64(31 - t // alpha)
    return out.astype(np.uint32)


def dsi_kernel_words(alpha: int, Z, digits: int = 64) -> np.ndarray:
    """K_alpha(x) of the Theorem (Sec. 5.3) at x = Z 2^-digits for words of `digits` digits
    (64 for interlaced nets): beta(x) = -floor(log2 x) is the position of the first nonzero
    digit, t_nu = 2^(-nu beta), and K_4's series sum_a wal_{2^a}(x) 8^-a runs over the
    `digits` digits (later digits 0): 8/7 - 2 sum_{a < digits, x_{a+1} = 1} 8^-a."""
    Zs = [int(z) for z in np.asarray(Z, dtype=np.uint64).ravel()]
    out = np.empty(len(Zs))
    for q, z in enumerate(Zs):
        if z == 0:
            beta, x, t1 = 0, 0.0, 0.0
        else:
            beta = digits - z.bit_length() + 1
            x = float(Fraction(z, 1 << digits))
            t1 = 2.0 ** -beta
        b = float(beta)
        t2, t3 = t1 * t1, t1 * t1 * t1
        if alpha == 1:
            out[q] = 1.0 - 3.0 * t1 if z else 1.0
        elif alpha == 2:
            out[q] = -1.0 - b * x + 2.5 * (1.0 - t1)
        elif alpha == 3:
            out[q] = -1.0 + b * x ** 2 - 5.0 * (1.0 - t1) * x + (43.0 / 18.0) * (1.0 - t2)
        elif alpha == 4:
            S = Fraction(8, 7)
            for a in range(digits):
                if (z >> (digits - 1 - a)) & 1:
                    S -= 2 * Fraction(1, 8 ** a)
            out[q] = (-1.0 - (2.0 / 3.0) * b * x ** 3 + 5.0 * (1.0 - t1) * x ** 2
                      - (43.0 / 9.0) * (1.0 - t2) * x + (701.0 / 294.0) * (1.0 - t3)
                      + b * (float(S) / 48.0 - 1.0 / 42.0))
        else:
            raise ValueError(f"DSI order {alpha} not supported")
    return out.reshape(np.shape(Z))


def ho_first_column(alpha_k: int, Xhat, c, zeta=1.0) -> np.ndarray:
    """k_1[i] = zeta prod_j (1 + c_j K_alpha(x_ij (-) x_0j)) for 64-digit points (Sec. 5.3-5.4)."""
    Xhat = np.asarray(Xhat, dtype=np.uint64)
    out = np.full(Xhat.shape[0], float(zeta))
    for j in range(Xhat.shape[1]):
        out *= 1.0 + c[j] * dsi_kernel_words(alpha_k, Xhat[:, j] ^ Xhat[0, j])
    return out


def ho_gram_dense(alpha_k: int, Xhat, c, zeta=1.0, eta=0.0) -> np.ndarray:
    """Dense Gram matrix of the product DSI kernel on 64-digit points, plus eta I."""
    Xhat = np.asarray(Xhat, dtype=np.uint64)
    n = Xhat.shape[0]
    K = np.full((n, n), float(zeta))
    for j in range(Xhat.shape[1]):
        Z = Xhat[:, j][:, None] ^ Xhat[None, :, j]
        K *= 1.0 + c[j] * dsi_kernel_words(alpha_k, Z)
    return K + eta * np.eye(n)


def ho_gram_weight_derivative(alpha_k: int, Xhat, c, j: int, zeta=1.0) -> np.ndarray:
    """dK/dc_j for the product DSI kernel on 64-digit points (dense)."""
    Xhat = np.asarray(Xhat, dtype=np.uint64)
    n = Xhat.shape[0]
    out = np.full((n, n), float(zeta))
    for jj in range(Xhat.shape[1]):
        Kv = dsi_kernel_words(alpha_k, Xhat[:, jj][:, None] ^ Xhat[None, :, jj])
        out *= Kv if jj == j else (1.0 + c[jj] * Kv)
    return out


def ho_mll_grad_dense(alpha_k: int, Xhat, y, c, eta, zeta=1.0):
    """dMLL/dc_j = c^T dK c / 2 - tr(K^-1 dK) / 2 and dMLL/deta for 64-digit points (dense,
    the textbook GP gradient as in mll_grad_dense)."""
    K = ho_gram_dense(alpha_k, Xhat, c, zeta, eta)
    n, d = Xhat.shape
    L = np.linalg.cholesky(K)
    cvec = scipy.linalg.cho_solve((L, True), y)
    Kinv = scipy.linalg.cho_solve((L, True), np.eye(n))
    dc = np.empty(d)
    for j in range(d):
        dK = ho_gram_weight_derivative(alpha_k, Xhat, c, j, zeta)
        dc[j] = 0.5 * cvec @ dK @ cvec - 0.5 * float(np.sum(Kinv * dK.T))
    deta = 0.5 * cvec @ cvec - 0.5 * float(np.trace(Kinv))
    return {"dc": dc, "deta": deta}
