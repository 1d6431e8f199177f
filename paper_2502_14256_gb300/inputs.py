"""Seeded synthetic inputs shared by the tests, the bench and the oracle checks.

This module holds no arithmetic of the method itself: it only draws random
integers and floats (SplitMix64, Steele, Lea & Flood 2014, "Fast splittable
pseudorandom number generators") and packs them into the arrays that the
method consumes:

* generator matrices of a base-2 digital net, one ``uint32`` word per column
  (bit 31 is the first output digit, i.e. the coefficient of 1/2),
* Matousek linear-scrambling matrices, one ``uint32`` row mask per row
  (bit 31 - u selects input digit u),
* digital shifts / lattice shifts as ``uint32`` words (value = word * 2^-32),
* lattice generating vectors, weights and right-hand sides.

Everything is a pure function of an integer seed, so the CUDA path and the
oracle are fed bit-identical inputs.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

M64 = (1 << 64) - 1
BASE_SEED = 20250220


class SplitMix64:
    """SplitMix64 stream (Steele, Lea & Flood 2014), vectorised over numpy uint64."""

    GOLDEN = np.uint64(0x9E3779B97F4A7C15)

    def __init__(self, seed: int):
        self.state = np.uint64(seed & M64)

    def next_u64(self, count: int) -> np.ndarray:
        count = int(count)
        with np.errstate(over="ignore"):
            k = np.arange(1, count + 1, dtype=np.uint64)
            z = self.state + k * self.GOLDEN
            self.state = self.state + np.uint64(count) * self.GOLDEN
            z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
            z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
            z = z ^ (z >> np.uint64(31))
        return z

    def u32(self, count: int) -> np.ndarray:
        return (self.next_u64(count) >> np.uint64(32)).astype(np.uint32)

    def uniform(self, count: int) -> np.ndarray:
        """Doubles in [0, 1) from the top 53 bits."""
        return (self.next_u64(count) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53

    def normal(self, count: int) -> np.ndarray:
        """Standard normals by the Box-Muller transform."""
        count = int(count)
        half = (count + 1) // 2
        u1 = 1.0 - self.uniform(half)  # (0, 1]
        u2 = self.uniform(half)
        r = np.sqrt(-2.0 * np.log(u1))
        z = np.concatenate([r * np.cos(2 * np.pi * u2), r * np.sin(2 * np.pi * u2)])
        return z[:count]

    def integers(self, lo: int, hi: int, count: int) -> np.ndarray:
        """Integers uniform in [lo, hi) (hi - lo <= 2^32), by 64-bit multiply-shift."""
        span = hi - lo
        u = self.u32(count).astype(np.uint64)
        return (lo + ((u * np.uint64(span)) >> np.uint64(32))).astype(np.int64)


# --------------------------------------------------------------------------- nets
def identity_columns() -> np.ndarray:
    """Columns of the 32x32 identity: column k has only output digit k (bit 31-k)."""
    return np.array([1 << (31 - k) for k in range(32)], dtype=np.uint32)


def random_upper_unit_columns(rng: SplitMix64) -> np.ndarray:
    """Columns of a random 32x32 upper-triangular unit-diagonal binary matrix.

    Column k may hold output digits t <= k (bits 31..31-k); digit k is 1.
    """
    words = rng.u32(32)
    cols = np.empty(32, dtype=np.uint32)
    for k in range(32):
        keep = ((1 << (k + 1)) - 1) << (31 - k)  # bits 31 .. 31-k
        cols[k] = (int(words[k]) & keep) | (1 << (31 - k))
    return cols


def random_lower_unit_rows(rng: SplitMix64) -> np.ndarray:
    """Row masks of a random lower-triangular unit-diagonal binary matrix (Matousek).

    Row t may hold input digits u <= t (bits 31..31-t); digit t is 1.
    """
    words = rng.u32(32)
    rows = np.empty(32, dtype=np.uint32)
    for t in range(32):
        keep = ((1 << (t + 1)) - 1) << (31 - t)
        rows[t] = (int(words[t]) & keep) | (1 << (31 - t))
    return rows


@dataclass
class NetInputs:
    d: int
    R: int
    C: np.ndarray      # (d, 32) uint32 generator columns
    S: np.ndarray      # (R, d, 32) uint32 LMS row masks
    D: np.ndarray      # (R, d) uint32 digital shifts
    order: str = "gray"


def make_net(seed: int, d: int, R: int, order: str = "gray") -> NetInputs:
    rng = SplitMix64(seed)
    C = np.empty((d, 32), dtype=np.uint32)
    C[0] = identity_columns()
    for j in range(1, d):
        C[j] = random_upper_unit_columns(rng)
    S = np.empty((R, d, 32), dtype=np.uint32)
    for r in range(R):
        for j in range(d):
            S[r, j] = random_lower_unit_rows(rng)
    D = rng.u32(R * d).reshape(R, d)
    return NetInputs(d=d, R=R, C=C, S=S, D=D, order=order)


@dataclass
class HONetInputs:
    d: int                    # dimensions of the interlaced (higher-order) net
    alpha: int                # interlacing order
    R: int
    C: np.ndarray             # (alpha d, 32) u32 generator columns of the underlying net
    S: np.ndarray             # (R, alpha d, 32) u32 LMS row masks
    D: np.ndarray             # (R, d) u64 digital shifts with 64 digits
    order: str


def make_ho_net(seed: int, d: int, alpha: int, R: int, order: str = "gray") -> HONetInputs:
    """Inputs of an order-alpha interlaced net in d dimensions: the alpha d generator matrices
    (the first the identity, the others random upper unit-triangular), an LMS scramble per
    randomization and matrix, and a 64-digit digital shift per randomization and dimension."""
    base = make_net(seed, alpha * d, R, order)
    rng = SplitMix64(seed + 0x5EED)
    hi = rng.u32(R * d).astype(np.uint64)
    lo = rng.u32(R * d).astype(np.uint64)
    D = ((hi << np.uint64(32)) | lo).reshape(R, d)
    return HONetInputs(d=d, alpha=alpha, R=R, C=base.C, S=base.S, D=D, order=order)


@dataclass
class LatticeInputs:
    d: int
    R: int
    g: np.ndarray      # (d,) uint32 odd generating vector
    D: np.ndarray      # (R, d) uint32 shifts on the 2^-32 grid


def make_lattice(seed: int, d: int, R: int, m_gen: int) -> LatticeInputs:
    """Generating vector of odd integers uniform in [1, 2^m_gen)."""
    rng = SplitMix64(seed)
    half = rng.integers(0, 1 << (m_gen - 1), d)
    g = (2 * half + 1).astype(np.uint32)
    D = rng.u32(R * d).reshape(R, d)
    return LatticeInputs(d=d, R=R, g=g, D=D)


# ------------------------------------------------------------ right-hand sides
def points_as_float(X: np.ndarray) -> np.ndarray:
    """uint32 point words -> doubles in [0, 1) (exact)."""
    return X.astype(np.float64) * 2.0 ** -32


def rhs_product(X: np.ndarray) -> np.ndarray:
    """y = prod_j (1 + (x_j - 1/2)/j^2) over the last axis of X (uint32 words)."""
    x = points_as_float(X)
    j = np.arange(1, X.shape[-1] + 1, dtype=np.float64)
    return np.prod(1.0 + (x - 0.5) / j ** 2, axis=-1)


def rhs_exp(X: np.ndarray, noise: np.ndarray | None = None) -> np.ndarray:
    """y = exp(sum_j x_j / j) - prod_j j (e^{1/j} - 1) (+ noise) over the last axis."""
    x = points_as_float(X)
    d = X.shape[-1]
    j = np.arange(1, d + 1, dtype=np.float64)
    const = float(np.prod(j * np.expm1(1.0 / j)))
    y = np.exp(np.sum(x / j, axis=-1)) - const
    if noise is not None:
        y = y + noise
    return y


# ----------------------------------------------------------------- workloads
@dataclass
class Workload:
    """One named synthetic workload (a row of the project's config table)."""
    name: str
    kind: str                 # "net" or "lattice"
    family: str               # "dsi" or "si"
    alpha: int
    d: int
    ms: list                  # log2 n per instance
    R: int
    nrhs: int
    gamma: np.ndarray         # (d,) product weights
    log_ls: np.ndarray        # (d,) log lengthscales (effective weight gamma*exp(log_ls))
    eta: float
    zeta: float = 1.0
    order: str = "gray"
    seed: int = BASE_SEED
    rhs: str = "product"      # "product" or "exp"
    noise_sigma: float = 0.0
    extra: dict = field(default_factory=dict)


def workload(name: str) -> Workload:
    """Synthetic workloads shaped like the paper's experiments.

    plain      net  n=2^10 d=4  DSI order 1, gamma_j=1/j^2, eta=1e-8, y=prod(1+(x_j-.5)/j^2)
    batch      net  m in 14..20, d=16, R=64, DSI order 2, gamma_j=0.9^j, 8 rhs (exp + N(0,1e-6))
    diff       lattice n=2^18 d=32, SI alpha=2, unit weights, log_ls=0, eta=e^-12
    diff_small the same at n=2^10 (dense oracle size)
    precision  net n=2^24 d=64 R=16, DSI order 4, gamma_j=j^-3, eta=1e-8
    solve20    net n=2^20 d=16 R=64, DSI order 2, gamma_j=0.9^j, eta=1e-8, 1 rhs
    """
    j = np.arange(1, 129, dtype=np.float64)
    if name == "plain":
        d = 4
        return Workload(name, "net", "dsi", 1, d, [10], 1, 1, 1.0 / j[:d] ** 2,
                        np.zeros(d), 1e-8, seed=BASE_SEED + 1)
    if name == "batch":
        d = 16
        rng = SplitMix64(BASE_SEED + 2)
        ms = [int(v) for v in rng.integers(14, 21, 32)]
        return Workload(name, "net", "dsi", 2, d, ms, 64, 8, 0.9 ** j[:d], np.zeros(d), 1e-8,
                        seed=BASE_SEED + 2, rhs="exp", noise_sigma=1e-3)
    if name in ("diff", "diff_small"):
        d = 32
        m = 18 if name == "diff" else 10
        return Workload(name, "lattice", "si", 2, d, [m], 1, 1, np.ones(d), np.zeros(d),
                        math.exp(-12.0), seed=BASE_SEED + 3, extra={"m_gen": 18})
    if name == "precision":
        d = 64
        return Workload(name, "net", "dsi", 4, d, [24], 16, 1, j[:d] ** -3.0, np.zeros(d), 1e-8,
                        seed=BASE_SEED + 4)
    if name == "solve20":
        d = 16
        return Workload(name, "net", "dsi", 2, d, [20], 64, 1, 0.9 ** j[:d], np.zeros(d), 1e-8,
                        seed=BASE_SEED + 6, rhs="exp", noise_sigma=1e-3)
    raise KeyError(name)


def mixed_batch(seed: int = BASE_SEED + 5, count: int = 256, m_lo: int = 12, m_hi: int = 22):
    """Mixed batch: half lattice + SI alpha=1, half net + DSI order 2.

    Each instance draws m uniform in [m_lo, m_hi] and d from {8, 32, 128}.
    Weights gamma_j = 1/j^2, eta = 1e-8, y = prod(1 + (x_j - .5)/j^2).
    """
    rng = SplitMix64(seed)
    ms = rng.integers(m_lo, m_hi + 1, count)
    ds = np.array([8, 32, 128])[rng.integers(0, 3, count)]
    out = []
    for t in range(count):
        d = int(ds[t])
        j = np.arange(1, d + 1, dtype=np.float64)
        if t % 2 == 0:
            out.append(Workload(f"mixed{t}", "lattice", "si", 1, d, [int(ms[t])], 1, 1,
                                1.0 / j ** 2, np.zeros(d), 1e-8, seed=seed + 1000 + t,
                                extra={"m_gen": int(ms[t])}))
        else:
            out.append(Workload(f"mixed{t}", "net", "dsi", 2, d, [int(ms[t])], 1, 1,
                                1.0 / j ** 2, np.zeros(d), 1e-8, seed=seed + 1000 + t))
    return out
