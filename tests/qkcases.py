"""Shared builders for the GPU parity tests: seeded inputs from the input module,
uploaded as raw 32-bit words, with the oracle's reference arrays beside them."""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch

from oracle import qk_oracle as o
from paper_2502_14256_gb300 import inputs


def dev():
    return torch.device("cuda:0")


def u32_tensor(a):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.uint32)).view(np.int32)).to(dev())


def u32_host(t):
    return t.detach().cpu().numpy().view(np.uint32)


def rel_err(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.max(np.abs(b))
    return float(np.max(np.abs(a - b)) / (den if den > 0 else 1.0))


@dataclass
class Case:
    kind: str
    family: str
    alpha: int
    d: int
    R: int
    order: str
    ps: object          # qk.PointSet
    Ct_ref: np.ndarray | None
    g: np.ndarray | None
    D: np.ndarray
    keep: list          # device tensors kept alive
    c: np.ndarray       # effective weights
    zeta: float

    def points_ref(self, r, idx, m):
        if self.kind == "net":
            return o.net_points(self.Ct_ref[r], self.D[r], idx, m, self.order)
        return o.lattice_points(self.g, self.D[r], idx)

    def k1_ref(self, r, m):
        X = self.points_ref(r, np.arange(1 << m), m)
        return o.first_column(self.family, self.alpha, X, self.c, self.zeta), X


def make_case(kind, family, alpha, d, R, seed, c=None, zeta=1.0, order="gray", m_gen=20):
    from paper_2502_14256_gb300 import qk
    keep = []
    if c is None:
        c = 1.0 / np.arange(1, d + 1) ** 2
    if kind == "net":
        net = inputs.make_net(seed, d, R, order)
        Cd, Sd, Dd = u32_tensor(net.C), u32_tensor(net.S), u32_tensor(net.D)
        Ct = torch.empty((R, d, 32), dtype=torch.int32, device=dev())
        qk.lms_setup(Cd, Sd, Ct)
        keep += [Cd, Sd, Dd, Ct]
        ps = qk.pointset(qk.QK_NET_B2, d, R, Ct=Ct, D=Dd, order=qk.QK_GRAY if order == "gray" else qk.QK_NATURAL)
        Ct_ref = o.lms_scramble(net.C, net.S)
        return Case(kind, family, alpha, d, R, order, ps, Ct_ref, None, net.D, keep, np.asarray(c, float), zeta)
    lat = inputs.make_lattice(seed, d, R, m_gen)
    gd, Dd = u32_tensor(lat.g), u32_tensor(lat.D)
    keep += [gd, Dd]
    ps = qk.pointset(qk.QK_LATTICE, d, R, g=gd, D=Dd)
    return Case(kind, family, alpha, d, R, "natural", ps, None, lat.g, lat.D, keep, np.asarray(c, float), zeta)


def kernel_of(case):
    from paper_2502_14256_gb300 import qk
    w = torch.tensor(case.c, dtype=torch.float64, device=dev())
    case.keep.append(w)
    fam = qk.QK_DSI if case.family == "dsi" else qk.QK_SI
    return qk.kernel(fam, case.alpha, w, case.zeta)


def lam_elementwise_ok(got, want, rel, eps, m, factor=8.0):
    """Every eigenvalue within rel of the reference, or within the absolute rounding floor of
    an eps-precision transform of the first column, factor * sqrt(m + 1) * eps * max|lambda|
    (the normwise check alone admits that much error on every eigenvalue, the smallest
    included; this one bounds each by its own size first)."""
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    floor = factor * np.sqrt(m + 1) * eps * np.max(np.abs(want))
    return bool(np.all(np.abs(got - want) <= rel * np.abs(want) + floor))


def lam_elementwise_report(got, want):
    err = np.abs(np.asarray(got) - np.asarray(want))
    k = int(np.argmax(err / np.abs(want)))
    return {"worst_rel": float(err[k] / abs(want[k])), "at_lambda": float(want[k]), "max_lambda": float(np.max(np.abs(want))),
            "abs_err": float(err[k])}


def ff_column_floor(lam, d):
    """Absolute perturbation of every eigenvalue by a float-float first column: about 2^-46
    per operation, ~5 operations per factor and d factors in a random walk, times ~6 for the
    largest of n Gaussian-like errors, applied to each entry of p (rms ||lambda_{w>0}|| / n),
    summed by the transform (sqrt(n)): 2^-46 sqrt(5 d) 6 ||lambda_{w>0}||_2 / sqrt(n)."""
    lam = np.asarray(lam, dtype=np.float64)
    n = lam.shape[-1]
    return 2.0 ** -46 * math.sqrt(5 * d) * 6.0 * float(np.linalg.norm(lam[1:])) / math.sqrt(n)


def cond_tol(lam, base, eps, factor=20.0):
    """Forward-error tolerance for a solve with spectrum lam: the larger of the target
    and factor * cond * eps (a backward-stable solve loses about cond * eps)."""
    lam = np.asarray(lam, dtype=np.float64)
    cond = float(np.max(np.abs(lam)) / np.min(np.abs(lam)))
    return max(base, factor * cond * eps)


EPS64 = 2.0 ** -53
EPS32 = 2.0 ** -24
