"""qk_eigs_static, the eigenvalue entry point for callers that cannot allocate device
memory (its scratch is a static device array owned by the library), against qk_eigs,
which takes a caller workspace.  Collected last so that a run stopping at the first
failure has run every other test; it also passes on its own in a fresh process."""
import ctypes as C

import numpy as np
import pytest
import torch

from tests import qkcases as qc

pytestmark = pytest.mark.gpu

F64, F32 = torch.float64, torch.float32


@pytest.fixture(scope="module")
def qk():
    from paper_2502_14256_gb300 import build
    build.build()
    from paper_2502_14256_gb300 import qk as q
    return q


@pytest.mark.parametrize("kind,family,alpha,m,dt", [("net", "dsi", 2, 14, F64), ("net", "dsi", 4, 17, F32),
                                                    ("lattice", "si", 2, 12, F64), ("lattice", "si", 1, 15, F32)])
def test_static_scratch_eigenvalues_match_the_workspace_entry_point(qk, kind, family, alpha, m, dt):
    d, R, eta, zeta = 4, 2, 1e-6, 1.3
    case = qc.make_case(kind, family, alpha, d, R, seed=7000 + m, c=0.7 ** np.arange(1, d + 1), zeta=zeta)
    kern = qc.kernel_of(case)
    fam = qk.QK_DSI if family == "dsi" else qk.QK_SI
    col = torch.empty((R, 1 << m), dtype=dt, device=qc.dev())
    qk.kernel_col(case.ps, kern, 0, R, m, col, form=qk.QK_COL_P)
    tol = 1e-12 if dt == F64 else 1e-6
    # two calls in a row on different columns: the second must not see the first's data
    for r in (0, 1, 0):
        one = col[r:r + 1].contiguous()
        ref = torch.empty((1, 1 << m), dtype=F64, device=qc.dev())
        qk.eigs(fam, m, one, ref, zeta=zeta, eta=eta, form=qk.QK_COL_P)
        got = torch.full_like(ref, float("nan"))
        qk.eigs_static(fam, m, one, got, zeta=zeta, eta=eta, form=qk.QK_COL_P)
        torch.cuda.synchronize()
        assert qc.rel_err(got.cpu().numpy(), ref.cpu().numpy()) < tol
    # and the whole batch at once
    ref = torch.empty((R, 1 << m), dtype=F64, device=qc.dev())
    qk.eigs(fam, m, col, ref, zeta=zeta, eta=eta, form=qk.QK_COL_P)
    got = torch.full_like(ref, float("nan"))
    qk.eigs_static(fam, m, col, got, zeta=zeta, eta=eta, form=qk.QK_COL_P)
    assert qc.rel_err(got.cpu().numpy(), ref.cpu().numpy()) < tol


def test_static_scratch_refuses_requests_beyond_its_size(qk):
    fake = C.c_void_p(0x1000)
    # 2^20 FP64 net elements need 8 MiB, twice the static array: refused before any launch
    rc = qk.LIB.qk_eigs_static(qk.QK_DSI, 20, 1, qk.QK_F64, qk.QK_COL_K1, fake, 1.0, 0.0, fake, None, None)
    assert rc == qk.QK_EINVAL
    assert "static array" in qk.last_error()
