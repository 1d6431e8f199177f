"""qk_fwht_ws (two-pass launches or one persistent launch with a ticket queue), its tuner
and its bounded wait: bit-identical to qk_fwht (the same butterflies in the same order) for
every plan, equal to the oracle's Hadamard transform, and a wait that runs out returns a
status instead of hanging."""
import numpy as np
import pytest
import torch

from oracle import qk_oracle as o

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qk():
    from paper_2502_14256_gb300 import build
    build.build()
    from paper_2502_14256_gb300 import qk as q
    return q


def _data(nvec, m, dtype, seed):
    g = torch.Generator(device="cuda:0").manual_seed(seed)
    return torch.randn((nvec, 1 << m), dtype=dtype, device="cuda:0", generator=g)


CASES = [(torch.float32, 14, 1), (torch.float32, 16, 37), (torch.float32, 20, 9), (torch.float32, 21, 3),
         (torch.float64, 13, 5), (torch.float64, 17, 11), (torch.float64, 19, 2), (torch.float64, 20, 3)]


@pytest.mark.parametrize("dtype,m,nvec", CASES)
def test_every_plan_is_bitwise_qk_fwht(qk, dtype, m, nvec):
    x = _data(nvec, m, dtype, seed=m * 100 + nvec)
    ref = qk.fwht(m, x.clone())
    plans = [dict(mode=qk.QK_FWHT_TWO_PASS)] + [dict(mode=qk.QK_FWHT_PERSISTENT, lag=lag, ctas_per_sm=cps)
                                                 for lag in (0, 1, 2, nvec + 5) for cps in (0, 1, 3)]
    status = torch.zeros(1, dtype=torch.int32, device="cuda:0")
    for plan in plans:
        got = qk.fwht_ws(m, x.clone(), plan=plan, status=status)
        qk.read_status(status)
        assert torch.equal(got, ref), plan


def test_tuned_plan_is_used_and_exact(qk):
    m, nvec, dtype = 18, 24, torch.float32
    scratch = _data(nvec, m, dtype, seed=1)
    plan = qk.fwht_tune(m, scratch)
    assert plan["ms"] > 0
    x = _data(nvec, m, dtype, seed=2)
    ref = qk.fwht(m, x.clone())
    got = qk.fwht_ws(m, x.clone())
    assert torch.equal(got, ref), plan


def test_persistent_matches_oracle(qk):
    m, nvec = 15, 3
    x = _data(nvec, m, torch.float64, seed=3)
    got = qk.fwht_ws(m, x.clone(), plan=dict(mode=qk.QK_FWHT_PERSISTENT, lag=1, ctas_per_sm=2)).cpu().numpy()
    xs = x.cpu().numpy()
    for v in range(nvec):
        want = o.hadamard_apply(xs[v]) / np.sqrt(1 << m)
        assert np.max(np.abs(got[v] - want)) < 1e-13 * np.max(np.abs(want)) * m


def test_wait_that_runs_out_returns_timeout_status(qk):
    """Column tiles with no published low tile: every bounded wait expires, each tile is
    skipped, QK_STATUS_TIMEOUT is reported, and the context keeps working."""
    m, nvec = 15, 2
    x = _data(nvec, m, torch.float32, seed=4)
    before = x.clone()
    status = torch.zeros(1, dtype=torch.int32, device="cuda:0")
    qk.fwht_wait_selftest(m, x, 1 << 12, status)
    torch.cuda.synchronize()
    assert int(status.item()) & qk.QK_STATUS_TIMEOUT
    assert torch.equal(x, before)
    with pytest.raises(qk.QKError) as e:
        qk.read_status(status)
    assert e.value.code == qk.QK_ETIMEOUT
    assert int(status.item()) == 0
    ref = qk.fwht(m, x.clone())
    assert torch.equal(qk.fwht_ws(m, x.clone()), ref)
