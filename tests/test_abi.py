"""The C-ABI library builds, loads and exports every entry point include/qk.h declares.

No compute calls here (no GPU in this environment); argument validation that returns
before any launch is exercised with NULL pointers.
"""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "qk.h")


def _declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^QK_API\s+\w+\s+(qk_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2502_14256_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for need in ("qk_gen_points", "qk_kernel_col", "qk_eigs", "qk_solve", "qk_mll", "qk_batch_run"):
        assert need in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (qk_\w+)$", out, flags=re.M))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_binding_loads_and_names_match(lib_path):
    from paper_2502_14256_gb300 import qk
    assert sorted(qk.EXPORTED) == _declared()
    assert qk.version() >= 100


def test_invalid_arguments_are_rejected_before_any_launch(lib_path):
    from paper_2502_14256_gb300 import qk
    lib = qk.LIB
    # NULL point set
    assert lib.qk_gen_points(None, 0, 1, 0, 16, None, None) == qk.QK_EINVAL
    ps = qk.PointSet(qk.QK_NET_B2, qk.QK_GRAY, 0, 1, None, None, None)
    assert lib.qk_gen_points(C.byref(ps), 0, 1, 0, 16, None, None) == qk.QK_EINVAL
    assert "d = 0" in qk.last_error()
    # m too large, bad dtype, missing workspace
    size = C.c_size_t(0)
    assert lib.qk_workspace_bytes(0, qk.QK_DSI, 31, 1, 1, qk.QK_F64, 4, C.byref(size)) == qk.QK_EINVAL
    assert lib.qk_workspace_bytes(0, qk.QK_DSI, 10, 1, 1, 7, 4, C.byref(size)) == qk.QK_EINVAL
    assert lib.qk_workspace_bytes(0, qk.QK_DSI, 10, 2, 1, qk.QK_F32, 4, C.byref(size)) == qk.QK_OK
    assert size.value >= 2 * 1024 * 4
    fake = C.c_void_p(0x1000)
    rc = lib.qk_eigs(qk.QK_DSI, 10, 2, qk.QK_F32, 0, fake, 1.0, 0.0, fake, None, 0, None, None)
    assert rc == qk.QK_EWORKSPACE
    # DSI kernel on a lattice is refused
    ps = qk.PointSet(qk.QK_LATTICE, qk.QK_NATURAL, 2, 1, None, fake, None)
    k = qk.Kernel(qk.QK_DSI, 2, 2, fake, 1.0)
    assert lib.qk_kernel_col(C.byref(ps), C.byref(k), 0, 1, 4, qk.QK_F64, 0, fake, None) == qk.QK_EINVAL
    # solve refinement bound
    rc = lib.qk_solve(qk.QK_DSI, 4, 1, 1, qk.QK_F32, fake, fake, fake, 99, fake, 1 << 20, None)
    assert rc == qk.QK_EINVAL
    # batch run without a plan
    assert lib.qk_batch_run(fake, 0, None, None) == qk.QK_EINVAL


def test_documented_argument_errors_of_the_extension_and_scheduling_calls(lib_path):
    """Errors include/qk.h documents for the doubling updates, the static-scratch
    eigenvalues and the schedule / FWHT plans, all raised before any launch."""
    from paper_2502_14256_gb300 import qk
    lib = qk.LIB
    a, b = C.c_void_p(0x100000), C.c_void_p(0x100000 + 64)  # overlapping ranges
    fake = C.c_void_p(0x2000000)
    ps = qk.PointSet(qk.QK_NET_B2, qk.QK_GRAY, 2, 1, fake, None, fake)
    k = qk.Kernel(qk.QK_DSI, 2, 2, fake, 1.0)
    # positions of an extended point set start at multiples of 2048
    assert lib.qk_kernel_col_at(C.byref(ps), C.byref(k), 0, 1, C.c_uint64(100), 4, qk.QK_F64, 0, fake,
                                None) == qk.QK_EINVAL
    assert "2048" in qk.last_error()
    # the extended eigenvalues must not overlap the old ones
    assert lib.qk_eigs_extend(qk.QK_DSI, 10, 1, qk.QK_F64, 0, fake, C.c_double(1.0), C.c_double(0.0), a, b,
                              fake, C.c_size_t(1 << 30), None, None) == qk.QK_EINVAL
    # transform extensions: out must not overlap the inputs, nor x_new xt_old
    for fn in (lib.qk_fwht_extend, lib.qk_fftbr_extend):
        assert fn(10, C.c_uint64(1), qk.QK_F32, a, fake, b, None) == qk.QK_EINVAL
        assert "out must not overlap" in qk.last_error()
        assert fn(10, C.c_uint64(1), qk.QK_F32, a, b, fake, None) == qk.QK_EINVAL
        assert "x_new" in qk.last_error()
    # static scratch: a request beyond its size is refused
    assert lib.qk_eigs_static(qk.QK_DSI, 20, 8, qk.QK_F64, 0, fake, C.c_double(1.0), C.c_double(0.0), fake,
                              None, None) == qk.QK_EINVAL
    # unknown schedule and FWHT plan modes
    assert lib.qk_batch_schedule(fake, C.c_size_t(1 << 20), 7, 1) == qk.QK_EINVAL
    plan = qk.FwhtPlan(7, 0, 0, 0.0)
    assert lib.qk_fwht_ws(16, C.c_uint64(4), qk.QK_F32, fake, fake, C.c_size_t(1 << 20), C.byref(plan), None,
                          None) == qk.QK_EINVAL
    # the bounded-wait self-test needs a status word
    assert lib.qk_fwht_wait_selftest(16, C.c_uint64(4), qk.QK_F32, fake, fake, C.c_size_t(1 << 20), 10, None,
                                     None) == qk.QK_EINVAL


def test_no_cpu_fallback_in_the_binding():
    """The product binding never imports the oracle and never computes on the host."""
    src = open(os.path.join(ROOT, "paper_2502_14256_gb300", "qk.py")).read()
    assert "oracle" not in src
    assert "numpy" not in src
