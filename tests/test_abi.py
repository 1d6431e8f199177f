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
    text = open(HEADER).read()
    for name in ("QK_MAX_M", "QK_MAX_D"):
        assert int(re.search(rf"#define {name} (\d+)", text).group(1)) == getattr(qk, name)


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


def test_point_set_kernel_and_spectrum_argument_errors(lib_path):
    """Limits include/qk.h states for point sets, kernels and the spectrum: positions below
    2^32, 1 <= d <= QK_MAX_D, randomizations within R, lattices in natural order, matching
    kernel and point-set d, DSI orders 1-4 and SI 1-2, zeta > 0, m <= QK_MAX_M, known column
    forms and families, 256-byte aligned workspaces.  Each returns QK_EINVAL before a launch."""
    from paper_2502_14256_gb300 import qk
    lib = qk.LIB
    fake = C.c_void_p(0x2000000)

    def ps(kind=qk.QK_NET_B2, order=qk.QK_GRAY, d=2, R=2):
        net = kind == qk.QK_NET_B2
        return C.byref(qk.PointSet(kind, order, d, R, fake if net else None, None if net else fake, fake))

    def kern(fam=qk.QK_DSI, alpha=2, d=2, zeta=1.0):
        return C.byref(qk.Kernel(fam, alpha, d, fake, zeta))

    u64 = C.c_uint64
    cases = [
        lib.qk_gen_points(ps(), 0, 1, u64((1 << 32) - 4), u64(8), fake, None),
        lib.qk_gen_points(ps(d=qk.QK_MAX_D + 1), 0, 1, u64(0), u64(8), fake, None),
        lib.qk_gen_points(ps(R=2), 1, 2, u64(0), u64(8), fake, None),
        lib.qk_gen_points(ps(kind=qk.QK_LATTICE, order=qk.QK_GRAY), 0, 1, u64(0), u64(8), fake, None),
        lib.qk_kernel_col(ps(d=2), kern(d=3), 0, 1, 4, qk.QK_F64, 0, fake, None),
        lib.qk_kernel_col(ps(), kern(alpha=5), 0, 1, 4, qk.QK_F64, 0, fake, None),
        lib.qk_kernel_col(ps(kind=qk.QK_LATTICE, order=qk.QK_NATURAL), kern(fam=qk.QK_SI, alpha=3), 0, 1, 4,
                          qk.QK_F64, 0, fake, None),
        lib.qk_kernel_col(ps(), kern(zeta=0.0), 0, 1, 4, qk.QK_F64, 0, fake, None),
        lib.qk_kernel_col(ps(), kern(), 0, 1, qk.QK_MAX_M + 1, qk.QK_F64, 0, fake, None),
        lib.qk_kernel_col(ps(), kern(), 0, 1, 4, qk.QK_F64, 9, fake, None),
        lib.qk_lms_setup(0, 1, fake, fake, fake, None),
        lib.qk_lms_setup(2, 1, None, fake, fake, None),
        lib.qk_eigs(qk.QK_DSI, 4, 1, qk.QK_F64, 0, fake, C.c_double(0.0), C.c_double(0.0), fake, fake,
                    C.c_size_t(1 << 20), None, None),
        lib.qk_eigs(7, 4, 1, qk.QK_F64, 0, fake, C.c_double(1.0), C.c_double(0.0), fake, fake,
                    C.c_size_t(1 << 20), None, None),
        lib.qk_eigs(qk.QK_DSI, 4, 1, qk.QK_F64, 0, fake, C.c_double(1.0), C.c_double(0.0), fake,
                    C.c_void_p(0x2000010), C.c_size_t(1 << 20), None, None),
    ]
    assert cases == [qk.QK_EINVAL] * len(cases), cases


def test_no_cpu_fallback_in_the_binding():
    """The product binding never imports the oracle and never computes on the host."""
    src = open(os.path.join(ROOT, "paper_2502_14256_gb300", "qk.py")).read()
    assert "oracle" not in src
    assert "numpy" not in src


def test_student_t_quantile_host_code_matches_scipy(lib_path):
    """The library's host Student-t quantile (incomplete-beta CDF, bisection) against scipy."""
    scipy_stats = pytest.importorskip("scipy.stats")
    from paper_2502_14256_gb300 import qk
    for df in (1, 2, 3, 5, 9, 14, 30, 63, 1000):
        for p in (0.5, 0.6, 0.9, 0.95, 0.975, 0.995, 0.9995, 0.05, 0.005):
            got = qk.student_t_quantile(df, p)
            want = float(scipy_stats.t.ppf(p, df))
            assert abs(got - want) <= 1e-12 * max(1.0, abs(want)), (df, p, got, want)
    q = C.c_double(0.0)
    assert qk.LIB.qk_student_t_quantile(0.0, 0.9, C.byref(q)) == qk.QK_EINVAL
    assert qk.LIB.qk_student_t_quantile(5.0, 1.0, C.byref(q)) == qk.QK_EINVAL


def test_rqmc_and_discrepancy_argument_errors(lib_path):
    from paper_2502_14256_gb300 import qk
    lib = qk.LIB
    fake = C.c_void_p(0x2000000)
    u64 = C.c_uint64
    net1 = qk.PointSet(qk.QK_NET_B2, qk.QK_GRAY, 3, 1, fake, None, fake)
    cases = [
        lib.qk_integrand(C.byref(net1), 0, 1, u64(0), u64(16), qk.QK_F_SIMPLE1, 0, qk.QK_F64, fake, None),  # d != 1
        lib.qk_integrand(C.byref(net1), 0, 1, u64(0), u64(16), qk.QK_F_OAKLEY, 0, qk.QK_F64, fake, None),   # d != 2
        lib.qk_integrand(C.byref(net1), 0, 1, u64(0), u64(16), 9, 0, qk.QK_F64, fake, None),
        lib.qk_integrand(C.byref(net1), 0, 1, u64((1 << 32) - 4), u64(8), qk.QK_F_GFUN, 0, qk.QK_F64, fake, None),
        lib.qk_rqmc(1, u64(16), qk.QK_F64, fake, C.c_double(0.05), fake, None),
        lib.qk_rqmc(4, u64(16), qk.QK_F64, fake, C.c_double(1.5), fake, None),
        lib.qk_discrepancy(qk.QK_DSI, 4, 1, qk.QK_F64, 7, fake, C.c_double(1.0), fake, None),
        lib.qk_discrepancy(qk.QK_DSI, 4, 1, qk.QK_F64, qk.QK_COL_P, fake, C.c_double(0.0), fake, None),
    ]
    assert cases == [qk.QK_EINVAL] * len(cases), cases
    assert lib.qk_discrepancy_weights(qk.QK_SI, 10, 2, 3, qk.QK_F64, fake, fake, C.c_double(1.0), fake, None,
                                      C.c_size_t(0), None) == qk.QK_EWORKSPACE


def test_workspace_sizes_saturate_instead_of_wrapping(lib_path):
    """batch 2^30 of 2^30-point lattice columns in FP64 (16-byte complex elements) needs 2^64
    bytes: the size saturates, so the static-scratch call refuses it and qk_eigs refuses a NULL
    or small workspace (a wrapped size of 0 would accept it)."""
    from paper_2502_14256_gb300 import qk
    lib = qk.LIB
    fake = C.c_void_p(0x2000000)
    size = C.c_size_t(0)
    assert lib.qk_workspace_bytes(0, qk.QK_SI, 30, 1 << 30, 1, qk.QK_F64, 1, C.byref(size)) == qk.QK_OK
    assert size.value == (1 << 64) - 1
    assert lib.qk_eigs_static(qk.QK_SI, 30, 1 << 30, qk.QK_F64, 0, fake, C.c_double(1.0), C.c_double(0.0), fake,
                              None, None) == qk.QK_EINVAL
    assert lib.qk_eigs(qk.QK_SI, 30, 1 << 30, qk.QK_F64, 0, fake, C.c_double(1.0), C.c_double(0.0), fake, None,
                       C.c_size_t(0), None, None) == qk.QK_EWORKSPACE
    assert lib.qk_eigs(qk.QK_SI, 30, 1 << 30, qk.QK_F64, 0, fake, C.c_double(1.0), C.c_double(0.0), fake, fake,
                       C.c_size_t(1 << 40), None, None) == qk.QK_EWORKSPACE


def test_persistent_schedule_takes_a_subset_of_the_plan(lib_path):
    """Host side of QK_SCHED_PERSISTENT on mixed plans: the persistent launch takes the fused
    DSI nets of one order, so a plan of a lattice and a net outside the fused size range has
    none (QK_EINVAL, nothing launched) and reserves no persistent region, while adding one
    fused net reserves it.  Plans are recorded on a fake workspace: nothing touches it."""
    from paper_2502_14256_gb300 import qk
    lib = qk.LIB
    fake = C.c_void_p(0x2000000)
    ws = C.c_void_p(0x40000000)  # 256-byte aligned, never dereferenced by plan or refusal

    def net(m, alpha=2):
        ps = qk.PointSet(qk.QK_NET_B2, qk.QK_GRAY, 2, 2, fake, None, fake)
        return qk.Task(ps, qk.Kernel(qk.QK_DSI, alpha, 2, fake, 1.0), m, 1, 1e-8, fake, fake, None, fake, fake)

    def lattice(m):
        ps = qk.PointSet(qk.QK_LATTICE, qk.QK_NATURAL, 2, 2, None, fake, fake)
        return qk.Task(ps, qk.Kernel(qk.QK_SI, 1, 2, fake, 1.0), m, 1, 1e-8, fake, fake, None, fake, fake)

    def bytes_of(tasks):
        arr = (qk.Task * len(tasks))(*tasks)
        out = C.c_size_t(0)
        assert lib.qk_batch_workspace_bytes(arr, len(tasks), qk.QK_F32, C.byref(out)) == qk.QK_OK
        return arr, out.value

    arr, nb = bytes_of([lattice(14), net(12)])
    assert lib.qk_batch_plan(arr, 2, qk.QK_F32, 1, ws, C.c_size_t(nb), None) == qk.QK_OK
    assert lib.qk_batch_schedule(ws, C.c_size_t(nb), qk.QK_SCHED_PERSISTENT, 1) == qk.QK_EINVAL
    assert "fused DSI net" in qk.last_error()
    assert lib.qk_batch_schedule(ws, C.c_size_t(nb), qk.QK_SCHED_LAUNCHES, 0) == qk.QK_OK
    _, nb_fused = bytes_of([lattice(14), net(12), net(16)])
    assert nb_fused > nb
