"""Thin Python binding of libqk.so (include/qk.h), by ctypes.

Each function takes torch tensors that live on the GPU, passes their raw
device pointers and sizes to the C entry point of the same name, and raises
QKError on a non-zero status.  Nothing here computes: every step of the path
runs in the library's CUDA kernels.  The library must have been built
(``python -m paper_2502_14256_gb300.build``); importing this module without
it raises immediately instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libqk.so")

QK_OK, QK_EINVAL, QK_ENOTPD, QK_ECUDA, QK_ETIMEOUT, QK_EWORKSPACE = range(6)
QK_STATUS_NOTPD, QK_STATUS_TIMEOUT, QK_STATUS_FLOOR = 1, 2, 4
QK_NET_B2, QK_LATTICE = 0, 1
QK_NATURAL, QK_GRAY = 0, 1
QK_DSI, QK_SI = 0, 1
QK_F64, QK_F32, QK_F32W = 0, 1, 2
# Precision name for QK_F32W (FP32 data, float-float first column): pass it where a torch
# dtype names the schedule's precision (batch_workspace_bytes, batch_plan; kernel_col(wide=True)).
F32W = "float32w"
QK_COL_K1, QK_COL_P = 0, 1
QK_MLL_QUAD, QK_MLL_LOGDET, QK_MLL_MLL, QK_MLL_MEAN, QK_MLL_VAR, QK_MLL_NOUT = range(6)
OP_EIGS, OP_SOLVE, OP_MATVEC, OP_MLL, OP_FWHT, OP_DISCREPANCY = 0, 1, 2, 3, 4, 5
QK_FWHT_TWO_PASS, QK_FWHT_PERSISTENT = 0, 1
QK_SCHED_LAUNCHES, QK_SCHED_PERSISTENT = 0, 1
QK_MAX_M, QK_MAX_D = 30, 256

EXPORTED = ["qk_lms_setup", "qk_gen_points", "qk_kernel_col", "qk_eigs", "qk_solve", "qk_matvec", "qk_mll",
            "qk_batch_workspace_bytes", "qk_batch_plan", "qk_batch_run", "qk_workspace_bytes",
            "qk_read_status", "qk_last_error", "qk_version", "qk_fwht", "qk_fftbr", "qk_ifftbr",
            "qk_launch_count", "qk_eigs_static", "qk_batch_timing", "qk_batch_kernel_ms", "qk_fwht_ws",
            "qk_fwht_tune", "qk_fwht_wait_selftest", "qk_batch_run_host", "qk_batch_schedule",
            "qk_kernel_col_at", "qk_eigs_extend", "qk_fwht_extend", "qk_fftbr_extend", "qk_batch_tune",
            "qk_integrand", "qk_rqmc", "qk_student_t_quantile", "qk_discrepancy", "qk_discrepancy_weights",
            "qk_interlace", "qk_gen_points_ho", "qk_kernel_col_ho", "qk_mll_spectrum", "qk_mll_ho",
            "qk_fftbr_ws", "qk_ratio_selftest"]
QK_F_SIMPLE1, QK_F_SIMPLE2, QK_F_OAKLEY, QK_F_GFUN, QK_F_GENZ_OSC, QK_F_GENZ_CP = range(6)
INTEGRANDS = {"simple1": QK_F_SIMPLE1, "simple2": QK_F_SIMPLE2, "oakley": QK_F_OAKLEY, "gfun": QK_F_GFUN,
              "genz_osc": QK_F_GENZ_OSC, "genz_cp": QK_F_GENZ_CP}


class QKError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libqk status {code}: {msg}")
        self.code = code


class PointSet(C.Structure):
    _fields_ = [("kind", C.c_int32), ("order", C.c_int32), ("d", C.c_uint32), ("R", C.c_uint32),
                ("Ct", C.c_void_p), ("g", C.c_void_p), ("D", C.c_void_p)]


class Kernel(C.Structure):
    _fields_ = [("family", C.c_int32), ("alpha", C.c_int32), ("d", C.c_uint32), ("weights", C.c_void_p),
                ("zeta", C.c_double)]


class HOPointSet(C.Structure):
    _fields_ = [("order", C.c_int32), ("d", C.c_uint32), ("R", C.c_uint32), ("Chat", C.c_void_p), ("D", C.c_void_p)]


class FwhtPlan(C.Structure):
    _fields_ = [("mode", C.c_int32), ("lag", C.c_uint32), ("ctas_per_sm", C.c_uint32), ("ms", C.c_float)]


class HostIO(C.Structure):
    _fields_ = [("y", C.c_void_p), ("c", C.c_void_p), ("lam", C.c_void_p), ("out", C.c_void_p),
                ("grad", C.c_void_p)]


class Task(C.Structure):
    _fields_ = [("ps", PointSet), ("k", Kernel), ("m", C.c_uint32), ("nrhs", C.c_uint32), ("eta", C.c_double),
                ("y", C.c_void_p), ("c", C.c_void_p), ("lam", C.c_void_p), ("out", C.c_void_p),
                ("grad", C.c_void_p)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_2502_14256_gb300.build`")
    lib = C.CDLL(LIB_PATH)
    P, u32, u64, i32, dbl, sz = C.c_void_p, C.c_uint32, C.c_uint64, C.c_int32, C.c_double, C.c_size_t
    sig = {
        "qk_lms_setup": [u32, u32, P, P, P, P],
        "qk_gen_points": [C.POINTER(PointSet), u32, u32, u64, u64, P, P],
        "qk_kernel_col": [C.POINTER(PointSet), C.POINTER(Kernel), u32, u32, u32, i32, i32, P, P],
        "qk_eigs": [i32, u32, u32, i32, i32, P, dbl, dbl, P, P, sz, P, P],
        "qk_solve": [i32, u32, u32, u32, i32, P, P, P, i32, P, sz, P],
        "qk_matvec": [i32, u32, u32, u32, i32, P, P, P, P, sz, P],
        "qk_mll": [C.POINTER(PointSet), C.POINTER(Kernel), u32, u32, u32, u32, i32, dbl, P, P, P, P, P, sz, P, P],
        "qk_batch_workspace_bytes": [C.POINTER(Task), u32, i32, C.POINTER(sz)],
        "qk_batch_plan": [C.POINTER(Task), u32, i32, i32, P, sz, P],
        "qk_batch_run": [P, sz, P, P],
        "qk_workspace_bytes": [i32, i32, u32, u32, u32, i32, u32, C.POINTER(sz)],
        "qk_read_status": [P, P],
        "qk_last_error": [C.c_char_p, sz],
        "qk_version": [],
        "qk_fwht": [u32, u64, i32, P, P],
        "qk_fftbr": [u32, u64, i32, P, P],
        "qk_ifftbr": [u32, u64, i32, P, P],
        "qk_launch_count": [],
        "qk_eigs_static": [i32, u32, u32, i32, i32, P, dbl, dbl, P, P, P],
        "qk_batch_timing": [P, u32],
        "qk_batch_kernel_ms": [P, u32, C.c_char_p, sz, C.POINTER(u32), C.POINTER(dbl)],
        "qk_fwht_ws": [u32, u64, i32, P, P, sz, C.POINTER(FwhtPlan), P, P],
        "qk_fftbr_ws": [u32, u64, i32, i32, P, P, sz, u32, P, P],
        "qk_ratio_selftest": [P, P, P, u64, P],
        "qk_fwht_tune": [u32, u64, i32, P, P, sz, C.POINTER(FwhtPlan), P],
        "qk_fwht_wait_selftest": [u32, u64, i32, P, P, sz, u32, P, P],
        "qk_batch_run_host": [P, sz, C.POINTER(HostIO), u32, P, P],
        "qk_batch_schedule": [P, sz, i32, u32],
        "qk_batch_tune": [P, sz, C.POINTER(i32), C.POINTER(u32), C.POINTER(C.c_float), P],
        "qk_kernel_col_at": [C.POINTER(PointSet), C.POINTER(Kernel), u32, u32, u64, u32, i32, i32, P, P],
        "qk_eigs_extend": [i32, u32, u32, i32, i32, P, dbl, dbl, P, P, P, sz, P, P],
        "qk_fwht_extend": [u32, u64, i32, P, P, P, P],
        "qk_fftbr_extend": [u32, u64, i32, P, P, P, P],
        "qk_integrand": [C.POINTER(PointSet), u32, u32, u64, u64, i32, i32, i32, P, P],
        "qk_rqmc": [u32, u64, i32, P, dbl, P, P],
        "qk_student_t_quantile": [dbl, dbl, C.POINTER(dbl)],
        "qk_discrepancy": [i32, u32, u32, i32, i32, P, dbl, P, P],
        "qk_discrepancy_weights": [i32, u32, u32, u32, i32, P, P, dbl, P, P, sz, P],
        "qk_interlace": [u32, u32, u32, P, P, P],
        "qk_gen_points_ho": [C.POINTER(HOPointSet), u32, u32, u64, u64, P, P],
        "qk_kernel_col_ho": [C.POINTER(HOPointSet), C.POINTER(Kernel), u32, u32, u32, i32, i32, P, P],
        "qk_mll_spectrum": [i32, u32, u32, u32, i32, dbl, P, P, P, P, sz, P],
        "qk_mll_ho": [C.POINTER(HOPointSet), C.POINTER(Kernel), u32, u32, u32, u32, i32, P, P, P, P, P, sz, P],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = None if name == "qk_last_error" else (C.c_uint64 if name == "qk_launch_count" else C.c_int)
    return lib


LIB = _load()


def last_error() -> str:
    buf = C.create_string_buffer(512)
    LIB.qk_last_error(buf, 512)
    return buf.value.decode(errors="replace")


def _check(rc: int):
    if rc != QK_OK:
        raise QKError(rc, last_error())


def _ptr(t) -> int | None:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("libqk takes device tensors")
    if not t.is_contiguous():
        raise ValueError("libqk takes contiguous tensors")
    return t.data_ptr()


def _stream(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def dtype_code(dt) -> int:
    if isinstance(dt, str):
        if dt == F32W:
            return QK_F32W
        raise ValueError(f"unsupported precision {dt!r}")
    if dt == torch.float64:
        return QK_F64
    if dt == torch.float32:
        return QK_F32
    raise ValueError(f"unsupported dtype {dt}")


def data_dtype(dt) -> torch.dtype:
    """The torch dtype of the y / c arrays of a schedule of precision dt."""
    return torch.float32 if dt == F32W else dt


# --------------------------------------------------------------- structures
def pointset(kind: int, d: int, R: int, Ct=None, g=None, D=None, order: int = QK_GRAY) -> PointSet:
    return PointSet(kind, order if kind == QK_NET_B2 else QK_NATURAL, d, R, _ptr(Ct), _ptr(g), _ptr(D))


def kernel(family: int, alpha: int, weights, zeta: float = 1.0) -> Kernel:
    return Kernel(family, alpha, weights.numel(), _ptr(weights), float(zeta))


# --------------------------------------------------------------- entry points
def lms_setup(C_cols, S_rows, Ct_out, stream=None):
    d = C_cols.shape[0]
    R = S_rows.shape[0]
    _check(LIB.qk_lms_setup(d, R, _ptr(C_cols), _ptr(S_rows), _ptr(Ct_out), _stream(stream)))
    return Ct_out


def gen_points(ps: PointSet, r0: int, nr: int, i0: int, n: int, X, stream=None):
    _check(LIB.qk_gen_points(C.byref(ps), r0, nr, i0, n, _ptr(X), _stream(stream)))
    return X


def _col_code(col, wide: bool) -> int:
    if wide:
        if col.dtype != torch.float64:
            raise ValueError("the float-float column (wide=True) is written as float64")
        return QK_F32W
    return dtype_code(col.dtype)


def kernel_col(ps: PointSet, k: Kernel, r0: int, nr: int, m: int, col, form: int = QK_COL_K1, stream=None,
               wide: bool = False):
    """First column; wide=True computes it in float-float arithmetic (FP32 pipes) into a
    float64 tensor (QK_F32W)."""
    _check(LIB.qk_kernel_col(C.byref(ps), C.byref(k), r0, nr, m, _col_code(col, wide), form, _ptr(col),
                             _stream(stream)))
    return col


def kernel_col_at(ps: PointSet, k: Kernel, r0: int, nr: int, i0: int, m: int, col, form: int = QK_COL_K1,
                  stream=None, wide: bool = False):
    """First-column entries of the 2^m points at positions i0 .. i0 + 2^m - 1."""
    _check(LIB.qk_kernel_col_at(C.byref(ps), C.byref(k), r0, nr, i0, m, _col_code(col, wide), form, _ptr(col),
                                _stream(stream)))
    return col


def eigs_extend(family: int, m: int, col_new, lam_old, lam, zeta: float = 1.0, eta: float = 0.0,
                form: int = QK_COL_K1, ws=None, status=None, stream=None):
    """Eigenvalues of the doubled point set (2^(m+1) points) from those of the first 2^m."""
    batch = col_new.numel() >> m
    if ws is None:
        ws = workspace(workspace_bytes(OP_EIGS, family, m, batch, 1, col_new.dtype), col_new.device)
    _check(LIB.qk_eigs_extend(family, m, batch, dtype_code(col_new.dtype), form, _ptr(col_new), zeta, eta,
                              _ptr(lam_old), _ptr(lam), _ptr(ws), ws.numel(), _ptr(status), _stream(stream)))
    return lam


def fwht_extend(m: int, xt_old, x_new, out, stream=None):
    _check(LIB.qk_fwht_extend(m, _nvec_m(xt_old, m, False), dtype_code(xt_old.dtype), _ptr(xt_old), _ptr(x_new),
                              _ptr(out), _stream(stream)))
    return out


def fftbr_extend(m: int, xt_old, x_new, out, stream=None):
    _check(LIB.qk_fftbr_extend(m, _nvec_m(xt_old, m, True), dtype_code(xt_old.dtype), _ptr(xt_old), _ptr(x_new),
                               _ptr(out), _stream(stream)))
    return out


def workspace_bytes(op: int, family: int, m: int, batch: int, nrhs: int, dtype: torch.dtype, d: int = 0) -> int:
    out = C.c_size_t(0)
    _check(LIB.qk_workspace_bytes(op, family, m, batch, nrhs, dtype_code(dtype), d, C.byref(out)))
    return out.value


def workspace(nbytes: int, device="cuda"):
    """A 256-byte aligned device byte buffer (torch allocations are 512-byte aligned)."""
    return torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device)


def eigs(family: int, m: int, col, lam, zeta: float = 1.0, eta: float = 0.0, form: int = QK_COL_K1,
         ws=None, status=None, stream=None):
    batch = _check_spectrum_args(m, col, lam)
    if ws is None:
        ws = workspace(workspace_bytes(OP_EIGS, family, m, batch, 1, col.dtype), col.device)
    _check(LIB.qk_eigs(family, m, batch, dtype_code(col.dtype), form, _ptr(col), zeta, eta, _ptr(lam), _ptr(ws),
                       ws.numel(), _ptr(status), _stream(stream)))
    return lam


def _check_spectrum_args(m: int, col, lam) -> int:
    """Batch count of a (batch, 2^m) column and its (batch, 2^m) float64 eigenvalue output on
    the current device; ValueError on a mismatch (the C side trusts these sizes)."""
    n = 1 << m
    if col.numel() % n != 0:
        raise ValueError(f"column holds {col.numel()} elements, not a multiple of 2^{m}")
    if lam.dtype != torch.float64 or lam.numel() != col.numel():
        raise ValueError("lam must be a float64 tensor with as many elements as the column")
    dev = torch.cuda.current_device()
    for name, t in (("col", col), ("lam", lam)):
        if not t.is_cuda or t.device.index != dev:
            raise ValueError(f"{name} must live on the current CUDA device (cuda:{dev})")
    return col.numel() // n


def eigs_static(family: int, m: int, col, lam, zeta: float = 1.0, eta: float = 0.0, form: int = QK_COL_K1,
                status=None, stream=None):
    """qk_eigs without a workspace: the library's static device scratch is used
    (for callers that cannot allocate; see include/qk.h for its size limit)."""
    batch = _check_spectrum_args(m, col, lam)
    _check(LIB.qk_eigs_static(family, m, batch, dtype_code(col.dtype), form, _ptr(col), zeta, eta, _ptr(lam),
                              _ptr(status), _stream(stream)))
    return lam


def solve(family: int, m: int, lam, y, c, refine_steps: int = 0, ws=None, stream=None):
    batch = lam.numel() >> m
    nrhs = (y.numel() >> m) // batch
    if ws is None:
        ws = workspace(workspace_bytes(OP_SOLVE, family, m, batch, nrhs, y.dtype), y.device)
    _check(LIB.qk_solve(family, m, batch, nrhs, dtype_code(y.dtype), _ptr(lam), _ptr(y), _ptr(c), refine_steps,
                        _ptr(ws), ws.numel(), _stream(stream)))
    return c


def matvec(family: int, m: int, lam, y, u, ws=None, stream=None):
    batch = lam.numel() >> m
    nrhs = (y.numel() >> m) // batch
    if ws is None:
        ws = workspace(workspace_bytes(OP_MATVEC, family, m, batch, nrhs, y.dtype), y.device)
    _check(LIB.qk_matvec(family, m, batch, nrhs, dtype_code(y.dtype), _ptr(lam), _ptr(y), _ptr(u), _ptr(ws),
                         ws.numel(), _stream(stream)))
    return u


def mll(ps: PointSet, k: Kernel, r0: int, nr: int, m: int, nrhs: int, eta: float, lam, y, out, grad=None,
        ws=None, status=None, stream=None):
    if ws is None:
        ws = workspace(workspace_bytes(OP_MLL, k.family, m, nr, nrhs, y.dtype, ps.d), y.device)
    _check(LIB.qk_mll(C.byref(ps), C.byref(k), r0, nr, m, nrhs, dtype_code(y.dtype), eta, _ptr(lam), _ptr(y),
                      _ptr(out), _ptr(grad), _ptr(ws), ws.numel(), _ptr(status), _stream(stream)))
    return out


def read_status(status, stream=None):
    _check(LIB.qk_read_status(_ptr(status), _stream(stream)))


def version() -> int:
    return LIB.qk_version()


def launch_count() -> int:
    return LIB.qk_launch_count()


def _nvec_m(x, m, complex_data):
    per = (2 << m) if complex_data else (1 << m)
    return x.numel() // per


def fwht(m: int, x, stream=None):
    """x <- H x / sqrt(n) in place over the last axis (length 2^m)."""
    _check(LIB.qk_fwht(m, _nvec_m(x, m, False), dtype_code(x.dtype), _ptr(x), _stream(stream)))
    return x


def fftbr(m: int, x, stream=None):
    """In place; x holds interleaved (re, im) pairs, natural-order input."""
    _check(LIB.qk_fftbr(m, _nvec_m(x, m, True), dtype_code(x.dtype), _ptr(x), _stream(stream)))
    return x


def ifftbr(m: int, x, stream=None):
    _check(LIB.qk_ifftbr(m, _nvec_m(x, m, True), dtype_code(x.dtype), _ptr(x), _stream(stream)))
    return x


def fwht_workspace(nvec: int, device="cuda"):
    return workspace(workspace_bytes(OP_FWHT, QK_DSI, 0, nvec, 1, torch.float32), device)


def fwht_ws(m: int, x, ws=None, plan=None, status=None, stream=None):
    """qk_fwht with a workspace: the tuned (or the given) two-pass or persistent single-launch
    form; plan = dict(mode=QK_FWHT_*, lag=.., ctas_per_sm=..) pins one."""
    nvec = _nvec_m(x, m, False)
    if ws is None:
        ws = fwht_workspace(nvec, x.device)
    pp = None
    if plan is not None:
        pp = C.byref(FwhtPlan(plan["mode"], plan.get("lag", 0), plan.get("ctas_per_sm", 0), 0.0))
    _check(LIB.qk_fwht_ws(m, nvec, dtype_code(x.dtype), _ptr(x), _ptr(ws), ws.numel(), pp, _ptr(status),
                          _stream(stream)))
    return x


def fftbr_ws(m: int, x, inverse=False, ws=None, lag=0, status=None, stream=None):
    """qk_fftbr (or qk_ifftbr) with a workspace: one persistent launch for FP32 and
    16 <= m <= 20 (the same results bit for bit), the plain transform otherwise."""
    nvec = _nvec_m(x, m, True)
    if ws is None:
        ws = fwht_workspace(nvec, x.device)
    _check(LIB.qk_fftbr_ws(m, nvec, dtype_code(x.dtype), 1 if inverse else 0, _ptr(x), _ptr(ws), ws.numel(),
                           lag, _ptr(status), _stream(stream)))
    return x


def ratio_selftest(a, b, stream=None):
    """q = a / b as the FP64 gradient sweeps form it (test support); a, b: FP64 device tensors."""
    if a.dtype != torch.float64 or b.dtype != torch.float64 or a.shape != b.shape:
        raise ValueError("ratio_selftest needs two FP64 tensors of one shape")
    a, b = a.contiguous(), b.contiguous()
    q = torch.empty_like(a)
    _check(LIB.qk_ratio_selftest(_ptr(a), _ptr(b), _ptr(q), a.numel(), _stream(stream)))
    return q


def fwht_tune(m: int, x, ws=None, stream=None) -> dict:
    """Autotune qk_fwht_ws for x's shape (x is overwritten); returns the chosen plan."""
    nvec = _nvec_m(x, m, False)
    if ws is None:
        ws = fwht_workspace(nvec, x.device)
    plan = FwhtPlan()
    _check(LIB.qk_fwht_tune(m, nvec, dtype_code(x.dtype), _ptr(x), _ptr(ws), ws.numel(), C.byref(plan),
                            _stream(stream)))
    return {"mode": "persistent" if plan.mode == QK_FWHT_PERSISTENT else "two_pass", "lag": plan.lag,
            "ctas_per_sm": plan.ctas_per_sm, "ms": plan.ms}


def fwht_wait_selftest(m: int, x, spin_limit: int, status, ws=None, stream=None):
    nvec = _nvec_m(x, m, False)
    if ws is None:
        ws = fwht_workspace(nvec, x.device)
    _check(LIB.qk_fwht_wait_selftest(m, nvec, dtype_code(x.dtype), _ptr(x), _ptr(ws), ws.numel(), spin_limit,
                                     _ptr(status), _stream(stream)))


# ------------------------------------------------------------------ batching
def task_array(tasks):
    arr = (Task * len(tasks))(*tasks)
    return arr


def batch_workspace_bytes(tasks, dtype: torch.dtype) -> int:
    arr = task_array(tasks)
    out = C.c_size_t(0)
    _check(LIB.qk_batch_workspace_bytes(arr, len(tasks), dtype_code(dtype), C.byref(out)))
    return out.value


def batch_plan(tasks, dtype: torch.dtype, refine_steps: int, ws, stream=None):
    arr = task_array(tasks)
    _check(LIB.qk_batch_plan(arr, len(tasks), dtype_code(dtype), refine_steps, _ptr(ws), ws.numel(),
                             _stream(stream)))


def batch_run(ws, status=None, stream=None):
    _check(LIB.qk_batch_run(_ptr(ws), ws.numel(), _ptr(status), _stream(stream)))


def batch_schedule(ws, mode: int, lag: int = 0):
    """Choose how batch_run executes the recorded plan (QK_SCHED_LAUNCHES / QK_SCHED_PERSISTENT)."""
    _check(LIB.qk_batch_schedule(_ptr(ws), ws.numel(), mode, lag))


def batch_tune(ws, stream=None) -> dict:
    """Time the launch sequence and the persistent launch (each lag) of the recorded plan and
    keep the fastest; returns {"mode": ..., "lag": ..., "ms": ...}."""
    mode, lag, ms = C.c_int32(0), C.c_uint32(0), C.c_float(0.0)
    _check(LIB.qk_batch_tune(_ptr(ws), ws.numel(), C.byref(mode), C.byref(lag), C.byref(ms), _stream(stream)))
    return {"mode": "persistent" if mode.value == QK_SCHED_PERSISTENT else "launches", "lag": lag.value,
            "ms": ms.value}


def batch_run_host(ws, host_io, chunk_r: int, status=None, stream=None):
    """Run the planned schedule from host tensors: host_io is a list (one per task) of dicts
    with CPU tensors y (required), out (required), c, lam, grad (optional); copies in and out
    overlap the compute chunk by chunk (pinned tensors for overlap)."""
    arr = (HostIO * len(host_io))()
    for i, h in enumerate(host_io):
        arr[i] = HostIO(*[h[k].data_ptr() if h.get(k) is not None else None for k in ("y", "c", "lam", "out", "grad")])
    _check(LIB.qk_batch_run_host(_ptr(ws), ws.numel(), arr, chunk_r, _ptr(status), _stream(stream)))


def batch_timing(ws, runs: int):
    """Record CUDA events around each kernel of the next `runs` batch_run calls."""
    _check(LIB.qk_batch_timing(_ptr(ws), runs))


def batch_kernel_ms(ws):
    """{kernel name: (launches, summed ms)} of the recorded runs."""
    out, idx = {}, 0
    while True:
        name = C.create_string_buffer(64)
        cnt = C.c_uint32(0)
        ms = C.c_double(0.0)
        rc = LIB.qk_batch_kernel_ms(_ptr(ws), idx, name, 64, C.byref(cnt), C.byref(ms))
        if rc != QK_OK:
            break
        out[name.value.decode()] = (cnt.value, ms.value)
        idx += 1
    return out


# ------------------------------------------------------------- RQMC integration
def integrand(ps: PointSet, r0: int, nr: int, i0: int, n: int, f, y, baker: bool = False, stream=None):
    """y (nr, n) <- f at the points (f: a name of INTEGRANDS or its QK_F_* code)."""
    code = INTEGRANDS[f] if isinstance(f, str) else int(f)
    _check(LIB.qk_integrand(C.byref(ps), r0, nr, i0, n, code, 1 if baker else 0, dtype_code(y.dtype), _ptr(y),
                            _stream(stream)))
    return y


def rqmc(y, tau: float, out=None, stream=None):
    """RQMC estimate of y (R, n): device doubles [mu, sigma, half width, t, mu_1 .. mu_R]."""
    R, n = y.shape
    if out is None:
        out = torch.empty(4 + R, dtype=torch.float64, device=y.device)
    _check(LIB.qk_rqmc(R, n, dtype_code(y.dtype), _ptr(y), float(tau), _ptr(out), _stream(stream)))
    return out


def student_t_quantile(df: float, p: float) -> float:
    q = C.c_double(0.0)
    _check(LIB.qk_student_t_quantile(float(df), float(p), C.byref(q)))
    return q.value


def discrepancy(family: int, m: int, col, zeta: float = 1.0, form: int = QK_COL_P, out=None, stream=None):
    """Squared worst-case error for equal and optimal weights from first columns (batch, 2^m):
    (batch, 3) doubles [equal, optimal, optimal weight]."""
    batch = col.numel() >> m
    if col.numel() != batch << m:
        raise ValueError(f"column holds {col.numel()} elements, not a multiple of 2^{m}")
    if out is None:
        out = torch.empty((batch, 3), dtype=torch.float64, device=col.device)
    _check(LIB.qk_discrepancy(family, m, batch, dtype_code(col.dtype), form, _ptr(col), float(zeta), _ptr(out),
                              _stream(stream)))
    return out


def discrepancy_weights(family: int, m: int, lam, w, zeta: float = 1.0, out=None, ws=None, stream=None):
    """Squared worst-case error of weights w (batch, nw, 2^m) given eigenvalues lam (batch, 2^m)."""
    batch = lam.numel() >> m
    nw = (w.numel() >> m) // batch
    if out is None:
        out = torch.empty((batch, nw), dtype=torch.float64, device=w.device)
    if ws is None:
        ws = workspace(workspace_bytes(OP_DISCREPANCY, family, m, batch, nw, w.dtype), w.device)
    _check(LIB.qk_discrepancy_weights(family, m, batch, nw, dtype_code(w.dtype), _ptr(lam), _ptr(w), float(zeta),
                                      _ptr(out), _ptr(ws), ws.numel(), _stream(stream)))
    return out


# ------------------------------------------------------------ higher-order nets
def interlace(alpha: int, Ct, Chat, stream=None):
    """Chat (R, d, 32) int64 <- interlacing of order alpha of Ct (R, alpha d, 32) int32."""
    R, ad = Ct.shape[0], Ct.shape[1]
    if ad % alpha != 0:
        raise ValueError("Ct holds alpha d matrices per randomization")
    _check(LIB.qk_interlace(ad // alpha, R, alpha, _ptr(Ct), _ptr(Chat), _stream(stream)))
    return Chat


def ho_pointset(d: int, R: int, Chat, D=None, order: int = QK_GRAY) -> HOPointSet:
    return HOPointSet(order, d, R, _ptr(Chat), _ptr(D))


def gen_points_ho(ps: HOPointSet, r0: int, nr: int, i0: int, n: int, X, stream=None):
    _check(LIB.qk_gen_points_ho(C.byref(ps), r0, nr, i0, n, _ptr(X), _stream(stream)))
    return X


def kernel_col_ho(ps: HOPointSet, k: Kernel, r0: int, nr: int, m: int, col, form: int = QK_COL_K1, stream=None):
    _check(LIB.qk_kernel_col_ho(C.byref(ps), C.byref(k), r0, nr, m, dtype_code(col.dtype), form, _ptr(col),
                                _stream(stream)))
    return col


def mll_spectrum(family: int, m: int, lam, y, out, zeta: float = 1.0, ws=None, stream=None):
    """MLL pieces from eigenvalues lam (nr, 2^m) and y (nr, nrhs, 2^m), without a point set."""
    nr = lam.numel() >> m
    nrhs = (y.numel() >> m) // nr
    if ws is None:
        ws = workspace(workspace_bytes(OP_MLL, family, m, nr, nrhs, y.dtype, 0), y.device)
    _check(LIB.qk_mll_spectrum(family, m, nr, nrhs, dtype_code(y.dtype), float(zeta), _ptr(lam), _ptr(y), _ptr(out),
                               _ptr(ws), ws.numel(), _stream(stream)))
    return out


def mll_ho(ps: HOPointSet, k: Kernel, r0: int, nr: int, m: int, nrhs: int, lam, y, out, grad=None, ws=None,
           stream=None):
    """qk_mll for a higher-order net (MLL pieces and, with grad, the gradient block)."""
    if ws is None:
        ws = workspace(workspace_bytes(OP_MLL, QK_DSI, m, nr, nrhs, y.dtype, ps.d), y.device)
    _check(LIB.qk_mll_ho(C.byref(ps), C.byref(k), r0, nr, m, nrhs, dtype_code(y.dtype), _ptr(lam), _ptr(y), _ptr(out),
                         _ptr(grad), _ptr(ws), ws.numel(), _stream(stream)))
    return out
