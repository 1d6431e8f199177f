// extern "C" entry points of libqk.so (declared in include/qk.h): argument
// validation on the host, then dispatch to the launchers.  No entry point
// allocates device memory or synchronises, except qk_batch_plan (a host ->
// device copy of the work list) and qk_read_status (reads the status word).
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "qk_common.cuh"
#include "qk_internal.h"

namespace qk {

static thread_local char g_err[512];
static std::atomic<uint64_t> g_launches{0};

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

int sm_count() {
  constexpr int kMaxDev = 64;
  static std::atomic<int> cache[kMaxDev];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) dev = 0;
  int v = cache[dev].load(std::memory_order_relaxed);
  if (v <= 0) {
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 1;
    cache[dev].store(v, std::memory_order_relaxed);
  }
  return v;
}

void set_error(const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

int fail(int code, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

int cuda_fail(cudaError_t e, const char *what) {
  set_error("%s: CUDA error %d (%s)", what, (int)e, cudaGetErrorString(e));
  return QK_ECUDA;
}

static int check_dtype(int32_t dtype) {
  return (dtype == QK_F64 || dtype == QK_F32) ? QK_OK : fail(QK_EINVAL, "dtype must be QK_F64 or QK_F32");
}
// Column entry points also take QK_F32W (float-float arithmetic, FP64 output).
static int check_col_dtype(int32_t dtype) {
  return (dtype == QK_F64 || dtype == QK_F32 || dtype == QK_F32W)
             ? QK_OK
             : fail(QK_EINVAL, "dtype must be QK_F64, QK_F32 or QK_F32W");
}
static int check_family(int32_t family) {
  return (family == QK_DSI || family == QK_SI) ? QK_OK : fail(QK_EINVAL, "family must be QK_DSI or QK_SI");
}
static int check_m(uint32_t m) {
  return m <= QK_MAX_M ? QK_OK : fail(QK_EINVAL, "m = %u exceeds QK_MAX_M = %d", m, QK_MAX_M);
}
int check_ws(const void *ws, size_t have, size_t need) {
  if (need == 0) return QK_OK;
  if (!ws) return fail(QK_EWORKSPACE, "workspace is NULL (%zu bytes needed)", need);
  if (have < need) return fail(QK_EWORKSPACE, "workspace has %zu bytes, %zu needed", have, need);
  if (((uintptr_t)ws & 255u) != 0) return fail(QK_EINVAL, "workspace must be 256-byte aligned");
  return QK_OK;
}

int check_pointset(const qk_pointset *ps, uint32_t r0, uint32_t nr) {
  if (!ps) return fail(QK_EINVAL, "point set is NULL");
  if (ps->d < 1 || ps->d > QK_MAX_D) return fail(QK_EINVAL, "d = %u outside 1..%d", ps->d, QK_MAX_D);
  if ((uint64_t)r0 + nr > ps->R) return fail(QK_EINVAL, "randomizations %u..%u exceed R = %u", r0, r0 + nr, ps->R);
  if (ps->kind == QK_NET_B2) {
    if (!ps->Ct) return fail(QK_EINVAL, "net point set without scrambled columns Ct");
    if (ps->order != QK_NATURAL && ps->order != QK_GRAY) return fail(QK_EINVAL, "order must be natural or Gray");
  } else if (ps->kind == QK_LATTICE) {
    if (!ps->g) return fail(QK_EINVAL, "lattice point set without generating vector g");
    if (ps->order != QK_NATURAL) return fail(QK_EINVAL, "lattices are generated in natural order");
  } else {
    return fail(QK_EINVAL, "unknown point-set kind %d", ps->kind);
  }
  return QK_OK;
}

int check_kernel(const qk_kernel *k, const qk_pointset *ps) {
  if (!k) return fail(QK_EINVAL, "kernel is NULL");
  if (check_family(k->family)) return QK_EINVAL;
  if (k->d != ps->d) return fail(QK_EINVAL, "kernel d = %u differs from point-set d = %u", k->d, ps->d);
  if (!k->weights) return fail(QK_EINVAL, "kernel weights are NULL");
  if (!(k->zeta > 0.0)) return fail(QK_EINVAL, "zeta must be > 0");
  if (k->family == QK_DSI) {
    if (ps->kind != QK_NET_B2) return fail(QK_EINVAL, "DSI kernels pair with digital nets (Sec. 5.3)");
    if (k->alpha < 1 || k->alpha > 4) return fail(QK_EINVAL, "DSI order must be 1..4");
  } else {
    if (ps->kind != QK_LATTICE) return fail(QK_EINVAL, "SI kernels pair with lattices (Sec. 5.2)");
    if (k->alpha < 1 || k->alpha > 2) return fail(QK_EINVAL, "SI smoothness must be 1 or 2");
  }
  return QK_OK;
}

ColJob make_job(const qk_pointset *ps, const qk_kernel *k, uint32_t r0, uint32_t nr, uint32_t m) {
  ColJob j;
  j.kind = ps->kind;
  j.order = ps->order;
  j.d = ps->d;
  j.m = m;
  j.Ct = ps->kind == QK_NET_B2 ? ps->Ct + (size_t)r0 * ps->d * 32 : nullptr;
  j.g = ps->g;
  j.w = k->weights;
  j.zeta = k->zeta;
  j.family = k->family;
  j.alpha = k->alpha;
  j.nr = nr;
  return j;
}

}  // namespace qk

using namespace qk;

#define QK_TRY(x)        \
  do {                   \
    int rc_ = (x);       \
    if (rc_) return rc_; \
  } while (0)

extern "C" {

int qk_version(void) { return 100; }

uint64_t qk_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

static int transform_entry(int kind, uint32_t m, uint64_t nvec, int32_t dtype, void *x, qk_stream stream) {
  g_err[0] = 0;
  QK_TRY(check_dtype(dtype));
  QK_TRY(check_m(m));
  if (nvec == 0) return QK_OK;
  if (!x) return fail(QK_EINVAL, "transform data is NULL");
  return op_transform(kind, m, nvec, dtype, x, (cudaStream_t)stream);
}

int qk_fwht(uint32_t m, uint64_t nvec, int32_t dtype, void *x, qk_stream stream) {
  return transform_entry(0, m, nvec, dtype, x, stream);
}
int qk_fftbr(uint32_t m, uint64_t nvec, int32_t dtype, void *x, qk_stream stream) {
  return transform_entry(1, m, nvec, dtype, x, stream);
}
int qk_ifftbr(uint32_t m, uint64_t nvec, int32_t dtype, void *x, qk_stream stream) {
  return transform_entry(2, m, nvec, dtype, x, stream);
}

void qk_last_error(char *buf, size_t len) {
  if (!buf || len == 0) return;
  strncpy(buf, g_err, len - 1);
  buf[len - 1] = 0;
}

int qk_lms_setup(uint32_t d, uint32_t R, const uint32_t *C, const uint32_t *S, uint32_t *Ct, qk_stream stream) {
  g_err[0] = 0;
  if (d < 1 || d > QK_MAX_D) return fail(QK_EINVAL, "d = %u outside 1..%d", d, QK_MAX_D);
  if (!C || !S || !Ct) return fail(QK_EINVAL, "qk_lms_setup: NULL array");
  return launch_lms(d, R, C, S, Ct, (cudaStream_t)stream);
}

int qk_gen_points(const qk_pointset *ps, uint32_t r0, uint32_t nr, uint64_t i0, uint64_t n, uint32_t *X,
                  qk_stream stream) {
  g_err[0] = 0;
  QK_TRY(check_pointset(ps, r0, nr));
  if (!X && n && nr) return fail(QK_EINVAL, "qk_gen_points: X is NULL");
  if (i0 + n > (1ull << 32)) return fail(QK_EINVAL, "positions beyond 2^32");
  return launch_gen_points(ps, r0, nr, i0, n, X, (cudaStream_t)stream);
}

int qk_kernel_col(const qk_pointset *ps, const qk_kernel *k, uint32_t r0, uint32_t nr, uint32_t m, int32_t dtype,
                  int32_t form, void *col, qk_stream stream) {
  g_err[0] = 0;
  QK_TRY(check_pointset(ps, r0, nr));
  QK_TRY(check_kernel(k, ps));
  QK_TRY(check_col_dtype(dtype));
  QK_TRY(check_m(m));
  if (form != QK_COL_K1 && form != QK_COL_P) return fail(QK_EINVAL, "form must be QK_COL_K1 or QK_COL_P");
  if (!col && nr) return fail(QK_EINVAL, "qk_kernel_col: output is NULL");
  return launch_kernel_col(make_job(ps, k, r0, nr, m), dtype, form, col, (cudaStream_t)stream);
}

int qk_kernel_col_at(const qk_pointset *ps, const qk_kernel *k, uint32_t r0, uint32_t nr, uint64_t i0, uint32_t m,
                     int32_t dtype, int32_t form, void *col, qk_stream stream) {
  g_err[0] = 0;
  QK_TRY(check_pointset(ps, r0, nr));
  QK_TRY(check_kernel(k, ps));
  QK_TRY(check_col_dtype(dtype));
  QK_TRY(check_m(m));
  if (form != QK_COL_K1 && form != QK_COL_P) return fail(QK_EINVAL, "form must be QK_COL_K1 or QK_COL_P");
  if (i0 % 2048 != 0) return fail(QK_EINVAL, "qk_kernel_col_at: i0 = %llu is not a multiple of 2048", (unsigned long long)i0);
  if (i0 + (1ull << m) > (1ull << 32)) return fail(QK_EINVAL, "qk_kernel_col_at: positions beyond 2^32");
  if (!col && nr) return fail(QK_EINVAL, "qk_kernel_col_at: output is NULL");
  ColJob job = make_job(ps, k, r0, nr, m);
  job.i0 = i0;
  return launch_kernel_col(job, dtype, form, col, (cudaStream_t)stream);
}

int qk_eigs_extend(int32_t family, uint32_t m, uint32_t batch, int32_t dtype, int32_t form, const void *col_new,
                   double zeta, double eta, const double *lam_old, double *lam, void *ws, size_t ws_bytes,
                   uint32_t *status, qk_stream stream) {
  g_err[0] = 0;
  QK_TRY(check_family(family));
  QK_TRY(check_dtype(dtype));
  QK_TRY(check_m(m));
  if (m + 1 > QK_MAX_M) return fail(QK_EINVAL, "qk_eigs_extend: 2^(m+1) exceeds 2^%d", QK_MAX_M);
  if (form != QK_COL_K1 && form != QK_COL_P) return fail(QK_EINVAL, "form must be QK_COL_K1 or QK_COL_P");
  if (batch == 0) return QK_OK;
  if (!col_new || !lam_old || !lam) return fail(QK_EINVAL, "qk_eigs_extend: NULL array");
  if (!(zeta > 0.0)) return fail(QK_EINVAL, "zeta must be > 0");
  const uint64_t n = 1ull << m;
  const double *lo = lam_old, *hi = lam_old + (uint64_t)batch * n;
  if (!(lam + ((uint64_t)batch << (m + 1)) <= lo || lam >= hi))
    return fail(QK_EINVAL, "qk_eigs_extend: lam must not overlap lam_old");
  QK_TRY(check_ws(ws, ws_bytes, ws_eigs(family, m, batch, dtype)));
  return op_eigs_extend(family, m, batch, dtype, form, col_new, zeta, eta, lam_old, lam, ws, status,
                        (cudaStream_t)stream);
}

static int transform_extend_entry(int kind, uint32_t m, uint64_t nvec, int32_t dtype, const void *xt_old, void *x_new,
                                  void *out, qk_stream stream) {
  g_err[0] = 0;
  QK_TRY(check_dtype(dtype));
  QK_TRY(check_m(m));
  if (m + 1 > QK_MAX_M) return fail(QK_EINVAL, "2^(m+1) exceeds 2^%d", QK_MAX_M);
  if (nvec == 0) return QK_OK;
  if (!xt_old || !x_new || !out) return fail(QK_EINVAL, "transform extension: NULL array");
  // byte ranges: xt_old and x_new hold nvec x n elements, out nvec x 2n (complex for FFTBR)
  const uint64_t half = elem_bytes(kind == 0 ? QK_DSI : QK_SI, dtype) * (nvec << m);
  auto disjoint = [](const void *a, uint64_t na, const void *b, uint64_t nb) {
    const uintptr_t pa = (uintptr_t)a, pb = (uintptr_t)b;
    return pa + na <= pb || pb + nb <= pa;
  };
  if (!disjoint(out, 2 * half, xt_old, half) || !disjoint(out, 2 * half, x_new, half))
    return fail(QK_EINVAL, "transform extension: out must not overlap xt_old or x_new");
  if (!disjoint(x_new, half, xt_old, half))
    return fail(QK_EINVAL, "transform extension: x_new (transformed in place) must not overlap xt_old");
  return op_transform_extend(kind, m, nvec, dtype, xt_old, x_new, out, (cudaStream_t)stream);
}

int qk_fwht_extend(uint32_t m, uint64_t nvec, int32_t dtype, const void *xt_old, void *x_new, void *out,
                   qk_stream stream) {
  return transform_extend_entry(0, m, nvec, dtype, xt_old, x_new, out, stream);
}

int qk_fftbr_extend(uint32_t m, uint64_t nvec, int32_t dtype, const void *xt_old, void *x_new, void *out,
                    qk_stream stream) {
  return transform_extend_entry(1, m, nvec, dtype, xt_old, x_new, out, stream);
}

int qk_workspace_bytes(int32_t op, int32_t family, uint32_t m, uint32_t batch, uint32_t nrhs, int32_t dtype,
                       uint32_t d, size_t *bytes) {
  g_err[0] = 0;
  QK_TRY(check_family(family));
  QK_TRY(check_dtype(dtype));
  QK_TRY(check_m(m));
  if (!bytes) return fail(QK_EINVAL, "bytes is NULL");
  switch (op) {
    case 0: *bytes = ws_eigs(family, m, batch, dtype); break;
    case 1: *bytes = ws_solve(family, m, batch, nrhs, dtype); break;
    case 2: *bytes = ws_matvec(family, m, batch, nrhs, dtype); break;
    case 3: *bytes = ws_mll(family, m, batch, nrhs, dtype, d); break;
    case 4: *bytes = persist_wht_ws_bytes(batch); break;
    case 5: *bytes = ws_discrepancy(family, m, batch, nrhs, dtype); break;
    default: return fail(QK_EINVAL, "unknown op %d", op);
  }
  return QK_OK;
}

int qk_eigs(int32_t family, uint32_t m, uint32_t batch, int32_t dtype, int32_t form, const void *col, double zeta,
            double eta, double *lam, void *ws, size_t ws_bytes, uint32_t *status, qk_stream stream) {
  g_err[0] = 0;
  QK_TRY(check_family(family));
  QK_TRY(check_dtype(dtype));
  QK_TRY(check_m(m));
  if (form != QK_COL_K1 && form != QK_COL_P) return fail(QK_EINVAL, "form must be QK_COL_K1 or QK_COL_P");
  if (batch == 0) return QK_OK;
  if (!col || !lam) return fail(QK_EINVAL, "qk_eigs: NULL array");
  if (!(zeta > 0.0)) return fail(QK_EINVAL, "zeta must be > 0");
  QK_TRY(check_ws(ws, ws_bytes, ws_eigs(family, m, batch, dtype)));
  return op_eigs(family, m, batch, dtype, form, col, zeta, eta, lam, ws, status, (cudaStream_t)stream);
}

int qk_solve(int32_t family, uint32_t m, uint32_t batch, uint32_t nrhs, int32_t dtype, const double *lam,
             const void *y, void *c, int32_t refine_steps, void *ws, size_t ws_bytes, qk_stream stream) {
  g_err[0] = 0;
  QK_TRY(check_family(family));
  QK_TRY(check_dtype(dtype));
  QK_TRY(check_m(m));
  if (batch == 0 || nrhs == 0) return QK_OK;
  if (!lam || !y || !c) return fail(QK_EINVAL, "qk_solve: NULL array");
  if (refine_steps < 0 || refine_steps > 8) return fail(QK_EINVAL, "refine_steps must be 0..8");
  QK_TRY(check_ws(ws, ws_bytes, ws_solve(family, m, batch, nrhs, dtype)));
  return op_solve(family, m, batch, nrhs, dtype, lam, y, c, refine_steps, ws, (cudaStream_t)stream);
}

int qk_matvec(int32_t family, uint32_t m, uint32_t batch, uint32_t nrhs, int32_t dtype, const double *lam,
              const void *y, void *u, void *ws, size_t ws_bytes, qk_stream stream) {
  g_err[0] = 0;
  QK_TRY(check_family(family));
  QK_TRY(check_dtype(dtype));
  QK_TRY(check_m(m));
  if (batch == 0 || nrhs == 0) return QK_OK;
  if (!lam || !y || !u) return fail(QK_EINVAL, "qk_matvec: NULL array");
  QK_TRY(check_ws(ws, ws_bytes, ws_matvec(family, m, batch, nrhs, dtype)));
  return op_matvec(family, m, batch, nrhs, dtype, lam, y, u, ws, (cudaStream_t)stream);
}

int qk_mll(const qk_pointset *ps, const qk_kernel *k, uint32_t r0, uint32_t nr, uint32_t m, uint32_t nrhs,
           int32_t dtype, double eta, const double *lam, const void *y, double *out, double *grad, void *ws,
           size_t ws_bytes, uint32_t *status, qk_stream stream) {
  g_err[0] = 0;
  (void)eta;
  (void)status;
  QK_TRY(check_pointset(ps, r0, nr));
  QK_TRY(check_kernel(k, ps));
  QK_TRY(check_dtype(dtype));
  QK_TRY(check_m(m));
  if (nr == 0 || nrhs == 0) return QK_OK;
  if (!lam || !y || !out) return fail(QK_EINVAL, "qk_mll: NULL array");
  QK_TRY(check_ws(ws, ws_bytes, ws_mll(k->family, m, nr, nrhs, dtype, ps->d)));
  return op_mll(make_job(ps, k, r0, nr, m), nrhs, dtype, lam, y, out, grad, ws, (cudaStream_t)stream);
}

int qk_read_status(uint32_t *status, qk_stream stream) {
  g_err[0] = 0;
  if (!status) return QK_OK;
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "qk_read_status sync");
  uint32_t h = 0;
  e = cudaMemcpy(&h, status, sizeof(h), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "qk_read_status copy");
  const uint32_t zero = 0;
  e = cudaMemcpy(status, &zero, sizeof(zero), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "qk_read_status clear");
  if (h & QK_STATUS_TIMEOUT) return fail(QK_ETIMEOUT, "a bounded device wait expired");
  if (h & QK_STATUS_NOTPD) return fail(QK_ENOTPD, "an eigenvalue was <= 0: K is not positive definite");
  return QK_OK;
}

}  // extern "C"
