// Batched schedules over many (point set, kernel, randomization, right-hand
// side) tasks of uneven n.  qk_batch_plan validates the host task list, sizes
// the workspace, and records the plan; qk_batch_run issues kernel launches
// only (no allocation, no host synchronisation), so it can be captured into a
// CUDA graph and replayed.
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "qk_common.cuh"
#include "qk_internal.h"

namespace qk {


// Event pairs recorded around launches when timing is on (qk_batch_timing).
struct EventTimer : LaunchTimer {
  struct Rec {
    std::string name;
    cudaEvent_t a = nullptr, b = nullptr;
  };
  std::vector<Rec> recs;
  uint32_t runs_left = 0;
  bool active = false;
  void begin(const char *name, cudaStream_t st) override {
    Rec r;
    r.name = name;
    cudaEventCreate(&r.a);
    cudaEventCreate(&r.b);
    cudaEventRecord(r.a, st);
    recs.push_back(r);
  }
  void end(cudaStream_t st) override { cudaEventRecord(recs.back().b, st); }
  void clear() {
    for (Rec &r : recs) {
      cudaEventDestroy(r.a);
      cudaEventDestroy(r.b);
    }
    recs.clear();
  }
  ~EventTimer() override { clear(); }
};

struct Plan {
  std::vector<qk_task> tasks;
  int32_t dtype = QK_F64;
  int32_t refine = 0;
  size_t scratch = 0;   // bytes of the shared scratch region
  size_t lam_off = 0;   // offset of the eigenvalue buffer
  size_t persist_off = 0, persist_bytes = 0;  // region of the persistent schedule (if eligible)
  std::vector<qk_task> persist_tasks;   // the tasks the persistent launch takes (see persist_subset)
  std::vector<uint8_t> in_persist;      // per task: 1 if it is one of them
  size_t total = 0;
  int32_t mode = QK_SCHED_LAUNCHES;
  PersistState persist;
  std::shared_ptr<EventTimer> timer;
};

constexpr uint32_t kMaxPersistLag = 2;  // the workspace is sized for lags up to this

static std::mutex g_mu;
static std::unordered_map<const void *, Plan> g_plans;

// A task runs fused (qk_fused.cu) when its family and size allow it; otherwise it
// runs as the sequence of standalone ops.
static bool use_fused(const qk_task &t, int dtype, int refine) {
  (void)refine;
  return fused_supported(t, dtype);
}

// Lattice tasks run as column, eigenvalues and one combined MLL + gradient + solve pass on
// pairs of vectors (qk_spectral.cu); an FP32 solve with refinement steps keeps the separate
// refined solve.
static bool use_lattice(const qk_task &t, int dtype, int refine) {
  return t.k.family == QK_SI && (dtype != QK_F32 || refine == 0 || !t.c);
}

static size_t task_scratch(const qk_task &t, int dtype, int refine) {
  if (use_fused(t, dtype, refine)) return fused_ws_bytes(t, dtype, refine);
  const uint32_t R = t.ps.R;
  if (use_lattice(t, dtype, refine)) {
    const size_t col = align256((dtype == QK_F32 ? 4 : 8) * ((uint64_t)R << t.m));
    size_t s = ws_eigs(t.k.family, t.m, R, dtype == QK_F32 ? QK_F32 : QK_F64);
    const size_t mw = ws_mll_si(t.m, R, t.nrhs, dtype, t.ps.d, t.c != nullptr);
    return col + (mw > s ? mw : s);
  }
  if (dtype == QK_F32W) {
    // float-float column stored as FP64, FP64 eigenvalues and spectral sums, FP32 solve
    // with refinement and FP32 gradient sweep
    const size_t col = align256(8 * ((uint64_t)R << t.m));
    size_t s = ws_eigs(t.k.family, t.m, R, QK_F64);
    const size_t mw = ws_mll(t.k.family, t.m, R, t.nrhs, QK_F32W, t.ps.d);
    if (mw > s) s = mw;
    if (t.c) {
      const size_t sw = ws_solve(t.k.family, t.m, R, t.nrhs, QK_F32);
      if (sw > s) s = sw;
    }
    return col + s;
  }
  const size_t tb = dtype == QK_F64 ? 8 : 4;
  const size_t col = align256(tb * ((uint64_t)R << t.m));
  size_t s = ws_eigs(t.k.family, t.m, R, dtype);
  const size_t mw = ws_mll(t.k.family, t.m, R, t.nrhs, dtype, t.ps.d);
  if (mw > s) s = mw;
  if (t.c) {
    const size_t sw = ws_solve(t.k.family, t.m, R, t.nrhs, dtype);
    if (sw > s) s = sw;
  }
  return col + s;
}

// The tasks one persistent launch can take: fused DSI nets of the order of the plan's first
// such task.  The others (lattices, sizes outside the fused range, other orders) run as
// their launch sequence after it.
static void persist_subset(Plan &p) {
  p.persist_tasks.clear();
  p.in_persist.assign(p.tasks.size(), 0);
  int alpha = 0;
  for (size_t i = 0; i < p.tasks.size(); ++i) {
    const qk_task &t = p.tasks[i];
    if (!fused_supported(t, p.dtype)) continue;
    if (!alpha) alpha = t.k.alpha;
    if (t.k.alpha != alpha) continue;
    p.persist_tasks.push_back(t);
    p.in_persist[i] = 1;
  }
}

static int make_plan(const qk_task *tasks, uint32_t ntasks, int32_t dtype, int32_t refine, Plan &p) {
  if (!tasks && ntasks) return fail(QK_EINVAL, "task list is NULL");
  if (dtype != QK_F64 && dtype != QK_F32 && dtype != QK_F32W)
    return fail(QK_EINVAL, "dtype must be QK_F64, QK_F32 or QK_F32W");
  p.tasks.assign(tasks, tasks + ntasks);
  p.dtype = dtype;
  p.refine = refine;
  size_t scratch = 0, lam = 0;
  for (uint32_t i = 0; i < ntasks; ++i) {
    const qk_task &t = tasks[i];
    int rc = check_pointset(&t.ps, 0, t.ps.R);
    if (rc) return fail(rc, "task %u: %s", i, "invalid point set");
    if ((rc = check_kernel(&t.k, &t.ps))) return fail(rc, "task %u: invalid kernel", i);
    if (t.m > QK_MAX_M) return fail(QK_EINVAL, "task %u: m = %u too large", i, t.m);
    if (t.nrhs == 0 || !t.y || !t.out) return fail(QK_EINVAL, "task %u: needs nrhs >= 1, y and out", i);
    const size_t s = task_scratch(t, dtype, refine);
    if (s > scratch) scratch = s;
    if (!t.lam && !use_fused(t, dtype, refine)) {
      const size_t l = align256(sizeof(double) * ((uint64_t)t.ps.R << t.m));
      if (l > lam) lam = l;
    }
  }
  p.scratch = align256(scratch);
  p.lam_off = p.scratch;
  p.total = p.scratch + lam;
  p.persist_off = align256(p.total);
  p.persist_bytes = 0;
  persist_subset(p);
  if (persist_eligible(p.persist_tasks, dtype)) {
    for (uint32_t lag = 1; lag <= kMaxPersistLag; ++lag) {
      const size_t b = persist_ws_bytes(p.persist_tasks, dtype, refine, lag);
      if (b > p.persist_bytes) p.persist_bytes = b;
    }
    p.total = p.persist_off + p.persist_bytes;
  }
  return QK_OK;
}

// Brackets one standalone op of the unfused path when timing is on.
struct OpScope {
  LaunchTimer *tm;
  cudaStream_t st;
  OpScope(LaunchTimer *t, const char *name, cudaStream_t s) : tm(t), st(s) {
    if (tm) tm->begin(name, st);
  }
  ~OpScope() {
    if (tm) tm->end(st);
  }
};

// One task (or a range of its randomizations, see sub_task) through its kernels.
static int run_task(const Plan &p, const qk_task &t, unsigned char *ws, uint32_t *status, cudaStream_t st,
                    LaunchTimer *tm) {
  {
    const uint32_t R = t.ps.R;
    const size_t tb = p.dtype == QK_F32 ? 4 : 8;  // stored column (QK_F32W: FP64 from float-float)
    unsigned char *col = ws;
    unsigned char *scr = ws + align256(tb * ((uint64_t)R << t.m));
    double *lam = t.lam ? t.lam : (double *)(ws + p.lam_off);
    const ColJob job = make_job(&t.ps, &t.k, 0, R, t.m);
    if (use_fused(t, p.dtype, p.refine)) return run_fused(t, job, p.dtype, p.refine, ws, status, st, tm);
    int rc;
    if (use_lattice(t, p.dtype, p.refine)) {
      const int eig_dtype = p.dtype;  // QK_F32W: float-float transforms of the float-float column
      {
        OpScope s(tm, p.dtype == QK_F32W ? "op_kernel_col_ff" : "op_kernel_col", st);
        if ((rc = launch_kernel_col(job, p.dtype, QK_COL_P, col, st))) return rc;
      }
      {
        OpScope s(tm, "op_eigs", st);
        if ((rc = op_eigs(t.k.family, t.m, R, eig_dtype, QK_COL_P, col, t.k.zeta, t.eta, lam, scr, status, st)))
          return rc;
      }
      OpScope s(tm, "op_mll_solve", st);
      // the gradient sweep reads the stored column (FP64 for QK_F64 and QK_F32W)
      const double *pcol = p.dtype == QK_F32 ? nullptr : reinterpret_cast<const double *>(col);
      return op_mll_solve_si(job, t.nrhs, p.dtype, lam, t.y, t.out, t.grad, t.c, scr, st, pcol);
    }
    if (p.dtype == QK_F32W) {
      {
        OpScope s(tm, "op_kernel_col_ff", st);
        if ((rc = launch_kernel_col(job, QK_F32W, QK_COL_P, col, st))) return rc;
      }
      {
        OpScope s(tm, "op_eigs", st);
        if ((rc = op_eigs(t.k.family, t.m, R, QK_F64, QK_COL_P, col, t.k.zeta, t.eta, lam, scr, status, st)))
          return rc;
      }
      {
        OpScope s(tm, "op_mll", st);
        if ((rc = op_mll(job, t.nrhs, QK_F32W, lam, t.y, t.out, t.grad, scr, st))) return rc;
      }
      if (t.c) {
        OpScope s(tm, "op_solve", st);
        const int refine = p.refine > 0 ? p.refine : 1;
        if ((rc = op_solve(t.k.family, t.m, R, t.nrhs, QK_F32, lam, t.y, t.c, refine, scr, st))) return rc;
      }
      return QK_OK;
    }
    {
      OpScope s(tm, "op_kernel_col", st);
      if ((rc = launch_kernel_col(job, p.dtype, QK_COL_P, col, st))) return rc;
    }
    {
      OpScope s(tm, "op_eigs", st);
      if ((rc = op_eigs(t.k.family, t.m, R, p.dtype, QK_COL_P, col, t.k.zeta, t.eta, lam, scr, status, st))) return rc;
    }
    {
      OpScope s(tm, "op_mll", st);
      if ((rc = op_mll(job, t.nrhs, p.dtype, lam, t.y, t.out, t.grad, scr, st))) return rc;
    }
    if (t.c) {
      OpScope s(tm, "op_solve", st);
      if ((rc = op_solve(t.k.family, t.m, R, t.nrhs, p.dtype, lam, t.y, t.c, p.refine, scr, st))) return rc;
    }
  }
  return QK_OK;
}

static int run_plan(const Plan &p, unsigned char *ws, uint32_t *status, cudaStream_t st, LaunchTimer *tm) {
  const bool persistent = p.mode == QK_SCHED_PERSISTENT && p.persist.ok;
  if (persistent) {
    int rc = persist_run(p.persist, status, st, tm);
    if (rc) return rc;
  }
  for (size_t i = 0; i < p.tasks.size(); ++i) {
    if (persistent && p.in_persist[i]) continue;  // done by the persistent launch
    int rc = run_task(p, p.tasks[i], ws, status, st, tm);
    if (rc) return rc;
  }
  return QK_OK;
}

// Randomizations [r0, r0 + nr) of task t as a task of their own (pointers offset).
static qk_task sub_task(const qk_task &t, uint32_t r0, uint32_t nr, size_t elem) {
  qk_task s = t;
  const uint64_t n = 1ull << t.m, d = t.ps.d;
  s.ps.R = nr;
  if (t.ps.Ct) s.ps.Ct = t.ps.Ct + (size_t)r0 * d * 32;
  if (t.ps.D) s.ps.D = t.ps.D + (size_t)r0 * d;
  s.y = (const unsigned char *)t.y + elem * r0 * t.nrhs * n;
  if (t.c) s.c = (unsigned char *)t.c + elem * r0 * t.nrhs * n;
  if (t.lam) s.lam = t.lam + (size_t)r0 * n;
  s.out = t.out + (size_t)r0 * t.nrhs * QK_MLL_NOUT;
  if (t.grad) s.grad = t.grad + (size_t)r0 * t.nrhs * (2 * d + 2);
  return s;
}

// Streams and events of the host-buffer runner, created once per device: copies in, copies
// back, and two compute streams that alternating chunks run on.
struct HostRunner {
  cudaStream_t in = nullptr, out = nullptr, cmp[2] = {nullptr, nullptr};
  std::vector<cudaEvent_t> ev;
  int ensure(size_t nev) {
    if (!in) {
      cudaError_t e = cudaStreamCreateWithFlags(&in, cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&out, cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cmp[0], cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cmp[1], cudaStreamNonBlocking);
      if (e != cudaSuccess) return cuda_fail(e, "qk_batch_run_host: stream creation");
    }
    while (ev.size() < nev) {
      cudaEvent_t x;
      cudaError_t e = cudaEventCreateWithFlags(&x, cudaEventDisableTiming);
      if (e != cudaSuccess) return cuda_fail(e, "qk_batch_run_host: event creation");
      ev.push_back(x);
    }
    return QK_OK;
  }
};
static std::mutex g_host_mu;
static std::unordered_map<int, HostRunner> g_host_runners;

// Chunk sizes (randomizations) for R randomizations with chunks of at most chunk_r: a half
// chunk at both ends (computing starts after a short first copy in, and the last copy back
// is short), chunk_r in between; uniform chunks when R is too small.  A chunk's kernels fill
// whole waves of resident CTAs only for some sizes, so the caller picks chunk_r (bench.py
// times a few).
static std::vector<uint32_t> host_chunks(uint32_t R, uint32_t chunk_r) {
  const uint32_t h = chunk_r / 2;
  std::vector<uint32_t> out;
  if (h == 0 || R < chunk_r + 2 * h) {
    for (uint32_t r0 = 0; r0 < R; r0 += chunk_r) out.push_back(R - r0 < chunk_r ? R - r0 : chunk_r);
    return out;
  }
  out.push_back(h);
  uint32_t mid = R - 2 * h;
  while (mid) {
    const uint32_t c = mid < chunk_r ? mid : chunk_r;
    out.push_back(c);
    mid -= c;
  }
  out.push_back(h);
  return out;
}

}  // namespace qk

using namespace qk;

extern "C" {

int qk_batch_workspace_bytes(const qk_task *tasks, uint32_t ntasks, int32_t dtype, size_t *bytes) {
  if (!bytes) return fail(QK_EINVAL, "bytes is NULL");
  Plan p;
  int rc = make_plan(tasks, ntasks, dtype, 0, p);
  if (rc) return rc;
  Plan pr;  // refinement may need the larger unfused workspace
  if ((rc = make_plan(tasks, ntasks, dtype, 1, pr))) return rc;
  *bytes = p.total > pr.total ? p.total : pr.total;
  return QK_OK;
}

int qk_batch_plan(const qk_task *tasks, uint32_t ntasks, int32_t dtype, int32_t refine_steps, void *ws,
                  size_t ws_bytes, qk_stream stream) {
  (void)stream;
  if (refine_steps < 0 || refine_steps > 8) return fail(QK_EINVAL, "refine_steps must be 0..8");
  Plan p;
  int rc = make_plan(tasks, ntasks, dtype, refine_steps, p);
  if (rc) return rc;
  if (p.total && (!ws || ws_bytes < p.total))
    return fail(QK_EWORKSPACE, "batch workspace has %zu bytes, %zu needed", ws_bytes, p.total);
  if (((uintptr_t)ws & 255u) != 0) return fail(QK_EINVAL, "workspace must be 256-byte aligned");
  std::lock_guard<std::mutex> lk(g_mu);
  g_plans[ws] = std::move(p);
  return QK_OK;
}

int qk_batch_run(void *ws, size_t ws_bytes, uint32_t *status, qk_stream stream) {
  Plan p;
  LaunchTimer *tm = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_plans.find(ws);
    if (it == g_plans.end()) return fail(QK_EINVAL, "no plan recorded for this workspace (call qk_batch_plan)");
    p = it->second;
    if (p.timer && p.timer->runs_left > 0) {
      --p.timer->runs_left;
      tm = p.timer.get();
    }
  }
  if (ws_bytes < p.total) return fail(QK_EWORKSPACE, "batch workspace has %zu bytes, %zu needed", ws_bytes, p.total);
  return run_plan(p, (unsigned char *)ws, status, (cudaStream_t)stream, tm);
}

int qk_batch_schedule(void *ws, size_t ws_bytes, int32_t mode, uint32_t lag) {
  if (mode != QK_SCHED_LAUNCHES && mode != QK_SCHED_PERSISTENT)
    return fail(QK_EINVAL, "mode must be QK_SCHED_LAUNCHES or QK_SCHED_PERSISTENT");
  if (lag > kMaxPersistLag) return fail(QK_EINVAL, "lag must be 0..%u", kMaxPersistLag);
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_plans.find(ws);
  if (it == g_plans.end()) return fail(QK_EINVAL, "no plan recorded for this workspace (call qk_batch_plan)");
  Plan &p = it->second;
  if (ws_bytes < p.total) return fail(QK_EWORKSPACE, "batch workspace has %zu bytes, %zu needed", ws_bytes, p.total);
  if (mode == QK_SCHED_LAUNCHES) {
    p.mode = mode;
    return QK_OK;
  }
  if (!p.persist_bytes)
    return fail(QK_EINVAL, "the persistent schedule needs at least one task that is a fused DSI net");
  PersistState st;
  int rc = persist_setup(p.persist_tasks, p.dtype, p.refine, lag ? lag : 1, (unsigned char *)ws + p.persist_off,
                         p.persist_bytes, st);
  if (rc) return rc;
  p.persist = st;
  p.mode = mode;
  return QK_OK;
}

int qk_batch_tune(void *ws, size_t ws_bytes, int32_t *mode_out, uint32_t *lag_out, float *ms_out, qk_stream stream) {
  cudaStream_t st = (cudaStream_t)stream;
  Plan base;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_plans.find(ws);
    if (it == g_plans.end()) return fail(QK_EINVAL, "no plan recorded for this workspace (call qk_batch_plan)");
    base = it->second;
  }
  if (ws_bytes < base.total) return fail(QK_EWORKSPACE, "batch workspace has %zu bytes, %zu needed", ws_bytes, base.total);
  struct Cand {
    int32_t mode;
    uint32_t lag;
    float ms;
  };
  std::vector<Cand> cand = {{QK_SCHED_LAUNCHES, 0, 0.f}};
  if (base.persist_bytes)
    for (uint32_t lag = 1; lag <= kMaxPersistLag; ++lag) cand.push_back({QK_SCHED_PERSISTENT, lag, 0.f});
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  int rc = QK_OK;
  Cand best{QK_SCHED_LAUNCHES, 0, 1e30f};
  for (Cand &c : cand) {
    if ((rc = qk_batch_schedule(ws, ws_bytes, c.mode, c.lag))) break;
    Plan p;
    {
      std::lock_guard<std::mutex> lk(g_mu);
      p = g_plans[ws];
    }
    if ((rc = run_plan(p, (unsigned char *)ws, nullptr, st, nullptr))) break;  // warm-up
    const int reps = 3;
    cudaEventRecord(a, st);
    for (int r = 0; r < reps && !rc; ++r) rc = run_plan(p, (unsigned char *)ws, nullptr, st, nullptr);
    cudaEventRecord(b, st);
    if (rc) break;
    cudaError_t e = cudaEventSynchronize(b);
    if (e != cudaSuccess) {
      rc = cuda_fail(e, "qk_batch_tune");
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    c.ms = ms / reps;
    if (c.ms < best.ms) best = c;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (rc) return rc;
  if ((rc = qk_batch_schedule(ws, ws_bytes, best.mode, best.lag))) return rc;
  if (mode_out) *mode_out = best.mode;
  if (lag_out) *lag_out = best.lag;
  if (ms_out) *ms_out = best.ms;
  return QK_OK;
}

int qk_batch_run_host(void *ws, size_t ws_bytes, const qk_host_io *io, uint32_t chunk_r, uint32_t *status,
                      qk_stream stream) {
  Plan p;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_plans.find(ws);
    if (it == g_plans.end()) return fail(QK_EINVAL, "no plan recorded for this workspace (call qk_batch_plan)");
    p = it->second;
  }
  if (ws_bytes < p.total) return fail(QK_EWORKSPACE, "batch workspace has %zu bytes, %zu needed", ws_bytes, p.total);
  if (!io && !p.tasks.empty()) return fail(QK_EINVAL, "qk_batch_run_host: io is NULL");
  if (chunk_r == 0) return fail(QK_EINVAL, "qk_batch_run_host: chunk_r must be >= 1");
  const size_t elem = p.dtype == QK_F64 ? 8 : 4;
  size_t nchunks = 0;
  std::vector<std::vector<uint32_t>> chunks(p.tasks.size());
  for (size_t i = 0; i < p.tasks.size(); ++i) {
    const qk_task &t = p.tasks[i];
    if (!io[i].y || !io[i].out) return fail(QK_EINVAL, "task %zu: host y and out are required", i);
    if ((io[i].c && !t.c) || (io[i].lam && !t.lam) || (io[i].grad && !t.grad))
      return fail(QK_EINVAL, "task %zu: a host output whose device buffer was not planned", i);
    chunks[i] = host_chunks(t.ps.R, chunk_r);
    nchunks += chunks[i].size();
  }
  // Two chunks in flight: when every task runs fused and two chunks' scratch fits in front of
  // the workspace's persistent-schedule region, consecutive chunks compute on two library
  // streams, each with its own scratch slot, so that one chunk's kernels fill the SMs that
  // the other's last wave leaves idle (a chunk's launches end in partial waves).  A slot is
  // reused only by the chunk two on, on the same stream.
  size_t slot = 0;
  bool dual = true;
  for (size_t i = 0; i < p.tasks.size() && dual; ++i) {
    const qk_task &t = p.tasks[i];
    if (!use_fused(t, p.dtype, p.refine)) dual = false;
    for (const uint32_t nr : chunks[i]) {
      const size_t b = align256(task_scratch(sub_task(t, 0, nr, elem), p.dtype, p.refine));
      if (b > slot) slot = b;
    }
  }
  const size_t avail = p.persist_bytes ? p.persist_off : p.total;
  if (nchunks < 2 || 2 * slot > avail) dual = false;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_host_mu);
  HostRunner &hr = g_host_runners[dev];
  int rc = hr.ensure(2 * nchunks + 1);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  // the copies and the compute streams must not start before earlier work on the caller's
  // stream
  cudaEvent_t start = hr.ev[2 * nchunks];
  cudaError_t e = cudaEventRecord(start, st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(hr.in, start, 0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(hr.out, start, 0);
  for (int c = 0; c < 2 && dual && e == cudaSuccess; ++c) e = cudaStreamWaitEvent(hr.cmp[c], start, 0);
  if (e != cudaSuccess) return cuda_fail(e, "qk_batch_run_host");
  size_t k = 0;
  auto cp = [&](void *dst, const void *src, size_t bytes, cudaMemcpyKind kind, cudaStream_t s) -> int {
    if (!bytes) return QK_OK;
    cudaError_t ce = cudaMemcpyAsync(dst, src, bytes, kind, s);
    return ce == cudaSuccess ? QK_OK : cuda_fail(ce, "qk_batch_run_host: copy");
  };
  for (size_t i = 0; i < p.tasks.size(); ++i) {
    const qk_task &t = p.tasks[i];
    const uint64_t n = 1ull << t.m, d = t.ps.d;
    uint32_t r0 = 0;
    for (const uint32_t nr : chunks[i]) {
      const qk_task s = sub_task(t, r0, nr, elem);
      const size_t ybytes = elem * nr * t.nrhs * n, yoff = elem * (size_t)r0 * t.nrhs * n;
      // host -> device: this chunk's right-hand sides
      if ((rc = cp((void *)s.y, (const unsigned char *)io[i].y + yoff, ybytes, cudaMemcpyHostToDevice, hr.in)))
        return rc;
      if ((e = cudaEventRecord(hr.ev[2 * k], hr.in)) != cudaSuccess) return cuda_fail(e, "qk_batch_run_host");
      // compute once the chunk has landed: on the caller's stream, or on compute stream k mod 2
      // with scratch slot k mod 2
      cudaStream_t cs = dual ? hr.cmp[k & 1] : st;
      unsigned char *wsk = (unsigned char *)ws + (dual ? (k & 1) * slot : 0);
      if ((e = cudaStreamWaitEvent(cs, hr.ev[2 * k], 0)) != cudaSuccess) return cuda_fail(e, "qk_batch_run_host");
      if ((rc = run_task(p, s, wsk, status, cs, nullptr))) return rc;
      if ((e = cudaEventRecord(hr.ev[2 * k + 1], cs)) != cudaSuccess) return cuda_fail(e, "qk_batch_run_host");
      // device -> host: this chunk's results, overlapping the next chunk's compute
      if ((e = cudaStreamWaitEvent(hr.out, hr.ev[2 * k + 1], 0)) != cudaSuccess)
        return cuda_fail(e, "qk_batch_run_host");
      if (io[i].c && (rc = cp((unsigned char *)io[i].c + yoff, s.c, ybytes, cudaMemcpyDeviceToHost, hr.out)))
        return rc;
      if (io[i].lam && (rc = cp(io[i].lam + (size_t)r0 * n, s.lam, 8 * nr * n, cudaMemcpyDeviceToHost, hr.out)))
        return rc;
      if ((rc = cp(io[i].out + (size_t)r0 * t.nrhs * QK_MLL_NOUT, s.out, 8 * nr * t.nrhs * QK_MLL_NOUT,
                   cudaMemcpyDeviceToHost, hr.out)))
        return rc;
      if (io[i].grad && (rc = cp(io[i].grad + (size_t)r0 * t.nrhs * (2 * d + 2), s.grad,
                                 8 * nr * t.nrhs * (2 * d + 2), cudaMemcpyDeviceToHost, hr.out)))
        return rc;
      r0 += nr;
      ++k;
    }
  }
  // the caller's stream completes only after the last copy back
  if (k) {
    if ((e = cudaEventRecord(hr.ev[2 * (k - 1)], hr.out)) != cudaSuccess) return cuda_fail(e, "qk_batch_run_host");
    if ((e = cudaStreamWaitEvent(st, hr.ev[2 * (k - 1)], 0)) != cudaSuccess) return cuda_fail(e, "qk_batch_run_host");
  }
  return QK_OK;
}

int qk_batch_timing(void *ws, uint32_t runs) {
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_plans.find(ws);
  if (it == g_plans.end()) return fail(QK_EINVAL, "no plan recorded for this workspace (call qk_batch_plan)");
  if (!it->second.timer) it->second.timer = std::make_shared<EventTimer>();
  it->second.timer->clear();
  it->second.timer->runs_left = runs;
  return QK_OK;
}

int qk_batch_kernel_ms(void *ws, uint32_t idx, char *name, size_t name_len, uint32_t *launches, double *ms) {
  std::shared_ptr<EventTimer> tm;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_plans.find(ws);
    if (it == g_plans.end()) return fail(QK_EINVAL, "no plan recorded for this workspace (call qk_batch_plan)");
    tm = it->second.timer;
  }
  if (!tm) return fail(QK_EINVAL, "timing was not enabled (call qk_batch_timing)");
  std::vector<std::string> names;
  for (const auto &r : tm->recs) {
    bool seen = false;
    for (const auto &nm : names) seen |= nm == r.name;
    if (!seen) names.push_back(r.name);
  }
  if (idx >= names.size()) return fail(QK_EINVAL, "kernel index %u beyond %zu recorded names", idx, names.size());
  uint32_t cnt = 0;
  double tot = 0.0;
  for (const auto &r : tm->recs) {
    if (r.name != names[idx]) continue;
    cudaError_t e = cudaEventSynchronize(r.b);
    if (e != cudaSuccess) return cuda_fail(e, "qk_batch_kernel_ms");
    float t = 0.f;
    e = cudaEventElapsedTime(&t, r.a, r.b);
    if (e != cudaSuccess) return cuda_fail(e, "qk_batch_kernel_ms");
    ++cnt;
    tot += t;
  }
  if (name && name_len) {
    strncpy(name, names[idx].c_str(), name_len - 1);
    name[name_len - 1] = 0;
  }
  if (launches) *launches = cnt;
  if (ms) *ms = tot;
  return QK_OK;
}

}  // extern "C"
