// Batched FWHT with a workspace (qk_fwht_ws) and its autotuner (qk_fwht_tune).
//
// For LOGT < m <= 2 LOGT - LOGL the transform is two tile passes (low bits on contiguous
// tiles, high bits on column tiles).  They run either as two launches over the whole
// batch, or as one persistent launch that queues a vector's column tiles `lag` vectors
// after its low tiles (qk_fused.cu).  Which is faster, and with which lag and number of
// resident CTAs per SM, depends on m, the batch and the GPU's L2, so the tuner times the
// candidates on the caller's buffer and remembers the fastest per (device, m, dtype,
// nvec).  Other sizes go to the generic multi-pass transform.
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "qk_common.cuh"
#include "qk_internal.h"

namespace qk {

using TuneKey = std::tuple<int, uint32_t, int32_t, uint64_t>;
static std::mutex g_tune_mu;
static std::map<TuneKey, qk_fwht_plan> g_tuned;

static int current_device() {
  int dev = 0;
  cudaGetDevice(&dev);
  return dev;
}

static int run_plan_wht(const qk_fwht_plan &p, uint32_t m, uint64_t nvec, int32_t dtype, void *x, void *ws,
                        uint32_t *status, cudaStream_t st) {
  const double scale = 1.0 / std::sqrt((double)(1ull << m));
  if (p.mode == QK_FWHT_TWO_PASS) return tiled_wht(x, m, nvec, dtype, scale, st);
  return persist_wht(x, m, nvec, dtype, scale, ws, status, st, p.lag, p.ctas_per_sm);
}

static qk_fwht_plan default_plan() {
  qk_fwht_plan p;
  p.mode = QK_FWHT_PERSISTENT;
  p.lag = 0;  // chosen from m, nvec and the grid at launch
  p.ctas_per_sm = 0;
  p.ms = -1.0f;
  return p;
}

}  // namespace qk

using namespace qk;

extern "C" {

int qk_fwht_ws(uint32_t m, uint64_t nvec, int32_t dtype, void *x, void *ws, size_t ws_bytes,
               const qk_fwht_plan *plan, uint32_t *status, qk_stream stream) {
  set_error("%s", "");
  if (dtype != QK_F64 && dtype != QK_F32) return fail(QK_EINVAL, "dtype must be QK_F64 or QK_F32");
  if (m > QK_MAX_M) return fail(QK_EINVAL, "m = %u exceeds QK_MAX_M = %d", m, QK_MAX_M);
  if (nvec == 0) return QK_OK;
  if (!x) return fail(QK_EINVAL, "transform data is NULL");
  if (!tiled_wht_supported(m, dtype)) return op_transform(0 /* WHT */, m, nvec, dtype, x, (cudaStream_t)stream);
  const size_t need = persist_wht_ws_bytes(nvec);
  if (!ws || ws_bytes < need) return fail(QK_EWORKSPACE, "qk_fwht_ws: workspace has %zu bytes, %zu needed", ws_bytes, need);
  if (((uintptr_t)ws & 255u) != 0) return fail(QK_EINVAL, "workspace must be 256-byte aligned");
  qk_fwht_plan p = default_plan();
  if (plan) {
    if (plan->mode != QK_FWHT_TWO_PASS && plan->mode != QK_FWHT_PERSISTENT)
      return fail(QK_EINVAL, "plan mode must be QK_FWHT_TWO_PASS or QK_FWHT_PERSISTENT");
    p = *plan;
  } else {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(TuneKey(current_device(), m, dtype, nvec));
    if (it != g_tuned.end()) p = it->second;
  }
  return run_plan_wht(p, m, nvec, dtype, x, ws, status, (cudaStream_t)stream);
}

int qk_fftbr_ws(uint32_t m, uint64_t nvec, int32_t dtype, int32_t inverse, void *x, void *ws, size_t ws_bytes,
                uint32_t lag, uint32_t *status, qk_stream stream) {
  set_error("%s", "");
  if (dtype != QK_F64 && dtype != QK_F32) return fail(QK_EINVAL, "dtype must be QK_F64 or QK_F32");
  if (m > QK_MAX_M) return fail(QK_EINVAL, "m = %u exceeds QK_MAX_M = %d", m, QK_MAX_M);
  if (inverse != 0 && inverse != 1) return fail(QK_EINVAL, "inverse must be 0 or 1");
  if (nvec == 0) return QK_OK;
  if (!x) return fail(QK_EINVAL, "transform data is NULL");
  const int kind = inverse ? 2 /* IFFTBR */ : 1 /* FFTBR */;
  if (!persist_fft_supported(m, dtype)) return op_transform(kind, m, nvec, dtype, x, (cudaStream_t)stream);
  const size_t need = persist_wht_ws_bytes(nvec);
  if (!ws || ws_bytes < need) return fail(QK_EWORKSPACE, "qk_fftbr_ws: workspace has %zu bytes, %zu needed", ws_bytes, need);
  if (((uintptr_t)ws & 255u) != 0) return fail(QK_EINVAL, "workspace must be 256-byte aligned");
  return persist_fft(kind, x, m, nvec, 1.0 / std::sqrt((double)(1ull << m)), (uint32_t *)ws, status, lag,
                     (cudaStream_t)stream);
}

int qk_fwht_tune(uint32_t m, uint64_t nvec, int32_t dtype, void *x, void *ws, size_t ws_bytes, qk_fwht_plan *best,
                 qk_stream stream) {
  set_error("%s", "");
  if (dtype != QK_F64 && dtype != QK_F32) return fail(QK_EINVAL, "dtype must be QK_F64 or QK_F32");
  if (m > QK_MAX_M) return fail(QK_EINVAL, "m = %u exceeds QK_MAX_M = %d", m, QK_MAX_M);
  if (nvec == 0 || !x) return fail(QK_EINVAL, "qk_fwht_tune needs nvec >= 1 and data");
  if (!tiled_wht_supported(m, dtype)) {
    if (best) *best = default_plan();
    return QK_OK;  // nothing to choose: the generic transform
  }
  const size_t need = persist_wht_ws_bytes(nvec);
  if (!ws || ws_bytes < need) return fail(QK_EWORKSPACE, "qk_fwht_tune: workspace has %zu bytes, %zu needed", ws_bytes, need);
  if (((uintptr_t)ws & 255u) != 0) return fail(QK_EINVAL, "workspace must be 256-byte aligned");
  cudaStream_t st = (cudaStream_t)stream;
  const int occ = persist_wht_max_ctas_per_sm(dtype);
  if (occ <= 0) return fail(QK_ECUDA, "qk_fwht_tune: occupancy query failed");
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, current_device());

  std::vector<qk_fwht_plan> cand;
  qk_fwht_plan two = default_plan();
  two.mode = QK_FWHT_TWO_PASS;
  cand.push_back(two);
  const uint64_t bytes = (dtype == QK_F64 ? 8ull : 4ull) << m;
  for (int cps = 1; cps <= occ; ++cps) {
    const uint32_t dl = persist_wht_default_lag(m, nvec, dtype, (uint32_t)(sms * cps));
    const uint32_t base = dl > 1 ? dl / 2 : 1;  // candidates: half, once and twice the default
    uint32_t prev = 0;
    for (uint32_t mult : {1u, 2u, 4u}) {
      uint64_t lag = (uint64_t)base * mult;
      if (lag > nvec) lag = nvec;
      if (lag * bytes > (96ull << 20) && mult > 1) continue;  // keep the waiting output within L2
      if (lag == prev) continue;
      prev = (uint32_t)lag;
      qk_fwht_plan p = default_plan();
      p.lag = (uint32_t)lag;
      p.ctas_per_sm = (uint32_t)cps;
      cand.push_back(p);
    }
  }

  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  qk_fwht_plan win = cand[0];
  float win_ms = 1e30f;
  int rc = QK_OK;
  for (qk_fwht_plan &p : cand) {
    if ((rc = run_plan_wht(p, m, nvec, dtype, x, ws, nullptr, st))) break;  // warm-up
    const int reps = 3;
    cudaEventRecord(a, st);
    for (int r = 0; r < reps && !rc; ++r) rc = run_plan_wht(p, m, nvec, dtype, x, ws, nullptr, st);
    cudaEventRecord(b, st);
    if (rc) break;
    cudaError_t e = cudaEventSynchronize(b);
    if (e != cudaSuccess) {
      rc = cuda_fail(e, "qk_fwht_tune");
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    p.ms = ms / reps;
    if (p.ms < win_ms) {
      win_ms = p.ms;
      win = p;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (rc) return rc;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[TuneKey(current_device(), m, dtype, nvec)] = win;
  }
  if (best) *best = win;
  return QK_OK;
}

int qk_fwht_wait_selftest(uint32_t m, uint64_t nvec, int32_t dtype, void *x, void *ws, size_t ws_bytes,
                          uint32_t spin_limit, uint32_t *status, qk_stream stream) {
  set_error("%s", "");
  if (dtype != QK_F64 && dtype != QK_F32) return fail(QK_EINVAL, "dtype must be QK_F64 or QK_F32");
  if (!tiled_wht_supported(m, dtype)) return fail(QK_EINVAL, "m = %u is not a two-pass size", m);
  if (nvec == 0 || !x || !status) return fail(QK_EINVAL, "qk_fwht_wait_selftest needs nvec >= 1, data, status");
  if (spin_limit == 0 || spin_limit > kSpinLimit) return fail(QK_EINVAL, "spin_limit must be 1..%u", kSpinLimit);
  const size_t need = persist_wht_ws_bytes(nvec);
  if (!ws || ws_bytes < need) return fail(QK_EWORKSPACE, "workspace has %zu bytes, %zu needed", ws_bytes, need);
  if (((uintptr_t)ws & 255u) != 0) return fail(QK_EINVAL, "workspace must be 256-byte aligned");
  return persist_wht(x, m, nvec, dtype, 1.0, ws, status, (cudaStream_t)stream, 0, 0, spin_limit, true);
}

}  // extern "C"
