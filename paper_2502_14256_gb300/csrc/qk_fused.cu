// Host side of the fused net pipeline (arXiv 2502.14256, Sec. 5.3-5.4): workspace layout,
// dispatch by precision, the persistent whole-plan schedule's tables, and the batched
// two-pass and persistent FWHT kernels.  The pipeline's kernels live in qk_fused.cuh.
#include <cmath>
#include <type_traits>
#include <utility>
#include <vector>

#include "qk_fused.cuh"

namespace qk {

QK_FUSED_PRECISIONS(QK_FUSED_EXTERN)

// ------------------------------------------------- standalone batched WHT
// x <- H x * scale for vectors of n = 2^m with LOGT < m <= 2 LOGT - LOGL, in place, in two
// tile passes: low LOGT bits on contiguous tiles, the high bits on column tiles.
template <typename T>
__global__ void __launch_bounds__(kFNT, 5) k_wht_low(T *__restrict__ x) {
  constexpr int LOGT = FCfg<T>::LOGT, L = FCfg<T>::L;
  extern __shared__ __align__(16) unsigned char smem[];
  T *sm = reinterpret_cast<T *>(smem);
  T *xb = x + ((uint64_t)blockIdx.x << LOGT);  // tiles of all vectors, contiguous
  const int t = threadIdx.x;
  T v[L];
#pragma unroll
  for (int l = 0; l < L; ++l) v[l] = xb[e_of<T>(0, t, l)];
  xwht_full<T>(v, sm, 0);
#pragma unroll
  for (int l = 0; l < L; ++l) xb[e_of<T>(2, t, l)] = v[l];
}

template <typename T, int M>
__global__ void __launch_bounds__(kFNT) k_wht_high(T *__restrict__ x, T scale) {
  constexpr int LOGT = FCfg<T>::LOGT, L = FCfg<T>::L;
  extern __shared__ __align__(16) unsigned char smem[];
  T *sm = reinterpret_cast<T *>(smem);
  constexpr int c = 2 * LOGT - M;
  const int t = threadIdx.x;
  constexpr uint32_t tiles = 1u << (M - LOGT);
  const uint32_t tau = blockIdx.x & (tiles - 1);
  T *xv = x + ((uint64_t)(blockIdx.x >> (M - LOGT)) << M);
  const uint32_t tcol = tau << c;
  auto widx = [&](uint32_t e) -> uint32_t { return ((e >> c) << LOGT) | tcol | (e & ((1u << c) - 1)); };
  T v[L];
#pragma unroll
  for (int l = 0; l < L; ++l) v[l] = xv[widx(e_of<T>(0, t, l))];
  xwht_col<T>(v, sm, c, 0);
#pragma unroll
  for (int l = 0; l < L; ++l) xv[widx(e_of<T>(2, t, l))] = v[l] * scale;
}

// ------------------------------------------- persistent batched WHT (one launch)
// Both tile passes of every vector in a single launch of resident CTAs that take work
// items in ticket order (WhtSched) from a global counter: the low-pass tiles first, a
// vector's column tiles `lag` vectors later.  Past the wait limit a column tile is skipped
// and QK_STATUS_TIMEOUT is raised.
template <typename T, int M>
__global__ void __launch_bounds__(kFNT, 5) k_wht_persist(T *__restrict__ x, T scale, WhtSched sc,
                                                         uint32_t *__restrict__ ctr, uint32_t *status,
                                                         uint32_t spin_limit, uint32_t first_item) {
  constexpr int LOGT = FCfg<T>::LOGT, L = FCfg<T>::L, m = M, c = 2 * LOGT - M;
  extern __shared__ __align__(16) unsigned char smem[];
  // s_item[k & 1] and s_ok[k & 1] belong to this CTA's item k: thread 0 claims item
  // k + 1 while item k is processed.  Every path through an item passes a barrier after
  // its slots are read, so a slot is rewritten (two items on) only after all threads
  // have read it, and the loop needs no barrier of its own.
  __shared__ uint32_t s_item[2], s_ok[2];
  T *sm = reinterpret_cast<T *>(smem);
  uint32_t *ticket = ctr, *done = ctr + 1;
  const int t = threadIdx.x;
  const uint32_t total = sc.total(), T_ = 1u << sc.lt;
  if (t == 0) s_item[0] = first_item + atomicAdd(ticket, 1u);
  __syncthreads();
  for (int k = 0;; ++k) {
    const uint32_t it = s_item[k & 1];
    if (it >= total) break;
    if (t == 0) s_item[(k + 1) & 1] = first_item + atomicAdd(ticket, 1u);
    uint32_t v, tile;
    bool high;
    sc.decode(it, v, tile, high);
    T *xv = x + ((uint64_t)v << m);
    T r[L];
    if (!high) {
      T *xb = xv + ((uint64_t)tile << LOGT);
#pragma unroll
      for (int l = 0; l < L; ++l) r[l] = xb[e_of<T>(0, t, l)];
      xwht_full<T>(r, sm, 0);
#pragma unroll
      for (int l = 0; l < L; ++l) xb[e_of<T>(2, t, l)] = r[l];
      __syncthreads();  // every thread's stores precede thread 0's release below
      if (t == 0) red_release_add_u32(&done[v], 1u);
    } else {
      if (t == 0) {
        uint32_t tries = 0, ok = 1;
        while (ld_acquire_u32(&done[v]) < T_) {
          if (++tries > spin_limit) {
            ok = 0;
            if (status) atomicOr(status, (uint32_t)QK_STATUS_TIMEOUT);
            break;
          }
          __nanosleep(128);
        }
        s_ok[k & 1] = ok;
      }
      __syncthreads();
      if (s_ok[k & 1]) {
        const uint32_t tcol = tile << c;
        auto widx = [&](uint32_t e) -> uint32_t { return ((e >> c) << LOGT) | tcol | (e & ((1u << c) - 1)); };
#pragma unroll
        for (int l = 0; l < L; ++l) r[l] = __ldcg(&xv[widx(e_of<T>(0, t, l))]);  // L2, never a stale L1 line
        xwht_col<T>(r, sm, c, 0);
#pragma unroll
        for (int l = 0; l < L; ++l) xv[widx(e_of<T>(2, t, l))] = r[l] * scale;
      }
    }
  }
}

size_t persist_wht_ws_bytes(uint64_t nvec) { return align256(sizeof(uint32_t) * (1 + nvec)); }

// Every m of the two-pass range gets its own instantiation: with the tile split known at
// compile time, column-tile addressing folds into immediate offsets and the butterfly
// stage selection into straight-line code.
template <typename T> struct WhtKernels {
  void (*low)(T *);  // the same for every m
  void (*high)(T *, T);
  void (*persist)(T *, T, WhtSched, uint32_t *, uint32_t *, uint32_t, uint32_t);
};
template <typename T, int M>
static WhtKernels<T> wht_kernels_m() {
  return WhtKernels<T>{k_wht_low<T>, k_wht_high<T, M>, k_wht_persist<T, M>};
}
template <typename T, int... I>
static WhtKernels<T> wht_pick(int m, std::integer_sequence<int, I...>) {
  constexpr int LO = FCfg<T>::LOGT + 1;
  WhtKernels<T> out{nullptr, nullptr, nullptr};
  ((m == LO + I ? (void)(out = wht_kernels_m<T, LO + I>()) : (void)0), ...);
  return out;
}
template <typename T>
static WhtKernels<T> wht_kernels(int m) {
  constexpr int LOGT = FCfg<T>::LOGT;
  return wht_pick<T>(m, std::make_integer_sequence<int, two_pass_max_m<T>() - LOGT>());
}

bool tiled_wht_supported(uint32_t m, int dtype) {
  const int LOGT = dtype == QK_F64 ? FCfg<double>::LOGT : FCfg<float>::LOGT;
  const int MX = dtype == QK_F64 ? two_pass_max_m<double>() : two_pass_max_m<float>();
  return (int)m > LOGT && (int)m <= MX;
}

// Vectors may be processed in chunks (chunk_bytes) so that the second pass could find
// the first pass's output in L2; on GB300 a sweep of 8 MB .. unchunked (64 x 2^20 FP32)
// measured 1.17 .. 2.96 TB/s algorithmic, best unchunked (each pass then streams at
// ~87% of the measured copy bandwidth), so the default is one launch per pass.
template <typename T>
static int tiled_wht_t(T *x, uint32_t m, uint64_t nvec, double scale, cudaStream_t st, size_t chunk_bytes) {
  constexpr int LOGT = FCfg<T>::LOGT;
  const size_t sm = xtile_bytes<T>();
  const uint64_t n = 1ull << m;
  uint64_t chunk = chunk_bytes / (n * sizeof(T));
  if (chunk < 1) chunk = 1;
  const WhtKernels<T> K = wht_kernels<T>(m);
  for (uint64_t v0 = 0; v0 < nvec; v0 += chunk) {
    const uint64_t nv = (nvec - v0) < chunk ? (nvec - v0) : chunk;
    const uint64_t blocks = nv << (m - LOGT);
    K.low<<<(unsigned)blocks, kFNT, sm, st>>>(x + v0 * n);
    int rc = check_launch("wht low");
    if (rc) return rc;
    K.high<<<(unsigned)blocks, kFNT, sm, st>>>(x + v0 * n, (T)scale);
    if ((rc = check_launch("wht high"))) return rc;
  }
  return QK_OK;
}

int tiled_wht(void *x, uint32_t m, uint64_t nvec, int dtype, double scale, cudaStream_t st, size_t chunk_bytes) {
  return dtype == QK_F64 ? tiled_wht_t<double>((double *)x, m, nvec, scale, st, chunk_bytes)
                         : tiled_wht_t<float>((float *)x, m, nvec, scale, st, chunk_bytes);
}

template <typename T>
static int persist_occupancy() {
  static int occ = -1;
  if (occ < 0) {
    // every instantiation has the same launch bounds and shared memory; query one
    constexpr int M = two_pass_max_m<T>() - 1;
    const size_t sm = xtile_bytes<T>();
    smem_optin<k_wht_persist<T, M>>(sm);
    int o = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_wht_persist<T, M>, kFNT, sm) != cudaSuccess) return -1;
    occ = o;
  }
  return occ;
}

int persist_wht_max_ctas_per_sm(int dtype) {
  return dtype == QK_F64 ? persist_occupancy<double>() : persist_occupancy<float>();
}

// Lag (in vectors) after which a vector's column tiles are queued: enough tickets between
// a vector's last low tile and its first column tile that the low tile has finished when
// the column tile is taken (lag tiles-per-vector >= resident CTAs), plus three vectors of
// slack (measured), and at most 48 MB of first-pass output waiting in L2.
uint32_t persist_wht_default_lag(uint32_t m, uint64_t nvec, int dtype, uint32_t ctas) {
  const int LOGT = dtype == QK_F64 ? FCfg<double>::LOGT : FCfg<float>::LOGT;
  const uint64_t T = 1ull << (m - LOGT), bytes = (dtype == QK_F64 ? 8ull : 4ull) << m;
  uint64_t lag = (ctas + T - 1) / T + 3;  // measured best for 64 x 2^20 FP32 at 4 CTAs/SM: 8
  const uint64_t cap = (48ull << 20) / bytes;
  if (lag > cap) lag = cap;
  if (lag < 1) lag = 1;
  if (lag > nvec) lag = nvec;
  return (uint32_t)lag;
}

template <typename T>
static int persist_wht_t(T *x, uint32_t m, uint64_t nvec, double scale, uint32_t *ctr, uint32_t *status,
                         cudaStream_t st, uint32_t lag, uint32_t ctas_per_sm, uint32_t spin_limit,
                         bool columns_only) {
  constexpr int LOGT = FCfg<T>::LOGT;
  const int occ = persist_occupancy<T>();
  if (occ <= 0) return fail(QK_ECUDA, "persistent WHT: occupancy query failed");
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // default: at most 4 CTAs per SM (measured: a fifth resident CTA gains nothing and
  // lengthens the lag the queue needs)
  const uint32_t cps = ctas_per_sm == 0 ? (occ < 4 ? (uint32_t)occ : 4u)
                                        : ((int)ctas_per_sm > occ ? (uint32_t)occ : ctas_per_sm);
  const uint64_t items = (2ull * nvec) << (m - LOGT);
  if (items >= (1ull << 31)) return fail(QK_EINVAL, "persistent WHT: %llu work items exceed 2^31",
                                         (unsigned long long)items);
  const uint32_t grid = (uint32_t)sms * cps;
  if (lag == 0) lag = persist_wht_default_lag(m, nvec, sizeof(T) == 8 ? QK_F64 : QK_F32, grid);
  if (lag > nvec) lag = (uint32_t)nvec;
  WhtSched sc{(uint32_t)nvec, (uint32_t)(m - LOGT), lag};
  cudaError_t e = cudaMemsetAsync(ctr, 0, sizeof(uint32_t) * (1 + nvec), st);
  if (e != cudaSuccess) return cuda_fail(e, "persistent WHT: counter reset");
  // columns_only starts the tickets at the first column tile with every vector's low
  // tiles left unpublished: each column tile's wait must then run out (a test of the
  // bounded wait; the data are left untouched).
  if (columns_only) sc.lag = (uint32_t)nvec;
  const uint32_t first = columns_only ? (uint32_t)(nvec << (m - LOGT)) : 0u;
  wht_kernels<T>((int)m).persist<<<grid, kFNT, xtile_bytes<T>(), st>>>(x, (T)scale, sc, ctr, status, spin_limit,
                                                                        first);
  return check_launch("wht persistent");
}

int persist_wht(void *x, uint32_t m, uint64_t nvec, int dtype, double scale, void *ws, uint32_t *status,
                cudaStream_t st, uint32_t lag, uint32_t ctas_per_sm, uint32_t spin_limit, bool columns_only) {
  if (nvec == 0) return QK_OK;
  return dtype == QK_F64 ? persist_wht_t<double>((double *)x, m, nvec, scale, (uint32_t *)ws, status, st, lag,
                                                 ctas_per_sm, spin_limit, columns_only)
                         : persist_wht_t<float>((float *)x, m, nvec, scale, (uint32_t *)ws, status, st, lag,
                                                ctas_per_sm, spin_limit, columns_only);
}

// ------------------------------------------------------------------ host side
bool fused_supported(const qk_task &t, int dtype) {
  if (t.k.family != QK_DSI || t.ps.kind != QK_NET_B2) return false;
  if (dtype == QK_F32W) dtype = QK_F32;
  const int LOGT = dtype == QK_F64 ? FCfg<double>::LOGT : FCfg<float>::LOGT;
  const int MX = dtype == QK_F64 ? two_pass_max_m<double>() : two_pass_max_m<float>();
  return (int)t.m > LOGT && (int)t.m <= MX;
}

static size_t fused_elem(int dtype) { return dtype == QK_F64 ? 8 : 4; }

size_t fused_ws_bytes(const qk_task &t, int dtype, int refine) {
  const int LOGT = dtype == QK_F64 ? FCfg<double>::LOGT : FCfg<float>::LOGT;
  const uint64_t R = t.ps.R, n = 1ull << t.m, tiles = n >> LOGT, nv = R * t.nrhs;
  const size_t e = fused_elem(dtype);
  size_t s = 2 * align256(e * R * n) + 2 * align256(e * nv * n);
  s += 2 * align256(8 * R * tiles) + align256(8 * nv * tiles) + align256(16 * nv * tiles);
  s += align256(8 * nv * tiles * 2 * (uint64_t)t.ps.d);
  if ((refine > 0 && dtype == QK_F32) || dtype == QK_F32W) s += align256(e * nv * n);  // lo parts of y'
  if (dtype == QK_F32W) s += align256(e * R * n);                                      // lo parts of p'
  return s;
}

// The fused view of a task: its pointers and the scratch buffers carved from ws (in the
// order and sizes of fused_ws_bytes).
static FTask make_ftask(const qk_task &t, const ColJob &job, int dtype, int refine, void *ws, uint32_t *status) {
  const int LOGT = dtype == QK_F64 ? FCfg<double>::LOGT : FCfg<float>::LOGT;
  const uint64_t R = t.ps.R, n = 1ull << t.m, tiles = n >> LOGT, nv = R * t.nrhs;
  const size_t e = fused_elem(dtype);
  unsigned char *p = (unsigned char *)ws;
  FTask ft;
  ft.job = job;
  ft.nrhs = t.nrhs;
  ft.tiles = (uint32_t)tiles;
  ft.cB = 2 * LOGT - (int)t.m;
  ft.eta = t.eta;
  ft.y = t.y;
  ft.c = t.c;
  ft.lam = t.lam;
  ft.out = t.out;
  ft.grad = t.grad;
  ft.status = status;
  ft.p = p, p += align256(e * R * n);
  ft.pT = p, p += align256(e * R * n);
  ft.yT = p, p += align256(e * nv * n);
  ft.gT = p, p += align256(e * nv * n);
  ft.sp = (double *)p, p += align256(8 * R * tiles);
  ft.ld = (double *)p, p += align256(8 * R * tiles);
  ft.sy = (double *)p, p += align256(8 * nv * tiles);
  ft.qg = (double *)p, p += align256(16 * nv * tiles);
  ft.gr = (double *)p;
  p += align256(8 * nv * tiles * 2 * (uint64_t)t.ps.d);
  ft.yL = nullptr;
  ft.pTL = nullptr;
  if ((dtype == QK_F32 && refine > 0) || dtype == QK_F32W) {
    ft.yL = p;
    p += align256(e * nv * n);
  }
  if (dtype == QK_F32W) ft.pTL = p;
  return ft;
}

int run_fused(const qk_task &t, const ColJob &job, int dtype, int refine, void *ws, uint32_t *status,
              cudaStream_t st, LaunchTimer *tm) {
  const FTask ft = make_ftask(t, job, dtype, refine, ws, status);
  // FP64 needs no refinement; FP32 with refine >= 1 runs the compensated variant
  // (one exact-residual step; further steps change nothing at FP32 resolution)
  if (dtype == QK_F64) return dispatch_fused<double, false>(ft, st, tm);
  if (dtype == QK_F32W) return dispatch_fused<float, true, true>(ft, st, tm);  // always refined
  if (refine > 0) return dispatch_fused<float, true>(ft, st, tm);
  return dispatch_fused<float, false>(ft, st, tm);
}

static int persist_launch(const PSched &ps, int dtype, int refine, int alpha, uint32_t dmax, cudaStream_t st) {
  if (dtype == QK_F64) return persist_dispatch<double, false, false>(ps, alpha, dmax, st);
  if (dtype == QK_F32W) return persist_dispatch<float, true, true>(ps, alpha, dmax, st);
  if (refine > 0) return persist_dispatch<float, true, false>(ps, alpha, dmax, st);
  return persist_dispatch<float, false, false>(ps, alpha, dmax, st);
}

// Host side: the unit table, step table and counters live in the workspace region given
// to persist_setup (tables uploaded once, synchronously); persist_run resets the counters
// and launches.
bool persist_eligible(const std::vector<qk_task> &tasks, int dtype) {
  if (tasks.empty()) return false;
  for (const qk_task &t : tasks)
    if (!fused_supported(t, dtype) || t.k.alpha != tasks[0].k.alpha) return false;
  return true;
}

static size_t unit_scratch(const qk_task &t, int dtype, int refine) {
  qk_task one = t;
  one.ps.R = 1;
  return align256(fused_ws_bytes(one, dtype, refine));
}

static uint32_t persist_nslot(uint32_t lag) { return 2 * lag + 3; }

size_t persist_ws_bytes(const std::vector<qk_task> &tasks, int dtype, int refine, uint32_t lag) {
  if (lag == 0) lag = 1;
  size_t slot = 0, U = 0;
  for (const qk_task &t : tasks) {
    const size_t b = unit_scratch(t, dtype, refine);
    if (b > slot) slot = b;
    U += t.ps.R;
  }
  const size_t S = U + 2 * lag + 2;
  return persist_nslot(lag) * slot + align256(sizeof(PUnit) * U) + align256(sizeof(uint32_t) * (S + 1)) +
         align256(sizeof(uint32_t) * (2 + 4 * U));
}

int persist_setup(const std::vector<qk_task> &tasks, int dtype, int refine, uint32_t lag, void *region, size_t bytes,
                  PersistState &out) {
  if (lag == 0) lag = 1;
  if (!persist_eligible(tasks, dtype))
    return fail(QK_EINVAL, "persistent schedule: tasks are not all fused DSI nets of one order");
  if (bytes < persist_ws_bytes(tasks, dtype, refine, lag))
    return fail(QK_EWORKSPACE, "persistent schedule: workspace too small");
  const int LOGT = dtype == QK_F64 ? FCfg<double>::LOGT : FCfg<float>::LOGT;
  size_t slot = 0;
  uint32_t U = 0, dmax = 0;
  for (const qk_task &t : tasks) {
    const size_t b = unit_scratch(t, dtype, refine);
    if (b > slot) slot = b;
    U += t.ps.R;
    if (t.ps.d > dmax) dmax = t.ps.d;
  }
  const uint32_t nslot = persist_nslot(lag), S = U + 2 * lag + 2;
  unsigned char *base = (unsigned char *)region;
  unsigned char *units_d = base + nslot * slot;
  unsigned char *steps_d = units_d + align256(sizeof(PUnit) * U);
  unsigned char *ctr_d = steps_d + align256(sizeof(uint32_t) * (S + 1));
  std::vector<PUnit> units;
  units.reserve(U);
  const size_t elem = dtype == QK_F64 ? 8 : 4;
  for (const qk_task &t : tasks) {
    const uint64_t n = 1ull << t.m, d = t.ps.d;
    for (uint32_t r = 0; r < t.ps.R; ++r) {
      qk_task one = t;  // randomization r as a task of its own
      one.ps.R = 1;
      if (t.ps.Ct) one.ps.Ct = t.ps.Ct + (size_t)r * d * 32;
      one.y = (const unsigned char *)t.y + elem * (size_t)r * t.nrhs * n;
      if (t.c) one.c = (unsigned char *)t.c + elem * (size_t)r * t.nrhs * n;
      if (t.lam) one.lam = t.lam + (size_t)r * n;
      one.out = t.out + (size_t)r * t.nrhs * QK_MLL_NOUT;
      if (t.grad) one.grad = t.grad + (size_t)r * t.nrhs * (2 * d + 2);
      const ColJob job = make_job(&one.ps, &one.k, 0, 1, one.m);
      PUnit pu;
      pu.ft = make_ftask(one, job, dtype, refine, base + (size_t)(units.size() % nslot) * slot, nullptr);
      pu.tiles = (uint32_t)(n >> LOGT);
      pu.nrhs = t.nrhs;
      pu.ncv = (t.c || t.grad) ? pu.tiles * t.nrhs : 0;
      units.push_back(pu);
    }
  }
  std::vector<uint32_t> off(S + 1, 0);
  for (uint32_t s = 0; s < S; ++s) {
    uint64_t c = 0;
    if (s < U) c += units[s].tiles;
    if (s >= lag && s - lag < U) c += units[s - lag].tiles;
    if (s >= 2 * lag && s - 2 * lag < U) c += units[s - 2 * lag].ncv;
    if (s >= 2 * lag + 1 && s - 2 * lag - 1 < U) c += units[s - 2 * lag - 1].nrhs;
    if (off[s] + c >= (1ull << 31)) return fail(QK_EINVAL, "persistent schedule: more than 2^31 work items");
    off[s + 1] = off[s] + (uint32_t)c;
  }
  cudaError_t e = cudaMemcpy(units_d, units.data(), sizeof(PUnit) * U, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(steps_d, off.data(), sizeof(uint32_t) * (S + 1), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "persistent schedule: table upload");
  out.units = units_d;
  out.steps = steps_d;
  out.ctr = ctr_d;
  out.ctr_bytes = sizeof(uint32_t) * (2 + 4 * (size_t)U);
  out.U = U, out.S = S, out.lag = lag, out.nslot = nslot, out.dmax = dmax;
  out.dtype = dtype, out.refine = refine, out.alpha = tasks[0].k.alpha;
  out.ok = true;
  return QK_OK;
}

int persist_run(const PersistState &p, uint32_t *status, cudaStream_t st, LaunchTimer *tm, uint32_t spin_limit) {
  cudaError_t e = cudaMemsetAsync(p.ctr, 0, p.ctr_bytes, st);
  if (e != cudaSuccess) return cuda_fail(e, "persistent schedule: counter reset");
  PSched ps;
  ps.units = (const PUnit *)p.units;
  ps.step_off = (const uint32_t *)p.steps;
  ps.U = p.U, ps.S = p.S, ps.lag = p.lag, ps.nslot = p.nslot;
  ps.ctr = (uint32_t *)p.ctr;
  ps.status = status;
  ps.spin_limit = spin_limit;
  if (tm) tm->begin("k_fused_persist", st);
  int rc = persist_launch(ps, p.dtype, p.refine, p.alpha, p.dmax, st);
  if (tm) tm->end(st);
  return rc;
}

}  // namespace qk
