// Fused solve + marginal log-likelihood + gradient for digital nets with DSI
// kernels (arXiv 2502.14256, Sec. 5.3-5.4), n = 2^m with LOGT < m <= 2 LOGT - 5.
//
// The length-n Hadamard transform is split at bit LOGT (tile = 2^LOGT elements:
// 8192 FP32 / 4096 FP64).  Three phases per randomization r:
//   A  (contiguous tiles)  first column p = k_1/zeta - 1 by the column sweep, stored;
//      low LOGT bits of the WHT of p and of every right-hand side y -> p', y';
//      FP64 partial sums of p and y.
//   B  (column tiles: the m - LOGT high bits x a run of contiguous low indices)
//      high bits of the WHT -> lambda = zeta H p + zeta n [w = 0] + eta (and
//      log lambda), Y = H y; epilogue c^_w = Y_w/(n lambda_w),
//      g_w = (Y_w^2/(n lambda_w^2) - 1/lambda_w)/2 with partial sums of the
//      quadratic form and of g; high bits of the inverse WHT of c^ and g.
//   C  (contiguous tiles)  low bits of the inverse -> c = K^-1 y (stored) and
//      u = H g; gradient sweep sum_i u_i dk1_i/dc_j, sum_i dk1_i/dc_j, with the
//      factors recomputed and k_1 from the stored p.
// A final kernel reduces the partial sums into the MLL outputs and gradient.
//
// Inside a tile every thread holds the L elements e = threadIdx.x + 256 l: the
// tile bits carried by l (the top log2 L bits) are transformed in registers, the
// low 8 bits in padded shared memory in radix-16 rounds.
#include <cmath>
#include <vector>

#include "qk_column.cuh"
#include "qk_common.cuh"
#include "qk_factors.cuh"
#include "qk_internal.h"

namespace qk {

template <typename T> struct FCfg;
template <> struct FCfg<float> { static constexpr int LOGT = 13, LOGL = 5, L = 32, PAD = 5; };
template <> struct FCfg<double> { static constexpr int LOGT = 12, LOGL = 4, L = 16, PAD = 4; };
constexpr int kFNT = 256, kLOGNT = 8;

struct FTask {
  ColJob job;
  uint32_t nrhs, tiles;  // tiles = n >> LOGT
  int cB;                // phase-B contiguous column bits (= 2 LOGT - m)
  double eta;
  const void *y;
  void *c;
  double *lam, *out, *grad;
  void *p, *pT, *yT, *gT;               // (R, n), (R, n), (R, nrhs, n), (R, nrhs, n)
  void *yL;                             // (R, nrhs, n): low parts of the compensated y' (refinement)
  double *sp, *sy, *ld, *qg, *gr;       // partial sums
  uint32_t *status;
};

template <typename T>
__device__ __forceinline__ int fpad(int e) { return e + (e >> FCfg<T>::PAD); }

template <typename T>
__host__ __device__ constexpr size_t tile_smem_bytes() {
  return (size_t)((1 << FCfg<T>::LOGT) + ((1 << FCfg<T>::LOGT) >> FCfg<T>::PAD)) * sizeof(T);
}

// Radix-2^R WHT round on tile bits [b, b+R) held in shared memory.
template <typename T, int R>
__device__ __forceinline__ void smem_round(T *sm, int b) {
  constexpr int G = (1 << FCfg<T>::LOGT) >> R;
  for (int g = threadIdx.x; g < G; g += kFNT) {
    const int e0 = (g & ((1 << b) - 1)) | ((g >> b) << (b + R));
    T v[1 << R];
#pragma unroll
    for (int q = 0; q < (1 << R); ++q) v[q] = sm[fpad<T>(e0 | (q << b))];
#pragma unroll
    for (int h = 0; h < R; ++h)
#pragma unroll
      for (int q = 0; q < (1 << R); ++q)
        if (!(q & (1 << h))) {
          const T a = v[q], bb = v[q | (1 << h)];
          v[q] = a + bb;
          v[q | (1 << h)] = a - bb;
        }
#pragma unroll
    for (int q = 0; q < (1 << R); ++q) sm[fpad<T>(e0 | (q << b))] = v[q];
  }
}

// WHT butterflies over tile bits [c, LOGT) of the tile held as v[l] at e = tid + 256 l;
// the result is returned in v with the same mapping.  sm: the padded tile scratch.
template <typename T>
__device__ __forceinline__ void tile_wht(T (&v)[FCfg<T>::L], T *sm, int c) {
  constexpr int L = FCfg<T>::L, LOGL = FCfg<T>::LOGL;
#pragma unroll
  for (int h = 0; h < LOGL; ++h) {
    if (kLOGNT + h >= c) {
#pragma unroll
      for (int q = 0; q < L; ++q)
        if (!(q & (1 << h))) {
          const T a = v[q], b = v[q | (1 << h)];
          v[q] = a + b;
          v[q | (1 << h)] = a - b;
        }
    }
  }
  if (c < kLOGNT) {
#pragma unroll
    for (int l = 0; l < L; ++l) sm[fpad<T>(threadIdx.x + (l << kLOGNT))] = v[l];
    __syncthreads();
    for (int b = c; b < kLOGNT; b += 4) {
      const int r = (kLOGNT - b) < 4 ? (kLOGNT - b) : 4;
      if (r == 4) smem_round<T, 4>(sm, b);
      else if (r == 3) smem_round<T, 3>(sm, b);
      else if (r == 2) smem_round<T, 2>(sm, b);
      else smem_round<T, 1>(sm, b);
      __syncthreads();
    }
#pragma unroll
    for (int l = 0; l < L; ++l) v[l] = sm[fpad<T>(threadIdx.x + (l << kLOGNT))];
    __syncthreads();
  }
}

// s + c tracks a sum with the rounding error of each addition carried in c (Kahan).
template <typename T>
__device__ __forceinline__ void kahan_add(T &s, T &c, T v) {
  const T y = v - c;
  const T t = s + y;
  c = (t - s) - y;
  s = t;
}

// Error-free sum: s + e == a + b exactly (Knuth's TwoSum; no ordering of |a|, |b| needed).
template <typename T>
__device__ __forceinline__ void two_sum(T a, T b, T &s, T &e) {
  s = a + b;
  const T bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// Compensated butterfly on (hi, lo) pairs: the rounding error of each hi sum is added
// to the lo parts, so hi + lo carries the transform to about twice the precision of T.
template <typename T>
__device__ __forceinline__ void cbfly(T &ah, T &al, T &bh, T &bl) {
  T s, e1, d, e2;
  two_sum(ah, bh, s, e1);
  two_sum(ah, -bh, d, e2);
  const T sl = (al + bl) + e1, dl = (al - bl) + e2;
  ah = s, al = sl, bh = d, bl = dl;
}

template <typename T, int R>
__device__ __forceinline__ void smem_round2(T *sh, T *sl, int b) {
  constexpr int G = (1 << FCfg<T>::LOGT) >> R;
  for (int g = threadIdx.x; g < G; g += kFNT) {
    const int e0 = (g & ((1 << b) - 1)) | ((g >> b) << (b + R));
    T vh[1 << R], vl[1 << R];
#pragma unroll
    for (int q = 0; q < (1 << R); ++q) {
      vh[q] = sh[fpad<T>(e0 | (q << b))];
      vl[q] = sl[fpad<T>(e0 | (q << b))];
    }
#pragma unroll
    for (int h = 0; h < R; ++h)
#pragma unroll
      for (int q = 0; q < (1 << R); ++q)
        if (!(q & (1 << h))) cbfly(vh[q], vl[q], vh[q | (1 << h)], vl[q | (1 << h)]);
#pragma unroll
    for (int q = 0; q < (1 << R); ++q) {
      sh[fpad<T>(e0 | (q << b))] = vh[q];
      sl[fpad<T>(e0 | (q << b))] = vl[q];
    }
  }
}

// tile_wht on compensated pairs (hi, lo); shl: a second padded tile for the lo parts.
template <typename T>
__device__ __forceinline__ void tile_wht2(T (&vh)[FCfg<T>::L], T (&vl)[FCfg<T>::L], T *sh, T *shl, int c) {
  constexpr int L = FCfg<T>::L, LOGL = FCfg<T>::LOGL;
#pragma unroll
  for (int h = 0; h < LOGL; ++h) {
    if (kLOGNT + h >= c) {
#pragma unroll
      for (int q = 0; q < L; ++q)
        if (!(q & (1 << h))) cbfly(vh[q], vl[q], vh[q | (1 << h)], vl[q | (1 << h)]);
    }
  }
  if (c < kLOGNT) {
#pragma unroll
    for (int l = 0; l < L; ++l) {
      sh[fpad<T>(threadIdx.x + (l << kLOGNT))] = vh[l];
      shl[fpad<T>(threadIdx.x + (l << kLOGNT))] = vl[l];
    }
    __syncthreads();
    for (int b = c; b < kLOGNT; b += 4) {
      const int r = (kLOGNT - b) < 4 ? (kLOGNT - b) : 4;
      if (r == 4) smem_round2<T, 4>(sh, shl, b);
      else if (r == 3) smem_round2<T, 3>(sh, shl, b);
      else if (r == 2) smem_round2<T, 2>(sh, shl, b);
      else smem_round2<T, 1>(sh, shl, b);
      __syncthreads();
    }
#pragma unroll
    for (int l = 0; l < L; ++l) {
      vh[l] = sh[fpad<T>(threadIdx.x + (l << kLOGNT))];
      vl[l] = shl[fpad<T>(threadIdx.x + (l << kLOGNT))];
    }
    __syncthreads();
  }
}

__device__ __forceinline__ float fused_log(float v) { return logf(v); }
__device__ __forceinline__ double fused_log(double v) { return log(v); }

// ------------------------------------------------------------------ phase A
template <typename T, int FAM, int ALPHA, bool COMP>
__global__ void __launch_bounds__(kFNT) k_fused_A(FTask ft) {
  constexpr int LOGT = FCfg<T>::LOGT, L = FCfg<T>::L;
  extern __shared__ __align__(16) unsigned char smem[];
  const ColJob &job = ft.job;
  const uint32_t d = job.d;
  double *wd;
  DiffTables tb;
  carve_tables<L>(smem, d, &wd, tb);
  T *wT = reinterpret_cast<T *>(wd);
  T *sm = reinterpret_cast<T *>(smem + align256(col_smem_bytes<L>(d)));
  double *red = reinterpret_cast<double *>(smem + align256(col_smem_bytes<L>(d)) +
                                           (COMP ? 2 : 1) * tile_smem_bytes<T>());
  const uint32_t r = blockIdx.y, tile = blockIdx.x;
  const uint64_t n = 1ull << job.m, base = (uint64_t)tile << LOGT;
  const int t = threadIdx.x;
  for (uint32_t q = t; q < d; q += kFNT) wT[q] = (T)job.w[q];
  build_all<T, FAM, ALPHA, L>(job, job.Ct + (size_t)r * d * 32, job.g, base, tb);
  __syncthreads();
  uint32_t bi[L];
#pragma unroll
  for (int l = 0; l < L; ++l) bi[l] = __brev((uint32_t)(base + t + (l << kLOGNT)));
  T p[L];
  column_sweep<T, FAM, ALPHA, L>(job, tb, wT, bi, p);
  T *P = reinterpret_cast<T *>(ft.p) + (uint64_t)r * n + base;
  T ps = T(0), pc = T(0);  // compensated (Kahan) thread partial: the sum cancels
#pragma unroll
  for (int l = 0; l < L; ++l) {
    P[t + (l << kLOGNT)] = p[l];
    kahan_add(ps, pc, p[l]);
  }
  const double sps = block_sum((double)ps - (double)pc, red);
  if (t == 0) ft.sp[(uint64_t)r * ft.tiles + tile] = sps;
  tile_wht<T>(p, sm, 0);
  T *PT = reinterpret_cast<T *>(ft.pT) + (uint64_t)r * n + base;
#pragma unroll
  for (int l = 0; l < L; ++l) PT[t + (l << kLOGNT)] = p[l];
  for (uint32_t q = 0; q < ft.nrhs; ++q) {
    const uint64_t v = (uint64_t)r * ft.nrhs + q;
    const T *Y = reinterpret_cast<const T *>(ft.y) + v * n + base;
    T yv[L];
    T ys = T(0), yc = T(0);
#pragma unroll
    for (int l = 0; l < L; ++l) {
      yv[l] = Y[t + (l << kLOGNT)];
      kahan_add(ys, yc, yv[l]);
    }
    const double sys = block_sum((double)ys - (double)yc, red);
    if (t == 0) ft.sy[v * ft.tiles + tile] = sys;
    T *YT = reinterpret_cast<T *>(ft.yT) + v * n + base;
    if constexpr (COMP) {
      T yl[L];
#pragma unroll
      for (int l = 0; l < L; ++l) yl[l] = T(0);
      tile_wht2<T>(yv, yl, sm, sm + tile_smem_bytes<T>() / sizeof(T), 0);
      T *YL = reinterpret_cast<T *>(ft.yL) + v * n + base;
#pragma unroll
      for (int l = 0; l < L; ++l) {
        YT[t + (l << kLOGNT)] = yv[l];
        YL[t + (l << kLOGNT)] = yl[l];
      }
    } else {
      tile_wht<T>(yv, sm, 0);
#pragma unroll
      for (int l = 0; l < L; ++l) YT[t + (l << kLOGNT)] = yv[l];
    }
  }
}

// ------------------------------------------------------------------ phase B
template <typename T, bool COMP>
__global__ void __launch_bounds__(kFNT, 2) k_fused_B(FTask ft) {
  constexpr int LOGT = FCfg<T>::LOGT, L = FCfg<T>::L;
  extern __shared__ __align__(16) unsigned char smem[];
  T *sm = reinterpret_cast<T *>(smem);
  T *lmv = reinterpret_cast<T *>(smem + tile_smem_bytes<T>());      // lambda, tile layout
  T *gst = reinterpret_cast<T *>(smem + 2 * tile_smem_bytes<T>());  // g before its transform
  double *red = reinterpret_cast<double *>(smem + 3 * tile_smem_bytes<T>());
  const uint32_t r = blockIdx.y, tau = blockIdx.x;
  const int c = ft.cB, t = threadIdx.x;
  const uint64_t n = 1ull << ft.job.m;
  // element (t, l) of the tile is w = (row << LOGT) | (tau << c) | col, e = t + 256 l
  const uint32_t tcol = tau << c;  // fused sizes keep n <= 2^(2 LOGT - 5) < 2^32
  auto widx = [&](int l) -> uint32_t {
    const uint32_t e = t + (l << kLOGNT);
    return ((e >> c) << LOGT) | tcol | (e & ((1u << c) - 1));
  };
  const T *PT = reinterpret_cast<const T *>(ft.pT) + (uint64_t)r * n;
  T lam[L];
#pragma unroll
  for (int l = 0; l < L; ++l) lam[l] = PT[widx(l)];
  tile_wht<T>(lam, sm, c);
  const T zeta = (T)ft.job.zeta, eta = (T)ft.eta, zn = (T)(ft.job.zeta * (double)n);
  bool bad = false;
  T lds = T(0);
  double *LAM = ft.lam ? ft.lam + (uint64_t)r * n : nullptr;
#pragma unroll
  for (int l = 0; l < L; ++l) {
    const uint32_t wl = widx(l);
    T v = fmadd(zeta, lam[l], eta);
    if (wl == 0) v += zn;
    bad |= !(v > T(0));
    lds += fused_log(v);
    if (LAM) LAM[wl] = (double)v;
    lmv[fpad<T>(t + (l << kLOGNT))] = v;  // each thread reads back only its own entries
  }
  if (bad && ft.status) atomicOr(ft.status, (uint32_t)QK_STATUS_NOTPD);
  const double ldsum = block_sum((double)lds, red);
  if (t == 0) ft.ld[(uint64_t)r * ft.tiles + tau] = ldsum;
  const T inv_n = T(1) / (T)n;
  for (uint32_t q = 0; q < ft.nrhs; ++q) {
    const uint64_t v = (uint64_t)r * ft.nrhs + q;
    T *YT = reinterpret_cast<T *>(ft.yT) + v * n;
    T *GT = reinterpret_cast<T *>(ft.gT) + v * n;
    T y[L];
#pragma unroll
    for (int l = 0; l < L; ++l) y[l] = YT[widx(l)];
    T ylo[COMP ? L : 1];
    if constexpr (COMP) {
      const T *YL = reinterpret_cast<const T *>(ft.yL) + v * n;
#pragma unroll
      for (int l = 0; l < L; ++l) ylo[l] = YL[widx(l)];
      tile_wht2<T>(y, ylo, sm, gst, c);  // gst doubles as the lo tile here
    } else {
      tile_wht<T>(y, sm, c);
    }
    T quad = T(0), gs = T(0);
#pragma unroll
    for (int l = 0; l < L; ++l) {
      const int e = fpad<T>(t + (l << kLOGNT));  // this thread's own entries only
      const T lw = lmv[e];
      const T il = T(1) / lw;
      const T sc = inv_n * il;          // 1 / (n lambda_w)
      T ch = y[l] * sc;                 // c^_w = Y_w / (n lambda_w)
      const T a = ch * y[l];            // Y_w^2 / (n lambda_w)
      quad += a;
      const T gg = T(0.5) * (a - T(1)) * il;
      gs += gg;
      if constexpr (COMP) {
        // refinement: the exact residual of the division plus the forward transform's
        // own rounding error (the lo part), divided once more, corrects c^ before the
        // inverse transform: the solve then equals one step of iterative refinement
        // with an exact residual, up to the rounding of the inverse transform.
        const T nl = (T)n * lw;                       // exact: n is a power of two
        const T rho = fmadd(-ch, nl, y[l]);           // Y_hi - c^ n lambda_w
        ch = fmadd(rho + ylo[l], sc, ch);
      }
      y[l] = ch;
      gst[e] = gg;
    }
    tile_wht<T>(y, sm, c);
#pragma unroll
    for (int l = 0; l < L; ++l) YT[widx(l)] = y[l];
#pragma unroll
    for (int l = 0; l < L; ++l) y[l] = gst[fpad<T>(t + (l << kLOGNT))];
    tile_wht<T>(y, sm, c);
#pragma unroll
    for (int l = 0; l < L; ++l) GT[widx(l)] = y[l];
    const double sq = block_sum((double)quad, red);
    const double sg = block_sum((double)gs, red);
    if (t == 0) {
      ft.qg[(v * ft.tiles + tau) * 2 + 0] = sq;
      ft.qg[(v * ft.tiles + tau) * 2 + 1] = sg;
    }
  }
}

// ------------------------------------------------------------------ phase C
template <typename T, int FAM, int ALPHA>
__global__ void __launch_bounds__(kFNT, 2) k_fused_C(FTask ft) {
  constexpr int LOGT = FCfg<T>::LOGT, L = FCfg<T>::L;
  extern __shared__ __align__(16) unsigned char smem[];
  const ColJob &job = ft.job;
  const uint32_t d = job.d;
  double *wd;
  DiffTables tb;
  carve_tables<L>(smem, d, &wd, tb);
  T *wT = reinterpret_cast<T *>(wd);
  T *sm = reinterpret_cast<T *>(smem + align256(col_smem_bytes<L>(d)));
  double *red = reinterpret_cast<double *>(smem + align256(col_smem_bytes<L>(d)) + tile_smem_bytes<T>());
  const uint32_t v = blockIdx.y, r = v / ft.nrhs, tile = blockIdx.x;
  const uint64_t n = 1ull << job.m, base = (uint64_t)tile << LOGT;
  const int t = threadIdx.x;
  const T *YT = reinterpret_cast<const T *>(ft.yT) + (uint64_t)v * n + base;
  const T *GT = reinterpret_cast<const T *>(ft.gT) + (uint64_t)v * n + base;
  T cc[L], uu[L];
#pragma unroll
  for (int l = 0; l < L; ++l) cc[l] = YT[t + (l << kLOGNT)];
  tile_wht<T>(cc, sm, 0);
  if (ft.c) {
    T *Cv = reinterpret_cast<T *>(ft.c) + (uint64_t)v * n + base;
#pragma unroll
    for (int l = 0; l < L; ++l) Cv[t + (l << kLOGNT)] = cc[l];
  }
  if (!ft.grad) return;
#pragma unroll
  for (int l = 0; l < L; ++l) uu[l] = GT[t + (l << kLOGNT)];
  tile_wht<T>(uu, sm, 0);
  for (uint32_t q = t; q < d; q += kFNT) wT[q] = (T)job.w[q];
  build_all<T, FAM, ALPHA, L>(job, job.Ct + (size_t)r * d * 32, job.g, base, tb);
  const T *P = reinterpret_cast<const T *>(ft.p) + (uint64_t)r * n + base;
  const T zeta = (T)job.zeta;
  T k1[L];
  uint32_t bi[L];
  bool ok[L];
#pragma unroll
  for (int l = 0; l < L; ++l) {
    k1[l] = zeta * (T(1) + P[t + (l << kLOGNT)]);
    bi[l] = __brev((uint32_t)(base + t + (l << kLOGNT)));
    ok[l] = true;
    uu[l] *= k1[l];  // from here on uu holds u k1
  }
  __syncthreads();
  // u itself stays in the transform tile (sm) after tile_wht; each thread reads its own
  gradient_sweep<T, FAM, ALPHA, L>(job, tb, wT, bi, k1, uu, ok,
                                   [&](int l) { return sm[fpad<T>(t + (l << kLOGNT))]; }, red);
  __syncthreads();
  double *dst = ft.gr + ((uint64_t)v * ft.tiles + tile) * 2 * d;
  for (uint32_t q = t; q < 2 * d; q += kFNT) {
    double s = 0.0;
#pragma unroll
    for (int wp = 0; wp < kFNT / 32; ++wp) s += red[(size_t)wp * 2 * d + q];
    dst[q] = s;
  }
}

// ------------------------------------------------------------------ final
__global__ void __launch_bounds__(256) k_fused_final(FTask ft) {
  __shared__ double sh[32];
  const uint32_t v = blockIdx.x, r = v / ft.nrhs;
  const uint32_t tiles = ft.tiles, d = ft.job.d;
  const double n = (double)(1ull << ft.job.m), zeta = ft.job.zeta;
  double q = 0, gsum = 0, ld = 0, sp = 0, sy = 0;
  for (uint32_t b = threadIdx.x; b < tiles; b += blockDim.x) {
    q += ft.qg[((uint64_t)v * tiles + b) * 2 + 0];
    gsum += ft.qg[((uint64_t)v * tiles + b) * 2 + 1];
    ld += ft.ld[(uint64_t)r * tiles + b];
    sp += ft.sp[(uint64_t)r * tiles + b];
    sy += ft.sy[(uint64_t)v * tiles + b];
  }
  q = block_sum(q, sh);
  gsum = block_sum(gsum, sh);
  ld = block_sum(ld, sh);
  sp = block_sum(sp, sh);
  sy = block_sum(sy, sh);
  __shared__ double res[5];
  if (threadIdx.x == 0) {
    res[0] = q, res[1] = gsum, res[2] = ld, res[3] = sp, res[4] = sy;
  }
  __syncthreads();
  const double lam0 = zeta * (n + res[3]) + ft.eta;  // lambda_0 from the FP64 sum of p
  const double mfac = -zeta * res[4] / (lam0 * lam0);
  if (threadIdx.x == 0) {
    double *o = ft.out + (uint64_t)v * QK_MLL_NOUT;
    o[QK_MLL_QUAD] = res[0];
    o[QK_MLL_LOGDET] = res[2];
    o[QK_MLL_MLL] = -0.5 * res[0] - 0.5 * res[2] - 0.5 * n * 1.8378770664093454836;
    o[QK_MLL_MEAN] = zeta * res[4] / lam0;
    o[QK_MLL_VAR] = zeta * ((zeta * res[3] + ft.eta) / lam0);  // zeta (lambda_0 - zeta n) / lambda_0
  }
  if (!ft.grad) return;
  double *g = ft.grad + (uint64_t)v * (2 * d + 2);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (uint32_t j = warp; j < 2 * d; j += blockDim.x >> 5) {
    double s = 0.0;
    for (uint32_t b = lane; b < tiles; b += 32) s += ft.gr[((uint64_t)v * tiles + b) * 2 * d + j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
      if (j < d) g[j] = s;
      else g[d + 1 + (j - d)] = mfac * s;
    }
  }
  if (threadIdx.x == 0) {
    g[d] = res[1];
    g[2 * d + 1] = mfac;
  }
}

// ------------------------------------------------------------------ host side
bool fused_supported(const qk_task &t, int dtype) {
  if (t.k.family != QK_DSI || t.ps.kind != QK_NET_B2) return false;
  const int LOGT = dtype == QK_F64 ? FCfg<double>::LOGT : FCfg<float>::LOGT;
  return (int)t.m > LOGT && (int)t.m <= 2 * LOGT - 5;
}

static size_t fused_elem(int dtype) { return dtype == QK_F64 ? 8 : 4; }

size_t fused_ws_bytes(const qk_task &t, int dtype, int refine) {
  const int LOGT = dtype == QK_F64 ? FCfg<double>::LOGT : FCfg<float>::LOGT;
  const uint64_t R = t.ps.R, n = 1ull << t.m, tiles = n >> LOGT, nv = R * t.nrhs;
  const size_t e = fused_elem(dtype);
  size_t s = 2 * align256(e * R * n) + 2 * align256(e * nv * n);
  s += 2 * align256(8 * R * tiles) + align256(8 * nv * tiles) + align256(16 * nv * tiles);
  s += align256(8 * nv * tiles * 2 * (uint64_t)t.ps.d);
  if (refine > 0 && dtype == QK_F32) s += align256(e * nv * n);  // lo parts of y'
  return s;
}

template <typename T, int FAM, int ALPHA, bool COMP>
static int launch_fused_t(const FTask &ft, cudaStream_t st) {
  constexpr int L = FCfg<T>::L;
  const uint32_t R = ft.job.nr, d = ft.job.d;
  const size_t colb = align256(col_smem_bytes<L>(d));
  // phase A keeps a second tile for the lo parts when compensating
  const size_t smA = colb + (COMP ? 2 : 1) * tile_smem_bytes<T>() + 32 * sizeof(double);
  const size_t smB = 3 * tile_smem_bytes<T>() + 32 * sizeof(double);
  const size_t smC = colb + tile_smem_bytes<T>() + (size_t)(kFNT / 32) * 2 * d * sizeof(double);
  smem_optin<k_fused_A<T, FAM, ALPHA, COMP>>(smA);
  smem_optin<k_fused_B<T, COMP>>(smB);
  smem_optin<k_fused_C<T, FAM, ALPHA>>(smC);
  k_fused_A<T, FAM, ALPHA, COMP><<<dim3(ft.tiles, R), kFNT, smA, st>>>(ft);
  int rc = check_launch("fused A");
  if (rc) return rc;
  k_fused_B<T, COMP><<<dim3(ft.tiles, R), kFNT, smB, st>>>(ft);
  if ((rc = check_launch("fused B"))) return rc;
  if (ft.c || ft.grad) {
    k_fused_C<T, FAM, ALPHA><<<dim3(ft.tiles, R * ft.nrhs), kFNT, smC, st>>>(ft);
    if ((rc = check_launch("fused C"))) return rc;
  }
  k_fused_final<<<R * ft.nrhs, 256, 0, st>>>(ft);
  return check_launch("fused final");
}

template <typename T, bool COMP>
static int dispatch_fused(const FTask &ft, cudaStream_t st) {
  switch (ft.job.alpha) {
    case 1: return launch_fused_t<T, 0, 1, COMP>(ft, st);
    case 2: return launch_fused_t<T, 0, 2, COMP>(ft, st);
    case 3: return launch_fused_t<T, 0, 3, COMP>(ft, st);
    case 4: return launch_fused_t<T, 0, 4, COMP>(ft, st);
    default: return fail(QK_EINVAL, "DSI order must be 1..4");
  }
}

int run_fused(const qk_task &t, const ColJob &job, int dtype, int refine, void *ws, uint32_t *status,
              cudaStream_t st) {
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
  // FP64 needs no refinement; FP32 with refine >= 1 runs the compensated variant
  // (one exact-residual step; further steps change nothing at FP32 resolution)
  if (dtype == QK_F64) return dispatch_fused<double, false>(ft, st);
  if (refine > 0) {
    ft.yL = p;
    return dispatch_fused<float, true>(ft, st);
  }
  return dispatch_fused<float, false>(ft, st);
}

}  // namespace qk
