// Device code of the fused net pipeline (phases A, B, C, final) and of its persistent
// whole-plan schedule, with their launch templates.  Shared by qk_fused.cu (host side and
// the batched WHT) and the qk_fused_*.cu files, each of which instantiates the kernels of
// one precision so that the translation units compile in parallel.
//
// Fused solve + marginal log-likelihood + gradient for digital nets with DSI
// kernels (arXiv 2502.14256, Sec. 5.3-5.4), n = 2^m with LOGT < m <= 2 LOGT - LOGL
// (2^13 < n <= 2^21 in FP32, 2^12 < n <= 2^20 in FP64).
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
#pragma once

#include <cmath>
#include <type_traits>
#include <utility>
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
// Largest m of the two-pass split: the column tiles need at least L contiguous elements
// (c = 2 LOGT - m >= LOGL).
template <typename T> constexpr int two_pass_max_m() { return 2 * FCfg<T>::LOGT - FCfg<T>::LOGL; }

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
  void *pTL;                            // (R, n): low parts of p' (float-float first column)
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

// s + e tracks a sum exactly up to the rounding of e: the error of each addition to s
// (TwoSum) is accumulated in e.  (Kahan's single correction term is not enough here: its
// s - c keeps an error of ~u sum|v| per partial, and Sum y of a centred integrand is a
// small difference of large terms.)
template <typename T>
__device__ __forceinline__ void ff_add(T &s, T &e, T v) {
  T t, r;
  two_sum(s, v, t, r);
  s = t;
  e += r;
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

// ---------------------------------------------------------- register-tiled WHT
// Three thread layouts of a 2^LOGT-element tile (L = 2^LOGL elements per thread,
// 256 threads):
//   L0: e = t + 256 l                                   (l carries bits [8, LOGT))
//   L1: e = L t + l                                     (l carries bits [0, LOGL))
//   L2: e = (t mod L) + L l + L^2 (t div L)             (l carries bits [LOGL, 2 LOGL))
// L0 and L2 give coalesced global accesses.  Every transformed bit is butterflied in
// exactly one layout: [c, LOGL) in L1, [max(c, LOGL), 8) in L2, [max(c, 8), LOGT) in
// L0, with conflict-free transposes through a tile padded by 4 words per L elements
// (L1 side in 128-bit vectors).
template <typename T> struct Lay {
  static constexpr int L = FCfg<T>::L, LOGL = FCfg<T>::LOGL, LOGT = FCfg<T>::LOGT;
  static constexpr int PADE = 16 / sizeof(T);  // 4 words per row of L elements
  static constexpr int VEC = 16 / sizeof(T);   // elements per 128-bit access
};
template <typename T>
__host__ __device__ constexpr size_t xtile_bytes() {
  return (size_t)((1 << FCfg<T>::LOGT) + Lay<T>::PADE * ((1 << FCfg<T>::LOGT) >> FCfg<T>::LOGL)) * sizeof(T);
}
template <typename T>
__device__ __forceinline__ int xpad(int e) { return e + Lay<T>::PADE * (e >> Lay<T>::LOGL); }
template <typename T>
__device__ __forceinline__ int e_of(int lay, int t, int l) {
  constexpr int LOGL = Lay<T>::LOGL, L = Lay<T>::L;
  if (lay == 0) return t + (l << 8);
  if (lay == 1) return (t << LOGL) + l;
  return (t & (L - 1)) + (l << LOGL) + ((t >> LOGL) << (2 * LOGL));
}

// Two FP32 butterflies in one packed instruction pair: (a0, a1) +- (b0, b1) (sm_100+ f32x2).
__device__ __forceinline__ void bfly_x2(float &a0, float &a1, float &b0, float &b1) {
  unsigned long long A, B, S, D;
  asm("mov.b64 %0, {%1, %2};" : "=l"(A) : "f"(a0), "f"(a1));
  asm("mov.b64 %0, {%1, %2};" : "=l"(B) : "f"(b0), "f"(b1));
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(S) : "l"(A), "l"(B));
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(D) : "l"(A), "l"(B));
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a0), "=f"(a1) : "l"(S));
  asm("mov.b64 {%0, %1}, %2;" : "=f"(b0), "=f"(b1) : "l"(D));
}

// Butterflies on the register bits h whose tile bit (bit0 + h) lies in [lo, hi).  FP32
// stages on bits h >= 1 pair neighbouring registers into packed f32x2 adds (the same
// roundings as scalar adds, half the instructions).
template <typename T>
__device__ __forceinline__ void reg_stages(T (&v)[FCfg<T>::L], int bit0, int lo, int hi) {
  constexpr int L = FCfg<T>::L, LOGL = FCfg<T>::LOGL;
#pragma unroll
  for (int h = 0; h < LOGL; ++h) {
    if (bit0 + h >= lo && bit0 + h < hi) {
      if constexpr (sizeof(T) == 4) {
        if (h > 0) {
#pragma unroll
          for (int q = 0; q < L; q += 2)
            if (!(q & (1 << h))) bfly_x2(v[q], v[q + 1], v[q | (1 << h)], v[(q | (1 << h)) + 1]);
          continue;
        }
      }
#pragma unroll
      for (int q = 0; q < L; ++q)
        if (!(q & (1 << h))) {
          const T a = v[q], b = v[q | (1 << h)];
          v[q] = a + b;
          v[q | (1 << h)] = a - b;
        }
    }
  }
}

// Padded tile index of element (t, l) of a layout = base(t) + stride * l.
template <typename T>
__device__ __forceinline__ int xbase(int lay, int t) {
  constexpr int LOGL = Lay<T>::LOGL, L = Lay<T>::L, P = Lay<T>::PADE;
  if (lay == 0) return t + P * (t >> LOGL);
  if (lay == 1) return (t << LOGL) + P * t;
  return (t & (L - 1)) + ((t >> LOGL) << (2 * LOGL)) + P * ((t >> LOGL) << LOGL);
}
template <typename T>
__host__ __device__ constexpr int xstride(int lay) {
  return lay == 0 ? 256 + Lay<T>::PADE * (256 >> Lay<T>::LOGL) : (lay == 1 ? 1 : Lay<T>::L + Lay<T>::PADE);
}

// v (layout `from`) -> v (layout `to`) through the padded tile.
template <typename T>
__device__ __forceinline__ void xpose(T (&v)[FCfg<T>::L], T *sm, int from, int to) {
  constexpr int L = FCfg<T>::L, V = Lay<T>::VEC;
  using V4 = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
  const int t = threadIdx.x;
  T *w = sm + xbase<T>(from, t);
  if (from == 1) {
#pragma unroll
    for (int l = 0; l < L; l += V) *reinterpret_cast<V4 *>(w + l) = *reinterpret_cast<V4 *>(&v[l]);
  } else if (from == 0) {
#pragma unroll
    for (int l = 0; l < L; ++l) w[l * xstride<T>(0)] = v[l];
  } else {
#pragma unroll
    for (int l = 0; l < L; ++l) w[l * xstride<T>(2)] = v[l];
  }
  __syncthreads();
  const T *rd = sm + xbase<T>(to, t);
  if (to == 1) {
#pragma unroll
    for (int l = 0; l < L; l += V) *reinterpret_cast<V4 *>(&v[l]) = *reinterpret_cast<const V4 *>(rd + l);
  } else if (to == 0) {
#pragma unroll
    for (int l = 0; l < L; ++l) v[l] = rd[l * xstride<T>(0)];
  } else {
#pragma unroll
    for (int l = 0; l < L; ++l) v[l] = rd[l * xstride<T>(2)];
  }
  __syncthreads();
}

// ------------------------------------- FP32 full-tile transposes through a warp-major tile
// An FP32 tile (8192 elements, 256 threads x 32) exchanges the lane bits of layout L0 with
// its register bits inside each warp (a per-warp region of the tile, __syncwarp), and only
// the warp bits across the CTA (__syncthreads): two CTA barriers per full-tile transform
// instead of four.  Element e sits at ((e >> 5) & 7) 1152 + (e >> 8) 36 + (e & 31): region =
// warp bits (5-7), row = bits 8-12, column = lane bits, rows padded to 36 words so that
// 128-bit row accesses of 8 lanes hit distinct banks.  Layout L1w: thread (lane, w) holds
// e = l + 32 w + 256 lane in register l (bits 0-4), i.e. row `lane` of region w.  Every
// function ends with its reads complete in all warps where a later write could reach them.
constexpr int kWReg = 1152, kWRow = 36;

__device__ __forceinline__ void xw_L0_to_L1w(float (&v)[32], float *sm) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float *rg = sm + w * kWReg;
#pragma unroll
  for (int l = 0; l < 32; ++l) rg[l * kWRow + lane] = v[l];  // e = lane + 32 w + 256 l
  __syncwarp();
#pragma unroll
  for (int l = 0; l < 32; l += 4)
    *reinterpret_cast<float4 *>(&v[l]) = *reinterpret_cast<const float4 *>(rg + lane * kWRow + l);
}

__device__ __forceinline__ void xw_L1w_to_L2(float (&v)[32], float *sm) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float *row = sm + w * kWReg + lane * kWRow;
#pragma unroll
  for (int l = 0; l < 32; l += 4) *reinterpret_cast<float4 *>(row + l) = *reinterpret_cast<const float4 *>(&v[l]);
  __syncthreads();
#pragma unroll
  for (int l = 0; l < 32; ++l) v[l] = sm[(l & 7) * kWReg + ((l >> 3) + 4 * w) * kWRow + lane];  // e = lane + 32 l + 1024 w
  __syncthreads();
}

__device__ __forceinline__ void xw_L2_to_L1w(float (&v)[32], float *sm) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int l = 0; l < 32; ++l) sm[(l & 7) * kWReg + ((l >> 3) + 4 * w) * kWRow + lane] = v[l];
  __syncthreads();
  const float *row = sm + w * kWReg + lane * kWRow;
#pragma unroll
  for (int l = 0; l < 32; l += 4) *reinterpret_cast<float4 *>(&v[l]) = *reinterpret_cast<const float4 *>(row + l);
}

__device__ __forceinline__ void xw_L1w_to_L0(float (&v)[32], float *sm) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float *rg = sm + w * kWReg;
#pragma unroll
  for (int l = 0; l < 32; l += 4)
    *reinterpret_cast<float4 *>(rg + lane * kWRow + l) = *reinterpret_cast<const float4 *>(&v[l]);
  __syncwarp();
#pragma unroll
  for (int l = 0; l < 32; ++l) v[l] = rg[l * kWRow + lane];
  __syncthreads();
}

// Full tile WHT (bits [0, LOGT)): from L0 to L2 (dir 0) or from L2 to L0 (dir 1).
template <typename T>
__device__ __forceinline__ void xwht_full(T (&v)[FCfg<T>::L], T *sm, int dir) {
  constexpr int LOGL = Lay<T>::LOGL, LOGT = Lay<T>::LOGT;
  if constexpr (sizeof(T) == 4) {  // warp-major tile: the same butterflies in the same order
    if (dir == 0) {
      reg_stages<T>(v, 8, 8, LOGT);
      xw_L0_to_L1w(v, sm);
      reg_stages<T>(v, 0, 0, LOGL);
      xw_L1w_to_L2(v, sm);
      reg_stages<T>(v, LOGL, LOGL, 8);
    } else {
      reg_stages<T>(v, LOGL, LOGL, 8);
      xw_L2_to_L1w(v, sm);
      reg_stages<T>(v, 0, 0, LOGL);
      xw_L1w_to_L0(v, sm);
      reg_stages<T>(v, 8, 8, LOGT);
    }
    return;
  }
  if (dir == 0) {
    reg_stages<T>(v, 8, 8, LOGT);
    xpose<T>(v, sm, 0, 1);
    reg_stages<T>(v, 0, 0, LOGL);
    xpose<T>(v, sm, 1, 2);
    reg_stages<T>(v, LOGL, LOGL, 8);
  } else {
    reg_stages<T>(v, LOGL, LOGL, 8);
    xpose<T>(v, sm, 2, 1);
    reg_stages<T>(v, 0, 0, LOGL);
    xpose<T>(v, sm, 1, 0);
    reg_stages<T>(v, 8, 8, LOGT);
  }
}

// Column-tile WHT on bits [c, LOGT), c >= LOGL: from L0 to L2 (dir 0) or L2 to L0 (dir 1).
template <typename T>
__device__ __forceinline__ void xwht_col(T (&v)[FCfg<T>::L], T *sm, int c, int dir) {
  constexpr int LOGL = Lay<T>::LOGL, LOGT = Lay<T>::LOGT;
  if (dir == 0) {
    reg_stages<T>(v, 8, c, LOGT);
    xpose<T>(v, sm, 0, 2);
    reg_stages<T>(v, LOGL, c, 8);
  } else {
    reg_stages<T>(v, LOGL, c, 8);
    xpose<T>(v, sm, 2, 0);
    reg_stages<T>(v, 8, c, LOGT);
  }
}

// Packed FP32 pairs (sm_100+ f32x2 adds): the same roundings as the scalar operations.
__device__ __forceinline__ unsigned long long pk2(float a, float b) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void upk2(unsigned long long v, float &a, float &b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ unsigned long long add2(unsigned long long x, unsigned long long y) {
  unsigned long long r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(x), "l"(y));
  return r;
}
__device__ __forceinline__ unsigned long long sub2(unsigned long long x, unsigned long long y) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(x), "l"(y));
  return r;
}

// Two compensated butterflies (registers q and q + 1 of the same stage) in packed
// arithmetic: exactly cbfly applied to each.
__device__ __forceinline__ void cbfly_x2(float &ah0, float &ah1, float &al0, float &al1, float &bh0, float &bh1,
                                         float &bl0, float &bl1) {
  const unsigned long long A = pk2(ah0, ah1), B = pk2(bh0, bh1), Al = pk2(al0, al1), Bl = pk2(bl0, bl1);
  const unsigned long long S = add2(A, B), bb = sub2(S, A);
  const unsigned long long e1 = add2(sub2(A, sub2(S, bb)), sub2(B, bb));  // TwoSum(a, b)
  const unsigned long long D = sub2(A, B), dd = sub2(D, A);
  const unsigned long long e2 = sub2(sub2(A, sub2(D, dd)), add2(B, dd));  // TwoSum(a, -b)
  const unsigned long long SL = add2(add2(Al, Bl), e1), DL = add2(sub2(Al, Bl), e2);
  upk2(S, ah0, ah1);
  upk2(SL, al0, al1);
  upk2(D, bh0, bh1);
  upk2(DL, bl0, bl1);
}

template <typename T>
__device__ __forceinline__ void reg_stages2(T (&vh)[FCfg<T>::L], T (&vl)[FCfg<T>::L], int bit0, int lo, int hi) {
  constexpr int L = FCfg<T>::L, LOGL = FCfg<T>::LOGL;
#pragma unroll
  for (int h = 0; h < LOGL; ++h) {
    if (bit0 + h >= lo && bit0 + h < hi) {
      if constexpr (sizeof(T) == 4) {
        if (h > 0) {
#pragma unroll
          for (int q = 0; q < L; q += 2)
            if (!(q & (1 << h))) {
              const int p = q | (1 << h);
              cbfly_x2(vh[q], vh[q + 1], vl[q], vl[q + 1], vh[p], vh[p + 1], vl[p], vl[p + 1]);
            }
          continue;
        }
      }
#pragma unroll
      for (int q = 0; q < L; ++q)
        if (!(q & (1 << h))) cbfly(vh[q], vl[q], vh[q | (1 << h)], vl[q | (1 << h)]);
    }
  }
}

// Compensated (hi, lo) versions of xwht_full / xwht_col; sml: the padded tile for the lo
// parts (may be sm itself: each transpose ends with a barrier, so the lo parts then pass
// through the same tile after the hi parts).
template <typename T>
__device__ __forceinline__ void xwht_full2(T (&vh)[FCfg<T>::L], T (&vl)[FCfg<T>::L], T *sm, T *sml, int dir) {
  constexpr int LOGL = Lay<T>::LOGL, LOGT = Lay<T>::LOGT;
  if constexpr (sizeof(T) == 4) {  // warp-major tile (sm); the hi then the lo parts pass through it
    (void)sml;
    if (dir == 0) {
      reg_stages2<T>(vh, vl, 8, 8, LOGT);
      xw_L0_to_L1w(vh, sm);
      __syncwarp();  // every lane has read its hi row before the lo parts overwrite the region
      xw_L0_to_L1w(vl, sm);
      reg_stages2<T>(vh, vl, 0, 0, LOGL);
      xw_L1w_to_L2(vh, sm);
      xw_L1w_to_L2(vl, sm);
      reg_stages2<T>(vh, vl, LOGL, LOGL, 8);
    } else {
      reg_stages2<T>(vh, vl, LOGL, LOGL, 8);
      xw_L2_to_L1w(vh, sm);
      __syncthreads();  // every warp has read its hi rows before the lo parts fill the tile
      xw_L2_to_L1w(vl, sm);
      reg_stages2<T>(vh, vl, 0, 0, LOGL);
      __syncthreads();
      xw_L1w_to_L0(vh, sm);
      xw_L1w_to_L0(vl, sm);
      reg_stages2<T>(vh, vl, 8, 8, LOGT);
    }
    return;
  }
  const int a = dir == 0 ? 0 : 2, b = dir == 0 ? 2 : 0;
  const int a0 = dir == 0 ? 8 : LOGL, a1 = dir == 0 ? LOGT : 8, b0 = dir == 0 ? LOGL : 8, b1 = dir == 0 ? 8 : LOGT;
  reg_stages2<T>(vh, vl, a0, a0, a1);
  xpose<T>(vh, sm, a, 1);
  xpose<T>(vl, sml, a, 1);
  reg_stages2<T>(vh, vl, 0, 0, LOGL);
  xpose<T>(vh, sm, 1, b);
  xpose<T>(vl, sml, 1, b);
  reg_stages2<T>(vh, vl, b0, b0, b1);
}

template <typename T>
__device__ __forceinline__ void xwht_col2(T (&vh)[FCfg<T>::L], T (&vl)[FCfg<T>::L], T *sm, T *sml, int c, int dir) {
  constexpr int LOGL = Lay<T>::LOGL, LOGT = Lay<T>::LOGT;
  if (dir == 0) {
    reg_stages2<T>(vh, vl, 8, c, LOGT);
    xpose<T>(vh, sm, 0, 2);
    xpose<T>(vl, sml, 0, 2);
    reg_stages2<T>(vh, vl, LOGL, c, 8);
  } else {
    reg_stages2<T>(vh, vl, LOGL, c, 8);
    xpose<T>(vh, sm, 2, 0);
    xpose<T>(vl, sml, 2, 0);
    reg_stages2<T>(vh, vl, 8, c, LOGT);
  }
}

// log lambda for the log-determinant: FP32 tiles take the hardware log2 approximation
// (absolute error ~2^-22 per term, about 1e-8 relative on a log det summed over 2^20
// eigenvalues even if every term erred the same way; the sum itself is FP64), FP64 tiles
// the full-precision log.  1 / lambda likewise: the FP32 tiles' reciprocal estimate plus one
// Newton step (within 1 ulp); the solve's exact-residual correction below absorbs it.
__device__ __forceinline__ float fused_log(float v) { return __logf(v); }
__device__ __forceinline__ double fused_log(double v) { return log(v); }
__device__ __forceinline__ float fused_rcp(float v) {
  const float r = rcp_approx(v);
  return fmaf(fmaf(-v, r, 1.f), r, r);
}
__device__ __forceinline__ double fused_rcp(double v) { return 1.0 / v; }

// ------------------------------------------------------------------ phase A
template <typename T, int FAM, int ALPHA, bool COMP, bool WIDE>
__device__ __forceinline__ void fused_A_item(const FTask &ft, uint32_t r, uint32_t tile, unsigned char *smem) {
  static_assert(!WIDE || (COMP && sizeof(T) == 4), "the float-float column runs on the compensated FP32 path");
  constexpr int LOGT = FCfg<T>::LOGT, L = FCfg<T>::L;
  const ColJob &job = ft.job;
  const uint32_t d = job.d;
  double *wd;
  DiffTables tb;
  carve_tables<L>(smem, d, &wd, tb);
  T *wT = reinterpret_cast<T *>(wd);
  T *sm = reinterpret_cast<T *>(smem + align256(col_smem_bytes<L>(d)));
  T *sml = sm;  // the compensated transforms pass the lo parts through the same tile
  double *red = reinterpret_cast<double *>(smem + align256(col_smem_bytes<L>(d)) + xtile_bytes<T>());
  const uint64_t n = 1ull << job.m, base = (uint64_t)tile << LOGT;
  const int t = threadIdx.x;
  if constexpr (WIDE) {
    float2 *wff = reinterpret_cast<float2 *>(wd);
    for (uint32_t q = t; q < d; q += kFNT) wff[q] = ff_split(job.w[q]);
    build_all_ff<FAM, ALPHA, L>(job, job.Ct + (size_t)r * d * 32, job.g, base, tb);
  } else {
    for (uint32_t q = t; q < d; q += kFNT) wT[q] = (T)job.w[q];
    build_all<T, FAM, ALPHA, L>(job, job.Ct + (size_t)r * d * 32, job.g, base, tb);
  }
  __syncthreads();
  uint32_t bi[L];
#pragma unroll
  for (int l = 0; l < L; ++l) bi[l] = __brev((uint32_t)(base + t + (l << kLOGNT)));
  T p[L];
  T pl[WIDE ? L : 1];  // float-float column: low parts
  if constexpr (WIDE) column_sweep_ff<FAM, ALPHA, L>(job, tb, reinterpret_cast<const float2 *>(wd), bi, p, pl);
  else column_sweep<T, FAM, ALPHA, L>(job, tb, wT, bi, p);
  T *P = reinterpret_cast<T *>(ft.p) + (uint64_t)r * n + base;
  T *PT = reinterpret_cast<T *>(ft.pT) + (uint64_t)r * n + base;
  if constexpr (WIDE) {
#pragma unroll
    for (int l = 0; l < L; ++l) P[t + (l << kLOGNT)] = p[l];  // phase C's k_1 needs p to FP32 only
    xwht_full2<T>(p, pl, sm, sml, 0);  // L0 -> L2, compensated
    // the tile sum of p is the transform's element 0 (thread 0, register 0 of layout L2),
    // already a compensated pair: no separate sum
    if (t == 0) ft.sp[(uint64_t)r * ft.tiles + tile] = f2d_exact(p[0]) + f2d_exact(pl[0]);
    T *PTL = reinterpret_cast<T *>(ft.pTL) + (uint64_t)r * n + base;
#pragma unroll
    for (int l = 0; l < L; ++l) {
      PT[e_of<T>(2, t, l)] = p[l];
      PTL[e_of<T>(2, t, l)] = pl[l];
    }
  } else {
    T ps = T(0), pe = T(0);  // compensated thread partial: the sum cancels
#pragma unroll
    for (int l = 0; l < L; ++l) {
      P[t + (l << kLOGNT)] = p[l];  // phase C's k_1 needs p to FP32 precision only
      ff_add(ps, pe, p[l]);
    }
    const double sps = block_sum_c(ps, pe, red);
    if (t == 0) ft.sp[(uint64_t)r * ft.tiles + tile] = sps;
    xwht_full<T>(p, sm, 0);  // L0 -> L2
#pragma unroll
    for (int l = 0; l < L; ++l) PT[e_of<T>(2, t, l)] = p[l];
  }
  for (uint32_t q = 0; q < ft.nrhs; ++q) {
    const uint64_t v = (uint64_t)r * ft.nrhs + q;
    const T *Y = reinterpret_cast<const T *>(ft.y) + v * n + base;
    T yv[L];
#pragma unroll
    for (int l = 0; l < L; ++l) yv[l] = Y[t + (l << kLOGNT)];
    if constexpr (!COMP) {
      T ys = T(0), ye = T(0);
#pragma unroll
      for (int l = 0; l < L; ++l) ff_add(ys, ye, yv[l]);
      const double sys = block_sum_c(ys, ye, red);
      if (t == 0) ft.sy[v * ft.tiles + tile] = sys;
    }
    T *YT = reinterpret_cast<T *>(ft.yT) + v * n + base;
    if constexpr (COMP) {
      T yl[L];
#pragma unroll
      for (int l = 0; l < L; ++l) yl[l] = T(0);
      xwht_full2<T>(yv, yl, sm, sml, 0);
      // the tile sum of y: element 0 of the compensated transform (a float-float pair)
      if (t == 0) ft.sy[v * ft.tiles + tile] = f2d_exact(yv[0]) + f2d_exact(yl[0]);
      T *YL = reinterpret_cast<T *>(ft.yL) + v * n + base;
#pragma unroll
      for (int l = 0; l < L; ++l) {
        YT[e_of<T>(2, t, l)] = yv[l];
        YL[e_of<T>(2, t, l)] = yl[l];
      }
    } else {
      xwht_full<T>(yv, sm, 0);
#pragma unroll
      for (int l = 0; l < L; ++l) YT[e_of<T>(2, t, l)] = yv[l];
    }
  }
}

template <typename T, int FAM, int ALPHA, bool COMP, bool WIDE>
__global__ void __launch_bounds__(kFNT, WIDE ? 1 : 3) k_fused_A(FTask ft) {
  extern __shared__ __align__(16) unsigned char smem[];
  fused_A_item<T, FAM, ALPHA, COMP, WIDE>(ft, blockIdx.y, blockIdx.x, smem);
}

// ------------------------------------------------------------------ phase B
template <typename T, bool COMP, bool WIDE>
__device__ __forceinline__ void fused_B_item(const FTask &ft, uint32_t r, uint32_t tau, unsigned char *smem,
                                             uint32_t *status) {
  constexpr int LOGT = FCfg<T>::LOGT, L = FCfg<T>::L;
  T *sm = reinterpret_cast<T *>(smem);
  T *lmv = reinterpret_cast<T *>(smem + xtile_bytes<T>());      // lambda (own entries)
  T *gst = reinterpret_cast<T *>(smem + 2 * xtile_bytes<T>());  // g (own entries) / lo tile
  double *red = reinterpret_cast<double *>(smem + 3 * xtile_bytes<T>());
  const int c = ft.cB, t = threadIdx.x;
  const uint64_t n = 1ull << ft.job.m;
  // element (t, l) of the tile is w = (row << LOGT) | (tau << c) | col, e = t + 256 l
  const uint32_t tcol = tau << c;  // fused sizes keep n <= 2^(2 LOGT - LOGL) < 2^32
  // tile element e -> index in the vector; wi0 / wi2: the elements (t, l) of layouts L0 / L2
  auto widx = [&](uint32_t e) -> uint32_t { return ((e >> c) << LOGT) | tcol | (e & ((1u << c) - 1)); };
  // L0 element (t, l) has e = t + 256 l; for c <= 8 its index is w0 + l * S0
  const bool lin = c <= kLOGNT;
  const uint32_t w0 = widx((uint32_t)t), S0 = 1u << (LOGT + kLOGNT - c);
  auto wi0 = [&](int l) -> uint32_t { return lin ? w0 + (uint32_t)l * S0 : widx(e_of<T>(0, t, l)); };
  auto wi2 = [&](int l) -> uint32_t { return widx(e_of<T>(2, t, l)); };
  const T *PT = reinterpret_cast<const T *>(ft.pT) + (uint64_t)r * n;
  T lam[L];
#pragma unroll
  for (int l = 0; l < L; ++l) lam[l] = __ldcg(&PT[wi0(l)]);
  T laml[WIDE ? L : 1];  // float-float column: low parts of the transform
  if constexpr (WIDE) {
    const T *PTL = reinterpret_cast<const T *>(ft.pTL) + (uint64_t)r * n;
#pragma unroll
    for (int l = 0; l < L; ++l) laml[l] = __ldcg(&PTL[wi0(l)]);
    xwht_col2<T>(lam, laml, sm, gst, c, 0);  // L0 -> L2, compensated (gst: the lo tile)
  } else {
    xwht_col<T>(lam, sm, c, 0);  // L0 -> L2
  }
  const T zeta = (T)ft.job.zeta, eta = (T)ft.eta, zn = (T)(ft.job.zeta * (double)n);
  bool bad = false;
  T lds = T(0);
  double *LAM = ft.lam ? ft.lam + (uint64_t)r * n : nullptr;
  bool floored = false;
#pragma unroll
  for (int l = 0; l < L; ++l) {
    T v;
    if constexpr (WIDE) {
      // lambda = zeta (H p) + zeta n [w = 0] + eta in float-float, then rounded once: the
      // small eigenvalues keep FP32 relative precision
      const float2 zf = ff_split(ft.job.zeta), ef = ff_split(ft.eta);
      FF<float> x = ff_mul(FF<float>{lam[l], laml[l]}, FF<float>{zf.x, zf.y});
      if (l == 0 && t == 0 && tau == 0) {
        const float2 nf = ff_split(ft.job.zeta * (double)n);
        x = ff_add(x, FF<float>{nf.x, nf.y});
      }
      x = ff_add(x, FF<float>{ef.x, ef.y});
      if (eta > T(0) && !(x.h >= eta)) {  // K + eta I has no eigenvalue below eta: rounding
        x = FF<float>{ef.x, ef.y};
        floored = true;
      }
      v = x.h;
      if (LAM) LAM[wi2(l)] = f2d_exact(x.h) + f2d_exact(x.l);
    } else {
      v = fmadd(zeta, lam[l], eta);
      if (l == 0 && t == 0 && tau == 0) v += zn;  // w = 0 (e = 0 in every layout)
      if (eta > T(0) && !(v >= eta)) {  // K + eta I has no eigenvalue below eta: rounding
        v = eta;
        floored = true;
      }
      if (LAM) LAM[wi2(l)] = f2d_exact(v);
    }
    bad |= !(v > T(0));
    lds += fused_log(v);
    lmv[t + (l << kLOGNT)] = v;  // each thread reads back only its own entries
  }
  if (bad && status) atomicOr(status, (uint32_t)QK_STATUS_NOTPD);
  if (floored && status) atomicOr(status, (uint32_t)QK_STATUS_FLOOR);
  const double ldsum = block_sum_c(lds, T(0), red);
  if (t == 0) ft.ld[(uint64_t)r * ft.tiles + tau] = ldsum;
  const T inv_n = T(1) / (T)n;
  for (uint32_t q = 0; q < ft.nrhs; ++q) {
    const uint64_t v = (uint64_t)r * ft.nrhs + q;
    T *YT = reinterpret_cast<T *>(ft.yT) + v * n;
    T *GT = reinterpret_cast<T *>(ft.gT) + v * n;
    T y[L];
#pragma unroll
    for (int l = 0; l < L; ++l) y[l] = __ldcg(&YT[wi0(l)]);
    T ylo[COMP ? L : 1];
    if constexpr (COMP) {
      const T *YL = reinterpret_cast<const T *>(ft.yL) + v * n;
#pragma unroll
      for (int l = 0; l < L; ++l) ylo[l] = __ldcg(&YL[wi0(l)]);
      xwht_col2<T>(y, ylo, sm, gst, c, 0);  // gst doubles as the lo tile here
    } else {
      xwht_col<T>(y, sm, c, 0);
    }
    T quad = T(0), gs = T(0);
#pragma unroll
    for (int l = 0; l < L; ++l) {
      const int e = t + (l << kLOGNT);  // this thread's own entries only
      const T lw = lmv[e];
      const T il = fused_rcp(lw);
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
    // inverse high bits of c^, then of g: one copy of the transform's code for both (the
    // kernel's time goes to instruction fetch more than to arithmetic)
#pragma unroll 1
    for (int k = 0; k < 2; ++k) {
      if (k) {
#pragma unroll
        for (int l = 0; l < L; ++l) y[l] = gst[t + (l << kLOGNT)];
      }
      xwht_col<T>(y, sm, c, 1);  // L2 -> L0
      T *dst = k ? GT : YT;
#pragma unroll
      for (int l = 0; l < L; ++l) dst[wi0(l)] = y[l];
    }
    const double sq = block_sum_c(quad, T(0), red);
    const double sg = block_sum_c(gs, T(0), red);
    if (t == 0) {
      ft.qg[(v * ft.tiles + tau) * 2 + 0] = sq;
      ft.qg[(v * ft.tiles + tau) * 2 + 1] = sg;
    }
  }
}

template <typename T, bool COMP, bool WIDE>
__global__ void __launch_bounds__(kFNT, 2) k_fused_B(FTask ft) {
  extern __shared__ __align__(16) unsigned char smem[];
  fused_B_item<T, COMP, WIDE>(ft, blockIdx.y, blockIdx.x, smem, ft.status);
}

// ------------------------------------------------------------------ phase C
template <typename T, int FAM, int ALPHA>
__device__ __forceinline__ void fused_C_item(const FTask &ft, uint32_t v, uint32_t tile, unsigned char *smem) {
  constexpr int LOGT = FCfg<T>::LOGT, L = FCfg<T>::L;
  const ColJob &job = ft.job;
  const uint32_t d = job.d;
  double *wd;
  DiffTables tb;
  carve_tables<L>(smem, d, &wd, tb);
  T *wT = reinterpret_cast<T *>(wd);
  T *sm = reinterpret_cast<T *>(smem + align256(col_smem_bytes<L>(d)));
  double *red = reinterpret_cast<double *>(smem + align256(col_smem_bytes<L>(d)) + xtile_bytes<T>());
  const uint32_t r = v / ft.nrhs;
  const uint64_t n = 1ull << job.m, base = (uint64_t)tile << LOGT;
  const int t = threadIdx.x;
  const T *YT = reinterpret_cast<const T *>(ft.yT) + (uint64_t)v * n + base;
  const T *GT = reinterpret_cast<const T *>(ft.gT) + (uint64_t)v * n + base;
  T cc[L], uu[L];
#pragma unroll
  for (int l = 0; l < L; ++l) cc[l] = __ldcg(&YT[e_of<T>(2, t, l)]);
  xwht_full<T>(cc, sm, 1);  // L2 -> L0: the thread's own points
  if (ft.c) {
    T *Cv = reinterpret_cast<T *>(ft.c) + (uint64_t)v * n + base;
#pragma unroll
    for (int l = 0; l < L; ++l) Cv[t + (l << kLOGNT)] = cc[l];
  }
  if (!ft.grad) return;
#pragma unroll
  for (int l = 0; l < L; ++l) uu[l] = __ldcg(&GT[e_of<T>(2, t, l)]);
  xwht_full<T>(uu, sm, 1);
#pragma unroll
  for (int l = 0; l < L; ++l) sm[t + (l << kLOGNT)] = uu[l];  // own entries, for the rare fallback
  for (uint32_t q = t; q < d; q += kFNT) wT[q] = (T)job.w[q];
  build_all<T, FAM, ALPHA, L>(job, job.Ct + (size_t)r * d * 32, job.g, base, tb);
  const T *P = reinterpret_cast<const T *>(ft.p) + (uint64_t)r * n + base;
  const T zeta = (T)job.zeta;
  T k1[L];
  uint32_t bi[L];
  bool ok[L];
#pragma unroll
  for (int l = 0; l < L; ++l) {
    k1[l] = zeta * (T(1) + __ldcg(&P[t + (l << kLOGNT)]));
    bi[l] = __brev((uint32_t)(base + t + (l << kLOGNT)));
    ok[l] = true;
    uu[l] *= k1[l];  // from here on uu holds u k1
  }
  __syncthreads();
  // u itself stays in the transform tile (sm) after tile_wht; each thread reads its own
  gradient_sweep<T, FAM, ALPHA, L, true>(job, tb, wT, bi, k1, uu, ok,
                                   [&](int l) { return sm[t + (l << kLOGNT)]; }, red);
  __syncthreads();
  double *dst = ft.gr + ((uint64_t)v * ft.tiles + tile) * 2 * d;
  for (uint32_t q = t; q < 2 * d; q += kFNT) dst[q] = red_total<T>(red, kFNT / 32, 2 * d, q);
}

template <typename T, int FAM, int ALPHA>
__global__ void __launch_bounds__(kFNT, 2) k_fused_C(FTask ft) {
  extern __shared__ __align__(16) unsigned char smem[];
  fused_C_item<T, FAM, ALPHA>(ft, blockIdx.y, blockIdx.x, smem);
}

// ------------------------------------------------------------------ final
__device__ __forceinline__ void fused_final_item(const FTask &ft, uint32_t v) {
  __shared__ double sh[32];
  const uint32_t r = v / ft.nrhs;
  const uint32_t tiles = ft.tiles, d = ft.job.d;
  const double n = (double)(1ull << ft.job.m), zeta = ft.job.zeta;
  double q = 0, gsum = 0, ld = 0, sp = 0, sy = 0;
  for (uint32_t b = threadIdx.x; b < tiles; b += blockDim.x) {
    q += __ldcg(&ft.qg[((uint64_t)v * tiles + b) * 2 + 0]);
    gsum += __ldcg(&ft.qg[((uint64_t)v * tiles + b) * 2 + 1]);
    ld += __ldcg(&ft.ld[(uint64_t)r * tiles + b]);
    sp += __ldcg(&ft.sp[(uint64_t)r * tiles + b]);
    sy += __ldcg(&ft.sy[(uint64_t)v * tiles + b]);
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
    for (uint32_t b = lane; b < tiles; b += 32) s += __ldcg(&ft.gr[((uint64_t)v * tiles + b) * 2 * d + j]);
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

static __global__ void __launch_bounds__(256) k_fused_final(FTask ft) { fused_final_item(ft, blockIdx.x); }

// -------------------------------------- persistent whole-pipeline schedule (one launch)
// Every randomization of every task is a unit u with four kinds of work items: A tiles,
// B column tiles, C tiles (x right-hand sides) and F (the final reduction, one per
// right-hand side).  Resident CTAs take items in ticket order; step s of the sequence
// holds A(s), B(s - lag), C(s - 2 lag), F(s - 2 lag - 1), so a unit's phases follow each
// other while its intermediate vectors are in L2.  Units cycle through nslot scratch
// slots; A(u) reuses the slot of u - nslot once F(u - nslot) has finished.
//
// Item dependencies: B(u) after all A(u), C(u) after all B(u), F(u) after all C(u) (after
// all B(u) when the unit wants neither c nor the gradient), A(u) after all F(u - nslot).
// Each is on items with smaller tickets (nslot > 2 lag + 1), a CTA waits only while it
// holds no unpublished item, and those items were claimed by CTAs that are running: the
// waits end.  They are bounded all the same: past the limit the CTA raises
// QK_STATUS_TIMEOUT and the shared abort flag, and every later wait gives up at once, so
// the launch finishes.
struct PUnit {
  FTask ft;                   // one randomization: r = 0, scratch in slot u mod nslot
  uint32_t tiles, nrhs, ncv;  // ncv: C items (tiles x nrhs, 0 when neither c nor grad is wanted)
};
struct PSched {
  const PUnit *units;
  const uint32_t *step_off;  // S + 1 prefix counts of items per step
  uint32_t U, S, lag, nslot;
  uint32_t *ctr;  // ticket, abort flag, then cntA, cntB, cntC, cntF (U each)
  uint32_t *status;
  uint32_t spin_limit;
};
enum { PK_A = 0, PK_B = 1, PK_C = 2, PK_F = 3 };

__device__ __forceinline__ void psched_decode(const PSched &ps, uint32_t it, uint32_t &kind, uint32_t &u,
                                              uint32_t &idx) {
  uint32_t lo = 0, hi = ps.S;  // step_off[lo] <= it < step_off[hi]
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (ps.step_off[mid] <= it) lo = mid;
    else hi = mid;
  }
  const uint32_t s = lo, L = ps.lag;
  uint32_t k = it - ps.step_off[s];
  if (s < ps.U) {
    const uint32_t nA = ps.units[s].tiles;
    if (k < nA) {
      kind = PK_A, u = s, idx = k;
      return;
    }
    k -= nA;
  }
  if (s >= L && s - L < ps.U) {
    const uint32_t nB = ps.units[s - L].tiles;
    if (k < nB) {
      kind = PK_B, u = s - L, idx = k;
      return;
    }
    k -= nB;
  }
  if (s >= 2 * L && s - 2 * L < ps.U) {
    const uint32_t nC = ps.units[s - 2 * L].ncv;
    if (k < nC) {
      kind = PK_C, u = s - 2 * L, idx = k;
      return;
    }
    k -= nC;
  }
  kind = PK_F, u = s - 2 * L - 1, idx = k;
}

// Thread 0: wait until *cnt >= need (bounded); false if this item must be skipped.
__device__ __forceinline__ bool psched_wait(const PSched &ps, const uint32_t *cnt, uint32_t need) {
  volatile uint32_t *abort_flag = ps.ctr + 1;
  uint32_t k = 0;
  while (ld_acquire_u32(cnt) < need) {
    if (*abort_flag) return false;
    if (++k > ps.spin_limit) {
      atomicExch(ps.ctr + 1, 1u);
      if (ps.status) atomicOr(ps.status, (uint32_t)QK_STATUS_TIMEOUT);
      return false;
    }
    __nanosleep(128);
  }
  return true;
}

template <typename T, int FAM, int ALPHA, bool COMP, bool WIDE>
__global__ void __launch_bounds__(kFNT, 2) k_fused_persist(PSched ps) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ uint32_t s_it, s_ok;
  const int t = threadIdx.x;
  const uint32_t total = ps.step_off[ps.S];
  uint32_t *cntA = ps.ctr + 2, *cntB = cntA + ps.U, *cntC = cntB + ps.U, *cntF = cntC + ps.U;
  for (;;) {
    if (t == 0) s_it = atomicAdd(ps.ctr, 1u);
    __syncthreads();
    const uint32_t it = s_it;
    if (it >= total) break;
    uint32_t kind, u, idx;
    psched_decode(ps, it, kind, u, idx);
    const PUnit &pu = ps.units[u];
    if (t == 0) {
      bool ok = true;
      if (kind == PK_A && u >= ps.nslot) ok = psched_wait(ps, cntF + (u - ps.nslot), ps.units[u - ps.nslot].nrhs);
      else if (kind == PK_B) ok = psched_wait(ps, cntA + u, pu.tiles);
      else if (kind == PK_C) ok = psched_wait(ps, cntB + u, pu.tiles);
      else if (kind == PK_F)  // after C, or after B when the unit has no C items
        ok = pu.ncv ? psched_wait(ps, cntC + u, pu.ncv) : psched_wait(ps, cntB + u, pu.tiles);
      s_ok = ok;
    }
    __syncthreads();
    if (!s_ok) continue;  // uniform; the loop's first barrier separates s_ok's next write
    if (kind == PK_A) {
      fused_A_item<T, FAM, ALPHA, COMP, WIDE>(pu.ft, 0, idx, smem);
    } else if (kind == PK_B) {
      fused_B_item<T, COMP, WIDE>(pu.ft, 0, idx, smem, ps.status);
    } else if (kind == PK_C) {
      fused_C_item<T, FAM, ALPHA>(pu.ft, idx / pu.tiles, idx % pu.tiles, smem);
    } else {
      fused_final_item(pu.ft, idx);
    }
    __syncthreads();  // every thread's stores (and shared-memory reads) are done
    if (t == 0)
      red_release_add_u32((kind == PK_A ? cntA : kind == PK_B ? cntB : kind == PK_C ? cntC : cntF) + u, 1u);
  }
}

template <typename T, int FAM, int ALPHA, bool COMP, bool WIDE>
int launch_fused_t(const FTask &ft, cudaStream_t st, LaunchTimer *tm) {
  constexpr int L = FCfg<T>::L;
  const uint32_t R = ft.job.nr, d = ft.job.d;
  const size_t colb = align256(col_smem_bytes<L>(d));
  // phase A keeps a second tile for the lo parts when compensating
  const size_t smA = colb + xtile_bytes<T>() + 32 * sizeof(double);
  const size_t smB = 3 * xtile_bytes<T>() + 32 * sizeof(double);
  const size_t smC = colb + xtile_bytes<T>() + (size_t)(kFNT / 32) * 2 * d * sizeof(double);
  smem_optin<k_fused_A<T, FAM, ALPHA, COMP, WIDE>>(smA);
  smem_optin<k_fused_B<T, COMP, WIDE>>(smB);
  smem_optin<k_fused_C<T, FAM, ALPHA>>(smC);
  if (tm) tm->begin("k_fused_A", st);
  k_fused_A<T, FAM, ALPHA, COMP, WIDE><<<dim3(ft.tiles, R), kFNT, smA, st>>>(ft);
  if (tm) tm->end(st);
  int rc = check_launch("fused A");
  if (rc) return rc;
  if (tm) tm->begin("k_fused_B", st);
  k_fused_B<T, COMP, WIDE><<<dim3(ft.tiles, R), kFNT, smB, st>>>(ft);
  if (tm) tm->end(st);
  if ((rc = check_launch("fused B"))) return rc;
  if (ft.c || ft.grad) {
    if (tm) tm->begin("k_fused_C", st);
    k_fused_C<T, FAM, ALPHA><<<dim3(ft.tiles, R * ft.nrhs), kFNT, smC, st>>>(ft);
    if (tm) tm->end(st);
    if ((rc = check_launch("fused C"))) return rc;
  }
  if (tm) tm->begin("k_fused_final", st);
  k_fused_final<<<R * ft.nrhs, 256, 0, st>>>(ft);
  if (tm) tm->end(st);
  return check_launch("fused final");
}

template <typename T, bool COMP, bool WIDE = false>
int dispatch_fused(const FTask &ft, cudaStream_t st, LaunchTimer *tm) {
  switch (ft.job.alpha) {
    case 1: return launch_fused_t<T, 0, 1, COMP, WIDE>(ft, st, tm);
    case 2: return launch_fused_t<T, 0, 2, COMP, WIDE>(ft, st, tm);
    case 3: return launch_fused_t<T, 0, 3, COMP, WIDE>(ft, st, tm);
    case 4: return launch_fused_t<T, 0, 4, COMP, WIDE>(ft, st, tm);
    default: return fail(QK_EINVAL, "DSI order must be 1..4");
  }
}

template <typename T, int FAM, int ALPHA, bool COMP, bool WIDE = false>
int persist_launch_t(const PSched &ps, uint32_t dmax, cudaStream_t st) {
  constexpr int L = FCfg<T>::L;
  const size_t colb = align256(col_smem_bytes<L>(dmax));
  const size_t smA = colb + xtile_bytes<T>() + 32 * sizeof(double);
  const size_t smB = 3 * xtile_bytes<T>() + 32 * sizeof(double);
  const size_t smC = colb + xtile_bytes<T>() + (size_t)(kFNT / 32) * 2 * dmax * sizeof(double);
  size_t sm = smA > smB ? smA : smB;
  if (smC > sm) sm = smC;
  smem_optin<k_fused_persist<T, FAM, ALPHA, COMP, WIDE>>(sm);
  int occ = 0, dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_fused_persist<T, FAM, ALPHA, COMP, WIDE>, kFNT, sm);
  if (e != cudaSuccess || occ < 1)
    return fail(QK_ECUDA, "persistent schedule: %zu bytes of shared memory per CTA do not fit", sm);
  k_fused_persist<T, FAM, ALPHA, COMP, WIDE><<<(unsigned)(sms * occ), kFNT, sm, st>>>(ps);
  return check_launch("fused persistent");
}

// The persistent launch for one precision (T, COMP, WIDE) and the DSI order of the plan.
template <typename T, bool COMP, bool WIDE>
int persist_dispatch(const PSched &ps, int alpha, uint32_t dmax, cudaStream_t st) {
  switch (alpha) {
    case 1: return persist_launch_t<T, 0, 1, COMP, WIDE>(ps, dmax, st);
    case 2: return persist_launch_t<T, 0, 2, COMP, WIDE>(ps, dmax, st);
    case 3: return persist_launch_t<T, 0, 3, COMP, WIDE>(ps, dmax, st);
    case 4: return persist_launch_t<T, 0, 4, COMP, WIDE>(ps, dmax, st);
    default: return fail(QK_EINVAL, "DSI order must be 1..4");
  }
}

// Kernels are instantiated in qk_fused_f64.cu, qk_fused_f32.cu, qk_fused_f32c.cu and
// qk_fused_f32w.cu only.
#define QK_FUSED_PRECISIONS(X) X(double, false, false) X(float, false, false) X(float, true, false) X(float, true, true)
#define QK_FUSED_EXTERN(T, C, W)                                                   \
  extern template int dispatch_fused<T, C, W>(const FTask &, cudaStream_t, LaunchTimer *); \
  extern template int persist_dispatch<T, C, W>(const PSched &, int, uint32_t, cudaStream_t);
#define QK_FUSED_INSTANTIATE(T, C, W)                                              \
  template int dispatch_fused<T, C, W>(const FTask &, cudaStream_t, LaunchTimer *);        \
  template int persist_dispatch<T, C, W>(const PSched &, int, uint32_t, cudaStream_t);

}  // namespace qk
