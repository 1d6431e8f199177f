// Per-CTA difference-word tables and the first-column sweep (arXiv 2502.14256,
// Sec. 5.4: k_1[i] = K(x_i, x_0)), shared by the standalone column / gradient
// kernels and the fused pipeline.
//
// Digital nets: X_i (+) X_0 = XOR_{bit k of h(i)} Ct[k] with h(i) = i (natural) or
// i ^ (i >> 1) (Gray), linear over GF(2).  A CTA of NT = 256 threads covers
// NT * L consecutive positions i = tile | (l << 8) | (warp << 5) | lane (disjoint
// bit fields), so the difference word is Z(h(lane)) ^ Z(h(warp << 5)) ^ Z(h(tile | l << 8)):
// three shared tables, one broadcast load and one XOR per (point, dimension).
// Lattices: X_i (-) X_0 = v(i) 2^32 g mod 2^32 = brev(i) * g (wrapping multiply).
#pragma once

#include "qk_common.cuh"
#include "qk_factors.cuh"
#include "qk_internal.h"

namespace qk {

constexpr int kColNT = 256;

__device__ __forceinline__ uint32_t order_map(int order, uint32_t v) {
  return order == QK_GRAY ? (v ^ (v >> 1)) : v;
}

__device__ __forceinline__ uint32_t xor_columns(const uint32_t *col, uint32_t v) {
  uint32_t acc = 0;
  while (v) {
    acc ^= col[__ffs(v) - 1];
    v &= v - 1;
  }
  return acc;
}

struct DiffTables {
  uint32_t *zlane;  // [j][lane]
  uint32_t *zwarp;  // [warp][j]
  uint32_t *zl;     // [l][j]
  uint32_t *gs;     // lattices: [j]
};

// Shared bytes: weights (d doubles) + tables ((32 + 8 + L) d words).
template <int L>
__host__ __device__ inline size_t col_smem_bytes(uint32_t d) {
  return (size_t)d * sizeof(double) + (size_t)(32 + kColNT / 32 + L) * d * sizeof(uint32_t);
}

template <int L>
__device__ __forceinline__ void carve_tables(unsigned char *smem, uint32_t d, double **w, DiffTables &tb) {
  *w = reinterpret_cast<double *>(smem);
  uint32_t *u = reinterpret_cast<uint32_t *>(smem + (size_t)d * sizeof(double));
  tb.zlane = u;
  tb.zwarp = tb.zlane + 32 * d;
  tb.zl = tb.zwarp + (kColNT / 32) * d;
  tb.gs = u;
}

// Fill the tables for one CTA tile (Cr = this randomization's d x 32 columns).
template <int L>
__device__ void build_tables(const ColJob &job, const uint32_t *Cr, const uint32_t *g, uint64_t tile_base,
                             DiffTables &tb) {
  const uint32_t d = job.d;
  if (job.kind == QK_NET_B2) {
    for (uint32_t q = threadIdx.x; q < 32 * d; q += kColNT) {
      const uint32_t j = q >> 5, ln = q & 31;
      tb.zlane[q] = xor_columns(Cr + j * 32, order_map(job.order, ln));
    }
    for (uint32_t q = threadIdx.x; q < (kColNT / 32) * d; q += kColNT) {
      const uint32_t w = q / d, j = q - w * d;
      tb.zwarp[q] = xor_columns(Cr + j * 32, order_map(job.order, w << 5));
    }
    for (uint32_t q = threadIdx.x; q < L * d; q += kColNT) {
      const uint32_t l = q / d, j = q - l * d;
      tb.zl[q] = xor_columns(Cr + j * 32, order_map(job.order, (uint32_t)(tile_base | ((uint64_t)l << 8))));
    }
  } else {
    for (uint32_t q = threadIdx.x; q < d; q += kColNT) tb.gs[q] = g[q];
  }
}

// Difference word of this thread's point l in dimension j.
template <int FAM, int L>
__device__ __forceinline__ uint32_t diff_word(const DiffTables &tb, uint32_t d, uint32_t base, uint32_t bi, int l,
                                              uint32_t j) {
  if constexpr (FAM == 0) return base ^ tb.zl[l * d + j];
  else return bi * tb.gs[j];
}

// p[l] = prod_j (1 + c_j K_j(point l)) - 1 for the L points of this thread.
template <typename T, int FAM, int ALPHA, int L>
__device__ __forceinline__ void column_sweep(const ColJob &job, const DiffTables &tb, const T *wT,
                                             const uint32_t (&bi)[L], T (&p)[L]) {
  const uint32_t d = job.d;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int l = 0; l < L; ++l) p[l] = T(0);
  for (uint32_t j = 0; j < d; ++j) {
    const T wj = wT[j];
    uint32_t base = 0;
    if constexpr (FAM == 0) base = tb.zlane[j * 32 + lane] ^ tb.zwarp[warp * d + j];
#pragma unroll
    for (int l = 0; l < L; ++l) {
      const T a = wj * factor<T, FAM, ALPHA>(diff_word<FAM, L>(tb, d, base, bi[l], l, (FAM == 0) ? j : j));
      p[l] = pm1_step(p[l], a);
    }
  }
}

// dk_1/dc_j by the explicit product (used only where 1 + c_j K_j == 0 exactly).
template <typename T, int FAM, int ALPHA, int L>
__device__ T dk_explicit(const ColJob &job, const DiffTables &tb, const T *wT, uint32_t bi_l, int l, uint32_t jx) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T prod = (T)job.zeta;
  for (uint32_t j = 0; j < job.d; ++j) {
    uint32_t base = 0;
    if constexpr (FAM == 0) base = tb.zlane[j * 32 + lane] ^ tb.zwarp[warp * job.d + j];
    const T K = factor<T, FAM, ALPHA>(diff_word<FAM, L>(tb, job.d, base, bi_l, l, j));
    prod *= (j == jx) ? K : (T(1) + wT[j] * K);
  }
  return prod;
}

// Gradient sweep: for each dimension j, warp-reduced FP64 sums over this warp's
// points of u_i dk1_i/dc_j and dk1_i/dc_j, written to red[warp][2d].
template <typename T, int FAM, int ALPHA, int L>
__device__ __forceinline__ void gradient_sweep(const ColJob &job, const DiffTables &tb, const T *wT,
                                               const uint32_t (&bi)[L], const T (&k1)[L], const T (&uu)[L],
                                               const bool (&ok)[L], double *red) {
  const uint32_t d = job.d;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (uint32_t j = 0; j < d; ++j) {
    const T wj = wT[j];
    T su = T(0), s1 = T(0);
    uint32_t base = 0;
    if constexpr (FAM == 0) base = tb.zlane[j * 32 + lane] ^ tb.zwarp[warp * d + j];
#pragma unroll
    for (int l = 0; l < L; ++l) {
      const T K = factor<T, FAM, ALPHA>(diff_word<FAM, L>(tb, d, base, bi[l], l, j));
      const T f = T(1) + wj * K;
      T dk = (f != T(0)) ? k1[l] * K / f : dk_explicit<T, FAM, ALPHA, L>(job, tb, wT, bi[l], l, j);
      if (!ok[l]) dk = T(0);
      su += uu[l] * dk;
      s1 += dk;
    }
    double du = (double)su, d1 = (double)s1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      du += __shfl_xor_sync(0xffffffffu, du, o);
      d1 += __shfl_xor_sync(0xffffffffu, d1, o);
    }
    if (lane == 0) {
      red[(size_t)warp * 2 * d + j] = du;
      red[(size_t)warp * 2 * d + d + j] = d1;
    }
  }
}

}  // namespace qk
