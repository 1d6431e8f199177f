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

// DSI kernels as polynomials in the converted word fz = (T)Z with coefficients that
// depend only on beta, i.e. on clz(Z) (the Theorem of Sec. 5.3; x = fz 2^-32):
//   order 1: K = 1 - 3 t1                         (1 at Z = 0)
//   order 2: K = (3/2 - 5/2 t1) - beta 2^-32 fz
//   order 3: K = (-1 + 43/18 (1 - t2)) - 5 (1 - t1) 2^-32 fz + beta 2^-64 fz^2
//   order 4: K = (-1 + 701/294 (1 - t3)) - 43/9 (1 - t2) 2^-32 fz + 5 (1 - t1) 2^-64 fz^2
//                - 2/3 beta 2^-96 fz^3 - beta/24 S'(Z)
// Row r = clz(Z) in 0..32 (r = 32 is Z = 0: beta = t = 0); rows are padded to a
// power-of-two stride so that each lookup is one (or two) vector loads.
// S'(Z) = sum of 8^-a over set digits x_{a+1} is read from a 256-entry byte table:
// S' = T[b0] + 2^-24 T[b1] + 2^-48 T[b2] + ... for the bytes b0, b1, ... of Z.
constexpr int kTabRows = 33, kTabNC = 8, kOctRows = 256;

// Row stride (elements) for order alpha: 1, 2, 4, 8 -> rows load as one vector.
__host__ __device__ constexpr int tab_stride(int alpha) { return alpha == 1 ? 1 : (alpha == 2 ? 2 : (alpha == 3 ? 4 : 8)); }

template <typename T>
__host__ __device__ inline size_t dsi_tab_bytes() {
  return (size_t)(kTabRows * kTabNC + kOctRows) * sizeof(T);
}

struct DiffTables {
  uint32_t *zlane;  // [j][lane]
  uint32_t *zwarp;  // [warp][j]
  uint32_t *zl;     // [j][l]
  uint32_t *gs;     // lattices: [j]
  void *ktab;       // DSI coefficient rows [33][kTabNC] then the byte table [256], of T
};

// Shared bytes: weights (d doubles) + DSI tables (as doubles) + index tables ((32 + 8 + L) d words).
__host__ __device__ inline size_t weights_bytes(uint32_t d) { return ((size_t)d * sizeof(double) + 15) & ~(size_t)15; }

template <int L>
__host__ __device__ inline size_t col_smem_bytes(uint32_t d) {
  return weights_bytes(d) + dsi_tab_bytes<double>() + (size_t)(32 + kColNT / 32 + L) * d * sizeof(uint32_t);
}

template <int L>
__device__ __forceinline__ void carve_tables(unsigned char *smem, uint32_t d, double **w, DiffTables &tb) {
  *w = reinterpret_cast<double *>(smem);
  tb.ktab = smem + weights_bytes(d);  // 16-byte aligned for the vector row loads
  uint32_t *u = reinterpret_cast<uint32_t *>(smem + weights_bytes(d) + dsi_tab_bytes<double>());
  tb.zlane = u;
  tb.zwarp = tb.zlane + 32 * d;
  tb.zl = tb.zwarp + (kColNT / 32) * d;
  tb.gs = u;
}

// DSI coefficient rows.  They depend only on beta and the order (the weights enter
// later, as c_j K), so they are computed once, at compile time, in double precision
// (the Theorem's beta-dependent coefficients, stored as T); every CTA copies them into
// shared memory.  Rows of order 3 and 4 carry the rounding residuals of their constant
// (and, for order 4, linear) coefficients, so that FP32 rows add no per-row bias.
constexpr int kDsiTabLen = kTabRows * kTabNC + kOctRows;
template <typename T> struct DsiTable { T v[kDsiTabLen]; };

__host__ __device__ constexpr double pow2neg(int e) {
  double r = 1.0;
  for (int i = 0; i < e; ++i) r *= 0.5;
  return r;
}

template <typename T, int ALPHA>
__host__ __device__ constexpr DsiTable<T> make_dsi_table() {
  DsiTable<T> tab{};
  constexpr int S = tab_stride(ALPHA);
  for (int q = 0; q < kTabRows; ++q) {
    const int beta = q < 32 ? q + 1 : 0;
    const double t1 = q < 32 ? pow2neg(beta) : 0.0, t2 = t1 * t1, t3 = t2 * t1;
    const double b = (double)beta;
    double A = 0, B = 0, C = 0, D = 0, E = 0;
    if (ALPHA == 1) {
      A = q < 32 ? 1.0 - 3.0 * t1 : 1.0;
    } else if (ALPHA == 2) {
      A = 1.5 - 2.5 * t1;
      B = -b * pow2neg(32);
    } else if (ALPHA == 3) {
      A = -1.0 + (43.0 / 18.0) * (1.0 - t2);
      B = -5.0 * (1.0 - t1) * pow2neg(32);
      C = b * pow2neg(64);
    } else {
      A = -1.0 + (701.0 / 294.0) * (1.0 - t3);
      B = -(43.0 / 9.0) * (1.0 - t2) * pow2neg(32);
      C = 5.0 * (1.0 - t1) * pow2neg(64);
      D = -(2.0 / 3.0) * b * pow2neg(96);
      E = -b / 24.0;
    }
    const double co[5] = {A, B, C, D, E};
    for (int k = 0; k < S && k < 5; ++k) tab.v[q * S + k] = (T)co[k];
    if (ALPHA == 3) tab.v[q * S + 3] = (T)(A - (double)(T)A);
    if (ALPHA == 4) {
      tab.v[q * S + 5] = (T)(A - (double)(T)A);
      tab.v[q * S + 6] = (T)(B - (double)(T)B);
    }
  }
  for (int byte = 0; byte < kOctRows; ++byte) {  // S' of the 8 digits of one byte (a = 0..7)
    double sum = 0.0;
    for (int a = 0; a < 8; ++a)
      if ((byte >> (7 - a)) & 1) sum += pow2neg(3 * a);
    tab.v[kTabRows * kTabNC + byte] = (T)sum;
  }
  return tab;
}

static __device__ const DsiTable<float> g_dsi_f[4] = {make_dsi_table<float, 1>(), make_dsi_table<float, 2>(),
                                                      make_dsi_table<float, 3>(), make_dsi_table<float, 4>()};
static __device__ const DsiTable<double> g_dsi_d[4] = {make_dsi_table<double, 1>(), make_dsi_table<double, 2>(),
                                                       make_dsi_table<double, 3>(), make_dsi_table<double, 4>()};

// Float-float rows of the same polynomials in fz (the float-float first column): per row the
// pairs (h, l) of A, B, C, D, E (orders 2 and 3 use a prefix), padded to 12 floats so that
// a row loads as three 128-bit vectors, then the octal byte table (exact in FP32).
constexpr int kFFStride = 12;
constexpr int kDsiFFLen = kTabRows * kFFStride + kOctRows;
struct DsiTableFF { float v[kDsiFFLen]; };
static_assert(sizeof(DsiTableFF) <= kDsiTabLen * sizeof(double), "float-float rows fit the shared table region");

template <int ALPHA>
__host__ __device__ constexpr DsiTableFF make_dsi_table_ff() {
  DsiTableFF tab{};
  for (int q = 0; q < kTabRows; ++q) {
    const int beta = q < 32 ? q + 1 : 0;
    const double t1 = q < 32 ? pow2neg(beta) : 0.0, t2 = t1 * t1, t3 = t2 * t1;
    const double b = (double)beta;
    double co[5] = {0, 0, 0, 0, 0};
    if (ALPHA == 1) {
      co[0] = q < 32 ? 1.0 - 3.0 * t1 : 1.0;
    } else if (ALPHA == 2) {
      co[0] = 1.5 - 2.5 * t1;
      co[1] = -b * pow2neg(32);
    } else if (ALPHA == 3) {
      co[0] = -1.0 + (43.0 / 18.0) * (1.0 - t2);
      co[1] = -5.0 * (1.0 - t1) * pow2neg(32);
      co[2] = b * pow2neg(64);
    } else {
      co[0] = -1.0 + (701.0 / 294.0) * (1.0 - t3);
      co[1] = -(43.0 / 9.0) * (1.0 - t2) * pow2neg(32);
      co[2] = 5.0 * (1.0 - t1) * pow2neg(64);
      co[3] = -(2.0 / 3.0) * b * pow2neg(96);
      co[4] = -b / 24.0;
    }
    for (int k = 0; k < 5; ++k) {
      const float h = (float)co[k];
      tab.v[q * kFFStride + 2 * k] = h;
      tab.v[q * kFFStride + 2 * k + 1] = (float)(co[k] - (double)h);
    }
  }
  for (int byte = 0; byte < kOctRows; ++byte) {
    double sum = 0.0;
    for (int a = 0; a < 8; ++a)
      if ((byte >> (7 - a)) & 1) sum += pow2neg(3 * a);
    tab.v[kTabRows * kFFStride + byte] = (float)sum;  // at most 22 significant bits: exact
  }
  return tab;
}

static __device__ const DsiTableFF g_dsi_ff[4] = {make_dsi_table_ff<1>(), make_dsi_table_ff<2>(),
                                                  make_dsi_table_ff<3>(), make_dsi_table_ff<4>()};

template <int ALPHA>
__device__ void build_dsi_tab_ff(float *tab) {
  const float *src = g_dsi_ff[ALPHA - 1].v;
  for (int q = threadIdx.x; q < kDsiFFLen; q += kColNT) tab[q] = src[q];
}

// Copy the DSI coefficient rows of this order into shared memory.
template <typename T, int ALPHA>
__device__ void build_dsi_tab(T *tab) {
  const T *src;
  if constexpr (sizeof(T) == 4) src = g_dsi_f[ALPHA - 1].v;
  else src = g_dsi_d[ALPHA - 1].v;
  for (int q = threadIdx.x; q < kDsiTabLen; q += kColNT) tab[q] = src[q];
}

__device__ __forceinline__ float word_to(float, uint32_t Z) { return __uint2float_rn(Z); }
__device__ __forceinline__ double word_to(double, uint32_t Z) {
  return __hiloint2double(0x43300000, (int)Z) - 4503599627370496.0;  // exact
}

// K_alpha(Z) for a DSI kernel from the shared coefficient rows (vector row loads).
template <typename T, int ALPHA>
__device__ __forceinline__ T dsi_tab_eval(const T *tab, uint32_t Z) {
  constexpr int S = tab_stride(ALPHA);
  const T *row = tab + __clz(Z) * S;
  if constexpr (ALPHA == 1) {
    return row[0];
  } else {
    const T fz = word_to(T(), Z);
    if constexpr (ALPHA == 2) {
      T a, b;
      if constexpr (sizeof(T) == 4) {
        const float2 v = *reinterpret_cast<const float2 *>(row);
        a = v.x, b = v.y;
      } else {
        const double2 v = *reinterpret_cast<const double2 *>(row);
        a = v.x, b = v.y;
      }
      return fmadd(b, fz, a);
    } else {
      T c0, c1, c2, c3;
      if constexpr (sizeof(T) == 4) {
        const float4 v = *reinterpret_cast<const float4 *>(row);
        c0 = v.x, c1 = v.y, c2 = v.z, c3 = v.w;
      } else {
        const double2 v0 = *reinterpret_cast<const double2 *>(row);
        const double2 v1 = *reinterpret_cast<const double2 *>(row + 2);
        c0 = v0.x, c1 = v0.y, c2 = v1.x, c3 = v1.y;
      }
      if constexpr (ALPHA == 3) {
        return fmadd(fmadd(c2, fz, c1), fz, c0) + c3;  // c3: residual of c0
      } else {
        const T *oct = tab + kTabRows * kTabNC;
        T sp = oct[Z >> 24] + T(0x1p-24) * oct[(Z >> 16) & 255u];
        if constexpr (sizeof(T) == 8) sp += T(0x1p-48) * oct[(Z >> 8) & 255u];
        T c4, c5, c6;
        if constexpr (sizeof(T) == 4) {
          const float4 v = *reinterpret_cast<const float4 *>(row + 4);
          c4 = v.x, c5 = v.y, c6 = v.z;
        } else {
          const double2 v = *reinterpret_cast<const double2 *>(row + 4);
          c4 = v.x, c5 = v.y, c6 = row[6];
        }
        const T poly = fmadd(fmadd(c3, fz, c2), fz, c1) * fz + c0;
        return fmadd(c4, sp, poly) + fmadd(c6, fz, c5);
      }
    }
  }
}

// K_alpha for either family: DSI from the table, SI from the Bernoulli form.
template <typename T, int FAM, int ALPHA>
__device__ __forceinline__ T kfac(const DiffTables &tb, uint32_t w) {
  if constexpr (FAM == 0) return dsi_tab_eval<T, ALPHA>(reinterpret_cast<const T *>(tb.ktab), w);
  else return si_factor<T, ALPHA>(w);
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
      const uint32_t j = q / L, l = q - j * L;
      tb.zl[q] = xor_columns(Cr + j * 32, order_map(job.order, (uint32_t)(tile_base | ((uint64_t)l << 8))));
    }
  } else {
    for (uint32_t q = threadIdx.x; q < d; q += kColNT) tb.gs[q] = g[q];
  }
}

// All per-CTA tables: index tables plus, for DSI kernels, the coefficient rows.
template <typename T, int FAM, int ALPHA, int L>
__device__ __forceinline__ void build_all(const ColJob &job, const uint32_t *Cr, const uint32_t *g,
                                          uint64_t tile_base, DiffTables &tb) {
  build_tables<L>(job, Cr, g, tile_base, tb);
  if constexpr (FAM == 0) build_dsi_tab<T, ALPHA>(reinterpret_cast<T *>(tb.ktab));
}

// Difference word of this thread's point l in dimension j.
template <int FAM, int L>
__device__ __forceinline__ uint32_t diff_word(const DiffTables &tb, uint32_t d, uint32_t base, uint32_t bi, int l,
                                              uint32_t j) {
  if constexpr (FAM == 0) return base ^ tb.zl[j * L + l];  // l is a compile-time offset
  else return bi * tb.gs[j];
}

// Difference words of this thread's points l .. l + 3 in dimension j.  Nets read the four
// table words with one 128-bit shared load: carve_tables places zl at a multiple of 16
// bytes from the (16-byte aligned) shared base, and a row holds L words, L a multiple of 4.
template <int FAM, int L>
__device__ __forceinline__ void diff_words4(const DiffTables &tb, uint32_t base, const uint32_t (&bi)[L], int l,
                                            uint32_t j, uint32_t (&z)[4]) {
  static_assert(L % 4 == 0, "rows of whole quads");
  if constexpr (FAM == 0) {
    const uint4 q = *reinterpret_cast<const uint4 *>(tb.zl + j * L + l);
    z[0] = base ^ q.x, z[1] = base ^ q.y, z[2] = base ^ q.z, z[3] = base ^ q.w;
  } else {
    const uint32_t gj = tb.gs[j];
#pragma unroll
    for (int i = 0; i < 4; ++i) z[i] = bi[l + i] * gj;
  }
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
    if constexpr (sizeof(T) == 4 && L % 4 == 0) {
      // two points per packed f32x2 multiply / add / fma: the same roundings as below
      const unsigned long long W = pack_f2(wj, wj);
#pragma unroll
      for (int l = 0; l < L; l += 4) {
        uint32_t z[4];
        diff_words4<FAM, L>(tb, base, bi, l, j, z);
#pragma unroll
        for (int i = 0; i < 4; i += 2) {
          const T k0 = kfac<T, FAM, ALPHA>(tb, z[i]), k1 = kfac<T, FAM, ALPHA>(tb, z[i + 1]);
          const unsigned long long A = mul_f2(W, pack_f2(k0, k1)), P = pack_f2(p[l + i], p[l + i + 1]);
          unpack_f2(fma_f2(P, A, add_f2(P, A)), p[l + i], p[l + i + 1]);
        }
      }
    } else if constexpr (L % 4 == 0) {
#pragma unroll
      for (int l = 0; l < L; l += 4) {
        uint32_t z[4];
        diff_words4<FAM, L>(tb, base, bi, l, j, z);
#pragma unroll
        for (int i = 0; i < 4; ++i) p[l + i] = pm1_step(p[l + i], wj * kfac<T, FAM, ALPHA>(tb, z[i]));
      }
    } else {
#pragma unroll
      for (int l = 0; l < L; ++l) {
        const T a = wj * kfac<T, FAM, ALPHA>(tb, diff_word<FAM, L>(tb, d, base, bi[l], l, j));
        p[l] = pm1_step(p[l], a);
      }
    }
  }
}

// --------------------------------------------- float-float first column (pairs of points)
// The 32-bit word Z as a normalised float-float pair: Z & ~255 (at most 24 significant bits)
// and Z & 255 convert exactly; one fast TwoSum normalises the pair.
__device__ __forceinline__ FF<F2> word_ff2(uint32_t Z0, uint32_t Z1) {
  const F2 zh = vpack(__uint2float_rn(Z0 & ~255u), __uint2float_rn(Z1 & ~255u));
  const F2 zl = vpack(small_int_to(0.f, Z0 & 255u), small_int_to(0.f, Z1 & 255u));
  return ff_fast_two_sum(zh, zl);
}

// K_alpha of two points in float-float from the float-float rows (the polynomial in fz of
// the FP32 rows, Horner in float-float).  S'(Z) = T[b0] + 2^-24 T[b1] + 2^-48 T[b2] (the
// bytes b of Z) enters as the pair (T[b0], 2^-24 T[b1] + 2^-48 T[b2]): T[b0] is 0 or at
// least 2^-21, above the second part, so one fast TwoSum normalises it.
template <int ALPHA>
__device__ __forceinline__ FF<F2> dsi_ff2(const float *tab, uint32_t Z0, uint32_t Z1) {
  const float *r0 = tab + __clz(Z0) * kFFStride, *r1 = tab + __clz(Z1) * kFFStride;
  const float4 a0 = *reinterpret_cast<const float4 *>(r0), a1 = *reinterpret_cast<const float4 *>(r1);
  const FF<F2> A = {vpack(a0.x, a1.x), vpack(a0.y, a1.y)};
  if constexpr (ALPHA == 1) {
    return A;
  } else {
    const FF<F2> B = {vpack(a0.z, a1.z), vpack(a0.w, a1.w)};
    const FF<F2> fz = word_ff2(Z0, Z1);
    if constexpr (ALPHA == 2) {
      return ff_add(A, ff_mul(B, fz));
    } else {
      const float4 b0 = *reinterpret_cast<const float4 *>(r0 + 4), b1 = *reinterpret_cast<const float4 *>(r1 + 4);
      const FF<F2> C = {vpack(b0.x, b1.x), vpack(b0.y, b1.y)};
      if constexpr (ALPHA == 3) {
        return ff_add(ff_mul(ff_add(ff_mul(C, fz), B), fz), A);
      } else {
        static_assert(ALPHA == 4, "DSI order 1..4");
        const FF<F2> D = {vpack(b0.z, b1.z), vpack(b0.w, b1.w)};
        const float2 e0 = *reinterpret_cast<const float2 *>(r0 + 8), e1 = *reinterpret_cast<const float2 *>(r1 + 8);
        const FF<F2> E = {vpack(e0.x, e1.x), vpack(e0.y, e1.y)};
        FF<F2> t = ff_add(ff_mul(D, fz), C);
        t = ff_add(ff_mul(t, fz), B);
        t = ff_add(ff_mul(t, fz), A);
        const float *oct = tab + kTabRows * kFFStride;
        const F2 sh = vpack(oct[Z0 >> 24], oct[Z1 >> 24]);
        const F2 sl = vfma(vsplat(0x1p-48f), vpack(oct[(Z0 >> 8) & 255u], oct[(Z1 >> 8) & 255u]),
                           vmul(vsplat(0x1p-24f), vpack(oct[(Z0 >> 16) & 255u], oct[(Z1 >> 16) & 255u])));
        return ff_add(t, ff_mul(E, ff_fast_two_sum(sh, sl)));
      }
    }
  }
}

// SI kernels in float-float: x = W 2^-32 (exact pair), q = x (1 - x),
// K_1 = pi^2/3 - 2 pi^2 q, K_2 = pi^4/45 - 2 pi^4/3 q^2 (Sec. 5.2, Bernoulli B_2 and B_4);
// the constants are the pairs of their FP64 values.
template <int ALPHA>
__device__ __forceinline__ FF<F2> si_ff2(uint32_t W0, uint32_t W1) {
  FF<F2> x = word_ff2(W0, W1);
  x.h = vmul(x.h, vsplat(0x1p-32f));
  x.l = vmul(x.l, vsplat(0x1p-32f));
  FF<F2> omx = ff_two_sum(vsplat(1.f), vneg(x.h));
  omx.l = vsub(omx.l, x.l);
  FF<F2> q = ff_mul(x, omx);
  auto cst = [](double v) -> FF<F2> {
    const float2 s = ff_split(v);
    return {vsplat(s.x), vsplat(s.y)};
  };
  if constexpr (ALPHA == 1) {
    return ff_add(cst(3.2898681336964528729), ff_mul(cst(-19.739208802178717238), q));
  } else {
    static_assert(ALPHA == 2, "SI smoothness 1..2");
    return ff_add(cst(2.1646464674222763831), ff_mul(cst(-64.939394022668291491), ff_mul(q, q)));
  }
}

template <int FAM, int ALPHA>
__device__ __forceinline__ FF<F2> kfac_ff2(const DiffTables &tb, uint32_t w0, uint32_t w1) {
  if constexpr (FAM == 0) return dsi_ff2<ALPHA>(reinterpret_cast<const float *>(tb.ktab), w0, w1);
  else return si_ff2<ALPHA>(w0, w1);
}

// Tables of the float-float sweep: the index tables and, for DSI kernels, the float-float rows.
template <int FAM, int ALPHA, int L>
__device__ __forceinline__ void build_all_ff(const ColJob &job, const uint32_t *Cr, const uint32_t *g,
                                             uint64_t tile_base, DiffTables &tb) {
  build_tables<L>(job, Cr, g, tile_base, tb);
  if constexpr (FAM == 0) build_dsi_tab_ff<ALPHA>(reinterpret_cast<float *>(tb.ktab));
}

// p = prod_j (1 + c_j K_j) - 1 for the L points of this thread as float-float pairs
// (ph[l] + pl[l], about 2^-46 relative per factor), two points per packed f32x2 operation.
// wff: the weights c_j as pairs (h, l).
template <int FAM, int ALPHA, int L>
__device__ __forceinline__ void column_sweep_ff(const ColJob &job, const DiffTables &tb, const float2 *wff,
                                                const uint32_t (&bi)[L], float (&ph)[L], float (&pl)[L]) {
  static_assert(L % 4 == 0, "quads of points");
  const uint32_t d = job.d;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  FF<F2> P[L / 2];
  const F2 zero = vsplat(0.f), one = vsplat(1.f);
#pragma unroll
  for (int h = 0; h < L / 2; ++h) P[h] = {zero, zero};
  for (uint32_t j = 0; j < d; ++j) {
    const float2 w = wff[j];
    const FF<F2> W = {vsplat(w.x), vsplat(w.y)};
    uint32_t base = 0;
    if constexpr (FAM == 0) base = tb.zlane[j * 32 + lane] ^ tb.zwarp[warp * d + j];
#pragma unroll
    for (int h = 0; h < L / 2; h += 2) {
      uint32_t z[4];
      diff_words4<FAM, L>(tb, base, bi, 2 * h, j, z);
      P[h] = ff_pm1_step(P[h], ff_mul(W, kfac_ff2<FAM, ALPHA>(tb, z[0], z[1])), one);
      P[h + 1] = ff_pm1_step(P[h + 1], ff_mul(W, kfac_ff2<FAM, ALPHA>(tb, z[2], z[3])), one);
    }
  }
#pragma unroll
  for (int h = 0; h < L / 2; ++h) {
    vunpack(P[h].h, ph[2 * h], ph[2 * h + 1]);
    vunpack(P[h].l, pl[2 * h], pl[2 * h + 1]);
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
    const T K = kfac<T, FAM, ALPHA>(tb, diff_word<FAM, L>(tb, job.d, base, bi_l, l, j));
    prod *= (j == jx) ? K : (T(1) + wT[j] * K);
  }
  return prod;
}

__device__ __forceinline__ float ratio(float a, float b) { return __fdividef(a, b); }  // 2 ulp
// Approximate reciprocal (PTX rcp.approx.ftz.f32, max 1 ulp; subnormals flush to 0): 1/0 = inf.
__device__ __forceinline__ float rcp_approx(float a) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
  return r;
}
// a / b in FP64 without the FP64 divide (GB300 has about two FP64 lanes per SM and cycle):
// the reciprocal of b by two Newton-Raphson steps r <- r + r (1 - b r), each squaring the
// relative error, from the FP32 reciprocal estimate of b (b's leading 24 bits, rel. error
// below 2^-22); the second step's error is below one unit in the last place, then one
// product: within 2 ulp of the rounded quotient (checked against the divide by
// qk_ratio_selftest).  Five FP64 operations; b outside [2^-100, 2^100] in magnitude, zero,
// subnormal, inf or NaN, takes the divide.
__device__ __forceinline__ double ratio(double a, double b) {
  const uint32_t hi = (uint32_t)__double2hiint(b), lo = (uint32_t)__double2loint(b);
  const uint32_t ex = (hi >> 20) & 0x7FFu;
  if (ex - 923u > 200u) return a / b;
  const uint32_t fb = (hi & 0x80000000u) | ((ex - 896u) << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29);
  double r = f2d_exact(rcp_approx(__uint_as_float(fb)));
  double e = fma(-b, r, 1.0);
  r = fma(r, e, r);
  e = fma(-b, r, 1.0);
  r = fma(r, e, r);
  return a * r;
}

// Warp sums of four per-lane values, the pair (a0, a1) of one dimension and (b0, b1) of
// the next, by a reduce-scatter: at the xor-16 step a lane keeps one dimension's pair and
// sends the other's, at the xor-8 step it keeps one value of that pair, and the last three
// steps finish one sum per group of 8 lanes.  Lane 0 ends with the total of a0, lane 8 of
// a1, lane 16 of b0 and lane 24 of b1 (every lane of a group of 8 holds its group's total).
// Each sum is formed in the same order of additions as a full xor butterfly, so the FP64
// totals equal those of one butterfly per value; FP32 totals are float-float pairs (s, e).
// 5 shuffle steps for 4 values instead of 20.
__device__ __forceinline__ void warp_sum4_ff(float a0, float a1, float b0, float b1, float &s, float &e) {
  const int lane = threadIdx.x & 31;
  const bool h16 = lane & 16, h8 = lane & 8;
  const float k0 = h16 ? b0 : a0, k1 = h16 ? b1 : a1;
  const float r0 = __shfl_xor_sync(0xffffffffu, h16 ? a0 : b0, 16);
  const float r1 = __shfl_xor_sync(0xffffffffu, h16 ? a1 : b1, 16);
  float s0, e0, s1, e1;
  two_sum(k0, r0, s0, e0);
  two_sum(k1, r1, s1, e1);
  s = h8 ? s1 : s0, e = h8 ? e1 : e0;
  const float rs = __shfl_xor_sync(0xffffffffu, h8 ? s0 : s1, 8);
  const float re = __shfl_xor_sync(0xffffffffu, h8 ? e0 : e1, 8);
  ff_merge(s, e, rs, re);
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) {
    const float s2 = __shfl_xor_sync(0xffffffffu, s, o), e2 = __shfl_xor_sync(0xffffffffu, e, o);
    ff_merge(s, e, s2, e2);
  }
}
__device__ __forceinline__ double warp_sum4(double a0, double a1, double b0, double b1) {
  const int lane = threadIdx.x & 31;
  const bool h16 = lane & 16, h8 = lane & 8;
  const double s0 = (h16 ? b0 : a0) + __shfl_xor_sync(0xffffffffu, h16 ? a0 : b0, 16);
  const double s1 = (h16 ? b1 : a1) + __shfl_xor_sync(0xffffffffu, h16 ? a1 : b1, 16);
  double s = (h8 ? s1 : s0) + __shfl_xor_sync(0xffffffffu, h8 ? s0 : s1, 8);
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// Gradient sweep: for each dimension j, warp-reduced sums over this warp's points of
// u_i dk1_i/dc_j and dk1_i/dc_j (float-float pairs in FP32 sweeps, doubles in FP64
// sweeps), written to red[warp][2d] and totalled by red_total, with
// dk1_i/dc_j = k1_i K_ij / (1 + c_j K_ij).  wk[l] = u_l k1_l, both zero for points with
// !ok[l]; uget(l) returns u_l and is called only for the rare exact zero of
// 1 + c_j K_ij, handled after the loop by the explicit product over the other dimensions.
// ALL_OK (unpacked sweeps): every point is valid, so no per-point validity select.
// Dimensions are reduced in pairs (warp_sum4*): an even dimension's two lane sums wait in
// registers for the next dimension's; an odd d leaves the last dimension to a butterfly.
template <typename T, int FAM, int ALPHA, int L, bool ALL_OK = false, typename UF>
__device__ __forceinline__ void gradient_sweep(const ColJob &job, const DiffTables &tb, const T *wT,
                                               const uint32_t (&bi)[L], const T (&k1)[L], const T (&wk)[L],
                                               const bool (&ok)[L], UF uget, double *red) {
  const uint32_t d = job.d;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr bool PACKED = sizeof(T) == 4 && L % 4 == 0;
  // packed form: points (2h, 2h+1) share one f32x2 fma / mul, with the two halves summed
  // separately; a zero 1 + c_j K gives an infinite reciprocal, so the sums come out
  // non-finite and the exact fallback below runs instead of a per-point zero test.
  // Points with !ok[l] carry wk[l] = k1[l] = 0 and add nothing (or a NaN, which again
  // sends the thread to the fallback, where they are skipped).
  unsigned long long WK[PACKED ? L / 2 : 1], K1[PACKED ? L / 2 : 1];
  if constexpr (PACKED) {
#pragma unroll
    for (int h = 0; h < L / 2; ++h) {
      WK[h] = pack_f2(wk[2 * h], wk[2 * h + 1]);
      K1[h] = pack_f2(k1[2 * h], k1[2 * h + 1]);
    }
  }
  T cu = T(0), c1 = T(0);  // lane sums of the even dimension of the current pair
  for (uint32_t j = 0; j < d; ++j) {
    const T wj = wT[j];
    T su = T(0), s1 = T(0);
    uint32_t base = 0;
    if constexpr (FAM == 0) base = tb.zlane[j * 32 + lane] ^ tb.zwarp[warp * d + j];
    bool anyzero = false;
    if constexpr (PACKED) {
      const unsigned long long W = pack_f2(wj, wj), ONE = pack_f2(1.f, 1.f);
      unsigned long long SU = pack_f2(0.f, 0.f), S1 = SU;
#pragma unroll
      for (int l = 0; l < L; l += 4) {
        uint32_t z[4];
        diff_words4<FAM, L>(tb, base, bi, l, j, z);
#pragma unroll
        for (int i = 0; i < 4; i += 2) {
          const int h = (l + i) >> 1;
          const T ka = kfac<T, FAM, ALPHA>(tb, z[i]), kb = kfac<T, FAM, ALPHA>(tb, z[i + 1]);
          const unsigned long long KK = pack_f2(ka, kb);
          float fa, fb;
          unpack_f2(fma_f2(W, KK, ONE), fa, fb);
          const unsigned long long Q = mul_f2(KK, pack_f2(rcp_approx(fa), rcp_approx(fb)));
          SU = fma_f2(WK[h], Q, SU);
          S1 = fma_f2(K1[h], Q, S1);
        }
      }
      float a, b;
      unpack_f2(SU, a, b);
      su = a + b;
      unpack_f2(S1, a, b);
      s1 = a + b;
      anyzero = !(isfinite(su) && isfinite(s1));
    } else {
      auto step = [&](int l, uint32_t z) {
        const T K = kfac<T, FAM, ALPHA>(tb, z);
        const T f = fmadd(wj, K, T(1));
        anyzero |= f == T(0);
        T q = ratio(K, f);
        if constexpr (!ALL_OK) q = ok[l] ? q : T(0);
        su = fmadd(wk[l], q, su);
        s1 = fmadd(k1[l], q, s1);
      };
      if constexpr (L % 4 == 0) {
#pragma unroll
        for (int l = 0; l < L; l += 4) {
          uint32_t z[4];
          diff_words4<FAM, L>(tb, base, bi, l, j, z);
#pragma unroll
          for (int i = 0; i < 4; ++i) step(l + i, z[i]);
        }
      } else {
#pragma unroll
        for (int l = 0; l < L; ++l) step(l, diff_word<FAM, L>(tb, d, base, bi[l], l, j));
      }
    }
    if (anyzero) {  // exact zeros of 1 + c_j K: use prod_{j' != j} (1 + c_j' K_j') directly
      su = T(0), s1 = T(0);
#pragma unroll
      for (int l = 0; l < L; ++l) {
        if (!ok[l]) continue;
        const T K = kfac<T, FAM, ALPHA>(tb, diff_word<FAM, L>(tb, d, base, bi[l], l, j));
        const T f = fmadd(wj, K, T(1));
        const T dk = f == T(0) ? dk_explicit<T, FAM, ALPHA, L>(job, tb, wT, bi[l], l, j) : k1[l] * ratio(K, f);
        su = fmadd(uget(l), dk, su);
        s1 += dk;
      }
    }
    if (!(j & 1) && j + 1 < d) {  // uniform over the warp: wait for the pair's odd dimension
      cu = su, c1 = s1;
      continue;
    }
    if constexpr (sizeof(T) == 4) {
      // float-float warp sums, kept as (hi, lo) pairs: no FP64 arithmetic per dimension
      float2 *r2 = reinterpret_cast<float2 *>(red) + (size_t)warp * 2 * d;
      if (j & 1) {
        float s, e;
        warp_sum4_ff(cu, c1, su, s1, s, e);
        if (!(lane & 7)) r2[((lane & 8) ? d : 0) + j - ((lane & 16) ? 0 : 1)] = make_float2(s, e);
      } else {
        float ue = 0.f, oe = 0.f;
        warp_sum_ff(su, ue);
        warp_sum_ff(s1, oe);
        if (lane == 0) {
          r2[j] = make_float2(su, ue);
          r2[d + j] = make_float2(s1, oe);
        }
      }
    } else {
      double *rw = red + (size_t)warp * 2 * d;
      if (j & 1) {
        const double s = warp_sum4(cu, c1, su, s1);
        if (!(lane & 7)) rw[((lane & 8) ? d : 0) + j - ((lane & 16) ? 0 : 1)] = s;
      } else {
        double du = su, d1 = s1;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          du += __shfl_xor_sync(0xffffffffu, du, o);
          d1 += __shfl_xor_sync(0xffffffffu, d1, o);
        }
        if (lane == 0) {
          rw[j] = du;
          rw[d + j] = d1;
        }
      }
    }
  }
}

// Entry q of the per-warp gradient partials red[warp][nq] summed over the warps: FP32
// sweeps leave float-float pairs (summed in float-float, converted once), FP64 sweeps
// doubles.
template <typename T>
__device__ __forceinline__ double red_total(const double *red, int warps, uint32_t nq, uint32_t q) {
  if constexpr (sizeof(T) == 4) {
    const float2 *r2 = reinterpret_cast<const float2 *>(red);
    float s = 0.f, e = 0.f;
    for (int w = 0; w < warps; ++w) {
      const float2 p = r2[(size_t)w * nq + q];
      ff_merge(s, e, p.x, p.y);
    }
    return (double)s + (double)e;
  } else {
    double s = 0.0;
    for (int w = 0; w < warps; ++w) s += red[(size_t)w * nq + q];
    return s;
  }
}

}  // namespace qk
