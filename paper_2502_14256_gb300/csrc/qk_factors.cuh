// One-dimensional kernel factors K_alpha evaluated from 32-bit words, in T =
// float or double, and the product-minus-one recurrence for the first column.
//
// DSI (arXiv 2502.14256, Sec. 5.3, Theorem; x = Z 2^-32, beta(x) = -floor(log2 x),
// t_nu = 2^(-nu beta), beta(0) = t_nu(0) = 0):
//   K_1 = 1 - 3 t_1 (Z != 0), K_1(0) = 1    (first-order Walsh kernel; the paper
//                                            defers order 1 to Dick & Pillichshammer)
//   K_2 = -1 - beta x + 5/2 (1 - t_1)
//   K_3 = -1 + beta x^2 - 5 (1 - t_1) x + 43/18 (1 - t_2)
//   K_4 = -1 - 2/3 beta x^3 + 5 (1 - t_1) x^2 - 43/9 (1 - t_2) x + 701/294 (1 - t_3)
//         + beta (S/48 - 1/42),  S = sum_a wal_{2^a}(x) 8^-a.
// With 32 digits S = 8/7 - 2 S', S' = sum over set digits x_{a+1} of 8^-a, so the
// last term equals -beta S'/24 (no cancellation between S/48 and 1/42).  S' is
// read off the word by spreading its leading bits three apart (octal digits).
//
// SI (Sec. 5.2): K_alpha(x) = (2 pi)^(2 alpha) / ((-1)^(alpha+1) (2 alpha)!) B_2alpha(x):
//   K_1 = pi^2/3 - 2 pi^2 x (1 - x),   K_2 = pi^4/45 - 2 pi^4/3 (x (1 - x))^2.
#pragma once

#include "qk_common.cuh"

namespace qk {

// Exact small integer -> T by the mantissa trick (one add, no conversion unit).
__device__ __forceinline__ float small_int_to(float, uint32_t v) {
  return __int_as_float(0x4B000000 | (int)v) - 8388608.0f;  // v < 2^23
}
__device__ __forceinline__ double small_int_to(double, uint32_t v) {
  return __hiloint2double(0x43300000, (int)v) - 4503599627370496.0;  // v < 2^32
}

// S' = sum_{a >= 0, bit (31-a) of Z set} 8^-a, to the precision of T.
__device__ __forceinline__ float octal_tail(float, uint32_t Z) {
  return __uint2float_rn(spread3_10(Z >> 22)) * 0x1p-27f;  // a = 0..9
}
__device__ __forceinline__ double octal_tail(double, uint32_t Z) {
  const uint32_t hi = spread3_10(Z >> 22);                     // a = 0..9
  const uint32_t t11 = (Z >> 11) & 0x7FFu;                     // a = 10..20
  const uint32_t lo = spread3_10(t11) | ((t11 >> 10) << 30);
  return small_int_to(0.0, hi) * 0x1p-27 + small_int_to(0.0, lo) * 0x1p-60;
}

template <typename T, int ALPHA>
__device__ __forceinline__ T dsi_factor(uint32_t Z) {
  const bool nz = Z != 0u;
  const int beta = nz ? (__clz(Z) + 1) : 0;
  const T t1 = nz ? exp2neg(T(), beta) : T(0);
  if constexpr (ALPHA == 1) {
    return nz ? (T(1) - T(3) * t1) : T(1);
  } else {
    const T x = word_to_unit(T(), Z);
    const T b = small_int_to(T(), (uint32_t)beta);
    if constexpr (ALPHA == 2) {
      return T(1.5) - b * x - T(2.5) * t1;
    } else if constexpr (ALPHA == 3) {
      const T t2 = t1 * t1;
      return T(-1) + b * x * x - T(5) * (T(1) - t1) * x + T(43.0 / 18.0) * (T(1) - t2);
    } else {
      static_assert(ALPHA == 4, "DSI order 1..4");
      const T t2 = t1 * t1;
      const T t3 = t2 * t1;
      const T x2 = x * x;
      const T sp = octal_tail(T(), Z);
      return T(-1) - T(2.0 / 3.0) * b * x2 * x + T(5) * (T(1) - t1) * x2 -
             T(43.0 / 9.0) * (T(1) - t2) * x + T(701.0 / 294.0) * (T(1) - t3) -
             b * sp * T(1.0 / 24.0);
    }
  }
}

template <typename T, int ALPHA>
__device__ __forceinline__ T si_factor(uint32_t W) {
  const T x = word_to_unit(T(), W);
  // x (1 - x): in FP64, 1 - x is exact (x has 32 significant bits), so x * (1 - x) and the
  // fused x - x * x both round the same real number once; the fused form is one operation
  T q;
  if constexpr (sizeof(T) == 8) q = fma(-x, x, x);
  else q = x * (T(1) - x);
  if constexpr (ALPHA == 1) {
    return T(3.2898681336964528729) - T(19.739208802178717238) * q;  // pi^2/3, 2 pi^2
  } else {
    static_assert(ALPHA == 2, "SI smoothness 1..2");
    return T(2.1646464674222763831) - T(64.939394022668291491) * (q * q);  // pi^4/45, 2pi^4/3
  }
}

// Family dispatch: FAM 0 = DSI (argument is the XOR difference word), 1 = SI
// (argument is the mod-2^32 difference word).
template <typename T, int FAM, int ALPHA>
__device__ __forceinline__ T factor(uint32_t w) {
  if constexpr (FAM == 0) return dsi_factor<T, ALPHA>(w);
  else return si_factor<T, ALPHA>(w);
}

// Fused multiply-add in the precision of the arguments (never promoted).
__device__ __forceinline__ float fmadd(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmadd(double a, double b, double c) { return fma(a, b, c); }

// p <- (1 + p)(1 + a) - 1, keeping p = prod(1 + a_j) - 1 with relative precision.
template <typename T>
__device__ __forceinline__ T pm1_step(T p, T a) { return fmadd(p, a, p + a); }

}  // namespace qk
