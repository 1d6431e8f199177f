// Batched radix-2 transforms of length n = 2^m, tiled through shared memory.
//
//   WHT: multiplication by the Hadamard matrix H_m (arXiv 2502.14256, Sec. 5.3),
//        butterflies (a, b) -> (a + b, a - b); unnormalised.
//   DIT: FFTBR (Sec. 5.2): radix-2 decimation-in-time FFT whose input is already
//        in bit-reversed order (natural-order lattice data), output in natural
//        frequency order; butterfly (a, b) -> (a + W b, a - W b), W = e^{-2 pi i j/2^(b+1)}.
//   DIF: IFFTBR: decimation-in-frequency inverse FFT, natural-order frequency
//        input, bit-reversed (natural point order) output; conjugate twiddles.
//        Unnormalised (the caller applies 1/n).
//
// A pass applies the butterflies of k consecutive bits [s, s+k) of the element
// index.  A CTA loads one tile of 2^LOGE elements into shared memory with
// coalesced accesses: 2^c contiguous "column" elements (untransformed low bits)
// times 2^k "rows" at stride 2^s, or, for short vectors (m <= LOGE), 2^(LOGE-m)
// whole vectors.  Inside the tile the row bits are processed in rounds of up to
// 4 bits, each round a radix-16 transform held in registers, with a padded
// shared-memory layout between rounds.  The WHT stages commute; the FFTs run
// their stages in increasing (DIT) or decreasing (DIF) bit order, passes too.
#pragma once

#include <type_traits>
#include <vector>

#include "qk_common.cuh"

namespace qk {

enum XformKind { XF_WHT = 0, XF_DIT = 1, XF_DIF = 2 };

struct PassDesc {
  int m;              // log2 n
  int s;              // first transformed bit
  int k;              // transformed bits
  int c;              // contiguous column bits (multi-pass tiles)
  int small;          // 1: tile holds whole vectors (m <= LOGE)
  uint64_t vstride;   // elements between vectors
  uint64_t nvec;      // vectors
  double scale;       // multiply every stored element (last pass only)
};

template <typename E> struct ElemTraits;
template <> struct ElemTraits<float> { static constexpr int LOGE = 13, CMIN = 5, PAD = 5; };
template <> struct ElemTraits<double> { static constexpr int LOGE = 12, CMIN = 4, PAD = 4; };
template <> struct ElemTraits<float2> { static constexpr int LOGE = 12, CMIN = 4, PAD = 4; };
template <> struct ElemTraits<double2> { static constexpr int LOGE = 11, CMIN = 3, PAD = 3; };

template <typename E> struct ScalarOf;
template <> struct ScalarOf<float> { using type = float; };
template <> struct ScalarOf<double> { using type = double; };
template <> struct ScalarOf<float2> { using type = float; };
template <> struct ScalarOf<double2> { using type = double; };

// A complex value in float-float arithmetic on the FP32 pipes: h = (Re_h, Im_h) and
// l = (Re_l, Im_l) as packed f32x2 pairs, Re = Re_h + Re_l to about 2^-46 relative.  The
// transforms of the float-float column path run in it: GB300's FP64 rate is a small
// fraction of its FP32 rate, and a float-float butterfly costs a few dozen FP32 operations.
struct __align__(16) FFC {
  F2 h, l;
};
template <> struct ElemTraits<FFC> { static constexpr int LOGE = 11, CMIN = 3, PAD = 3; };
template <> struct ScalarOf<FFC> { using type = double; };

// ------------------------------------------------------------ element algebra
// FP32 complex addition as one packed f32x2 instruction (the same IEEE operation on both
// halves: the same results as two scalar additions, in half the instructions)
__device__ __forceinline__ float2 operator+(float2 a, float2 b) {
  float2 r;
  vunpack(vadd(vpack(a.x, a.y), vpack(b.x, b.y)), r.x, r.y);
  return r;
}
__device__ __forceinline__ float2 operator-(float2 a, float2 b) {
  float2 r;
  vunpack(vsub(vpack(a.x, a.y), vpack(b.x, b.y)), r.x, r.y);
  return r;
}
__device__ __forceinline__ double2 operator+(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 operator-(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 w) {
  return make_float2(fmaf(a.x, w.x, -a.y * w.y), fmaf(a.x, w.y, a.y * w.x));
}
__device__ __forceinline__ double2 cmul(double2 a, double2 w) {
  return make_double2(fma(a.x, w.x, -a.y * w.y), fma(a.x, w.y, a.y * w.x));
}
__device__ __forceinline__ float scale_elem(float a, double s) { return a * (float)s; }
__device__ __forceinline__ double scale_elem(double a, double s) { return a * s; }
__device__ __forceinline__ float2 scale_elem(float2 a, double s) { return make_float2(a.x * (float)s, a.y * (float)s); }
__device__ __forceinline__ double2 scale_elem(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
template <typename E> __device__ __forceinline__ E zero_elem();
template <> __device__ __forceinline__ float zero_elem<float>() { return 0.f; }
template <> __device__ __forceinline__ double zero_elem<double>() { return 0.0; }
template <> __device__ __forceinline__ float2 zero_elem<float2>() { return make_float2(0.f, 0.f); }
template <> __device__ __forceinline__ double2 zero_elem<double2>() { return make_double2(0.0, 0.0); }

__device__ __forceinline__ FFC operator+(FFC a, FFC b) {
  const FF<F2> r = ff_add(FF<F2>{a.h, a.l}, FF<F2>{b.h, b.l});
  return {r.h, r.l};
}
__device__ __forceinline__ FFC operator-(FFC a, FFC b) { return a + FFC{vneg(b.h), vneg(b.l)}; }
__device__ __forceinline__ F2 vswap(F2 a) {
  float x, y;
  vunpack(a, x, y);
  return vpack(y, x);
}
// a w = (a.re, a.im) (w.re, w.re) + (a.im, a.re) (-w.im, w.im), each product a float-float
// product of packed pairs
__device__ __forceinline__ FFC cmul(FFC a, FFC w) {
  float wrh, wih, wrl, wil;
  vunpack(w.h, wrh, wih);
  vunpack(w.l, wrl, wil);
  const FF<F2> p1 = ff_mul(FF<F2>{a.h, a.l}, FF<F2>{vpack(wrh, wrh), vpack(wrl, wrl)});
  const FF<F2> p2 = ff_mul(FF<F2>{vswap(a.h), vswap(a.l)}, FF<F2>{vpack(-wih, wih), vpack(-wil, wil)});
  const FF<F2> r = ff_add(p1, p2);
  return {r.h, r.l};
}
// the pair of two doubles (re, im): h = fl32(v), l = fl32(v - h)
__device__ __forceinline__ FFC ffc_from(double re, double im) {
  const float rh = __double2float_rn(re), ih = __double2float_rn(im);
  return {vpack(rh, ih), vpack(__double2float_rn(re - (double)rh), __double2float_rn(im - (double)ih))};
}
__device__ __forceinline__ double ffc_re(FFC a) {
  float h, i, l, j;
  vunpack(a.h, h, i);
  vunpack(a.l, l, j);
  return f2d_exact(h) + f2d_exact(l);
}
__device__ __forceinline__ double ffc_im(FFC a) {
  float h, i, l, j;
  vunpack(a.h, h, i);
  vunpack(a.l, l, j);
  return f2d_exact(i) + f2d_exact(j);
}
__device__ __forceinline__ FFC scale_elem(FFC a, double s) {
  const float2 sp = ff_split(s);
  const FF<F2> r = ff_mul(FF<F2>{a.h, a.l}, FF<F2>{vsplat(sp.x), vsplat(sp.y)});
  return {r.h, r.l};
}
template <> __device__ __forceinline__ FFC zero_elem<FFC>() { return {vsplat(0.f), vsplat(0.f)}; }

// Twiddle e^{sign i pi j / 2^b} for 0 <= j < 2^b.
__device__ __forceinline__ float2 twiddle(float2, uint64_t j, int b, float sign) {
  float sv, cv;
  sincospif(sign * __ull2float_rn(j) * exp2neg(0.f, b), &sv, &cv);
  return make_float2(cv, sv);
}
__device__ __forceinline__ double2 twiddle(double2, uint64_t j, int b, double sign) {
  double sv, cv;
  sincospi(sign * (double)j * exp2neg(0.0, b), &sv, &cv);
  return make_double2(cv, sv);
}
__device__ __forceinline__ FFC twiddle(FFC, uint64_t j, int b, double sign) {
  double sv, cv;
  sincospi(sign * (double)j * exp2neg(0.0, b), &sv, &cv);
  return ffc_from(cv, sv);
}

// e^{sign i pi k / 8} for k = 0..7: cos and sin of multiples of pi/8 (k is a compile-time
// constant wherever this is called, so the switch folds away).
template <typename E, typename S>
__device__ __forceinline__ E root8(int k, S sign) {
  constexpr double C1 = 0.92387953251128675613, S1 = 0.38268343236508977173, R2 = 0.70710678118654752440;
  double c = 1.0, s = 0.0;
  switch (k & 7) {
    case 1: c = C1, s = S1; break;
    case 2: c = R2, s = R2; break;
    case 3: c = S1, s = C1; break;
    case 4: c = 0.0, s = 1.0; break;
    case 5: c = -S1, s = C1; break;
    case 6: c = -R2, s = R2; break;
    case 7: c = -C1, s = S1; break;
    default: break;
  }
  E w;
  w.x = (S)c;
  w.y = (S)(sign * s);
  return w;
}

template <>
__device__ __forceinline__ FFC root8<FFC, double>(int k, double sign) {
  const double2 w = root8<double2>(k, sign);
  const float2 c = ff_split(w.x), s = ff_split(w.y);
  return {vpack(c.x, s.x), vpack(c.y, s.y)};
}

template <typename E>
__device__ __forceinline__ int pad_index(int e) { return e + (e >> ElemTraits<E>::PAD); }

// Global offset of tile element e and its index inside its vector.
struct TileMap {
  uint64_t base;       // offset of tile element 0
  uint64_t gbase;      // index within the vector of element 0
  int c, k, s;
  int small;
  uint64_t vstride;
  uint64_t first_vec, nvec;
  int m;
  __device__ __forceinline__ bool valid(int e) const {
    if (!small) return true;
    return first_vec + (uint64_t)(e >> m) < nvec;
  }
  __device__ __forceinline__ uint64_t offset(int e) const {
    if (small) return base + (uint64_t)(e >> m) * vstride + (uint64_t)(e & ((1 << m) - 1));
    const int col = e & ((1 << c) - 1);
    const int row = e >> c;
    return base + ((uint64_t)row << s) + (uint64_t)col;
  }
  __device__ __forceinline__ uint64_t gindex(int e) const {
    if (small) return (uint64_t)(e & ((1 << m) - 1));
    const int col = e & ((1 << c) - 1);
    const int row = e >> c;
    return gbase + ((uint64_t)row << s) + (uint64_t)col;
  }
};

__device__ __forceinline__ TileMap make_tilemap(const PassDesc &p, int LOGE, uint64_t blk) {
  TileMap t;
  t.c = p.c;
  t.k = p.k;
  t.s = p.s;
  t.small = p.small;
  t.vstride = p.vstride;
  t.nvec = p.nvec;
  t.m = p.m;
  if (p.small) {
    const uint64_t per = 1ull << (LOGE - p.m);
    t.first_vec = blk * per;
    t.base = t.first_vec * p.vstride;
    t.gbase = 0;
  } else {
    const int other = p.m - p.k - p.c;
    const uint64_t tiles = 1ull << other;
    const uint64_t v = blk >> other;
    const uint64_t tau = blk & (tiles - 1);
    const int lo_bits = p.s - p.c;
    const uint64_t olo = tau & ((1ull << lo_bits) - 1);
    const uint64_t ohi = tau >> lo_bits;
    t.first_vec = v;
    t.gbase = (ohi << (p.s + p.k)) + (olo << p.c);
    t.base = v * p.vstride + t.gbase;
  }
  return t;
}

// Radix-2^R butterflies over R row bits starting at tile bit position `pos`
// (global bit gb0), on the 2^R elements v[] of one group.
template <int KIND, int R, typename E>
__device__ __forceinline__ void radix_round(E (&v)[1 << R], uint64_t glow, int gb0) {
  using S = typename ScalarOf<E>::type;
  if constexpr (KIND == XF_WHT) {
#pragma unroll
    for (int h = 0; h < R; ++h) {
#pragma unroll
      for (int q = 0; q < (1 << R); ++q) {
        if (!(q & (1 << h))) {
          const E a = v[q], b = v[q | (1 << h)];
          v[q] = a + b;
          v[q | (1 << h)] = a - b;
        }
      }
    }
  } else if constexpr (KIND == XF_DIT) {
    // the twiddle of stage bg for j = glow + (ql << gb0) factors into e^{-i pi glow / 2^bg}
    // (one per stage and group) times e^{-i pi ql / 2^h}, an eighth root of -1 (constant);
    // the per-stage factors are successive squares of the top stage's
    E bases[R];
    bases[R - 1] = twiddle(E(), glow, gb0 + R - 1, S(-1));
#pragma unroll
    for (int h = R - 2; h >= 0; --h) bases[h] = cmul(bases[h + 1], bases[h + 1]);
#pragma unroll
    for (int h = 0; h < R; ++h) {
      const E base = bases[h];
#pragma unroll
      for (int q = 0; q < (1 << R); ++q) {
        if (!(q & (1 << h))) {
          const int ql = q & ((1 << h) - 1);
          const E w = ql == 0 ? base : cmul(base, root8<E>(ql << (3 - h), S(-1)));
          const E a = v[q], b = cmul(v[q | (1 << h)], w);
          v[q] = a + b;
          v[q | (1 << h)] = a - b;
        }
      }
    }
  } else {
    E bases[R];
    bases[R - 1] = twiddle(E(), glow, gb0 + R - 1, S(1));
#pragma unroll
    for (int h = R - 2; h >= 0; --h) bases[h] = cmul(bases[h + 1], bases[h + 1]);
#pragma unroll
    for (int h = R - 1; h >= 0; --h) {
      const E base = bases[h];
#pragma unroll
      for (int q = 0; q < (1 << R); ++q) {
        if (!(q & (1 << h))) {
          const int ql = q & ((1 << h) - 1);
          const E w = ql == 0 ? base : cmul(base, root8<E>(ql << (3 - h), S(1)));
          const E a = v[q], b = v[q | (1 << h)];
          v[q] = a + b;
          v[q | (1 << h)] = cmul(a - b, w);
        }
      }
    }
  }
}

// One round over R row bits [b, b+R) of the tile (tile bit position c + b).
template <int KIND, int R, typename E, int LOGE, int NT>
__device__ __forceinline__ void tile_round(E *sm, const TileMap &tm, int b) {
  constexpr int E_ = 1 << LOGE;
  constexpr int G = E_ >> R;
  const int pos = (tm.small ? 0 : tm.c) + b;
  const int gb0 = tm.s + b;
  for (int g = threadIdx.x; g < G; g += NT) {
    const int lowmask = (1 << pos) - 1;
    const int e0 = (g & lowmask) | ((g >> pos) << (pos + R));
    E v[1 << R];
#pragma unroll
    for (int q = 0; q < (1 << R); ++q) v[q] = sm[pad_index<E>(e0 | (q << pos))];
    uint64_t glow = 0;
    if constexpr (KIND != XF_WHT) glow = tm.gindex(e0) & ((1ull << gb0) - 1);
    radix_round<KIND, R>(v, glow, gb0);
#pragma unroll
    for (int q = 0; q < (1 << R); ++q) sm[pad_index<E>(e0 | (q << pos))] = v[q];
  }
}

template <int KIND, typename E, int LOGE, int NT>
__device__ __forceinline__ void tile_rounds(E *sm, const TileMap &tm, int k) {
  auto run = [&](int b, int r) {
    switch (r) {
      case 1: tile_round<KIND, 1, E, LOGE, NT>(sm, tm, b); break;
      case 2: tile_round<KIND, 2, E, LOGE, NT>(sm, tm, b); break;
      case 3: tile_round<KIND, 3, E, LOGE, NT>(sm, tm, b); break;
      default: tile_round<KIND, 4, E, LOGE, NT>(sm, tm, b); break;
    }
    __syncthreads();
  };
  if constexpr (KIND == XF_DIF) {
    // descending bit order: rounds from the top
    int b = k;
    while (b > 0) {
      const int r = b >= 4 ? 4 : b;
      b -= r;
      run(b, r);
    }
  } else {
    for (int b = 0; b < k; b += 4) run(b, (k - b) >= 4 ? 4 : (k - b));
  }
}

template <int KIND, typename E, int NT>
__global__ void __launch_bounds__(NT) k_transform_pass(E *__restrict__ x, PassDesc p) {
  constexpr int LOGE = ElemTraits<E>::LOGE;
  constexpr int E_ = 1 << LOGE;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  E *sm = reinterpret_cast<E *>(smem_raw);
  const TileMap tm = make_tilemap(p, LOGE, blockIdx.x);
  constexpr int PER = E_ / NT;  // elements per thread; all loads issued before any is used
  E r[PER];
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int e = threadIdx.x + i * NT;
    r[i] = tm.valid(e) ? x[tm.offset(e)] : zero_elem<E>();
  }
#pragma unroll
  for (int i = 0; i < PER; ++i) sm[pad_index<E>(threadIdx.x + i * NT)] = r[i];
  __syncthreads();
  tile_rounds<KIND, E, LOGE, NT>(sm, tm, p.k);
  const bool do_scale = p.scale != 1.0;
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int e = threadIdx.x + i * NT;
    E v = sm[pad_index<E>(e)];
    if (do_scale) v = scale_elem(v, p.scale);
    if (tm.valid(e)) x[tm.offset(e)] = v;
  }
}

// FP32 complex passes (FFTBR / IFFTBR) that keep the tile in registers between rounds:
// 4096 elements, 256 threads x 16.  A pass over K = 4..8 or 12 row bits (c = 12 - K
// contiguous column bits) runs its butterflies in rounds of up to 4 row bits on the
// thread's registers; between rounds one padded shared-memory transpose regroups the
// elements so that the next round's bits are in registers.  Register layout at row-bit
// offset b: thread t = col | rowlow << c | rowhigh << (c + b) holds register l at row
// rowlow | l << b | rowhigh << (b + 4).  Rounds follow k_transform_pass: DIT upwards from
// bit 0, the last round holding the R = K mod 4 top bits (layout b = K - 4, register bits
// [4 - R, 4)); DIF downwards from the top, the last round holding the R bottom bits (layout
// b = 0, register bits [0, R)); each partial round runs for every value of the other
// register bits.  Global loads and stores use a
// layout in which a warp covers whole 128-byte lines: the round layout itself where
// c >= 4, and b = 8 (element t + 256 l) for K = 12, whose b = 0 end takes one more
// transpose.  Butterflies and twiddles are those of radix_round: the same results as
// k_transform_pass, bit for bit.
template <int K>
__device__ __forceinline__ int fft_reg_elem(int t, int b, int l) {
  constexpr int C = 12 - K;
  const int col = t & ((1 << C) - 1);
  const int rowlow = (t >> C) & ((1 << b) - 1);
  const int rowhigh = t >> (C + b);
  return col | ((rowlow | (l << b) | (rowhigh << (b + 4))) << C);
}

template <int K>
__device__ __forceinline__ void fft_reg_relayout(float2 (&v)[16], float2 *sm, int from_b, int to_b) {
  const int t = threadIdx.x;
#pragma unroll
  for (int l = 0; l < 16; ++l) sm[pad_index<float2>(fft_reg_elem<K>(t, from_b, l))] = v[l];
  __syncthreads();
#pragma unroll
  for (int l = 0; l < 16; ++l) v[l] = sm[pad_index<float2>(fft_reg_elem<K>(t, to_b, l))];
  __syncthreads();
}

// Butterflies on register bits [H0, H0 + R) in layout b, for each value of the other bits.
template <int KIND, int K, int R, int H0>
__device__ __forceinline__ void fft_reg_round(float2 (&v)[16], const TileMap &tm, int b) {
  constexpr int NO = 1 << (4 - R);  // values of the other register bits
  const int gb0 = tm.s + b + H0;
#pragma unroll
  for (int o = 0; o < NO; ++o) {
    // other bits: below H0 they are o's low bits, above H0 + R its high bits
    const int olow = o & ((1 << H0) - 1), ohigh = o >> H0;
    float2 g[1 << R];
#pragma unroll
    for (int q = 0; q < (1 << R); ++q) g[q] = v[olow | (q << H0) | (ohigh << (H0 + R))];
    const uint64_t glow = tm.gindex(fft_reg_elem<K>(threadIdx.x, b, olow | (ohigh << (H0 + R)))) &
                          ((1ull << gb0) - 1);
    radix_round<KIND, R, float2>(g, glow, gb0);
#pragma unroll
    for (int q = 0; q < (1 << R); ++q) v[olow | (q << H0) | (ohigh << (H0 + R))] = g[q];
  }
}

// One tile of a pass: load, all rounds, store (times scale).  CG: loads bypass L1 (data
// written by other CTAs of the same launch).
template <int KIND, int K, bool CG>
__device__ __forceinline__ void fft_reg_tile(float2 *__restrict__ x, const TileMap &tm, float2 *sm, double scale) {
  static_assert((K >= 4 && K <= 8) || K == 12, "4..8 or 12 row bits");
  constexpr int F = K / 4, RP = K % 4;  // full rounds, bits of the partial round
  // DIT: full rounds at b = 0, 4, ..., then the top RP bits in layout K - 4.
  // DIF: full rounds at b = K - 4, K - 8, ..., then the bottom RP bits in layout 0.
  constexpr int B_FIRST = KIND == XF_DIF ? K - 4 : 0;
  constexpr int B_LAST = KIND == XF_DIF ? 0 : K - 4;
  constexpr int B_IO_IN = K == 12 ? 8 : B_FIRST;
  constexpr int B_IO_OUT = K == 12 ? 8 : B_LAST;
  const int t = threadIdx.x;
  float2 v[16];
#pragma unroll
  for (int l = 0; l < 16; ++l) {
    const float2 *src = x + tm.offset(fft_reg_elem<K>(t, B_IO_IN, l));
    v[l] = CG ? __ldcg(src) : *src;
  }
  if constexpr (B_IO_IN != B_FIRST) fft_reg_relayout<K>(v, sm, B_IO_IN, B_FIRST);
  int bcur = B_FIRST;
#pragma unroll
  for (int rd = 0; rd < F; ++rd) {
    const int b = KIND == XF_DIF ? K - 4 - 4 * rd : 4 * rd;
    if (b != bcur) {
      fft_reg_relayout<K>(v, sm, bcur, b);
      bcur = b;
    }
    fft_reg_round<KIND, K, 4, 0>(v, tm, b);
  }
  if constexpr (RP > 0) {
    if (bcur != B_LAST) {
      fft_reg_relayout<K>(v, sm, bcur, B_LAST);
      bcur = B_LAST;
    }
    if constexpr (KIND == XF_DIF) fft_reg_round<KIND, K, RP, 0>(v, tm, 0);
    else fft_reg_round<KIND, K, RP, 4 - RP>(v, tm, K - 4);
  }
  if (bcur != B_IO_OUT) fft_reg_relayout<K>(v, sm, bcur, B_IO_OUT);
  const bool do_scale = scale != 1.0;
#pragma unroll
  for (int l = 0; l < 16; ++l) {
    float2 w = v[l];
    if (do_scale) w = scale_elem(w, scale);
    x[tm.offset(fft_reg_elem<K>(t, B_IO_OUT, l))] = w;
  }
}

template <int KIND, int K>
__global__ void __launch_bounds__(256) k_fft_reg(float2 *__restrict__ x, PassDesc p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  fft_reg_tile<KIND, K, false>(x, make_tilemap(p, 12, blockIdx.x), reinterpret_cast<float2 *>(smem_raw), p.scale);
}

// Both passes of an FP32 complex transform of n = 2^(12 + KH) (KH = 4..8) in ONE launch of
// resident CTAs taking tiles in WhtSched ticket order: FFTBR runs the contiguous 12-bit
// tiles first and the column tiles of the high KH bits second, IFFTBR the reverse; the
// second pass of a vector starts after all its first-pass tiles are published (bounded
// wait: past spin_limit tries the tile is skipped and QK_STATUS_TIMEOUT set).  The same
// tiles and butterflies as the two launches: the same results, bit for bit.
template <int KIND, int KH>
__global__ void __launch_bounds__(256) k_fft_persist(float2 *__restrict__ x, double scale, WhtSched sc,
                                                     uint32_t *__restrict__ ctr, uint32_t *status,
                                                     uint32_t spin_limit) {
  constexpr int M = 12 + KH;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ uint32_t s_item[2], s_ok[2];  // as in the persistent FWHT: item k's slots are k & 1
  float2 *sm = reinterpret_cast<float2 *>(smem_raw);
  uint32_t *ticket = ctr, *done = ctr + 1;
  const int t = threadIdx.x;
  const uint32_t total = sc.total(), T_ = 1u << sc.lt;
  const PassDesc plo{M, 0, 12, 0, 0, 1ull << M, sc.nvec, 1.0};
  const PassDesc phi{M, 12, KH, 12 - KH, 0, 1ull << M, sc.nvec, 1.0};
  if (t == 0) s_item[0] = atomicAdd(ticket, 1u);
  __syncthreads();
  for (int k = 0;; ++k) {
    const uint32_t it = s_item[k & 1];
    if (it >= total) break;
    if (t == 0) s_item[(k + 1) & 1] = atomicAdd(ticket, 1u);
    uint32_t v, tile;
    bool second;
    sc.decode(it, v, tile, second);
    const uint64_t blk = ((uint64_t)v << sc.lt) + tile;
    if (!second) {
      if constexpr (KIND == XF_DIF) fft_reg_tile<KIND, KH, false>(x, make_tilemap(phi, 12, blk), sm, 1.0);
      else fft_reg_tile<KIND, 12, false>(x, make_tilemap(plo, 12, blk), sm, 1.0);
      __syncthreads();  // every thread's stores precede thread 0's release
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
        if constexpr (KIND == XF_DIF) fft_reg_tile<KIND, 12, true>(x, make_tilemap(plo, 12, blk), sm, scale);
        else fft_reg_tile<KIND, KH, true>(x, make_tilemap(phi, 12, blk), sm, scale);
      }
    }
  }
}

// Host: split the m bits into passes.
template <typename E>
inline std::vector<PassDesc> plan_passes(int m, uint64_t vstride, uint64_t nvec) {
  constexpr int LOGE = ElemTraits<E>::LOGE, CMIN = ElemTraits<E>::CMIN;
  std::vector<PassDesc> out;
  if (m <= LOGE) {
    out.push_back(PassDesc{m, 0, m, 0, 1, vstride, nvec, 1.0});
    return out;
  }
  out.push_back(PassDesc{m, 0, LOGE, 0, 0, vstride, nvec, 1.0});
  int s = LOGE, rem = m - LOGE;
  const int kmax = LOGE - CMIN;
  while (rem > 0) {
    // balance the remaining bits over the fewest passes
    const int np = (rem + kmax - 1) / kmax;
    const int kk = (rem + np - 1) / np;
    out.push_back(PassDesc{m, s, kk, LOGE - kk, 0, vstride, nvec, 1.0});
    s += kk;
    rem -= kk;
  }
  return out;
}

template <typename E>
inline uint64_t pass_blocks(const PassDesc &p) {
  constexpr int LOGE = ElemTraits<E>::LOGE;
  if (p.small) {
    const uint64_t per = 1ull << (LOGE - p.m);
    return (p.nvec + per - 1) / per;
  }
  return p.nvec << (p.m - p.k - p.c);
}

template <typename E>
inline size_t pass_smem() {
  constexpr int LOGE = ElemTraits<E>::LOGE, PAD = ElemTraits<E>::PAD;
  return (size_t)((1 << LOGE) + ((1 << LOGE) >> PAD)) * sizeof(E);
}

// Run a complete transform of `nvec` vectors of length 2^m, in place.
template <int KIND, typename E>
int run_transform(E *x, int m, uint64_t vstride, uint64_t nvec, double scale, cudaStream_t st) {
  constexpr int NT = 256;
  std::vector<PassDesc> passes = plan_passes<E>(m, vstride, nvec);
  if (KIND == XF_DIF) {
    std::vector<PassDesc> rev(passes.rbegin(), passes.rend());
    passes.swap(rev);
  }
  passes.back().scale = scale;
  const size_t smem = pass_smem<E>();
  smem_optin<k_transform_pass<KIND, E, NT>>(smem);
  for (const PassDesc &p : passes) {
    const uint64_t blocks = pass_blocks<E>(p);
    if (blocks == 0) continue;
    if (blocks > 0x7FFFFFFFull) return fail(QK_EINVAL, "transform grid too large");
    if constexpr (KIND != XF_WHT && std::is_same<E, float2>::value) {
      // FP32 complex tiles of 4..8 or 12 row bits: registers between rounds
      if (!p.small && p.c + p.k == 12 && ((p.k >= 4 && p.k <= 8) || p.k == 12)) {
        switch (p.k) {
          case 4: k_fft_reg<KIND, 4><<<(unsigned)blocks, NT, smem, st>>>(x, p); break;
          case 5: k_fft_reg<KIND, 5><<<(unsigned)blocks, NT, smem, st>>>(x, p); break;
          case 6: k_fft_reg<KIND, 6><<<(unsigned)blocks, NT, smem, st>>>(x, p); break;
          case 7: k_fft_reg<KIND, 7><<<(unsigned)blocks, NT, smem, st>>>(x, p); break;
          case 8: k_fft_reg<KIND, 8><<<(unsigned)blocks, NT, smem, st>>>(x, p); break;
          default: k_fft_reg<KIND, 12><<<(unsigned)blocks, NT, smem, st>>>(x, p); break;
        }
        int rc = check_launch("transform pass (registers)");
        if (rc) return rc;
        continue;
      }
    }
    k_transform_pass<KIND, E, NT><<<(unsigned)blocks, NT, smem, st>>>(x, p);
    int rc = check_launch("transform pass");
    if (rc) return rc;
  }
  return QK_OK;
}

}  // namespace qk
