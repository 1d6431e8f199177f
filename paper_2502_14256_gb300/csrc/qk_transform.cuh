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

// ------------------------------------------------------------ element algebra
__device__ __forceinline__ float2 operator+(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 operator-(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
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
    k_transform_pass<KIND, E, NT><<<(unsigned)blocks, NT, smem, st>>>(x, p);
    int rc = check_launch("transform pass");
    if (rc) return rc;
  }
  return QK_OK;
}

}  // namespace qk
