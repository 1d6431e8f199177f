// Spectral operations of arXiv 2502.14256, Sec. 5.4, on top of the tile
// transforms: eigenvalues, solves, matrix-vector products, and the marginal
// log-likelihood with its gradient carried back through the transform.
//
// Normalisation: the transforms are unnormalised (H y, or the DFT of the data
// in linear order).  With Y = H y (or DFT(y_lin)):
//   lambda = H k_1 + eta,  K^-1 y = H (Y / lambda) / n,  K y = H (Y * lambda) / n,
//   y^T K^-1 y = sum |Y_w|^2 / (n lambda_w),  log det K = sum log lambda_w,
//   dMLL/dlambda_w = g_w = (|Y_w|^2 / (n lambda_w^2) - 1 / lambda_w) / 2,
//   dMLL/dc_j = sum_i (H g)_i dk1_i/dc_j,  dMLL/deta = sum_w g_w.
// For lattices H is replaced by the DIT FFT on natural-order input (FFTBR) and
// the inverse by the conjugate DIF FFT with natural-order output (IFFTBR); the
// kernel column is real and symmetric in linear order, so lambda and H g are real.
#include <cmath>
#include <cstring>
#include <type_traits>

#include "qk_common.cuh"
#include "qk_internal.h"
#include "qk_transform.cuh"

namespace qk {

// ------------------------------------------------------------- small kernels
template <typename T>
__device__ __forceinline__ double re(T v) { return (double)v; }
__device__ __forceinline__ double re(float2 v) { return (double)v.x; }
__device__ __forceinline__ double re(double2 v) { return v.x; }
template <typename T>
__device__ __forceinline__ double abs2(T v) { return (double)v * (double)v; }
__device__ __forceinline__ double abs2(float2 v) { return (double)v.x * v.x + (double)v.y * v.y; }
__device__ __forceinline__ double abs2(double2 v) { return v.x * v.x + v.y * v.y; }
template <typename E> __device__ __forceinline__ E from_real(double v);
template <> __device__ __forceinline__ float from_real<float>(double v) { return (float)v; }
template <> __device__ __forceinline__ double from_real<double>(double v) { return v; }
template <> __device__ __forceinline__ float2 from_real<float2>(double v) { return make_float2((float)v, 0.f); }
template <> __device__ __forceinline__ double2 from_real<double2>(double v) { return make_double2(v, 0.0); }
template <typename E> __device__ __forceinline__ E mul_real(E v, double s);
template <> __device__ __forceinline__ float mul_real<float>(float v, double s) { return (float)((double)v * s); }
template <> __device__ __forceinline__ double mul_real<double>(double v, double s) { return v * s; }
template <> __device__ __forceinline__ float2 mul_real<float2>(float2 v, double s) {
  return make_float2((float)((double)v.x * s), (float)((double)v.y * s));
}
template <> __device__ __forceinline__ double2 mul_real<double2>(double2 v, double s) {
  return make_double2(v.x * s, v.y * s);
}

__device__ __forceinline__ uint64_t gtid() { return (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ uint64_t gstride() { return (uint64_t)gridDim.x * blockDim.x; }

// real T -> element E (copy or complex with zero imaginary part)
template <typename T, typename E>
__global__ void k_load_real(const T *__restrict__ in, E *__restrict__ out, uint64_t count) {
  for (uint64_t i = gtid(); i < count; i += gstride()) out[i] = from_real<E>((double)in[i]);
}

// real part of E -> T, times scale
template <typename E, typename T>
__global__ void k_store_real(const E *__restrict__ in, T *__restrict__ out, uint64_t count, double scale) {
  for (uint64_t i = gtid(); i < count; i += gstride()) out[i] = (T)(re(in[i]) * scale);
}

// Real transform values x > 0 (finite) tested without FP64 compares.
__device__ __forceinline__ bool pos_finite(float x) { return x > 0.f && x <= 3.4028234663852886e38f; }
__device__ __forceinline__ bool pos_finite(double x) {
  const long long b = __double_as_longlong(x);
  return b > 0 && b < 0x7FF0000000000000ll;
}

// lambda = zmul * Re(X) + [form P] zeta n delta_{w0} + eta, with the sign test.  Real
// transforms take a short path for the usual entry (x > 0 away from w = 0, zmul > 0,
// eta > 0): then lambda >= eta > 0 exactly, so neither test can fire, and lambda costs one
// FP64 FMA on x widened by integer operations (GB300's FP64 conversion and compare run at
// the rate of its FP64 adder).  The value is the same FMA as the general path's.
template <typename E>
__global__ void k_lam_final(const E *__restrict__ X, double *__restrict__ lam, uint64_t total, int m,
                            double zmul, double dc, double eta, uint32_t *status) {
  bool bad = false, floored = false;
  const uint64_t mask = (1ull << m) - 1;
  const bool shortcut = zmul > 0.0 && eta > 0.0;
  for (uint64_t i = gtid(); i < total; i += gstride()) {
    if constexpr (std::is_same<E, float>::value || std::is_same<E, double>::value) {
      const E x = X[i];
      if (shortcut && (i & mask) != 0 && pos_finite(x)) {
        lam[i] = fma(zmul, f2d_exact(x), eta);
        continue;
      }
    }
    double v = fma(zmul, re(X[i]), eta);
    if ((i & mask) == 0) v += dc;
    if (eta > 0.0 && !(v >= eta)) {  // K + eta I has no eigenvalue below eta: rounding
      v = eta;
      floored = true;
    }
    lam[i] = v;
    bad |= !(v > 0.0);
  }
  if (bad && status) atomicOr(status, (uint32_t)QK_STATUS_NOTPD);
  if (floored && status) atomicOr(status, (uint32_t)QK_STATUS_FLOOR);
}

// X[v][w] *= fac / lambda[v / nrhs][w] (mode 0) or fac * lambda (mode 1), in FP64.
template <typename E>
__global__ void k_scale_lam(E *__restrict__ X, const double *__restrict__ lam, uint64_t total, int m,
                            uint32_t nrhs, double fac, int mode) {
  const uint64_t mask = (1ull << m) - 1;
  for (uint64_t i = gtid(); i < total; i += gstride()) {
    const uint64_t v = i >> m, w = i & mask;
    const double l = lam[((v / nrhs) << m) + w];
    X[i] = mul_real(X[i], mode == 0 ? fac / l : fac * l);
  }
}

template <typename E, typename T>
__global__ void k_residual(const T *__restrict__ y, const E *__restrict__ Kc, T *__restrict__ r, uint64_t count,
                           double scale) {
  for (uint64_t i = gtid(); i < count; i += gstride()) r[i] = (T)((double)y[i] - re(Kc[i]) * scale);
}

template <typename T>
__global__ void k_add(T *__restrict__ c, const T *__restrict__ dc, uint64_t count) {
  for (uint64_t i = gtid(); i < count; i += gstride()) c[i] += dc[i];
}

constexpr int kRedNT = 256;

// Per vector: FP64 partial sums of y over gridDim.x contiguous chunks, out[v][chunk] (the
// posterior mean needs the sum with relative accuracy, and for a centred integrand it is
// a small difference of large terms; k_mll_final adds the chunks).
template <typename T>
__global__ void k_sum_rows(const T *__restrict__ y, int m, double *__restrict__ out) {
  __shared__ double sh[32];
  const uint64_t n = 1ull << m, chunk = (n + gridDim.x - 1) / gridDim.x;
  const uint64_t lo = (uint64_t)blockIdx.x * chunk, hi = lo + chunk < n ? lo + chunk : n;
  const T *yv = y + (uint64_t)blockIdx.y * n;
  double s = 0.0;
  for (uint64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) s += (double)yv[i];
  const double t = block_sum(s, sh);
  if (threadIdx.x == 0) out[(uint64_t)blockIdx.y * gridDim.x + blockIdx.x] = t;
}

// Per vector: quad and sum g partials; overwrite X with g (real); keep Re Y_0.
template <typename E>
__global__ void k_mll_spectral(E *__restrict__ X, const double *__restrict__ lam, int m, uint32_t nrhs,
                               double *__restrict__ part, double *__restrict__ y0) {
  __shared__ double sh[32];
  const uint64_t n = 1ull << m;
  const uint32_t v = blockIdx.y;
  const double *lr = lam + (uint64_t)(v / nrhs) * n;
  E *xv = X + (uint64_t)v * n;
  double q = 0.0, gs = 0.0;
  const double inv_n = 1.0 / (double)n;
  for (uint64_t w = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; w < n; w += (uint64_t)gridDim.x * blockDim.x) {
    const E Y = xv[w];
    const double l = lr[w];
    const double a = abs2(Y) * inv_n / l;
    q += a;
    const double g = 0.5 * (a - 1.0) / l;
    gs += g;
    xv[w] = from_real<E>(g);
  }
  const double sq = block_sum(q, sh);
  const double sg = block_sum(gs, sh);
  if (threadIdx.x == 0) {
    part[((uint64_t)v * gridDim.x + blockIdx.x) * 2 + 0] = sq;
    part[((uint64_t)v * gridDim.x + blockIdx.x) * 2 + 1] = sg;
  }
}

// ------------------------------------------ lattices: two real vectors per complex transform
// The DFT is linear and maps a real vector a to a Hermitian A (A_{n-k} = conj A_k).  So two
// real vectors a, b travel as the one complex vector z = a + i b, whose transform Z = A + i B
// splits per frequency pair (k, n - k) as
//   A_k = (Z_k + conj Z_{n-k}) / 2,   B_k = (Z_k - conj Z_{n-k}) / (2 i),
// and the inverse transform of C + i D with C, D Hermitian is c + i d with c, d real.  The
// kernel column is real and symmetric in linear order, so its transform is real: A = Re Z,
// B = Im Z directly.  Vector v of a batch of nvec lives in pair v / 2 as its real (v even) or
// imaginary (v odd) part; an odd batch leaves the last pair's imaginary part zero.  Every
// lattice transform thus runs on half as many complex vectors.

__host__ __device__ inline uint64_t npairs_of(uint64_t nvec) { return (nvec + 1) >> 1; }

template <typename E>
__device__ __forceinline__ E cplx(double re_, double im_) {
  E z;
  z.x = (decltype(z.x))re_;
  z.y = (decltype(z.y))im_;
  return z;
}
template <>
__device__ __forceinline__ FFC cplx<FFC>(double re_, double im_) {
  return ffc_from(re_, im_);
}
__device__ __forceinline__ double cre(float2 z) { return (double)z.x; }
__device__ __forceinline__ double cim(float2 z) { return (double)z.y; }
__device__ __forceinline__ double cre(double2 z) { return z.x; }
__device__ __forceinline__ double cim(double2 z) { return z.y; }
__device__ __forceinline__ double cre(FFC z) { return ffc_re(z); }
__device__ __forceinline__ double cim(FFC z) { return ffc_im(z); }

// out[q] = in[2q] + i in[2q+1] (real vectors of T, n = 2^m each)
template <typename T, typename E>
__global__ void k_load_pairs(const T *__restrict__ in, E *__restrict__ out, uint64_t nvec, int m) {
  const uint64_t total = npairs_of(nvec) << m, mask = (1ull << m) - 1;
  for (uint64_t i = gtid(); i < total; i += gstride()) {
    const uint64_t q = i >> m, w = i & mask;
    const uint64_t vb = 2 * q + 1;
    out[i] = cplx<E>((double)in[((2 * q) << m) + w], vb < nvec ? (double)in[(vb << m) + w] : 0.0);
  }
}

// out[2q] = Re in[q] * scale, out[2q+1] = Im in[q] * scale
template <typename E, typename T>
__global__ void k_store_pairs(const E *__restrict__ in, T *__restrict__ out, uint64_t nvec, int m, double scale) {
  const uint64_t total = npairs_of(nvec) << m, mask = (1ull << m) - 1;
  for (uint64_t i = gtid(); i < total; i += gstride()) {
    const uint64_t q = i >> m, w = i & mask;
    const uint64_t vb = 2 * q + 1;
    const E z = in[i];
    out[((2 * q) << m) + w] = (T)((double)z.x * scale);
    if (vb < nvec) out[(vb << m) + w] = (T)((double)z.y * scale);
  }
}

// lambda of column 2q from Re Z, of column 2q+1 from Im Z; as k_lam_final otherwise.
template <typename E>
__global__ void k_lam_pairs(const E *__restrict__ X, double *__restrict__ lam, uint64_t nvec, int m,
                            double zmul, double dc, double eta, uint32_t *status) {
  bool bad = false, floored = false;
  const uint64_t total = npairs_of(nvec) << m, mask = (1ull << m) - 1;
  for (uint64_t i = gtid(); i < total; i += gstride()) {
    const uint64_t q = i >> m, w = i & mask;
    const E z = X[i];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const uint64_t v = 2 * q + h;
      if (v >= nvec) break;
      double val = zmul * (h ? cim(z) : cre(z)) + eta;
      if (w == 0) val += dc;
      if (eta > 0.0 && !(val >= eta)) {
        val = eta;
        floored = true;
      }
      lam[(v << m) + w] = val;
      bad |= !(val > 0.0);
    }
  }
  if (bad && status) atomicOr(status, (uint32_t)QK_STATUS_NOTPD);
  if (floored && status) atomicOr(status, (uint32_t)QK_STATUS_FLOOR);
}

// The two transforms held by pair element k and its partner kk = n - k (mod n): A_k, B_k
// (A_kk = conj A_k, B_kk = conj B_k).
template <typename E>
__device__ __forceinline__ void split_pair(E zk, E zkk, double2 &a, double2 &b) {
  const double kr = cre(zk), ki = cim(zk), kkr = cre(zkk), kki = cim(zkk);
  a = make_double2(0.5 * (kr + kkr), 0.5 * (ki - kki));
  b = make_double2(0.5 * (ki + kki), -0.5 * (kr - kkr));
}
// c + i d for complex c, d
__device__ __forceinline__ double2 join_pair(double2 c, double2 d) { return make_double2(c.x - d.y, c.y + d.x); }

// Per frequency pair (k, n - k), k = 0 .. n/2, of pair q: the vectors' transforms
// Y_v = A or B; X <- Y / lambda * fac (mode 0) or Y * lambda * fac (mode 1), re-joined
// (the products stay Hermitian, so the inverse transform returns real vectors again).
template <typename E>
__global__ void k_scale_pairs(E *__restrict__ X, const double *__restrict__ lam, uint64_t nvec, int m,
                              uint32_t nrhs, double fac, int mode) {
  const uint64_t n = 1ull << m, half = n >> 1, per = half + 1;
  const uint64_t total = npairs_of(nvec) * per;
  for (uint64_t i = gtid(); i < total; i += gstride()) {
    const uint64_t q = i / per, k = i - q * per, kk = (n - k) & (n - 1);
    E *xq = X + (q << m);
    double2 a, b;
    split_pair(xq[k], xq[kk], a, b);
    double sk[2], skk[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const uint64_t v = 2 * q + h < nvec ? 2 * q + h : 2 * q;  // an absent half scales a zero
      const double *lr = lam + ((v / nrhs) << m);
      sk[h] = mode == 0 ? fac / lr[k] : fac * lr[k];
      skk[h] = mode == 0 ? fac / lr[kk] : fac * lr[kk];
    }
    const double2 ck = make_double2(a.x * sk[0], a.y * sk[0]), dk = make_double2(b.x * sk[1], b.y * sk[1]);
    const double2 ckk = make_double2(a.x * skk[0], -a.y * skk[0]), dkk = make_double2(b.x * skk[1], -b.y * skk[1]);
    const double2 wk = join_pair(ck, dk), wkk = join_pair(ckk, dkk);
    xq[k] = cplx<E>(wk.x, wk.y);
    if (kk != k) xq[kk] = cplx<E>(wkk.x, wkk.y);
  }
}

// r = y - part(Kc) (residual of the refinement step, pair layout of Kc)
template <typename E, typename T>
__global__ void k_residual_pairs(const T *__restrict__ y, const E *__restrict__ Kc, T *__restrict__ r,
                                 uint64_t nvec, int m, double scale) {
  const uint64_t total = npairs_of(nvec) << m, mask = (1ull << m) - 1;
  for (uint64_t i = gtid(); i < total; i += gstride()) {
    const uint64_t q = i >> m, w = i & mask;
    const E z = Kc[i];
    const uint64_t ia = ((2 * q) << m) + w, vb = 2 * q + 1;
    r[ia] = (T)((double)y[ia] - (double)z.x * scale);
    if (vb < nvec) r[(vb << m) + w] = (T)((double)y[(vb << m) + w] - (double)z.y * scale);
  }
}

// MLL spectral step on pairs: per vector v the partial sums of y^T K^-1 y = sum |Y|^2/(n lam)
// and of g = (|Y|^2/(n lam) - 1) / (2 lam); G <- g_a + i g_b (real, symmetric: its inverse
// transform is u_a + i u_b); with C != nullptr also C <- Y_a/(n lam) + i Y_b/(n lam) (the
// solve).  G may alias X (each thread reads its pair elements before writing them).
template <typename E, typename EG, typename EO>
__global__ void k_mll_spectral_pairs(const E *X, const double *__restrict__ lam, uint64_t nvec, int m,
                                     uint32_t nrhs, double *__restrict__ part, EG *G, EO *__restrict__ C) {
  __shared__ double sh[32];
  const uint64_t n = 1ull << m, half = n >> 1;
  const uint64_t q = blockIdx.y;
  const E *xq = X + (q << m);
  EG *gq = G + (q << m);
  EO *cq = C ? C + (q << m) : nullptr;
  const double inv_n = 1.0 / (double)n;
  double qs[2] = {0.0, 0.0}, gs[2] = {0.0, 0.0};
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k <= half;
       k += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t kk = (n - k) & (n - 1);
    double2 y[2];
    split_pair(xq[k], xq[kk], y[0], y[1]);
    double gk[2], gkk[2], ck[2][2], ckk[2][2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const uint64_t v = 2 * q + h;
      gk[h] = gkk[h] = 0.0;
      ck[h][0] = ck[h][1] = ckk[h][0] = ckk[h][1] = 0.0;
      if (v >= nvec) continue;
      const double *lr = lam + ((v / nrhs) << m);
      // one division per eigenvalue; inv_n is a power of two, so sk = inv_n / lambda exactly
      // as k_scale_pairs rounds it (the same solve as qk_solve, bit for bit)
      const double rk = 1.0 / lr[k], rkk = 1.0 / lr[kk];
      const double sk = inv_n * rk, skk = inv_n * rkk;
      const double y2 = y[h].x * y[h].x + y[h].y * y[h].y;
      const double ak = y2 * sk;
      gk[h] = 0.5 * (ak - 1.0) * rk;
      qs[h] += ak;
      gs[h] += gk[h];
      ck[h][0] = y[h].x * sk;
      ck[h][1] = y[h].y * sk;
      if (kk != k) {
        const double akk = y2 * skk;
        gkk[h] = 0.5 * (akk - 1.0) * rkk;
        qs[h] += akk;
        gs[h] += gkk[h];
        ckk[h][0] = y[h].x * skk;
        ckk[h][1] = -y[h].y * skk;
      }
    }
    gq[k] = cplx<EG>(gk[0], gk[1]);
    if (kk != k) gq[kk] = cplx<EG>(gkk[0], gkk[1]);
    if (cq) {
      const double2 wk = join_pair(make_double2(ck[0][0], ck[0][1]), make_double2(ck[1][0], ck[1][1]));
      cq[k] = cplx<EO>(wk.x, wk.y);
      if (kk != k) {
        const double2 wkk = join_pair(make_double2(ckk[0][0], ckk[0][1]), make_double2(ckk[1][0], ckk[1][1]));
        cq[kk] = cplx<EO>(wkk.x, wkk.y);
      }
    }
  }
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const double sq = block_sum(qs[h], sh);
    const double sg = block_sum(gs[h], sh);
    const uint64_t v = 2 * q + h;
    if (threadIdx.x == 0 && v < nvec) {
      part[(v * gridDim.x + blockIdx.x) * 2 + 0] = sq;
      part[(v * gridDim.x + blockIdx.x) * 2 + 1] = sg;
    }
  }
}

template <bool FAST_LOG>
__global__ void k_logdet(const double *__restrict__ lam, int m, double *__restrict__ part) {
  __shared__ double sh[32];
  const uint64_t n = 1ull << m;
  const double *lr = lam + (uint64_t)blockIdx.y * n;
  double s = 0.0;
  for (uint64_t w = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; w < n; w += (uint64_t)gridDim.x * blockDim.x)
    s += FAST_LOG ? (double)logf((float)lr[w]) : log(lr[w]);
  const double t = block_sum(s, sh);
  if (threadIdx.x == 0) part[(uint64_t)blockIdx.y * gridDim.x + blockIdx.x] = t;
}

struct FinalArgs {
  uint32_t nvec, nrhs, d, bspec, blog, bgrad, by0;
  int m;
  double zeta;
  const double *lam, *spec_part, *log_part, *grad_part, *y0;  // y0: (nvec, by0) partial sums of y
  double *out, *grad;
};

constexpr int kFinNT = 256;

// One CTA per vector: the partial sums of the spectral step, the log-determinant, y and the
// gradient sweep added up (threads over the blocks, then over (entry, block group)).
__global__ void __launch_bounds__(kFinNT) k_mll_final(FinalArgs a) {
  __shared__ double sh[32];
  __shared__ double gsh[kFinNT];
  const uint32_t v = blockIdx.x, t = threadIdx.x;
  const uint32_t r = v / a.nrhs;
  const double n = (double)(1ull << a.m);
  double quad = 0.0, gsum = 0.0, ld = 0.0, sy = 0.0;
  for (uint32_t b = t; b < a.bspec; b += kFinNT) {
    quad += a.spec_part[((uint64_t)v * a.bspec + b) * 2 + 0];
    gsum += a.spec_part[((uint64_t)v * a.bspec + b) * 2 + 1];
  }
  for (uint32_t b = t; b < a.blog; b += kFinNT) ld += a.log_part[(uint64_t)r * a.blog + b];
  for (uint32_t b = t; b < a.by0; b += kFinNT) sy += a.y0[(uint64_t)v * a.by0 + b];
  quad = block_sum(quad, sh);
  gsum = block_sum(gsum, sh);
  ld = block_sum(ld, sh);
  sy = block_sum(sy, sh);
  __shared__ double s_sumy;
  if (t == 0) s_sumy = sy;
  __syncthreads();
  const double sumy = s_sumy;
  const double lam0 = a.lam[(uint64_t)r << a.m];
  if (t == 0) {
    double *o = a.out + (uint64_t)v * QK_MLL_NOUT;
    o[QK_MLL_QUAD] = quad;
    o[QK_MLL_LOGDET] = ld;
    o[QK_MLL_MLL] = -0.5 * quad - 0.5 * ld - 0.5 * n * 1.8378770664093454836;  // log(2 pi)
    o[QK_MLL_MEAN] = a.zeta * sumy / lam0;
    o[QK_MLL_VAR] = a.zeta * ((lam0 - a.zeta * n) / lam0);
  }
  if (!a.grad) return;
  double *g = a.grad + (uint64_t)v * (2 * a.d + 2);
  const double mfac = -a.zeta * sumy / (lam0 * lam0);
  if (t == 0) {
    g[a.d] = gsum;
    g[2 * a.d + 1] = mfac;
  }
  // entries q in [0, 2d): thread t takes entry q0 + t % nq over the blocks b = t / nq mod ng
  const uint32_t nq2 = 2 * a.d;
  const uint32_t nq = nq2 < (uint32_t)kFinNT ? nq2 : (uint32_t)kFinNT, ng = kFinNT / nq;
  const double *gp = a.grad_part + (uint64_t)v * a.bgrad * nq2;
  for (uint32_t q0 = 0; q0 < nq2; q0 += nq) {
    const uint32_t q = q0 + t % nq, grp = t / nq;
    double s = 0.0;
    if (grp < ng && q < nq2)
      for (uint32_t b = grp; b < a.bgrad; b += ng) s += gp[(uint64_t)b * nq2 + q];
    gsh[t] = s;
    __syncthreads();
    if (t < nq && q < nq2) {
      double tot = 0.0;
      for (uint32_t k = 0; k < ng; ++k) tot += gsh[k * nq + t];
      if (q < a.d) g[q] = tot;
      else g[a.d + 1 + (q - a.d)] = mfac * tot;
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------ host helpers
static unsigned grid_for(uint64_t count) {
  uint64_t b = (count + 255) / 256;
  const uint64_t cap = (uint64_t)sm_count() * 32;
  return (unsigned)(b < 1 ? 1 : (b > cap ? cap : b));
}

template <typename E, int KIND>
static int xform(E *x, int m, uint64_t nvec, double scale, cudaStream_t st) {
  return run_transform<KIND, E>(x, m, 1ull << m, nvec, scale, st);
}

template <typename E> struct IsCplx { static constexpr bool value = false; };
template <> struct IsCplx<float2> { static constexpr bool value = true; };
template <> struct IsCplx<double2> { static constexpr bool value = true; };

// Forward transform (in place): WHT for real elements (nets), FFTBR (DIT) for
// complex elements (lattices); the element type encodes the family.
template <typename E>
static int fwd(int family, E *x, int m, uint64_t nvec, cudaStream_t st) {
  (void)family;
  if constexpr (IsCplx<E>::value) return xform<E, XF_DIT>(x, m, nvec, 1.0, st);
  else return xform<E, XF_WHT>(x, m, nvec, 1.0, st);
}
template <typename E>
static int inv(int family, E *x, int m, uint64_t nvec, double scale, cudaStream_t st) {
  (void)family;
  if constexpr (IsCplx<E>::value) return xform<E, XF_DIF>(x, m, nvec, scale, st);
  else return xform<E, XF_WHT>(x, m, nvec, scale, st);
}

// count * bytes, rounded up to 256, saturating at SIZE_MAX: a workspace size that does not
// fit size_t must not wrap to a small number (callers compare it with what they hold).
static size_t sized(uint64_t count_hi, uint32_t m, size_t bytes) {
  const size_t cap = SIZE_MAX - 255;
  if (count_hi != 0 && (bytes == 0 ? false : count_hi > ((cap / bytes) >> m))) return SIZE_MAX;
  return align256(bytes * (count_hi << m));
}
static size_t add_sat(size_t a, size_t b) { return a > SIZE_MAX - b ? SIZE_MAX : a + b; }

size_t elem_bytes(int family, int dtype) {
  // QK_F32W: FP64 columns (nets) and float-float complex transforms (lattices), 8 per part
  const size_t s = (dtype == QK_F64 || dtype == QK_F32W) ? 8 : 4;
  return family == QK_SI ? 2 * s : s;
}

// Workspace sizes (bytes) per op; see qk_workspace_bytes.
size_t ws_eigs(int family, uint32_t m, uint32_t batch, int dtype) {
  return sized(batch, m, elem_bytes(family, dtype));
}
size_t ws_solve(int family, uint32_t m, uint32_t batch, uint32_t nrhs, int dtype) {
  const uint64_t nv = (uint64_t)batch * nrhs;
  // X (E) + residual path: FP64 element buffer + T buffer
  return add_sat(add_sat(sized(nv, m, elem_bytes(family, dtype)), sized(nv, m, elem_bytes(family, QK_F64))),
                 sized(nv, m, dtype == QK_F64 ? 8 : 4));
}
size_t ws_matvec(int family, uint32_t m, uint32_t batch, uint32_t nrhs, int dtype) {
  return sized((uint64_t)batch * nrhs, m, elem_bytes(family, dtype));
}
uint32_t spec_blocks(uint32_t m) {
  const uint64_t b = ((1ull << m) + 4095) / 4096;
  return (uint32_t)(b > 256 ? 256 : b);
}
// dtype QK_F32W: FP32 y and gradient sweep, FP64 transforms and spectral sums.
size_t ws_mll_si(uint32_t m, uint32_t nr, uint32_t nrhs, int dtype, uint32_t d, bool with_c);
size_t ws_mll(int family, uint32_t m, uint32_t nr, uint32_t nrhs, int dtype, uint32_t d) {
  if (family == QK_SI) return ws_mll_si(m, nr, nrhs, dtype, d, false);
  const uint64_t nv = (uint64_t)nr * nrhs;
  size_t s = sized(nv, m, elem_bytes(family, dtype == QK_F32W ? QK_F64 : dtype));
  if (family == QK_SI || dtype == QK_F32W) s = add_sat(s, sized(nv, m, dtype == QK_F64 ? 8 : 4));  // real u
  s = add_sat(s, align256(nv * spec_blocks(m) * 2 * sizeof(double)));
  s = add_sat(s, align256((uint64_t)nr * spec_blocks(m) * sizeof(double)));
  s = add_sat(s, align256(nv * spec_blocks(m) * sizeof(double)));
  s = add_sat(s, align256(nv * grad_blocks(m) * 2 * (uint64_t)d * sizeof(double)));
  return s;
}

// --------------------------------------------------------------- operations
template <typename T, typename E>
static int eigs_t(int family, uint32_t m, uint32_t batch, int form, const void *col, double zeta, double eta,
                  double *lam, void *ws, uint32_t *status, cudaStream_t st) {
  const uint64_t cnt = (uint64_t)batch << m;
  E *X = (E *)ws;
  k_load_real<T, E><<<grid_for(cnt), 256, 0, st>>>((const T *)col, X, cnt);
  int rc = check_launch("eigs load");
  if (rc) return rc;
  if ((rc = fwd<E>(family, X, m, batch, st))) return rc;
  const double zmul = form == QK_COL_P ? zeta : 1.0;
  const double dc = form == QK_COL_P ? zeta * (double)(1ull << m) : 0.0;
  k_lam_final<E><<<grid_for(cnt), 256, 0, st>>>(X, lam, cnt, (int)m, zmul, dc, eta, status);
  return check_launch("eigs finalize");
}

// ------------------------------------------------ doubling updates (Sec. 5.4)
// With 2n = 2^(m+1) points whose first n are the n-point set, the transform of the
// doubled set splits into the transforms of the two halves:
//   conj(V_{m+1}) [a; b] = [conj(V_m) a + w (.) conj(V_m) b; conj(V_m) a - w (.) conj(V_m) b] / sqrt(2)
// with w_k = 1 (Hadamard, nets) or exp(-pi i k / n) (bit-reversed Fourier, lattices).

// Imaginary and real parts of w_k times a value (nets: w = 1).
template <typename E> struct Twid {
  static __device__ __forceinline__ void apply(E v, int, uint64_t, double &r, double &i) {
    r = (double)v;
    i = 0.0;
  }
};
template <> struct Twid<float2> {
  static __device__ __forceinline__ void apply(float2 v, int m, uint64_t k, double &r, double &i) {
    double s, c;
    sincospi(-(double)k / (double)(1ull << m), &s, &c);
    r = c * v.x - s * v.y;
    i = s * v.x + c * v.y;
  }
};
template <> struct Twid<double2> {
  static __device__ __forceinline__ void apply(double2 v, int m, uint64_t k, double &r, double &i) {
    double s, c;
    sincospi(-(double)k / (double)(1ull << m), &s, &c);
    r = c * v.x - s * v.y;
    i = s * v.x + c * v.y;
  }
};

// lambda' = [lambda + w (.) t, lambda - w (.) t] with t = zmul X (+ dc at k = 0) the
// unnormalised transform of the new half of the first column; the result is real.  The
// eigenvalue floor and sign test of k_lam_final apply to lambda'.
template <typename E>
__global__ void k_lam_extend(const E *__restrict__ X, const double *__restrict__ lam_old, double *__restrict__ lam,
                             uint64_t total, int m, double zmul, double dc, double eta, uint32_t *status) {
  bool bad = false, floored = false;
  const uint64_t mask = (1ull << m) - 1;
  for (uint64_t i = gtid(); i < total; i += gstride()) {
    const uint64_t b = i >> m, k = i & mask;
    double tr, ti;
    Twid<E>::apply(X[i], m, k, tr, ti);
    tr = zmul * tr + (k == 0 ? dc : 0.0);
    const double a = lam_old[i];
    double v[2] = {a + tr, a - tr};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (eta > 0.0 && !(v[h] >= eta)) {
        v[h] = eta;
        floored = true;
      }
      bad |= !(v[h] > 0.0);
      lam[(b << (m + 1)) + ((uint64_t)h << m) + k] = v[h];
    }
  }
  if (bad && status) atomicOr(status, (uint32_t)QK_STATUS_NOTPD);
  if (floored && status) atomicOr(status, (uint32_t)QK_STATUS_FLOOR);
}

template <typename T, typename E>
static int eigs_extend_t(int family, uint32_t m, uint32_t batch, int form, const void *col_new, double zeta,
                         double eta, const double *lam_old, double *lam, void *ws, uint32_t *status, cudaStream_t st) {
  const uint64_t cnt = (uint64_t)batch << m;
  E *X = (E *)ws;
  k_load_real<T, E><<<grid_for(cnt), 256, 0, st>>>((const T *)col_new, X, cnt);
  int rc = check_launch("eigs extend load");
  if (rc) return rc;
  if ((rc = fwd<E>(family, X, m, batch, st))) return rc;
  const double zmul = form == QK_COL_P ? zeta : 1.0;
  const double dc = form == QK_COL_P ? zeta * (double)(1ull << m) : 0.0;
  k_lam_extend<E><<<grid_for(cnt), 256, 0, st>>>(X, lam_old, lam, cnt, (int)m, zmul, dc, eta, status);
  return check_launch("eigs extend");
}

int op_eigs_extend(int family, uint32_t m, uint32_t batch, int dtype, int form, const void *col_new, double zeta,
                   double eta, const double *lam_old, double *lam, void *ws, uint32_t *status, cudaStream_t st) {
  if (family == QK_DSI)
    return dtype == QK_F64 ? eigs_extend_t<double, double>(family, m, batch, form, col_new, zeta, eta, lam_old, lam, ws, status, st)
                           : eigs_extend_t<float, float>(family, m, batch, form, col_new, zeta, eta, lam_old, lam, ws, status, st);
  return dtype == QK_F64 ? eigs_extend_t<double, double2>(family, m, batch, form, col_new, zeta, eta, lam_old, lam, ws, status, st)
                         : eigs_extend_t<float, float2>(family, m, batch, form, col_new, zeta, eta, lam_old, lam, ws, status, st);
}

// out = [xt_old + w (.) xt_new, xt_old - w (.) xt_new] / sqrt(2) per vector (normalised transforms).
template <typename E>
__global__ void k_xform_extend(const E *__restrict__ xt_old, const E *__restrict__ xt_new, E *__restrict__ out,
                               uint64_t total, int m) {
  const uint64_t mask = (1ull << m) - 1;
  const double r2 = 0.70710678118654752440;
  for (uint64_t i = gtid(); i < total; i += gstride()) {
    const uint64_t b = i >> m, k = i & mask;
    double tr, ti;
    Twid<E>::apply(xt_new[i], m, k, tr, ti);
    const E a = xt_old[i];
    E lo, hi;
    if constexpr (IsCplx<E>::value) {
      using S = decltype(a.x);
      lo.x = (S)(((double)a.x + tr) * r2), lo.y = (S)(((double)a.y + ti) * r2);
      hi.x = (S)(((double)a.x - tr) * r2), hi.y = (S)(((double)a.y - ti) * r2);
    } else {
      lo = (E)(((double)a + tr) * r2);
      hi = (E)(((double)a - tr) * r2);
    }
    out[(b << (m + 1)) + k] = lo;
    out[(b << (m + 1)) + (1ull << m) + k] = hi;
  }
}

int op_transform_extend(int kind, uint32_t m, uint64_t nvec, int dtype, const void *xt_old, void *x_new, void *out,
                        cudaStream_t st) {
  int rc = op_transform(kind, m, nvec, dtype, x_new, st);  // normalised forward transform of the new half
  if (rc) return rc;
  const uint64_t cnt = nvec << m;
  if (kind == XF_WHT) {
    if (dtype == QK_F64) k_xform_extend<double><<<grid_for(cnt), 256, 0, st>>>((const double *)xt_old, (const double *)x_new, (double *)out, cnt, (int)m);
    else k_xform_extend<float><<<grid_for(cnt), 256, 0, st>>>((const float *)xt_old, (const float *)x_new, (float *)out, cnt, (int)m);
  } else {
    if (dtype == QK_F64) k_xform_extend<double2><<<grid_for(cnt), 256, 0, st>>>((const double2 *)xt_old, (const double2 *)x_new, (double2 *)out, cnt, (int)m);
    else k_xform_extend<float2><<<grid_for(cnt), 256, 0, st>>>((const float2 *)xt_old, (const float2 *)x_new, (float2 *)out, cnt, (int)m);
  }
  return check_launch("transform extend");
}

// Lattices: two columns per complex transform (their transforms are real).
template <typename T, typename E>
static int eigs_si_t(uint32_t m, uint32_t batch, int form, const void *col, double zeta, double eta, double *lam,
                     void *ws, uint32_t *status, cudaStream_t st) {
  const uint64_t np = npairs_of(batch), cnt = np << m;
  E *X = (E *)ws;
  k_load_pairs<T, E><<<grid_for(cnt), 256, 0, st>>>((const T *)col, X, batch, (int)m);
  int rc = check_launch("eigs load");
  if (rc) return rc;
  if ((rc = xform<E, XF_DIT>(X, (int)m, np, 1.0, st))) return rc;
  const double zmul = form == QK_COL_P ? zeta : 1.0;
  const double dc = form == QK_COL_P ? zeta * (double)(1ull << m) : 0.0;
  k_lam_pairs<E><<<grid_for(cnt), 256, 0, st>>>(X, lam, batch, (int)m, zmul, dc, eta, status);
  return check_launch("eigs finalize");
}

int op_eigs(int family, uint32_t m, uint32_t batch, int dtype, int form, const void *col, double zeta, double eta,
            double *lam, void *ws, uint32_t *status, cudaStream_t st) {
  if (batch == 0) return QK_OK;
  if (family == QK_DSI) {
    if (dtype == QK_F32W) dtype = QK_F64;  // FP64 column, FP64 transform
    return dtype == QK_F64 ? eigs_t<double, double>(family, m, batch, form, col, zeta, eta, lam, ws, status, st)
                           : eigs_t<float, float>(family, m, batch, form, col, zeta, eta, lam, ws, status, st);
  }
  // QK_F32W: the float-float column (stored FP64) through float-float transforms
  if (dtype == QK_F32W) return eigs_si_t<double, FFC>(m, batch, form, col, zeta, eta, lam, ws, status, st);
  return dtype == QK_F64 ? eigs_si_t<double, double2>(m, batch, form, col, zeta, eta, lam, ws, status, st)
                         : eigs_si_t<float, float2>(m, batch, form, col, zeta, eta, lam, ws, status, st);
}

// c = K^-1 y (mode 0) or K y (mode 1) in precision of E; X is scratch of nvec * n E.
template <typename T, typename E>
static int apply_t(int family, uint32_t m, uint32_t nvec, uint32_t nrhs, const double *lam, const T *y, T *c,
                   E *X, int mode, cudaStream_t st) {
  const uint64_t cnt = (uint64_t)nvec << m;
  const double n = (double)(1ull << m);
  k_load_real<T, E><<<grid_for(cnt), 256, 0, st>>>(y, X, cnt);
  int rc = check_launch("solve load");
  if (rc) return rc;
  if ((rc = fwd<E>(family, X, m, nvec, st))) return rc;
  k_scale_lam<E><<<grid_for(cnt), 256, 0, st>>>(X, lam, cnt, (int)m, nrhs, 1.0 / n, mode);
  if ((rc = check_launch("solve scale"))) return rc;
  if ((rc = inv<E>(family, X, m, nvec, 1.0, st))) return rc;
  k_store_real<E, T><<<grid_for(cnt), 256, 0, st>>>(X, c, cnt, 1.0);
  return check_launch("solve store");
}

template <typename T, typename E, typename E64>
static int solve_t(int family, uint32_t m, uint32_t batch, uint32_t nrhs, const double *lam, const T *y, T *c,
                   int refine, void *ws, cudaStream_t st) {
  const uint32_t nvec = batch * nrhs;
  const uint64_t cnt = (uint64_t)nvec << m;
  unsigned char *p = (unsigned char *)ws;
  E *X = (E *)p;
  p += align256(sizeof(E) * cnt);
  E64 *X64 = (E64 *)p;
  p += align256(sizeof(E64) * cnt);
  T *tmp = (T *)p;
  int rc = apply_t<T, E>(family, m, nvec, nrhs, lam, y, c, X, 0, st);
  if (rc) return rc;
  const double n = (double)(1ull << m);
  for (int it = 0; it < refine; ++it) {
    // residual r = y - K c with FP64 transforms
    k_load_real<T, E64><<<grid_for(cnt), 256, 0, st>>>(c, X64, cnt);
    if ((rc = check_launch("refine load"))) return rc;
    if ((rc = fwd<E64>(family, X64, m, nvec, st))) return rc;
    k_scale_lam<E64><<<grid_for(cnt), 256, 0, st>>>(X64, lam, cnt, (int)m, nrhs, 1.0 / n, 1);
    if ((rc = check_launch("refine scale"))) return rc;
    if ((rc = inv<E64>(family, X64, m, nvec, 1.0, st))) return rc;
    k_residual<E64, T><<<grid_for(cnt), 256, 0, st>>>(y, X64, tmp, cnt, 1.0);
    if ((rc = check_launch("refine residual"))) return rc;
    if ((rc = apply_t<T, E>(family, m, nvec, nrhs, lam, tmp, tmp, X, 0, st))) return rc;
    k_add<T><<<grid_for(cnt), 256, 0, st>>>(c, tmp, cnt);
    if ((rc = check_launch("refine add"))) return rc;
  }
  return QK_OK;
}

// Lattices: c = K^-1 y (mode 0) or K y (mode 1) on pairs of vectors; X: (nvec + 1) / 2
// complex vectors of E.
template <typename T, typename E>
static int apply_si_t(uint32_t m, uint32_t nvec, uint32_t nrhs, const double *lam, const T *y, T *c, E *X, int mode,
                      cudaStream_t st) {
  const uint64_t np = npairs_of(nvec), cnt = np << m;
  const double n = (double)(1ull << m);
  k_load_pairs<T, E><<<grid_for(cnt), 256, 0, st>>>(y, X, nvec, (int)m);
  int rc = check_launch("solve load");
  if (rc) return rc;
  if ((rc = xform<E, XF_DIT>(X, (int)m, np, 1.0, st))) return rc;
  k_scale_pairs<E><<<grid_for(np * ((1ull << m) / 2 + 1)), 256, 0, st>>>(X, lam, nvec, (int)m, nrhs, 1.0 / n, mode);
  if ((rc = check_launch("solve scale"))) return rc;
  if ((rc = xform<E, XF_DIF>(X, (int)m, np, 1.0, st))) return rc;
  k_store_pairs<E, T><<<grid_for(cnt), 256, 0, st>>>(X, c, nvec, (int)m, 1.0);
  return check_launch("solve store");
}

template <typename T, typename E, typename E64>
static int solve_si_t(uint32_t m, uint32_t batch, uint32_t nrhs, const double *lam, const T *y, T *c, int refine,
                      void *ws, cudaStream_t st) {
  const uint32_t nvec = batch * nrhs;
  const uint64_t np = npairs_of(nvec), cnt = (uint64_t)nvec << m;
  unsigned char *p = (unsigned char *)ws;
  E *X = (E *)p;
  p += align256(sizeof(E) * (np << m));
  E64 *X64 = (E64 *)p;
  p += align256(sizeof(E64) * (np << m));
  T *tmp = (T *)p;
  int rc = apply_si_t<T, E>(m, nvec, nrhs, lam, y, c, X, 0, st);
  if (rc) return rc;
  const double n = (double)(1ull << m);
  for (int it = 0; it < refine; ++it) {
    // residual r = y - K c with FP64 transforms, then c += K^-1 r
    k_load_pairs<T, E64><<<grid_for(np << m), 256, 0, st>>>(c, X64, nvec, (int)m);
    if ((rc = check_launch("refine load"))) return rc;
    if ((rc = xform<E64, XF_DIT>(X64, (int)m, np, 1.0, st))) return rc;
    k_scale_pairs<E64><<<grid_for(np * ((1ull << m) / 2 + 1)), 256, 0, st>>>(X64, lam, nvec, (int)m, nrhs, 1.0 / n, 1);
    if ((rc = check_launch("refine scale"))) return rc;
    if ((rc = xform<E64, XF_DIF>(X64, (int)m, np, 1.0, st))) return rc;
    k_residual_pairs<E64, T><<<grid_for(np << m), 256, 0, st>>>(y, X64, tmp, nvec, (int)m, 1.0);
    if ((rc = check_launch("refine residual"))) return rc;
    if ((rc = apply_si_t<T, E>(m, nvec, nrhs, lam, tmp, tmp, X, 0, st))) return rc;
    k_add<T><<<grid_for(cnt), 256, 0, st>>>(c, tmp, cnt);
    if ((rc = check_launch("refine add"))) return rc;
  }
  return QK_OK;
}

int op_solve(int family, uint32_t m, uint32_t batch, uint32_t nrhs, int dtype, const double *lam, const void *y,
             void *c, int refine, void *ws, cudaStream_t st) {
  if ((uint64_t)batch * nrhs == 0) return QK_OK;
  if (family == QK_SI) {
    if (dtype == QK_F64)
      return solve_si_t<double, double2, double2>(m, batch, nrhs, lam, (const double *)y, (double *)c, refine, ws, st);
    return solve_si_t<float, float2, double2>(m, batch, nrhs, lam, (const float *)y, (float *)c, refine, ws, st);
  }
  if (family == QK_DSI) {
    if (dtype == QK_F64)
      return solve_t<double, double, double>(family, m, batch, nrhs, lam, (const double *)y, (double *)c, refine, ws, st);
    return solve_t<float, float, double>(family, m, batch, nrhs, lam, (const float *)y, (float *)c, refine, ws, st);
  }
  if (dtype == QK_F64)
    return solve_t<double, double2, double2>(family, m, batch, nrhs, lam, (const double *)y, (double *)c, refine, ws, st);
  return solve_t<float, float2, double2>(family, m, batch, nrhs, lam, (const float *)y, (float *)c, refine, ws, st);
}

// X <- the unnormalised forward transform (H, or the DFT of the data in linear order) of
// nvec real vectors `in` of dtype; X holds elements of the transform type (real for nets,
// complex for lattices) in the same precision.
int op_forward_real(int family, uint32_t m, uint64_t nvec, int dtype, const void *in, void *X, cudaStream_t st) {
  const uint64_t cnt = nvec << m;
  int rc;
  if (family == QK_DSI) {
    if (dtype == QK_F64) k_load_real<double, double><<<grid_for(cnt), 256, 0, st>>>((const double *)in, (double *)X, cnt);
    else k_load_real<float, float><<<grid_for(cnt), 256, 0, st>>>((const float *)in, (float *)X, cnt);
    if ((rc = check_launch("forward load"))) return rc;
    return dtype == QK_F64 ? fwd<double>(family, (double *)X, (int)m, nvec, st) : fwd<float>(family, (float *)X, (int)m, nvec, st);
  }
  if (dtype == QK_F64) k_load_real<double, double2><<<grid_for(cnt), 256, 0, st>>>((const double *)in, (double2 *)X, cnt);
  else k_load_real<float, float2><<<grid_for(cnt), 256, 0, st>>>((const float *)in, (float2 *)X, cnt);
  if ((rc = check_launch("forward load"))) return rc;
  return dtype == QK_F64 ? fwd<double2>(family, (double2 *)X, (int)m, nvec, st)
                         : fwd<float2>(family, (float2 *)X, (int)m, nvec, st);
}

int op_matvec(int family, uint32_t m, uint32_t batch, uint32_t nrhs, int dtype, const double *lam, const void *y,
              void *u, void *ws, cudaStream_t st) {
  const uint32_t nvec = batch * nrhs;
  if (nvec == 0) return QK_OK;
  if (family == QK_SI)
    return dtype == QK_F64 ? apply_si_t<double, double2>(m, nvec, nrhs, lam, (const double *)y, (double *)u, (double2 *)ws, 1, st)
                           : apply_si_t<float, float2>(m, nvec, nrhs, lam, (const float *)y, (float *)u, (float2 *)ws, 1, st);
  if (family == QK_DSI)
    return dtype == QK_F64 ? apply_t<double, double>(family, m, nvec, nrhs, lam, (const double *)y, (double *)u, (double *)ws, 1, st)
                           : apply_t<float, float>(family, m, nvec, nrhs, lam, (const float *)y, (float *)u, (float *)ws, 1, st);
  return dtype == QK_F64 ? apply_t<double, double2>(family, m, nvec, nrhs, lam, (const double *)y, (double *)u, (double2 *)ws, 1, st)
                         : apply_t<float, float2>(family, m, nvec, nrhs, lam, (const float *)y, (float *)u, (float2 *)ws, 1, st);
}

template <typename T, typename E>
static int mll_t(const ColJob &job, uint32_t nrhs, const double *lam, const T *y, double *out, double *grad,
                 void *ws, cudaStream_t st, int dtype) {
  const uint32_t m = job.m;
  const uint32_t nvec = job.nr * nrhs;
  const uint64_t cnt = (uint64_t)nvec << m;
  unsigned char *p = (unsigned char *)ws;
  E *X = (E *)p;
  p += align256(sizeof(E) * cnt);
  // the transform output is u itself when E == T (nets in the data precision); otherwise
  // (lattices: complex; FP64 transforms of FP32 data) its real part is stored as T
  constexpr bool SEP_U = !std::is_same<E, T>::value;
  T *u = (T *)X;
  if (SEP_U) {
    u = (T *)p;
    p += align256(sizeof(T) * cnt);
  }
  const uint32_t bs = spec_blocks(m);
  double *spec_part = (double *)p;
  p += align256((uint64_t)nvec * bs * 2 * sizeof(double));
  double *log_part = (double *)p;
  p += align256((uint64_t)job.nr * bs * sizeof(double));
  double *y0 = (double *)p;
  p += align256((uint64_t)nvec * bs * sizeof(double));
  double *grad_part = (double *)p;

  k_load_real<T, E><<<grid_for(cnt), 256, 0, st>>>(y, X, cnt);
  int rc = check_launch("mll load");
  if (rc) return rc;
  k_sum_rows<T><<<dim3(spec_blocks(m), nvec), 256, 0, st>>>(y, (int)m, y0);
  if ((rc = check_launch("mll sum y"))) return rc;
  if ((rc = fwd<E>(job.family, X, (int)m, nvec, st))) return rc;
  k_mll_spectral<E><<<dim3(bs, nvec), kRedNT, 0, st>>>(X, lam, (int)m, nrhs, spec_part, y0);
  if ((rc = check_launch("mll spectral"))) return rc;
  if (dtype == QK_F64)
    k_logdet<false><<<dim3(bs, job.nr), kRedNT, 0, st>>>(lam, (int)m, log_part);
  else  // FP32 logs of FP32-rounded eigenvalues: each log is off by ~eps32 (absolute)
    k_logdet<true><<<dim3(bs, job.nr), kRedNT, 0, st>>>(lam, (int)m, log_part);
  if ((rc = check_launch("mll logdet"))) return rc;
  if (grad) {
    // u = H g (nets) or the DFT of g read back in natural order (lattices); real.
    if ((rc = inv<E>(job.family, X, (int)m, nvec, 1.0, st))) return rc;
    if (SEP_U) {
      k_store_real<E, T><<<grid_for(cnt), 256, 0, st>>>(X, u, cnt, 1.0);
      if ((rc = check_launch("mll u"))) return rc;
    }
    if ((rc = launch_grad_partials(job, nrhs, sizeof(T) == 8 ? QK_F64 : QK_F32, u, grad_part, st))) return rc;
  }
  FinalArgs fa;
  fa.nvec = nvec;
  fa.nrhs = nrhs;
  fa.d = job.d;
  fa.bspec = bs;
  fa.blog = bs;
  fa.bgrad = grad_blocks(m);
  fa.m = (int)m;
  fa.zeta = job.zeta;
  fa.lam = lam;
  fa.spec_part = spec_part;
  fa.log_part = log_part;
  fa.grad_part = grad_part;
  fa.y0 = y0;
  fa.by0 = bs;
  fa.out = out;
  fa.grad = grad;
  k_mll_final<<<nvec, kFinNT, 0, st>>>(fa);
  return check_launch("mll final");
}

// Lattices: MLL, gradient and (with c) the solve on pairs of vectors.  Forward transforms in
// E, the spectral step in FP64, the inverse transforms of the gradient's g pairs (G; in
// place over the forward data when EG == E) and of the solve's pairs (C) in the data
// precision.  With the float-float column (QK_F32W) the forward transforms are FP64 and the
// inverses FP32: the gradient's accuracy is then set by the FP32 sweep over the points (its
// terms cancel near the nugget floor), which an FP64 inverse of g does not change
// (measured: the same 4e-4 .. 6e-4 relative error on dMLL/dc at n = 2^12, eta = 1e-6).
template <typename E, typename EG, typename EO>
static size_t ws_mll_si_t(uint32_t m, uint32_t nr, uint32_t nrhs, uint32_t d, bool with_c) {
  const uint64_t nv = (uint64_t)nr * nrhs, np = npairs_of(nv);
  size_t s = sized(np, m, sizeof(E));
  if (!std::is_same<E, EG>::value) s = add_sat(s, sized(np, m, sizeof(EG)));
  if (with_c) s = add_sat(s, sized(np, m, sizeof(EO)));
  s = add_sat(s, align256(nv * spec_blocks(m) * 2 * sizeof(double)));
  s = add_sat(s, align256((uint64_t)nr * spec_blocks(m) * sizeof(double)));
  s = add_sat(s, align256(nv * spec_blocks(m) * sizeof(double)));
  s = add_sat(s, align256(nv * grad_blocks(m) * 2 * (uint64_t)d * sizeof(double)));
  return s;
}

size_t ws_mll_si(uint32_t m, uint32_t nr, uint32_t nrhs, int dtype, uint32_t d, bool with_c) {
  if (dtype == QK_F64) return ws_mll_si_t<double2, double2, double2>(m, nr, nrhs, d, with_c);
  if (dtype == QK_F32W) return ws_mll_si_t<FFC, float2, float2>(m, nr, nrhs, d, with_c);
  return ws_mll_si_t<float2, float2, float2>(m, nr, nrhs, d, with_c);
}

template <typename T, typename E, typename EG, typename EO>
static int mll_si_t(const ColJob &job, uint32_t nrhs, const double *lam, const T *y, double *out, double *grad,
                    T *c, void *ws, cudaStream_t st, bool fast_log, const double *pcol) {
  static_assert(sizeof(EO) == 2 * sizeof(T) && sizeof(EG) == 2 * sizeof(T), "inverse transforms in the data precision");
  const uint32_t m = job.m;
  const uint64_t nvec = (uint64_t)job.nr * nrhs, np = npairs_of(nvec);
  if (nvec == 0) return QK_OK;
  unsigned char *p = (unsigned char *)ws;
  E *X = (E *)p;
  p += align256(sizeof(E) * (np << m));
  EG *G = reinterpret_cast<EG *>(X);
  if (!std::is_same<E, EG>::value) {
    G = (EG *)p;
    p += align256(sizeof(EG) * (np << m));
  }
  EO *C = nullptr;
  if (c) {
    C = (EO *)p;
    p += align256(sizeof(EO) * (np << m));
  }
  const uint32_t bs = spec_blocks(m);
  double *spec_part = (double *)p;
  p += align256(nvec * bs * 2 * sizeof(double));
  double *log_part = (double *)p;
  p += align256((uint64_t)job.nr * bs * sizeof(double));
  double *y0 = (double *)p;
  p += align256(nvec * bs * sizeof(double));
  double *grad_part = (double *)p;

  k_load_pairs<T, E><<<grid_for(np << m), 256, 0, st>>>(y, X, nvec, (int)m);
  int rc = check_launch("mll load");
  if (rc) return rc;
  k_sum_rows<T><<<dim3(spec_blocks(m), (unsigned)nvec), 256, 0, st>>>(y, (int)m, y0);
  if ((rc = check_launch("mll sum y"))) return rc;
  if ((rc = xform<E, XF_DIT>(X, (int)m, np, 1.0, st))) return rc;
  k_mll_spectral_pairs<E, EG, EO><<<dim3(bs, (unsigned)np), kRedNT, 0, st>>>(X, lam, nvec, (int)m, nrhs, spec_part,
                                                                             G, C);
  if ((rc = check_launch("mll spectral"))) return rc;
  if (fast_log)  // FP32 logs of the eigenvalues: each log off by ~eps32 (absolute)
    k_logdet<true><<<dim3(bs, job.nr), kRedNT, 0, st>>>(lam, (int)m, log_part);
  else
    k_logdet<false><<<dim3(bs, job.nr), kRedNT, 0, st>>>(lam, (int)m, log_part);
  if ((rc = check_launch("mll logdet"))) return rc;
  // G -> u_a + i u_b (real vectors of the gradient), C -> c_a + i c_b
  if (grad) {
    if ((rc = xform<EG, XF_DIF>(G, (int)m, np, 1.0, st))) return rc;
    if ((rc = launch_grad_partials(job, nrhs, sizeof(T) == 8 ? QK_F64 : QK_F32, G, grad_part, st, true, pcol)))
      return rc;
  }
  if (c && (rc = xform<EO, XF_DIF>(C, (int)m, np, 1.0, st))) return rc;
  if (c) {
    k_store_pairs<EO, T><<<grid_for(np << m), 256, 0, st>>>(C, c, nvec, (int)m, 1.0);
    if ((rc = check_launch("mll solve store"))) return rc;
  }
  FinalArgs fa;
  fa.nvec = (uint32_t)nvec;
  fa.nrhs = nrhs;
  fa.d = job.d;
  fa.bspec = bs;
  fa.blog = bs;
  fa.bgrad = grad_blocks(m);
  fa.m = (int)m;
  fa.zeta = job.zeta;
  fa.lam = lam;
  fa.spec_part = spec_part;
  fa.log_part = log_part;
  fa.grad_part = grad_part;
  fa.y0 = y0;
  fa.by0 = bs;
  fa.out = out;
  fa.grad = grad;
  k_mll_final<<<(unsigned)nvec, kFinNT, 0, st>>>(fa);
  return check_launch("mll final");
}

// MLL, gradient and solve of lattice tasks in one pass (dtype QK_F64, QK_F32W or QK_F32):
// c may be null (no solve), grad may be null.
int op_mll_solve_si(const ColJob &job, uint32_t nrhs, int dtype, const double *lam, const void *y, double *out,
                    double *grad, void *c, void *ws, cudaStream_t st, const double *pcol) {
  if (job.family != QK_SI) return fail(QK_EINVAL, "op_mll_solve_si: lattice tasks only");
  if (dtype == QK_F64)
    return mll_si_t<double, double2, double2, double2>(job, nrhs, lam, (const double *)y, out, grad, (double *)c, ws,
                                                       st, false, pcol);
  if (dtype == QK_F32W)
    return mll_si_t<float, FFC, float2, float2>(job, nrhs, lam, (const float *)y, out, grad, (float *)c, ws, st,
                                                true, pcol);
  return mll_si_t<float, float2, float2, float2>(job, nrhs, lam, (const float *)y, out, grad, (float *)c, ws, st,
                                                 true, pcol);
}

int op_mll(const ColJob &job, uint32_t nrhs, int dtype, const double *lam, const void *y, double *out, double *grad,
           void *ws, cudaStream_t st) {
  if (job.family == QK_SI) return op_mll_solve_si(job, nrhs, dtype, lam, y, out, grad, nullptr, ws, st);
  if (dtype == QK_F32W) return mll_t<float, double>(job, nrhs, lam, (const float *)y, out, grad, ws, st, dtype);
  return dtype == QK_F64 ? mll_t<double, double>(job, nrhs, lam, (const double *)y, out, grad, ws, st, dtype)
                         : mll_t<float, float>(job, nrhs, lam, (const float *)y, out, grad, ws, st, dtype);
}

// ------------------------------------------------ persistent FP32 FFTBR / IFFTBR
bool persist_fft_supported(uint32_t m, int dtype) { return dtype == QK_F32 && m >= 16 && m <= 20; }

template <int KIND, int KH>
static int persist_fft_t(float2 *x, uint32_t m, uint64_t nvec, double scale, uint32_t *ctr, uint32_t *status,
                         uint32_t lag, uint32_t spin_limit, cudaStream_t st) {
  const size_t smem = pass_smem<float2>();
  static int occ = -1;  // per instantiation; the same on every GB300
  if (occ < 0) {
    smem_optin<k_fft_persist<KIND, KH>>(smem);
    int o = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_fft_persist<KIND, KH>, 256, smem) != cudaSuccess || o < 1)
      return fail(QK_ECUDA, "persistent FFT: occupancy query failed");
    occ = o;
  }
  const uint32_t T = 1u << (m - 12);
  const uint64_t items = (2ull * nvec) * T;
  if (items >= (1ull << 31)) return fail(QK_EINVAL, "persistent FFT: %llu work items exceed 2^31",
                                         (unsigned long long)items);
  const uint32_t grid = (uint32_t)sm_count() * (uint32_t)occ;
  if (lag == 0) {
    // enough tickets between a vector's last first-pass tile and its first second-pass
    // tile that the former has finished (lag T >= resident CTAs), one vector of slack, at
    // most 24 MB of first-pass output waiting in L2 (measured, 64 x 2^20: lag 2-3 0.380 ms,
    // 5 0.414 ms, 8 0.424 ms)
    uint64_t lg = (grid + T - 1) / T + 1;
    const uint64_t cap = (24ull << 20) / (8ull << m);
    if (lg > cap) lg = cap;
    lag = (uint32_t)(lg < 1 ? 1 : lg);
  }
  if (lag > nvec) lag = (uint32_t)nvec;
  WhtSched sc{(uint32_t)nvec, m - 12, lag};
  cudaError_t e = cudaMemsetAsync(ctr, 0, sizeof(uint32_t) * (1 + nvec), st);
  if (e != cudaSuccess) return cuda_fail(e, "persistent FFT: counter reset");
  k_fft_persist<KIND, KH><<<grid, 256, smem, st>>>(x, scale, sc, ctr, status, spin_limit);
  return check_launch("persistent FFT");
}

template <int KIND>
static int persist_fft_kind(float2 *x, uint32_t m, uint64_t nvec, double scale, uint32_t *ctr, uint32_t *status,
                            uint32_t lag, uint32_t spin_limit, cudaStream_t st) {
  switch (m) {
    case 16: return persist_fft_t<KIND, 4>(x, m, nvec, scale, ctr, status, lag, spin_limit, st);
    case 17: return persist_fft_t<KIND, 5>(x, m, nvec, scale, ctr, status, lag, spin_limit, st);
    case 18: return persist_fft_t<KIND, 6>(x, m, nvec, scale, ctr, status, lag, spin_limit, st);
    case 19: return persist_fft_t<KIND, 7>(x, m, nvec, scale, ctr, status, lag, spin_limit, st);
    case 20: return persist_fft_t<KIND, 8>(x, m, nvec, scale, ctr, status, lag, spin_limit, st);
    default: return fail(QK_EINVAL, "persistent FFT: m = %u outside 16..20", m);
  }
}

int persist_fft(int kind, void *x, uint32_t m, uint64_t nvec, double scale, uint32_t *ctr, uint32_t *status,
                uint32_t lag, cudaStream_t st, uint32_t spin_limit) {
  if (nvec == 0) return QK_OK;
  if (kind == XF_DIT) return persist_fft_kind<XF_DIT>((float2 *)x, m, nvec, scale, ctr, status, lag, spin_limit, st);
  return persist_fft_kind<XF_DIF>((float2 *)x, m, nvec, scale, ctr, status, lag, spin_limit, st);
}

int op_transform(int kind, uint32_t m, uint64_t nvec, int dtype, void *x, cudaStream_t st) {
  const double scale = 1.0 / std::sqrt((double)(1ull << m));
  if (kind == XF_WHT && tiled_wht_supported(m, dtype)) return tiled_wht(x, m, nvec, dtype, scale, st);
  if (kind == XF_WHT)
    return dtype == QK_F64 ? xform<double, XF_WHT>((double *)x, (int)m, nvec, scale, st)
                           : xform<float, XF_WHT>((float *)x, (int)m, nvec, scale, st);
  if (kind == XF_DIT)
    return dtype == QK_F64 ? xform<double2, XF_DIT>((double2 *)x, (int)m, nvec, scale, st)
                           : xform<float2, XF_DIT>((float2 *)x, (int)m, nvec, scale, st);
  return dtype == QK_F64 ? xform<double2, XF_DIF>((double2 *)x, (int)m, nvec, scale, st)
                         : xform<float2, XF_DIF>((float2 *)x, (int)m, nvec, scale, st);
}

}  // namespace qk
