// Randomized QMC integration on top of the point sets (arXiv 2502.14256):
//   * the six test integrands of the numerical experiments (Sec. 6) evaluated at the points
//     of R randomizations, optionally through the baker transform x -> 1 - 2|x - 1/2|
//     (Sec. 4.2), without materialising the points;
//   * the RQMC estimate over R randomizations with its Student-t interval (Sec. 3.1);
//   * the squared worst-case error (generalized kernel discrepancy) of a cubature rule
//     (Sec. 3.2): closed forms for equal weights 1/n and the optimal weights K^-1 kappa,
//     and general weights through the spectrum (w^T K w = sum lambda |w~|^2, Sec. 5.4).
#include <cfloat>
#include <cmath>

#include "qk_column.cuh"
#include "qk_common.cuh"
#include "qk_internal.h"

namespace qk {

constexpr int kIntNT = 256, kIntRL = 8, kIntNP = kIntNT * kIntRL;  // points per CTA tile

template <typename T>
__device__ __forceinline__ T t_exp(T v) {
  if constexpr (sizeof(T) == 8) return exp(v);
  else return expf(v);
}
template <typename T>
__device__ __forceinline__ T t_cos(T v) {
  if constexpr (sizeof(T) == 8) return cos(v);
  else return cosf(v);
}
template <typename T>
__device__ __forceinline__ T t_pow(T a, T b) {
  if constexpr (sizeof(T) == 8) return pow(a, b);
  else return powf(a, b);
}

// Coordinate x = X 2^-32 of a word, or its baker transform 1 - 2|x - 1/2| = X' 2^-32 with
// X' = 2X (X < 2^31) or 2^33 - 2X (exact as a 33-bit integer), converted once to T.
template <typename T>
__device__ __forceinline__ T coord(uint32_t X, bool baker) {
  if (!baker) {
    if constexpr (sizeof(T) == 8) return (double)X * 0x1p-32;
    else return __uint2float_rn(X) * 0x1p-32f;
  }
  const uint64_t Xb = X < 0x80000000u ? 2ull * X : (1ull << 33) - 2ull * X;
  if constexpr (sizeof(T) == 8) return (double)Xb * 0x1p-32;
  else return __ull2float_rn(Xb) * 0x1p-32f;
}

// Running state of one point over its dimensions: the first two coordinates, a product
// (G-function) and a linear form (Genz).
template <typename T>
struct FState {
  T x1, x2, prod, lin;
};

template <typename T>
__device__ __forceinline__ void fstate_add(FState<T> &s, int f, uint32_t j, T x, const double *cf) {
  if (j == 0) s.x1 = x;
  if (j == 1) s.x2 = x;
  if (f == QK_F_GFUN) {
    const T a = (T)cf[j];
    s.prod *= (fabs(T(4) * x - T(2)) - a) / (T(1) + a);
  } else if (f == QK_F_GENZ_OSC || f == QK_F_GENZ_CP) {
    s.lin = fmadd((T)cf[j], x, s.lin);
  }
}

template <typename T>
__device__ __forceinline__ T fstate_value(const FState<T> &s, int f, uint32_t d) {
  switch (f) {
    case QK_F_SIMPLE1: return s.x1 * t_exp(s.x1) - T(1);
    case QK_F_SIMPLE2: return s.x2 * t_exp(s.x1 * s.x2) / T(0.71828182845904523536) - T(1);  // e - 2
    case QK_F_OAKLEY: {
      const T t1 = (s.x1 - T(0.5)) / T(50), t2 = (s.x2 - T(0.5)) / T(50);
      return T(5) + t1 + t2 + T(2) * t_cos(t1) + T(2) * t_cos(t2);
    }
    case QK_F_GFUN: return s.prod;
    case QK_F_GENZ_OSC: return t_cos(s.lin);  // cos(-s) = cos(s)
    default: return t_pow(T(1) + s.lin, -(T)(d + 1));
  }
}

// y[r][i] = f(x_i) for the points at positions i0 + [0, n) of randomization r0 + blockIdx.y.
// A CTA covers kIntNP consecutive positions aligned to kIntNP; a thread makes kIntRL
// consecutive points dimension by dimension (nets: seeded from the XOR tables of the tile,
// lane and warp bits, then one XOR per point with a column known at compile time, as in
// point generation; lattices: brev(i) g + D).
template <typename T, bool NET>
__global__ void __launch_bounds__(kIntNT) k_integrand(uint32_t d, int order, const uint32_t *__restrict__ Ct,
                                                      const uint32_t *__restrict__ g, const uint32_t *__restrict__ D,
                                                      uint32_t r0, uint64_t i0, uint64_t n, int f, int baker,
                                                      T *__restrict__ y) {
  extern __shared__ __align__(16) unsigned char ism[];
  double *cf = reinterpret_cast<double *>(ism);                  // (d) coefficients
  uint32_t *ztile = reinterpret_cast<uint32_t *>(cf + d);        // (d) tile words, shift included
  uint32_t *zlane = ztile + d;                                   // (32 d) nets
  uint32_t *zwarp = zlane + 32 * d;                              // (8 d) nets
  uint32_t *steps = zwarp + (kIntNT / 32) * d;                   // (3 d) nets: step columns
  const uint32_t rl = blockIdx.y, r = r0 + rl;
  const uint64_t base = ((i0 / kIntNP) + blockIdx.x) * kIntNP;  // < 2^32
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  // coefficients (FP64): Genz oscillatory / corner peak (Sec. 6), G-function a_j = (j - 2)/2
  if (t == 0) {
    if (f == QK_F_GENZ_OSC || f == QK_F_GENZ_CP) {
      double sum = 0.0;
      for (uint32_t j = 0; j < d; ++j) {
        const double ct = f == QK_F_GENZ_OSC ? exp((double)(j + 1) * log(1e-8) / (double)d)
                                             : 1.0 / ((double)(j + 1) * (double)(j + 1));
        cf[j] = ct;
        sum += ct;
      }
      const double scale = (f == QK_F_GENZ_OSC ? 4.5 : 0.25) / sum;
      for (uint32_t j = 0; j < d; ++j) cf[j] *= scale;
    } else {
      for (uint32_t j = 0; j < d; ++j) cf[j] = ((double)(j + 1) - 2.0) / 2.0;
    }
  }
  if constexpr (NET) {
    const uint32_t *Cr = Ct + (size_t)r * d * 32;
    for (uint32_t q = t; q < 32 * d; q += kIntNT) {
      const uint32_t j = q >> 5, ln = q & 31;
      zlane[q] = xor_columns(Cr + j * 32, order_map(order, ln * kIntRL));
    }
    for (uint32_t q = t; q < (kIntNT / 32) * d; q += kIntNT) {
      const uint32_t w = q / d, j = q - w * d;
      zwarp[w * d + j] = xor_columns(Cr + j * 32, order_map(order, (w * 32) * kIntRL));
    }
    for (uint32_t j = t; j < d; j += kIntNT) {
      ztile[j] = xor_columns(Cr + j * 32, order_map(order, (uint32_t)base)) ^ (D ? D[(size_t)r * d + j] : 0u);
      const uint32_t c0 = Cr[j * 32], c1 = Cr[j * 32 + 1], c2 = Cr[j * 32 + 2];
      steps[3 * j] = c0;
      steps[3 * j + 1] = order == QK_GRAY ? c1 : (c0 ^ c1);
      steps[3 * j + 2] = order == QK_GRAY ? c2 : (c0 ^ c1 ^ c2);
    }
  } else {
    for (uint32_t j = t; j < d; j += kIntNT) ztile[j] = D ? D[(size_t)r * d + j] : 0u;
  }
  __syncthreads();
  FState<T> st[kIntRL];
#pragma unroll
  for (int k = 0; k < kIntRL; ++k) st[k] = FState<T>{T(0), T(0), T(1), T(0)};
  const uint32_t i_first = (uint32_t)base + (uint32_t)t * kIntRL;
  for (uint32_t j = 0; j < d; ++j) {
    uint32_t w[kIntRL];
    if constexpr (NET) {
      const uint32_t s0 = steps[3 * j], s1 = steps[3 * j + 1], s2 = steps[3 * j + 2];
      uint32_t x = ztile[j] ^ zlane[j * 32 + lane] ^ zwarp[warp * d + j];
      w[0] = x;
      x ^= s0, w[1] = x;
      x ^= s1, w[2] = x;
      x ^= s0, w[3] = x;
      x ^= s2, w[4] = x;
      x ^= s0, w[5] = x;
      x ^= s1, w[6] = x;
      x ^= s0, w[7] = x;
    } else {
      const uint32_t gj = g[j], dj = ztile[j];
#pragma unroll
      for (int k = 0; k < kIntRL; ++k) w[k] = __brev(i_first + k) * gj + dj;
    }
#pragma unroll
    for (int k = 0; k < kIntRL; ++k) fstate_add(st[k], f, j, coord<T>(w[k], baker != 0), cf);
  }
  T *yr = y + (size_t)rl * n;
#pragma unroll
  for (int k = 0; k < kIntRL; ++k) {
    const uint64_t i = (uint64_t)i_first + k;
    if (i >= i0 && i < i0 + n) yr[i - i0] = fstate_value(st[k], f, d);
  }
}

template <typename T>
static int launch_integrand_t(const qk_pointset *ps, uint32_t r0, uint32_t nr, uint64_t i0, uint64_t n, int f,
                              int baker, T *y, cudaStream_t st) {
  const uint32_t d = ps->d;
  const uint64_t tiles = (i0 + n - 1) / kIntNP - i0 / kIntNP + 1;
  const size_t smem = sizeof(double) * d + sizeof(uint32_t) * ((size_t)d + 32 * d + (kIntNT / 32) * d + 3 * d);
  const bool net = ps->kind == QK_NET_B2;
  if (net) smem_optin<k_integrand<T, true>>(smem);
  else smem_optin<k_integrand<T, false>>(smem);
  for (uint32_t rc = 0; rc < nr; rc += 65535) {  // grid.y limit
    const uint32_t cnt = nr - rc < 65535 ? nr - rc : 65535;
    dim3 grid((unsigned)tiles, cnt);
    T *yc = y + (size_t)rc * n;
    if (net)
      k_integrand<T, true><<<grid, kIntNT, smem, st>>>(d, ps->order, ps->Ct, nullptr, ps->D, r0 + rc, i0, n, f, baker, yc);
    else
      k_integrand<T, false><<<grid, kIntNT, smem, st>>>(d, ps->order, nullptr, ps->g, ps->D, r0 + rc, i0, n, f, baker, yc);
    int rc_ = check_launch("qk_integrand");
    if (rc_) return rc_;
  }
  return QK_OK;
}

// ------------------------------------------------------------- RQMC estimate
// Per randomization: the FP64 sum of y over the n points (one CTA per randomization).
template <typename T>
__global__ void __launch_bounds__(1024) k_row_means(const T *__restrict__ y, uint64_t n, double *__restrict__ mu_r) {
  __shared__ double sh[32];
  const T *yr = y + (size_t)blockIdx.x * n;
  double s = 0.0;
  for (uint64_t i = threadIdx.x; i < n; i += blockDim.x) s += (double)yr[i];
  const double tot = block_sum(s, sh);
  if (threadIdx.x == 0) mu_r[blockIdx.x] = tot / (double)n;
}

// out = [mu, sigma, half width, t, mu_1 .. mu_R]: mu_r already in out[4 ..].
__global__ void k_rqmc_final(uint32_t R, double t_star, double *__restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double *mu_r = out + 4;
  double mu = 0.0;
  for (uint32_t r = 0; r < R; ++r) mu += mu_r[r];
  mu /= (double)R;
  double ss = 0.0;
  for (uint32_t r = 0; r < R; ++r) ss += (mu_r[r] - mu) * (mu_r[r] - mu);
  const double sigma = sqrt(ss / (double)(R - 1));
  out[0] = mu;
  out[1] = sigma;
  out[2] = t_star * sigma / sqrt((double)R);
  out[3] = t_star;
}

// ------------------------------------------------ Student-t quantile (host)
// Regularised incomplete beta I_x(a, b) by its continued fraction (evaluated with the
// modified Lentz method), using I_x(a, b) = 1 - I_{1-x}(b, a) where the fraction converges
// slowly (x > (a + 1)/(a + b + 2)).
static double inc_beta_cf(double a, double b, double x) {
  const double tiny = 1e-300;
  double c = 1.0, dd = 1.0 - (a + b) * x / (a + 1.0);
  if (std::fabs(dd) < tiny) dd = tiny;
  dd = 1.0 / dd;
  double h = dd;
  for (int k = 1; k <= 400; ++k) {
    // even step: k (b - k) x / ((a + 2k - 1)(a + 2k))
    double num = k * (b - k) * x / ((a + 2.0 * k - 1.0) * (a + 2.0 * k));
    dd = 1.0 + num * dd;
    c = 1.0 + num / c;
    if (std::fabs(dd) < tiny) dd = tiny;
    if (std::fabs(c) < tiny) c = tiny;
    dd = 1.0 / dd;
    h *= dd * c;
    // odd step: -(a + k)(a + b + k) x / ((a + 2k)(a + 2k + 1))
    num = -(a + k) * (a + b + k) * x / ((a + 2.0 * k) * (a + 2.0 * k + 1.0));
    dd = 1.0 + num * dd;
    c = 1.0 + num / c;
    if (std::fabs(dd) < tiny) dd = tiny;
    if (std::fabs(c) < tiny) c = tiny;
    dd = 1.0 / dd;
    const double del = dd * c;
    h *= del;
    if (std::fabs(del - 1.0) < 1e-16) break;
  }
  return h;
}

static double inc_beta(double a, double b, double x) {
  if (x <= 0.0) return 0.0;
  if (x >= 1.0) return 1.0;
  const double lbeta = std::lgamma(a) + std::lgamma(b) - std::lgamma(a + b);
  const double front = std::exp(a * std::log(x) + b * std::log1p(-x) - lbeta);
  if (x < (a + 1.0) / (a + b + 2.0)) return front * inc_beta_cf(a, b, x) / a;
  return 1.0 - front * inc_beta_cf(b, a, 1.0 - x) / b;
}

// P(T <= t) for Student's t with df degrees of freedom: for t >= 0,
// 1 - I_{df/(df + t^2)}(df/2, 1/2) / 2, and symmetry for t < 0.
static double student_t_cdf(double t, double df) {
  const double tail = 0.5 * inc_beta(0.5 * df, 0.5, df / (df + t * t));
  return t >= 0.0 ? 1.0 - tail : tail;
}

// The quantile by bisection on the monotone CDF (to the last bit of the bracket).
static double student_t_quantile(double df, double p) {
  if (p == 0.5) return 0.0;
  const bool lower = p < 0.5;
  const double q = lower ? 1.0 - p : p;
  double lo = 0.0, hi = 1.0;
  while (student_t_cdf(hi, df) < q && hi < 1e300) hi *= 2.0;
  for (int it = 0; it < 2000; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (student_t_cdf(mid, df) < q) lo = mid;
    else hi = mid;
  }
  const double v = 0.5 * (lo + hi);
  return lower ? -v : v;
}

// --------------------------------------------- squared worst-case error (Sec. 3.2)
// From the first column in form P (p = k_1/zeta - 1), per batch entry, with S = sum_i p_i
// (FP64 sums) and lambda_0 = zeta (n + S) for the kernel without nugget:
//   equal weights 1/n:        int int K - 2 zeta + 1^T K 1 / n^2 = zeta S / n
//   optimal weights K^-1 kappa = (zeta / lambda_0) 1:  zeta - zeta^2 n / lambda_0 = zeta S / (n + S)
// (kappa_i = int K(u, x_i) du = zeta and int int K = zeta: each one-dimensional K_alpha
// integrates to zero).  out (batch, 3) = [equal, optimal, optimal weight value].
template <typename T>
__global__ void __launch_bounds__(1024) k_discrepancy_closed(const T *__restrict__ col, int form, uint64_t n, double zeta,
                                                             double *__restrict__ out) {
  __shared__ double sh[32];
  const T *cr = col + (size_t)blockIdx.x * n;
  double s = 0.0;
  for (uint64_t i = threadIdx.x; i < n; i += blockDim.x)
    s += form == QK_COL_P ? (double)cr[i] : (double)cr[i] / zeta - 1.0;
  const double S = block_sum(s, sh);
  if (threadIdx.x == 0) {
    const double nn = (double)n;
    double *o = out + (size_t)blockIdx.x * 3;
    o[0] = zeta * S / nn;
    o[1] = zeta * S / (nn + S);
    o[2] = 1.0 / (nn + S);  // zeta / lambda_0
  }
}

__device__ __forceinline__ double sq_abs(float v) { return (double)v * (double)v; }
__device__ __forceinline__ double sq_abs(double v) { return v * v; }
__device__ __forceinline__ double sq_abs(float2 v) { return (double)v.x * v.x + (double)v.y * v.y; }
__device__ __forceinline__ double sq_abs(double2 v) { return v.x * v.x + v.y * v.y; }

// General weights: per vector v the partial sums of lambda_w |W_w|^2 / n (W = the
// unnormalised transform of the weights, so sum lambda |W|^2 / n = w^T K w) and of w.
template <typename E>
__global__ void k_quad_lambda(const E *__restrict__ X, const double *__restrict__ lam, int m, uint32_t nw,
                              double *__restrict__ part) {
  __shared__ double sh[32];
  const uint64_t n = 1ull << m;
  const uint32_t v = blockIdx.y;
  const double *lr = lam + (uint64_t)(v / nw) * n;
  const E *xv = X + (uint64_t)v * n;
  double q = 0.0;
  for (uint64_t w = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; w < n; w += (uint64_t)gridDim.x * blockDim.x)
    q += lr[w] * sq_abs(xv[w]);
  const double sq = block_sum(q, sh);
  if (threadIdx.x == 0) part[(uint64_t)v * gridDim.x + blockIdx.x] = sq / (double)n;
}

template <typename T>
__global__ void __launch_bounds__(1024) k_weight_sums(const T *__restrict__ w, uint64_t n, double *__restrict__ out) {
  __shared__ double sh[32];
  const T *wr = w + (size_t)blockIdx.x * n;
  double s = 0.0;
  for (uint64_t i = threadIdx.x; i < n; i += blockDim.x) s += (double)wr[i];
  const double tot = block_sum(s, sh);
  if (threadIdx.x == 0) out[blockIdx.x] = tot;
}

__global__ void k_discrepancy_final(uint32_t nvec, uint32_t blocks, double zeta, const double *__restrict__ part,
                                    const double *__restrict__ wsum, double *__restrict__ out) {
  const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nvec) return;
  double q = 0.0;
  for (uint32_t b = 0; b < blocks; ++b) q += part[(uint64_t)v * blocks + b];
  out[v] = zeta - 2.0 * zeta * wsum[v] + q;
}

constexpr uint32_t kDiscBlocks = 64;

template <typename T, typename E>
static int discrepancy_weights_t(int family, uint32_t m, uint32_t batch, uint32_t nw, const double *lam, const T *w,
                                 double zeta, double *out, void *ws, cudaStream_t st) {
  const uint32_t nvec = batch * nw;
  const uint64_t n = 1ull << m, cnt = (uint64_t)nvec << m;
  unsigned char *p = (unsigned char *)ws;
  E *X = (E *)p;
  p += align256(sizeof(E) * cnt);
  double *part = (double *)p;
  p += align256(sizeof(double) * nvec * kDiscBlocks);
  double *wsum = (double *)p;
  k_weight_sums<T><<<nvec, 1024, 0, st>>>(w, n, wsum);
  int rc = check_launch("discrepancy weight sums");
  if (rc) return rc;
  // unnormalised forward transform of the weights (the solve's first half)
  if ((rc = op_forward_real(family, m, nvec, sizeof(T) == 8 ? QK_F64 : QK_F32, w, X, st))) return rc;
  const uint32_t blocks = n < 256 * kDiscBlocks ? (uint32_t)((n + 255) / 256) : kDiscBlocks;
  k_quad_lambda<E><<<dim3(blocks, nvec), 256, 0, st>>>(X, lam, (int)m, nw, part);
  if ((rc = check_launch("discrepancy quadratic form"))) return rc;
  // part holds `blocks` entries per vector; the final sums that many
  k_discrepancy_final<<<(nvec + 127) / 128, 128, 0, st>>>(nvec, blocks, zeta, part, wsum, out);
  return check_launch("discrepancy final");
}

size_t ws_discrepancy(int family, uint32_t m, uint32_t batch, uint32_t nw, int dtype) {
  const uint64_t nvec = (uint64_t)batch * nw;
  return ws_matvec(family, m, batch, nw, dtype) + align256(sizeof(double) * nvec * kDiscBlocks) +
         align256(sizeof(double) * nvec);
}

}  // namespace qk

using namespace qk;

#define QK_TRY(x)        \
  do {                   \
    int rc_ = (x);       \
    if (rc_) return rc_; \
  } while (0)

extern "C" {

int qk_student_t_quantile(double df, double p, double *q) {
  set_error("%s", "");
  if (!q) return fail(QK_EINVAL, "qk_student_t_quantile: q is NULL");
  if (!(df > 0.0) || !std::isfinite(df)) return fail(QK_EINVAL, "degrees of freedom must be finite and > 0");
  if (!(p > 0.0 && p < 1.0)) return fail(QK_EINVAL, "p must lie in (0, 1)");
  *q = student_t_quantile(df, p);
  return QK_OK;
}

int qk_integrand(const qk_pointset *ps, uint32_t r0, uint32_t nr, uint64_t i0, uint64_t n, int32_t f, int32_t baker,
                 int32_t dtype, void *y, qk_stream stream) {
  set_error("%s", "");
  QK_TRY(check_pointset(ps, r0, nr));
  if (dtype != QK_F64 && dtype != QK_F32) return fail(QK_EINVAL, "dtype must be QK_F64 or QK_F32");
  if (f < QK_F_SIMPLE1 || f > QK_F_GENZ_CP) return fail(QK_EINVAL, "unknown integrand %d", f);
  if (f == QK_F_SIMPLE1 && ps->d != 1) return fail(QK_EINVAL, "the simple d = 1 integrand needs d = 1");
  if ((f == QK_F_SIMPLE2 || f == QK_F_OAKLEY) && ps->d != 2)
    return fail(QK_EINVAL, "this integrand is defined for d = 2 (point set has d = %u)", ps->d);
  if (i0 + n > (1ull << 32)) return fail(QK_EINVAL, "positions beyond 2^32");
  if (n == 0 || nr == 0) return QK_OK;
  if (!y) return fail(QK_EINVAL, "qk_integrand: y is NULL");
  const cudaStream_t st = (cudaStream_t)stream;
  return dtype == QK_F64 ? launch_integrand_t<double>(ps, r0, nr, i0, n, f, baker, (double *)y, st)
                         : launch_integrand_t<float>(ps, r0, nr, i0, n, f, baker, (float *)y, st);
}

int qk_rqmc(uint32_t R, uint64_t n, int32_t dtype, const void *y, double tau, double *out, qk_stream stream) {
  set_error("%s", "");
  if (dtype != QK_F64 && dtype != QK_F32) return fail(QK_EINVAL, "dtype must be QK_F64 or QK_F32");
  if (R < 2) return fail(QK_EINVAL, "the interval needs R >= 2 randomizations");
  if (n == 0) return fail(QK_EINVAL, "n must be >= 1");
  if (!(tau > 0.0 && tau < 1.0)) return fail(QK_EINVAL, "tau must lie in (0, 1)");
  if (!y || !out) return fail(QK_EINVAL, "qk_rqmc: NULL array");
  const double t_star = student_t_quantile((double)(R - 1), 1.0 - 0.5 * tau);
  const cudaStream_t st = (cudaStream_t)stream;
  if (dtype == QK_F64) k_row_means<double><<<R, 1024, 0, st>>>((const double *)y, n, out + 4);
  else k_row_means<float><<<R, 1024, 0, st>>>((const float *)y, n, out + 4);
  QK_TRY(check_launch("rqmc means"));
  k_rqmc_final<<<1, 32, 0, st>>>(R, t_star, out);
  return check_launch("rqmc interval");
}

int qk_discrepancy(int32_t family, uint32_t m, uint32_t batch, int32_t dtype, int32_t form, const void *col,
                   double zeta, double *out, qk_stream stream) {
  set_error("%s", "");
  if (family != QK_DSI && family != QK_SI) return fail(QK_EINVAL, "family must be QK_DSI or QK_SI");
  if (dtype != QK_F64 && dtype != QK_F32) return fail(QK_EINVAL, "dtype must be QK_F64 or QK_F32");
  if (m > QK_MAX_M) return fail(QK_EINVAL, "m = %u exceeds QK_MAX_M = %d", m, QK_MAX_M);
  if (form != QK_COL_K1 && form != QK_COL_P) return fail(QK_EINVAL, "form must be QK_COL_K1 or QK_COL_P");
  if (!(zeta > 0.0)) return fail(QK_EINVAL, "zeta must be > 0");
  if (batch == 0) return QK_OK;
  if (!col || !out) return fail(QK_EINVAL, "qk_discrepancy: NULL array");
  const cudaStream_t st = (cudaStream_t)stream;
  const uint64_t n = 1ull << m;
  if (dtype == QK_F64) k_discrepancy_closed<double><<<batch, 1024, 0, st>>>((const double *)col, form, n, zeta, out);
  else k_discrepancy_closed<float><<<batch, 1024, 0, st>>>((const float *)col, form, n, zeta, out);
  return check_launch("qk_discrepancy");
}

int qk_discrepancy_weights(int32_t family, uint32_t m, uint32_t batch, uint32_t nw, int32_t dtype, const double *lam,
                           const void *w, double zeta, double *out, void *ws, size_t ws_bytes, qk_stream stream) {
  set_error("%s", "");
  if (family != QK_DSI && family != QK_SI) return fail(QK_EINVAL, "family must be QK_DSI or QK_SI");
  if (dtype != QK_F64 && dtype != QK_F32) return fail(QK_EINVAL, "dtype must be QK_F64 or QK_F32");
  if (m > QK_MAX_M) return fail(QK_EINVAL, "m = %u exceeds QK_MAX_M = %d", m, QK_MAX_M);
  if (!(zeta > 0.0)) return fail(QK_EINVAL, "zeta must be > 0");
  if (batch == 0 || nw == 0) return QK_OK;
  if ((uint64_t)batch * nw > 0xFFFFFFFFull) return fail(QK_EINVAL, "batch x nw exceeds 2^32");
  if (!lam || !w || !out) return fail(QK_EINVAL, "qk_discrepancy_weights: NULL array");
  QK_TRY(check_ws(ws, ws_bytes, ws_discrepancy(family, m, batch, nw, dtype)));
  const cudaStream_t st = (cudaStream_t)stream;
  if (family == QK_DSI)
    return dtype == QK_F64 ? discrepancy_weights_t<double, double>(family, m, batch, nw, lam, (const double *)w, zeta, out, ws, st)
                           : discrepancy_weights_t<float, float>(family, m, batch, nw, lam, (const float *)w, zeta, out, ws, st);
  return dtype == QK_F64 ? discrepancy_weights_t<double, double2>(family, m, batch, nw, lam, (const double *)w, zeta, out, ws, st)
                         : discrepancy_weights_t<float, float2>(family, m, batch, nw, lam, (const float *)w, zeta, out, ws, st);
}

}  // extern "C"
