// Higher-order digital nets (arXiv 2502.14256, Sec. 4.3, "Digital interlacing for
// higher-order nets") and the DSI kernels on their points (Sec. 5.3):
//   * interlacing of order alpha: the alpha d (LMS-scrambled) generator matrices of a net
//     become d matrices whose digit t is digit floor(t / alpha) of matrix
//     alpha j + (t mod alpha) (0-based j); higher-order LMS is LMS on the alpha d matrices
//     (qk_lms_setup) followed by this interlacing;
//   * points as 64-digit words (t_max = min(64, 32 alpha); later digits lie below 2^-64);
//   * the first Gram column of the product DSI kernel on 64-digit difference words, with
//     beta = clz64(Z) + 1, x = Z 2^-64 and the order-4 digit series over 64 digits.
// The column feeds the spectral ops (eigenvalues, solve, MLL pieces) unchanged: an
// interlaced net is still a digital net, so its Gram matrix is RSBT and the FWHT applies.
#include "qk_column.cuh"
#include "qk_common.cuh"
#include "qk_factors.cuh"
#include "qk_internal.h"

namespace qk {

// ------------------------------------------------------------------ interlacing
// One CTA per (randomization, dimension), one thread per column k.
__global__ void k_interlace(uint32_t d, uint32_t alpha, const uint32_t *__restrict__ Ct,
                            uint64_t *__restrict__ Chat) {
  const uint32_t rj = blockIdx.x, r = rj / d, j = rj - r * d, k = threadIdx.x;
  const uint32_t *src = Ct + ((size_t)r * alpha * d + (size_t)alpha * j) * 32;  // matrices alpha j .. alpha j + alpha - 1
  const uint32_t tmax = 32 * alpha < 64 ? 32 * alpha : 64;
  uint64_t w = 0;
  for (uint32_t t = 0; t < tmax; ++t) {
    const uint32_t bit = (src[(t % alpha) * 32 + k] >> (31 - t / alpha)) & 1u;
    w |= (uint64_t)bit << (63 - t);
  }
  Chat[(size_t)rj * 32 + k] = w;
}

__device__ __forceinline__ uint64_t xor_columns64(const uint64_t *col, uint32_t v) {
  uint64_t acc = 0;
  while (v) {
    acc ^= col[__ffs(v) - 1];
    v &= v - 1;
  }
  return acc;
}

// ------------------------------------------------------------- point generation
// The tiled generator of qk_gen_points on 64-digit words: a CTA builds NP points of every
// dimension in shared memory (runs of 8 points per thread, one XOR per point), then writes
// them as one contiguous run.
constexpr int kHoNT = 256, kHoRL = 8, kHoWords = 4096;

static uint32_t ho_lognp(uint32_t d) {
  uint32_t l = 0;
  while ((2u << l) * d <= (uint32_t)kHoWords) ++l;
  return l < 3 ? 3 : l;
}

__global__ void __launch_bounds__(kHoNT) k_points_ho(uint32_t d, int order, const uint64_t *__restrict__ Chat,
                                                     const uint64_t *__restrict__ D, uint32_t r0, uint64_t i0,
                                                     uint64_t n, uint32_t lognp, uint64_t *__restrict__ X) {
  extern __shared__ __align__(16) unsigned char hsm[];
  const uint32_t NP = 1u << lognp, runs = (NP / kHoRL) * d;
  uint64_t *tile = reinterpret_cast<uint64_t *>(hsm);  // NP x d
  uint64_t *sC = tile + (size_t)NP * d;                // d x 32
  uint64_t *zrun = sC + 32 * d;                        // (NP / RL) x d
  uint64_t *ztile = zrun + runs;                       // d
  const uint32_t rl = blockIdx.y, r = r0 + rl;
  const uint64_t base = ((i0 >> lognp) + blockIdx.x) << lognp;
  const int t = threadIdx.x;
  for (uint32_t q = t; q < 32 * d; q += kHoNT) sC[q] = Chat[(size_t)r * d * 32 + q];
  __syncthreads();
  for (uint32_t w = t; w < runs; w += kHoNT) {
    const uint32_t q = w / d, j = w - q * d;
    zrun[w] = xor_columns64(sC + j * 32, order_map(order, q * kHoRL));
  }
  for (uint32_t j = t; j < d; j += kHoNT)
    ztile[j] = xor_columns64(sC + j * 32, order_map(order, (uint32_t)base)) ^ (D ? D[(size_t)r * d + j] : 0ull);
  __syncthreads();
  for (uint32_t w = t; w < runs; w += kHoNT) {
    const uint32_t q = w / d, j = w - q * d;
    uint64_t *dst = tile + (size_t)q * kHoRL * d + j;
    const uint64_t *cj = sC + j * 32;
    const uint64_t c0 = cj[0], c1 = cj[1], c2 = cj[2];
    const uint64_t s0 = c0, s1 = order == QK_GRAY ? c1 : (c0 ^ c1), s2 = order == QK_GRAY ? c2 : (c0 ^ c1 ^ c2);
    uint64_t x = ztile[j] ^ zrun[w];
    dst[0] = x;
    x ^= s0, dst[1 * d] = x;
    x ^= s1, dst[2 * d] = x;
    x ^= s0, dst[3 * d] = x;
    x ^= s2, dst[4 * d] = x;
    x ^= s0, dst[5 * d] = x;
    x ^= s1, dst[6 * d] = x;
    x ^= s0, dst[7 * d] = x;
  }
  __syncthreads();
  const uint64_t lo = base > i0 ? base : i0, hi = (base + NP) < (i0 + n) ? (base + NP) : (i0 + n);
  const uint64_t words = (hi - lo) * d;
  const uint64_t *src = tile + (lo - base) * d;
  uint64_t *out = X + ((uint64_t)rl * n + (lo - i0)) * d;
  for (uint64_t e = t; e < words; e += kHoNT) out[e] = src[e];
}

// ------------------------------------------------------------------ kernels
// K_alpha(x) of the Theorem at x = Z 2^-64 (64-digit words): beta = clz64(Z) + 1,
// t_nu = 2^(-nu beta) (products, so that FP32 underflows to 0 gracefully), and for order 4
// S' = sum over set digits a of 8^-a read from the top 21 (FP64) or 10 (FP32) digits (the
// rest lie below the precision of T: 8^-21 = 2^-63).
template <typename T, int ALPHA>
__device__ __forceinline__ T dsi_factor64(uint64_t Z) {
  if (Z == 0ull) {
    if constexpr (ALPHA == 1) return T(1);
    else if constexpr (ALPHA == 2) return T(1.5);
    else if constexpr (ALPHA == 3) return T(-1.0 + 43.0 / 18.0);
    else return T(-1.0 + 701.0 / 294.0);
  }
  const int beta = __clzll((long long)Z) + 1;
  const T t1 = exp2neg(T(), beta);
  if constexpr (ALPHA == 1) {
    return T(1) - T(3) * t1;
  } else {
    T x;
    if constexpr (sizeof(T) == 8) x = __ull2double_rn(Z) * 0x1p-64;
    else x = __ull2float_rn(Z) * 0x1p-64f;
    const T b = (T)beta;
    if constexpr (ALPHA == 2) {
      return T(1.5) - b * x - T(2.5) * t1;
    } else if constexpr (ALPHA == 3) {
      const T t2 = t1 * t1;
      return T(-1) + b * x * x - T(5) * (T(1) - t1) * x + T(43.0 / 18.0) * (T(1) - t2);
    } else {
      static_assert(ALPHA == 4, "DSI order 1..4");
      const T t2 = t1 * t1, t3 = t2 * t1, x2 = x * x;
      const T sp = octal_tail(T(), (uint32_t)(Z >> 32));
      return T(-1) - T(2.0 / 3.0) * b * x2 * x + T(5) * (T(1) - t1) * x2 - T(43.0 / 9.0) * (T(1) - t2) * x +
             T(701.0 / 294.0) * (T(1) - t3) - b * sp * T(1.0 / 24.0);
    }
  }
}

// First column of randomization r0 + blockIdx.y at 2048 consecutive positions per CTA
// (L = 8 per thread, positions tile | l << 8 | warp << 5 | lane), from three per-CTA
// tables of 64-digit difference words (the index map is linear over GF(2)).
constexpr int kHoColL = 8;

template <typename T, int ALPHA>
__global__ void __launch_bounds__(kHoNT) k_kernel_col_ho(uint32_t d, int order, uint32_t m, const uint64_t *__restrict__ Chat,
                                                         const double *__restrict__ w, double zeta, int form,
                                                         T *__restrict__ out) {
  extern __shared__ __align__(16) unsigned char csm[];
  double *wd = reinterpret_cast<double *>(csm);
  uint64_t *zlane = reinterpret_cast<uint64_t *>(wd + d);  // [j][lane]
  uint64_t *zwarp = zlane + 32 * d;                         // [warp][j]
  uint64_t *zl = zwarp + (kHoNT / 32) * d;                  // [j][l]
  const uint32_t rl = blockIdx.y;
  const uint64_t n = 1ull << m;
  const uint64_t tile_base = (uint64_t)blockIdx.x * (kHoNT * kHoColL);
  const uint64_t *Cr = Chat + (size_t)rl * d * 32;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  for (uint32_t q = t; q < d; q += kHoNT) wd[q] = w[q];
  for (uint32_t q = t; q < 32 * d; q += kHoNT) {
    const uint32_t j = q >> 5, ln = q & 31;
    zlane[q] = xor_columns64(Cr + j * 32, order_map(order, ln));
  }
  for (uint32_t q = t; q < (kHoNT / 32) * d; q += kHoNT) {
    const uint32_t ww = q / d, j = q - ww * d;
    zwarp[q] = xor_columns64(Cr + j * 32, order_map(order, ww << 5));
  }
  for (uint32_t q = t; q < kHoColL * d; q += kHoNT) {
    const uint32_t j = q / kHoColL, l = q - j * kHoColL;
    zl[q] = xor_columns64(Cr + j * 32, order_map(order, (uint32_t)(tile_base | ((uint64_t)l << 8))));
  }
  __syncthreads();
  T p[kHoColL];
#pragma unroll
  for (int l = 0; l < kHoColL; ++l) p[l] = T(0);
  for (uint32_t j = 0; j < d; ++j) {
    const T wj = (T)wd[j];
    const uint64_t b = zlane[j * 32 + lane] ^ zwarp[warp * d + j];
#pragma unroll
    for (int l = 0; l < kHoColL; ++l) p[l] = pm1_step(p[l], wj * dsi_factor64<T, ALPHA>(b ^ zl[j * kHoColL + l]));
  }
#pragma unroll
  for (int l = 0; l < kHoColL; ++l) {
    const uint64_t i = tile_base + t + ((uint64_t)l << 8);
    if (i < n) out[(size_t)rl * n + i] = form == QK_COL_P ? p[l] : (T)zeta * (T(1) + p[l]);
  }
}

template <typename T, int ALPHA>
static int launch_col_ho_t(const qk_hopointset *ps, const qk_kernel *k, uint32_t r0, uint32_t nr, uint32_t m, int form,
                           T *out, cudaStream_t st) {
  const uint32_t d = ps->d;
  const uint64_t n = 1ull << m;
  const size_t smem = sizeof(double) * d + sizeof(uint64_t) * ((size_t)32 * d + (kHoNT / 32) * d + kHoColL * d);
  smem_optin<k_kernel_col_ho<T, ALPHA>>(smem);
  for (uint32_t rc = 0; rc < nr; rc += 65535) {
    const uint32_t cnt = nr - rc < 65535 ? nr - rc : 65535;
    dim3 grid(ceil_div_u(n, kHoNT * kHoColL), cnt);
    k_kernel_col_ho<T, ALPHA><<<grid, kHoNT, smem, st>>>(d, ps->order, m, ps->Chat + (size_t)(r0 + rc) * d * 32,
                                                         k->weights, k->zeta, form, out + (size_t)rc * n);
    int rc_ = check_launch("qk_kernel_col_ho");
    if (rc_) return rc_;
  }
  return QK_OK;
}

template <typename T>
static int dispatch_col_ho(const qk_hopointset *ps, const qk_kernel *k, uint32_t r0, uint32_t nr, uint32_t m, int form,
                           T *out, cudaStream_t st) {
  switch (k->alpha) {
    case 1: return launch_col_ho_t<T, 1>(ps, k, r0, nr, m, form, out, st);
    case 2: return launch_col_ho_t<T, 2>(ps, k, r0, nr, m, form, out, st);
    case 3: return launch_col_ho_t<T, 3>(ps, k, r0, nr, m, form, out, st);
    case 4: return launch_col_ho_t<T, 4>(ps, k, r0, nr, m, form, out, st);
    default: return fail(QK_EINVAL, "DSI order must be 1..4");
  }
}

// ------------------------------------------------------- gradient partial sums
// For vector v = r nrhs + q (blockIdx.y) and the 2048 points of this CTA: per dimension j,
// sum_i u_i dk1_i/dc_j and sum_i dk1_i/dc_j with dk1_i/dc_j = k1_i K_ij / (1 + c_j K_ij)
// (the explicit product over the other dimensions where 1 + c_j K_ij = 0), the factors
// recomputed from the 64-digit words; written as partial[v][blockIdx.x][2d] (the layout
// of the 32-digit gradient partials, 2048 points per block).
template <typename T, int ALPHA>
__global__ void __launch_bounds__(kHoNT) k_grad_partials_ho(uint32_t d, int order, uint32_t m, uint32_t nrhs,
                                                            const uint64_t *__restrict__ Chat,
                                                            const double *__restrict__ w, double zeta,
                                                            const T *__restrict__ u, double *__restrict__ partial) {
  extern __shared__ __align__(16) unsigned char gsm2[];
  double *wd = reinterpret_cast<double *>(gsm2);
  double *red = wd + d;                                     // [warp][2d]
  uint64_t *zlane = reinterpret_cast<uint64_t *>(red + (kHoNT / 32) * 2 * d);
  uint64_t *zwarp = zlane + 32 * d;
  uint64_t *zl = zwarp + (kHoNT / 32) * d;
  const uint32_t v = blockIdx.y, rl = v / nrhs;
  const uint64_t n = 1ull << m;
  const uint64_t tile_base = (uint64_t)blockIdx.x * (kHoNT * kHoColL);
  const uint64_t *Cr = Chat + (size_t)rl * d * 32;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  for (uint32_t q = t; q < d; q += kHoNT) wd[q] = w[q];
  for (uint32_t q = t; q < 32 * d; q += kHoNT) {
    const uint32_t j = q >> 5, ln = q & 31;
    zlane[q] = xor_columns64(Cr + j * 32, order_map(order, ln));
  }
  for (uint32_t q = t; q < (kHoNT / 32) * d; q += kHoNT) {
    const uint32_t ww = q / d, j = q - ww * d;
    zwarp[q] = xor_columns64(Cr + j * 32, order_map(order, ww << 5));
  }
  for (uint32_t q = t; q < kHoColL * d; q += kHoNT) {
    const uint32_t j = q / kHoColL, l = q - j * kHoColL;
    zl[q] = xor_columns64(Cr + j * 32, order_map(order, (uint32_t)(tile_base | ((uint64_t)l << 8))));
  }
  __syncthreads();
  T p[kHoColL], uu[kHoColL], k1[kHoColL];
  bool ok[kHoColL];
#pragma unroll
  for (int l = 0; l < kHoColL; ++l) {
    const uint64_t i = tile_base + t + ((uint64_t)l << 8);
    ok[l] = i < n;
    uu[l] = ok[l] ? u[(size_t)v * n + i] : T(0);
    p[l] = T(0);
  }
  for (uint32_t j = 0; j < d; ++j) {
    const T wj = (T)wd[j];
    const uint64_t b = zlane[j * 32 + lane] ^ zwarp[warp * d + j];
#pragma unroll
    for (int l = 0; l < kHoColL; ++l) p[l] = pm1_step(p[l], wj * dsi_factor64<T, ALPHA>(b ^ zl[j * kHoColL + l]));
  }
#pragma unroll
  for (int l = 0; l < kHoColL; ++l) k1[l] = ok[l] ? (T)zeta * (T(1) + p[l]) : T(0);
  for (uint32_t j = 0; j < d; ++j) {
    const T wj = (T)wd[j];
    const uint64_t b = zlane[j * 32 + lane] ^ zwarp[warp * d + j];
    double su = 0.0, s1 = 0.0;
#pragma unroll
    for (int l = 0; l < kHoColL; ++l) {
      if (!ok[l]) continue;
      const uint64_t bl = b ^ zl[j * kHoColL + l];
      const T K = dsi_factor64<T, ALPHA>(bl);
      const T f = fmadd(wj, K, T(1));
      T dk;
      if (f != T(0)) {
        dk = k1[l] * (K / f);
      } else {  // 1 + c_j K = 0: the product of the other factors, explicitly
        dk = (T)zeta * K;
        for (uint32_t jj = 0; jj < d; ++jj) {
          if (jj == j) continue;
          const uint64_t bj = zlane[jj * 32 + lane] ^ zwarp[warp * d + jj] ^ zl[jj * kHoColL + l];
          dk *= T(1) + (T)wd[jj] * dsi_factor64<T, ALPHA>(bj);
        }
      }
      su += (double)uu[l] * (double)dk;
      s1 += (double)dk;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      su += __shfl_xor_sync(0xffffffffu, su, o);
      s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    }
    if (lane == 0) {
      red[(size_t)warp * 2 * d + j] = su;
      red[(size_t)warp * 2 * d + d + j] = s1;
    }
  }
  __syncthreads();
  double *dst = partial + ((size_t)v * gridDim.x + blockIdx.x) * 2 * d;
  for (uint32_t q = t; q < 2 * d; q += kHoNT) {
    double s = 0.0;
    for (int ww = 0; ww < kHoNT / 32; ++ww) s += red[(size_t)ww * 2 * d + q];
    dst[q] = s;
  }
}

template <typename T, int ALPHA>
static int launch_grad_ho_t(const ColJob &job, uint32_t nrhs, const T *u, double *partial, cudaStream_t st) {
  const uint32_t d = job.d;
  const uint64_t n = 1ull << job.m;
  const size_t smem = sizeof(double) * ((size_t)d + (kHoNT / 32) * 2 * d) +
                      sizeof(uint64_t) * ((size_t)32 * d + (kHoNT / 32) * d + kHoColL * d);
  smem_optin<k_grad_partials_ho<T, ALPHA>>(smem);
  const uint64_t nvec = (uint64_t)job.nr * nrhs;
  if (nvec > 65535) return fail(QK_EINVAL, "higher-order gradient: more than 65535 vectors per call");
  dim3 grid(ceil_div_u(n, kHoNT * kHoColL), (unsigned)nvec);
  k_grad_partials_ho<T, ALPHA><<<grid, kHoNT, smem, st>>>(d, job.order, job.m, nrhs, job.Chat, job.w, job.zeta, u,
                                                          partial);
  return check_launch("higher-order gradient partials");
}

template <typename T>
static int dispatch_grad_ho(const ColJob &job, uint32_t nrhs, const T *u, double *partial, cudaStream_t st) {
  switch (job.alpha) {
    case 1: return launch_grad_ho_t<T, 1>(job, nrhs, u, partial, st);
    case 2: return launch_grad_ho_t<T, 2>(job, nrhs, u, partial, st);
    case 3: return launch_grad_ho_t<T, 3>(job, nrhs, u, partial, st);
    case 4: return launch_grad_ho_t<T, 4>(job, nrhs, u, partial, st);
    default: return fail(QK_EINVAL, "DSI order must be 1..4");
  }
}

int launch_grad_partials_ho(const ColJob &job, uint32_t nrhs, int32_t dtype, const void *u, double *partial,
                            cudaStream_t st) {
  return dtype == QK_F64 ? dispatch_grad_ho<double>(job, nrhs, (const double *)u, partial, st)
                         : dispatch_grad_ho<float>(job, nrhs, (const float *)u, partial, st);
}

static int check_hopointset(const qk_hopointset *ps, uint32_t r0, uint32_t nr) {
  if (!ps) return fail(QK_EINVAL, "higher-order point set is NULL");
  if (ps->d < 1 || ps->d > QK_MAX_D) return fail(QK_EINVAL, "d = %u outside 1..%d", ps->d, QK_MAX_D);
  if ((uint64_t)r0 + nr > ps->R) return fail(QK_EINVAL, "randomizations %u..%u exceed R = %u", r0, r0 + nr, ps->R);
  if (!ps->Chat) return fail(QK_EINVAL, "higher-order point set without interlaced columns");
  if (ps->order != QK_NATURAL && ps->order != QK_GRAY) return fail(QK_EINVAL, "order must be natural or Gray");
  return QK_OK;
}

}  // namespace qk

using namespace qk;

#define QK_TRY(x)        \
  do {                   \
    int rc_ = (x);       \
    if (rc_) return rc_; \
  } while (0)

extern "C" {

int qk_interlace(uint32_t d, uint32_t R, uint32_t alpha, const uint32_t *Ct, uint64_t *Chat, qk_stream stream) {
  set_error("%s", "");
  if (d < 1 || d > QK_MAX_D) return fail(QK_EINVAL, "d = %u outside 1..%d", d, QK_MAX_D);
  if (alpha < 1 || alpha > 4) return fail(QK_EINVAL, "interlacing order must be 1..4");
  if ((uint64_t)alpha * d * 32 > 0xFFFFFFFFull) return fail(QK_EINVAL, "alpha d too large");
  if (R == 0) return QK_OK;
  if (!Ct || !Chat) return fail(QK_EINVAL, "qk_interlace: NULL array");
  if ((uint64_t)R * d >= (1ull << 31)) return fail(QK_EINVAL, "R d exceeds the grid");
  k_interlace<<<R * d, 32, 0, (cudaStream_t)stream>>>(d, alpha, Ct, Chat);
  return check_launch("qk_interlace");
}

int qk_gen_points_ho(const qk_hopointset *ps, uint32_t r0, uint32_t nr, uint64_t i0, uint64_t n, uint64_t *X,
                     qk_stream stream) {
  set_error("%s", "");
  QK_TRY(check_hopointset(ps, r0, nr));
  if (i0 + n > (1ull << 32)) return fail(QK_EINVAL, "positions beyond 2^32");
  if (n == 0 || nr == 0) return QK_OK;
  if (!X) return fail(QK_EINVAL, "qk_gen_points_ho: X is NULL");
  const uint32_t d = ps->d, lognp = ho_lognp(d), NP = 1u << lognp;
  const uint64_t tiles = ((i0 + n - 1) >> lognp) - (i0 >> lognp) + 1;
  const size_t smem = sizeof(uint64_t) * ((size_t)NP * d + 32 * d + (NP / kHoRL) * d + d);
  smem_optin<k_points_ho>(smem);
  for (uint32_t rc = 0; rc < nr; rc += 65535) {
    const uint32_t cnt = nr - rc < 65535 ? nr - rc : 65535;
    k_points_ho<<<dim3((unsigned)tiles, cnt), kHoNT, smem, (cudaStream_t)stream>>>(
        d, ps->order, ps->Chat, ps->D, r0 + rc, i0, n, lognp, X + (size_t)rc * n * d);
    QK_TRY(check_launch("qk_gen_points_ho"));
  }
  return QK_OK;
}

int qk_kernel_col_ho(const qk_hopointset *ps, const qk_kernel *k, uint32_t r0, uint32_t nr, uint32_t m, int32_t dtype,
                     int32_t form, void *col, qk_stream stream) {
  set_error("%s", "");
  QK_TRY(check_hopointset(ps, r0, nr));
  if (!k) return fail(QK_EINVAL, "kernel is NULL");
  if (k->family != QK_DSI) return fail(QK_EINVAL, "higher-order nets pair with DSI kernels (Sec. 5.3)");
  if (k->alpha < 1 || k->alpha > 4) return fail(QK_EINVAL, "DSI order must be 1..4");
  if (k->d != ps->d) return fail(QK_EINVAL, "kernel d = %u differs from point-set d = %u", k->d, ps->d);
  if (!k->weights) return fail(QK_EINVAL, "kernel weights are NULL");
  if (!(k->zeta > 0.0)) return fail(QK_EINVAL, "zeta must be > 0");
  if (dtype != QK_F64 && dtype != QK_F32) return fail(QK_EINVAL, "dtype must be QK_F64 or QK_F32");
  if (m > QK_MAX_M) return fail(QK_EINVAL, "m = %u exceeds QK_MAX_M = %d", m, QK_MAX_M);
  if (form != QK_COL_K1 && form != QK_COL_P) return fail(QK_EINVAL, "form must be QK_COL_K1 or QK_COL_P");
  if (nr == 0) return QK_OK;
  if (!col) return fail(QK_EINVAL, "qk_kernel_col_ho: output is NULL");
  const cudaStream_t st = (cudaStream_t)stream;
  return dtype == QK_F64 ? dispatch_col_ho<double>(ps, k, r0, nr, m, form, (double *)col, st)
                         : dispatch_col_ho<float>(ps, k, r0, nr, m, form, (float *)col, st);
}

int qk_mll_ho(const qk_hopointset *ps, const qk_kernel *k, uint32_t r0, uint32_t nr, uint32_t m, uint32_t nrhs,
              int32_t dtype, const double *lam, const void *y, double *out, double *grad, void *ws, size_t ws_bytes,
              qk_stream stream) {
  set_error("%s", "");
  QK_TRY(check_hopointset(ps, r0, nr));
  if (!k) return fail(QK_EINVAL, "kernel is NULL");
  if (k->family != QK_DSI) return fail(QK_EINVAL, "higher-order nets pair with DSI kernels (Sec. 5.3)");
  if (k->alpha < 1 || k->alpha > 4) return fail(QK_EINVAL, "DSI order must be 1..4");
  if (k->d != ps->d) return fail(QK_EINVAL, "kernel d = %u differs from point-set d = %u", k->d, ps->d);
  if (!k->weights) return fail(QK_EINVAL, "kernel weights are NULL");
  if (!(k->zeta > 0.0)) return fail(QK_EINVAL, "zeta must be > 0");
  if (dtype != QK_F64 && dtype != QK_F32) return fail(QK_EINVAL, "dtype must be QK_F64 or QK_F32");
  if (m > QK_MAX_M) return fail(QK_EINVAL, "m = %u exceeds QK_MAX_M = %d", m, QK_MAX_M);
  if (nr == 0 || nrhs == 0) return QK_OK;
  if (!lam || !y || !out) return fail(QK_EINVAL, "qk_mll_ho: NULL array");
  if (grad && (uint64_t)nr * nrhs > 65535) return fail(QK_EINVAL, "qk_mll_ho: nr nrhs > 65535 with a gradient");
  QK_TRY(check_ws(ws, ws_bytes, ws_mll(QK_DSI, m, nr, nrhs, dtype, ps->d)));
  ColJob job{};
  job.kind = kHONet;
  job.order = ps->order;
  job.d = ps->d;
  job.m = m;
  job.Chat = ps->Chat + (size_t)r0 * ps->d * 32;
  job.w = k->weights;
  job.zeta = k->zeta;
  job.family = QK_DSI;
  job.alpha = k->alpha;
  job.nr = nr;
  return op_mll(job, nrhs, dtype, lam, y, out, grad, ws, (cudaStream_t)stream);
}

int qk_mll_spectrum(int32_t family, uint32_t m, uint32_t nr, uint32_t nrhs, int32_t dtype, double zeta,
                    const double *lam, const void *y, double *out, void *ws, size_t ws_bytes, qk_stream stream) {
  set_error("%s", "");
  if (family != QK_DSI && family != QK_SI) return fail(QK_EINVAL, "family must be QK_DSI or QK_SI");
  if (dtype != QK_F64 && dtype != QK_F32) return fail(QK_EINVAL, "dtype must be QK_F64 or QK_F32");
  if (m > QK_MAX_M) return fail(QK_EINVAL, "m = %u exceeds QK_MAX_M = %d", m, QK_MAX_M);
  if (!(zeta > 0.0)) return fail(QK_EINVAL, "zeta must be > 0");
  if (nr == 0 || nrhs == 0) return QK_OK;
  if (!lam || !y || !out) return fail(QK_EINVAL, "qk_mll_spectrum: NULL array");
  QK_TRY(check_ws(ws, ws_bytes, ws_mll(family, m, nr, nrhs, dtype, 0)));
  ColJob job{};
  job.family = family;
  job.m = m;
  job.nr = nr;
  job.zeta = zeta;
  job.d = 0;
  return op_mll(job, nrhs, dtype, lam, y, out, nullptr, ws, (cudaStream_t)stream);
}

}  // extern "C"
