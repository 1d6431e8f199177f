// Point generation (arXiv 2502.14256, Sec. 4.2-4.3), first Gram columns
// (Sec. 5.4, k_1[i] = K(x_i, x_0)) and the gradient reductions that recompute
// the kernel factors instead of storing them.
//
// Digital nets: the point at sequence position i is
//   X_i = D (+) XOR_{bit k of h(i)} Ct[k],  h(i) = i (natural) or i ^ (i >> 1) (Gray),
// and h is linear over GF(2).  A CTA covers 2048 consecutive positions
// i = tile | (l << 8) | (warp << 5) | lane with disjoint bit fields, so
//   X_i (+) X_0 = Z(h(lane)) (+) Z(h(warp << 5)) (+) Z(h(tile | l << 8)),
// three small per-CTA tables in shared memory: each difference word costs one
// broadcast shared load and one XOR, and the outputs of a warp are contiguous.
// Lattices: X_i (-) X_0 = v(i) 2^32 g mod 2^32 = brev(i) * g (wrapping multiply).
#include <cstdio>

#include "qk_common.cuh"
#include "qk_factors.cuh"
#include "qk_internal.h"
#include "qk_column.cuh"

namespace qk {

constexpr int kNT = 256;  // threads per CTA
constexpr int kL = 8;     // points per thread
constexpr int kTile = kNT * kL;

// --------------------------------------------------------------- LMS setup
__global__ void k_lms(uint32_t d, const uint32_t *__restrict__ C, const uint32_t *__restrict__ S,
                      uint32_t *__restrict__ Ct) {
  const uint32_t rj = blockIdx.x;       // r * d + j
  const uint32_t j = rj % d;
  const int k = threadIdx.x;            // column
  __shared__ uint32_t rows[32];
  rows[k] = S[(size_t)rj * 32 + k];
  __syncthreads();
  const uint32_t col = C[(size_t)j * 32 + k];
  uint32_t out = 0;
#pragma unroll
  for (int t = 0; t < 32; ++t) out |= (uint32_t)(__popc(rows[t] & col) & 1) << (31 - t);
  Ct[(size_t)rj * 32 + k] = out;
}

int launch_lms(uint32_t d, uint32_t R, const uint32_t *C, const uint32_t *S, uint32_t *Ct,
               cudaStream_t st) {
  const uint64_t blocks = (uint64_t)d * R;
  if (blocks == 0) return QK_OK;
  k_lms<<<(unsigned)blocks, 32, 0, st>>>(d, C, S, Ct);
  return check_launch("qk_lms_setup");
}

// ---------------------------------------------------------- point generation
__global__ void k_points_net(uint32_t d, int order, const uint32_t *__restrict__ Ct,
                             const uint32_t *__restrict__ D, uint32_t r0, uint64_t i0, uint64_t n,
                             uint32_t *__restrict__ X) {
  extern __shared__ uint32_t sC[];
  const uint32_t rl = blockIdx.y;
  const uint32_t r = r0 + rl;
  for (uint32_t q = threadIdx.x; q < d * 32; q += blockDim.x) sC[q] = Ct[(size_t)r * d * 32 + q];
  __syncthreads();
  const uint64_t total = n * d;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += stride) {
    const uint64_t i = e / d;
    const uint32_t j = (uint32_t)(e - i * d);
    const uint32_t h = order_map(order, (uint32_t)(i0 + i));
    uint32_t v = xor_columns(sC + j * 32, h);
    if (D) v ^= D[(size_t)r * d + j];
    X[(size_t)rl * total + e] = v;
  }
}

__global__ void k_points_lattice(uint32_t d, const uint32_t *__restrict__ g,
                                 const uint32_t *__restrict__ D, uint32_t r0, uint64_t i0,
                                 uint64_t n, uint32_t *__restrict__ X) {
  const uint32_t rl = blockIdx.y;
  const uint32_t r = r0 + rl;
  const uint64_t total = n * d;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += stride) {
    const uint64_t i = e / d;
    const uint32_t j = (uint32_t)(e - i * d);
    uint32_t v = __brev((uint32_t)(i0 + i)) * g[j];
    if (D) v += D[(size_t)r * d + j];
    X[(size_t)rl * total + e] = v;
  }
}

int launch_gen_points(const qk_pointset *ps, uint32_t r0, uint32_t nr, uint64_t i0, uint64_t n,
                      uint32_t *X, cudaStream_t st) {
  if (n == 0 || nr == 0) return QK_OK;
  const uint64_t total = n * ps->d;
  uint64_t blocks = (total + 255) / 256;
  if (blocks > (uint64_t)kSMs * 64) blocks = (uint64_t)kSMs * 64;
  dim3 grid((unsigned)blocks, nr);
  if (ps->kind == QK_NET_B2) {
    const size_t smem = (size_t)ps->d * 32 * sizeof(uint32_t);
    smem_optin<k_points_net>(smem);
    k_points_net<<<grid, 256, smem, st>>>(ps->d, ps->order, ps->Ct, ps->D, r0, i0, n, X);
  } else {
    k_points_lattice<<<grid, 256, 0, st>>>(ps->d, ps->g, ps->D, r0, i0, n, X);
  }
  return check_launch("qk_gen_points");
}

template <typename T, int FAM, int ALPHA>
__global__ void __launch_bounds__(kNT) k_kernel_col(ColJob job, int form, T *__restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem[];
  double *wd;
  DiffTables tb;
  carve_tables<kL>(smem, job.d, &wd, tb);
  T *wT = reinterpret_cast<T *>(wd);
  const uint32_t rl = blockIdx.y;
  const uint64_t n = 1ull << job.m;
  // positions job.i0 + [0, n); job.i0 is a multiple of kTile, so position bits split into
  // disjoint tile, l, warp and lane fields for the XOR tables
  const uint64_t tile_base = job.i0 + (uint64_t)blockIdx.x * kTile;
  for (uint32_t q = threadIdx.x; q < job.d; q += kNT) wT[q] = (T)job.w[q];
  build_all<T, FAM, ALPHA, kL>(job, job.Ct ? job.Ct + (size_t)rl * job.d * 32 : nullptr, job.g, tile_base, tb);
  __syncthreads();
  uint32_t bi[kL];
#pragma unroll
  for (int l = 0; l < kL; ++l) bi[l] = __brev((uint32_t)(tile_base + threadIdx.x + (l << 8)));
  T p[kL];
  column_sweep<T, FAM, ALPHA, kL>(job, tb, wT, bi, p);
  const T zeta = (T)job.zeta;
#pragma unroll
  for (int l = 0; l < kL; ++l) {
    const uint64_t i = tile_base - job.i0 + threadIdx.x + ((uint64_t)l << 8);
    if (i < n) out[(size_t)rl * n + i] = form == QK_COL_P ? p[l] : zeta * (T(1) + p[l]);
  }
}

template <typename T, int FAM, int ALPHA>
static void launch_col_t(const ColJob &job, int form, T *out, cudaStream_t st) {
  const uint64_t n = 1ull << job.m;
  dim3 grid(ceil_div_u(n, kTile), job.nr);
  const size_t smem = col_smem_bytes<kL>(job.d);
  smem_optin<k_kernel_col<T, FAM, ALPHA>>(smem);
  k_kernel_col<T, FAM, ALPHA><<<grid, kNT, smem, st>>>(job, form, out);
}

template <typename T>
static int dispatch_col(const ColJob &job, int form, T *out, cudaStream_t st) {
  if (job.family == QK_DSI) {
    switch (job.alpha) {
      case 1: launch_col_t<T, 0, 1>(job, form, out, st); break;
      case 2: launch_col_t<T, 0, 2>(job, form, out, st); break;
      case 3: launch_col_t<T, 0, 3>(job, form, out, st); break;
      case 4: launch_col_t<T, 0, 4>(job, form, out, st); break;
      default: return fail(QK_EINVAL, "DSI order must be 1..4");
    }
  } else {
    switch (job.alpha) {
      case 1: launch_col_t<T, 1, 1>(job, form, out, st); break;
      case 2: launch_col_t<T, 1, 2>(job, form, out, st); break;
      default: return fail(QK_EINVAL, "SI smoothness must be 1 or 2");
    }
  }
  return check_launch("qk_kernel_col");
}

int launch_kernel_col(const ColJob &job, int32_t dtype, int32_t form, void *out, cudaStream_t st) {
  if (job.nr == 0) return QK_OK;
  return dtype == QK_F64 ? dispatch_col<double>(job, form, (double *)out, st)
                         : dispatch_col<float>(job, form, (float *)out, st);
}

// ------------------------------------------------------- gradient partials
// dk_1[i]/dc_j = zeta K_ij prod_{j' != j} f_ij' with f_ij = 1 + c_j K_ij, computed as
// zeta (1 + p_i) K_ij / f_ij (explicit product where f_ij == 0).
template <typename T, int FAM, int ALPHA>
__global__ void __launch_bounds__(kNT) k_grad_partials(ColJob job, uint32_t nrhs, const T *__restrict__ u,
                                                       double *__restrict__ partial) {
  extern __shared__ __align__(16) unsigned char smem[];
  double *wd;
  DiffTables tb;
  carve_tables<kL>(smem, job.d, &wd, tb);
  T *wT = reinterpret_cast<T *>(wd);
  const uint32_t d = job.d;
  double *red = reinterpret_cast<double *>(smem + col_smem_bytes<kL>(d));  // [warp][2d]
  const uint32_t v = blockIdx.y;  // vector = r * nrhs + rhs
  const uint32_t rl = v / nrhs;
  const uint64_t n = 1ull << job.m;
  const uint64_t tile_base = (uint64_t)blockIdx.x * kTile;
  for (uint32_t q = threadIdx.x; q < d; q += kNT) wT[q] = (T)job.w[q];
  build_all<T, FAM, ALPHA, kL>(job, job.Ct ? job.Ct + (size_t)rl * d * 32 : nullptr, job.g, tile_base, tb);
  __syncthreads();
  uint32_t bi[kL];
  T uu[kL], k1[kL];
  bool ok[kL];
#pragma unroll
  for (int l = 0; l < kL; ++l) {
    const uint64_t i = tile_base + threadIdx.x + ((uint64_t)l << 8);
    bi[l] = __brev((uint32_t)i);
    ok[l] = i < n;
    uu[l] = ok[l] ? u[(size_t)v * n + i] : T(0);
  }
  T p[kL];
  column_sweep<T, FAM, ALPHA, kL>(job, tb, wT, bi, p);
  const T zeta = (T)job.zeta;
  T wk[kL];
#pragma unroll
  for (int l = 0; l < kL; ++l) {
    k1[l] = ok[l] ? zeta * (T(1) + p[l]) : T(0);
    wk[l] = uu[l] * k1[l];
  }
  gradient_sweep<T, FAM, ALPHA, kL>(job, tb, wT, bi, k1, wk, ok, [&](int l) { return uu[l]; }, red);
  __syncthreads();
  double *dst = partial + ((size_t)v * gridDim.x + blockIdx.x) * 2 * d;
  for (uint32_t q = threadIdx.x; q < 2 * d; q += kNT) dst[q] = red_total<T>(red, kNT / 32, 2 * d, q);
}

uint32_t grad_blocks(uint32_t m) { return ceil_div_u(1ull << m, kTile); }

template <typename T, int FAM, int ALPHA>
static void launch_grad_t(const ColJob &job, uint32_t nrhs, const T *u, double *partial, cudaStream_t st) {
  dim3 grid(grad_blocks(job.m), job.nr * nrhs);
  const size_t smem = col_smem_bytes<kL>(job.d) + (size_t)(kNT / 32) * 2 * job.d * sizeof(double);
  smem_optin<k_grad_partials<T, FAM, ALPHA>>(smem);
  k_grad_partials<T, FAM, ALPHA><<<grid, kNT, smem, st>>>(job, nrhs, u, partial);
}

template <typename T>
static int dispatch_grad(const ColJob &job, uint32_t nrhs, const T *u, double *partial, cudaStream_t st) {
  if (job.family == QK_DSI) {
    switch (job.alpha) {
      case 1: launch_grad_t<T, 0, 1>(job, nrhs, u, partial, st); break;
      case 2: launch_grad_t<T, 0, 2>(job, nrhs, u, partial, st); break;
      case 3: launch_grad_t<T, 0, 3>(job, nrhs, u, partial, st); break;
      case 4: launch_grad_t<T, 0, 4>(job, nrhs, u, partial, st); break;
      default: return fail(QK_EINVAL, "DSI order must be 1..4");
    }
  } else {
    switch (job.alpha) {
      case 1: launch_grad_t<T, 1, 1>(job, nrhs, u, partial, st); break;
      case 2: launch_grad_t<T, 1, 2>(job, nrhs, u, partial, st); break;
      default: return fail(QK_EINVAL, "SI smoothness must be 1 or 2");
    }
  }
  return check_launch("gradient partials");
}

int launch_grad_partials(const ColJob &job, uint32_t nrhs, int32_t dtype, const void *u, double *partial,
                         cudaStream_t st) {
  if (job.nr == 0 || nrhs == 0) return QK_OK;
  return dtype == QK_F64 ? dispatch_grad<double>(job, nrhs, (const double *)u, partial, st)
                         : dispatch_grad<float>(job, nrhs, (const float *)u, partial, st);
}

}  // namespace qk
