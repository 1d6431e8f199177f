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
// By tiles: a CTA builds NP consecutive points (aligned to NP) of every dimension of one
// randomization in shared memory, row-major as in the output, then writes the part inside
// [i0, i0 + n) as one contiguous, coalesced run of words.  Inside the tile a thread makes a
// run of kGenRL = 8 consecutive points of one dimension:
//   nets: the index maps h(i) = i and i ^ (i >> 1) are linear over GF(2) and the tile, run
//   and step bits of i are disjoint, so the run's first point is the XOR of a per-tile word,
//   a per-run word (both tables built once per CTA) and the shift; each next point is one
//   XOR with a column known at compile time: Gray order changes digit ctz(k + 1) (Sec. 4.3,
//   Gray code), natural order all digits below it (the XOR of columns 0 .. ctz(k + 1));
//   lattices: X_i = brev(i) g + D, one multiply-add per point.
constexpr int kGenNT = 256, kGenRL = 8, kGenWords = 8192;

// log2 of the tile's point count: the largest power of two with NP d <= kGenWords (NP >= RL).
static uint32_t gen_lognp(uint32_t d) {
  uint32_t l = 0;
  while ((2u << l) * d <= (uint32_t)kGenWords) ++l;
  return l < 3 ? 3 : l;
}

template <bool NET>
__global__ void __launch_bounds__(kGenNT) k_points_tiled(uint32_t d, int order, const uint32_t *__restrict__ Ct,
                                                         const uint32_t *__restrict__ g, const uint32_t *__restrict__ D,
                                                         uint32_t r0, uint32_t nr, uint64_t i0, uint64_t n,
                                                         uint32_t lognp, uint32_t tiles, int direct,
                                                         uint32_t *__restrict__ X) {
  extern __shared__ __align__(16) uint32_t gsm[];
  const uint32_t NP = 1u << lognp, runs = (NP / kGenRL) * d;
  // direct: rows of d >= 16 words are written from registers (a warp's store covers whole
  // 64-byte row pieces); otherwise the tile is staged in shared memory first
  uint32_t *tile = gsm;             // NP x d (staged form only)
  uint32_t *sC = tile + (direct ? 0 : NP * d);  // nets: d x 32 columns; lattices: g
  uint32_t *zrun = sC + 32 * d;     // nets: (NP / RL) x d run words
  uint32_t *ztile = zrun + runs;    // d tile words (shift included)
  const int t = threadIdx.x;
  // work items (randomization, tile) in order; each CTA takes one contiguous chunk, so the
  // per-randomization set-up (columns, run words) is redone only where the chunk crosses
  // into the next randomization
  const uint64_t total = (uint64_t)nr * tiles, chunk = (total + gridDim.x - 1) / gridDim.x;
  const uint64_t it0 = (uint64_t)blockIdx.x * chunk, it1 = it0 + chunk < total ? it0 + chunk : total;
  uint32_t cur = 0xFFFFFFFFu;
  for (uint64_t it = it0; it < it1; ++it) {
    const uint32_t rl = (uint32_t)(it / tiles), tt = (uint32_t)(it - (uint64_t)rl * tiles), r = r0 + rl;
    if (rl != cur) {  // the previous item's run phase ended at a barrier: sC / zrun are free
      cur = rl;
      if constexpr (NET) {
        for (uint32_t q = t; q < 32 * d; q += kGenNT) sC[q] = Ct[(size_t)r * d * 32 + q];
        __syncthreads();
        for (uint32_t w = t; w < runs; w += kGenNT) {
          const uint32_t q = w / d, j = w - q * d;
          zrun[w] = xor_columns(sC + j * 32, order_map(order, q * kGenRL));
        }
      } else {
        for (uint32_t j = t; j < d; j += kGenNT) sC[j] = g[j];
      }
    }
    const uint64_t base = ((i0 >> lognp) + tt) << lognp;  // < 2^32 (i0 + n <= 2^32)
    if constexpr (NET) {
      // the tile word of dimension j: one warp XOR-reduces the columns selected by the
      // digits of h(base), lane k holding column k
      const uint32_t hb = order_map(order, (uint32_t)base), lane = t & 31;
      for (uint32_t j = t >> 5; j < d; j += kGenNT / 32) {
        const uint32_t v = __reduce_xor_sync(0xffffffffu, ((hb >> lane) & 1u) ? sC[j * 32 + lane] : 0u);
        if (lane == 0) ztile[j] = v ^ (D ? D[(size_t)r * d + j] : 0u);
      }
    } else {
      for (uint32_t j = t; j < d; j += kGenNT) ztile[j] = D ? D[(size_t)r * d + j] : 0u;
    }
    // also separates the previous item's copy-out (reads of the tile) from this item's writes
    __syncthreads();
    // run (q, j): points q RL .. q RL + 7 of the tile in dimension j
    const uint64_t lo = base > i0 ? base : i0, hi = (base + NP) < (i0 + n) ? (base + NP) : (i0 + n);
    auto run = [&](uint32_t q, uint32_t j, uint32_t w) {
      if (direct) {  // straight to the output rows, positions inside [i0, i0 + n) only
        const uint64_t p0 = base + (uint64_t)q * kGenRL;
        uint32_t *dst = X + ((uint64_t)rl * n) * d + j;
        uint32_t xs[kGenRL];
        if constexpr (NET) {
          const uint32_t *cj = sC + j * 32;
          const uint32_t c0 = cj[0], c1 = cj[1], c2 = cj[2];
          const uint32_t s0 = c0, s1 = order == QK_GRAY ? c1 : (c0 ^ c1), s2 = order == QK_GRAY ? c2 : (c0 ^ c1 ^ c2);
          xs[0] = ztile[j] ^ zrun[w];
          xs[1] = xs[0] ^ s0, xs[2] = xs[1] ^ s1, xs[3] = xs[2] ^ s0, xs[4] = xs[3] ^ s2;
          xs[5] = xs[4] ^ s0, xs[6] = xs[5] ^ s1, xs[7] = xs[6] ^ s0;
        } else {
          const uint32_t gj = sC[j], dj = ztile[j];
#pragma unroll
          for (int k = 0; k < kGenRL; ++k) xs[k] = __brev((uint32_t)p0 + k) * gj + dj;
        }
#pragma unroll
        for (int k = 0; k < kGenRL; ++k)
          if (p0 + k >= lo && p0 + k < hi) dst[(p0 + k - i0) * d] = xs[k];
        return;
      }
      uint32_t *dst = tile + q * kGenRL * d + j;
      if constexpr (NET) {
        const uint32_t *cj = sC + j * 32;
        const uint32_t c0 = cj[0], c1 = cj[1], c2 = cj[2];
        // step k -> k + 1 flips digit ctz(k + 1) of the Gray index, digits 0 .. ctz(k + 1) of i
        const uint32_t s0 = c0, s1 = order == QK_GRAY ? c1 : (c0 ^ c1), s2 = order == QK_GRAY ? c2 : (c0 ^ c1 ^ c2);
        uint32_t x = ztile[j] ^ zrun[w];
        dst[0] = x;
        x ^= s0, dst[1 * d] = x;
        x ^= s1, dst[2 * d] = x;
        x ^= s0, dst[3 * d] = x;
        x ^= s2, dst[4 * d] = x;
        x ^= s0, dst[5 * d] = x;
        x ^= s1, dst[6 * d] = x;
        x ^= s0, dst[7 * d] = x;
      } else {
        const uint32_t gj = sC[j], dj = ztile[j];
        const uint32_t i = (uint32_t)base + q * kGenRL;
#pragma unroll
        for (int k = 0; k < kGenRL; ++k) dst[k * d] = __brev(i + k) * gj + dj;
      }
    };
    if (kGenNT % d == 0) {  // a thread keeps its dimension and steps through the runs
      const uint32_t j = (uint32_t)t % d;
      for (uint32_t q = (uint32_t)t / d; q < NP / kGenRL; q += kGenNT / d) run(q, j, q * d + j);
    } else {
      for (uint32_t w = t; w < runs; w += kGenNT) {
        const uint32_t q = w / d;
        run(q, w - q * d, w);
      }
    }
    __syncthreads();
    if (direct) continue;  // the barrier above also separates this item's run phase from the next
    const uint64_t words = (hi - lo) * d, soff = (lo - base) * d;
    const uint32_t *src = tile + soff;
    uint32_t *out = X + ((uint64_t)rl * n + (lo - i0)) * d;
    if ((((uintptr_t)out | (uintptr_t)src) & 15u) == 0 && (words & 3u) == 0) {  // 16-byte rows
      const uint4 *s4 = reinterpret_cast<const uint4 *>(src);
      uint4 *o4 = reinterpret_cast<uint4 *>(out);
      for (uint64_t e = t; e < (words >> 2); e += kGenNT) o4[e] = s4[e];
    } else {
      for (uint64_t e = t; e < words; e += kGenNT) out[e] = src[e];
    }
  }
}

int launch_gen_points(const qk_pointset *ps, uint32_t r0, uint32_t nr, uint64_t i0, uint64_t n,
                      uint32_t *X, cudaStream_t st) {
  if (n == 0 || nr == 0) return QK_OK;
  const uint32_t d = ps->d, lognp = gen_lognp(d), NP = 1u << lognp;
  const uint64_t tiles = ((i0 + n - 1) >> lognp) - (i0 >> lognp) + 1;  // <= 2^29
  const int direct = d >= 16;
  const size_t smem = sizeof(uint32_t) * ((direct ? 0 : (size_t)NP * d) + 32 * d + (NP / kGenRL) * d + d);
  int occ = 0;
  if (ps->kind == QK_NET_B2) {
    smem_optin<k_points_tiled<true>>(smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_points_tiled<true>, kGenNT, smem);
  } else {
    smem_optin<k_points_tiled<false>>(smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_points_tiled<false>, kGenNT, smem);
  }
  if (occ < 1) occ = 1;
  // one wave of resident CTAs, each taking an equal contiguous chunk of the (r, tile) items
  const uint64_t total = (uint64_t)nr * tiles;
  uint64_t grid = (uint64_t)sm_count() * occ;
  if (grid > total) grid = total;
  if (ps->kind == QK_NET_B2)
    k_points_tiled<true><<<(unsigned)grid, kGenNT, smem, st>>>(d, ps->order, ps->Ct, nullptr, ps->D, r0, nr, i0, n,
                                                               lognp, (uint32_t)tiles, direct, X);
  else
    k_points_tiled<false><<<(unsigned)grid, kGenNT, smem, st>>>(d, ps->order, nullptr, ps->g, ps->D, r0, nr, i0, n,
                                                                lognp, (uint32_t)tiles, direct, X);
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

// The first column in float-float arithmetic on the FP32 pipes (about 2^-46 relative per
// factor), written as FP64: for spectra that reach far below eps32 ||k_1||, where an FP32
// column would perturb the small eigenvalues beyond the 1/lambda-weighted outputs' tolerance.
template <int FAM, int ALPHA>
__global__ void __launch_bounds__(kNT) k_kernel_col_ff(ColJob job, int form, double *__restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem[];
  double *wd;
  DiffTables tb;
  carve_tables<kL>(smem, job.d, &wd, tb);
  float2 *wff = reinterpret_cast<float2 *>(wd);
  const uint32_t rl = blockIdx.y;
  const uint64_t n = 1ull << job.m;
  const uint64_t tile_base = job.i0 + (uint64_t)blockIdx.x * kTile;
  for (uint32_t q = threadIdx.x; q < job.d; q += kNT) wff[q] = ff_split(job.w[q]);
  build_all_ff<FAM, ALPHA, kL>(job, job.Ct ? job.Ct + (size_t)rl * job.d * 32 : nullptr, job.g, tile_base, tb);
  __syncthreads();
  uint32_t bi[kL];
#pragma unroll
  for (int l = 0; l < kL; ++l) bi[l] = __brev((uint32_t)(tile_base + threadIdx.x + (l << 8)));
  float ph[kL], pl[kL];
  column_sweep_ff<FAM, ALPHA, kL>(job, tb, wff, bi, ph, pl);
#pragma unroll
  for (int l = 0; l < kL; ++l) {
    const uint64_t i = tile_base - job.i0 + threadIdx.x + ((uint64_t)l << 8);
    const double p = f2d_exact(ph[l]) + f2d_exact(pl[l]);
    if (i < n) out[(size_t)rl * n + i] = form == QK_COL_P ? p : job.zeta + job.zeta * p;
  }
}

template <int FAM, int ALPHA>
static void launch_col_ff(const ColJob &job, int form, double *out, cudaStream_t st) {
  const uint64_t n = 1ull << job.m;
  dim3 grid(ceil_div_u(n, kTile), job.nr);
  const size_t smem = col_smem_bytes<kL>(job.d);
  smem_optin<k_kernel_col_ff<FAM, ALPHA>>(smem);
  k_kernel_col_ff<FAM, ALPHA><<<grid, kNT, smem, st>>>(job, form, out);
}

static int dispatch_col_ff(const ColJob &job, int form, double *out, cudaStream_t st) {
  if (job.family == QK_DSI) {
    switch (job.alpha) {
      case 1: launch_col_ff<0, 1>(job, form, out, st); break;
      case 2: launch_col_ff<0, 2>(job, form, out, st); break;
      case 3: launch_col_ff<0, 3>(job, form, out, st); break;
      case 4: launch_col_ff<0, 4>(job, form, out, st); break;
      default: return fail(QK_EINVAL, "DSI order must be 1..4");
    }
  } else {
    switch (job.alpha) {
      case 1: launch_col_ff<1, 1>(job, form, out, st); break;
      case 2: launch_col_ff<1, 2>(job, form, out, st); break;
      default: return fail(QK_EINVAL, "SI smoothness must be 1 or 2");
    }
  }
  return check_launch("qk_kernel_col (float-float)");
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
  if (dtype == QK_F32W) return dispatch_col_ff(job, form, (double *)out, st);
  return dtype == QK_F64 ? dispatch_col<double>(job, form, (double *)out, st)
                         : dispatch_col<float>(job, form, (float *)out, st);
}

// ------------------------------------------------------- gradient partials
// dk_1[i]/dc_j = zeta K_ij prod_{j' != j} f_ij' with f_ij = 1 + c_j K_ij, computed as
// zeta (1 + p_i) K_ij / f_ij (explicit product where f_ij == 0).
template <typename T, int FAM, int ALPHA>
__global__ void __launch_bounds__(kNT) k_grad_partials(ColJob job, uint32_t nrhs, const T *__restrict__ u,
                                                       double *__restrict__ partial, int pairs,
                                                       const double *__restrict__ pcol) {
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
    const size_t ui = pairs ? ((((size_t)(v >> 1) * n) + i) << 1) + (v & 1) : (size_t)v * n + i;
    uu[l] = ok[l] ? u[ui] : T(0);
  }
  T p[kL];
  if (pcol) {  // the first column as computed before (p form, FP64): no second column sweep
#pragma unroll
    for (int l = 0; l < kL; ++l) {
      const uint64_t i = tile_base + threadIdx.x + ((uint64_t)l << 8);
      p[l] = ok[l] ? (T)pcol[(size_t)rl * n + i] : T(0);
    }
  } else {
    column_sweep<T, FAM, ALPHA, kL>(job, tb, wT, bi, p);
  }
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

__global__ void k_ratio_selftest(const double *__restrict__ a, const double *__restrict__ b, double *__restrict__ q,
                                 uint64_t n) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    q[i] = ratio(a[i], b[i]);
}

template <typename T, int FAM, int ALPHA>
static void launch_grad_t(const ColJob &job, uint32_t nrhs, const T *u, double *partial, int pairs,
                          const double *pcol, cudaStream_t st) {
  dim3 grid(grad_blocks(job.m), job.nr * nrhs);
  const size_t smem = col_smem_bytes<kL>(job.d) + (size_t)(kNT / 32) * 2 * job.d * sizeof(double);
  smem_optin<k_grad_partials<T, FAM, ALPHA>>(smem);
  k_grad_partials<T, FAM, ALPHA><<<grid, kNT, smem, st>>>(job, nrhs, u, partial, pairs, pcol);
}

template <typename T>
static int dispatch_grad(const ColJob &job, uint32_t nrhs, const T *u, double *partial, int pairs,
                         const double *pcol, cudaStream_t st) {
  if (job.family == QK_DSI) {
    switch (job.alpha) {
      case 1: launch_grad_t<T, 0, 1>(job, nrhs, u, partial, pairs, pcol, st); break;
      case 2: launch_grad_t<T, 0, 2>(job, nrhs, u, partial, pairs, pcol, st); break;
      case 3: launch_grad_t<T, 0, 3>(job, nrhs, u, partial, pairs, pcol, st); break;
      case 4: launch_grad_t<T, 0, 4>(job, nrhs, u, partial, pairs, pcol, st); break;
      default: return fail(QK_EINVAL, "DSI order must be 1..4");
    }
  } else {
    switch (job.alpha) {
      case 1: launch_grad_t<T, 1, 1>(job, nrhs, u, partial, pairs, pcol, st); break;
      case 2: launch_grad_t<T, 1, 2>(job, nrhs, u, partial, pairs, pcol, st); break;
      default: return fail(QK_EINVAL, "SI smoothness must be 1 or 2");
    }
  }
  return check_launch("gradient partials");
}

int launch_grad_partials(const ColJob &job, uint32_t nrhs, int32_t dtype, const void *u, double *partial,
                         cudaStream_t st, bool pairs, const double *pcol) {
  if (job.nr == 0 || nrhs == 0) return QK_OK;
  if (job.kind == kHONet) {
    if (pairs || pcol) return fail(QK_EINVAL, "gradient partials: pair layout and stored column are for lattices");
    return launch_grad_partials_ho(job, nrhs, dtype, u, partial, st);
  }
  return dtype == QK_F64 ? dispatch_grad<double>(job, nrhs, (const double *)u, partial, pairs ? 1 : 0, pcol, st)
                         : dispatch_grad<float>(job, nrhs, (const float *)u, partial, pairs ? 1 : 0, pcol, st);
}

}  // namespace qk

using namespace qk;

extern "C" int qk_ratio_selftest(const double *a, const double *b, double *q, uint64_t n, qk_stream stream) {
  set_error("%s", "");
  if (n == 0) return QK_OK;
  if (!a || !b || !q) return fail(QK_EINVAL, "qk_ratio_selftest: NULL array");
  uint64_t blocks = (n + 255) / 256;
  const uint64_t cap = (uint64_t)sm_count() * 8;
  if (blocks > cap) blocks = cap;
  k_ratio_selftest<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(a, b, q, n);
  return check_launch("qk_ratio_selftest");
}
