// Internal helpers shared by the libqk translation units: error reporting,
// launch checks, integer and floating-point device primitives.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/qk.h"

namespace qk {

// ------------------------------------------------------------------ host side
void set_error(const char *fmt, ...);
int fail(int code, const char *fmt, ...);
int cuda_fail(cudaError_t e, const char *what);

void count_launch();

// Call right after every kernel launch: counts it and reports launch errors.
inline int check_launch(const char *what) {
  count_launch();
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? QK_OK : cuda_fail(e, what);
}

inline unsigned ceil_div_u(uint64_t a, uint64_t b) { return (unsigned)((a + b - 1) / b); }

// Multiprocessors of the current device (queried once per device, cached).
int sm_count();

// Opt a kernel into more than 48 KB of dynamic shared memory, once per process
// and kernel (the call is skipped entirely below 48 KB, so launches that need
// no opt-in issue no extra runtime call, e.g. inside CUDA-graph capture).
template <auto FN>
inline void smem_optin(size_t bytes) {
  static size_t done = 0;  // one counter per kernel (FN is the kernel itself)
  if (bytes <= 48 * 1024 || bytes <= done) return;
  cudaFuncSetAttribute(FN, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  done = bytes;
}

// Round x up to a multiple of 256 bytes (workspace sub-allocation alignment).
__host__ __device__ inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// ---------------------------------------------------------------- device side
template <typename T> struct Cplx;
template <> struct Cplx<float> { using type = float2; };
template <> struct Cplx<double> { using type = double2; };

// Exact 2^-e for 0 <= e <= 96 (a power of two built from exponent bits).
__device__ __forceinline__ float exp2neg(float, int e) { return __int_as_float((127 - e) << 23); }
__device__ __forceinline__ double exp2neg(double, int e) {
  return __longlong_as_double((long long)(1023 - e) << 52);
}

// x = Z 2^-32 as T.  FP32: correctly rounded conversion.  FP64: exact, built as
// (1 + Z 2^-32) from the mantissa bits minus 1 (one add; GB300 converts u32 to
// f64 on its slow FP64 pipe at half the add rate).
__device__ __forceinline__ float word_to_unit(float, uint32_t Z) {
  return __uint2float_rn(Z) * 0x1p-32f;
}
__device__ __forceinline__ double word_to_unit(double, uint32_t Z) {
  return __hiloint2double((int)(0x3FF00000u | (Z >> 12)), (int)(Z << 20)) - 1.0;
}

// Sum of v over the CTA (blockDim.x a multiple of 32, at most 1024); the result is
// valid in thread 0.  sh: 32 doubles of shared scratch.  All threads must call it.
__device__ __forceinline__ double block_sum(double v, double *sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += sh[q];
  return s;
}

// Error-free sum: s + e == a + b exactly (Knuth's TwoSum; no ordering of |a|, |b| needed).
template <typename T>
__device__ __forceinline__ void two_sum(T a, T b, T &s, T &e) {
  s = a + b;
  const T bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// Float-float ("compensated") sums.  On GB300 an FP64 add costs about 40 FP32 adds, so
// FP32 reductions keep their partial sums as unevaluated pairs s + e (about 48 bits)
// and convert to FP64 once, at the end.
__device__ __forceinline__ void ff_merge(float &s, float &e, float s2, float e2) {
  float t, r;
  two_sum(s, s2, t, r);
  s = t;
  e = e + (e2 + r);
}
// Warp-wide sum of the pairs (s, e); every lane ends with the total.
__device__ __forceinline__ void warp_sum_ff(float &s, float &e) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float s2 = __shfl_xor_sync(0xffffffffu, s, o), e2 = __shfl_xor_sync(0xffffffffu, e, o);
    ff_merge(s, e, s2, e2);
  }
}
// CTA sum of thread partials: FP32 pairs (s, e) summed in float-float, FP64 partials in
// FP64.  The result is valid in thread 0.  sh: 32 doubles of shared scratch.  All
// threads must call it.
__device__ __forceinline__ double block_sum_c(float s, float e, double *sh) {
  float *f = reinterpret_cast<float *>(sh);
  warp_sum_ff(s, e);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
  __syncthreads();
  if (lane == 0) {
    f[2 * w] = s;
    f[2 * w + 1] = e;
  }
  __syncthreads();
  double out = 0.0;
  if (w == 0) {
    float a = lane < nw ? f[2 * lane] : 0.f, b = lane < nw ? f[2 * lane + 1] : 0.f;
    warp_sum_ff(a, b);
    if (lane == 0) out = (double)a + (double)b;
  }
  return out;
}
__device__ __forceinline__ double block_sum_c(double s, double e, double *sh) { return block_sum(s + e, sh); }

// Exact float -> double by integer operations for normal values (the FP64 conversion
// unit is as slow as the FP64 adder on GB300); zero, subnormal, inf and NaN inputs take
// the hardware conversion.
__device__ __forceinline__ double f2d_exact(float v) {
  const uint32_t u = __float_as_uint(v), ex = (u >> 23) & 0xFFu;
  if (ex == 0u || ex == 0xFFu) return (double)v;
  const uint32_t hi = (u & 0x80000000u) | ((ex + 896u) << 20) | ((u & 0x7FFFFFu) >> 3);
  return __hiloint2double((int)hi, (int)(u << 29));
}
__device__ __forceinline__ double f2d_exact(double v) { return v; }

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_add_u32(uint32_t *p, uint32_t v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Ticket order of a persistent two-pass tile transform (one launch for both passes of a
// batch of vectors): step s of the item sequence holds the first-pass tiles of vector s
// followed by the second-pass tiles of vector s - lag, so a vector's second pass runs
// while its first-pass output (written in place) is still in L2.  A second-pass tile of
// vector v waits until every first-pass tile of v has been published; those tiles hold
// smaller tickets, were claimed by CTAs that are running, and wait on nothing, so the
// wait ends (it is bounded all the same).
struct WhtSched {
  uint32_t nvec, lt, lag;  // lt = log2(tiles per vector and pass); 1 <= lag <= nvec
  __host__ __device__ uint32_t total() const { return (2u * nvec) << lt; }
  __device__ void decode(uint32_t i, uint32_t &v, uint32_t &tile, bool &second) const {
    const uint32_t T = 1u << lt, pre = lag << lt, mid = ((nvec - lag) << lt) * 2u;
    if (i < pre) {
      v = i >> lt, tile = i & (T - 1), second = false;
    } else if (i - pre < mid) {
      const uint32_t j = i - pre, s = j >> (lt + 1), k = j & (2 * T - 1);
      second = k >= T;
      v = second ? s : lag + s;
      tile = k & (T - 1);
    } else {
      const uint32_t j = i - pre - mid;
      v = (nvec - lag) + (j >> lt), tile = j & (T - 1), second = true;
    }
  }
};

// Packed FP32 pairs for the f32x2 arithmetic of sm_100+: one instruction applies the
// same IEEE operation (same rounding) to both halves.
__device__ __forceinline__ unsigned long long pack_f2(float a, float b) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void unpack_f2(unsigned long long v, float &a, float &b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ unsigned long long add_f2(unsigned long long x, unsigned long long y) {
  unsigned long long r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(x), "l"(y));
  return r;
}
__device__ __forceinline__ unsigned long long mul_f2(unsigned long long x, unsigned long long y) {
  unsigned long long r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(x), "l"(y));
  return r;
}
__device__ __forceinline__ unsigned long long fma_f2(unsigned long long x, unsigned long long y,
                                                     unsigned long long z) {
  unsigned long long r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(x), "l"(y), "l"(z));
  return r;
}

// Spread the low 10 bits of v so that bit p lands on bit 3p (30-bit result).
__device__ __forceinline__ uint32_t spread3_10(uint32_t v) {
  v &= 0x3FFu;
  v = (v | (v << 16)) & 0x030000FFu;
  v = (v | (v << 8)) & 0x0300F00Fu;
  v = (v | (v << 4)) & 0x030C30C3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}


// ------------------------------------------------------- float-float arithmetic
// Values carried as unevaluated pairs h + l of FP32 numbers (about 48 significant bits)
// on the FP32 pipes, from error-free transformations: TwoSum for additions and the
// product error fma(a, b, -a b) for multiplications (Dekker 1971; Knuth, TAOCP vol. 2).
// On GB300 an FP64 operation costs tens of FP32 operations, so float-float is the cheap
// way to more than FP32 precision.  Every operation is written for V = float (one value)
// or F2 (two values in one packed f32x2 register: the same IEEE operations on both
// halves), so that two points share each instruction.  The scalar forms use the _rn
// intrinsics, which the compiler never contracts into a fused multiply-add.
struct F2 {
  unsigned long long v;
};
__device__ __forceinline__ float vadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float vsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float vmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float vfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float vneg(float a) { return -a; }
__device__ __forceinline__ F2 vadd(F2 a, F2 b) { return {add_f2(a.v, b.v)}; }
__device__ __forceinline__ F2 vsub(F2 a, F2 b) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a.v), "l"(b.v));
  return {r};
}
__device__ __forceinline__ F2 vmul(F2 a, F2 b) { return {mul_f2(a.v, b.v)}; }
__device__ __forceinline__ F2 vfma(F2 a, F2 b, F2 c) { return {fma_f2(a.v, b.v, c.v)}; }
__device__ __forceinline__ F2 vneg(F2 a) { return {a.v ^ 0x8000000080000000ull}; }
__device__ __forceinline__ F2 vpack(float a, float b) { return {pack_f2(a, b)}; }
__device__ __forceinline__ F2 vsplat(float a) { return {pack_f2(a, a)}; }
__device__ __forceinline__ void vunpack(F2 x, float &a, float &b) { unpack_f2(x.v, a, b); }

template <typename V>
struct FF {
  V h, l;
};

// s + e == a + b exactly (no ordering of |a|, |b| needed).
template <typename V>
__device__ __forceinline__ FF<V> ff_two_sum(V a, V b) {
  const V s = vadd(a, b), bb = vsub(s, a);
  return {s, vadd(vsub(a, vsub(s, bb)), vsub(b, bb))};
}
// The same when |a| >= |b| or a == 0 (three operations).
template <typename V>
__device__ __forceinline__ FF<V> ff_fast_two_sum(V a, V b) {
  const V s = vadd(a, b);
  return {s, vsub(b, vsub(s, a))};
}
// x y, relative error about 2^-46 for normalised pairs (|l| <= ulp(h)/2).
template <typename V>
__device__ __forceinline__ FF<V> ff_mul(FF<V> x, FF<V> y) {
  const V p = vmul(x.h, y.h);
  V e = vfma(x.h, y.h, vneg(p));
  e = vfma(x.h, y.l, e);
  e = vfma(x.l, y.h, e);
  return ff_fast_two_sum(p, e);
}
// x + y, error about 2^-46 max(|x|, |y|).
template <typename V>
__device__ __forceinline__ FF<V> ff_add(FF<V> x, FF<V> y) {
  FF<V> s = ff_two_sum(x.h, y.h);
  return ff_fast_two_sum(s.h, vadd(s.l, vadd(x.l, y.l)));
}
// x (1 + a) + a = (1 + x)(1 + a) - 1: the product-minus-one recurrence of the first column.
template <typename V>
__device__ __forceinline__ FF<V> ff_pm1_step(FF<V> x, FF<V> a, V one) {
  FF<V> q = ff_two_sum(one, x.h);  // 1 + x, exact up to the rounding of q.l below
  q.l = vadd(q.l, x.l);
  return ff_add(x, ff_mul(a, q));
}
// The pair of a double (host or device constant): h = fl32(v), l = fl32(v - h).
__host__ __device__ inline float2 ff_split(double v) {
  const float h = (float)v;
  return make_float2(h, (float)(v - (double)h));
}

}  // namespace qk
