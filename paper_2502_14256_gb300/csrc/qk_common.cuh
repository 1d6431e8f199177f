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

constexpr int kSMs = 152;  // GB300: 2 dies x 76 SMs

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

// Spread the low 10 bits of v so that bit p lands on bit 3p (30-bit result).
__device__ __forceinline__ uint32_t spread3_10(uint32_t v) {
  v &= 0x3FFu;
  v = (v | (v << 16)) & 0x030000FFu;
  v = (v | (v << 8)) & 0x0300F00Fu;
  v = (v | (v << 4)) & 0x030C30C3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}

}  // namespace qk
