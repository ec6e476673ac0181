// Conversions between FP64 and FP32 by integer operations on the IEEE-754 layouts, for the
// FP32-arithmetic passes over FP64 vectors: on GB300 an SM retires two FP64 operations per
// clock, and these keep the element loops off the FP64 pipe.
//   f32_of: truncation toward zero to 23 mantissa bits; magnitudes below 2^-126 become a
//           signed zero, magnitudes of 2^128 and above (and non-finite values) infinity.
//   f64_of: exact; FP32 subnormals become a signed zero.
//   fixed54: the fixed-point form floor(|v| 2^(54 - esc)) of |v| < 2^esc.
// The same code compiles for the host, where tests/f32conv_host.cu checks it against the
// C library's conversions.
#pragma once
#include <cstdint>
#include <cstring>

#include <cuda_runtime.h>

namespace tnt {

__host__ __device__ __forceinline__ uint64_t bits_of(double x) {
#ifdef __CUDA_ARCH__
  return (uint64_t)__double_as_longlong(x);
#else
  uint64_t u;
  std::memcpy(&u, &x, sizeof u);
  return u;
#endif
}
__host__ __device__ __forceinline__ double double_of_bits(uint64_t u) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)u);
#else
  double x;
  std::memcpy(&x, &u, sizeof x);
  return x;
#endif
}
__host__ __device__ __forceinline__ unsigned bits_of(float x) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(x);
#else
  unsigned u;
  std::memcpy(&u, &x, sizeof u);
  return u;
#endif
}
__host__ __device__ __forceinline__ float float_of_bits(unsigned u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float x;
  std::memcpy(&x, &u, sizeof x);
  return x;
#endif
}

__host__ __device__ __forceinline__ float f32_of(double x) {
  const uint64_t u = bits_of(x);
  const unsigned hi = (unsigned)(u >> 32);
  const unsigned e = (hi >> 20) & 0x7ffu, sgn = hi & 0x80000000u;
  const unsigned m = (unsigned)(u >> 29) & 0x7fffffu;  // the 23 leading mantissa bits
  unsigned b = sgn | ((e - 896u) << 23) | m;           // exponent bias 1023 -> 127
  b = (e <= 896u) ? sgn : b;
  b = (e >= 1151u) ? (sgn | 0x7f800000u) : b;
  return float_of_bits(b);
}

__host__ __device__ __forceinline__ double f64_of(float f) {
  const unsigned b = bits_of(f);
  const unsigned e = (b >> 23) & 0xffu, sgn = b & 0x80000000u, m = b & 0x7fffffu;
  unsigned hi = sgn | ((e + 896u) << 20) | (m >> 3), lo = m << 29;
  if (e == 0u) {
    hi = sgn;
    lo = 0u;
  }
  if (e == 255u) hi = sgn | 0x7ff00000u | (m >> 3);
  return double_of_bits(((uint64_t)hi << 32) | lo);
}

// F = floor(|v| 2^(54 - esc)) for |v| < 2^esc: the 53-bit mantissa shifted (exact), the
// fixed-point form whose 6-bit groups are the slices of the FP64-accurate GEMM (oz.cu)
__host__ __device__ __forceinline__ uint64_t fixed54(double v, int esc) {
  const uint64_t u = bits_of(v);
  const int eb = (int)((u >> 52) & 0x7ff);
  uint64_t mant = u & ((1ull << 52) - 1);
  if (eb) mant |= 1ull << 52;
  const int sh = (eb ? eb : 1) - 1021 - esc;  // F = mant 2^sh, F < 2^54
  if (sh >= 0) return mant << sh;
  return sh <= -64 ? 0ull : mant >> (-sh);
}

#ifdef __CUDACC__
__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
#endif

}  // namespace tnt
