// Device helpers shared by the warp-packed kernels (FP64 solve and FP32-inner
// refinement): bit-pattern tests that avoid the FP64 pipe, segment-local
// shuffle sums and the schedule-driven SpMV.
#pragma once
#include "camp_internal.h"

namespace camp {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ bool is_finite_bits(double v) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(v);
  return ((u >> 52) & 0x7ffull) != 0x7ffull;
}
// |v| < 1e-300, on the bit pattern (no FP64 instruction)
__device__ __forceinline__ bool abs_tiny(double v) {
  const unsigned long long u =
      (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull;
  return u < 0x01a56e1fc2f8f359ull;  // bit pattern of 1e-300
}
// a <= b for a, b >= +0 (or NaN a: false), on the bit pattern
__device__ __forceinline__ bool le_nonneg(double a, double b) {
  return __double_as_longlong(a) <= __double_as_longlong(b);
}

// Sum NV values over the Lc lanes of each segment (xor butterfly; every lane
// of the segment ends with the same bits).
template <int NV>
__device__ __forceinline__ void seg_sum(double (&v)[NV], int Lc) {
  for (int off = Lc >> 1; off > 0; off >>= 1) {
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] += __shfl_xor_sync(kFull, v[q], off);
  }
}

// o[row] = sum_k A_s[k] g[col k] over this lane's slots of the schedule.
__device__ __forceinline__ void seg_spmv(const SchedWord *__restrict__ sch,
                                         int L, int Lc, const double *As,
                                         const double *gs, double *os) {
  double acc = 0.0;
#pragma unroll 4
  for (int j = 0; j < L; ++j) {
    const SchedWord w = sch[j * Lc];
    acc = fma(As[w.x & 0xffffu], gs[w.x >> 16], acc);
    if (w.y >> 16) {
      os[w.y & 0xffffu] = acc;
      acc = 0.0;
    }
  }
}

// float variant of the segment sum
template <int NV>
__device__ __forceinline__ void seg_sumf(float (&v)[NV], int Lc) {
  for (int off = Lc >> 1; off > 0; off >>= 1) {
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] += __shfl_xor_sync(kFull, v[q], off);
  }
}

// o[row] = sum_k A_s[k] g[col k] in FP32 (same schedule).
__device__ __forceinline__ void seg_spmvf(const SchedWord *__restrict__ sch,
                                          int L, int Lc, const float *As,
                                          const float *gs, float *os) {
  float acc = 0.0f;
#pragma unroll 4
  for (int j = 0; j < L; ++j) {
    const SchedWord w = sch[j * Lc];
    acc = fmaf(As[w.x & 0xffffu], gs[w.x >> 16], acc);
    if (w.y >> 16) {
      os[w.y & 0xffffu] = acc;
      acc = 0.0f;
    }
  }
}

// Round-to-nearest-even FP64 -> FP32 conversion on the bit pattern (integer
// pipe) for values whose FP32 result is a normal number; zeros, subnormal
// results, overflow, Inf and NaN take the hardware conversion.  IEEE 754
// rounding written from its definition: keep 23 of the 52 fraction bits and
// round on the 29 dropped bits (ties to even); a carry out of the fraction
// increments the exponent.
__device__ __forceinline__ float d2f_rn(double v) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(v);
  const int e = (int)((u >> 52) & 0x7ffull) - 1023;
  if (e < -126 || e > 126) return __double2float_rn(v);
  const unsigned long long frac = u & 0xfffffffffffffull;
  unsigned m = (unsigned)(frac >> 29);
  const unsigned rem = (unsigned)(frac & 0x1fffffffull);
  if (rem > 0x10000000u || (rem == 0x10000000u && (m & 1u))) ++m;
  const unsigned bits = ((unsigned)(u >> 63) << 31) + ((unsigned)(e + 127) << 23) + m;
  return __uint_as_float(bits);
}

// Exact FP32 -> FP64 widening on the bit pattern for normal numbers (zeros,
// subnormals, Inf and NaN take the hardware conversion).
__device__ __forceinline__ double f2d_exact(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned ef = (b >> 23) & 0xffu;
  if (ef == 0u || ef == 0xffu) return (double)f;
  const unsigned long long u = ((unsigned long long)(b >> 31) << 63) |
                               ((unsigned long long)(ef - 127 + 1023) << 52) |
                               ((unsigned long long)(b & 0x7fffffu) << 29);
  return __longlong_as_double((long long)u);
}

}  // namespace camp
