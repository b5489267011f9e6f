// Device helpers shared by the warp-packed kernels (FP64 solve and FP32-inner
// refinement): bit-pattern tests that avoid the FP64 pipe, segment-local
// shuffle sums and the schedule-driven SpMV.
#pragma once
#include "camp_internal.h"

namespace camp {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kSpmvUnroll = 4;  // SpMV pipeline block (slots per lane)

// Difficulty class of a cell from the high word of its estimate
// max_i |A_ii - 1| (a non-negative double, so its high words order as
// integers): the half-octave index (exponent and first fraction bit),
// largest first; estimates >= 12 share class 0, those below 2^-29 (and zero)
// the last class.
__device__ __forceinline__ int difficulty_class(unsigned hi) {
  const int idx = (int)(hi >> 19);  // 2 * biased exponent + top fraction bit
  const int top = ((1023 + 3) << 1) | 1;
  const int c = top - idx;
  return c < 0 ? 0 : (c >= kOrdClasses ? kOrdClasses - 1 : c);
}
__device__ __forceinline__ unsigned diag_departure_hi(double aii) {
  return (unsigned)((unsigned long long)__double_as_longlong(fabs(aii - 1.0)) >> 32);
}
// The same key from gamma itself (its magnitude, on the integer pipe).
__device__ __forceinline__ unsigned magnitude_hi(double v) {
  return (unsigned)(((unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull) >> 32);
}

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

// Two sums over the segment with log2(Lc) FP64 additions instead of
// 2 log2(Lc): at the first level each lane pair exchanges the value the other
// keeps (the lower lane keeps a, the upper keeps b), then one value is summed;
// a final exchange gives every lane both totals.
__device__ __forceinline__ void seg_sum2(double &a, double &b, int Lc) {
  if (Lc == 1) return;
  const int half = Lc >> 1;
  const bool up = (threadIdx.x & half) != 0;
  double keep = up ? b : a;
  const double send = up ? a : b;
  keep += __shfl_xor_sync(kFull, send, half);
  for (int off = half >> 1; off > 0; off >>= 1) keep += __shfl_xor_sync(kFull, keep, off);
  const double other = __shfl_xor_sync(kFull, keep, half);
  a = up ? other : keep;
  b = up ? keep : other;
}

// Three sums (a fourth slot is zero) with two transposing levels: 2 + 1 +
// (log2(Lc) - 2) FP64 additions for Lc >= 4.
__device__ __forceinline__ void seg_sum3(double &a, double &b, double &c, int Lc) {
  if (Lc < 4) {
    double v[3] = {a, b, c};
    seg_sum<3>(v, Lc);
    a = v[0]; b = v[1]; c = v[2];
    return;
  }
  const int h1 = Lc >> 1, h2 = Lc >> 2;
  const bool u1 = (threadIdx.x & h1) != 0;
  const bool u2 = (threadIdx.x & h2) != 0;
  // level 1: lower half keeps (a, b), upper half keeps (c, 0)
  double k0 = u1 ? c : a, k1 = u1 ? 0.0 : b;
  const double s0 = u1 ? a : c, s1 = u1 ? b : 0.0;
  k0 += __shfl_xor_sync(kFull, s0, h1);
  k1 += __shfl_xor_sync(kFull, s1, h1);
  // level 2: lower quarter keeps k0, upper keeps k1
  double k = u2 ? k1 : k0;
  const double s = u2 ? k0 : k1;
  k += __shfl_xor_sync(kFull, s, h2);
  for (int off = h2 >> 1; off > 0; off >>= 1) k += __shfl_xor_sync(kFull, k, off);
  // lane classes (u1, u2): (0,0) a, (0,1) b, (1,0) c, (1,1) zero
  const double x2 = __shfl_xor_sync(kFull, k, h2);
  const double x1 = __shfl_xor_sync(kFull, k, h1);
  const double x3 = __shfl_xor_sync(kFull, k, h1 | h2);
  // the lane whose class is (p, q) holds: own k, x2 = (p, !q), x1 = (!p, q), x3 = (!p, !q)
  const double va = (!u1 && !u2) ? k : (!u1 && u2) ? x2 : (u1 && !u2) ? x1 : x3;
  const double vb = (!u1 && u2) ? k : (!u1 && !u2) ? x2 : (u1 && u2) ? x1 : x3;
  const double vc = (u1 && !u2) ? k : (u1 && u2) ? x2 : (!u1 && !u2) ? x1 : x3;
  a = va; b = vb; c = vc;
}

__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }

// *p = v when flag != 0, as one predicated shared-memory store (no branch)
__device__ __forceinline__ void store_if(unsigned flag, double *p, double v) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %0, 0;\n\t@q st.shared.f64 [%1], %2;\n\t}"
               :: "r"(flag), "r"(a), "d"(v) : "memory");
}
__device__ __forceinline__ void store_if(unsigned flag, float *p, float v) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %0, 0;\n\t@q st.shared.f32 [%1], %2;\n\t}"
               :: "r"(flag), "r"(a), "f"(v) : "memory");
}

// os[row] = sum over this lane's slots of A_slot * gs[col] (os: shared
// memory).  sch and loadA(j) give this lane's word and A value of slot j.
// Software pipeline over blocks of P slots: the block's A values and gathers
// (its words were read one block earlier) and the next block's words are
// issued before the block's chain of multiply-adds, so the shared-memory
// latency runs under the FP64 chain; a row end is a predicated store and a
// select, without a branch.  Slots past L read word 0 and A = 0 (no row end
// follows them).
template <class T, class LoadA>
__device__ __forceinline__ void spmv_slots(const SchedWord *__restrict__ sch, int L, int Lc,
                                           LoadA loadA, const T *__restrict__ gs,
                                           T *__restrict__ os) {
  constexpr int P = kSpmvUnroll;
  SchedWord w[P];
#pragma unroll
  for (int u = 0; u < P; ++u) w[u] = u < L ? sch[u * Lc] : 0u;
  T acc = T(0);
  for (int j0 = 0; j0 < L; j0 += P) {
    T av[P], xv[P];
    SchedWord wn[P];
#pragma unroll
    for (int u = 0; u < P; ++u) {
      av[u] = j0 + u < L ? loadA(j0 + u) : T(0);
      xv[u] = gs[w[u] & 0x7ffu];
    }
#pragma unroll
    for (int u = 0; u < P; ++u) {
      const int j = j0 + P + u;
      wn[u] = j < L ? sch[j * Lc] : 0u;
    }
#pragma unroll
    for (int u = 0; u < P; ++u) {
      acc = fma_t(av[u], xv[u], acc);
      store_if(w[u] & kSlotEnd, os + ((w[u] >> 11) & 0x7ffu), acc);
      acc = (w[u] & kSlotEnd) ? T(0) : acc;
    }
#pragma unroll
    for (int u = 0; u < P; ++u) w[u] = wn[u];
  }
}

// o[row] = sum over this lane's slots of A_slot * g[col].  sch and As point at
// this lane's column of the schedule and of the slot-ordered A (stride Lc).
__device__ __forceinline__ void seg_spmv(const SchedWord *__restrict__ sch,
                                         int L, int Lc,
                                         const double *__restrict__ As,
                                         const double *__restrict__ gs,
                                         double *__restrict__ os) {
  spmv_slots<double>(sch, L, Lc, [&](int j) { return As[j * Lc]; }, gs, os);
}

// Same with A read from global memory through the slot's source entry.
__device__ __forceinline__ void seg_spmv_gather(const SchedWord *__restrict__ sch,
                                                const int *__restrict__ src,
                                                int L, int Lc,
                                                const double *__restrict__ Ag,
                                                const double *__restrict__ gs,
                                                double *__restrict__ os) {
  spmv_slots<double>(sch, L, Lc, [&](int j) {
    const int k = __ldg(src + j * Lc);
    return k >= 0 ? __ldg(Ag + k) : 0.0;
  }, gs, os);
}

// Coalesced, vectorised read of one cell's A row (CSR order), handed to
// put(slot, value) with the slot from the dst map.  The row is read in
// 16-byte pairs from its first 16-byte boundary (lane sl reads pairs sl,
// sl + Lc, ...); an entry before that boundary and an odd entry at the end
// are read alone by lane 0.  The loads of kStagePairs pairs are issued before
// any store, so a lane waits for memory once per batch rather than once per
// entry.
constexpr int kStagePairs = 8;
template <class Put>
__device__ __forceinline__ void stage_scatter(const double *__restrict__ Ac,
                                              const int *__restrict__ dst, int nnz,
                                              int sl, int Lc, bool live, Put put) {
  const int h = (int)((reinterpret_cast<size_t>(Ac) >> 3) & 1);  // entries before the boundary
  const int np = (nnz - h) >> 1;                                  // whole pairs
  const double2 *A2 = reinterpret_cast<const double2 *>(Ac + h);
  const int *d2 = dst + h;
  for (int p0 = sl; p0 < np; p0 += kStagePairs * Lc) {
    double2 v[kStagePairs];
    int d[2 * kStagePairs];
#pragma unroll
    for (int u = 0; u < kStagePairs; ++u) {
      const int p = p0 + u * Lc;
      const bool in = p < np;
      d[2 * u] = in ? __ldg(d2 + 2 * p) : -1;
      d[2 * u + 1] = in ? __ldg(d2 + 2 * p + 1) : -1;
      v[u] = (live && in) ? __ldg(A2 + p) : make_double2(0.0, 0.0);
    }
#pragma unroll
    for (int u = 0; u < kStagePairs; ++u) {
      if (d[2 * u] >= 0) put(d[2 * u], v[u].x);
      if (d[2 * u + 1] >= 0) put(d[2 * u + 1], v[u].y);
    }
  }
  if (sl == 0) {
    if (h) put(__ldg(dst), live ? __ldg(Ac) : 0.0);
    if ((nnz - h) & 1) put(__ldg(dst + nnz - 1), live ? __ldg(Ac + nnz - 1) : 0.0);
  }
}

// Zero this lane's padding slots of a slot-ordered A (never scatter targets).
template <class T>
__device__ __forceinline__ void zero_padding(T *__restrict__ Abase, const int *__restrict__ padfrom,
                                             int L, int Lc, int sl) {
  for (int t = __ldg(padfrom + sl) * Lc + sl; t < L * Lc; t += Lc) Abase[t] = T(0);
}

// float variant of the segment sum
template <int NV>
__device__ __forceinline__ void seg_sumf(float (&v)[NV], int Lc) {
  for (int off = Lc >> 1; off > 0; off >>= 1) {
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] += __shfl_xor_sync(kFull, v[q], off);
  }
}

// FP32 variant (slot-ordered A32).
__device__ __forceinline__ void seg_spmvf(const SchedWord *__restrict__ sch,
                                          int L, int Lc,
                                          const float *__restrict__ As,
                                          const float *__restrict__ gs,
                                          float *__restrict__ os) {
  spmv_slots<float>(sch, L, Lc, [&](int j) { return As[j * Lc]; }, gs, os);
}

// FP64 -> FP32 conversion, round to nearest even, entirely on the integer
// pipe (on this GPU a hardware F2F conversion occupies the FP64 pipe).  IEEE
// 754 rounding written from its definition: keep 23 of the 52 fraction bits
// and round on the 29 dropped bits, ties to even; a carry out of the fraction
// increments the exponent (and reaches infinity at the top of the range).
// Results below the FP32 normal range are flushed to a signed zero; Inf and
// NaN map to Inf and a quiet NaN.
__device__ __forceinline__ float d2f_rn(double v) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(v);
  const unsigned sign = (unsigned)(u >> 32) & 0x80000000u;
  const int ed = (int)((u >> 52) & 0x7ffull);
  const unsigned long long frac = u & 0xfffffffffffffull;
  const int ef = ed - 1023 + 127;
  unsigned m = (unsigned)(frac >> 29);
  const unsigned rem = (unsigned)(frac & 0x1fffffffull);
  m += (rem > 0x10000000u || (rem == 0x10000000u && (m & 1u))) ? 1u : 0u;
  unsigned bits = ((unsigned)ef << 23) + m;          // valid for 1 <= ef <= 254
  bits = (ef >= 255) ? 0x7f800000u : bits;            // overflow -> Inf
  bits = (ef <= 0) ? 0u : bits;                       // underflow -> 0
  bits = (ed == 0x7ff) ? (frac ? 0x7fc00000u : 0x7f800000u) : bits;
  return __uint_as_float(sign | bits);
}

// Exact FP32 -> FP64 widening on the integer pipe (FP32 subnormals, which
// d2f_rn never produces, are read as zero).
__device__ __forceinline__ double f2d_exact(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned ef = (b >> 23) & 0xffu;
  const unsigned long long sign = (unsigned long long)(b >> 31) << 63;
  const unsigned long long mant = (unsigned long long)(b & 0x7fffffu) << 29;
  unsigned long long u = sign | ((unsigned long long)(ef - 127 + 1023) << 52) | mant;
  u = (ef == 0u) ? sign : u;
  u = (ef == 0xffu) ? (sign | (0x7ffull << 52) | mant) : u;
  return __longlong_as_double((long long)u);
}

// x == 0 (either sign) on the bit pattern
__device__ __forceinline__ bool is_zero_bits(double v) {
  return ((unsigned long long)__double_as_longlong(v) << 1) == 0ull;
}

// 1/d in FP64 by Newton-Raphson iteration y <- y + y (1 - d y).  d = m 2^k
// with m in [1, 2) (m and k read from the bit pattern); an FP32
// rcp.approx of m (relative error about 2^-22) seeds STEPS Newton steps on m,
// each squaring the relative error (one step: about 2^-44; two: FP64
// rounding); the exponent of the result is then lowered by k on the bit
// pattern.  Only the 2*STEPS Newton FMAs use the FP64 pipe (a division costs
// about seven).  Zero gives Inf, Inf gives zero, NaN
// stays NaN; results that would leave the normal FP64 range (|d| above
// 2^1022 or below 2^-1022) are returned as zero or Inf.
template <int STEPS>
__device__ __forceinline__ double recip64n(double d) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(d);
  const unsigned long long sign = u & 0x8000000000000000ull;
  const int ed = (int)((u >> 52) & 0x7ffull);
  const unsigned long long frac = u & 0xfffffffffffffull;
  const double m = __longlong_as_double((long long)(frac | (1023ull << 52)));
  float yf;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(yf)
      : "f"(__uint_as_float(0x3f800000u | (unsigned)(frac >> 29))));
  double y = __longlong_as_double((long long)(((unsigned long long)(__float_as_uint(yf) & 0x7fffffu) << 29) |
                                              ((unsigned long long)(((__float_as_uint(yf) >> 23) & 0xffu) - 127 + 1023) << 52)));
#pragma unroll
  for (int s = 0; s < STEPS; ++s) {
    const double r = fma(-m, y, 1.0);
    y = fma(y, r, y);                     // 1/m in (0.5, 1]
  }
  const unsigned long long yu = (unsigned long long)__double_as_longlong(y);
  const int ey = (int)((yu >> 52) & 0x7ffull) - (ed - 1023);
  unsigned long long out = sign | ((unsigned long long)ey << 52) | (yu & 0xfffffffffffffull);
  out = (ey <= 0) ? sign : out;                                   // underflow
  out = (ey >= 0x7ff || ed == 0) ? (sign | (0x7ffull << 52)) : out;  // overflow, 1/0
  out = (ed == 0x7ff) ? (frac ? 0x7ff8000000000000ull : sign) : out;  // NaN, 1/Inf
  return __longlong_as_double((long long)out);
}

// Full-precision reciprocal (two Newton steps): the Jacobi preconditioner.
__device__ __forceinline__ double recip64(double d) { return recip64n<2>(d); }
// Scalars of the iteration (alpha, beta, omega): one step, relative error
// about 2^-44; x and r are updated with the same scalar, so they stay
// consistent and the true-residual test still decides convergence.
__device__ __forceinline__ double recip64s(double d) { return recip64n<1>(d); }

// Sum of v over the Lc lanes of each segment on the integer pipe.  Every
// term m 2^(e-1075) (53-bit integer m) is aligned to the segment's largest
// exponent as a signed 64-bit fixed-point number with 5 guard bits (room for
// 32 terms), the integers are summed exactly with xor shuffles, and the total
// is rounded once to FP64 (nearest, ties to even).  The error is at most one
// rounding plus 2^-57 of the largest term per term, every lane gets the same
// bits, and no FP64 instruction is issued.  Any NaN or Inf gives NaN; totals
// below the normal FP64 range flush to zero.
__device__ __forceinline__ double seg_sum_exact(double v, int Lc) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(v);
  const int e = (int)((u >> 52) & 0x7ffull);
  const unsigned long long frac = u & 0xfffffffffffffull;
  const unsigned long long m = e ? (frac | (1ull << 52)) : frac;
  const int ee = e ? e : 1;
  int emax = ee;
  for (int off = Lc >> 1; off > 0; off >>= 1) emax = max(emax, __shfl_xor_sync(kFull, emax, off));
  const int sh = emax - ee;
  long long f = sh >= 58 ? 0ll : (long long)((m << 5) >> sh);
  f = (u >> 63) ? -f : f;
  for (int off = Lc >> 1; off > 0; off >>= 1) f += __shfl_xor_sync(kFull, f, off);
  const unsigned long long neg = f < 0 ? 1ull : 0ull;
  const unsigned long long a = (unsigned long long)(f < 0 ? -f : f);
  const int lz = __clzll((long long)a);
  const unsigned long long an = a << (lz & 63);
  unsigned long long mant = an >> 11;
  const unsigned rem = (unsigned)(an & 0x7ffull);
  mant += (rem > 0x400u || (rem == 0x400u && (mant & 1ull))) ? 1ull : 0ull;
  int E = (63 - lz) + emax - 57;
  E += (mant >> 53) ? 1 : 0;                 // rounding carried into a new bit
  mant = (mant >> 53) ? (mant >> 1) : mant;
  unsigned long long out = (neg << 63) | ((unsigned long long)E << 52) | (mant & 0xfffffffffffffull);
  out = (E <= 0 || a == 0ull) ? (neg << 63) : out;            // zero / flush
  out = (E >= 0x7ff) ? ((neg << 63) | (0x7ffull << 52)) : out;  // overflow
  out = (emax == 0x7ff) ? 0x7ff8000000000000ull : out;         // NaN or Inf present
  return __longlong_as_double((long long)out);
}

// The same sum with the segment reductions done by full-warp redux.sync (one
// instruction per reduction, all lanes taking part): for each of the K =
// 32/Lc segments, the lanes of that segment contribute and the others add
// the neutral element.  The exponent maximum is reduced directly and the
// 64-bit fixed-point total as three 32-bit sums of its 20-bit digits (at
// most 32 lanes of 20-bit digits cannot overflow 32 bits), recombined
// exactly, so the result is bit-identical to seg_sum_exact.
template <int K>
__device__ __forceinline__ double seg_sum_exact_redux(double v) {
  constexpr int Lc = 32 / K;
  const int seg = (threadIdx.x & 31) / Lc;
  const unsigned long long u = (unsigned long long)__double_as_longlong(v);
  const int e = (int)((u >> 52) & 0x7ffull);
  const unsigned long long frac = u & 0xfffffffffffffull;
  const unsigned long long m = e ? (frac | (1ull << 52)) : frac;
  const int ee = e ? e : 1;
  int emax = 0;
#pragma unroll
  for (int s = 0; s < K; ++s) {
    const int r = (int)__reduce_max_sync(kFull, seg == s ? (unsigned)ee : 0u);
    emax = seg == s ? r : emax;
  }
  const int sh = emax - ee;
  long long f = sh >= 58 ? 0ll : (long long)((m << 5) >> sh);
  f = (u >> 63) ? -f : f;
  const unsigned d0 = (unsigned)(f & 0xfffffll);
  const unsigned d1 = (unsigned)((f >> 20) & 0xfffffll);
  const int d2 = (int)(f >> 40);
  unsigned s0 = 0, s1 = 0;
  int s2 = 0;
#pragma unroll
  for (int s = 0; s < K; ++s) {
    const bool mine = seg == s;
    const unsigned r0 = __reduce_add_sync(kFull, mine ? d0 : 0u);
    const unsigned r1 = __reduce_add_sync(kFull, mine ? d1 : 0u);
    const int r2 = __reduce_add_sync(kFull, mine ? d2 : 0);
    s0 = mine ? r0 : s0;
    s1 = mine ? r1 : s1;
    s2 = mine ? r2 : s2;
  }
  f = ((long long)s2 << 40) + ((long long)s1 << 20) + (long long)s0;
  const unsigned long long neg = f < 0 ? 1ull : 0ull;
  const unsigned long long a = (unsigned long long)(f < 0 ? -f : f);
  const int lz = __clzll((long long)a);
  const unsigned long long an = a << (lz & 63);
  unsigned long long mant = an >> 11;
  const unsigned rem = (unsigned)(an & 0x7ffull);
  mant += (rem > 0x400u || (rem == 0x400u && (mant & 1ull))) ? 1ull : 0ull;
  int E = (63 - lz) + emax - 57;
  E += (mant >> 53) ? 1 : 0;
  mant = (mant >> 53) ? (mant >> 1) : mant;
  unsigned long long out = (neg << 63) | ((unsigned long long)E << 52) | (mant & 0xfffffffffffffull);
  out = (E <= 0 || a == 0ull) ? (neg << 63) : out;
  out = (E >= 0x7ff) ? ((neg << 63) | (0x7ffull << 52)) : out;
  out = (emax == 0x7ff) ? 0x7ff8000000000000ull : out;
  return __longlong_as_double((long long)out);
}

// Exact segment sum.  With Lc known at compile time (LC > 0) and at most two
// cells per warp, the reductions run as full-warp redux.sync (one instruction
// each; a redux over part of a warp measured several times slower than
// shuffles); otherwise the shuffle form.  Both give the same bits.
template <int LC>
__device__ __forceinline__ double seg_sum_x(double v, int Lc) {
  if constexpr (LC >= 16) return seg_sum_exact_redux<32 / LC>(v);
  else return seg_sum_exact(v, Lc);
}

// A bounded wait ran out: raise the launch's time-out flag (device memory,
// read by the launch's last warp) and the host-mapped error word.
__device__ __forceinline__ void wait_timed_out(int *flag, int *err) {
  atomicExch(flag, 1);
  if (err) {
    *(volatile int *)err = 1;
    __threadfence_system();
  }
}

// Grid barrier of a cooperative launch, bounded in time: the CTA's threads
// meet, thread 0 publishes the CTA's writes and counts it in, then waits
// until the counter reaches target.  A wait longer than `limit` clocks (by
// default about a second; the CTAs of a cooperative launch are all resident,
// so a legitimate wait is microseconds) raises the time-out flags and goes on.
__device__ __forceinline__ void grid_barrier_bounded(unsigned *ctr, unsigned target,
                                                     int *flag, int *err, long long limit) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(ctr, 1u);
    const long long t0 = clock64();
    for (;;) {
      unsigned v;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(ctr) : "memory");
      if (v >= target) break;
      if (clock64() - t0 > limit) {
        wait_timed_out(flag, err);
        break;
      }
      __nanosleep(64);
    }
    __threadfence();
  }
  __syncthreads();
}

// In-launch difficulty ordering (run by every CTA of a cooperative solve
// launch before it solves; Args: WarpArgs or MixedArgs).  The estimate, the classes and the hardest-first
// order are those of the separate ordering pass: max_i |A_ii - 1| binned on
// half octaves, here over the sampled diagonal rows (or of |gamma_c|, see
// BY_GAMMA).  Each CTA classifies a contiguous share of the cells, counts them per class in shared memory and
// reserves its range inside each class with one global atomic per class;
// after a grid barrier it turns the class totals into class starts and
// writes its cells' order entries (cell + 1).  A warp that takes a group
// waits for the group's entries (written by whichever CTAs own those cells,
// all resident and past the barrier) and clears them once it has read them,
// so the order is all zero again for the next launch.
// sm: kOrdSmemBytes of this CTA's shared memory not yet in use.
// BY_GAMMA: classify by |gamma_c| instead (the fused assembly and Newton
// launches, whose matrices do not exist before a cell is assembled; gamma
// scales the off-identity part of A = I - gamma J, so it ranks the cells as
// the diagonal estimate does).
__device__ __forceinline__ const double *ord_gamma_of(const WarpArgs &a) { return a.gamma; }
__device__ __forceinline__ const double *ord_gamma_of(const MixedArgs &) { return nullptr; }
template <bool BY_GAMMA, class Args>
__device__ __forceinline__ void order_prologue(const Args &a, int *sm) {
  int *hist = sm;                       // per class: count, then class start
  int *base = sm + kOrdClasses;         // per class: this CTA's offset inside it
  unsigned long long *bkey = reinterpret_cast<unsigned long long *>(sm + 2 * kOrdClasses);
  // per cell of a pass: (estimate high word << 32 | sampled row), then its class word
  unsigned long long *key =
      reinterpret_cast<unsigned long long *>(reinterpret_cast<char *>(sm) + kOrdKeyOffset);
  unsigned *ctr = reinterpret_cast<unsigned *>(a.ord_ws + kOrdClasses);
  const int per = (a.cells + gridDim.x - 1) / gridDim.x;
  const int c0 = min(a.cells, (int)blockIdx.x * per), c1 = min(a.cells, c0 + per);
  const int nr = BY_GAMMA ? 1 : a.ord_nrows;
  // a share of one pass keeps its class words in shared memory
  const bool one_piece = c1 - c0 <= kOrdPiece;
  for (int i = threadIdx.x; i < kOrdClasses; i += blockDim.x) hist[i] = 0;
  if (threadIdx.x == 0) *bkey = 0ull;
  for (int p0 = c0; p0 < c1; p0 += kOrdPiece) {
    const int pc = min(kOrdPiece, c1 - p0);
    for (int i = threadIdx.x; i < pc; i += blockDim.x) key[i] = 0ull;
    __syncthreads();
    // the pass's sampled diagonal entries, flattened; each thread issues a
    // batch of independent loads before it folds them in
    const int m = pc * nr;
    for (int j0 = threadIdx.x; j0 < m; j0 += kOrdBatch * blockDim.x) {
      double v[kOrdBatch];
      int cl[kOrdBatch], q[kOrdBatch];
#pragma unroll
      for (int u = 0; u < kOrdBatch; ++u) {
        const int j = j0 + u * blockDim.x;
        cl[u] = j < m ? j / nr : -1;
        q[u] = j - cl[u] * nr;
        if (cl[u] >= 0)
          v[u] = BY_GAMMA ? __ldg(ord_gamma_of(a) + p0 + cl[u])
                          : __ldg(a.A + (size_t)(p0 + cl[u]) * a.nnz + __ldg(a.ord_rows + q[u]));
      }
#pragma unroll
      for (int u = 0; u < kOrdBatch; ++u)
        if (cl[u] >= 0)
          atomicMax(key + cl[u], (unsigned long long)(BY_GAMMA ? magnitude_hi(v[u])
                                                               : diag_departure_hi(v[u]))
                                         << 32 |
                                     (unsigned)q[u]);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < pc; i += blockDim.x) {
      const unsigned long long kk = key[i];
      const int k = difficulty_class((unsigned)(kk >> 32));
      const int w = k | atomicAdd(hist + k, 1) << 6;
      if (a.ord_hits) atomicMax(bkey, kk);
      if (one_piece) key[i] = (unsigned)w;
      else a.ord_cls[p0 + i] = w;
    }
    __syncthreads();
  }
  // where the CTA's hardest cell peaked (the host picks the rows to sample)
  if (a.ord_hits && threadIdx.x == 0 && c1 > c0) atomicAdd(a.ord_hits + (unsigned)*bkey, 1u);
  for (int k = threadIdx.x; k < kOrdClasses; k += blockDim.x)
    base[k] = hist[k] ? atomicAdd(a.ord_ws + k, hist[k]) : 0;
  grid_barrier_bounded(ctr, gridDim.x, a.ord_ws + kOrdFlag, a.ord_err, a.ord_wait);
  if (threadIdx.x < 32) {
    // exclusive prefix of the class totals, two classes per lane
    const int l = threadIdx.x;
    const int ta = __ldcg(a.ord_ws + 2 * l), tb = __ldcg(a.ord_ws + 2 * l + 1);
    int s = ta + tb;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(kFull, s, o);
      if (l >= o) s += t;
    }
    hist[2 * l] = s - ta - tb;
    hist[2 * l + 1] = s - tb;
  }
  __syncthreads();
  for (int c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
    const int w = one_piece ? (int)key[c - c0] : __ldcg(a.ord_cls + c);
    const int k = w & (kOrdClasses - 1);
    const int pos = hist[k] + base[k] + (w >> 6);
    if (pos < a.cells) __stcg(a.ord_out + pos, c + 1);  // in range unless the barrier timed out
  }
  __syncthreads();  // the warps' solve regions overlap the shared memory used here
}

// Wait, bounded in time as the barrier, until the in-launch ordering has
// written order entry *p.  The entry is the only datum passed, so a relaxed
// load suffices (an acquire would also invalidate the SM's L1 each time).
__device__ __forceinline__ void wait_order_entry(const int *p, int *flag, int *err,
                                                 long long limit) {
  const long long t0 = clock64();
  for (;;) {
    int v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    if (v != 0) return;
    if (clock64() - t0 > limit) {
      wait_timed_out(flag, err);
      return;
    }
    __nanosleep(32);
  }
}


// Next group of this warp in a launch with the dynamic queue (false when none
// is left).  An ordered launch (a.order set) first gives every warp one group
// of a stratified wave, or spreads the tickets over the order when there are
// fewer groups than warps (WarpArgs::ord_wave); `first` starts true.
template <class Args>
__device__ __forceinline__ bool take_group(const Args &a, int warp, int lane, bool &first,
                                           unsigned &g) {
  const bool strat = a.order && a.ord_stride == 0 && a.ord_wave > 0;
  if (first && strat) {
    first = false;
    const unsigned B = gridDim.x, b = blockIdx.x, w = (unsigned)warp;
    g = w * B + ((w & 1u) ? B - 1u - b : b);
    return true;
  }
  first = false;
  unsigned t = 0;
  if (lane == 0) t = atomicAdd(a.queue, 1u);
  t = __shfl_sync(kFull, t, 0);
  if (strat) t += (unsigned)a.ord_wave;
  if (t >= (unsigned)a.ngroups) return false;
  if (a.order && a.ord_stride && t < (unsigned)a.ord_wave)
    t = (unsigned)((unsigned long long)t * (unsigned)a.ord_stride % (unsigned)a.ord_wave);
  g = t;
  return true;
}

// In-launch ordering: lanes 0 .. k-1 wait for the order entries of group g's
// k cells; returns whether this lane owns one (to clear it after the solve).
template <class Args>
__device__ __forceinline__ bool await_order_entries(const Args &a, unsigned g, int k, int lane) {
  if (!a.ord_ws) return false;
  const int p = (int)g * k + lane;
  const bool mine = lane < k && p < a.cells;
  if (mine) wait_order_entry(a.order + p, a.ord_ws + kOrdFlag, a.ord_err, a.ord_wait);
  __syncwarp();
  return mine;
}

// End of a launch with the dynamic queue, called by every lane of every
// warp once it has no group left: the last warp to finish (every other warp
// has taken its last group before counting itself done, so every CTA is past
// its ordering prologue) resets the queue pair and, after an in-launch
// ordering, the ordering's workspace, so both are ready for the next launch
// in stream order.  If a wait of the ordering ran out, the order may have
// sent some cells to no warp and others to two: that warp then marks every
// cell of the launch CAMP_CELL_INVALID (status, when given) with a NaN
// residual and clears the order entries the launch left set.
template <class Args>
__device__ __forceinline__ void finish_queue(const Args &a, bool ordered, int warps_total,
                                             int lane) {
  unsigned last = 0;
  if (lane == 0) {
    __threadfence();
    last = atomicAdd(a.queue + 1, 1u) == (unsigned)warps_total - 1u ? 1u : 0u;
  }
  last = __shfl_sync(kFull, last, 0);
  if (!last) return;
  __threadfence();
  if (ordered && a.ord_ws && __ldcg(a.ord_ws + kOrdFlag) != 0) {
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    for (int c = lane; c < a.cells; c += 32) {
      a.ord_out[c] = 0;
      a.resid[c] = nan;
      if (a.status) a.status[c] = CAMP_CELL_INVALID;
    }
  }
  if (lane == 0) {
    atomicExch(a.queue, 0u);
    atomicExch(a.queue + 1, 0u);
    if (ordered && a.ord_ws)
      for (int i = 0; i < kOrdWords; ++i) atomicExch(a.ord_ws + i, 0);
  }
}

}  // namespace camp
