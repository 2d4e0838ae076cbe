// Double-float ("float-float") arithmetic: a value is the unevaluated sum hi + lo of
// two FP32 numbers with |lo| <= ulp(hi)/2, giving about 48 significant bits on the FP32
// pipes.  On GB300 the FP32 pipes issue 64 times more operations per clock than the
// FP64 pipe, so a transform written in double-float runs several times faster than in
// FP64 at an accuracy of a few units of 2^-48 relative to the data's norm.
//
// Building blocks (error-free transformations, round-to-nearest FP32, no reassociation;
// the build never passes --use_fast_math):
//   Fast2Sum (Dekker 1971): s = a + b, t = b - (s - a) is exact when |a| >= |b|;
//   2Sum (Knuth, TAOCP vol. 2): the same without the ordering condition, six operations;
//   2Prod with FMA: p = a b, e = fma(a, b, -p) is exact.
// Double-word addition is the "sloppy" variant (2Sum of the high parts, the low parts
// added and folded in by Fast2Sum); its error is bounded relative to |x| + |y|, which
// is what the norm-wise error analysis of an FFT needs.  Double-word multiplication
// uses the FMA-based product of the high parts plus the two cross terms (the lo*lo
// term is below the format's precision).  See Joldes, Muller and Popescu, "Tight and
// rigorous error bounds for basic building blocks of double-word arithmetic", ACM TOMS
// 44 (2017), for the analysis of these algorithms.
#pragma once

#include <cuda_runtime.h>

namespace aao {

struct dfl;
__host__ __device__ __forceinline__ dfl split_double(double x);
__host__ __device__ __forceinline__ double join_double(float hi, float lo);

struct dfl {
  float hi, lo;
  __host__ __device__ __forceinline__ dfl() : hi(0.f), lo(0.f) {}
  __host__ __device__ __forceinline__ dfl(float h, float l) : hi(h), lo(l) {}
  // a double-float within 2^-48 relative of x (hi + lo, |lo| <= ulp(hi)/2)
  __host__ __device__ __forceinline__ dfl(double x);
  __host__ __device__ __forceinline__ explicit operator double() const { return join_double(hi, lo); }
};

__host__ __device__ __forceinline__ dfl fast_two_sum(float a, float b) {
  const float s = a + b;
  const float t = b - (s - a);
  return dfl(s, t);
}

// Conversions between double and double-float.  Device code assembles the FP32 parts
// from the bit fields of the double with integer and FP32 operations, because GB300's
// narrow FP64 pipe also executes the FP64 <-> FP32 conversion instructions: with them a
// double-float transform spends half its time converting its input and output.
//   split: x = (-1)^s 2^E 1.m (52-bit m).  a = x with m truncated to 23 bits (an FP32
//   number, exact); the remainder x - a = (-1)^s r 2^(E-52) with the 29-bit integer
//   r = low bits of m, written as (r >> 6) 2^(E-46) + (r & 63) 2^(E-52): both integers
//   convert exactly by the 2^23 bias trick, the powers of two are exact FP32 scalings,
//   and one FMA rounds their sum; Fast2Sum renormalises (a, remainder).  Zero (and the
//   subnormal doubles) give 0; other exponents outside [-70, 120] take the conversion
//   instructions.
//   join: each FP32 part becomes a double by re-biasing its exponent and shifting its
//   mantissa (exact), then one FP64 addition.
__host__ __device__ __forceinline__ dfl split_double(double x) {
#ifdef __CUDA_ARCH__
  const unsigned hw = (unsigned)__double2hiint(x);
  const unsigned lw = (unsigned)__double2loint(x);
  const int E = (int)((hw >> 20) & 0x7FFu) - 1023;
  if (E == -1023) return dfl();  // zero (and subnormal doubles, far below the FP32 range)
  if (E < -70 || E > 120) {
    const float h = __double2float_rn(x);
    return dfl(h, __double2float_rn(x - (double)h));
  }
  const unsigned sign = hw & 0x80000000u;
  const float a = __uint_as_float(sign | ((unsigned)(E + 127) << 23) | ((hw & 0xFFFFFu) << 3) | (lw >> 29));
  const unsigned r = lw & 0x1FFFFFFFu;
  const float rh = __uint_as_float(0x4B000000u | (r >> 6)) - 8388608.f;
  const float rl = __uint_as_float(0x4B000000u | (r & 63u)) - 8388608.f;
  const float s1 = __uint_as_float((unsigned)(E - 46 + 127) << 23);
  const float s0 = __uint_as_float((unsigned)(E - 52 + 127) << 23);
  float l = fmaf(rh, s1, rl * s0);
  if (sign) l = -l;
  return fast_two_sum(a, l);
#else
  const float h = (float)x;
  return dfl(h, (float)(x - (double)h));
#endif
}

#ifdef __CUDA_ARCH__
__device__ __forceinline__ double float_to_double_bits(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xFFu;
  if ((u & 0x7FFFFFFFu) == 0u) return __hiloint2double((int)(u & 0x80000000u), 0);
  if (e == 0u || e == 0xFFu) return (double)f;  // subnormal, inf, nan
  const unsigned hw = (u & 0x80000000u) | ((e + 896u) << 20) | ((u & 0x7FFFFFu) >> 3);
  return __hiloint2double((int)hw, (int)((u & 7u) << 29));
}
#endif

__host__ __device__ __forceinline__ double join_double(float hi, float lo) {
#ifdef __CUDA_ARCH__
  return float_to_double_bits(hi) + float_to_double_bits(lo);
#else
  return (double)hi + (double)lo;
#endif
}

__host__ __device__ __forceinline__ dfl::dfl(double x) : hi(0.f), lo(0.f) { *this = split_double(x); }

__host__ __device__ __forceinline__ dfl two_sum(float a, float b) {
  const float s = a + b;
  const float ap = s - b;
  const float bp = s - ap;
  const float t = (a - ap) + (b - bp);
  return dfl(s, t);
}

__host__ __device__ __forceinline__ dfl operator+(dfl x, dfl y) {
  const dfl s = two_sum(x.hi, y.hi);
  const float v = x.lo + y.lo;
  return fast_two_sum(s.hi, s.lo + v);
}

__host__ __device__ __forceinline__ dfl operator-(dfl x) { return dfl(-x.hi, -x.lo); }
__host__ __device__ __forceinline__ dfl operator-(dfl x, dfl y) { return x + (-y); }

__host__ __device__ __forceinline__ dfl operator*(dfl x, dfl y) {
  const float p = x.hi * y.hi;
  float e = fmaf(x.hi, y.hi, -p);
  e = fmaf(x.hi, y.lo, e);
  e = fmaf(x.lo, y.hi, e);
  return fast_two_sum(p, e);
}

__host__ __device__ __forceinline__ dfl& operator*=(dfl& x, dfl y) { return x = x * y; }
__host__ __device__ __forceinline__ dfl& operator+=(dfl& x, dfl y) { return x = x + y; }

// a*b + c in the type at hand: one FMA for double and float, two rounded double-word
// operations for dfl.  (Deliberately not named fma: an aao::fma overload would hide
// the global double and float fma from unqualified calls inside the namespace.)
__host__ __device__ __forceinline__ double fmadd(double a, double b, double c) { return ::fma(a, b, c); }
__host__ __device__ __forceinline__ float fmadd(float a, float b, float c) { return ::fmaf(a, b, c); }
__host__ __device__ __forceinline__ dfl fmadd(dfl a, dfl b, dfl c) { return a * b + c; }

struct dfl2 {
  dfl x, y;
};

__host__ __device__ __forceinline__ dfl2 cadd(dfl2 a, dfl2 b) { return dfl2{a.x + b.x, a.y + b.y}; }
__host__ __device__ __forceinline__ dfl2 csub(dfl2 a, dfl2 b) { return dfl2{a.x - b.x, a.y - b.y}; }
__host__ __device__ __forceinline__ dfl2 cmul(dfl2 a, dfl2 b) {
  return dfl2{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
__host__ __device__ __forceinline__ dfl2 cmulc(dfl2 a, dfl2 b) {
  return dfl2{a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y};
}

}  // namespace aao
