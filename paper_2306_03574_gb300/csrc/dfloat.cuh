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

struct dfl {
  float hi, lo;
  __host__ __device__ __forceinline__ dfl() : hi(0.f), lo(0.f) {}
  __host__ __device__ __forceinline__ dfl(float h, float l) : hi(h), lo(l) {}
  // nearest double-float to x (hi = x rounded to FP32, lo = the remainder rounded)
  __host__ __device__ __forceinline__ dfl(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
  __host__ __device__ __forceinline__ explicit operator double() const { return (double)hi + (double)lo; }
};

__host__ __device__ __forceinline__ dfl fast_two_sum(float a, float b) {
  const float s = a + b;
  const float t = b - (s - a);
  return dfl(s, t);
}

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
