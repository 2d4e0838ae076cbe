// Conversions between FP64 and FP32 by integer operations on the IEEE bit fields.
//
// On GB300 the cvt instructions between double and float execute on the FP64 pipe,
// which issues 2 operations per clock per SM; a kernel that computes in FP32 on FP64
// vectors converts twice per value, and those conversions alone can keep the FP64 pipe
// busy for a large part of the kernel.  The functions below use a few integer
// operations instead (the exponent is re-biased by 1023 - 127 = 896 and the mantissa
// shifted); the FP32 pipes and the integer units have throughput to spare.
#pragma once

namespace aao {

// double -> float by integer operations on the bit fields: rounds to nearest (ties away
// from zero); |x| < 2^-126 gives a signed zero; valid for |x| < 2^128.
__device__ __forceinline__ float d2f_bits(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const unsigned long long a = u & 0x7FFFFFFFFFFFFFFFull;
  const unsigned sign = (unsigned)(u >> 32) & 0x80000000u;
  if (a < 0x3810000000000000ull) return __uint_as_float(sign);
  // re-bias the exponent by 1023 - 127 = 896, add half a unit of the 29 dropped bits
  const unsigned f = (unsigned)((a - 0x3800000000000000ull + 0x10000000ull) >> 29);
  return __uint_as_float(f | sign);
}

// float -> double by integer operations (exact for normal numbers; subnormals give a
// signed zero; finite inputs only)
__device__ __forceinline__ double f2d_bits(float v) {
  const unsigned f = __float_as_uint(v);
  const unsigned a = f & 0x7FFFFFFFu;
  const unsigned sign = f & 0x80000000u;
  if (a < 0x00800000u) return __hiloint2double((int)sign, 0);
  return __hiloint2double((int)(((a >> 3) + 0x38000000u) | sign), (int)(a << 29));
}

template <bool ICVT>
__device__ __forceinline__ float to_f32(double x) {
  if constexpr (ICVT) return d2f_bits(x);
  else return (float)x;
}
template <bool ICVT>
__device__ __forceinline__ double to_f64(float x) {
  if constexpr (ICVT) return f2d_bits(x);
  else return (double)x;
}


// load / store conversion of a kernel that computes in R on vectors of TIO.  CVM (FP32
// on FP64 vectors only): bit 0 converts the loads, bit 1 the stores by integer
// operations; the others stay cvt instructions.  Splitting them spreads the conversions
// over the FP64 pipe and the integer units.
template <typename R, typename TIO, int CVM>
struct Cvt {
  static __device__ __forceinline__ R load(TIO x) { return R(x); }
  static __device__ __forceinline__ TIO store(R x) { return TIO(x); }
};
template <int CVM>
struct Cvt<float, double, CVM> {
  static __device__ __forceinline__ float load(double x) { return to_f32<(CVM & 1) != 0>(x); }
  static __device__ __forceinline__ double store(float x) { return to_f64<(CVM & 2) != 0>(x); }
};

}  // namespace aao
