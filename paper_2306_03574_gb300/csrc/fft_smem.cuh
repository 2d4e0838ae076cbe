// Batched complex FFT of length L executed by a whole CTA on sequences held in
// shared memory: Stockham autosort, radix-4 stages and one radix-2 stage when
// log2(L) is odd, natural order in and out, forward = exp(-2 pi i jk/L),
// inverse = exp(+2 pi i jk/L), both unnormalised.
//
// Each stage first loads every value it needs into registers, synchronises,
// then writes the butterfly outputs back in place, so a single buffer serves
// all stages.
//
// Two shared-memory layouts of the batch (template parameter LAY):
//   0  sequence-major: element x of sequence q at q*L + x; the threads of a warp
//      walk x.  Stockham writes of stride RX then fall on one bank (a 32-way
//      conflict for radix 16), which costs little only where the FP64 pipe, not
//      shared memory, is the bottleneck.
//   1  interleaved and padded: element x of sequence q at NS*pad(x) + q with
//      pad(x) = x + floor(x/16); the threads of a warp walk q first.  Reads,
//      loads and stores touch consecutive words, the strided Stockham writes
//      are spread over all banks by the one-in-16 padding, and the lanes of a
//      warp share their twiddle factors (broadcast reads).
#pragma once

#include "aao_internal.cuh"

namespace aao {

template <int L, int NS, int LAY>
struct SLay {
  static constexpr int size = LAY ? NS * (L + L / 16) : NS * L;  // elements of the batch buffer
  static __device__ __forceinline__ int at(int q, int x) {
    return LAY ? NS * (x + (x >> 4)) + q : q * L + x;
  }
  // at(q, x + c) - at(q, x), valid when (x mod 16) + (c mod 16) < 16 (no carry into x/16)
  static constexpr int off(int c) { return LAY ? NS * (c + (c >> 4)) : c; }
  // task -> (sequence q, index j) for a pass with Q tasks per sequence
  template <int Q>
  static __device__ __forceinline__ void split(int task, int& q, int& j) {
    if (LAY) { q = task % NS; j = task / NS; }
    else { q = task / Q; j = task % Q; }
  }
};

template <int L>
struct Log2 {
  static constexpr int value = (L <= 1) ? 0 : 1 + Log2<L / 2>::value;
};
template <>
struct Log2<1> {
  static constexpr int value = 0;
};

// w -> w or conj(w)
template <bool INV, typename C>
AAO_HD C twid(C w) {
  if (INV) w.y = -w.y;
  return w;
}

// in-register 4-point DFT
template <bool INV, typename C>
AAO_HD void dft4(C& v0, C& v1, C& v2, C& v3) {
  C a0 = cadd(v0, v2), a1 = csub(v0, v2), a2 = cadd(v1, v3), a3 = csub(v1, v3);
  v0 = cadd(a0, a2);
  v2 = csub(a0, a2);
  if (!INV) {  // a1 -/+ i a3
    v1.x = a1.x + a3.y; v1.y = a1.y - a3.x;
    v3.x = a1.x - a3.y; v3.y = a1.y + a3.x;
  } else {
    v1.x = a1.x - a3.y; v1.y = a1.y + a3.x;
    v3.x = a1.x + a3.y; v3.y = a1.y - a3.x;
  }
}

// Forward 4-point DFT of (s0 v0, s1 v1, s2 v2, s3 v3) for real s_r: the products of
// the first butterflies' second operands are folded into multiply-adds (three
// operations per component pair instead of four).
template <typename C, typename R>
AAO_HD void dft4_scaled_fwd(C& v0, C& v1, C& v2, C& v3, R s0, R s1, R s2, R s3) {
  C p, q, a0, a1, a2, a3;
  p.x = v0.x * s0; p.y = v0.y * s0;
  q.x = v1.x * s1; q.y = v1.y * s1;
  a0.x = fmadd(s2, v2.x, p.x);  a0.y = fmadd(s2, v2.y, p.y);
  a1.x = fmadd(-s2, v2.x, p.x); a1.y = fmadd(-s2, v2.y, p.y);
  a2.x = fmadd(s3, v3.x, q.x);  a2.y = fmadd(s3, v3.y, q.y);
  a3.x = fmadd(-s3, v3.x, q.x); a3.y = fmadd(-s3, v3.y, q.y);
  v0 = cadd(a0, a2);
  v2 = csub(a0, a2);
  v1.x = a1.x + a3.y; v1.y = a1.y - a3.x;  // a1 - i a3
  v3.x = a1.x - a3.y; v3.y = a1.y + a3.x;  // a1 + i a3
}

// ---------------------------------------------------------------------------
// Higher radices: in-register 8- and 16-point DFTs and a generic radix-RX
// Stockham stage.  Fewer stages mean fewer shared-memory round trips and
// barriers; the internal twiddles of the 16-point DFT are the constants
// exp(-+ 2 pi i m / 16).
// ---------------------------------------------------------------------------

// v * exp(-+ 2 pi i m / 16) for the constant m (INV: the conjugate root)
// A compile-time constant in the arithmetic type R (for double-float the split is
// written out so that it folds at compile time instead of converting at run time).
template <typename R> AAO_HD R real_const(double x) { return R(x); }
template <> AAO_HD dfl real_const<dfl>(double x) { return dfl((float)x, (float)(x - (double)(float)x)); }

template <int M, bool INV, typename C>
AAO_HD C w16(C v) {
  using R = decltype(v.x);
  constexpr double c1 = 0.92387953251128675613;  // cos(pi/8)
  constexpr double s1 = 0.38268343236508977173;  // sin(pi/8)
  constexpr double h = 0.70710678118654752440;   // sqrt(2)/2
  constexpr int m = M & 15;
  if constexpr (m == 0) {
    return v;
  } else if constexpr (m == 4) {
    C o;
    if (!INV) { o.x = v.y; o.y = -v.x; } else { o.x = -v.y; o.y = v.x; }
    return o;
  } else if constexpr (m == 8) {
    C o; o.x = -v.x; o.y = -v.y;
    return o;
  } else {
    // exp(-2 pi i m/16) = cos - i sin
    constexpr double cr = m == 1 ? c1 : m == 2 ? h : m == 3 ? s1 : m == 5 ? -s1 : m == 6 ? -h : m == 7 ? -c1 : -c1;
    constexpr double ci0 = m == 1 ? -s1 : m == 2 ? -h : m == 3 ? -c1 : m == 5 ? -c1 : m == 6 ? -h : m == 7 ? -s1 : s1;
    constexpr double ci = INV ? -ci0 : ci0;
    static_assert(m == 1 || m == 2 || m == 3 || m == 5 || m == 6 || m == 7 || m == 9, "twiddle index");
    C w; w.x = real_const<R>(cr); w.y = real_const<R>(ci);
    return cmul(v, w);
  }
}

template <bool INV, typename C>
AAO_HD void dft8(C* v) {
  // radix-2 over even/odd inputs: X_k = E_k + W8^k O_k, X_{k+4} = E_k - W8^k O_k
  C e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  C o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4<INV>(e0, e1, e2, e3);
  dft4<INV>(o0, o1, o2, o3);
  o1 = w16<2, INV>(o1);
  o2 = w16<4, INV>(o2);
  o3 = w16<6, INV>(o3);
  v[0] = cadd(e0, o0); v[4] = csub(e0, o0);
  v[1] = cadd(e1, o1); v[5] = csub(e1, o1);
  v[2] = cadd(e2, o2); v[6] = csub(e2, o2);
  v[3] = cadd(e3, o3); v[7] = csub(e3, o3);
}

template <bool INV, typename C>
AAO_HD void dft16(C* v) {
  // 16 = 4 x 4: DFT4 over n1 (stride 4) for each n2, twiddle W16^{n2 k1}, DFT4 over n2;
  // X[k1 + 4 k2] = sum_n2 W4^{n2 k2} W16^{n2 k1} sum_n1 x[4 n1 + n2] W4^{n1 k1}
  C a[16];
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) {
    C x0 = v[n2], x1 = v[4 + n2], x2 = v[8 + n2], x3 = v[12 + n2];
    dft4<INV>(x0, x1, x2, x3);
    a[4 * n2 + 0] = x0; a[4 * n2 + 1] = x1; a[4 * n2 + 2] = x2; a[4 * n2 + 3] = x3;
  }
  a[5] = w16<1, INV>(a[5]);   a[6] = w16<2, INV>(a[6]);   a[7] = w16<3, INV>(a[7]);
  a[9] = w16<2, INV>(a[9]);   a[10] = w16<4, INV>(a[10]); a[11] = w16<6, INV>(a[11]);
  a[13] = w16<3, INV>(a[13]); a[14] = w16<6, INV>(a[14]); a[15] = w16<9, INV>(a[15]);
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    C y0 = a[k1], y1 = a[4 + k1], y2 = a[8 + k1], y3 = a[12 + k1];
    dft4<INV>(y0, y1, y2, y3);
    v[k1] = y0; v[k1 + 4] = y1; v[k1 + 8] = y2; v[k1 + 12] = y3;
  }
}

// Forward 16-point DFT (same 4 x 4 split as dft16) with the internal twiddles folded
// into fused multiply-adds.  In each column k1 of the second 4-point DFTs the
// non-trivial twiddles share one real factor: W^2 and W^6 are sqrt(2)/2 times
// (1 - i) and (-1 - i); W^1, W^3 and W^9 are cos(pi/8) times (1 - i t), (t - i) and
// (-1 + i t), t = tan(pi/8).  The short factors cost additions or one multiply-add
// each, and the common factor is applied by the multiply-adds that form the outputs
// instead of by separate products: 144 real operations instead of 160.
// With SCALED, the input element r is first multiplied by the real factor sc[r] (the
// diagonal scaling that precedes a transform), folded into the first butterflies.
template <bool SCALED = false, typename C, typename R = decltype(C::x)>
AAO_HD void dft16_fwd_fma(C* v, const R* sc = nullptr) {
  const R h = R(0.70710678118654752440);  // sqrt(2)/2
  const R c = R(0.92387953251128675613);  // cos(pi/8)
  const R t = R(0.41421356237309504880);  // tan(pi/8) = sqrt(2) - 1
  C a[16];
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) {
    C x0 = v[n2], x1 = v[4 + n2], x2 = v[8 + n2], x3 = v[12 + n2];
    if constexpr (SCALED) dft4_scaled_fwd(x0, x1, x2, x3, sc[n2], sc[4 + n2], sc[8 + n2], sc[12 + n2]);
    else dft4<false>(x0, x1, x2, x3);
    a[4 * n2 + 0] = x0; a[4 * n2 + 1] = x1; a[4 * n2 + 2] = x2; a[4 * n2 + 3] = x3;
  }
  {  // k1 = 0: no twiddles
    C y0 = a[0], y1 = a[4], y2 = a[8], y3 = a[12];
    dft4<false>(y0, y1, y2, y3);
    v[0] = y0; v[4] = y1; v[8] = y2; v[12] = y3;
  }
  {  // k1 = 2: (a2, a6 W^2, a10 W^4, a14 W^6), a10 W^4 = -i a10, a6 W^2 = h p, a14 W^6 = h r
    const C b0 = a[2], b2 = a[10], q6 = a[6], q14 = a[14];
    C e0, e1;
    e0.x = b0.x + b2.y; e0.y = b0.y - b2.x;
    e1.x = b0.x - b2.y; e1.y = b0.y + b2.x;
    const R px = q6.x + q6.y, py = q6.y - q6.x;
    const R rx = q14.y - q14.x, ry = -q14.x - q14.y;
    const R sx = px + rx, sy = py + ry, dx = px - rx, dy = py - ry;
    v[2].x = fmadd(h, sx, e0.x);   v[2].y = fmadd(h, sy, e0.y);     // e0 + h s
    v[10].x = fmadd(-h, sx, e0.x); v[10].y = fmadd(-h, sy, e0.y);   // e0 - h s
    v[6].x = fmadd(h, dy, e1.x);   v[6].y = fmadd(-h, dx, e1.y);    // e1 - i h d
    v[14].x = fmadd(-h, dy, e1.x); v[14].y = fmadd(h, dx, e1.y);    // e1 + i h d
  }
  {  // k1 = 1: (a1, a5 W^1, a9 W^2, a13 W^3); a5 W^1 +- a13 W^3 = c (o0 | o1)
    const C b0 = a[1], q9 = a[9], q5 = a[5], q13 = a[13];
    const R px = q9.x + q9.y, py = q9.y - q9.x;
    C e0, e1;
    e0.x = fmadd(h, px, b0.x);  e0.y = fmadd(h, py, b0.y);
    e1.x = fmadd(-h, px, b0.x); e1.y = fmadd(-h, py, b0.y);
    const R P = q5.x + q13.y, Q = q5.y + q13.x, Rr = q5.y - q13.x, S = q5.x - q13.y;
    const R o0x = fmadd(t, Q, P), o0y = fmadd(-t, S, Rr);
    const R o1x = fmadd(t, Rr, S), o1y = fmadd(-t, P, Q);
    v[1].x = fmadd(c, o0x, e0.x);   v[1].y = fmadd(c, o0y, e0.y);
    v[9].x = fmadd(-c, o0x, e0.x);  v[9].y = fmadd(-c, o0y, e0.y);
    v[5].x = fmadd(c, o1y, e1.x);   v[5].y = fmadd(-c, o1x, e1.y);
    v[13].x = fmadd(-c, o1y, e1.x); v[13].y = fmadd(c, o1x, e1.y);
  }
  {  // k1 = 3: (a3, a7 W^3, a11 W^6, a15 W^9); a7 W^3 +- a15 W^9 = c (o0 | o1)
    const C b0 = a[3], q11 = a[11], q7 = a[7], q15 = a[15];
    const R rx = q11.y - q11.x, ry = -q11.x - q11.y;
    C e0, e1;
    e0.x = fmadd(h, rx, b0.x);  e0.y = fmadd(h, ry, b0.y);
    e1.x = fmadd(-h, rx, b0.x); e1.y = fmadd(-h, ry, b0.y);
    const R P = q7.y - q15.x, Q = q7.x - q15.y, Rr = q7.x + q15.y, S = q7.y + q15.x;
    const R o0x = fmadd(t, Q, P), o0y = fmadd(t, S, -Rr);
    const R o1x = fmadd(t, Rr, S), o1y = fmadd(t, P, -Q);
    v[3].x = fmadd(c, o0x, e0.x);   v[3].y = fmadd(c, o0y, e0.y);
    v[11].x = fmadd(-c, o0x, e0.x); v[11].y = fmadd(-c, o0y, e0.y);
    v[7].x = fmadd(c, o1y, e1.x);   v[7].y = fmadd(-c, o1x, e1.y);
    v[15].x = fmadd(-c, o1y, e1.x); v[15].y = fmadd(c, o1x, e1.y);
  }
}

// The inverse through the forward transform: with swap(a + ib) = b + ia,
// IDFT(x) = swap(DFT(swap(x))); the swaps are register renames.
template <bool INV, typename C>
AAO_HD void dft16_fma(C* v) {
  if constexpr (INV) {
#pragma unroll
    for (int i = 0; i < 16; ++i) { const auto r = v[i].x; v[i].x = v[i].y; v[i].y = r; }
  }
  dft16_fwd_fma(v);
  if constexpr (INV) {
#pragma unroll
    for (int i = 0; i < 16; ++i) { const auto r = v[i].x; v[i].x = v[i].y; v[i].y = r; }
  }
}

// Native fused multiply-add: the folded 16-point DFT is shorter.  In double-float
// arithmetic a multiply-add is a product plus a sum, so there the folded form would
// add products and the plain one is kept.
template <typename C> struct FoldedDft16 { static constexpr bool value = true; };
template <> struct FoldedDft16<dfl2> { static constexpr bool value = false; };

template <int RX, bool INV, typename C>
AAO_HD void dft_r(C* v) {
  if constexpr (RX == 2) { C a = v[0]; v[0] = cadd(a, v[1]); v[1] = csub(a, v[1]); }
  else if constexpr (RX == 4) dft4<INV>(v[0], v[1], v[2], v[3]);
  else if constexpr (RX == 8) dft8<INV>(v);
  else if constexpr (FoldedDft16<C>::value) dft16_fma<INV>(v);
  else dft16<INV>(v);
}

// Forward radix-RX DFT (RX = 4 or 16) of the inputs scaled by real factors sc[r].
template <int RX, typename C, typename R>
AAO_HD void dft_r_scaled(C* v, const R* sc) {
  static_assert(RX == 4 || RX == 16, "scaled first stages are radix 4 or 16");
  if constexpr (FoldedDft16<C>::value) {
    if constexpr (RX == 4) dft4_scaled_fwd(v[0], v[1], v[2], v[3], sc[0], sc[1], sc[2], sc[3]);
    else dft16_fwd_fma<true>(v, sc);
  } else {  // double-float: a multiply-add is no cheaper than a product and a sum
#pragma unroll
    for (int r = 0; r < RX; ++r) { v[r].x = v[r].x * sc[r]; v[r].y = v[r].y * sc[r]; }
    dft_r<RX, false>(v);
  }
}

// One radix-RX Stockham stage with span LS (sub-transforms of length LS done):
// task j in [0, L/RX), k = j mod LS, v_r = x[j + r L/RX], v_r *= w^{r k L/(RX LS)},
// DFT_RX, y[(j - k) RX + k + r LS] = v_r.  Every thread computes one base index for
// its reads and one for its writes; the RX elements sit at compile-time offsets from
// them (in the padded layout the offsets hold because no element of a group crosses
// a 16-element padding boundary relative to its base: see the static_assert).
template <int L, int NS, int NT, int RX, bool INV, int LAY, int LS, typename C>
__device__ __forceinline__ void fft_stage_body(C* buf, const C* tw) {
  using Y = SLay<L, NS, LAY>;
  constexpr int Q = L / RX;
  constexpr int TASKS = NS * Q;
  static_assert(TASKS % NT == 0, "radix tasks must divide evenly among threads");
  static_assert(LS <= Q && (Q % 16 == 0 || 16 % Q == 0), "read offsets");
  static_assert(LS % 16 == 0 || RX * LS <= 16, "write offsets");
  constexpr int TPT = TASKS / NT;
  C v[TPT][RX];
#pragma unroll
  for (int t = 0; t < TPT; ++t) {
    int q, j;
    Y::template split<Q>(threadIdx.x + t * NT, q, j);
    const C* p = buf + Y::at(q, j);
#pragma unroll
    for (int r = 0; r < RX; ++r) v[t][r] = p[Y::off(r * Q)];
  }
  __syncthreads();
#pragma unroll
  for (int t = 0; t < TPT; ++t) {
    int q, j;
    Y::template split<Q>(threadIdx.x + t * NT, q, j);
    const int k = j & (LS - 1);
    if constexpr (LS > 1) {
      const int step = (Q / LS) * k;
#pragma unroll
      for (int r = 1; r < RX; ++r) v[t][r] = cmul(v[t][r], twid<INV>(tw[r * step]));
    }
    dft_r<RX, INV>(v[t]);
    C* o = buf + Y::at(q, (j - k) * RX + k);
#pragma unroll
    for (int r = 0; r < RX; ++r) o[Y::off(r * LS)] = v[t][r];
  }
  __syncthreads();
}

// Double-float stages are called rather than inlined: one radix-16 stage in
// double-word arithmetic is several thousand instructions, and inlining the four
// transforms of the time pipeline (and both passes of a DST) would overflow the
// instruction cache.  The call passes two pointers; everything else stays in the stage.
template <typename C> struct StageCalled { static constexpr bool value = false; };
template <> struct StageCalled<dfl2> { static constexpr bool value = true; };

template <int L, int NS, int NT, int RX, bool INV, int LAY, int LS, typename C>
__device__ __noinline__ void fft_stage_call(C* buf, const C* tw) {
  fft_stage_body<L, NS, NT, RX, INV, LAY, LS>(buf, tw);
}

template <int L, int NS, int NT, int RX, bool INV, int LAY, int LS, typename C>
__device__ __forceinline__ void fft_stage_r(C* buf, const C* tw) {
  if constexpr (StageCalled<C>::value) fft_stage_call<L, NS, NT, RX, INV, LAY, LS>(buf, tw);
  else fft_stage_body<L, NS, NT, RX, INV, LAY, LS>(buf, tw);
}

// First stage (span 1, so no twiddles) of a forward transform whose input element x
// is multiplied by the real factor sc[x] first: the diagonal scaling that precedes the
// transform costs no pass of its own.
template <int L, int NS, int NT, int RX, int LAY, typename C, typename R>
__device__ __forceinline__ void fft_stage1_scaled_body(C* buf, const R* sc) {
  using Y = SLay<L, NS, LAY>;
  constexpr int Q = L / RX;
  constexpr int TASKS = NS * Q;
  static_assert(TASKS % NT == 0, "radix tasks must divide evenly among threads");
  static_assert(Q % 16 == 0 || 16 % Q == 0, "read offsets");
  static_assert(RX <= 16, "write offsets");
  constexpr int TPT = TASKS / NT;
  C v[TPT][RX];
#pragma unroll
  for (int t = 0; t < TPT; ++t) {
    int q, j;
    Y::template split<Q>(threadIdx.x + t * NT, q, j);
    const C* p = buf + Y::at(q, j);
#pragma unroll
    for (int r = 0; r < RX; ++r) v[t][r] = p[Y::off(r * Q)];
  }
  __syncthreads();
#pragma unroll
  for (int t = 0; t < TPT; ++t) {
    int q, j;
    Y::template split<Q>(threadIdx.x + t * NT, q, j);
    R f[RX];
#pragma unroll
    for (int r = 0; r < RX; ++r) f[r] = sc[j + r * Q];
    dft_r_scaled<RX>(v[t], f);
    C* o = buf + Y::at(q, j * RX);
#pragma unroll
    for (int r = 0; r < RX; ++r) o[Y::off(r)] = v[t][r];
  }
  __syncthreads();
}

template <int L, int NS, int NT, int RX, int LAY, typename C, typename R>
__device__ __noinline__ void fft_stage1_scaled_call(C* buf, const R* sc) {
  fft_stage1_scaled_body<L, NS, NT, RX, LAY>(buf, sc);
}

template <int L, int NS, int NT, int RX, int LAY, typename C, typename R>
__device__ __forceinline__ void fft_stage1_scaled(C* buf, const R* sc) {
  if constexpr (StageCalled<C>::value) fft_stage1_scaled_call<L, NS, NT, RX, LAY>(buf, sc);
  else fft_stage1_scaled_body<L, NS, NT, RX, LAY>(buf, sc);
}

// Radix-4 stage plan from span LS on, with one radix-2 stage last when log2(L) is odd.
template <int L, int NS, int NT, bool INV, int LAY, int LS, typename C>
__device__ __forceinline__ void fft_r4_from(C* buf, const C* tw) {
  if constexpr (LS * 4 <= L) {
    fft_stage_r<L, NS, NT, 4, INV, LAY, LS>(buf, tw);
    fft_r4_from<L, NS, NT, INV, LAY, LS * 4>(buf, tw);
  } else if constexpr (LS * 2 == L) {
    fft_stage_r<L, NS, NT, 2, INV, LAY, LS>(buf, tw);
  }
}

// Full transform of NS sequences of length L by NT threads (radix-4 plan).  The caller
// must have synchronised after writing buf; on return buf is synchronised too.
template <int L, int NS, int NT, bool INV, int LAY = 0, typename C>
__device__ __forceinline__ void fft_block(C* buf, const C* tw) {
  fft_r4_from<L, NS, NT, INV, LAY, 1>(buf, tw);
}

// Stage plans with radix-16 first: 64 = 16*4, 128 = 16*8, 256 = 16*16,
// 512 = 16*16*2, 1024 = 16*16*4.  The stages after the first:
template <int L, int NS, int NT, bool INV, int LAY, typename C>
__device__ __forceinline__ void fft_block16_rest(C* buf, const C* tw) {
  if constexpr (L == 64) {
    fft_stage_r<L, NS, NT, 4, INV, LAY, 16>(buf, tw);
  } else if constexpr (L == 128) {
    fft_stage_r<L, NS, NT, 8, INV, LAY, 16>(buf, tw);
  } else if constexpr (L == 256) {
    fft_stage_r<L, NS, NT, 16, INV, LAY, 16>(buf, tw);
  } else if constexpr (L == 512) {
    fft_stage_r<L, NS, NT, 16, INV, LAY, 16>(buf, tw);
    fft_stage_r<L, NS, NT, 2, INV, LAY, 256>(buf, tw);
  } else {
    fft_stage_r<L, NS, NT, 16, INV, LAY, 16>(buf, tw);
    fft_stage_r<L, NS, NT, 4, INV, LAY, 256>(buf, tw);
  }
}

template <int L, int NS, int NT, bool INV, int LAY = 0, typename C>
__device__ __forceinline__ void fft_block16(C* buf, const C* tw) {
  fft_stage_r<L, NS, NT, 16, INV, LAY, 1>(buf, tw);
  fft_block16_rest<L, NS, NT, INV, LAY>(buf, tw);
}

// Forward transforms of diag(sc) x, the scaling folded into the first stage.
template <int L, int NS, int NT, int LAY = 0, typename C, typename R>
__device__ __forceinline__ void fft_block_scaled(C* buf, const C* tw, const R* sc) {
  fft_stage1_scaled<L, NS, NT, 4, LAY>(buf, sc);
  fft_r4_from<L, NS, NT, false, LAY, 4>(buf, tw);
}
template <int L, int NS, int NT, int LAY = 0, typename C, typename R>
__device__ __forceinline__ void fft_block16_scaled(C* buf, const C* tw, const R* sc) {
  fft_stage1_scaled<L, NS, NT, 16, LAY>(buf, sc);
  fft_block16_rest<L, NS, NT, false, LAY>(buf, tw);
}

}  // namespace aao
