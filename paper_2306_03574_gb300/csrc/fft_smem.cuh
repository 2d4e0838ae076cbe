// Batched complex FFT of length L executed by a whole CTA on sequences held in
// shared memory: Stockham autosort, radix-4 stages and one radix-2 stage when
// log2(L) is odd, natural order in and out, forward = exp(-2 pi i jk/L),
// inverse = exp(+2 pi i jk/L), both unnormalised.
//
// Each stage first loads every value it needs into registers, synchronises,
// then writes the butterfly outputs back in place, so a single buffer serves
// all stages.  Sequence q of the batch occupies buf[q*L .. q*L+L).
#pragma once

#include "aao_internal.cuh"

namespace aao {

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

// One radix-4 Stockham stage with span Ls (sub-transforms of length Ls done).
template <int L, int NS, int NT, bool INV, typename C>
__device__ __forceinline__ void fft_stage4(C* buf, const C* tw, int Ls) {
  constexpr int Q = L / 4;
  constexpr int TASKS = NS * Q;
  static_assert(TASKS % NT == 0, "radix-4 tasks must divide evenly among threads");
  constexpr int TPT = TASKS / NT;
  C v[TPT][4];
#pragma unroll
  for (int t = 0; t < TPT; ++t) {
    const int task = threadIdx.x + t * NT;
    const int q = task / Q, j = task % Q;
    const C* p = buf + q * L + j;
#pragma unroll
    for (int r = 0; r < 4; ++r) v[t][r] = p[r * Q];
  }
  __syncthreads();
#pragma unroll
  for (int t = 0; t < TPT; ++t) {
    const int task = threadIdx.x + t * NT;
    const int q = task / Q, j = task % Q;
    const int k = j & (Ls - 1);
    if (Ls > 1) {
      const int step = (Q / Ls) * k;  // twiddle exponent r*k*L/(4 Ls)
      v[t][1] = cmul(v[t][1], twid<INV>(tw[step]));
      v[t][2] = cmul(v[t][2], twid<INV>(tw[2 * step]));
      v[t][3] = cmul(v[t][3], twid<INV>(tw[3 * step]));
    }
    dft4<INV>(v[t][0], v[t][1], v[t][2], v[t][3]);
    C* o = buf + q * L + (j - k) * 4 + k;
#pragma unroll
    for (int r = 0; r < 4; ++r) o[r * Ls] = v[t][r];
  }
  __syncthreads();
}

// Final radix-2 stage (span L/2).
template <int L, int NS, int NT, bool INV, typename C>
__device__ __forceinline__ void fft_stage2_last(C* buf, const C* tw) {
  constexpr int Q = L / 2;
  constexpr int TASKS = NS * Q;
  static_assert(TASKS % NT == 0, "radix-2 tasks must divide evenly among threads");
  constexpr int TPT = TASKS / NT;
  C v[TPT][2];
#pragma unroll
  for (int t = 0; t < TPT; ++t) {
    const int task = threadIdx.x + t * NT;
    const int q = task / Q, j = task % Q;
    v[t][0] = buf[q * L + j];
    v[t][1] = buf[q * L + j + Q];
  }
  __syncthreads();
#pragma unroll
  for (int t = 0; t < TPT; ++t) {
    const int task = threadIdx.x + t * NT;
    const int q = task / Q, j = task % Q;
    const C b = cmul(v[t][1], twid<INV>(tw[j]));
    buf[q * L + j] = cadd(v[t][0], b);
    buf[q * L + j + Q] = csub(v[t][0], b);
  }
  __syncthreads();
}

// Full transform of NS sequences of length L by NT threads.  The caller must
// have synchronised after writing buf; on return buf is synchronised too.
template <int L, int NS, int NT, bool INV, typename C>
__device__ __forceinline__ void fft_block(C* buf, const C* tw) {
  constexpr int LG = Log2<L>::value;
#pragma unroll
  for (int s = 0; s < LG / 2; ++s) fft_stage4<L, NS, NT, INV>(buf, tw, 1 << (2 * s));
  if constexpr ((LG & 1) != 0) fft_stage2_last<L, NS, NT, INV>(buf, tw);
}

}  // namespace aao
