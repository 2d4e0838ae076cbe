// Time part of P_alpha^{-1} for every spatial mode j (Section 2.3 with the
// spatial DSTs factored out):
//     z_j = D^{-1} F^* G_j F D^2 F G_j F^* D^{-1} y_j,
// D = diag(alpha^{t/n}), F = (1/sqrt n)[theta^{tk}], theta = exp(2 pi i/n),
// G_j = diag_k Sigma_{k,j}^{-1/2}, Sigma_{k,j} = Lambda_j lambda_{1,k} + lambda_{2,k}.
// With FFT = sum_t exp(-2 pi i tk/n): F^* = FFT/sqrt(n) and F = sqrt(n) iFFT, so
// for real y the map is: D^{-1}; FFT; x G; iFFT; D^2; FFT; x conj(G); iFFT; D^{-1}
// (the second pass, F G F^*, equals iFFT(conj(G) FFT(.)) on real data).
//
// Two real modes a, b share one complex sequence z = y_a + i y_b.  With
// Z = FFT(z), multiplying mode a by G_a and mode b by G_b is
//     Y_k = A_k Z_k + B_k conj(Z_{n-k}),  A = (G_a + G_b)/(2n), B = (G_a - G_b)/(2n)
// (1/n of the inverse FFT folded in), and iFFT(Y) = result_a + i result_b.
// G_{n-k} = conj(G_k) gives A_{n-k} = conj(A_k), B_{n-k} = conj(B_k), so the
// table holds k = 0..n/2 only.  A CTA owns 2*NS consecutive modes, all n time
// levels of them staged in shared memory (coalesced rows of the time-major vector).
//
// Kernel variants (bits of the variant number): bit 0 = FFT stage plan (radix-4
// or radix-16 first), bit 1 = tile (4096/n mode pairs x 256 threads or 2048/n x
// 128), bit 2 = shared-memory layout of the batch (sequence-major or interleaved
// and padded, see fft_smem.cuh).  The interleaved variants also stage the CTA's
// slice of the spectral table in shared memory with asynchronous copies issued
// before the input load, so both spectral multiplies read it from there and its
// global-memory latency overlaps the load.  Double-float has four more, 8..11 (bit 3):
// the interleaved layout without the staged slice, whose 16-byte table entries would
// otherwise take a third of the shared memory and one resident CTA per SM.  All variants compute the same values;
// the translation units k_time64.cu / k_time32.cu instantiate them per precision.
#pragma once
#include <type_traits>

#include "aao_internal.cuh"
#include "convert_bits.cuh"
#include "dfloat.cuh"
#include "fft_smem.cuh"

namespace aao {

struct TimeArgs {
  int m, n, npairs;
};

// Y_k = A Z + B conj(W) (CONJ: with conj(A), conj(B))
template <bool CONJ, typename C>
__device__ __forceinline__ C mix(C A, C B, C Z, C W) {
  if (CONJ) { A.y = -A.y; B.y = -B.y; }
  C Y;
  Y.x = fmadd(A.x, Z.x, fmadd(-A.y, Z.y, fmadd(B.x, W.x, B.y * W.y)));
  Y.y = fmadd(A.x, Z.y, fmadd(A.y, Z.x, fmadd(B.y, W.x, -(B.x * W.y))));
  return Y;
}

// 16-byte asynchronous global -> shared copy; bytes past src_bytes are zero-filled
__device__ __forceinline__ void cp_async16(void* dst, const void* src, int src_bytes) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Copy the CTA's table slice ab[k][p0 + q][A|B], k = 0..L/2, q < NS, into tab[(k NS + q) 2 + {0,1}]
// (rows past the last mode pair are zero-filled).  Each (k, q) entry is 2 sizeof(C) bytes,
// a whole number of 16-byte chunks starting on a 16-byte boundary.
template <int L, int NS, int NT, typename C>
__device__ __forceinline__ void stage_table(C* tab, const C* __restrict__ ab, int npairs, int p0) {
  constexpr int H = L / 2;
  constexpr int CH = (2 * (int)sizeof(C)) / 16;  // 16-byte chunks per entry
  for (int task = threadIdx.x; task < NS * (H + 1) * CH; task += NT) {
    const int c = task % CH, e = task / CH;
    const int q = e % NS, k = e / NS;
    const bool ok = p0 + q < npairs;
    const C* src = ok ? ab + ((long long)k * npairs + p0 + q) * 2 : ab;
    cp_async16(reinterpret_cast<char*>(tab + (long long)e * 2) + 16 * c,
               reinterpret_cast<const char*>(src) + 16 * c, ok ? 16 : 0);
  }
  cp_async_commit();
}

// Principal square root in FP32, cancellation-free: for Re z >= 0,
// sqrt z = t + i Im(z)/(2t) with t = sqrt((|z| + Re z)/2); otherwise
// sqrt z = |Im z|/(2t) + i sign(Im z) t with t = sqrt((|z| - Re z)/2).
__device__ __forceinline__ float2 csqrt_principal_f(float2 z) {
  const float r = sqrtf(fmaf(z.x, z.x, z.y * z.y));
  float2 s;
  if (z.x >= 0.f) {
    const float t = sqrtf(0.5f * (r + z.x));
    s.x = t;
    s.y = (t > 0.f) ? z.y / (2.f * t) : 0.f;
  } else {
    const float t = sqrtf(0.5f * (r - z.x));
    s.x = fabsf(z.y) / (2.f * t);
    s.y = copysignf(t, z.y);
  }
  return s;
}

// The CTA's slice of the spectral table computed on the fly in FP32 instead of read
// from memory (same layout as stage_table): for mode pair p = p0 + q and frequency k,
// Sigma_{k,s} = (1 - a theta^k)^2 + (Lambda_s - 1)(1 + a^2 theta^{2k}) for the modes
// s = 2p, 2p+1 (the per-frequency terms and Lambda_s - 1 come from small FP32 tables),
// G = Sigma^{-1/2} on the principal branch, A = (G_a + G_b)/(2n), B = (G_a - G_b)/(2n)
// (eqs. (calphaprediagform), (calphasqrtdiagform)).
template <int L, int NS, int NT>
__device__ __forceinline__ void compute_table(float2* tab, const PrecTables<float>& tb, int m, int p0) {
  constexpr int H = L / 2;
  for (int task = threadIdx.x; task < NS * (H + 1); task += NT) {
    const int q = task % NS, k = task / NS;
    const float2 w2 = tb.wq[2 * k], qk = tb.wq[2 * k + 1];
    float2 G[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int sidx = 2 * (p0 + q) + e;
      if (sidx >= m) { G[e] = make_float2(0.f, 0.f); continue; }
      const float lm1 = tb.lm1[sidx];
      const float2 sg = make_float2(fmaf(lm1, qk.x, w2.x), fmaf(lm1, qk.y, w2.y));
      const float2 sq = csqrt_principal_f(sg);
      const float qq = fmaf(sq.x, sq.x, sq.y * sq.y);
      G[e] = make_float2(sq.x / qq, -sq.y / qq);  // 1 / sqrt(Sigma)
    }
    tab[2 * task] = make_float2((G[0].x + G[1].x) * tb.inv2n, (G[0].y + G[1].y) * tb.inv2n);
    tab[2 * task + 1] = make_float2((G[0].x - G[1].x) * tb.inv2n, (G[0].y - G[1].y) * tb.inv2n);
  }
}

// Spectral multiply of every sequence of the tile; the (A, B) entries come from the
// staged slice tab when STAGED, else from the table in global memory.
template <bool CONJ, int L, int NS, int NT, int LAY, bool STAGED, typename C>
__device__ __forceinline__ void mix_pass(C* cbuf, const C* __restrict__ ab, const C* tab, int npairs, int p0) {
  using Y = SLay<L, NS, LAY>;
  constexpr int H = L / 2;
  for (int task = threadIdx.x; task < NS * (H + 1); task += NT) {
    const int q = task % NS, k = task / NS;
    C A, B;
    if constexpr (STAGED) {
      A = tab[2 * task];
      B = tab[2 * task + 1];
    } else if (p0 + q < npairs) {  // tiles may extend past the last mode pair (zero data there)
      const long long row = ((long long)k * npairs + p0 + q) * 2;
      A = ab[row];
      B = ab[row + 1];
    } else {
      A.x = A.y = B.x = B.y = 0;
    }
    const int ik = Y::at(q, k);
    if (k == 0 || k == H) {
      const C Z = cbuf[ik];
      cbuf[ik] = mix<CONJ>(A, B, Z, Z);
    } else {
      const int im = Y::at(q, L - k);
      const C Zk = cbuf[ik], Zm = cbuf[im];
      cbuf[ik] = mix<CONJ>(A, B, Zk, Zm);
      cbuf[im] = mix<!CONJ>(A, B, Zm, Zk);
    }
  }
  __syncthreads();
}

// FFT stage plan: 0 = radix-4 stages (+ one radix-2), 1 = radix-16 first (fewer passes)
template <int FFTV, int L, int NS, int NT, bool INV, int LAY, typename C>
__device__ __forceinline__ void fft_run(C* buf, const C* tw) {
  if constexpr (FFTV == 0) fft_block<L, NS, NT, INV, LAY>(buf, tw);
  else fft_block16<L, NS, NT, INV, LAY>(buf, tw);
}
// Forward FFT of diag(sc) x (the D^{-1} and D^2 scalings ride on the first stage)
template <int FFTV, int L, int NS, int NT, int LAY, typename C, typename R>
__device__ __forceinline__ void fft_run_scaled(C* buf, const C* tw, const R* sc) {
  if constexpr (FFTV == 0) fft_block_scaled<L, NS, NT, LAY>(buf, tw, sc);
  else fft_block16_scaled<L, NS, NT, LAY>(buf, tw, sc);
}

// Where the D^{-1} and D^2 scalings go: into the first stage of the forward FFTs
// (multiply-adds, one shared-memory pass fewer) in FP64, whose kernel is bound by the
// FP64 pipe, and in FP32 up to n = 256; at n >= 512 the FP32 kernel needs more
// registers for the folded stage and loses a resident CTA per SM, which costs more than
// the pass (measured), and in double-float a multiply-add saves nothing.  Otherwise the
// load applies D^{-1} and a separate pass D^2.
template <typename R, int L> struct FoldScaling { static constexpr bool value = false; };
template <int L> struct FoldScaling<double, L> { static constexpr bool value = true; };
template <int L> struct FoldScaling<float, L> { static constexpr bool value = L <= 256; };

// Tile `tile` (mode pairs tile*NS ..) of one right-hand side: in and out point at it.
// ICVT: FP64 <-> FP32 conversions by integer operations (convert_bits.cuh) instead of
// cvt instructions on the FP64 pipe: bit 0 those of the loads, bit 1 those of the stores.
// PRELOAD > 0: the tile's loads batched in registers, PRELOAD tasks (two values each)
// per batch, every load of a batch issued before the first is converted.
// OTF (FP32 with PRELOAD and the staged layout): the table slice computed on the fly
// (compute_table) while the first batch of loads is in flight, instead of read.
template <typename R, typename TIO, int L, int NS, int NT, int FFTV, int LAY, int STG, int ICVT = 0,
          int PRELOAD = 0, bool OTF = false>
__device__ __forceinline__ void time_body(const TIO* in, TIO* out, const TimeArgs& a, const PrecTables<R>& tb,
                                          int tile) {
  using CV = Cvt<R, TIO, ICVT>;
  using C = typename Cplx<R>::T;
  using Y = SLay<L, NS, LAY>;
  constexpr bool STAGED = STG < 0 ? LAY == 1 : STG == 1;
  constexpr bool FOLD = FoldScaling<R, L>::value;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* cbuf = reinterpret_cast<C*>(smem_raw);
  C* tab = cbuf + Y::size;                           // staged table slice (STAGED only)
  C* tw = tab + (STAGED ? 2 * NS * (L / 2 + 1) : 0);
  R* dinv = reinterpret_cast<R*>(tw + L);
  R* d2 = dinv + L;

  const int tid = threadIdx.x;
  const int m = a.m;
  const int s0 = tile * (2 * NS);
  const int p0 = tile * NS;
  static_assert(!OTF || (PRELOAD > 0 && STAGED && std::is_same<R, float>::value), "on-the-fly table");
  if constexpr (STAGED && !OTF) stage_table<L, NS, NT>(tab, tb.ab, a.npairs, p0);
  if constexpr (PRELOAD > 0) {
    // Batches of PB tasks: every load of a batch is issued (into registers) before the
    // first is converted, the first batch before the table loads and the barrier.
    constexpr int TPT = NS * L / NT;
    constexpr int PB = TPT < PRELOAD ? TPT : PRELOAD;
    static_assert(NS * L % NT == 0 && TPT % PB == 0, "load batches");
    TIO xa[PB], xb[PB];
    auto load = [&](int b0) {
#pragma unroll
      for (int i = 0; i < PB; ++i) {
        const int task = tid + (b0 + i) * NT;
        const int q = task % NS, t = task / NS;
        const int sa = s0 + 2 * q;
        const TIO* p = in + (long long)t * m + sa;
        xa[i] = sa < m ? p[0] : TIO(0);
        xb[i] = sa + 1 < m ? p[1] : TIO(0);
      }
    };
    auto put = [&](int b0) {
#pragma unroll
      for (int i = 0; i < PB; ++i) {
        const int task = tid + (b0 + i) * NT;
        const int q = task % NS, t = task / NS;
        const R di = FOLD ? R(1) : dinv[t];
        C z;
        z.x = FOLD ? CV::load(xa[i]) : CV::load(xa[i]) * di;
        z.y = FOLD ? CV::load(xb[i]) : CV::load(xb[i]) * di;
        cbuf[Y::at(q, t)] = z;
      }
    };
    load(0);
    if constexpr (OTF) compute_table<L, NS, NT>(tab, tb, m, p0);
    for (int i = tid; i < L; i += NT) {
      tw[i] = tb.tw_time[i];
      dinv[i] = tb.dinv[i];
      d2[i] = tb.d2[i];
    }
    __syncthreads();
    put(0);
#pragma unroll 1
    for (int b0 = PB; b0 < TPT; b0 += PB) {
      load(b0);
      put(b0);
    }
  } else {
    for (int i = tid; i < L; i += NT) {
      tw[i] = tb.tw_time[i];
      dinv[i] = tb.dinv[i];
      d2[i] = tb.d2[i];
    }
    __syncthreads();

    // load, scaled by D^{-1} here or (FOLD) by the first FFT stage
    for (int task = tid; task < NS * L; task += NT) {
      const int q = task % NS, t = task / NS;
      const int sa = s0 + 2 * q;
      const TIO* p = in + (long long)t * m + sa;
      const R di = FOLD ? R(1) : dinv[t];
      C z;
      z.x = (sa < m) ? (FOLD ? CV::load(p[0]) : CV::load(p[0]) * di) : R();
      z.y = (sa + 1 < m) ? (FOLD ? CV::load(p[1]) : CV::load(p[1]) * di) : R();
      cbuf[Y::at(q, t)] = z;
    }
  }
  if constexpr (STAGED) cp_async_wait_all();
  __syncthreads();

  if constexpr (FOLD) fft_run_scaled<FFTV, L, NS, NT, LAY>(cbuf, tw, dinv);
  else fft_run<FFTV, L, NS, NT, false, LAY>(cbuf, tw);
  mix_pass<false, L, NS, NT, LAY, STAGED>(cbuf, tb.ab, tab, a.npairs, p0);
  fft_run<FFTV, L, NS, NT, true, LAY>(cbuf, tw);
  if constexpr (FOLD) {
    fft_run_scaled<FFTV, L, NS, NT, LAY>(cbuf, tw, d2);
  } else {
    for (int task = tid; task < NS * L; task += NT) {
      const int q = task % NS, t = task / NS;
      const int i = Y::at(q, t);
      C z = cbuf[i];
      z.x *= d2[t];
      z.y *= d2[t];
      cbuf[i] = z;
    }
    __syncthreads();
    fft_run<FFTV, L, NS, NT, false, LAY>(cbuf, tw);
  }
  mix_pass<true, L, NS, NT, LAY, STAGED>(cbuf, tb.ab, tab, a.npairs, p0);
  fft_run<FFTV, L, NS, NT, true, LAY>(cbuf, tw);

  // scale by D^{-1} and store
  for (int task = tid; task < NS * L; task += NT) {
    const int q = task % NS, t = task / NS;
    const int sa = s0 + 2 * q;
    TIO* p = out + (long long)t * m + sa;
    const C z = cbuf[Y::at(q, t)];
    const R di = dinv[t];
    if (sa < m) p[0] = CV::store(z.x * di);
    if (sa + 1 < m) p[1] = CV::store(z.y * di);
  }
}

template <typename R, typename TIO, int L, int NS, int NT, int FFTV, int LAY, int STG = -1, int ICVT = 0,
          int PRELOAD = 0, bool OTF = false>
__global__ void __launch_bounds__(NT) k_time(const TIO* in, TIO* out, TimeArgs a, PrecTables<R> tb) {
  const long long rb = (long long)blockIdx.y * L * a.m;
  time_body<R, TIO, L, NS, NT, FFTV, LAY, STG, ICVT, PRELOAD, OTF>(in + rb, out + rb, a, tb, blockIdx.x);
}

// The same built for MINB resident CTAs per SM (a register cap; the spills it may cause
// are the price of the occupancy)
template <typename R, typename TIO, int L, int NS, int NT, int FFTV, int LAY, int STG, int ICVT, int PRELOAD,
          bool OTF, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_time_occ(const TIO* in, TIO* out, TimeArgs a, PrecTables<R> tb) {
  const long long rb = (long long)blockIdx.y * L * a.m;
  time_body<R, TIO, L, NS, NT, FFTV, LAY, STG, ICVT, PRELOAD, OTF>(in + rb, out + rb, a, tb, blockIdx.x);
}

// Tile shapes: full = 4096/L modes-pairs x 256 threads, half = 2048/L x 128 threads.
template <typename R, typename TIO, int L, int NS, int NT, int FFTV, int LAY, int STG = -1, int ICVT = 0,
          int PRELOAD = 0, bool OTF = false, int MINB = 0>
static cudaError_t time_launch_cfg(const Plan& P, const TIO* in, TIO* out, int nrhs, cudaStream_t s) {
  using C = typename Cplx<R>::T;
  constexpr bool STAGED = STG < 0 ? LAY == 1 : STG == 1;
  const size_t smem = sizeof(C) * (SLay<L, NS, LAY>::size + (STAGED ? 2 * NS * (L / 2 + 1) : 0) + L) +
                      2 * sizeof(R) * L;
  TimeArgs a;
  a.m = P.m;
  a.n = P.n;
  a.npairs = P.npairs;
  const int ntile = (P.m + 2 * NS - 1) / (2 * NS);
  auto go = [&](auto kern) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kern<<<dim3(ntile, nrhs), NT, smem, s>>>(in, out, a, tables<R>(P));
  };
  if constexpr (MINB > 0) go(k_time_occ<R, TIO, L, NS, NT, FFTV, LAY, STG, ICVT, PRELOAD, OTF, MINB>);
  else go(k_time<R, TIO, L, NS, NT, FFTV, LAY, STG, ICVT, PRELOAD, OTF>);
  return cudaGetLastError();
}

template <typename R, typename TIO, int L>
static cudaError_t time_launch_L(const Plan& P, const TIO* in, TIO* out, int nrhs, cudaStream_t s) {
  const int v = std::is_same<R, double>::value  ? P.time_variant64
                : std::is_same<R, float>::value ? P.time_variant32
                                                : P.time_variant_ff;
  // small-problem tile: one warp, small_pairs(L) mode pairs, radix-4 plan, sequence-major
  if (v == TIME_VARIANT_SMALL)
    return time_launch_cfg<R, TIO, L, small_pairs(L), SMALL_NT, 0, 0>(P, in, out, nrhs, s);
  if constexpr (std::is_same<R, float>::value && std::is_same<TIO, float>::value) {
    // FP32 vectors: the variants of the FP64-vector kernel above 7 map to the classic
    // layout of their tile (full: 5, half: 7)
    if (v >= 8) return (v & 1) ? time_launch_cfg<R, TIO, L, 2048 / L, 128, 1, 1>(P, in, out, nrhs, s)
                               : time_launch_cfg<R, TIO, L, 4096 / L, 256, 1, 1>(P, in, out, nrhs, s);
  }
  if constexpr (std::is_same<R, float>::value && std::is_same<TIO, double>::value) {
    // FP32 arithmetic on FP64 vectors: 16, 17 = variants 5, 7 with integer conversions;
    // 18, 19 = variants 5, 7 with the loads batched 8 tasks at a time, 20, 21 16 at a time
    if (v == 16) return time_launch_cfg<R, TIO, L, 4096 / L, 256, 1, 1, -1, 3>(P, in, out, nrhs, s);
    if (v == 17) return time_launch_cfg<R, TIO, L, 2048 / L, 128, 1, 1, -1, 3>(P, in, out, nrhs, s);
    if (v == 18) return time_launch_cfg<R, TIO, L, 4096 / L, 256, 1, 1, -1, 0, 8>(P, in, out, nrhs, s);
    if (v == 19) return time_launch_cfg<R, TIO, L, 2048 / L, 128, 1, 1, -1, 0, 8>(P, in, out, nrhs, s);
    if (v == 20) return time_launch_cfg<R, TIO, L, 4096 / L, 256, 1, 1, -1, 0, 16>(P, in, out, nrhs, s);
    if (v == 21) return time_launch_cfg<R, TIO, L, 2048 / L, 128, 1, 1, -1, 0, 16>(P, in, out, nrhs, s);
    // 22, 23 = 18, 19 with the spectral table slice computed on the fly
    if (v == 22) return time_launch_cfg<R, TIO, L, 4096 / L, 256, 1, 1, -1, 0, 8, true>(P, in, out, nrhs, s);
    if (v == 23) return time_launch_cfg<R, TIO, L, 2048 / L, 128, 1, 1, -1, 0, 8, true>(P, in, out, nrhs, s);
    // 24, 25 = 18, 19 with the stores converted by integer operations; 26, 27 the loads;
    // 28, 29 both
    if (v == 24) return time_launch_cfg<R, TIO, L, 4096 / L, 256, 1, 1, -1, 2, 8>(P, in, out, nrhs, s);
    if (v == 25) return time_launch_cfg<R, TIO, L, 2048 / L, 128, 1, 1, -1, 2, 8>(P, in, out, nrhs, s);
    if (v == 26) return time_launch_cfg<R, TIO, L, 4096 / L, 256, 1, 1, -1, 1, 8>(P, in, out, nrhs, s);
    if (v == 27) return time_launch_cfg<R, TIO, L, 2048 / L, 128, 1, 1, -1, 1, 8>(P, in, out, nrhs, s);
    if (v == 28) return time_launch_cfg<R, TIO, L, 4096 / L, 256, 1, 1, -1, 3, 8>(P, in, out, nrhs, s);
    if (v == 29) return time_launch_cfg<R, TIO, L, 2048 / L, 128, 1, 1, -1, 3, 8>(P, in, out, nrhs, s);
    // 31, 32 = 27, 29 and 33 = 26 without the staged table slice (the mix passes read the
    // table from memory): half the shared memory, more CTAs per SM
    if (v == 31) return time_launch_cfg<R, TIO, L, 2048 / L, 128, 1, 1, 0, 1, 8>(P, in, out, nrhs, s);
    if (v == 32) return time_launch_cfg<R, TIO, L, 2048 / L, 128, 1, 1, 0, 3, 8>(P, in, out, nrhs, s);
    if (v == 33) return time_launch_cfg<R, TIO, L, 4096 / L, 256, 1, 1, 0, 1, 8>(P, in, out, nrhs, s);
  }
  if constexpr (std::is_same<R, dfl>::value) {
    // 12, 13 = variants 9, 11 with the loads batched 8 tasks at a time
    if (v == 12) return time_launch_cfg<R, TIO, L, 4096 / L, 256, 1, 1, 0, 0, 8>(P, in, out, nrhs, s);
    if (v == 13) return time_launch_cfg<R, TIO, L, 2048 / L, 128, 1, 1, 0, 0, 8>(P, in, out, nrhs, s);
    // 14 = 13 built for 5 CTAs per SM (the half tile's shared memory allows 5, its 120
    // registers 4)
    if (v == 14) return time_launch_cfg<R, TIO, L, 2048 / L, 128, 1, 1, 0, 0, 8, false, 5>(P, in, out, nrhs, s);
    if (v & 8) {  // interleaved layout without the staged table slice
      switch (v & 3) {
        case 0: return time_launch_cfg<R, TIO, L, 4096 / L, 256, 0, 1, 0>(P, in, out, nrhs, s);
        case 1: return time_launch_cfg<R, TIO, L, 4096 / L, 256, 1, 1, 0>(P, in, out, nrhs, s);
        case 2: return time_launch_cfg<R, TIO, L, 2048 / L, 128, 0, 1, 0>(P, in, out, nrhs, s);
        default: return time_launch_cfg<R, TIO, L, 2048 / L, 128, 1, 1, 0>(P, in, out, nrhs, s);
      }
    }
  }
  switch (v & 7) {
    case 0: return time_launch_cfg<R, TIO, L, 4096 / L, 256, 0, 0>(P, in, out, nrhs, s);
    case 1: return time_launch_cfg<R, TIO, L, 4096 / L, 256, 1, 0>(P, in, out, nrhs, s);
    case 2: return time_launch_cfg<R, TIO, L, 2048 / L, 128, 0, 0>(P, in, out, nrhs, s);
    case 3: return time_launch_cfg<R, TIO, L, 2048 / L, 128, 1, 0>(P, in, out, nrhs, s);
    case 4: return time_launch_cfg<R, TIO, L, 4096 / L, 256, 0, 1>(P, in, out, nrhs, s);
    case 5: return time_launch_cfg<R, TIO, L, 4096 / L, 256, 1, 1>(P, in, out, nrhs, s);
    case 6: return time_launch_cfg<R, TIO, L, 2048 / L, 128, 0, 1>(P, in, out, nrhs, s);
    default: return time_launch_cfg<R, TIO, L, 2048 / L, 128, 1, 1>(P, in, out, nrhs, s);
  }
}

template <typename R, typename TIO>
static cudaError_t time_dispatch(const Plan& P, const TIO* in, TIO* out, int nrhs, cudaStream_t s) {
  switch (P.n) {
    case 64: return time_launch_L<R, TIO, 64>(P, in, out, nrhs, s);
    case 128: return time_launch_L<R, TIO, 128>(P, in, out, nrhs, s);
    case 256: return time_launch_L<R, TIO, 256>(P, in, out, nrhs, s);
    case 512: return time_launch_L<R, TIO, 512>(P, in, out, nrhs, s);
    case 1024: return time_launch_L<R, TIO, 1024>(P, in, out, nrhs, s);
    default: return cudaErrorInvalidValue;
  }
}

template <typename R>
cudaError_t launch_time(const Plan& P, const R* in, R* out, int nrhs, cudaStream_t s, uint64_t* nl) {
  if (nl) ++*nl;
  return time_dispatch<R, R>(P, in, out, nrhs, s);
}

}  // namespace aao
