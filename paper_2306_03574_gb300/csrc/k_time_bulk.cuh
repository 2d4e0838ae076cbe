// Time part of P_alpha^{-1} in FP32/complex64 arithmetic on FP64 vectors, with the
// tile brought into shared memory by bulk asynchronous copies (the TMA engine) instead
// of per-thread loads.  The arithmetic (the pipeline of k_time.cuh) is unchanged:
// D^{-1}; FFT; x G; iFFT; D^2; FFT; x conj(G); iFFT; D^{-1}, two real modes per complex
// sequence, the interleaved padded shared-memory layout.
//
// Staging.  A CTA owns 2*NS consecutive modes s0 .. s0+2NS-1 and all L time levels.  Row
// t of the tile is the run in[t*m + s0 ..] of FP64 values; one elected warp issues one
// bulk copy per row (and, optionally, one per frequency row of the spectral-table slice)
// and a single mbarrier counts the bytes in.  Bulk copies need 16-byte aligned addresses
// and sizes: m = N^d is odd (N = 2^k - 1), so rows with odd t start 8 bytes past a
// 16-byte boundary.  Such a row is copied from one element earlier (and, inside the
// grid, to one element later), into a shared row of 2*NS + 2 doubles whose data then
// starts at offset 1; the last tile's ragged row ends are fetched with one plain load
// where the run would end off a boundary.  No copy reaches outside the vector.
//
// The FP64 -> FP32 conversion reads the staged rows into registers, a barrier passes, and
// the complex FP32 work buffer is written over the staging area (it is smaller).  The
// conversions can be done by integer operations on the bit fields (ICVT): on GB300 the
// FP64 pipe, which executes the cvt instructions, issues 2 operations per clock per SM,
// and the kernel converts two values per unknown.  The results are stored with plain
// coalesced stores.
#pragma once

#include "bulk_copy.cuh"
#include "convert_bits.cuh"
#include "k_time.cuh"

namespace aao {

template <int L, int NS, bool STAGE_T>
struct BulkTimeSmem {
  static constexpr int RS = 2 * NS + 2;  // doubles per staged row
  static constexpr size_t rows = (size_t)L * RS * sizeof(double);
  static constexpr size_t tab = STAGE_T ? (size_t)2 * NS * (L / 2 + 1) * sizeof(float2) : 0;
  static constexpr size_t bytes = rows + tab + (size_t)L * sizeof(float2) + 2 * (size_t)L * sizeof(float) + 16;
  static_assert((size_t)NS * (L + L / 16) * sizeof(float2) <= rows, "work buffer must fit the staging rows");
};

template <int L, int NS, int NT, int FFTV, bool STAGE_T, bool ICVT>
__global__ void __launch_bounds__(NT) k_time_bulk(const double* __restrict__ in, double* __restrict__ out,
                                                 TimeArgs a, PrecTables<float> tb) {
  using C = float2;
  using Y = SLay<L, NS, 1>;
  using SM = BulkTimeSmem<L, NS, STAGE_T>;
  constexpr int RS = SM::RS;
  constexpr bool FOLD = FoldScaling<float, L>::value;
  constexpr int TPT = NS * L / NT;
  static_assert(NS * L % NT == 0, "tasks per thread");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  double* rows = reinterpret_cast<double*>(smem_raw);
  C* cbuf = reinterpret_cast<C*>(smem_raw);  // over the rows once they are converted
  C* tab = reinterpret_cast<C*>(smem_raw + SM::rows);
  C* tw = reinterpret_cast<C*>(smem_raw + SM::rows + SM::tab);
  float* dinv = reinterpret_cast<float*>(tw + L);
  float* d2 = dinv + L;
  uint64_t* bar = reinterpret_cast<uint64_t*>(d2 + L);

  const int tid = threadIdx.x;
  const int m = a.m;
  const int s0 = blockIdx.x * (2 * NS);
  const int p0 = blockIdx.x * NS;
  const int cnt = min(2 * NS, m - s0);      // modes of this tile (odd only in the last tile)
  const int vp = min(NS, a.npairs - p0);    // mode pairs of this tile
  const long long rb = (long long)blockIdx.y * L * m;
  const double* inr = in + rb;
  double* outr = out + rb;
  // copy lengths (doubles) of even and odd rows: see the header comment
  const int len_even = cnt & ~1;
  const int len_odd = (cnt & 1) ? cnt + 1 : cnt + 2;

  if (tid == 0) mbar_init(bar, 1);
  __syncthreads();
  if (tid < 32) {
    if (tid == 0) {
      const uint32_t bytes = (uint32_t)((L / 2) * (len_even + len_odd) * sizeof(double)) +
                             (STAGE_T ? (uint32_t)((L / 2 + 1) * vp * 2 * sizeof(C)) : 0u);
      mbar_arrive_expect_tx(bar, bytes);
    }
    __syncwarp();
    for (int t = tid; t < L; t += 32) {
      double* dst = rows + (size_t)t * RS;
      const long long g = (long long)t * m + s0;
      if (t & 1) {
        bulk_load(dst, inr + g - 1, (uint32_t)(len_odd * sizeof(double)), bar);
      } else {
        if (len_even) bulk_load(dst, inr + g, (uint32_t)(len_even * sizeof(double)), bar);
        if (cnt & 1) dst[cnt - 1] = inr[g + cnt - 1];  // ragged end off a 16-byte boundary
      }
    }
    if constexpr (STAGE_T) {
      for (int k = tid; k <= L / 2; k += 32)
        bulk_load(tab + (size_t)k * 2 * NS, tb.ab + ((long long)k * a.npairs + p0) * 2,
                  (uint32_t)(vp * 2 * sizeof(C)), bar);
    }
  }
  for (int i = tid; i < L; i += NT) {
    tw[i] = tb.tw_time[i];
    dinv[i] = tb.dinv[i];
    d2[i] = tb.d2[i];
  }
  // bounded wait; a timeout (counted in g_wait_timeouts) abandons the tile after a
  // second bounded wait for the copies in flight
  const bool ok = mbar_wait(bar, 0);
  if (__syncthreads_or(!ok)) {
    mbar_wait(bar, 0);
    return;
  }

  // FP64 rows -> registers (FP32, scaled by D^{-1} unless the first FFT stage does it)
  C v[TPT];
#pragma unroll
  for (int i = 0; i < TPT; ++i) {
    const int task = tid + i * NT;
    const int q = task % NS, t = task / NS;
    const int j = 2 * q;
    const double* row = rows + (size_t)t * RS + (t & 1);
    const float di = FOLD ? 1.f : dinv[t];
    const float x0 = j < cnt ? to_f32<ICVT>(row[j]) : 0.f;
    const float x1 = j + 1 < cnt ? to_f32<ICVT>(row[j + 1]) : 0.f;
    v[i] = make_float2(FOLD ? x0 : x0 * di, FOLD ? x1 : x1 * di);
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < TPT; ++i) {
    const int task = tid + i * NT;
    cbuf[Y::at(task % NS, task / NS)] = v[i];
  }
  __syncthreads();

  if constexpr (FOLD) fft_run_scaled<FFTV, L, NS, NT, 1>(cbuf, tw, dinv);
  else fft_run<FFTV, L, NS, NT, false, 1>(cbuf, tw);
  mix_pass<false, L, NS, NT, 1, STAGE_T>(cbuf, tb.ab, tab, a.npairs, p0);
  fft_run<FFTV, L, NS, NT, true, 1>(cbuf, tw);
  if constexpr (FOLD) {
    fft_run_scaled<FFTV, L, NS, NT, 1>(cbuf, tw, d2);
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
    fft_run<FFTV, L, NS, NT, false, 1>(cbuf, tw);
  }
  mix_pass<true, L, NS, NT, 1, STAGE_T>(cbuf, tb.ab, tab, a.npairs, p0);
  fft_run<FFTV, L, NS, NT, true, 1>(cbuf, tw);

  // scale by D^{-1} and store
  for (int task = tid; task < NS * L; task += NT) {
    const int q = task % NS, t = task / NS;
    const int sa = s0 + 2 * q;
    double* p = outr + (long long)t * m + sa;
    const C z = cbuf[Y::at(q, t)];
    const float di = dinv[t];
    if (sa < m) p[0] = to_f64<ICVT>(z.x * di);
    if (sa + 1 < m) p[1] = to_f64<ICVT>(z.y * di);
  }
}

// Launch of the bulk-staged FP32 time pipeline: variant bits (after the base 8) select
// the tile (bit 0: 4096/L mode pairs x 256 threads or 2048/L x 128), the staged table
// slice (bit 1) and integer conversions (bit 2).
template <int L, int NS, int NT, bool STAGE_T, bool ICVT>
static cudaError_t time_bulk_cfg(const Plan& P, const double* in, double* out, int nrhs, cudaStream_t s) {
  const size_t smem = BulkTimeSmem<L, NS, STAGE_T>::bytes;
  TimeArgs a;
  a.m = P.m;
  a.n = P.n;
  a.npairs = P.npairs;
  auto kern = k_time_bulk<L, NS, NT, 1, STAGE_T, ICVT>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const int ntile = (P.m + 2 * NS - 1) / (2 * NS);
  kern<<<dim3(ntile, nrhs), NT, smem, s>>>(in, out, a, P.t32);
  return cudaGetLastError();
}

template <int L>
static cudaError_t time_bulk_L(int v, const Plan& P, const double* in, double* out, int nrhs, cudaStream_t s) {
  switch (v & 7) {
    case 0: return time_bulk_cfg<L, 4096 / L, 256, false, false>(P, in, out, nrhs, s);
    case 1: return time_bulk_cfg<L, 2048 / L, 128, false, false>(P, in, out, nrhs, s);
    case 2: return time_bulk_cfg<L, 4096 / L, 256, true, false>(P, in, out, nrhs, s);
    case 3: return time_bulk_cfg<L, 2048 / L, 128, true, false>(P, in, out, nrhs, s);
    case 4: return time_bulk_cfg<L, 4096 / L, 256, false, true>(P, in, out, nrhs, s);
    case 5: return time_bulk_cfg<L, 2048 / L, 128, false, true>(P, in, out, nrhs, s);
    case 6: return time_bulk_cfg<L, 4096 / L, 256, true, true>(P, in, out, nrhs, s);
    default: return time_bulk_cfg<L, 2048 / L, 128, true, true>(P, in, out, nrhs, s);
  }
}

static cudaError_t time_bulk_dispatch(int v, const Plan& P, const double* in, double* out, int nrhs,
                                      cudaStream_t s) {
  switch (P.n) {
    case 64: return time_bulk_L<64>(v, P, in, out, nrhs, s);
    case 128: return time_bulk_L<128>(v, P, in, out, nrhs, s);
    case 256: return time_bulk_L<256>(v, P, in, out, nrhs, s);
    case 512: return time_bulk_L<512>(v, P, in, out, nrhs, s);
    case 1024: return time_bulk_L<1024>(v, P, in, out, nrhs, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace aao
