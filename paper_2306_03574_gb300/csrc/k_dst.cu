// Orthonormal DST-I along one spatial axis (the matrix S = U-factor of Section 2.3:
// on a uniform grid the eigenvectors of L are the discrete sine transform).
//
// Two lines a, b of length N = M-1 are transformed by one complex FFT of length
// M = N+1.  For one real line x_1..x_N (x_0 = x_M = 0) put
//     y_j = sin(pi j/M)(x_j + x_{M-j}) + (x_j - x_{M-j})/2,   j = 0..M-1,
// and let Y_k = sum_j y_j exp(-2 pi i jk/M).  Then the DST-I
// X_k = sum_j x_j sin(pi jk/M) satisfies
//     X_{2k}   = -Im Y_k,
//     X_{2k+1} = X_{2k-1} + Re Y_k,   X_1 = Re Y_0 / 2,
// (the symmetric part of y feeds the cosine sums, the antisymmetric part the
// sine sums).  Lines a and b are packed as y^a + i y^b and separated after the
// FFT through Y^a_k = (C_k + conj C_{M-k})/2, Y^b_k = (C_k - conj C_{M-k})/(2i).
// The factor sqrt(2/M) and the 1/2 of the separation are folded into the
// pre-processing weights.  The odd outputs are a prefix sum over k, done per
// thread block of k and then across the threads of a line pair by shuffles.
//
// R is the arithmetic type (double, float or the double-float dfl), TIO the type of
// the vectors in memory (R itself, or double for the double-float kernels).
#include "aao_internal.cuh"
#include "dfloat.cuh"
#include "fft_smem.cuh"

namespace aao {

__device__ __forceinline__ double shfl_up(double v, int off, int w) { return __shfl_up_sync(0xffffffffu, v, off, w); }
__device__ __forceinline__ float shfl_up(float v, int off, int w) { return __shfl_up_sync(0xffffffffu, v, off, w); }
__device__ __forceinline__ dfl shfl_up(dfl v, int off, int w) {
  return dfl(__shfl_up_sync(0xffffffffu, v.hi, off, w), __shfl_up_sync(0xffffffffu, v.lo, off, w));
}

struct DstArgs {
  int N;            // line length
  long long nlines; // contiguous axis: number of lines (all rhs and time levels)
  int st;           // strided axis: stride = extent of the contiguous inner index
  long long nouter; // strided axis: number of outer blocks
};

// PRE: the pre-processing loads of a thread issued in batches of 4 tasks (16 values)
// before any of them is used, the first batch ahead of the table loads and the barrier.
// LAY: shared-memory layout of the line pairs (fft_smem.cuh: 0 sequence-major, 1
// interleaved and padded); with LAY 1 the threads of a warp walk the line pairs first in
// the pre-processing and the store too, so that their shared-memory accesses stay
// conflict-free (the global accesses then take whole 32-byte sectors of several lines).
template <typename R, typename TIO, int M, int NS, int NT, bool STRIDED, int FFTV, bool PRE = false, int LAY = 0>
__global__ void __launch_bounds__(NT) k_dst(const TIO* in, TIO* out, DstArgs a, PrecTables<R> tb) {
  using C = typename Cplx<R>::T;
  using Y = SLay<M, NS, LAY>;
  constexpr int H = M / 2;
  constexpr int TPS = NT / NS;     // threads per line pair in the post-processing
  constexpr int KQ = H / TPS;      // k values per thread
  static_assert(NT % NS == 0 && H % TPS == 0 && TPS <= 32 && (32 % TPS) == 0, "dst config");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* cbuf = reinterpret_cast<C*>(smem_raw);
  C* tw = cbuf + Y::size;
  R* sw = reinterpret_cast<R*>(tw + M);

  const int tid = threadIdx.x;
  const int N = a.N;

  // line addressing
  long long line0 = 0, obase = 0;
  int i0 = 0;
  if (!STRIDED) {
    line0 = (long long)blockIdx.x * (2 * NS);
  } else {
    obase = (long long)blockIdx.x * ((long long)a.st * N);
    i0 = blockIdx.y * (2 * NS);
  }

  // ---- pre-processing: y'_j, y'_{M-j} for j = 1..M/2 of lines a, b ----
  // task -> (line pair q, index j); the four inputs x_j, x_{M-j} of lines a, b
  auto task_qj = [&](int task, int& q, int& j) {
    if (!STRIDED && !LAY) { q = task / H; j = task % H + 1; }
    else { q = task % NS; j = task / NS + 1; }
  };
  auto load4 = [&](int task, TIO& a0, TIO& a1, TIO& b0, TIO& b1) {
    int q, j;
    task_qj(task, q, j);
    a0 = a1 = b0 = b1 = TIO(0);
    if (!STRIDED) {
      const long long la = line0 + 2 * q;
      if (la < a.nlines) {
        const TIO* p = in + la * N;
        a0 = p[j - 1];
        a1 = p[M - j - 1];
      }
      if (la + 1 < a.nlines) {
        const TIO* p = in + (la + 1) * N;
        b0 = p[j - 1];
        b1 = p[M - j - 1];
      }
    } else {
      const int ia = i0 + 2 * q;
      const TIO* p = in + obase + ia;
      if (ia < a.st) {
        a0 = p[(long long)(j - 1) * a.st];
        a1 = p[(long long)(M - j - 1) * a.st];
      }
      if (ia + 1 < a.st) {
        b0 = p[(long long)(j - 1) * a.st + 1];
        b1 = p[(long long)(M - j - 1) * a.st + 1];
      }
    }
  };
  auto weigh = [&](int task, R xa0, R xa1, R xb0, R xb1) {
    int q, j;
    task_qj(task, q, j);
    const R cq = tb.cq;
    const R w = sw[j];
    const R sa = xa0 + xa1, ta = cq * (xa0 - xa1);
    const R sb = xb0 + xb1, tbb = cq * (xb0 - xb1);
    C lo, hi;
    lo.x = fmadd(w, sa, ta);  lo.y = fmadd(w, sb, tbb);
    hi.x = fmadd(w, sa, -ta); hi.y = fmadd(w, sb, -tbb);
    cbuf[Y::at(q, j)] = lo;
    if (j != H) cbuf[Y::at(q, M - j)] = hi;
  };
  if constexpr (PRE) {
    constexpr int TPT = NS * H / NT, PB = 4;
    static_assert(NS * H % NT == 0 && TPT % PB == 0, "pre-processing batches");
    TIO x[PB][4];
#pragma unroll
    for (int i = 0; i < PB; ++i) load4(tid + i * NT, x[i][0], x[i][1], x[i][2], x[i][3]);
    for (int i = tid; i < M; i += NT) tw[i] = tb.tw_space[i];
    for (int i = tid; i <= H; i += NT) sw[i] = tb.sinw[i];
    __syncthreads();
#pragma unroll 1
    for (int b0 = 0; b0 < TPT; b0 += PB) {
      if (b0 > 0) {
#pragma unroll
        for (int i = 0; i < PB; ++i) load4(tid + (b0 + i) * NT, x[i][0], x[i][1], x[i][2], x[i][3]);
      }
#pragma unroll
      for (int i = 0; i < PB; ++i) weigh(tid + (b0 + i) * NT, R(x[i][0]), R(x[i][1]), R(x[i][2]), R(x[i][3]));
    }
  } else {
    for (int i = tid; i < M; i += NT) tw[i] = tb.tw_space[i];
    for (int i = tid; i <= H; i += NT) sw[i] = tb.sinw[i];
    __syncthreads();
    for (int task = tid; task < NS * H; task += NT) {
      TIO a0, a1, b0, b1;
      load4(task, a0, a1, b0, b1);
      weigh(task, R(a0), R(a1), R(b0), R(b1));
    }
  }
  for (int q = tid; q < NS; q += NT) { C z; z.x = R(); z.y = R(); cbuf[Y::at(q, 0)] = z; }
  __syncthreads();

  if constexpr (FFTV == 0) fft_block<M, NS, NT, false, LAY>(cbuf, tw);
  else fft_block16<M, NS, NT, false, LAY>(cbuf, tw);

  // ---- post-processing: separate the two lines, prefix sum for odd outputs ----
  const int q = tid / TPS, lq = tid % TPS;
  const int k0 = lq * KQ;
  R pa[KQ], pb[KQ], ia[KQ], ib[KQ];
  {
    R acc_a = R(), acc_b = R();
#pragma unroll
    for (int i = 0; i < KQ; ++i) {
      const int k = k0 + i;
      const C ck = cbuf[Y::at(q, k)];
      R ra, rb;
      if (k == 0) {
        ra = ck.x; rb = ck.y; ia[i] = R(); ib[i] = R();
      } else {
        const C cm = cbuf[Y::at(q, M - k)];
        ra = ck.x + cm.x; rb = ck.y + cm.y;
        ia[i] = cm.y - ck.y; ib[i] = ck.x - cm.x;
      }
      acc_a += ra; acc_b += rb;
      pa[i] = acc_a; pb[i] = acc_b;
    }
  }
  // exclusive scan of the per-thread totals across the TPS threads of line pair q
  R inc_a = pa[KQ - 1], inc_b = pb[KQ - 1];
#pragma unroll
  for (int off = 1; off < TPS; off <<= 1) {
    const R ua = shfl_up(inc_a, off, TPS);
    const R ub = shfl_up(inc_b, off, TPS);
    if (lq >= off) { inc_a += ua; inc_b += ub; }
  }
  R ex_a = shfl_up(inc_a, 1, TPS);
  R ex_b = shfl_up(inc_b, 1, TPS);
  if (lq == 0) { ex_a = R(); ex_b = R(); }
  __syncthreads();  // all reads of the spectrum are done
#pragma unroll
  for (int i = 0; i < KQ; ++i) {
    const int k = k0 + i;
    C odd; odd.x = pa[i] + ex_a; odd.y = pb[i] + ex_b;
    cbuf[Y::at(q, 2 * k)] = odd;          // X_{2k+1} -> index 2k
    if (k >= 1) {
      C ev; ev.x = ia[i]; ev.y = ib[i];
      cbuf[Y::at(q, 2 * k - 1)] = ev;     // X_{2k}   -> index 2k-1
    }
  }
  __syncthreads();

  // ---- store ----
  if (!STRIDED && LAY) {
    // lines fastest across the threads (conflict-free reads of the interleaved layout)
    const long long e0 = line0 * N;
    for (int task = tid; task < 2 * NS * N; task += NT) {
      const int l = task % (2 * NS), j = task / (2 * NS);
      if (line0 + l < a.nlines) {
        const C v = cbuf[Y::at(l >> 1, j)];
        out[e0 + (long long)l * N + j] = TIO((l & 1) ? v.y : v.x);
      }
    }
  } else if (!STRIDED) {
    // line by line (no division by the runtime length N); rows are contiguous in memory
    const long long e0 = line0 * N;
    for (int l = 0; l < 2 * NS; ++l) {
      if (line0 + l >= a.nlines) break;
      const C* row = cbuf + (l >> 1) * M;
      TIO* o = out + e0 + (long long)l * N;
      for (int j = tid; j < N; j += NT) {
        const C v = row[j];
        o[j] = TIO((l & 1) ? v.y : v.x);
      }
    }
  } else {
    for (int task = tid; task < 2 * NS * N; task += NT) {
      const int l = task % (2 * NS), j = task / (2 * NS);
      const int il = i0 + l;
      if (il < a.st) {
        const C v = cbuf[Y::at(l >> 1, j)];
        out[obase + (long long)j * a.st + il] = TIO((l & 1) ? v.y : v.x);
      }
    }
  }
}

// NS line pairs per CTA of NT threads (standard: 2048/M pairs, 128 threads)
template <typename R, typename TIO, int M, int FFTV, bool PRE, int NS = 2048 / M, int NT = 128, int LAY = 0>
static cudaError_t dst_launch_MV(const Plan& P, const TIO* in, TIO* out, int axis, int nrhs,
                                 cudaStream_t s) {
  using C = typename Cplx<R>::T;
  const PrecTables<R>& tb = tables<R>(P);
  const size_t smem = sizeof(C) * (SLay<M, NS, LAY>::size + M) + sizeof(R) * (M / 2 + 1);
  DstArgs a;
  a.N = P.N;
  long long stride = 1;
  for (int i = 0; i < axis; ++i) stride *= P.N;
  const long long total = (long long)nrhs * P.n * P.m;
  if (axis == 0) {
    a.nlines = total / P.N;
    a.st = 1;
    a.nouter = 0;
    auto kern = k_dst<R, TIO, M, NS, NT, false, FFTV, PRE, LAY>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const long long nb = (a.nlines + 2 * NS - 1) / (2 * NS);
    kern<<<dim3((unsigned)nb), NT, smem, s>>>(in, out, a, tb);
  } else {
    a.st = (int)stride;
    a.nouter = total / (stride * P.N);
    a.nlines = 0;
    auto kern = k_dst<R, TIO, M, NS, NT, true, FFTV, PRE, LAY>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int ntile = (int)((stride + 2 * NS - 1) / (2 * NS));
    kern<<<dim3((unsigned)a.nouter, (unsigned)ntile), NT, smem, s>>>(in, out, a, tb);
  }
  return cudaGetLastError();
}

template <typename R, typename TIO, int M>
static cudaError_t dst_launch_M(const Plan& P, const TIO* in, TIO* out, int axis, int nrhs,
                                cudaStream_t s) {
  // bit 0: radix-16 stage plan; bit 1: batched pre-processing loads; bit 2: interleaved
  // padded shared-memory layout; or the small tile (one warp, small_pairs(M) line
  // pairs, radix-4 plan)
  constexpr int NS = 2048 / M, NT = 128;
  if (P.dst_variant == DST_VARIANT_SMALL)
    return dst_launch_MV<R, TIO, M, 0, false, small_pairs(M), SMALL_NT>(P, in, out, axis, nrhs, s);
  switch (P.dst_variant & 7) {
    case 0: return dst_launch_MV<R, TIO, M, 0, false>(P, in, out, axis, nrhs, s);
    case 1: return dst_launch_MV<R, TIO, M, 1, false>(P, in, out, axis, nrhs, s);
    case 2: return dst_launch_MV<R, TIO, M, 0, true>(P, in, out, axis, nrhs, s);
    case 3: return dst_launch_MV<R, TIO, M, 1, true>(P, in, out, axis, nrhs, s);
    case 4: return dst_launch_MV<R, TIO, M, 0, false, NS, NT, 1>(P, in, out, axis, nrhs, s);
    case 5: return dst_launch_MV<R, TIO, M, 1, false, NS, NT, 1>(P, in, out, axis, nrhs, s);
    case 6: return dst_launch_MV<R, TIO, M, 0, true, NS, NT, 1>(P, in, out, axis, nrhs, s);
    default: return dst_launch_MV<R, TIO, M, 1, true, NS, NT, 1>(P, in, out, axis, nrhs, s);
  }
}

template <typename R, typename TIO>
static cudaError_t dst_dispatch(const Plan& P, const TIO* in, TIO* out, int axis, int nrhs, cudaStream_t s) {
  switch (P.M) {
    case 64: return dst_launch_M<R, TIO, 64>(P, in, out, axis, nrhs, s);
    case 128: return dst_launch_M<R, TIO, 128>(P, in, out, axis, nrhs, s);
    case 256: return dst_launch_M<R, TIO, 256>(P, in, out, axis, nrhs, s);
    case 512: return dst_launch_M<R, TIO, 512>(P, in, out, axis, nrhs, s);
    default: return cudaErrorInvalidValue;
  }
}

template <typename R>
cudaError_t launch_dst_axis(const Plan& P, const R* in, R* out, int axis, int nrhs,
                            cudaStream_t s, uint64_t* nl) {
  if (nl) ++*nl;
  return dst_dispatch<R, R>(P, in, out, axis, nrhs, s);
}

cudaError_t launch_dst_axis_ff(const Plan& P, const double* in, double* out, int axis, int nrhs,
                               cudaStream_t s, uint64_t* nl) {
  if (nl) ++*nl;
  return dst_dispatch<dfl, double>(P, in, out, axis, nrhs, s);
}

template cudaError_t launch_dst_axis<double>(const Plan&, const double*, double*, int, int,
                                             cudaStream_t, uint64_t*);
template cudaError_t launch_dst_axis<float>(const Plan&, const float*, float*, int, int,
                                            cudaStream_t, uint64_t*);

}  // namespace aao
